"""Autotuned schedules kept as a JSON table, so that a tuning run's choices can be reused.

An entry is keyed by (op, n, bits, full) -- the operation name of `moma.OPS`, the transform length
(for the element-wise ops the schedule holds for every length, and n is recorded as 0), the
container width and whether the context is a full-width one -- and holds the `moma_config` fields
the autotuner chose with its time per call.  `tune` runs `moma_autotune` and records the result,
`apply` sets every entry of one width and kind on a context with `moma_ctx_set_config`.  File
layout:

    {"format": "moma-schedules", "version": 1,
     "entries": [{"op": "ntt_fwd", "n": 1048576, "bits": 256, "full": false,
                  "config": {"engine": 2, "tile_log": 10, ...}, "us": 241.7}, ...]}

Host bookkeeping only; the schedules themselves are run by the library's kernels.
"""
from __future__ import annotations

import json
import os

from . import moma

FORMAT = "moma-schedules"
VERSION = 1
VEC_OPS = ("add", "sub", "mul", "axpy")
CONFIG_FIELDS = tuple(f for f, _ in moma.moma_config._fields_)


def _key(op: str, n: int, bits: int, full: bool) -> tuple:
    if op not in moma.OPS:
        raise ValueError(f"unknown operation {op!r}")
    return (op, 0 if op in VEC_OPS else int(n), int(bits), bool(full))


class Table:
    """(op, n, bits, full) -> {"config": {...}, "us": float}."""

    def __init__(self):
        self.entries: dict[tuple, dict] = {}

    def record(self, op: str, n: int, bits: int, full: bool, config: dict, us: float | None = None):
        cfg = {f: int(config.get(f, 0)) for f in CONFIG_FIELDS}
        self.entries[_key(op, n, bits, full)] = {"config": cfg, "us": None if us is None else float(us)}

    def lookup(self, op: str, n: int, bits: int, full: bool = False) -> dict | None:
        e = self.entries.get(_key(op, n, bits, full))
        return None if e is None else dict(e["config"])

    def to_json(self) -> dict:
        rows = [{"op": k[0], "n": k[1], "bits": k[2], "full": k[3], "config": v["config"], "us": v["us"]}
                for k, v in sorted(self.entries.items())]
        return {"format": FORMAT, "version": VERSION, "entries": rows}

    @classmethod
    def from_json(cls, doc: dict) -> "Table":
        if doc.get("format") != FORMAT or doc.get("version") != VERSION:
            raise ValueError("not a moma schedule table of a known version")
        t = cls()
        for r in doc["entries"]:
            unknown = set(r["config"]) - set(CONFIG_FIELDS)
            if unknown:
                raise ValueError(f"unknown schedule fields {sorted(unknown)}")
            t.record(r["op"], r["n"], r["bits"], r["full"], r["config"], r.get("us"))
        return t

    def save(self, path: str):
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.to_json(), f, indent=1)
        os.replace(tmp, path)

    @classmethod
    def load(cls, path: str) -> "Table":
        with open(path) as f:
            return cls.from_json(json.load(f))


def tune(table: Table, ctx, bits: int, op: str, n: int, count: int = 1, full: bool = False, stream=None) -> dict:
    """Run the library's autotuner for (op, n) on `ctx` (which keeps the winner) and record it."""
    best, us = moma.moma_autotune(ctx, op, n, count, stream)
    table.record(op, n, bits, full, best, us)
    return best


def apply(table: Table, ctx, bits: int, full: bool = False) -> int:
    """Set every schedule of this width and context kind on `ctx`; returns how many were set."""
    k = 0
    for (op, n, b, f), e in sorted(table.entries.items()):
        if b == bits and f == bool(full):
            moma.moma_ctx_set_config(ctx, op, n if n else 1, **e["config"])
            k += 1
    return k
