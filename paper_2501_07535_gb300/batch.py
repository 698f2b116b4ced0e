"""Building and running mixed job sets (the uneven batched workload) through the C ABI.

A job set is a list of `inputs.Job` (op, width, n, seed, prime_seed).  `JobSet` holds one
context per modulus, the device inputs and outputs of every job, and runs the set either as
one persistent batch launch (moma_batch_*) or as plain per-call launches (each job its own
moma_ntt_* / moma_polymul / moma_vec_* call), so that the two forms can be compared on the
same buffers.  Argument marshalling only; all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import inputs, moma

_CALLS = {
    "ntt_fwd": lambda c, n, a, b, o, al, s: moma.moma_ntt_fwd(c, n, a, o, s),
    "ntt_inv": lambda c, n, a, b, o, al, s: moma.moma_ntt_inv(c, n, a, o, s),
    "polymul": lambda c, n, a, b, o, al, s: moma.moma_polymul(c, n, a, b, o, s),
    "add": lambda c, n, a, b, o, al, s: moma.moma_vec_addmod(c, n, a, b, o, s),
    "sub": lambda c, n, a, b, o, al, s: moma.moma_vec_submod(c, n, a, b, o, s),
    "mul": lambda c, n, a, b, o, al, s: moma.moma_vec_mulmod(c, n, a, b, o, s),
    "axpy": lambda c, n, a, b, o, al, s: moma.moma_vec_axpymod(c, n, al, a, b, o, s),
}
TWO_OPERANDS = {"polymul", "add", "sub", "mul", "axpy"}


class Contexts:
    """One library context per (width, prime seed), created on first use."""

    def __init__(self):
        self._h = {}

    def get(self, width: int, prime_seed: int = 0) -> int:
        key = (width, prime_seed)
        if key not in self._h:
            self._h[key] = moma.moma_ctx_create(inputs.prime(width, prime_seed).q, width)
        return self._h[key]

    def handles(self) -> list[int]:
        return list(self._h.values())

    def close(self):
        for h in self._h.values():
            moma.moma_ctx_destroy(h)
        self._h.clear()


class JobSet:
    """The jobs of one rank: with world_size > 1 the set keeps only its cost-balanced share
    (replicas.shard_balanced), so N ranks on N GPUs together run the whole list once."""

    def __init__(self, jobs, contexts: Contexts | None = None, device="cuda", rank: int = 0, world_size: int = 1):
        from . import replicas
        self.jobs = replicas.shard_balanced(jobs, rank, world_size, replicas.job_cost)
        self.ctx = contexts or Contexts()
        self.a, self.b, self.out, self.alpha, self.host_a, self.host_b = [], [], [], [], [], []
        for j in self.jobs:
            p = inputs.prime(j.width, j.prime_seed)
            ha = inputs.residues(p.q, p.L, j.n, j.seed)
            hb = inputs.residues(p.q, p.L, j.n, j.seed + 7) if j.op in TWO_OPERANDS else None
            self.host_a.append(ha)
            self.host_b.append(hb)
            da = moma.to_device(ha, device)
            self.a.append(da)
            self.b.append(moma.to_device(hb, device) if hb is not None else None)
            self.out.append(torch.empty_like(da))
            self.alpha.append(inputs.scalar_residue(p.q, j.seed + 11) if j.op == "axpy" else None)
        self.batch = None

    def job_dicts(self):
        return [{"op": j.op, "ctx": self.ctx.get(j.width, j.prime_seed), "n": j.n, "a": self.a[i],
                 "b": self.b[i], "out": self.out[i], "alpha": self.alpha[i]} for i, j in enumerate(self.jobs)]

    def create_batch(self):
        if self.batch is None:
            self.batch = moma.moma_batch_create(self.job_dicts())
        return self.batch

    def run_batched(self, stream=None):
        moma.moma_batch_run(self.create_batch(), stream)

    def run_plain(self, stream=None):
        for i, j in enumerate(self.jobs):
            _CALLS[j.op](self.ctx.get(j.width, j.prime_seed), j.n, self.a[i], self.b[i], self.out[i],
                         self.alpha[i], stream)

    def status(self) -> int:
        return moma.moma_batch_sync_status(self.batch) if self.batch else 0

    def close(self):
        if self.batch:
            moma.moma_batch_destroy(self.batch)
            self.batch = None

    def work_units(self) -> dict:
        """Counts used for throughput: transforms (a cyclic product is three) and vector elements."""
        nt = sum(3 if j.op == "polymul" else 1 for j in self.jobs if j.op in ("ntt_fwd", "ntt_inv", "polymul"))
        ve = sum(j.n for j in self.jobs if j.op in ("add", "sub", "mul", "axpy"))
        return {"transforms": nt, "vector_elements": ve, "jobs": len(self.jobs)}
