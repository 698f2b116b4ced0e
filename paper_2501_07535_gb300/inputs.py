"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle's tests.

This module only draws random numbers and converts between Python integers and the
limb-major uint32 layout.  It holds none of the modular arithmetic of the method:
no addition, subtraction or multiplication modulo q, no transform.

Layout (used everywhere in this project): a vector of n residues, each an L-limb
integer with 32-bit limbs, is stored limb-major as ``uint32[L][n]``; limb 0 is the
least significant word.  The paper writes multi-word integers most significant word
first (Sec. 2.2, Eq. def_mp; Sec. 3, Eq. def_moma); that is notation only, memory
order here is little-endian.

Distributions follow the paper's workloads (Sec. 5): residues uniform in [0, q);
moduli of B = W - 4 bits inside a W-bit container (Sec. 5.2).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np

WIDTHS = (64, 128, 256, 384, 512, 768, 1024)
_HERE = os.path.dirname(os.path.abspath(__file__))
# the seed-generated moduli (input data, not results), written by tests/golden/make_primes.py
PRIMES_JSON = os.path.join(_HERE, "primes.json")


def limbs_of(width_bits: int) -> int:
    """Number of 32-bit limbs of a W-bit container (W/32)."""
    if width_bits % 32:
        raise ValueError("width must be a multiple of 32")
    return width_bits // 32


def int_to_limbs(x: int, L: int) -> list[int]:
    """Little-endian 32-bit limbs of a non-negative integer x < 2^(32L)."""
    if x < 0 or x >> (32 * L):
        raise ValueError("value does not fit in L limbs")
    return [(x >> (32 * i)) & 0xFFFFFFFF for i in range(L)]


def limbs_to_int(limbs) -> int:
    out = 0
    for i, w in enumerate(limbs):
        out |= int(w) << (32 * i)
    return out


def from_ints(values, L: int) -> np.ndarray:
    """Python ints -> uint32[L][n] limb-major array."""
    n = len(values)
    arr = np.zeros((L, n), dtype=np.uint32)
    for i, v in enumerate(values):
        v = int(v)
        if v < 0 or v >> (32 * L):
            raise ValueError("value does not fit in L limbs")
        for j in range(L):
            arr[j, i] = (v >> (32 * j)) & 0xFFFFFFFF
    return arr


def to_ints(arr: np.ndarray) -> list[int]:
    """uint32[L][n] limb-major array -> list of Python ints (vectorised over limbs)."""
    arr = np.asarray(arr, dtype=np.uint32)
    L, n = arr.shape
    # Build in 64-bit halves to keep the Python-level work to one int op per limb pair.
    out = [0] * n
    cols = [arr[j].tolist() for j in range(L)]
    for j in range(L - 1, -1, -1):
        c = cols[j]
        out = [(o << 32) | w for o, w in zip(out, c)]
    return out


def sample_ints(arr: np.ndarray, idx) -> list[int]:
    """Integers at selected columns of a limb-major array (cheap for big arrays)."""
    arr = np.asarray(arr)
    sub = arr[:, np.asarray(idx, dtype=np.int64)]
    return to_ints(sub)


# ----------------------------------------------------------------------------- moduli

@dataclass(frozen=True)
class Prime:
    width: int      # container width W (bits)
    seed: int
    q: int
    bits: int       # bit length of q: W - 4 (Barrett contexts) or W (full-width contexts)
    two_adicity: int

    @property
    def L(self) -> int:
        return limbs_of(self.width)


def load_primes(path: str = PRIMES_JSON) -> dict[tuple[int, int], Prime]:
    """Committed table of seed-generated primes, keyed by (W, seed)."""
    with open(path) as f:
        doc = json.load(f)
    out = {}
    for e in doc["primes"]:
        p = Prime(width=e["width"], seed=e["seed"], q=int(e["q"], 16), bits=e["bits"],
                  two_adicity=e["two_adicity"])
        out[(p.width, p.seed)] = p
    return out


_TABLES: dict[str, tuple] = {}  # parsed tables of PRIMES_JSON (Prime is immutable)


def _tables() -> tuple:
    if PRIMES_JSON not in _TABLES:
        _TABLES[PRIMES_JSON] = (load_primes(PRIMES_JSON), load_full_primes(PRIMES_JSON))
    return _TABLES[PRIMES_JSON]


def prime(width: int, seed: int = 0) -> Prime:
    """The committed (W - 4)-bit prime for (W, seed); the table is read once per process."""
    return _tables()[0][(width, seed)]


def load_full_primes(path: str = PRIMES_JSON) -> dict[tuple[int, int], Prime]:
    """Committed table of full-width primes (exactly W bits), keyed by (W, seed)."""
    with open(path) as f:
        doc = json.load(f)
    out = {}
    for e in doc.get("full_primes", []):
        p = Prime(width=e["width"], seed=e["seed"], q=int(e["q"], 16), bits=e["bits"],
                  two_adicity=e["two_adicity"])
        out[(p.width, p.seed)] = p
    return out


def prime_full(width: int, seed: int = 0) -> Prime:
    """The committed full-width (W-bit) prime for (W, seed)."""
    return _tables()[1][(width, seed)]


# ----------------------------------------------------------------------------- residues

def _less_than(draw: np.ndarray, ql: list[int]) -> np.ndarray:
    """Column-wise draw < q, comparing limbs from the most significant one down."""
    L = draw.shape[0]
    less = draw[L - 1] < np.uint32(ql[L - 1])
    tie = np.nonzero(draw[L - 1] == np.uint32(ql[L - 1]))[0]
    for j in range(L - 2, -1, -1):
        if tie.size == 0:
            break
        col = draw[j, tie]
        less[tie[col < np.uint32(ql[j])]] = True
        tie = tie[col == np.uint32(ql[j])]
    return less


def residues(q: int, L: int, n: int, seed: int) -> np.ndarray:
    """n residues uniform in [0, q) as uint32[L][n], from numpy PCG64(seed).

    Raw limbs are drawn uniformly, the top limb masked to the bit length of q, and
    columns that are >= q are redrawn (rejection keeps the distribution exactly
    uniform).  The comparison with q is lexicographic from the top limb.
    """
    if q <= 0 or q.bit_length() > 32 * L:
        raise ValueError("q does not fit in L limbs")
    top_bits = q.bit_length() - 32 * (L - 1)
    if top_bits <= 0:
        raise ValueError("q shorter than L-1 limbs; use fewer limbs")
    mask = np.uint32((1 << top_bits) - 1) if top_bits < 32 else np.uint32(0xFFFFFFFF)
    rng = np.random.Generator(np.random.PCG64(seed))
    ql = int_to_limbs(q, L)
    out = rng.integers(0, 1 << 32, size=(L, n), dtype=np.uint32)
    out[L - 1] &= mask
    todo = np.nonzero(~_less_than(out, ql))[0]
    while todo.size:
        draw = rng.integers(0, 1 << 32, size=(L, todo.size), dtype=np.uint32)
        draw[L - 1] &= mask
        ok = _less_than(draw, ql)
        out[:, todo[ok]] = draw[:, ok]
        todo = todo[~ok]
    return out


def scalar_residue(q: int, seed: int) -> int:
    """One residue uniform in [0, q) (used for the axpy scalar alpha)."""
    L = (q.bit_length() + 31) // 32
    return to_ints(residues(q, L, 1, seed))[0]


# ----------------------------------------------------------------------------- job mixes

@dataclass(frozen=True)
class Job:
    op: str          # 'ntt_fwd', 'ntt_inv', 'polymul', 'add', 'sub', 'mul', 'axpy'
    width: int
    n: int
    seed: int
    prime_seed: int = 0


def uneven_batch(n_jobs: int = 256, seed: int = 0, log_n_range=(10, 20),
                 widths=(128, 256, 384), ops=("ntt_fwd", "ntt_inv", "polymul")) -> list[Job]:
    """Mixed job list: log2 n uniform on the range, width uniform on the set, op uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for i in range(n_jobs):
        lg = int(rng.integers(log_n_range[0], log_n_range[1] + 1))
        w = int(widths[int(rng.integers(0, len(widths)))])
        op = ops[int(rng.integers(0, len(ops)))]
        jobs.append(Job(op=op, width=w, n=1 << lg, seed=1000 + i))
    return jobs


def served_stream(n_jobs: int = 10000, seed: int = 0, rate_per_s: float = 1000.0,
                  ntt_log_range=(12, 22), vec_log_range=(16, 24), widths=(256, 384, 768),
                  moduli_per_width: int = 2):
    """Poisson arrivals (exponential gaps) of a seeded mix of NTT and BLAS jobs.

    Returns (arrival_times_s, jobs).  Half the jobs are transforms, half are
    mulmod/axpy vectors, widths uniform on the set, a few moduli per width.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=n_jobs)
    t = np.cumsum(gaps)
    jobs = []
    for i in range(n_jobs):
        w = int(widths[int(rng.integers(0, len(widths)))])
        ps = int(rng.integers(0, moduli_per_width))
        if rng.random() < 0.5:
            lg = int(rng.integers(ntt_log_range[0], ntt_log_range[1] + 1))
            op = "ntt_fwd" if rng.random() < 0.5 else "ntt_inv"
        else:
            lg = int(rng.integers(vec_log_range[0], vec_log_range[1] + 1))
            op = "mul" if rng.random() < 0.5 else "axpy"
        jobs.append(Job(op=op, width=w, n=1 << lg, seed=50000 + i, prime_seed=ps))
    return t.tolist(), jobs


def log2_exact(n: int) -> int:
    k = int(math.log2(n)) if n > 0 else -1
    if n <= 0 or (1 << k) != n:
        raise ValueError("n must be a power of two")
    return k
