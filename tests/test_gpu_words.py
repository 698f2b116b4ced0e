"""The word-level building blocks against integer arithmetic and against the bounds the method
relies on (through moma_word_probe, raw outputs before any final reduction).

- add/sub (rules (addqdd), (adc), (subddd); the recursion of Sec. 3.2): exact sum with its carry
  word, exact difference mod 2^W with its borrow;
- the double-width product by every engine (Sec. 2.2 Eq. muls, Eq. mulk; rule (mulqdd)): exact;
- the truncated high half: floor(a*b / 2^W) or one less (the Barrett quotient estimate);
- Barrett reduction (Sec. 3.1 Eq. barrett): the exact residue, and its final correction fires at
  most once (one conditional subtraction suffices for a (W-4)-bit modulus);
- the fixed-multiplicand product before its corrections: congruent to a*w and below 3q, its
  quotient estimate the oracle reading's (oracle.barrett_fixed_steps) or one less;
- the Montgomery product: a*b*R^-1 mod q (full-width contexts);
- the word-based Barrett reduction of full-width contexts: r = a*b - s*q before its two final
  subtractions lies in [0, 4q) with s within 3 of floor(a*b/q) and equal to the oracle reading's
  estimate (oracle.barrett_full_steps) or one less, and the reduced product is exact,
  for moduli whose top word is 1 (the largest constant floor(2^(2W)/q)) and for 2^W - 1.
Operands are edge values (0, 1, all-ones words, q - 1, 2^W - 1 where allowed) and seeded draws.
"""
import random

import numpy as np
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu

WIDTHS = [64, 128, 256, 384, 512, 768]


def _vals(W, bound, rng, n):
    top = (1 << W) - 1
    edge = [0, 1, 2, top, top - 1, (1 << (W - 1)), (1 << 32) - 1, top ^ 0xFFFFFFFF, bound - 1, bound // 2]
    edge = [v for v in edge if 0 <= v < bound]
    vals = edge + [rng.randrange(bound) for _ in range(n - len(edge))]
    rng.shuffle(vals)
    return vals


def _probe(gpu, ctx, op, engine, a, b, L):
    n = len(a)
    da, db = gpu.to_device(inputs.from_ints(a, L)), gpu.to_device(inputs.from_ints(b, L))
    out = torch.zeros((2 * L + 1, n), dtype=torch.int32, device="cuda")
    gpu.moma_word_probe(ctx, op, engine, n, da, db, out)
    torch.cuda.synchronize()
    o = gpu.to_host(out)
    return o


def _planes(o, lo, hi):
    return inputs.to_ints(np.ascontiguousarray(o[lo:hi]))


@pytest.mark.parametrize("width", WIDTHS)
def test_word_add_sub_and_products(gpu, width):
    L = width // 32
    W = width
    rng = random.Random(width)
    q = inputs.prime(width).q
    ctx = gpu.moma_ctx_create(q, width)
    try:
        n = 1500
        a, b = _vals(W, 1 << W, rng, n), _vals(W, 1 << W, rng, n)
        o = _probe(gpu, ctx, "add", 0, a, b, L)
        s = _planes(o, 0, L)
        carry = [int(x) for x in o[L]]
        assert [x + y for x, y in zip(a, b)] == [v + (c << W) for v, c in zip(s, carry)]
        o = _probe(gpu, ctx, "sub", 0, a, b, L)
        d = _planes(o, 0, L)
        borrow = [int(x) for x in o[L]]
        assert d == [(x - y) % (1 << W) for x, y in zip(a, b)]
        assert borrow == [int(x < y) for x, y in zip(a, b)]
        for engine in (1, 2, 3):
            o = _probe(gpu, ctx, "mul", engine, a, b, L)
            assert _planes(o, 0, 2 * L) == [x * y for x, y in zip(a, b)], engine
        for engine in (1, 2):
            o = _probe(gpu, ctx, "mul_hi", engine, a, b, L)
            h = _planes(o, 0, L)
            exact = [(x * y) >> W for x, y in zip(a, b)]
            assert all(e - 1 <= v <= e for v, e in zip(h, exact)), engine
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", WIDTHS)
def test_word_barrett_one_correction_and_fixed_bound(gpu, width):
    L = width // 32
    rng = random.Random(width + 1)
    q = inputs.prime(width).q
    ctx = gpu.moma_ctx_create(q, width)
    try:
        n = 2000
        a, b = _vals(width, q, rng, n), _vals(width, q, rng, n)
        for engine in (1, 2):
            o = _probe(gpu, ctx, "barrett", engine, a, b, L)
            assert _planes(o, 0, L) == [x * y % q for x, y in zip(a, b)], engine
            fired = [int(x) for x in o[L]]
            assert set(fired) <= {0, 1}
        # the fixed multiplicand w = b[0]; a ranges over all L-word values
        aw = _vals(width, 1 << width, rng, n)
        w = b[0] if b[0] else 1
        bb = [w] + b[1:]
        for engine in (1, 2):
            o = _probe(gpu, ctx, "fixed", engine, aw, bb, L)
            r = _planes(o, 0, L)
            assert all(0 <= v < 3 * q for v in r), engine
            assert all((v - x * w) % q == 0 for v, x in zip(r, aw)), engine
            # the kernel's quotient estimate is the oracle reading's exact one or one less (its
            # high half is truncated)
            for x, v in zip(aw, r):
                s_or = oracle.barrett_fixed_steps(x, w, q, width)[2]
                assert (x * w - v) // q in (s_or, s_or - 1), engine
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", WIDTHS)
def test_word_montgomery(gpu, width):
    L = width // 32
    rng = random.Random(width + 2)
    q = inputs.prime_full(width).q
    rinv = pow(1 << width, -1, q)
    ctx = gpu.moma_ctx_create_full(q, width)
    try:
        n = 2000
        a, b = _vals(width, q, rng, n), _vals(width, q, rng, n)
        o = _probe(gpu, ctx, "mont", 0, a, b, L)
        assert _planes(o, 0, L) == [x * y * rinv % q for x, y in zip(a, b)]
        with pytest.raises(gpu.MomaError):  # Barrett blocks need a Barrett context
            _probe(gpu, ctx, "barrett", 1, a[:4], b[:4], L)
    finally:
        gpu.moma_ctx_destroy(ctx)


def _full_moduli(width):
    """Odd full-width moduli (BLAS needs no prime): the test prime, the smallest top word, 2^W - 1."""
    return [inputs.prime_full(width).q, (1 << (width - 32)) + 12345, (1 << width) - 1]


@pytest.mark.parametrize("width", WIDTHS)
def test_word_barrett_full_bound(gpu, width):
    L = width // 32
    rng = random.Random(width + 3)
    for q in _full_moduli(width):
        ctx = gpu.moma_ctx_create_full(q, width)
        try:
            n = 1500
            a, b = _vals(width, q, rng, n), _vals(width, q, rng, n)
            want = [x * y % q for x, y in zip(a, b)]
            for engine in (1, 2, 3):
                o = _probe(gpu, ctx, "barrett_full", engine, a, b, L)
                r = _planes(o, 0, L + 1)
                assert _planes(o, L + 1, 2 * L + 1) == want, (hex(q), engine)
                for x, y, v in zip(a, b, r):
                    t = x * y
                    assert 0 <= v < 4 * q and (t - v) % q == 0, (hex(q), engine)
                    assert t // q - 3 <= (t - v) // q <= t // q
                    # the oracle reading's exact estimate, or one less (truncated high half)
                    s_or = oracle.barrett_full_steps(x, y, q, L)[2]
                    assert (t - v) // q in (s_or, s_or - 1), (hex(q), engine)
            with pytest.raises(gpu.MomaError):  # the W-4 bit Barrett block needs a Barrett context
                _probe(gpu, ctx, "barrett", 1, a[:4], b[:4], L)
        finally:
            gpu.moma_ctx_destroy(ctx)
