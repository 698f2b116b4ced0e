"""Parity of the modular BLAS kernels (C ABI) with the oracle, bit-exact.

Sizes span several CTAs and a ragged tail; the aligned (vectorised) and unaligned
(scalar) paths are both exercised; the full 2^24-element workload is checked on a
seeded sample of its outputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu
WIDTHS = [64, 128, 256, 384, 512, 768, 1024]
OPS = ["add", "sub", "mul", "axpy"]


def _ref(op, a, b, q, alpha):
    if op == "add":
        return oracle.vec_addmod(a, b, q)
    if op == "sub":
        return oracle.vec_submod(a, b, q)
    if op == "mul":
        return oracle.vec_mulmod(a, b, q)
    return oracle.vec_axpy(alpha, a, b, q)


def _run(gpu, ctx, op, n, da, db, dc, alpha):
    if op == "add":
        gpu.moma_vec_addmod(ctx, n, da, db, dc)
    elif op == "sub":
        gpu.moma_vec_submod(ctx, n, da, db, dc)
    elif op == "mul":
        gpu.moma_vec_mulmod(ctx, n, da, db, dc)
    else:
        gpu.moma_vec_axpymod(ctx, n, alpha, da, db, dc)


def _edge_values(q):
    """Canonical edge residues: the ends of the range, halves, and words that are all ones or a
    power of two (those not below q, possible for the 60-bit modulus, are dropped)."""
    vals = [0, 1, 2, q - 1, q - 2, q // 2, (q + 1) // 2, (1 << 32) - 1, (1 << 32), (1 << 64) - 1,
            q - (1 << 32), q >> 1 | 1, q - (1 << 31)]
    return [v for v in vals if 0 <= v < q]


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("op", OPS)
def test_blas_parity_small_and_ragged(gpu, width, op):
    p = inputs.prime(width)
    q, L = p.q, p.L
    ctx = gpu.moma_ctx_create(q, width)
    try:
        alpha = inputs.scalar_residue(q, seed=3)
        for n, seed in ((1, 1), (3, 2), (4, 3), (1000, 3), ((1 << 16) + 5, 4)):
            a = inputs.residues(q, L, n, seed)
            b = inputs.residues(q, L, n, seed + 100)
            da, db = gpu.to_device(a), gpu.to_device(b)
            dc = torch.empty_like(da)
            _run(gpu, ctx, op, n, da, db, dc, alpha)
            torch.cuda.synchronize()
            got = inputs.to_ints(gpu.to_host(dc))
            assert got == _ref(op, inputs.to_ints(a), inputs.to_ints(b), q, alpha), (width, op, n)
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("op", OPS)
def test_blas_edge_values(gpu, width, op):
    p = inputs.prime(width)
    q, L = p.q, p.L
    ev = _edge_values(q)
    av = [x for x in ev for _ in ev]
    bv = [y for _ in ev for y in ev]
    ctx = gpu.moma_ctx_create(q, width)
    try:
        for alpha in (0, 1, q - 1, ev[5]):
            da, db = gpu.to_device(inputs.from_ints(av, L)), gpu.to_device(inputs.from_ints(bv, L))
            dc = torch.empty_like(da)
            _run(gpu, ctx, op, len(av), da, db, dc, alpha)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(dc)) == _ref(op, av, bv, q, alpha)
            if op != "axpy":
                break
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", [128, 256])
def test_blas_unaligned_and_inplace(gpu, width):
    p = inputs.prime(width)
    q, L = p.q, p.L
    n = 4099
    a = inputs.residues(q, L, n, 7)
    b = inputs.residues(q, L, n, 8)
    ctx = gpu.moma_ctx_create(q, width)
    try:
        # planes offset by one word: 4-byte aligned only -> scalar path
        buf_a = torch.zeros(L * n + 1, dtype=torch.int32, device="cuda")
        buf_b = torch.zeros(L * n + 1, dtype=torch.int32, device="cuda")
        va = buf_a[1:].view(L, n)
        vb = buf_b[1:].view(L, n)
        va.copy_(gpu.to_device(a))
        vb.copy_(gpu.to_device(b))
        gpu.moma_vec_mulmod(ctx, n, va, vb, va)  # in place, c == a
        torch.cuda.synchronize()
        assert inputs.to_ints(gpu.to_host(va)) == oracle.vec_mulmod(inputs.to_ints(a), inputs.to_ints(b), q)
        alpha = inputs.scalar_residue(q, 9)
        gpu.moma_vec_axpymod(ctx, n, alpha, vb, va, va)  # out aliases y
        torch.cuda.synchronize()
        ref = oracle.vec_axpy(alpha, inputs.to_ints(b), oracle.vec_mulmod(inputs.to_ints(a), inputs.to_ints(b), q), q)
        assert inputs.to_ints(gpu.to_host(va)) == ref
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", WIDTHS)
def test_blas_full_size_sampled(gpu, width):
    """The 2^24-element workload in the launch configuration the benchmark uses."""
    p = inputs.prime(width)
    q, L = p.q, p.L
    n = 1 << 24
    a = inputs.residues(q, L, n, 1)
    b = inputs.residues(q, L, n, 2)
    alpha = inputs.scalar_residue(q, 3)
    rng = np.random.Generator(np.random.PCG64(width))
    idx = np.unique(np.concatenate([rng.integers(0, n, 3000), np.arange(8), np.arange(n - 8, n)]))
    sa, sb = inputs.sample_ints(a, idx), inputs.sample_ints(b, idx)
    ctx = gpu.moma_ctx_create(q, width)
    try:
        da, db = gpu.to_device(a), gpu.to_device(b)
        dc = torch.empty_like(da)
        didx = torch.from_numpy(idx).cuda()
        for op in OPS:
            _run(gpu, ctx, op, n, da, db, dc, alpha)
            torch.cuda.synchronize()
            got = inputs.to_ints(gpu.to_host(dc[:, didx]))
            assert got == _ref(op, sa, sb, q, alpha), (width, op)
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_blas_argument_errors(gpu):
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        a = gpu.to_device(inputs.residues(p.q, 8, 16, 1))
        lib = gpu.lib()
        assert lib.moma_vec_addmod(ctx, 16, None, a.data_ptr(), a.data_ptr(), None) == 1   # INVALID_ARG
        assert lib.moma_vec_addmod(ctx, 16, a.data_ptr() + 2, a.data_ptr(), a.data_ptr(), None) == 4  # ALIGN
        assert lib.moma_vec_addmod(ctx, 0, None, None, None, None) == 0                  # n = 0: no-op
        assert lib.moma_vec_addmod(None, 16, a.data_ptr(), a.data_ptr(), a.data_ptr(), None) == 1
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_ctx_rejects_bad_moduli(gpu):
    import ctypes
    lib = gpu.lib()
    h = ctypes.c_void_p()
    for q, bits in ((inputs.prime(256).q, 384), (inputs.prime(256).q + 1, 256), (1 << 251, 256), (3, 128)):
        L = bits // 32
        arr = (ctypes.c_uint32 * L)(*inputs.int_to_limbs(q % (1 << (32 * L)), L))
        assert lib.moma_ctx_create(ctypes.cast(arr, ctypes.c_void_p), bits, ctypes.byref(h)) == 2  # MODULUS
    arr = (ctypes.c_uint32 * 8)(*inputs.int_to_limbs(inputs.prime(256).q, 8))
    assert lib.moma_ctx_create(ctypes.cast(arr, ctypes.c_void_p), 200, ctypes.byref(h)) == 1
