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


STAGED_TILES = {64: (10,), 128: (10,), 256: (9,), 384: (8,)}


@pytest.mark.parametrize("width", [64, 128, 256, 384])
@pytest.mark.parametrize("op", OPS)
def test_blas_staged_parity(gpu, width, op):
    """Operands staged in shared memory by bulk copies: every tile size and product engine, sizes
    with several tiles per CTA and a ragged tail past the last whole tile (n a multiple of 4, so
    the staged path is taken), against the oracle."""
    p = inputs.prime(width)
    q, L = p.q, p.L
    ctx = gpu.moma_ctx_create(q, width)
    engines = {"mul": (1, 2, 3), "axpy": (1, 2)}.get(op, (1,))
    try:
        alpha = inputs.scalar_residue(q, seed=5)
        for tile in STAGED_TILES[width]:
            for eng in engines:
                gpu.moma_ctx_set_config(ctx, op, 1 << 20, engine=eng, tile_log=tile)
                cfg = gpu.moma_ctx_get_config(ctx, op, 1 << 20)
                assert (cfg["engine"], cfg["tile_log"]) == (eng, tile)
                # the largest size gives every CTA of the persistent grid more tiles than stages
                for n, seed in ((4, 1), (1 << tile, 2), (3 * (1 << tile) + 4, 3), (3 * (1 << 20) + 1028, 4)):
                    a = inputs.residues(q, L, n, seed)
                    b = inputs.residues(q, L, n, seed + 50)
                    da, db = gpu.to_device(a), gpu.to_device(b)
                    dc = torch.empty_like(da)
                    _run(gpu, ctx, op, n, da, db, dc, alpha)
                    torch.cuda.synchronize()
                    if n < 1 << 16:
                        got = inputs.to_ints(gpu.to_host(dc))
                        ref = _ref(op, inputs.to_ints(a), inputs.to_ints(b), q, alpha)
                    else:  # a seeded sample, the first tiles and the ragged end
                        rng = np.random.Generator(np.random.PCG64(n + tile))
                        idx = np.unique(np.concatenate([rng.integers(0, n, 3000), np.arange(2048),
                                                        np.arange(n - 3000, n)]))
                        got = inputs.to_ints(gpu.to_host(dc[:, torch.from_numpy(idx).cuda()]))
                        ref = _ref(op, inputs.sample_ints(a, idx), inputs.sample_ints(b, idx), q, alpha)
                    assert got == ref, (width, op, tile, eng, n)
        assert gpu.moma_ctx_sync_status(ctx) == 0
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_blas_staged_fallback_and_inplace(gpu):
    """A staged schedule with operands that cannot be bulk-copied (planes not 16-byte aligned, n not
    a multiple of 4) takes the direct loads; in-place calls (c == a, out == y) stay exact."""
    p = inputs.prime(256)
    q, L = p.q, p.L
    ctx = gpu.moma_ctx_create(q, 256)
    try:
        gpu.moma_ctx_set_config(ctx, "mul", 1, engine=3, tile_log=9)
        gpu.moma_ctx_set_config(ctx, "axpy", 1, engine=2, tile_log=9)
        for n, off in ((4099, 0), (4096, 1), (8192, 0)):
            a = inputs.residues(q, L, n, 11)
            b = inputs.residues(q, L, n, 12)
            buf_a = torch.zeros(L * n + off, dtype=torch.int32, device="cuda")
            buf_b = torch.zeros(L * n + off, dtype=torch.int32, device="cuda")
            va, vb = buf_a[off:].view(L, n), buf_b[off:].view(L, n)
            va.copy_(gpu.to_device(a))
            vb.copy_(gpu.to_device(b))
            gpu.moma_vec_mulmod(ctx, n, va, vb, va)
            torch.cuda.synchronize()
            ab = oracle.vec_mulmod(inputs.to_ints(a), inputs.to_ints(b), q)
            assert inputs.to_ints(gpu.to_host(va)) == ab, (n, off)
            alpha = inputs.scalar_residue(q, 13)
            gpu.moma_vec_axpymod(ctx, n, alpha, vb, va, va)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(va)) == oracle.vec_axpy(alpha, inputs.to_ints(b), ab, q), (n, off)
        assert gpu.moma_ctx_sync_status(ctx) == 0
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_blas_staged_wait_runs_out(gpu):
    """The bounded wait of the staged kernel: the test hook arms one stage for 16 bytes that never
    arrive, the wait gives up after the (short) limit, the status reports MOMA_ERR_TIMEOUT, the
    kernel ends, and the next launch is exact again."""
    p = inputs.prime(256)
    q, L = p.q, p.L
    n = 1 << 20
    ctx = gpu.moma_ctx_create(q, 256)
    try:
        gpu.moma_ctx_set_config(ctx, "mul", n, engine=3, tile_log=9)
        lib = gpu.lib()
        assert lib.moma_ctx_set_wait_limit(ctx, 0) == 1 and lib.moma_ctx_set_wait_limit(None, 5) == 1
        assert lib.moma_ctx_inject_missing_copy(None) == 1
        gpu.moma_ctx_set_wait_limit(ctx, 2_000_000)  # 2 ms
        a = inputs.residues(q, L, n, 21)
        b = inputs.residues(q, L, n, 22)
        da, db = gpu.to_device(a), gpu.to_device(b)
        dc = torch.empty_like(da)
        gpu.moma_ctx_inject_missing_copy(ctx)
        gpu.moma_vec_mulmod(ctx, n, da, db, dc)
        assert gpu.moma_ctx_sync_status(ctx) == 7  # MOMA_ERR_TIMEOUT
        assert gpu.moma_ctx_sync_status(ctx) == 0  # cleared
        gpu.moma_vec_mulmod(ctx, n, da, db, dc)
        torch.cuda.synchronize()
        idx = np.arange(0, n, 997)
        got = inputs.to_ints(gpu.to_host(dc[:, torch.from_numpy(idx).cuda()]))
        assert got == oracle.vec_mulmod(inputs.sample_ints(a, idx), inputs.sample_ints(b, idx), q)
        assert gpu.moma_ctx_sync_status(ctx) == 0
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_default_stream_is_torchs_current_stream(gpu):
    """stream=None launches on torch's current stream: the handle the binding passes equals
    torch.cuda.current_stream() outside and inside a stream context, and a call inside the
    context is ordered on that stream."""
    from paper_2501_07535_gb300 import moma
    assert moma._current_stream_handle() == torch.cuda.current_stream().cuda_stream
    s = torch.cuda.Stream()
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        a = gpu.to_device(inputs.residues(p.q, p.L, 1 << 12, seed=1))
        b = gpu.to_device(inputs.residues(p.q, p.L, 1 << 12, seed=2))
        c = torch.empty_like(a)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            assert moma._current_stream_handle() == s.cuda_stream != torch.cuda.default_stream().cuda_stream
            gpu.moma_vec_mulmod(ctx, 1 << 12, a, b, c)
        s.synchronize()
        assert inputs.to_ints(gpu.to_host(c)) == oracle.vec_mulmod(inputs.to_ints(gpu.to_host(a)),
                                                                   inputs.to_ints(gpu.to_host(b)), p.q)
        assert moma._current_stream_handle() == torch.cuda.current_stream().cuda_stream
    finally:
        gpu.moma_ctx_destroy(ctx)
