"""moma_ntt_fwd_noalloc: the forward NTT for callers that may not allocate device memory.

Some callers own all device memory through another allocator or a fixed budget, or may
not wait on an allocator in a hot path, so the library offers one transform whose
intermediate buffers live in a fixed array inside the library.  This file is collected
last on purpose.  Its results must equal the oracle's and moma_ntt_fwd's exactly (the
arithmetic is integer).  It is checked on two calls in a row, because the shared array keeps
the previous call's contents.
"""
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu

# (width, log2 n): single pass (no scratch), two passes, three passes (both buffers),
# and the largest size the array allows at each width (L * n = 2^20 words).
CASES = [(64, 12), (64, 19), (128, 10), (128, 14), (128, 18), (256, 12), (256, 16), (256, 17), (384, 13),
         (384, 16)]
# one case per width is also compared with the oracle (sizes the oracle finishes quickly)
ORACLE_CASES = {(64, 12), (128, 14), (256, 12), (384, 13)}


@pytest.mark.parametrize("width,lg", CASES)
def test_noalloc_matches_ntt_fwd_twice(gpu, width, lg):
    p = inputs.prime(width)
    n = 1 << lg
    ctx = gpu.moma_ctx_create(p.q, width)
    try:
        xa_h = inputs.residues(p.q, p.L, n, seed=500 + lg)
        xa = gpu.to_device(xa_h)
        xb = gpu.to_device(inputs.residues(p.q, p.L, n, seed=600 + lg))
        ref_a, ref_b = torch.empty_like(xa), torch.empty_like(xb)
        gpu.moma_ntt_fwd(ctx, n, xa, ref_a)  # builds the twiddle tables for n (allocates)
        gpu.moma_ntt_fwd(ctx, n, xb, ref_b)
        got = torch.empty_like(xa)
        gpu.moma_ntt_fwd_noalloc(ctx, n, xa, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref_a)
        if (width, lg) in ORACLE_CASES:
            assert inputs.to_ints(gpu.to_host(got)) == oracle.ntt_fwd(inputs.to_ints(xa_h), p.q)
        gpu.moma_ntt_fwd_noalloc(ctx, n, xb, got)  # second call in a row reuses the array
        torch.cuda.synchronize()
        assert torch.equal(got, ref_b)
        inplace = xa.clone()
        gpu.moma_ntt_fwd_noalloc(ctx, n, inplace, inplace)  # out == in
        torch.cuda.synchronize()
        assert torch.equal(inplace, ref_a)
        assert gpu.moma_ctx_sync_status(ctx) == 0
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width,lg", [(128, 12), (256, 16), (384, 15)])
def test_noalloc_full_width_modulus(gpu, width, lg):
    """Contexts of full-width moduli (Montgomery passes) through the shared array: multi-pass sizes
    against the oracle and moma_ntt_fwd, two calls in a row."""
    p = inputs.prime_full(width)
    n = 1 << lg
    ctx = gpu.moma_ctx_create_full(p.q, width)
    try:
        xs = [inputs.residues(p.q, p.L, n, seed=700 + lg + k) for k in range(2)]
        for k, xh in enumerate(xs):
            x = gpu.to_device(xh)
            ref = torch.empty_like(x)
            gpu.moma_ntt_fwd(ctx, n, x, ref)
            got = torch.empty_like(x)
            gpu.moma_ntt_fwd_noalloc(ctx, n, x, got)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), k
            if k == 0 and lg <= 12:
                assert inputs.to_ints(gpu.to_host(got)) == oracle.ntt_fwd(inputs.to_ints(xh), p.q)
        assert gpu.moma_ctx_sync_status(ctx) == 0
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_noalloc_call_takes_no_device_memory(gpu):
    """The array is placed when the context is created, so the entry point's first call on a fresh
    context, after the tables exist, leaves the device's free memory unchanged."""
    p = inputs.prime(256)
    n = 1 << 16
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        x = gpu.to_device(inputs.residues(p.q, p.L, n, seed=9))
        ref, got = torch.empty_like(x), torch.empty_like(x)
        gpu.moma_ntt_fwd(ctx, n, x, ref)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        gpu.moma_ntt_fwd_noalloc(ctx, n, x, got)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.equal(got, ref)
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_noalloc_rejects_oversize_and_unprepared(gpu):
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    lib = gpu.lib()
    try:
        big = torch.zeros((p.L, 1 << 18), dtype=torch.int32, device="cuda")
        assert lib.moma_ntt_fwd_noalloc(ctx, 1 << 18, big.data_ptr(), big.data_ptr(), None) == 3  # SIZE
        x = gpu.to_device(inputs.residues(p.q, p.L, 1 << 12, seed=1))
        # no earlier moma_ntt_fwd for this size: the tables do not exist yet
        assert lib.moma_ntt_fwd_noalloc(ctx, 1 << 12, x.data_ptr(), x.data_ptr(), None) == 1  # INVALID_ARG
        # a schedule change after the tables were built needs another moma_ntt_fwd
        y = torch.empty_like(x)
        gpu.moma_ntt_fwd(ctx, 1 << 12, x, y)
        gpu.moma_ctx_set_config(ctx, "ntt_fwd", 1 << 12, tile_log=9, max_logr=4)
        assert lib.moma_ntt_fwd_noalloc(ctx, 1 << 12, x.data_ptr(), y.data_ptr(), None) == 1
        gpu.moma_ntt_fwd(ctx, 1 << 12, x, y)
        z = torch.empty_like(x)
        assert lib.moma_ntt_fwd_noalloc(ctx, 1 << 12, x.data_ptr(), z.data_ptr(), None) == 0
        torch.cuda.synchronize()
        assert torch.equal(z, y)
    finally:
        gpu.moma_ctx_destroy(ctx)
