"""moma_ntt_fwd_noalloc: the forward NTT for callers that may not allocate device memory.

Some callers own all device memory through another allocator or a fixed budget, or may
not wait on an allocator in a hot path, so the library offers one transform whose
intermediate buffers live in a fixed array inside the library.  This file is collected
last on purpose.  Its results must equal moma_ntt_fwd's exactly (the arithmetic is integer).
It is checked on two calls in a row, because the shared array keeps the previous call's
contents.
"""
import pytest
import torch

from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu

# (width, log2 n): single pass (no scratch), two passes, three passes (both buffers),
# and the largest size the array allows at each width (L * n = 2^20 words).
CASES = [(128, 10), (128, 14), (128, 18), (256, 12), (256, 16), (256, 17), (384, 13), (384, 16)]


@pytest.mark.parametrize("width,lg", CASES)
def test_noalloc_matches_ntt_fwd_twice(gpu, width, lg):
    p = inputs.prime(width)
    n = 1 << lg
    ctx = gpu.moma_ctx_create(p.q, width)
    try:
        xa = gpu.to_device(inputs.residues(p.q, p.L, n, seed=500 + lg))
        xb = gpu.to_device(inputs.residues(p.q, p.L, n, seed=600 + lg))
        ref_a, ref_b = torch.empty_like(xa), torch.empty_like(xb)
        gpu.moma_ntt_fwd(ctx, n, xa, ref_a)  # builds the twiddle tables for n (allocates)
        gpu.moma_ntt_fwd(ctx, n, xb, ref_b)
        got = torch.empty_like(xa)
        gpu.moma_ntt_fwd_noalloc(ctx, n, xa, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref_a)
        gpu.moma_ntt_fwd_noalloc(ctx, n, xb, got)  # second call in a row reuses the array
        torch.cuda.synchronize()
        assert torch.equal(got, ref_b)
        assert gpu.moma_ctx_sync_status(ctx) == 0
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
    finally:
        gpu.moma_ctx_destroy(ctx)
