"""Full-width moduli (W bits, Montgomery contexts) on the GPU, bit-exact against the oracle.

The oracle computes the definitions (a + b, a - b, a * b, alpha * x + y mod q, Eq. ntt, the
cyclic product); nothing on the GPU side is Barrett-specific here, every product is a
Montgomery product.  Edge values include q - 1 (sums that carry out of the container) and
residues with all-ones words.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu

WIDTHS = [64, 128, 256, 384, 512, 768, 1024]


@pytest.fixture(scope="module")
def fctx(gpu):
    ctxs = {w: gpu.moma_ctx_create_full(inputs.prime_full(w).q, w) for w in WIDTHS}
    yield ctxs
    for h in ctxs.values():
        gpu.moma_ctx_destroy(h)


def _edge_values(q, W, rng, n):
    L = W // 32
    ones = (1 << (32 * (L - 1))) - 1  # all-ones low words
    base = [0, 1, 2, q - 1, q - 2, q // 2, (q + 1) // 2, ones, q - ones, (1 << (W - 1)) % q]
    vals = [base[i % len(base)] for i in range(n // 2)] + [rng.randrange(q) for _ in range(n - n // 2)]
    rng.shuffle(vals)
    return vals


def test_create_full_checks_modulus(gpu):
    assert gpu.moma_ctx_is_full(0) == 0
    q = inputs.prime_full(256).q
    with pytest.raises(gpu.MomaError):
        gpu.moma_ctx_create_full(q + 1, 256)  # even
    with pytest.raises(gpu.MomaError):
        gpu.moma_ctx_create_full((1 << 200) + 1, 256)  # top limb empty
    h = gpu.moma_ctx_create_full(inputs.prime(256).q, 256)  # a (W-4)-bit modulus is full-width too
    try:
        assert gpu.moma_ctx_is_full(h) == 1
    finally:
        gpu.moma_ctx_destroy(h)
    with pytest.raises(gpu.MomaError):
        gpu.moma_ctx_create(q, 256)  # the Barrett context keeps its W-4 bit contract


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("n", [1, 7, 1000, 4099])
def test_full_width_blas(gpu, fctx, width, n):
    import random
    rng = random.Random(width * 7 + n)
    q = inputs.prime_full(width).q
    L = width // 32
    a = _edge_values(q, width, rng, n)
    b = _edge_values(q, width, rng, n)
    alpha = rng.randrange(q)
    da, db = gpu.to_device(inputs.from_ints(a, L)), gpu.to_device(inputs.from_ints(b, L))
    h = fctx[width]
    for name, fn, want in (("add", gpu.moma_vec_addmod, oracle.vec_addmod(a, b, q)),
                           ("sub", gpu.moma_vec_submod, oracle.vec_submod(a, b, q)),
                           ("mul", gpu.moma_vec_mulmod, oracle.vec_mulmod(a, b, q))):
        dc = torch.empty_like(da)
        fn(h, n, da, db, dc)
        torch.cuda.synchronize()
        assert inputs.to_ints(gpu.to_host(dc)) == want, name
    dc = torch.empty_like(da)
    gpu.moma_vec_axpymod(h, n, alpha, da, db, dc)
    torch.cuda.synchronize()
    assert inputs.to_ints(gpu.to_host(dc)) == oracle.vec_axpy(alpha, a, b, q)


@pytest.mark.parametrize("width", WIDTHS)
def test_full_width_blas_large_sampled(gpu, fctx, width):
    q = inputs.prime_full(width).q
    L = width // 32
    n = 1 << 20
    a = inputs.residues(q, L, n, 1)
    b = inputs.residues(q, L, n, 2)
    da, db = gpu.to_device(a), gpu.to_device(b)
    dc = torch.empty_like(da)
    gpu.moma_vec_mulmod(fctx[width], n, da, db, dc)
    torch.cuda.synchronize()
    idx = np.random.default_rng(width).choice(n, 2000, replace=False)
    ai, bi = inputs.sample_ints(a, idx), inputs.sample_ints(b, idx)
    got = inputs.sample_ints(gpu.to_host(dc), idx)
    assert got == [x * y % q for x, y in zip(ai, bi)]


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("lg", [1, 5, 10, 12, 13, 15])
def test_full_width_ntt(gpu, fctx, width, lg):
    if width >= 512 and lg > 13:
        pytest.skip("the oracle transform at 2^15 and 512 bits or more is slow; 2^13 has the same two-pass split")
    q = inputs.prime_full(width).q
    L = width // 32
    n = 1 << lg
    x = inputs.residues(q, L, n, seed=lg + width)
    xi = inputs.to_ints(x)
    h = fctx[width]
    dx = gpu.to_device(x)
    dy, dz = torch.empty_like(dx), torch.empty_like(dx)
    gpu.moma_ntt_fwd(h, n, dx, dy)
    gpu.moma_ntt_inv(h, n, dy, dz)
    torch.cuda.synchronize()
    assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(xi, q)
    assert torch.equal(dz, dx)
    w = gpu.moma_ctx_root(h, n)
    assert w == oracle.root_of_unity(q, n)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("lg", [3, 11])
def test_full_width_polymul_and_many(gpu, fctx, width, lg):
    q = inputs.prime_full(width).q
    L = width // 32
    n = 1 << lg
    a = inputs.residues(q, L, n, 5)
    b = inputs.residues(q, L, n, 6)
    ai, bi = inputs.to_ints(a), inputs.to_ints(b)
    h = fctx[width]
    da, db = gpu.to_device(a), gpu.to_device(b)
    dc = torch.empty_like(da)
    gpu.moma_polymul(h, n, da, db, dc)
    torch.cuda.synchronize()
    assert inputs.to_ints(gpu.to_host(dc)) == oracle.polymul_cyclic(ai, bi, q)
    # three transforms in one call equal three single calls
    xs = np.stack([inputs.residues(q, L, n, 40 + t) for t in range(3)])
    dx = gpu.to_device(xs)
    dy = torch.empty_like(dx)
    gpu.moma_ntt_fwd_many(h, n, 3, dx, dy)
    torch.cuda.synchronize()
    for t in range(3):
        assert inputs.to_ints(gpu.to_host(dy[t])) == oracle.ntt_fwd(inputs.to_ints(xs[t]), q)


def test_full_width_noalloc(gpu, fctx):
    q = inputs.prime_full(256).q
    h = fctx[256]
    n = 1 << 12
    x = gpu.to_device(inputs.residues(q, 8, n, 9))
    want, got = torch.empty_like(x), torch.empty_like(x)
    gpu.moma_ntt_fwd(h, n, x, want)
    gpu.moma_ntt_fwd_noalloc(h, n, x, got)
    torch.cuda.synchronize()
    assert torch.equal(want, got)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("lg", [1, 6, 11])
def test_full_width_negacyclic(gpu, fctx, width, lg):
    """psi tables in Montgomery form; forward = evaluation at the odd powers of psi."""
    q = inputs.prime_full(width).q
    L = width // 32
    n = 1 << lg
    h = fctx[width]
    a = inputs.residues(q, L, n, 70 + lg)
    b = inputs.residues(q, L, n, 80 + lg)
    ai, bi = inputs.to_ints(a), inputs.to_ints(b)
    da, db = gpu.to_device(a), gpu.to_device(b)
    fa, back, prod = torch.empty_like(da), torch.empty_like(da), torch.empty_like(da)
    gpu.moma_ntt_fwd_negacyclic(h, n, da, fa)
    gpu.moma_ntt_inv_negacyclic(h, n, fa, back)
    gpu.moma_polymul_negacyclic(h, n, da, db, prod)
    torch.cuda.synchronize()
    assert inputs.to_ints(gpu.to_host(fa)) == oracle.ntt_fwd_negacyclic(ai, q)
    assert torch.equal(back, da)
    assert inputs.to_ints(gpu.to_host(prod)) == oracle.negacyclic_convolution_naive(ai, bi, q)


def test_full_width_batch_jobs(gpu):
    """Full-width jobs in a batch (per-call kernels after the persistent launch) next to Barrett jobs;
    direct run, then graph capture and replay, against the oracle."""
    from paper_2501_07535_gb300 import moma
    specs = [("ntt_fwd", 256, 1 << 10, True), ("polymul", 384, 1 << 9, True), ("mul", 768, 3001, True),
             ("axpy", 128, 4096, True), ("ntt_inv", 256, 1 << 11, False), ("add", 256, 999, True)]
    hs, dev, host, alphas = [], [], [], []
    try:
        for i, (op, w, n, full) in enumerate(specs):
            q = inputs.prime_full(w).q if full else inputs.prime(w).q
            h = gpu.moma_ctx_create_full(q, w) if full else gpu.moma_ctx_create(q, w)
            hs.append(h)
            a = inputs.residues(q, w // 32, n, 300 + i)
            b = inputs.residues(q, w // 32, n, 400 + i)
            host.append((q, a, b))
            dev.append((gpu.to_device(a), gpu.to_device(b), torch.empty((w // 32, n), dtype=torch.int32,
                                                                        device="cuda")))
            alphas.append(inputs.scalar_residue(q, 500 + i) if op == "axpy" else None)
        jobs = [{"op": op, "ctx": hs[i], "n": n, "a": dev[i][0], "b": dev[i][1], "out": dev[i][2],
                 "alpha": alphas[i]} for i, (op, w, n, full) in enumerate(specs)]
        bh = moma.moma_batch_create(jobs)
        s = torch.cuda.Stream()
        try:
            with torch.cuda.stream(s):
                for _ in range(3):
                    for d in dev:
                        d[2].zero_()
                    moma.moma_batch_run(bh, s)
            s.synchronize()
            assert moma.moma_batch_sync_status(bh) == 0
        finally:
            moma.moma_batch_destroy(bh)
        for i, (op, w, n, full) in enumerate(specs):
            q, a, b = host[i]
            ai, bi = inputs.to_ints(a), inputs.to_ints(b)
            want = {"ntt_fwd": lambda: oracle.ntt_fwd(ai, q), "ntt_inv": lambda: oracle.ntt_inv(ai, q),
                    "polymul": lambda: oracle.polymul_cyclic(ai, bi, q), "mul": lambda: oracle.vec_mulmod(ai, bi, q),
                    "add": lambda: oracle.vec_addmod(ai, bi, q),
                    "axpy": lambda: oracle.vec_axpy(alphas[i], ai, bi, q)}[op]()
            assert inputs.to_ints(gpu.to_host(dev[i][2])) == want, (op, w, full)
    finally:
        for h in hs:
            gpu.moma_ctx_destroy(h)


def test_full_width_autotune(gpu, fctx):
    q = inputs.prime_full(384).q
    h = fctx[384]
    n = 1 << 12
    best, us = gpu.moma_autotune(h, "ntt_fwd", n, 2)
    assert us > 0
    x = inputs.residues(q, 12, n, 3)
    dx = gpu.to_device(x)
    dy = torch.empty_like(dx)
    gpu.moma_ntt_fwd(h, n, dx, dy)
    torch.cuda.synchronize()
    assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), q)


@pytest.mark.parametrize("width", WIDTHS)
def test_full_width_mulmod_engines_and_moduli(gpu, width):
    """mulmod of full-width contexts by each product engine with the word-based Barrett reduction
    and by two Montgomery products (engine 4): identical, and equal to a * b mod q, for the test
    prime, an odd modulus whose top word is 1 and 2^W - 1."""
    import random
    rng = random.Random(width * 11)
    L = width // 32
    n = 3001
    for q in (inputs.prime_full(width).q, (1 << (width - 32)) + 12345, (1 << width) - 1):
        h = gpu.moma_ctx_create_full(q, width)
        try:
            a = _edge_values(q, width, rng, n)
            b = _edge_values(q, width, rng, n)
            want = [x * y % q for x, y in zip(a, b)]
            da, db = gpu.to_device(inputs.from_ints(a, L)), gpu.to_device(inputs.from_ints(b, L))
            for engine in (1, 2, 3, 4):
                gpu.moma_ctx_set_config(h, "mul", n, engine=engine)
                assert gpu.moma_ctx_get_config(h, "mul", n)["engine"] == engine
                dc = torch.empty_like(da)
                gpu.moma_vec_mulmod(h, n, da, db, dc)
                torch.cuda.synchronize()
                assert inputs.to_ints(gpu.to_host(dc)) == want, (hex(q), engine)
        finally:
            gpu.moma_ctx_destroy(h)


def test_montgomery_engine_only_for_full_width_mulmod(gpu, fctx):
    q = inputs.prime(256).q
    h = gpu.moma_ctx_create(q, 256)
    try:
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(h, "mul", 1024, engine=4)
    finally:
        gpu.moma_ctx_destroy(h)
    with pytest.raises(gpu.MomaError):
        gpu.moma_ctx_set_config(fctx[256], "add", 1024, engine=4)
    with pytest.raises(gpu.MomaError):
        gpu.moma_ctx_set_config(fctx[256], "mul", 1024, engine=5)
