"""Kernel schedules (product engine, tile, radix split, vector width) and the autotuner.

Every schedule must give bit-identical results; the autotuner's choice is checked the
same way against the oracle.
"""
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [128, 256, 384])
@pytest.mark.parametrize("engine", [1, 2])
def test_ntt_every_engine_and_split(gpu, width, engine):
    p = inputs.prime(width)
    ctx = gpu.moma_ctx_create(p.q, width)
    try:
        for lg, tile, rmax, th, tight in ((10, 11, 6, 256, 0), (13, 10, 5, 256, 0), (13, 11, 8, 128, 0),
                                          (15, 12, 7, 256, 0), (13, 8, 5, 32, 1), (16, 9, 6, 64, 0),
                                          (10, 10, 7, 128, 1), (7, 8, 5, 32, 0), (14, 9, 5, 128, 1)):
            if tile > 12 and p.L == 12:
                continue
            n = 1 << lg
            kw = dict(engine=engine, tile_log=tile, max_logr=rmax, cta_threads=th, tight_regs=tight)
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", n, **kw)
            gpu.moma_ctx_set_config(ctx, "ntt_inv", n, **kw)
            cfg = gpu.moma_ctx_get_config(ctx, "ntt_fwd", n)
            assert (cfg["engine"], cfg["tile_log"], cfg["max_logr"], cfg["cta_threads"], cfg["tight_regs"]) == \
                (engine, tile, rmax, th, tight)
            x = inputs.residues(p.q, p.L, n, seed=lg + engine)
            dx = gpu.to_device(x)
            dy = torch.empty_like(dx)
            gpu.moma_ntt_fwd(ctx, n, dx, dy)
            dz = torch.empty_like(dx)
            gpu.moma_ntt_inv(ctx, n, dy, dz)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), p.q), (lg, tile, rmax)
            assert torch.equal(dz, dx)
    finally:
        gpu.moma_ctx_destroy(ctx)


WIDE_SCHEDULES = {
    # (log2 n, tile_log, max_logr, cta_threads, tight_regs); tiles within shared memory at each width
    512: ((13, 10, 5, 128, 0), (14, 11, 6, 256, 0), (12, 9, 4, 64, 0)),
    768: ((13, 9, 4, 128, 1), (14, 10, 5, 128, 1), (13, 11, 7, 256, 0), (12, 10, 5, 64, 0), (11, 8, 4, 32, 1)),
    1024: ((13, 9, 5, 128, 0), (12, 10, 6, 256, 0)),
}


@pytest.mark.parametrize("width", [512, 768, 1024])
@pytest.mark.parametrize("engine", [1, 2])
def test_ntt_wide_schedules(gpu, width, engine):
    """Schedules other than the default at 512 to 1024 bits (the autotuner's candidates), forward
    against the oracle and round trip; from 512 bits the whole-product rows and the register cap
    exist at 768 bits only, elsewhere they fall back to carry chains."""
    p = inputs.prime(width)
    ctx = gpu.moma_ctx_create(p.q, width)
    try:
        for lg, tile, rmax, th, tight in WIDE_SCHEDULES[width]:
            n = 1 << lg
            kw = dict(engine=engine, tile_log=tile, max_logr=rmax, cta_threads=th, tight_regs=tight)
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", n, **kw)
            gpu.moma_ctx_set_config(ctx, "ntt_inv", n, **kw)
            x = inputs.residues(p.q, p.L, n, seed=lg + 7 * engine)
            dx = gpu.to_device(x)
            dy, dz = torch.empty_like(dx), torch.empty_like(dx)
            gpu.moma_ntt_fwd(ctx, n, dx, dy)
            gpu.moma_ntt_inv(ctx, n, dy, dz)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), p.q), (lg, tile, rmax, th)
            assert torch.equal(dz, dx)
    finally:
        gpu.moma_ctx_destroy(ctx)


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
@pytest.mark.parametrize("engine", [1, 2])
def test_blas_every_engine_and_width(gpu, width, engine):
    p = inputs.prime(width)
    ctx = gpu.moma_ctx_create(p.q, width)
    try:
        n = 4096 + 4
        a = inputs.residues(p.q, p.L, n, 1)
        b = inputs.residues(p.q, p.L, n, 2)
        ai, bi = inputs.to_ints(a), inputs.to_ints(b)
        alpha = inputs.scalar_residue(p.q, 5)
        da, db = gpu.to_device(a), gpu.to_device(b)
        for vw in (1, 2, 4):
            for op in ("mul", "axpy"):
                gpu.moma_ctx_set_config(ctx, op, n, engine=engine, vec_width=vw)
            dc = torch.empty_like(da)
            gpu.moma_vec_mulmod(ctx, n, da, db, dc)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(dc)) == oracle.vec_mulmod(ai, bi, p.q), vw
            gpu.moma_vec_axpymod(ctx, n, alpha, da, db, dc)
            torch.cuda.synchronize()
            assert inputs.to_ints(gpu.to_host(dc)) == oracle.vec_axpy(alpha, ai, bi, p.q), vw
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_autotune_ntt_and_mul(gpu):
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        n = 1 << 14
        best, us = gpu.moma_autotune(ctx, "ntt_fwd", n, 4)
        assert best["engine"] in (1, 2) and us > 0
        assert gpu.moma_ctx_get_config(ctx, "ntt_fwd", n) == best
        x = inputs.residues(p.q, p.L, n, 3)
        dx = gpu.to_device(x)
        dy = torch.empty_like(dx)
        gpu.moma_ntt_fwd(ctx, n, dx, dy)
        torch.cuda.synchronize()
        assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), p.q)
        best, us = gpu.moma_autotune(ctx, "mul", 1 << 16)
        assert best["vec_width"] in (1, 2, 4) and us > 0
        best, us = gpu.moma_autotune(ctx, "polymul", 1 << 12)
        assert us > 0
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_config_rejects_invalid(gpu):
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", 1 << 10, tile_log=30)
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", 1 << 10, engine=7)
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, "mul", 1 << 10, vec_width=3)
        with pytest.raises(gpu.MomaError):  # the staged tile is fixed per width (2^9 at 256 bits)
            gpu.moma_ctx_set_config(ctx, "mul", 1 << 10, tile_log=8)
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", 1 << 10, engine=3)
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, 99, 1 << 10)
        with pytest.raises(gpu.MomaError):
            gpu.moma_ctx_set_config(ctx, "ntt_fwd", 1 << 10, cta_threads=256, tight_regs=1)
    finally:
        gpu.moma_ctx_destroy(ctx)


def test_schedule_table_round_trip(gpu, tmp_path):
    """Autotuned schedules saved as JSON, loaded and applied to a fresh context: the same effective
    schedules, and the transform under them still equals the oracle's."""
    from paper_2501_07535_gb300 import schedules
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    ctx2 = gpu.moma_ctx_create(p.q, 256)
    try:
        n = 1 << 13
        t = schedules.Table()
        best = schedules.tune(t, ctx, 256, "ntt_fwd", n, count=2)
        schedules.tune(t, ctx, 256, "mul", 4096)
        path = str(tmp_path / "schedules.json")
        t.save(path)
        assert schedules.apply(schedules.Table.load(path), ctx2, 256) == 2
        assert gpu.moma_ctx_get_config(ctx2, "ntt_fwd", n) == best
        assert gpu.moma_ctx_get_config(ctx2, "mul", 4096) == gpu.moma_ctx_get_config(ctx, "mul", 4096)
        x = inputs.residues(p.q, p.L, n, 21)
        dx = gpu.to_device(x)
        dy = torch.empty_like(dx)
        gpu.moma_ntt_fwd(ctx2, n, dx, dy)
        torch.cuda.synchronize()
        assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), p.q)
    finally:
        gpu.moma_ctx_destroy(ctx)
        gpu.moma_ctx_destroy(ctx2)


def test_autotune_keeps_only_the_winners_plan(gpu):
    """The autotuner builds a plan (twiddle tables) per candidate split (more than twenty of them);
    the losers' plans are freed, so the context holds at most one more plan than before (the
    winner's, whose tables can be a little larger than the default split's), and the winner's
    schedule still gives the oracle's transform."""
    p = inputs.prime(256)
    ctx = gpu.moma_ctx_create(p.q, 256)
    try:
        n = 1 << 14
        x = inputs.residues(p.q, p.L, n, 31)
        dx = gpu.to_device(x)
        dy = torch.empty_like(dx)
        gpu.moma_ntt_fwd(ctx, n, dx, dy)  # the default schedule's plan
        torch.cuda.synchronize()
        base = gpu.moma_ctx_device_bytes(ctx)
        gpu.moma_autotune(ctx, "ntt_fwd", n, 1)
        after = gpu.moma_ctx_device_bytes(ctx)
        assert base <= after <= 2.5 * base
        gpu.moma_ntt_fwd(ctx, n, dx, dy)
        torch.cuda.synchronize()
        assert inputs.to_ints(gpu.to_host(dy)) == oracle.ntt_fwd(inputs.to_ints(x), p.q)
    finally:
        gpu.moma_ctx_destroy(ctx)
