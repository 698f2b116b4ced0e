"""The persistent batch launch: uneven sizes, mixed widths, fused cyclic products, graph replay.

Every job's output must equal the oracle and the same job run alone through the plain
per-call API (bit-exact); a missing dependency must end in MOMA_ERR_TIMEOUT, not a hang.
"""
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import batch, inputs, moma

pytestmark = pytest.mark.gpu


def _oracle(job, a, b, alpha, q):
    if job.op == "ntt_fwd":
        return oracle.ntt_fwd(a, q)
    if job.op == "ntt_inv":
        return oracle.ntt_inv(a, q)
    if job.op == "polymul":
        return oracle.polymul_cyclic(a, b, q)
    if job.op == "add":
        return oracle.vec_addmod(a, b, q)
    if job.op == "sub":
        return oracle.vec_submod(a, b, q)
    if job.op == "mul":
        return oracle.vec_mulmod(a, b, q)
    return oracle.vec_axpy(alpha, a, b, q)


def _mixed_jobs():
    jobs = inputs.uneven_batch(n_jobs=24, seed=5, log_n_range=(1, 13), widths=(128, 256, 384))
    jobs += [inputs.Job(op=op, width=w, n=n, seed=3000 + i)
             for i, (op, w, n) in enumerate([("add", 768, 5000), ("sub", 128, 4099), ("mul", 256, 2048),
                                             ("axpy", 384, 3), ("mul", 768, 777), ("axpy", 128, 10000),
                                             ("ntt_fwd", 768, 1 << 10), ("ntt_inv", 768, 1 << 12),
                                             ("polymul", 768, 1 << 9), ("ntt_fwd", 768, 2)])]
    return jobs


def test_batch_matches_oracle_and_plain(gpu):
    js = batch.JobSet(_mixed_jobs())
    try:
        js.run_batched(torch.cuda.current_stream())
        assert js.status() == 0
        torch.cuda.synchronize()
        got = [moma.to_host(o).copy() for o in js.out]
        for i, j in enumerate(js.jobs):
            q = inputs.prime(j.width, j.prime_seed).q
            a = inputs.to_ints(js.host_a[i])
            b = inputs.to_ints(js.host_b[i]) if js.host_b[i] is not None else None
            assert inputs.to_ints(got[i]) == _oracle(j, a, b, js.alpha[i], q), (i, j)
        # the same jobs through the plain per-call API give the same words
        for o in js.out:
            o.zero_()
        js.run_plain()
        torch.cuda.synchronize()
        for i in range(len(js.jobs)):
            assert (moma.to_host(js.out[i]) == got[i]).all(), i
        # graph replay (second run of the same batch) on a side stream
        for o in js.out:
            o.zero_()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            js.run_batched(s)
            js.run_batched(s)
        s.synchronize()
        assert js.status() == 0
        for i in range(len(js.jobs)):
            assert (moma.to_host(js.out[i]) == got[i]).all(), i
    finally:
        js.close()
        js.ctx.close()


def test_batch_of_768bit_transforms_only(gpu):
    """768-bit transforms run as per-pass launches after the persistent launch; a batch with
    nothing else skips the persistent launch.  Direct run, then graph capture and replay."""
    jobs = [inputs.Job(op=op, width=768, n=n, seed=4000 + i)
            for i, (op, n) in enumerate([("ntt_fwd", 1 << 11), ("polymul", 1 << 8), ("ntt_inv", 1 << 9)])]
    js = batch.JobSet(jobs)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for _ in range(3):
                for o in js.out:
                    o.zero_()
                js.run_batched(s)
        s.synchronize()
        assert js.status() == 0
        for i, j in enumerate(js.jobs):
            q = inputs.prime(j.width, j.prime_seed).q
            a = inputs.to_ints(js.host_a[i])
            b = inputs.to_ints(js.host_b[i]) if js.host_b[i] is not None else None
            assert inputs.to_ints(moma.to_host(js.out[i])) == _oracle(j, a, b, None, q), (i, j)
    finally:
        js.close()
        js.ctx.close()


def test_uneven_workload_reduced_sizes(gpu):
    """The uneven mix (fwd / inv / cyclic products at 128-384 bits), sizes 2^10..2^14."""
    jobs = inputs.uneven_batch(n_jobs=32, seed=0, log_n_range=(10, 14))
    js = batch.JobSet(jobs)
    try:
        js.run_batched(torch.cuda.current_stream())
        assert js.status() == 0
        torch.cuda.synchronize()
        for i, j in enumerate(js.jobs):
            q = inputs.prime(j.width).q
            a = inputs.to_ints(js.host_a[i])
            b = inputs.to_ints(js.host_b[i]) if js.host_b[i] is not None else None
            assert inputs.to_ints(moma.to_host(js.out[i])) == _oracle(j, a, b, None, q), (i, j)
    finally:
        js.close()
        js.ctx.close()


def test_batch_bounded_wait_reports_timeout(gpu):
    jobs = [inputs.Job(op="ntt_fwd", width=256, n=1 << 12, seed=1), inputs.Job(op="polymul", width=128, n=1 << 11, seed=2)]
    js = batch.JobSet(jobs)
    try:
        b = js.create_batch()
        moma.moma_batch_set_wait_limit(b, 1 << 12)
        moma.moma_batch_inject_missing_dependency(b)
        moma.moma_batch_run(b, torch.cuda.current_stream())
        assert moma.moma_batch_sync_status(b) == 7  # MOMA_ERR_TIMEOUT, and the launch ended
        assert moma.moma_batch_sync_status(b) == 0  # cleared
    finally:
        js.close()
    js2 = batch.JobSet(jobs, js.ctx)
    try:
        js2.run_batched(torch.cuda.current_stream())
        assert js2.status() == 0  # a fresh batch of the same jobs completes normally
    finally:
        js2.close()
        js.ctx.close()


def test_batch_argument_errors(gpu):
    ctx = moma.moma_ctx_create(inputs.prime(256).q, 256)
    try:
        x = moma.to_device(inputs.residues(inputs.prime(256).q, 8, 64, 1))
        with pytest.raises(moma.MomaError):
            moma.moma_batch_create([{"op": 9, "ctx": ctx, "n": 64, "a": x, "out": x}])
        with pytest.raises(moma.MomaError):
            moma.moma_batch_create([{"op": "ntt_fwd", "ctx": ctx, "n": 63, "a": x, "out": x}])
        with pytest.raises(moma.MomaError):
            moma.moma_batch_create([{"op": "polymul", "ctx": ctx, "n": 64, "a": x, "out": x}])  # no b
        assert moma.moma_batch_submit([{"op": "ntt_fwd", "ctx": ctx, "n": 64, "a": x, "out": x}]) == 0
    finally:
        moma.moma_ctx_destroy(ctx)
