"""The server on the GPU: every job's result in the mix equals the job run alone."""
import pytest
import torch

import oracle
from paper_2501_07535_gb300 import batch, inputs, moma, serve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["fifo", "class"])
def test_served_results_equal_alone(gpu, policy):
    arrivals, jobs = inputs.served_stream(n_jobs=160, seed=3, rate_per_s=20000.0, ntt_log_range=(6, 12),
                                          vec_log_range=(8, 14))
    assert any(j.width == 768 and j.op.startswith("ntt") for j in jobs)
    ctxs = batch.Contexts()
    ex = serve.GpuExecutor(ctxs, slots=4, keep_outputs=True, master_log=12)
    try:
        ex.prewarm(jobs)
        st = serve.serve(arrivals, jobs, ctxs, slots=4, max_batch_jobs=16, executor=ex, policy=policy)
        torch.cuda.synchronize()
        assert st.completed == len(jobs) and st.rejected == 0
        assert st.max_concurrent_batches >= 1
        for j in jobs:
            got = ex.outputs[j.seed]
            a = ex.operand(j, 0)
            alone = torch.empty_like(a)
            c = ctxs.get(j.width, j.prime_seed)
            if j.op == "ntt_fwd":
                moma.moma_ntt_fwd(c, j.n, a, alone)
            elif j.op == "ntt_inv":
                moma.moma_ntt_inv(c, j.n, a, alone)
            elif j.op == "mul":
                moma.moma_vec_mulmod(c, j.n, a, ex.operand(j, 1), alone)
            else:
                al = inputs.scalar_residue(inputs.prime(j.width, j.prime_seed).q, j.seed)
                moma.moma_vec_axpymod(c, j.n, al, a, ex.operand(j, 1), alone)
            torch.cuda.synchronize()
            assert torch.equal(got, alone), j
        # spot-check a few against the oracle
        for j in jobs[:6]:
            q = inputs.prime(j.width, j.prime_seed).q
            a = inputs.to_ints(moma.to_host(ex.operand(j, 0)))
            got = inputs.to_ints(moma.to_host(ex.outputs[j.seed]))
            if j.op == "ntt_fwd":
                assert got == oracle.ntt_fwd(a, q)
            elif j.op == "ntt_inv":
                assert got == oracle.ntt_inv(a, q)
            elif j.op == "mul":
                assert got == oracle.vec_mulmod(a, inputs.to_ints(moma.to_host(ex.operand(j, 1))), q)
    finally:
        ctxs.close()
