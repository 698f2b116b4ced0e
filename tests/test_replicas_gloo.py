"""Replica helpers with two gloo ranks on CPU (the N > 1 path without GPUs)."""
import os
import socket

import torch.multiprocessing as mp

from paper_2501_07535_gb300 import inputs, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world_size, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world_size),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    replicas.init("gloo")
    replicas.barrier()
    mx = replicas.max_over_ranks(float(rank + 1))
    sm = replicas.sum_over_ranks(float(10 * (rank + 1)))
    jobs = inputs.uneven_batch(n_jobs=10, seed=1)
    mine = [j.seed for j in replicas.shard(jobs, rank, world_size)]
    replicas.barrier()
    replicas.finalize()
    out[rank] = (mx, sm, mine)


def test_two_gloo_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == out[1][1] == 30.0
    seeds = sorted(out[0][2] + out[1][2])
    assert seeds == sorted(j.seed for j in inputs.uneven_batch(n_jobs=10, seed=1))
    assert not set(out[0][2]) & set(out[1][2])


def _serve_rank_main(rank, world_size, port, out):
    """One rank of a replicated server: schedules its share of a served stream through the CPU
    Scheduler with a fake executor, and its share of an uneven batch by cost."""
    import torch.distributed as dist

    from paper_2501_07535_gb300 import serve
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world_size),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    replicas.init("gloo")

    class Fake:
        def start(self, t0):
            self.launched = []

        def footprint(self, job):
            return 4 * (job.width // 32) * job.n

        def launch(self, jobs):
            self.launched += [j.seed for j in jobs]
            return True

        def poll(self, handle):
            return 0.0

    arrivals, jobs = inputs.served_stream(n_jobs=300, seed=5, rate_per_s=1e6)
    ex = Fake()
    st = serve.serve(arrivals, jobs, None, slots=2, executor=ex, policy="class", rank=rank, world_size=world_size)
    mine_batch = [j.seed for j in replicas.shard_balanced(inputs.uneven_batch(n_jobs=64, seed=2), rank, world_size,
                                                          replicas.job_cost)]
    gathered = [None] * world_size
    dist.all_gather_object(gathered, (sorted(ex.launched), st.completed, mine_batch))
    replicas.finalize()
    out[rank] = gathered


def test_two_gloo_ranks_share_served_stream_and_batch():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_serve_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]  # every rank saw the same gathered result
    (s0, c0, b0), (s1, c1, b1) = out[0]
    _, jobs = inputs.served_stream(n_jobs=300, seed=5, rate_per_s=1e6)
    assert not set(s0) & set(s1) and sorted(s0 + s1) == sorted(j.seed for j in jobs)
    assert c0 + c1 == 300 and abs(c0 - c1) <= 1
    batch = inputs.uneven_batch(n_jobs=64, seed=2)
    assert not set(b0) & set(b1) and sorted(b0 + b1) == sorted(j.seed for j in batch)
    cost = {j.seed: replicas.job_cost(j) for j in batch}
    loads = [sum(cost[s] for s in b0), sum(cost[s] for s in b1)]
    assert max(loads) - min(loads) <= max(cost.values())  # greedy balance: within one job
