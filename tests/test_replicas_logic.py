"""Sharding helpers of the replicated runs on CPU (no process group): the cost-balanced share of an
uneven batch and the round-robin share of a served stream are disjoint, complete and deterministic."""
from paper_2501_07535_gb300 import inputs, replicas, serve


def test_shard_balanced_partitions_and_balances():
    jobs = inputs.uneven_batch(n_jobs=200, seed=4)
    for world in (1, 2, 3, 8):
        shares = [replicas.shard_balanced(jobs, r, world, replicas.job_cost) for r in range(world)]
        seeds = [j.seed for sh in shares for j in sh]
        assert sorted(seeds) == sorted(j.seed for j in jobs) and len(seeds) == len(set(seeds))
        for sh in shares:  # each share keeps the original order
            pos = [jobs.index(j) for j in sh]
            assert pos == sorted(pos)
        loads = [sum(replicas.job_cost(j) for j in sh) for sh in shares]
        assert max(loads) - min(loads) <= max(replicas.job_cost(j) for j in jobs)
        # the same assignment on every call (every rank computes it alone)
        assert shares == [replicas.shard_balanced(jobs, r, world, replicas.job_cost) for r in range(world)]


def test_job_cost_orders_work():
    small = inputs.Job(op="ntt_fwd", width=128, n=1 << 10, seed=0)
    big = inputs.Job(op="ntt_fwd", width=384, n=1 << 20, seed=1)
    prod = inputs.Job(op="polymul", width=384, n=1 << 20, seed=2)
    vec = inputs.Job(op="mul", width=384, n=1 << 20, seed=3)
    assert replicas.job_cost(small) < replicas.job_cost(vec) < replicas.job_cost(big) < replicas.job_cost(prod)
    assert replicas.job_cost(prod) == 3 * replicas.job_cost(big)


def test_rank_share_of_a_stream():
    arrivals, jobs = inputs.served_stream(n_jobs=101, seed=2, rate_per_s=1000.0)
    parts = [serve.rank_share(arrivals, jobs, r, 3) for r in range(3)]
    got = sorted((a, j.seed) for arr, js in parts for a, j in zip(arr, js))
    assert got == sorted((a, j.seed) for a, j in zip(arrivals, jobs))
    assert [len(p[1]) for p in parts] == [34, 34, 33]
    for arr, _ in parts:
        assert arr == sorted(arr)
    assert serve.rank_share(arrivals, jobs, 0, 1) == (list(arrivals), list(jobs))
