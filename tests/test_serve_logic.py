"""Host logic of the server (admission by memory budget, slots, FIFO, latencies) with a fake
executor: no GPU involved."""
import time

from paper_2501_07535_gb300 import inputs, serve


class FakeExecutor:
    """Each batch takes `per_job_s` per job; completion is visible once the host clock passes it."""

    def __init__(self, per_job_s=2e-4, footprint=lambda j: j.n, clock=time.perf_counter):
        self.per_job = per_job_s
        self.fp = footprint
        self.clock = clock
        self.launches = []

    def start(self, t0):
        self.t0 = t0

    def footprint(self, job):
        return self.fp(job)

    def launch(self, jobs):
        now = self.clock() - self.t0
        done = now + self.per_job * len(jobs)
        self.launches.append((now, done, [j.seed for j in jobs]))
        return done

    def poll(self, handle):
        return handle if self.clock() - self.t0 >= handle else None


def _jobs(n, size=100):
    return [inputs.Job(op="mul", width=256, n=size, seed=i) for i in range(n)]


def test_all_jobs_complete_fifo_and_latency_nonnegative():
    jobs = _jobs(300)
    arrivals = [i * 1e-4 for i in range(300)]
    ex = FakeExecutor()
    st = serve.Scheduler(ex, budget_bytes=10**9, slots=3, max_batch_jobs=16).run(arrivals, jobs)
    assert st.completed == 300 and st.rejected == 0
    assert all(lat >= -1e-9 for lat in st.latencies_s)
    order = [s for _, _, seeds in ex.launches for s in seeds]
    assert order == sorted(order)  # admitted in arrival order
    assert st.max_concurrent_batches <= 3


def test_budget_is_respected_and_oversize_rejected():
    jobs = _jobs(40, size=100) + [inputs.Job(op="mul", width=256, n=10**6, seed=99)]
    arrivals = [0.0] * len(jobs)
    ex = FakeExecutor()
    sched = serve.Scheduler(ex, budget_bytes=450, slots=4, max_batch_jobs=64)
    st = sched.run(arrivals, jobs)
    assert st.rejected == 1 and sched.rejected == [40]
    assert st.completed == 40
    assert st.max_inflight_bytes <= 450
    assert all(len(seeds) <= 4 for _, _, seeds in ex.launches)  # 4 jobs of 100 fit the budget


def test_continuous_batching_admits_while_others_run():
    jobs = _jobs(200)
    arrivals = [i * 5e-5 for i in range(200)]
    ex = FakeExecutor(per_job_s=1e-3)
    st = serve.Scheduler(ex, budget_bytes=10**9, slots=4, max_batch_jobs=8).run(arrivals, jobs)
    assert st.completed == 200
    assert st.max_concurrent_batches >= 2
    # some batch was launched while an earlier one was still running
    overlaps = sum(1 for k in range(1, len(ex.launches)) if ex.launches[k][0] < ex.launches[k - 1][1])
    assert overlaps > 0


def test_served_stream_shape():
    arrivals, jobs = serve.served_jobs(n_jobs=2000, seed=0, rate_per_s=1000.0)
    assert len(jobs) == 2000 and arrivals == sorted(arrivals)
    assert abs(arrivals[-1] / 2000 - 1e-3) < 2e-4  # Poisson rate
    assert {j.width for j in jobs} == {256, 384, 768}
    assert {j.width for j in jobs if j.op.startswith("ntt")} == {256, 384, 768}
    for j in jobs:
        if j.op in ("ntt_fwd", "ntt_inv"):
            assert j.width in (256, 384, 768) and 1 << 12 <= j.n <= 1 << 22
        else:
            assert j.op in ("mul", "axpy") and 1 << 16 <= j.n <= 1 << 24


class CostExecutor(FakeExecutor):
    """A batch takes the sum of its jobs' costs (job.n microseconds)."""

    def cost(self, job):
        return job.n * 1e-6

    def launch(self, jobs):
        now = time.perf_counter() - self.t0
        done = now + sum(self.cost(j) for j in jobs)
        self.launches.append((now, done, [j.seed for j in jobs]))
        return done


def _mixed(n, seed=3):
    import random
    rng = random.Random(seed)
    # 1 in 8 jobs is large (3 ms), the rest small (0.05 ms)
    return [inputs.Job(op="mul", width=256, n=3000 if rng.random() < 0.125 else 50, seed=i) for i in range(n)]


def _small_latencies(st, jobs):
    lat = st.latencies_s
    return sorted(lat[i] for i, j in enumerate(jobs) if j.n == 50)


def test_class_policy_keeps_small_jobs_out_of_large_batches():
    jobs = _mixed(400)
    arrivals = [i * 1.2e-4 for i in range(len(jobs))]
    ex = CostExecutor(footprint=lambda j: 1)
    st = serve.Scheduler(ex, budget_bytes=10**9, slots=4, max_batch_jobs=32, policy="class",
                         large_cost=5e-4, cost_cap=1e-3).run(arrivals, jobs)
    assert st.completed == len(jobs) and st.rejected == 0
    for _, _, seeds in ex.launches:  # every micro-batch is one size class
        assert len({jobs[s].n for s in seeds}) == 1
    # the head of the queue opens each batch: batch heads leave in arrival order
    heads = [seeds[0] for _, _, seeds in ex.launches]
    assert heads == sorted(heads)
    fifo_ex = CostExecutor(footprint=lambda j: 1)
    fifo = serve.Scheduler(fifo_ex, budget_bytes=10**9, slots=4, max_batch_jobs=32).run(arrivals, jobs)
    cls_small, fifo_small = _small_latencies(st, jobs), _small_latencies(fifo, jobs)
    q = int(0.9 * len(cls_small))
    assert cls_small[q] < fifo_small[q]  # small jobs no longer wait for a large one in their batch


def test_class_policy_respects_budget_and_rejects_oversize():
    jobs = _mixed(120) + [inputs.Job(op="mul", width=256, n=10**7, seed=999)]
    arrivals = [0.0] * len(jobs)
    ex = CostExecutor(footprint=lambda j: j.n)
    sched = serve.Scheduler(ex, budget_bytes=7000, slots=4, max_batch_jobs=64, policy="class")
    st = sched.run(arrivals, jobs)
    assert st.rejected == 1 and sched.rejected == [120]
    assert st.completed == 120
    assert st.max_inflight_bytes <= 7000


class SimClock:
    """Simulated time: each reading advances it by a microsecond, a sleep by its length."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-6
        return self.t

    def sleep(self, s):
        self.t += max(s, 1e-6)


def test_latency_grows_with_offered_load(monkeypatch):
    """Two slots of 4-job batches at 1 ms per job serve 2000 jobs/s.  At a quarter of that every
    job runs almost alone (latency about its own 1 ms); at twice that the queue grows through
    the stream and the makespan is set by the capacity."""
    capacity = 2 * 4 / (4 * 1e-3)

    def run(load):
        clk = SimClock()
        monkeypatch.setattr(serve.time, "sleep", clk.sleep)
        ex = FakeExecutor(per_job_s=1e-3, clock=clk)
        arrivals = [i / (load * capacity) for i in range(400)]
        sched = serve.Scheduler(ex, budget_bytes=10**9, slots=2, max_batch_jobs=4, clock=clk, idle_sleep_s=1e-5)
        return sched.run(arrivals, _jobs(400)).summary()

    lo, hi = run(0.25), run(2.0)
    assert lo["completed"] == hi["completed"] == 400
    assert lo["p99_ms"] < 2.5 and lo["mean_ms"] < 1.5
    assert hi["mean_ms"] > 20 * lo["mean_ms"] and hi["p99_ms"] > 20 * lo["p99_ms"]
    assert 0.9 * capacity < hi["jobs_per_s"] < 1.05 * capacity


def test_resident_memory_is_charged_to_the_budget():
    """Tables and operand masters the executor keeps resident count against the budget: beside 250
    resident bytes only two 100-byte jobs fit a 450-byte budget at a time, so the rest wait for
    batches to complete (deferred), and a job that would fit the budget alone but not beside the
    resident memory is refused."""

    class ResidentExecutor(FakeExecutor):
        def resident_bytes(self):
            return 250

    for policy in ("fifo", "class"):
        jobs = _jobs(12, size=100)
        ex = ResidentExecutor()
        st = serve.Scheduler(ex, budget_bytes=450, slots=4, max_batch_jobs=64, policy=policy).run([0.0] * 12, jobs)
        assert st.completed == 12 and st.rejected == 0, policy
        assert all(len(seeds) <= 2 for _, _, seeds in ex.launches), policy
        assert st.resident_bytes == 250 and st.max_inflight_bytes <= 200, policy
        assert st.resident_bytes + st.max_inflight_bytes <= 450
        assert st.deferred_for_memory > 0, policy
        summ = st.summary()
        assert summ["max_total_gb"] <= 450 / 1e9 + 1e-12
        big = [inputs.Job(op="mul", width=256, n=300, seed=50)]
        st2 = serve.Scheduler(ResidentExecutor(), budget_bytes=450, slots=4, policy=policy).run([0.0], big)
        assert st2.rejected == 1 and st2.completed == 0, policy


def test_class_batches_grow_with_the_backlog():
    """With more than `backlog_jobs` queued the cost cap is `backlog_cost_cap`: 300 small jobs
    (0.05 ms each) queued at once leave in 64-job micro-batches (3.2 ms, the job limit) while the
    queue is deep, then in batches of at most 10 (the 0.5 ms cap) once 128 or fewer are queued."""
    jobs = [inputs.Job(op="mul", width=256, n=50, seed=i) for i in range(300)]
    ex = CostExecutor(footprint=lambda j: 1)
    st = serve.Scheduler(ex, budget_bytes=10**9, slots=1, max_batch_jobs=64, policy="class", large_cost=5e-4,
                         cost_cap=5e-4, backlog_jobs=128, backlog_cost_cap=4e-3).run([0.0] * 300, jobs)
    assert st.completed == 300
    sizes = [len(seeds) for _, _, seeds in ex.launches]
    assert sizes[:2] == [64, 64]  # 300 and 236 queued
    queued, deep = 300, []
    for k in sizes:
        deep.append(queued > 128)
        queued -= k
    assert all(k <= 10 for k, d in zip(sizes, deep) if not d)
    assert sum(sizes) == 300 and max(sizes) == 64
    # the same stream with the cap alone never exceeds 10 jobs per micro-batch
    ex2 = CostExecutor(footprint=lambda j: 1)
    serve.Scheduler(ex2, budget_bytes=10**9, slots=1, max_batch_jobs=64, policy="class", cost_cap=5e-4,
                    backlog_jobs=10**6).run([0.0] * 300, jobs)
    assert max(len(s) for _, _, s in ex2.launches) <= 10
