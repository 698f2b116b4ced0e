"""Benchmark: 256-bit 2^20-point NTT throughput and 2^24-element mulmod throughput on GB300.

One JSON line on rank 0.  `value` is forward 2^20-point NTTs per second over a 252-bit
prime (256-bit container, L = 8 limbs), steady state over batches of 16 transforms per
step (the paper reports steady-state batched runs, Sec. 5.1).  The mulmod figure
(Gelem/s over 2^24 elements, same modulus) and its roofline are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: CUDA events on the launching stream, W untimed warm-up steps, K timed steps
bracketed by a barrier and a device synchronisation; inputs are larger than L2 (512 MiB
per NTT step, 1.5 GiB per mulmod step).  For N > 1 (torchrun) every rank runs its own
replica (the work is independent per transform) and the time is the max over ranks.
`--impl reference` times the CPU oracle (Python big integers) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "256-bit 2^20 NTT/s & mulmod Gelem/s vs roofline; batched/plain speedup; p99 latency"
WIDTH = 256
LOGN = 20
NTT_BATCH = 16
VEC_N = 1 << 24
L = WIDTH // 32


# DRAM bytes per pass launch of the dominant kernel (ntt_pass_kernel<8>, 16 transforms of 2^20):
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of a pass over 8 transforms, x 2;
# valid for this schedule and kernel version (None otherwise).
NTT_PASS_TRAFFIC_BYTES = 961_867_776
NTT_PASS_TRAFFIC_SCHEDULE = {"engine": 2, "tile_log": 10, "max_logr": 5, "cta_threads": 128, "tight_regs": 0}

# Integer-multiply peak from the unit counts: the multiply pipe (fmaheavy) of each of the 4 SM
# sub-partitions takes one whole 32x32->64 product (mad.wide) per 4 cycles per warp, i.e. 8 lane
# products per clock, 32 per SM per clock (moma_probe_imad measures the 4 cycles).
PRODUCTS_PER_CLK_PER_SM = 32


def word_products_per_mulmod(L):
    """Algorithmic 32x32->64 word products of one L-limb modular multiplication: 2L^2 + L."""
    return 2 * L * L + L


def product_peak(sms, sm_mhz):
    """Unit-count integer-multiply peak in word products per second."""
    return sms * PRODUCTS_PER_CLK_PER_SM * sm_mhz * 1e6


def ntt_roofline(n, limbs, batch, step_s, prod_peak):
    """Transform region: algorithmic word products per second ((n/2) log2 n mulmods of 2L^2 + L
    products for each of `batch` transforms in `step_s` seconds) against the product peak."""
    logn = n.bit_length() - 1
    prod = word_products_per_mulmod(limbs) * (n // 2) * logn * batch
    achieved = prod / step_s / 1e12
    peak = prod_peak / 1e12
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "T word-products/s",
            "frac": round(achieved / peak, 4)}


def vec_roofline(limbs, n, step_s, hbm_gbs, prod_peak, products=True):
    """Element-wise op over n elements in `step_s` seconds: the roofline time is the slower of its
    bytes (two operands read, one written) at the HBM peak and, for products, its 2L^2 + L word
    products per element at the product peak."""
    nbytes = 3 * 4 * limbs * n
    prod = word_products_per_mulmod(limbs) * n if products else 0
    t_hbm = nbytes / (hbm_gbs * 1e9) if hbm_gbs else 0.0
    t_prod = prod / prod_peak
    roof = max(t_hbm, t_prod)
    return {"bound": "hbm" if t_hbm >= t_prod else "alu", "time_us": round(roof * 1e6, 2),
            "achieved_us": round(step_s * 1e6, 2), "frac": round(roof / step_s, 4),
            "hbm_gbs_achieved": round(nbytes / step_s / 1e9, 1), "hbm_gbs_peak": hbm_gbs,
            "products_t_achieved": round(prod / step_s / 1e12, 3), "products_t_peak": round(prod_peak / 1e12, 3)}


# ----------------------------------------------------------------------------- CPU oracle

def _oracle_ntt_worker(args):
    q, logn, seed = args
    import oracle
    from paper_2501_07535_gb300 import inputs
    x = inputs.to_ints(inputs.residues(q, L, 1 << logn, seed))
    t = time.perf_counter()
    oracle.ntt_fwd(x, q)
    return time.perf_counter() - t


def _oracle_mulmod_worker(args):
    q, n, seed = args
    import oracle
    from paper_2501_07535_gb300 import inputs
    a = inputs.to_ints(inputs.residues(q, L, n, seed))
    b = inputs.to_ints(inputs.residues(q, L, n, seed + 1))
    t = time.perf_counter()
    oracle.vec_mulmod(a, b, q)
    return time.perf_counter() - t


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_ntt_rate(pool, cores, q, logn=LOGN):
    """All cores each run one full-size forward NTT; NTT/s = cores / wall time."""
    t = time.perf_counter()
    pool.map(_oracle_ntt_worker, [(q, logn, 1000 + i) for i in range(cores)])
    wall = time.perf_counter() - t
    return cores / wall, wall


def oracle_mulmod_rate(pool, cores, q, n=1 << 19):
    t = time.perf_counter()
    pool.map(_oracle_mulmod_worker, [(q, n, 2000 + 2 * i) for i in range(cores)])
    wall = time.perf_counter() - t
    return cores * n / wall / 1e9, wall


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling (every 20 ms) around the measured phase; waits for the first sample."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def _reader(self):
        for ln in self.proc.stdout:
            if ln.strip():
                self.lines.append(ln)

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._reader, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 10:
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def bench_config(world=1):
    """The workload the line's value is quoted on (shared by both arms)."""
    return {"workload": f"forward cyclic NTT, n=2^{LOGN}, 256-bit container (252-bit prime), {NTT_BATCH} transforms "
                        f"per step", "n": 1 << LOGN, "bits": WIDTH, "limbs": L, "batch": NTT_BATCH,
            "l2": "inputs larger than L2 (512 MiB per NTT step, 1.5 GiB per mulmod step)",
            "parallelism": f"replicas x{world}"}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2501_07535_gb300 import build, inputs, moma, replicas

    world, rank, local = replicas.world()
    if world > 1:
        torch.cuda.set_device(local)
        replicas.init("nccl")

    # CPU oracle pool: spawned before any GPU work (rank 0 only)
    pool = None
    cores = _cores()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)

    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    p = inputs.prime(WIDTH)
    q = p.q
    ctx = moma.moma_ctx_create(q, WIDTH)
    st = torch.cuda.current_stream()
    n = 1 << LOGN
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, dev)

    # ---- inputs (resident in HBM)
    xs = np.stack([inputs.residues(q, L, n, seed=10 + t + 100 * rank) for t in range(NTT_BATCH)])
    dx = moma.to_device(xs, dev)
    dy = torch.empty_like(dx)
    a = moma.to_device(inputs.residues(q, L, VEC_N, seed=1 + 10 * rank), dev)
    b = moma.to_device(inputs.residues(q, L, VEC_N, seed=2 + 10 * rank), dev)
    c = torch.empty_like(a)

    # plan set-up (twiddle tables) happens on the first call, outside the timed region
    moma.moma_ntt_fwd_many(ctx, n, NTT_BATCH, dx, dy)
    torch.cuda.synchronize()
    ntt_cfg = moma.moma_ctx_get_config(ctx, "ntt_fwd", n)
    mul_cfg = moma.moma_ctx_get_config(ctx, "mul", VEC_N)
    n_pass_launches = _pass_count(ntt_cfg, LOGN)

    # ---- integer-multiply peak (same run, same GPU): the fastest word-product form measured
    # (mad.wide gives one 32x32->64 product per instruction; a lo/hi carry-chain pair needs two)
    probe = {}
    for variant, per_op in ((5, 1.0), (0, 0.5)):
        pms, pops = moma.moma_probe_imad(variant, sms * 8, 256, 2000)
        probe[variant] = pops * per_op / (pms * 1e-3)
    probe_peak = max(probe.values())  # word products / s, fastest form measured in this run
    sm_max_mhz = _measured_peaks().get("sm_max_mhz") or 2070.0
    prod_peak = product_peak(sms, sm_max_mhz)  # unit-count peak at the max SM clock
    hbm = _measured_peaks().get("hbm_gbs")

    # ---- NTT region
    def ntt_step():
        moma.moma_ntt_fwd_many(ctx, n, NTT_BATCH, dx, dy)

    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        ntt_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ntt_step()
    e1.record(st)
    barrier()
    ntt_ms = max_over_ranks(e0.elapsed_time(e1))
    ntt_per_s = world * NTT_BATCH * args.steps / (ntt_ms * 1e-3)

    # ---- mulmod region
    def mul_step():
        moma.moma_vec_mulmod(ctx, VEC_N, a, b, c)

    for _ in range(args.warmup):
        mul_step()
    barrier()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(st)
    for _ in range(args.steps):
        mul_step()
    m1.record(st)
    barrier()
    mul_ms = max_over_ranks(m0.elapsed_time(m1))
    gelem = world * VEC_N * args.steps / (mul_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the region
    e2e_ms_local, e2e_ok = measure_e2e(ctx, xs, n, args.steps, args.warmup, barrier)
    assert e2e_ok
    e2e_ms = max_over_ranks(e2e_ms_local)
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    e2e = world * NTT_BATCH * args.steps / (e2e_ms * 1e-3)
    step_bytes = NTT_BATCH * L * n * 4
    del xs, dx, dy, a, b, c
    torch.cuda.empty_cache()

    # ---- roofline
    roof = ntt_roofline(n, L, NTT_BATCH, ntt_ms * 1e-3 / args.steps, prod_peak)
    mul_roof = vec_roofline(L, VEC_N, mul_ms * 1e-3 / args.steps, hbm, prod_peak)
    launches = args.steps * n_pass_launches  # pass kernels in the timed NTT region

    # ---- the other workloads (bulky tables first in the line, the headline block last)
    sens = run_sensitivity()
    c3 = run_c3_sweep(prod_peak) if not args.quick else None
    c2 = run_c2_table(hbm, prod_peak) if not args.quick else None
    c1 = run_c1_latency()
    c4 = run_uneven_batch(max(3, args.steps // 2), 2)
    c5 = run_served(n_jobs=args.serve_jobs) if args.serve_jobs > 0 else None

    result = {
        "metric": METRIC,
        "value": round(ntt_per_s, 2),
        "unit": "NTT/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ntt_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic: seeded uniform residues mod a seed-generated 252-bit prime q = c*2^32+1",
        "config": bench_config(world),
        "sensitivity": sens,
        "c3_ntt_sweep": c3,
        "c2_blas": c2,
        "c1_single_ntt": c1,
        "batched_vs_plain": c4,
        "served": c5,
        "multiply_probe": {"wide_t_products_per_s": round(probe[5] / 1e12, 3),
                           "carry_chain_t_products_per_s": round(probe[0] / 1e12, 3), "sms": sms},
        "schedule": {"ntt_fwd": ntt_cfg, "mul": mul_cfg},
        "e2e": {"value": round(e2e, 2), "unit": "NTT/s", "h2d_bytes_per_step": step_bytes,
                "d2h_bytes_per_step": step_bytes},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {**roof,
                     "traffic": NTT_PASS_TRAFFIC_BYTES if all(ntt_cfg.get(k) == v for k, v in
                                                              NTT_PASS_TRAFFIC_SCHEDULE.items()) else None,
                     "peak_source": f"{sms} SMs x {PRODUCTS_PER_CLK_PER_SM} whole 32x32->64 products (mad.wide) "
                                    f"per clock per SM x {sm_max_mhz:.0f} MHz max SM clock",
                     "peak_probe": round(probe_peak / 1e12, 3),
                     "frac_of_probe": round(roof["achieved"] / (probe_peak / 1e12), 4),
                     "algorithmic": f"(n/2)log2(n) mulmods x (2L^2+L) = {word_products_per_mulmod(L)} word "
                                    f"products per mulmod, {NTT_BATCH} transforms per step",
                     "mulmod": {"gelem_s": round(gelem, 3), "n": VEC_N, "bits": WIDTH,
                                "ms_per_step": round(mul_ms / args.steps, 4), **mul_roof}},
    }
    if pool is not None:
        rate, wall = oracle_ntt_rate(pool, cores, q)
        mrate, mwall = oracle_mulmod_rate(pool, cores, q)
        pool.close()
        result["cpu_baseline"] = {"value": round(rate, 4), "unit": "NTT/s", "cores": cores, "kind": "oracle",
                                  "sample": f"{cores} full 2^{LOGN}-point forward NTTs, one per core "
                                            f"({wall:.1f} s wall)",
                                  "mulmod": {"value": round(mrate, 6), "unit": "Gelem/s",
                                             "sample": f"{cores} x 2^19-element mulmod ({mwall:.1f} s wall)"}}
    result["headline"] = headline(result)
    if rank == 0:
        print(json.dumps(result), flush=True)
    moma.moma_ctx_destroy(ctx)
    replicas.finalize()


def headline(r):
    """The four parts of the metric in one short block, printed last in the line."""
    m = r["roofline"]["mulmod"]
    h = {"ntt_per_s": r["value"], "ntt_roofline_frac": r["roofline"]["frac"], "e2e_ntt_per_s": r["e2e"]["value"],
         "mulmod_gelem_s": m["gelem_s"], "mulmod_roofline_frac": m["frac"]}
    if r.get("batched_vs_plain"):
        h["batched_over_plain"] = r["batched_vs_plain"]["speedup"]
    s = r.get("served")
    if s:
        h.update({"served_over_plain": s["served_over_plain"], "served_p50_ms": s["p50_ms"],
                  "served_p99_ms_median": s["p99_ms_median"], "served_p99_ms_max": s["p99_ms_max"],
                  "served_p99_ms_runs": s["open_loop"]["p99_ms_runs"]})
    if r.get("c1_single_ntt"):
        h["c1_latency_us"] = min(r["c1_single_ntt"]["us_per_call"], r["c1_single_ntt"]["tuned_us_per_call"])
    if r.get("cpu_baseline"):
        h["cpu_oracle_ntt_per_s"] = r["cpu_baseline"]["value"]
    return h


# Each step's transforms are copied in, transformed and copied out in E2E_CHUNKS chunks that rotate
# over E2E_STREAMS streams (measured on GB300 with 16 transforms of 2^20 points: 1 chunk per stream
# 1.8k NTT/s, whole steps alternating on 2 streams 3.2k, 8 chunks on 4 streams 4.4k = the device rate).
E2E_CHUNKS = 8
E2E_STREAMS = 4


def measure_e2e(ctx, xs, n, steps, warmup, barrier, chunks=None, nstreams=None):
    """Forward NTTs of `xs` (count x L x n, host) through the C ABI with pinned host buffers: every
    step copies its inputs in, transforms them and copies the results out, all inside the timed
    region.  The step is cut in chunks that rotate over several streams, so the copy engines (in
    and out) and the SMs work on different chunks at the same time.  Returns (ms, results equal the
    device results)."""
    import numpy as np
    import torch

    from paper_2501_07535_gb300 import moma
    chunks = chunks or E2E_CHUNKS
    nstreams = nstreams or E2E_STREAMS
    count = xs.shape[0]
    per = count // chunks
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    hx = torch.from_numpy(xs.view(np.int32)).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    dxs = [torch.empty((per,) + tuple(xs.shape[1:]), dtype=torch.int32, device="cuda") for _ in range(nstreams)]
    dys = [torch.empty_like(d) for d in dxs]

    def step():
        for c in range(chunks):
            k = c % nstreams
            s_ = streams[k]
            with torch.cuda.stream(s_):
                dxs[k].copy_(hx[c * per:(c + 1) * per], non_blocking=True)
                moma.moma_ntt_fwd_many(ctx, n, per, dxs[k], dys[k], s_)
                hy[c * per:(c + 1) * per].copy_(dys[k], non_blocking=True)

    st = torch.cuda.current_stream()
    for _ in range(max(2, warmup)):
        step()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for s_ in streams:
        s_.wait_event(t0)
    for _ in range(steps):
        step()
    for s_ in streams:
        ev_ = torch.cuda.Event()
        ev_.record(s_)
        st.wait_event(ev_)
    t1.record(st)
    barrier()
    ref = torch.empty_like(hx, device="cuda")
    moma.moma_ntt_fwd_many(ctx, n, count, hx.cuda(), ref)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), bool(torch.equal(hy, ref.cpu()))


def run_profile(args):
    """Small cases for ncu captures (each op: one untimed call first, then `steps` calls):
    ntt: batched forward NTTs of 2^--profile-ntt-logn points (--ntt-batch transforms, --profile-bits
    wide);
    mul / add / sub / axpy: the vector op on 2^--profile-logn elements at --profile-bits;
    ntt768: 768-bit 2^16 NTTs (batch 8); mont_ntt / mont_mul: the 256-bit NTT and mulmod over a
    full-width modulus (its context's default schedule: Montgomery twiddles, word-based Barrett
    mulmod); mont_mul_redc: the same mulmod as two Montgomery products (engine 4); batch: the uneven batch at reduced sizes (2^10..2^16, 64 jobs); batch_large:
    128 jobs of the uneven mix at its full size range (2^10..2^20)."""
    import numpy as np
    import torch

    from paper_2501_07535_gb300 import batch, build, inputs, moma
    build.build()
    op = args.profile_op
    if op in ("batch", "batch_large"):
        nj, lr = (64, (10, 16)) if op == "batch" else (128, (10, 20))
        jobs = inputs.uneven_batch(n_jobs=nj, seed=0, log_n_range=lr)
        js = batch.JobSet(jobs)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for _ in range(1 + args.steps):
                js.run_batched(st)
        st.synchronize()
        status = js.status()
        js.close()
        js.ctx.close()
        print(json.dumps({"profile": op, "jobs": nj, "calls": 1 + args.steps, "status": status}))
        return
    full = op.startswith("mont_")
    redc = op == "mont_mul_redc"
    width = 768 if op == "ntt768" else args.profile_bits
    p = inputs.prime_full(width) if full else inputs.prime(width)
    q, Lw = p.q, p.L
    ctx = (moma.moma_ctx_create_full if full else moma.moma_ctx_create)(q, width)
    if op in ("mul", "add", "sub", "axpy", "mont_mul", "mont_mul_redc"):
        vn = 1 << args.profile_logn
        if redc:
            moma.moma_ctx_set_config(ctx, "mul", vn, engine=4)
        elif args.profile_tile:  # operands staged in shared memory by bulk copies
            cur = moma.moma_ctx_get_config(ctx, op, vn)
            moma.moma_ctx_set_config(ctx, op, vn, engine=cur["engine"], tile_log=args.profile_tile)
        a = moma.to_device(inputs.residues(q, Lw, vn, seed=1))
        b = moma.to_device(inputs.residues(q, Lw, vn, seed=2))
        c = torch.empty_like(a)
        alpha = inputs.scalar_residue(q, 3)
        for _ in range(1 + args.steps):
            if op == "add":
                moma.moma_vec_addmod(ctx, vn, a, b, c)
            elif op == "sub":
                moma.moma_vec_submod(ctx, vn, a, b, c)
            elif op == "axpy":
                moma.moma_vec_axpymod(ctx, vn, alpha, a, b, c)
            else:
                moma.moma_vec_mulmod(ctx, vn, a, b, c)
        torch.cuda.synchronize()
        cfg = moma.moma_ctx_get_config(ctx, "mul" if op.endswith("mul") or redc else op, vn)
        moma.moma_ctx_destroy(ctx)
        print(json.dumps({"profile": op, "bits": width, "n": vn, "calls": 1 + args.steps, "schedule": cfg}))
        return
    n = 1 << (16 if op == "ntt768" else args.profile_ntt_logn)
    xs = np.stack([inputs.residues(q, Lw, n, seed=10 + t) for t in range(args.ntt_batch)])
    dx = moma.to_device(xs)
    dy = torch.empty_like(dx)
    for _ in range(1 + args.steps):
        moma.moma_ntt_fwd_many(ctx, n, args.ntt_batch, dx, dy)
    torch.cuda.synchronize()
    cfg = moma.moma_ctx_get_config(ctx, "ntt_fwd", n)
    moma.moma_ctx_destroy(ctx)
    print(json.dumps({"profile": op, "bits": width, "n": n, "batch": args.ntt_batch, "calls": 1 + args.steps,
                      "passes_per_call": _pass_count(cfg, n.bit_length() - 1), "schedule": cfg}))
    return


def _pass_count(cfg, logn):
    if logn <= cfg["tile_log"]:
        return 1
    return math.ceil(logn / cfg["max_logr"])


def _timer(steps):
    """Mean milliseconds of fn() over `steps` calls after one untimed call (CUDA events)."""
    import torch

    def timed(fn, warm=1):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps
    return timed


C2_WIDTHS = (128, 256, 384, 768)
C2_OPS = ("add", "sub", "mul", "axpy")


def run_c2_table(hbm_gbs, prod_peak, steps=5, n=VEC_N):
    """The element-wise BLAS workload: addmod, submod, mulmod and axpy on 2^24 seeded residues at
    128/256/384/768 bits (each context's default schedule).  Per cell: time per call, Gelem/s,
    achieved HBM GB/s and word products/s, and the roofline fraction (the slower of 12L bytes per
    element at the HBM peak and, for mul and axpy, 2L^2 + L word products at the product peak).
    Inputs (1.5 to 4.8 GiB per call) are larger than L2.  `steps` timed calls per cell after one
    warm-up call."""
    import torch

    from paper_2501_07535_gb300 import inputs, moma
    timed = _timer(steps)
    rows = []
    for w in C2_WIDTHS:
        p = inputs.prime(w)
        ctx = moma.moma_ctx_create(p.q, w)
        a = moma.to_device(inputs.residues(p.q, p.L, n, 1))
        b = moma.to_device(inputs.residues(p.q, p.L, n, 2))
        c = torch.empty_like(a)
        alpha = inputs.scalar_residue(p.q, 3)
        calls = {"add": lambda: moma.moma_vec_addmod(ctx, n, a, b, c),
                 "sub": lambda: moma.moma_vec_submod(ctx, n, a, b, c),
                 "mul": lambda: moma.moma_vec_mulmod(ctx, n, a, b, c),
                 "axpy": lambda: moma.moma_vec_axpymod(ctx, n, alpha, a, b, c)}
        for op in C2_OPS:
            ms = timed(calls[op])
            r = vec_roofline(p.L, n, ms * 1e-3, hbm_gbs, prod_peak, products=op in ("mul", "axpy"))
            cfg = moma.moma_ctx_get_config(ctx, op, n)
            rows.append({"bits": w, "op": op, "us": r["achieved_us"], "gelem_s": round(n / ms / 1e6, 2),
                         "gbs": r["hbm_gbs_achieved"], "t_products_s": r["products_t_achieved"], "bound": r["bound"],
                         "roofline_us": r["time_us"], "frac": r["frac"],
                         "schedule": [cfg["engine"], cfg["vec_width"], cfg["tile_log"]]})
        assert moma.moma_ctx_sync_status(ctx) == 0
        moma.moma_ctx_destroy(ctx)
        del a, b, c
        torch.cuda.empty_cache()
    return {"n": n, "steps": steps, "schedule_fields": ["engine", "vec_width", "staged_tile_log"], "rows": rows}


C3_LOGN = tuple(range(14, 25))
C3_WIDTHS = (256, 384)
C3_BATCHES = (1, 2, 4, 8, 16)


def run_c3_sweep(prod_peak, steps=2):
    """The plain transform sweep: forward then inverse NTT, n = 2^14..2^24 at 256 and 384 bits,
    batch 1..16, every transform a separate call (moma_ntt_fwd / moma_ntt_inv, the default
    schedule).  One seeded transform per (n, width), copied into every batch slot on the device
    (identical work per slot).  Per cell: milliseconds per step (b forward + b inverse calls),
    transforms per second (forward and inverse each counted) and the fraction of the unit-count
    product peak ((n/2) log2 n mulmods of 2L^2 + L word products per transform).  `steps` timed
    steps per cell after one warm-up step; the round trip is checked once per (n, width)."""
    import torch

    from paper_2501_07535_gb300 import inputs, moma
    timed = _timer(steps)
    rows = []
    for w in C3_WIDTHS:
        p = inputs.prime(w)
        ctx = moma.moma_ctx_create(p.q, w)
        cap = max(C3_BATCHES) * p.L << max(C3_LOGN)
        fin = torch.empty(cap, dtype=torch.int32, device="cuda")
        fout = torch.empty_like(fin)
        for lg in C3_LOGN:
            n = 1 << lg
            bmax = max(C3_BATCHES)
            din = fin[:bmax * p.L * n].view(bmax, p.L, n)
            dout = fout[:bmax * p.L * n].view(bmax, p.L, n)
            din.copy_(moma.to_device(inputs.residues(p.q, p.L, n, seed=lg + w)).unsqueeze(0).expand(bmax, -1, -1))
            moma.moma_ntt_fwd(ctx, n, din[0], dout[0])
            moma.moma_ntt_inv(ctx, n, dout[0], dout[0])
            torch.cuda.synchronize()
            ok = bool(torch.equal(dout[0], din[0]))
            for bsz in C3_BATCHES:
                def step():
                    for t in range(bsz):
                        moma.moma_ntt_fwd(ctx, n, din[t], dout[t])
                    for t in range(bsz):
                        moma.moma_ntt_inv(ctx, n, dout[t], dout[t])
                ms = timed(step)
                roof = ntt_roofline(n, p.L, 2 * bsz, ms * 1e-3, prod_peak)
                rows.append([lg, w, bsz, round(ms, 4), round(2 * bsz / ms * 1e3, 1), roof["frac"], ok])
        assert moma.moma_ctx_sync_status(ctx) == 0
        moma.moma_ctx_destroy(ctx)
        del fin, fout, din, dout
        torch.cuda.empty_cache()
    return {"steps": steps, "fields": ["log2_n", "bits", "batch", "ms_per_step", "transforms_per_s", "frac",
                                       "round_trip_exact"], "rows": rows}


def run_c1_latency(calls=200):
    """The single small transform: one forward cyclic NTT of 2^12 points at 256 bits, issued as
    `calls` back-to-back calls on one stream; microseconds per call (launch and kernel) with the
    default schedule, the same calls captured once in a CUDA graph and replayed, and the calls with
    the schedule the autotuner picks for one transform of this size."""
    import torch

    from paper_2501_07535_gb300 import inputs, moma
    p = inputs.prime(256)
    n = 1 << 12
    ctx = moma.moma_ctx_create(p.q, 256)
    x = moma.to_device(inputs.residues(p.q, p.L, n, 0))
    y = torch.empty_like(x)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        f = lambda: moma.moma_ntt_fwd(ctx, n, x, y, st)  # noqa: E731
        ms = _timer(calls)(f, warm=5)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                for _ in range(20):
                    f()
            gms = _timer(max(1, calls // 20))(g.replay, warm=2)
        except RuntimeError:
            gms = None
        default_cfg = moma.moma_ctx_get_config(ctx, "ntt_fwd", n)
        tuned_cfg, _ = moma.moma_autotune(ctx, "ntt_fwd", n, 1, st)  # the autotuner's pick for one transform
        tms = _timer(calls)(f, warm=5)
    st.synchronize()
    assert moma.moma_ctx_sync_status(ctx) == 0
    moma.moma_ctx_destroy(ctx)
    keys = ("engine", "tile_log", "max_logr", "cta_threads", "tight_regs")
    return {"n": n, "bits": 256, "calls": calls, "us_per_call": round(ms * 1e3, 2),
            "graph_us_per_call": round(gms * 1e3 / 20, 2) if gms is not None else None,
            "schedule": [default_cfg[k] for k in keys], "tuned_us_per_call": round(tms * 1e3, 2),
            "tuned_schedule": [tuned_cfg[k] for k in keys]}


def run_uneven_batch(steps, warmup, n_jobs=256, seed=0):
    """The uneven batched workload: n_jobs transforms / cyclic products, n = 2^10..2^20 log-uniform,
    widths 128/256/384; one persistent launch (graph replay) against the same jobs as per-call launches."""
    import torch

    from paper_2501_07535_gb300 import batch, inputs

    jobs = inputs.uneven_batch(n_jobs=n_jobs, seed=seed, log_n_range=(10, 20))
    js = batch.JobSet(jobs)
    st = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    try:
        with torch.cuda.stream(st):
            for _ in range(warmup):
                js.run_plain(st)
            st.synchronize()
            e0, e1 = ev(), ev()
            e0.record(st)
            for _ in range(steps):
                js.run_plain(st)
            e1.record(st)
            st.synchronize()
            plain_ms = e0.elapsed_time(e1) / steps
            plain_out = [o.clone() for o in js.out]
            for o in js.out:
                o.zero_()
            for _ in range(warmup):
                js.run_batched(st)
            st.synchronize()
            b0, b1 = ev(), ev()
            b0.record(st)
            for _ in range(steps):
                js.run_batched(st)
            b1.record(st)
            st.synchronize()
            batched_ms = b0.elapsed_time(b1) / steps
        status = js.status()
        same = all(torch.equal(a, b) for a, b in zip(plain_out, js.out))
        units = js.work_units()
        return {"jobs": n_jobs, "transforms": units["transforms"], "batched_ms": round(batched_ms, 3),
                "plain_ms": round(plain_ms, 3), "speedup": round(plain_ms / batched_ms, 3),
                "batched_transforms_per_s": round(units["transforms"] / batched_ms * 1e3, 1),
                "identical_results": bool(same), "device_status": status,
                "plain_launches_per_step": None}
    finally:
        js.close()
        js.ctx.close()


def run_sensitivity(steps=5):
    """Sec. 5.4 analogues on seeded residues: (1) forward NTT runtime against width at n = 4096 from
    64 to 1024 bits (batches of 256, ns per butterfly = 2t/(n log2 n) as in Sec. 5.3), with the slowdown per
    doubling of the width as the paper reports it; (2) mulmod with schoolbook carry chains,
    whole mad.wide products and Karatsuba (Eq. mulk) at each width, 2^22 elements; (3) the same
    mulmod and transform over a full-width modulus: mulmod by the word-based Barrett reduction and
    by two Montgomery products (Sec. 5.2), the transform with Montgomery twiddle products."""
    import torch

    from paper_2501_07535_gb300 import inputs, moma
    out = {"ntt_n4096": [], "mulmod_engines": [], "full_width_montgomery": []}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    prev = None
    for w in (64, 128, 256, 384, 512, 768, 1024):
        p = inputs.prime(w)
        ctx = moma.moma_ctx_create(p.q, w)
        n, cnt = 4096, 256
        x = moma.to_device(inputs.residues(p.q, p.L, n * cnt, 40 + w).reshape(p.L, cnt, n).transpose(1, 0, 2).copy())
        y = torch.empty_like(x)
        ms = timed(lambda: moma.moma_ntt_fwd_many(ctx, n, cnt, x, y))
        ns_bfly = ms * 1e6 / cnt * 2 / (n * 12)
        row = {"bits": w, "ms_per_256": round(ms, 4), "ns_per_butterfly": round(ns_bfly, 4),
               "slowdown_vs_previous_width": round(ns_bfly / prev, 2) if prev else None}
        prev = ns_bfly
        out["ntt_n4096"].append(row)
        vn = 1 << 22
        a = moma.to_device(inputs.residues(p.q, p.L, vn, 1))
        b = moma.to_device(inputs.residues(p.q, p.L, vn, 2))
        c = torch.empty_like(a)
        eng = {}
        for e, name in ((1, "schoolbook_carry"), (2, "schoolbook_wide"), (3, "karatsuba")):
            moma.moma_ctx_set_config(ctx, "mul", vn, engine=e, vec_width=1)
            eng[name] = round(vn / timed(lambda: moma.moma_vec_mulmod(ctx, vn, a, b, c)) / 1e6, 2)
        out["mulmod_engines"].append({"bits": w, "gelem_s": eng,
                                      "karatsuba_over_schoolbook": round(eng["karatsuba"] / eng["schoolbook_carry"], 3)})
        # full-width modulus (W bits) against the (W-4)-bit Barrett context: mulmod by the default
        # word-based Barrett reduction with an (L+1)-word constant and by two Montgomery products
        # (engine 4); transforms with Montgomery twiddle products
        pf = inputs.prime_full(w)
        fctx = moma.moma_ctx_create_full(pf.q, w)
        fa = moma.to_device(inputs.residues(pf.q, pf.L, vn, 1))
        fb = moma.to_device(inputs.residues(pf.q, pf.L, vn, 2))
        full_gelem = vn / timed(lambda: moma.moma_vec_mulmod(fctx, vn, fa, fb, c)) / 1e6
        moma.moma_ctx_set_config(fctx, "mul", vn, engine=4)
        mont_gelem = vn / timed(lambda: moma.moma_vec_mulmod(fctx, vn, fa, fb, c)) / 1e6
        fx = moma.to_device(inputs.residues(pf.q, pf.L, n * cnt, 50 + w).reshape(pf.L, cnt, n).transpose(1, 0, 2).copy())
        fms = timed(lambda: moma.moma_ntt_fwd_many(fctx, n, cnt, fx, y))
        out["full_width_montgomery"].append({
            "bits": w, "mulmod_gelem_s": round(full_gelem, 2),
            "mulmod_over_barrett": round(full_gelem / max(eng.values()), 3),
            "mulmod_two_montgomery_gelem_s": round(mont_gelem, 2),
            "word_barrett_over_montgomery": round(full_gelem / mont_gelem, 3),
            "ntt_n4096_ns_per_butterfly": round(fms * 1e6 / cnt * 2 / (n * 12), 4),
            "ntt_over_barrett_time": round(fms / ms, 3)})
        moma.moma_ctx_destroy(fctx)
        moma.moma_ctx_destroy(ctx)
    # the paper's sweep doubles the width (Sec. 5.4): 64 -> 128 -> 256 -> 512 -> 1024 bits
    by = {r["bits"]: r["ns_per_butterfly"] for r in out["ntt_n4096"]}
    out["ntt_n4096_slowdown_per_doubling"] = {f"{w}->{2 * w}": round(by[2 * w] / by[w], 2)
                                              for w in (64, 128, 256, 512)}
    return out


def median_run(runs):
    """The run whose p99 is the median of the runs' p99 (the lower middle one for an even count)."""
    return sorted(runs, key=lambda r: r["p99_ms"])[(len(runs) - 1) // 2]


def run_served(n_jobs=10000, seed=0, load=0.8, slots=4, repeats=3):
    """The served stream: Poisson arrivals of n_jobs transforms (2^12..2^22) and mulmod/axpy
    vectors (2^16..2^24) at 256/384/768 bits, continuous batching under a 40 GB budget, with
    size-class micro-batches (serve.Scheduler policy "class").  Capacity is measured closed-loop
    (all requests present at t = 0); the open-loop runs offer load x capacity, `repeats` times under
    each policy (size classes, plain FIFO micro-batches), alternating; the median-p99 run of each is
    reported with every run's p99 beside it; one more run each at 0.5 and 1.0 x capacity gives the
    latency against the offered load.  The same jobs as plain per-call launches give the per-call
    throughput."""
    import torch

    from paper_2501_07535_gb300 import batch, serve
    unit_arrivals, jobs = serve.served_jobs(n_jobs=n_jobs, seed=seed, rate_per_s=1.0)
    ctxs = batch.Contexts()
    ex = serve.GpuExecutor(ctxs, slots=slots)
    try:
        ex.prewarm(jobs)
        closed = serve.serve([0.0] * n_jobs, jobs, ctxs, slots=slots, executor=ex, policy="class").summary()
        capacity = closed["jobs_per_s"]
        rate = load * capacity
        arrivals = [a / rate for a in unit_arrivals]
        # open loop: the two policies alternate `repeats` times on the same arrivals; the run with the
        # median p99 of each policy is reported, every run's p99 beside it
        runs = {"class": [], "fifo": []}
        for _ in range(repeats):
            for pol in ("class", "fifo"):
                runs[pol].append(serve.serve(arrivals, jobs, ctxs, slots=slots, executor=ex, policy=pol).summary())
        torch.cuda.synchronize()
        opened, fifo = (median_run(runs[pol]) for pol in ("class", "fifo"))
        opened["p99_ms_runs"] = [r["p99_ms"] for r in runs["class"]]
        fifo["p99_ms_runs"] = [r["p99_ms"] for r in runs["fifo"]]
        # the same arrivals at half and at full capacity (size classes, one run each)
        sweep = []
        for lo in (0.5, 1.0):
            r = serve.serve([a / (lo * capacity) for a in unit_arrivals], jobs, ctxs, slots=slots, executor=ex,
                            policy="class").summary()
            sweep.append({"offered_load": lo, "offered_jobs_per_s": round(lo * capacity, 1),
                          "jobs_per_s": r["jobs_per_s"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                          "mean_ms": r["mean_ms"]})
        torch.cuda.synchronize()
        plain_s = serve.run_plain(jobs, ex)
        return {"jobs": n_jobs, "policy": "class", "capacity_jobs_per_s": capacity,
                "plain_per_call_jobs_per_s": round(n_jobs / plain_s, 1),
                "served_over_plain": round(capacity / (n_jobs / plain_s), 3), "offered_load": load,
                "offered_jobs_per_s": round(rate, 1), "closed_loop": closed, "open_loop": opened,
                "open_loop_fifo": fifo, "load_sweep": sweep, "p50_ms": opened["p50_ms"], "p99_ms": opened["p99_ms"],
                "p99_ms_median": opened["p99_ms"], "p99_ms_min": min(opened["p99_ms_runs"]),
                "p99_ms_max": max(opened["p99_ms_runs"]), "budget_gb": 40, "slots": slots,
                "resident_gb": round(ex.resident_bytes() / 1e9, 3)}
    finally:
        ctxs.close()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    from paper_2501_07535_gb300 import inputs
    q = inputs.prime(WIDTH).q
    cores = _cores()
    pool = mp.get_context("spawn").Pool(cores)
    for _ in range(args.warmup):
        pool.map(_oracle_ntt_worker, [(q, LOGN - 4, 1 + i) for i in range(cores)])
    t = time.perf_counter()
    for k in range(args.steps):
        pool.map(_oracle_ntt_worker, [(q, LOGN, 1000 + 100 * k + i) for i in range(cores)])
    wall = time.perf_counter() - t
    pool.close()
    rate = cores * args.steps / wall
    out = {"metric": METRIC, "value": round(rate, 4), "unit": "NTT/s", "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "python-int",
           "data": "synthetic: seeded uniform residues mod a seed-generated 252-bit prime",
           "config": bench_config(world),
           "cpu_baseline": {"value": round(rate, 4), "unit": "NTT/s", "cores": cores, "kind": "oracle",
                            "sample": f"{cores} full 2^{LOGN}-point forward NTTs per step, one per host core "
                                      f"(warm-up steps at 2^{LOGN - 4})"},
           "e2e": {"value": round(rate, 4), "unit": "NTT/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="small NTT-only case for ncu captures")
    ap.add_argument("--ntt-batch", type=int, default=8)
    ap.add_argument("--profile-op", default="ntt",
                    choices=["ntt", "mul", "add", "sub", "axpy", "ntt768", "mont_ntt", "mont_mul", "mont_mul_redc",
                             "batch", "batch_large"])
    ap.add_argument("--profile-bits", type=int, default=WIDTH, help="container width of the profiled op")
    ap.add_argument("--profile-logn", type=int, default=24, help="log2 elements of the profiled vector op")
    ap.add_argument("--profile-ntt-logn", type=int, default=LOGN, help="log2 points of the profiled transforms (ntt)")
    ap.add_argument("--profile-tile", type=int, default=0, help="staged tile (log2) of the profiled vector op (0: direct)")
    ap.add_argument("--serve-jobs", type=int, default=10000, help="requests in the served stream (0: skip)")
    ap.add_argument("--quick", action="store_true", help="skip the BLAS table and the transform sweep")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
