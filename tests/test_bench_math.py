"""The roofline arithmetic of bench.py on CPU: the unit-count peak, the transform's algorithmic
product rate and the element-wise roofline (the slower of bytes at the HBM peak and word products at
the product peak), on hand-computed cases."""
import math

import pytest

import bench


def test_word_products_and_peak():
    assert [bench.word_products_per_mulmod(L) for L in (4, 8, 12, 24)] == [36, 136, 300, 1176]
    # 152 SMs x 32 products per clock x 2070 MHz
    assert bench.product_peak(152, 2070.0) == pytest.approx(152 * 32 * 2.07e9)


def test_ntt_roofline_counts_every_butterfly():
    peak = bench.product_peak(152, 2070.0)
    n, L, batch = 1 << 20, 8, 16
    prod = (n // 2) * 20 * 136 * batch  # (n/2) log2 n mulmods x (2L^2 + L) products x batch
    step_s = prod / (0.5 * peak)  # a step at half the peak
    r = bench.ntt_roofline(n, L, batch, step_s, peak)
    assert r["bound"] == "alu" and r["unit"] == "T word-products/s"
    assert r["frac"] == pytest.approx(0.5, abs=1e-4)
    assert r["achieved"] == pytest.approx(prod / step_s / 1e12, abs=1e-3)
    # twice the transform length: (2n/2) log2(2n) products, i.e. 2 x 21/20 the work
    r2 = bench.ntt_roofline(2 * n, L, batch, step_s, peak)
    assert r2["achieved"] / r["achieved"] == pytest.approx(2 * 21 / 20, rel=1e-3)


@pytest.mark.parametrize("L,bound", [(4, "hbm"), (8, "hbm"), (12, "alu"), (24, "alu")])
def test_vec_roofline_bound_switches_with_width(L, bound):
    """At 6657.6 GB/s and 10.07 T products/s: 2^24 mulmods are byte-bound up to 256 bits and
    product-bound from 384 bits (12L bytes against 2L^2 + L products per element)."""
    peak = bench.product_peak(152, 2070.0)
    n = 1 << 24
    t_hbm = 12 * L * n / 6657.6e9
    t_prod = (2 * L * L + L) * n / peak
    r = bench.vec_roofline(L, n, 2 * max(t_hbm, t_prod), 6657.6, peak)
    assert r["bound"] == bound
    assert r["frac"] == pytest.approx(0.5, abs=1e-4)
    assert r["time_us"] == pytest.approx(max(t_hbm, t_prod) * 1e6, abs=0.01)


def test_vec_roofline_additions_are_byte_bound():
    peak = bench.product_peak(152, 2070.0)
    r = bench.vec_roofline(8, 1 << 24, 1e-3, 6657.6, peak, products=False)
    assert r["bound"] == "hbm" and r["products_t_achieved"] == 0
    assert r["hbm_gbs_achieved"] == pytest.approx(12 * 8 * (1 << 24) / 1e-3 / 1e9, abs=0.1)
    assert math.isclose(r["frac"], 12 * 8 * (1 << 24) / 6657.6e9 / 1e-3, rel_tol=1e-3)


def test_headline_holds_every_part_of_the_metric():
    """The headline block names the transform rate and its fraction, the mulmod rate and its
    fraction, batched/plain, served/plain with p50 and the median and worst p99, and the C1
    latency (the faster of the default and the tuned schedule)."""
    r = {"value": 4276.0, "roofline": {"frac": 0.606, "mulmod": {"gelem_s": 39.0, "frac": 0.552}},
         "e2e": {"value": 4429.0}, "batched_vs_plain": {"speedup": 1.37},
         "served": {"served_over_plain": 1.05, "p50_ms": 4.7, "p99_ms_median": 37.6, "p99_ms_max": 40.4,
                    "open_loop": {"p99_ms_runs": [40.4, 37.6, 37.5]}},
         "c1_single_ntt": {"us_per_call": 23.3, "tuned_us_per_call": 23.4}, "cpu_baseline": {"value": 1.53}}
    h = bench.headline(r)
    assert h["ntt_per_s"] == 4276.0 and h["ntt_roofline_frac"] == 0.606
    assert h["mulmod_gelem_s"] == 39.0 and h["mulmod_roofline_frac"] == 0.552
    assert h["batched_over_plain"] == 1.37 and h["served_over_plain"] == 1.05
    assert (h["served_p50_ms"], h["served_p99_ms_median"], h["served_p99_ms_max"]) == (4.7, 37.6, 40.4)
    assert h["served_p99_ms_runs"] == [40.4, 37.6, 37.5]
    assert h["c1_latency_us"] == 23.3 and h["e2e_ntt_per_s"] == 4429.0
    # without the optional sections the block still carries the two kernel rates
    h2 = bench.headline({k: r[k] for k in ("value", "roofline", "e2e")})
    assert set(h2) == {"ntt_per_s", "ntt_roofline_frac", "e2e_ntt_per_s", "mulmod_gelem_s", "mulmod_roofline_frac"}
