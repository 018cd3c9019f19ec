"""The benchmark's per-kernel roofline bookkeeping on the host: the work
units each kernel is credited with, the bound it is judged against, the
fraction computed from them, and the traffic figure that is withdrawn once
the kernel's source changes.  The statistics are made up, so no GPU is
needed."""
import pytest

import bench

CLK = 2000.0  # MHz
HBM = 6000.0  # GB/s


def fake_stats(D):
    base = {"base_interactions": 4.0e12, "base_expanded": 3.0e12, "ms_base": 1500.0, "ms_base_tc": 1200.0,
            "farfield_terms": 1.0e9, "ms_farfield": 2.0, "local_terms": 2.0e9, "ms_local": 3.0,
            "f2l_terms": 5.0e8, "ms_f2l": 0.5, "pairs_visited": 1.0e9, "ms_classify": 100.0, "ms_post": 4.0}
    other = dict(base, ms_base=1700.0, ms_base_tc=1300.0)  # a second step: means are taken
    if D <= 5:
        for s in (base, other):
            s["base_expanded"] = 0.0
            s["ms_base_tc"] = 0.0
    return [base, other]


def fake_tinfo():
    return [{"n_nodes": 1000, "depth": 20, "n_coeff": 16, "ms_levels": 5.0, "ms_moments": 1.0}] * 2


def test_low_dimension_exact_sums_against_the_ex2_peak():
    out = bench.roofline_by_kernel(fake_stats(3), fake_tinfo(), 10 ** 6, 3, 4, CLK, HBM)
    assert "k_base_tc" not in out and "k_base_hd" not in out
    k = out["k_base"]
    ex2_peak = 152 * 32 * CLK * 1e6
    assert k["peak"] == pytest.approx(ex2_peak)
    assert k["ms_per_step"] == pytest.approx(1600.0)  # mean of the two steps
    assert k["achieved"] == pytest.approx(4.0e12 / 1.6)
    assert k["frac"] == pytest.approx(4.0e12 / 1.6 / ex2_peak)
    assert k["bound"] == "alu"


def test_high_dimension_splits_the_two_forms():
    D = 16
    out = bench.roofline_by_kernel(fake_stats(D), fake_tinfo(), 10 ** 6, D, 8, CLK, HBM)
    tc, hd = out["k_base_tc"], out["k_base_hd"]
    # tensor form: its own interactions and time, one ex2 each
    assert tc["units_per_step"] == pytest.approx(3.0e12)
    assert tc["ms_per_step"] == pytest.approx(1250.0)
    assert tc["peak"] == pytest.approx(152 * 32 * CLK * 1e6)
    # direct form: the rest of the interactions and of the exact-sum time,
    # 2D + 2 FMA-pipe operations each, against the FMA peak
    assert hd["units_per_step"] == pytest.approx(1.0e12 * (2 * D + 2))
    assert hd["ms_per_step"] == pytest.approx(1600.0 - 1250.0)
    fma_peak = 152 * 128 * CLK * 1e6
    assert hd["peak"] == pytest.approx(fma_peak)
    assert hd["frac"] == pytest.approx(1.0e12 * (2 * D + 2) / 0.35 / fma_peak)
    assert "k_base" not in out


def test_memory_bound_kernels_use_the_copy_bandwidth():
    D = 3
    out = bench.roofline_by_kernel(fake_stats(D), fake_tinfo(), 10 ** 6, D, 4, CLK, HBM)
    tr = out["k_traverse"]
    assert tr["units_per_step"] == pytest.approx(1.0e9 * (16 * D + 16))
    assert tr["peak"] == pytest.approx(HBM * 1e9)
    assert tr["frac"] == pytest.approx(1.0e9 * (16 * D + 16) / 0.1 / (HBM * 1e9))
    post = out["k_post"]
    assert post["units_per_step"] == pytest.approx(4 * 10 ** 6 * 16 + 4 * 1000 * 16 * 8)
    # D = 3 rows are padded to 4 floats
    assert out["k_build_levels"]["units_per_step"] == pytest.approx(20 * 10 ** 6 * (2 * 4 * 4 + 8))
    assert out["k_moments"]["units_per_step"] == pytest.approx(10 ** 6 * 4 * 4 + 1000 * 16 * 12)


def test_kernels_without_time_or_work_are_left_out():
    stats = fake_stats(3)
    for s in stats:
        s["ms_f2l"] = 0.0
        s["local_terms"] = 0.0
    out = bench.roofline_by_kernel(stats, fake_tinfo(), 10 ** 6, 3, 4, CLK, HBM)
    assert "k_f2l" not in out and "k_local" not in out
    assert "k_farfield" in out


def test_traffic_is_withdrawn_when_the_source_changes(monkeypatch):
    sha = bench.source_sha("base_tc.cu")
    assert sha and len(sha) == 16
    monkeypatch.setattr(bench, "K_BASE_TRAFFIC", {"w_same": ("base_tc.cu", sha, 123),
                                                  "w_changed": ("base_tc.cu", "0" * 16, 456),
                                                  "w_unset": ("actions.cu", "", 789)})
    assert bench.base_traffic("w_same") == 123
    assert bench.base_traffic("w_changed") is None
    assert bench.base_traffic("w_unset") is None
    assert bench.base_traffic("not_listed") is None
