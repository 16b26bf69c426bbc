"""The roofline arithmetic bench.py reports, checked on the host: the algorithmic counts of each
stage against their closed forms, the fractions against the definitions (achieved / peak), the
whole-evaluation bound, the traffic figure's source-digest guard and the launch count."""
import hashlib
import importlib.util
import os
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _problem(n, m, mv, d=8):
    return types.SimpleNamespace(X=np.zeros((n, d)), Z=np.zeros((m, d)), mv=mv)


def test_stage_counts_follow_the_closed_forms(bench):
    n, m, q = 500_000, 500, 20
    P = _problem(n, m, q)
    fpad = 512                                  # m + 1 = 501 rounded up to 64
    f, b = bench.stage_algorithmic(P, "lowrank_A")
    assert f == pytest.approx(n * m * (m + 1)) and b == 4 * n * m
    f, b = bench.stage_algorithmic(P, "vecchia_factor")
    # residual Gram of the (q+1) rows over m columns (lower triangle incl. diagonal), the F row
    # (q m), the q x q Cholesky (q^3 / 6), 2 flops each
    assert f == pytest.approx(2 * n * ((q + 1) * (q + 2) / 2 * m + q * m + q ** 3 / 6))
    assert b == 4 * n * m + 4 * n * fpad
    f, b = bench.stage_algorithmic(P, "gram_FtF")
    assert f == pytest.approx(n * (m + 1) * (m + 2)) and b == 4 * n * fpad
    # the whole evaluation: ~3.8e11 flops and ~4.0 GB
    tot_f = sum(bench.stage_algorithmic(P, s)[0] for s in ("lowrank_A", "vecchia_factor", "gram_FtF"))
    tot_b = sum(bench.stage_algorithmic(P, s)[1] for s in ("lowrank_A", "vecchia_factor", "gram_FtF"))
    assert 3.7e11 < tot_f < 3.9e11 and 4.0e9 <= tot_b < 4.1e9


def test_fractions_are_achieved_over_peak(bench):
    P = _problem(500_000, 500, 20)
    med = {"lowrank_A": 1.35, "vecchia_factor": 7.04, "gram_FtF": 2.05}
    pk = {"bf16_tflops": 1903.1, "hbm_gbs": 6795.5}
    r = bench.roofline_block(P, med, 12.07, pk)
    assert r["kernel"] == "vecchia_factor"     # the longest stage
    for st, dtype, peak in (("lowrank_A", "f16", 1903.1), ("vecchia_factor", "tf32", 1903.1 / 2),
                            ("gram_FtF", "tf32", 1903.1 / 2)):
        s = r["per_stage"][st]
        f, b = bench.stage_algorithmic(P, st)
        t = med[st] * 1e-3
        assert s["tensor_dtype"] == dtype and s["peak_tflops"] == pytest.approx(peak)
        assert s["tflops"] == pytest.approx(f / t / 1e12)
        assert s["frac_tensor"] == pytest.approx(f / t / 1e12 / peak)
        assert s["frac_hbm"] == pytest.approx(b / t / 1e9 / 6795.5)
        assert s["frac"] == max(s["frac_tensor"], s["frac_hbm"])
    assert r["frac"] == r["per_stage"]["vecchia_factor"]["frac_tensor"]
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    w = r["whole_eval"]
    t_tensor = sum(bench.stage_algorithmic(P, st)[0] / (r["per_stage"][st]["peak_tflops"] * 1e12)
                   for st in med)
    assert w["roofline_ms"] == pytest.approx(max(t_tensor, w["algorithmic_bytes"] / 6795.5e9) * 1e3)
    assert w["frac_whole_eval"] == pytest.approx(w["roofline_ms"] / 12.07)
    # the tensor-core factor path is held to the float16 peak
    r2 = bench.roofline_block(P, med, 12.07, pk, factor_path=2)
    assert r2["per_stage"]["vecchia_factor"]["peak_tflops"] == pytest.approx(1903.1)
    assert r2["traffic"] is None


def test_traffic_is_reported_only_for_the_captured_source(bench, monkeypatch):
    with open(os.path.join(ROOT, "paper_2507_05064_gb300", "csrc", "vif_factor.cu"), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    monkeypatch.setattr(bench, "FACTOR_TRAFFIC", {"bytes_per_point": 1000.0, "source_sha256": digest})
    assert bench.factor_traffic(123) == pytest.approx(123000.0)
    monkeypatch.setattr(bench, "FACTOR_TRAFFIC", {"bytes_per_point": 1000.0, "source_sha256": "0" * 64})
    assert bench.factor_traffic(123) is None


def test_committed_traffic_figure_matches_the_committed_source(bench):
    """The stored per-point DRAM figure belongs to the factor kernel source as committed."""
    assert bench.factor_traffic(100_000) == pytest.approx(bench.FACTOR_TRAFFIC["bytes_per_point"] * 1e5)


def test_launches_per_evaluation(bench):
    # m = 500: 16-wide Cholesky of Sigma_m (32 panels, 31 updates) and of the (m+1) capacitance
    # matrix (32, 31), 16 block diagonals of the 32-wide triangular inverse (1 + 2 x 15), 10 others
    assert bench.launches_per_eval(500) == 169
    assert bench.launches_per_eval(16) == 2 + 1 + 1 + 1 + 2 + 1 + 1 + 2 + 2 + 3 + 1
