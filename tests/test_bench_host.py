"""Host-side arithmetic of bench.py, without a GPU: the roofline work models,
the ALU peak, the downsampling expectation, the traffic record keyed to the
kernel's sources, the clock sampler's parsing, the whole-job rate and the
oracle's proportional shares (on a small graph)."""
import json
import os

import numpy as np
import pytest

import bench
from paper_2302_07084_gb300 import synth


def test_walk_ops_per_sample_closed_forms():
    # T = 1: one Philox block (words r, sigma, coin, w3), no step, 12 bookkeeping ops
    assert bench.walk_ops_per_sample({"s": [1.0]}) == 40.0 + 12.0
    # r = 3 only: ceil(5 / 4) = 2 blocks, 2 steps
    assert bench.walk_ops_per_sample({"s": [0.0, 0.0, 1.0]}) == 80.0 + 10.0 + 12.0
    # uniform over r = 1..4: r + 2 words, so blocks 1, 1, 2, 2; steps 0..3
    want = np.mean([40 + 0 + 12, 40 + 5 + 12, 80 + 10 + 12, 80 + 15 + 12])
    assert bench.walk_ops_per_sample({"s": [1, 1, 1, 1]}) == pytest.approx(want)


def test_kernel_models_are_the_algorithmic_byte_counts():
    g = synth.sbm(300, 3, 0.05, 0.01, seed=1)
    params = dict(d=32, oversample=16, precision=0)
    counts = dict(total_samples=1000.0, nnz_M=5000)
    bound, work, unit, _ = bench.kernel_model("walk_count", g, params, counts)
    assert (bound, work, unit) == ("hbm", 8.0 * 1000, "GB/s")
    _, work, _, _ = bench.kernel_model("spmm", g, params, counts)
    assert work == 8.0 * 5000 + g.n * 48 * (4 + 4)
    params["precision"] = 1
    _, work, _, _ = bench.kernel_model("spmm", g, params, counts)
    assert work == 8.0 * 5000 + g.n * 48 * (2 + 4)
    _, work, _, _ = bench.kernel_model("graph_spmm", g, params, counts)
    assert work == 8.0 * g.n_arcs + g.n * 32 * 8.0
    assert bench.kernel_model("jacobi_reg", g, params, counts) is None


def test_alu_peak_is_lanes_times_clock():
    assert bench.alu_peak_gops(152, 2070.0) == pytest.approx(152 * 128 * 2.07)


def test_expected_kept_draws():
    g = synth.sbm(200, 2, 0.1, 0.02, seed=2)
    p = {"samples": 1e5}
    assert bench.expected_kept_draws(g, p) == 1e5
    p["downsample_C"] = 1e9                    # every p_e = 1
    assert bench.expected_kept_draws(g, p) == pytest.approx(1e5)
    p["downsample_C"] = 0.5
    deg = g.degrees().astype(np.float64)
    src = np.repeat(np.arange(g.n), deg.astype(np.int64))
    pe = np.minimum(1.0, 0.5 * (1 / deg[src] + 1 / deg[g.indices]))
    assert bench.expected_kept_draws(g, p) == pytest.approx(1e5 * pe.mean())


def test_recorded_traffic_is_dropped_when_the_sources_change(monkeypatch):
    rec = dict(bench.RECORDED_TRAFFIC["walk_count"])
    rec["sha16"] = bench.source_sha16(rec["sources"])
    monkeypatch.setitem(bench.RECORDED_TRAFFIC, "walk_count", rec)
    assert bench.recorded_traffic("walk_count") == rec["bytes"]
    monkeypatch.setitem(bench.RECORDED_TRAFFIC, "walk_count", dict(rec, sha16="0" * 16))
    assert bench.recorded_traffic("walk_count") is None
    assert bench.recorded_traffic("no_such_kernel") is None


def test_clock_sampler_parses_nvidia_smi_rows(tmp_path):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 1100.5, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1800, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage"]
    f = open(tmp_path / "clocks.csv", "w+")
    f.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc, cs.file = Done(), f
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_whole_job_rate():
    assert bench.whole_job_rate(1, 6.68e8, 20.0) == pytest.approx(3.34e10)
    assert bench.whole_job_rate(4, 1e6, 500.0) == pytest.approx(8e6)


def test_bench_config_names_the_workload():
    g = synth.sbm(100, 2, 0.1, 0.02, seed=3)
    params = dict(samples=1e6, T=10, d=128, q=1, k=10)
    cfg = bench.bench_config(g, params, 2)
    assert cfg["workload"] == bench.WORKLOAD and cfg["parallelism"] == "replicas2"
    assert {"n", "m", "samples", "T", "d", "q", "k", "l2"} <= set(cfg)
    json.dumps(cfg)


def test_oracle_shares_cover_the_workload():
    """F proportional shares of a small workload: every arc range, pair range
    and row block is visited once, and each share runs (positive time)."""
    g = synth.sbm(400, 2, 0.05, 0.01, seed=5)
    params = dict(T=4, s=[0.25] * 4, samples=20.0 * g.n_arcs, b=1.0, d=8, oversample=8, q=1, k=3,
                  theta=0.5, mu=0.2, seed=1)
    ob = bench.OracleBaseline(g, params, F=4)
    assert ob.setup["nnz_M"] == int(ob.M[0][-1]) and ob.setup["nnz_pairs"] == ob.pairs[0].size
    F = ob.F
    arcs = [(k * g.n_arcs // F, (k + 1) * g.n_arcs // F) for k in range(F)]
    assert arcs[0][0] == 0 and arcs[-1][1] == g.n_arcs and all(a[1] == b[0] for a, b in zip(arcs, arcs[1:]))
    for k in range(F):
        assert ob.share(k) > 0.0
    assert f"{F} proportional shares" in ob.describe()
