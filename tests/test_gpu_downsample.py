"""Edge downsampling (Sec. 4.1, Algorithm 3) on the GPU against the oracle.

A draw of arc u -> v walks only if its coin word is below thr_e =
min(2^32, floor(p_e 2^32)), p_e = min(1, C (1/d_u + 1/d_v)), and then counts
with weight 1/p_e, held as floor(2^32 / p_e + 1/2) in 2^-32 units:

* raw draws: dropped draws read (-1, -1), kept draws equal the oracle's;
* weight sums per pair bit-exact (uint64) for the dense-table and the sort
  aggregation, including n = 2^B where the sort's drop marker needs one more
  key bit; the bucket aggregation refuses downsampling;
* the trunc_log CSR: structure and keep decisions exact, values within 1e-6;
* C so large that p_e = 1 everywhere reproduces the plain sparsifier;
* keep decisions exact for entries placed on v = 1 to the last bits (also
  without downsampling);
* the whole method (lne_embed) follows the oracle's downsampled embedding.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import assert_subspace, make_params, to_np

pytestmark = pytest.mark.gpu

VAL_RTOL = 1e-6
VAL_ATOL = 1e-7


def _ctx(agg):
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    c.set_option(lne.OPT_AGGREGATION, agg)
    return c


@pytest.fixture(scope="module", params=["table", "sort"])
def ctx(request):
    c = _ctx({"table": lne.AGG_TABLE, "sort": lne.AGG_SORT}[request.param])
    yield c
    c.close()


GRAPHS = {
    "sbm600": synth.sbm(600, 3, 0.05, 0.005, seed=3),
    "chunglu2k": synth.chung_lu(2000, 12000, 2.1, seed=4, n_labels=5),
    "lollipop": synth.lollipop_tiny(),
    "ring1024": synth.ring(1024),   # n = 2^B: the pair (1023, 1023) exists
}


def _params(g, T=10, rate=20.0, C=1.0, seed=9):
    p = make_params(T, synth.dirichlet_weights(T, 5), rate * g.n_arcs, seed=seed)
    p.downsample_C = C
    return p


def _check_counts(ctx, g, p):
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    x, y, w = oracle.sparsifier_counts(g.indptr, g.indices, p.T, p.s, p.samples, p.seed, C=p.downsample_C)
    assert "count" not in res
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["y"]).astype(np.int64), y)
    assert np.array_equal(to_np(res["weight"]).view(np.uint64), w)
    return res


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("C", [0.05, 0.5, 3.0])
def test_sample_pairs_drop_markers(ctx, name, C):
    g = GRAPHS[name]
    p = _params(g, T=5, rate=2.5, C=C, seed=77)
    dg = lne.DeviceGraph.from_graph(g)
    thr, _ = oracle.arc_downsample(g.indptr, g.indices, C)
    for a0, a1 in [(0, g.n_arcs), (g.n_arcs // 3, g.n_arcs - 1)]:
        u1, v1 = ctx.sample_pairs(dg, p, a0, a1)
        tr = oracle.sample_trace(g.indptr, g.indices, p.T, p.s, p.samples, p.seed, a0, a1,
                                 fields=("arc", "u1", "v1", "coin"))
        drop = tr["coin"].astype(np.uint64) >= thr[tr["arc"]]
        assert np.array_equal(to_np(u1).astype(np.int64), np.where(drop, -1, tr["u1"]))
        assert np.array_equal(to_np(v1).astype(np.int64), np.where(drop, -1, tr["v1"]))
        if C < 0.1:
            assert drop.mean() > 0.5      # most draws of a sparse graph are dropped


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("C", [0.05, 0.5, 3.0])
def test_weights_bit_exact(ctx, name, C):
    _check_counts(ctx, GRAPHS[name], _params(GRAPHS[name], C=C))


def test_weights_sbm_small_workload(ctx):
    """The 10k-node SBM workload (T=10, s_r=1/T, S=10 T m), downsampled."""
    g = synth.sbm_small()
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, seed=1)
    p.downsample_C = 2.0
    _check_counts(ctx, g, p)


def test_certain_coin_is_plain_counting(ctx):
    """p_e = 1 on every arc (C >= max degree / 2): weights are 2^32 per draw
    and the CSR is the plain sparsifier's."""
    g = GRAPHS["chunglu2k"]
    deg = np.diff(g.indptr)
    p = _params(g, C=float(deg.max()))
    res = _check_counts(ctx, g, p)
    p0 = _params(g, C=0.0)
    plain = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p0)
    assert np.array_equal(to_np(res["x"]), to_np(plain["x"]))
    assert np.array_equal(to_np(res["weight"]).view(np.uint64),
                          to_np(plain["count"]).astype(np.uint64) << np.uint64(32))
    a = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    b = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p0)
    assert np.array_equal(to_np(a["indptr"]), to_np(b["indptr"]))
    assert np.array_equal(to_np(a["indices"]), to_np(b["indices"]))
    np.testing.assert_allclose(to_np(a["data"]), to_np(b["data"]), rtol=VAL_RTOL, atol=VAL_ATOL)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("C", [0.2, 2.0])
def test_csr_matches_oracle(ctx, name, C):
    g = GRAPHS[name]
    p = _params(g, rate=20.0, C=C, seed=4)
    out = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    sp = oracle.sparsifier(g.indptr, g.indices, p.T, p.s, p.samples, p.seed, p.b, C=C)
    assert np.array_equal(to_np(out["indptr"]), sp["indptr"])
    assert np.array_equal(to_np(out["indices"]).astype(np.int64), sp["indices"])
    np.testing.assert_allclose(to_np(out["data"]), sp["data"], rtol=VAL_RTOL, atol=VAL_ATOL)


def test_bucket_aggregation_refuses():
    c = _ctx(lne.AGG_BUCKET)
    try:
        g = GRAPHS["sbm600"]
        with pytest.raises(lne.LneError) as e:
            c.sparsifier_counts(lne.DeviceGraph.from_graph(g), _params(g, C=1.0))
        assert e.value.code == -5
        # plain counting still works on the same context
        assert c.sparsifier_counts(lne.DeviceGraph.from_graph(g), _params(g, C=0.0))["count"].numel() > 0
    finally:
        c.close()


def test_bad_constant_rejected(ctx):
    g = GRAPHS["sbm600"]
    dg = lne.DeviceGraph.from_graph(g)
    for C in [-1.0, float("nan"), float("inf")]:
        with pytest.raises(lne.LneError) as e:
            ctx.sparsifier_counts(dg, _params(g, C=C))
        assert e.value.code == -1


def test_embed_downsampled_sbm_small(ctx):
    """Whole method with downsampling on the 10k-node SBM against the oracle."""
    g = synth.sbm_small()
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    p.downsample_C = 2.0
    ref = oracle.embed(g.indptr, g.indices, 10, p.s, p.samples, 32, 1, 10, 0.5, 0.2, 1, C=2.0)
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    assert_subspace(X, ref["X"], tag="downsampled embed")


def test_bench_workload_unbiased_and_sparse(ctx):
    """BlogCatalog-shaped graph, S = 200 T m = 6.68e8 draws, C = ln n (the
    paper's choice). Properties that hold at any size:

    * Thm 1 (unbiasedness): the summed weights estimate the number of draws,
      |z| < 6 against the variance sum_draws (1 - p_e) / p_e;
    * the kept draws number sum_arcs n_e p_e in expectation (|z| < 6), and
      sum over arcs of p_e <= 2 C n (each vertex's arcs add at most C), the
      O(n log n) size bound of Sec. 4.1."""
    g = synth.blogcatalog_like()
    n = g.n
    C = lne.default_downsample_C(n)
    assert C == float(np.log(n))
    p = make_params(10, synth.dirichlet_weights(10, seed=3), 200.0 * 10 * g.m, seed=2, d=128)
    p.downsample_C = C
    dg = lne.DeviceGraph.from_graph(g)
    res = ctx.sparsifier_counts(dg, p)
    thr, w = oracle.arc_downsample(g.indptr, g.indices, C)
    pe = np.minimum(thr.astype(np.float64) / 2.0 ** 32, 1.0)
    n_e = oracle.arc_samples(g.n_arcs, p.samples, p.seed).astype(np.float64)
    assert res["total_samples"] == int(n_e.sum())
    wsum = to_np(res["weight"]).view(np.uint64)
    est = float(np.sum(wsum.astype(np.float64))) * 2.0 ** -32
    var = float(np.sum(n_e * (1.0 - pe) / pe))
    z = (est - n_e.sum()) / np.sqrt(max(var, 1.0))
    print(f"downsampled weight total {est:.6e} vs draws {n_e.sum():.6e}, z = {z:.2f}")
    assert abs(z) < 6.0
    assert np.sum(pe) <= 2.0 * C * n + 1e-6
    # kept draws per arc from raw output on a few arc ranges (-1 marks a drop)
    rng = np.random.default_rng(1)
    kept, mean, v = 0, 0.0, 0.0
    for _ in range(4):
        a0 = int(rng.integers(0, g.n_arcs - 20000))
        u1, _ = ctx.sample_pairs(dg, p, a0, a0 + 20000)
        kept += int((u1 >= 0).sum())
        ne, pp = n_e[a0:a0 + 20000], pe[a0:a0 + 20000]
        mean += float(np.sum(ne * pp))
        v += float(np.sum(ne * pp * (1.0 - pp)))
    assert abs(kept - mean) < 6.0 * np.sqrt(max(v, 1.0))
    out = ctx.sparsifier_csr(dg, p)
    ip = to_np(out["indptr"])
    assert ip[0] == 0 and ip[-1] == out["nnz"] and np.all(np.diff(ip) >= 0)
    assert bool((out["data"] > 0).all())


@pytest.mark.parametrize("name", ["ring1024", "sbm600"])
@pytest.mark.parametrize("C", [0.0, 0.5])
def test_keep_decisions_at_the_threshold(ctx, name, C):
    """b chosen so that a common (K, d_x d_y) lands on v = 1 to the last bits:
    the keep decisions there (fl(fl(K alpha) / fl(d_x d_y)) > 1 in FP64) must
    equal the oracle's exactly, with and without downsampling."""
    g = GRAPHS[name]
    p = _params(g, T=4, rate=6.0, C=C, seed=21)
    x, y, cnt = oracle.sparsifier_counts(g.indptr, g.indices, p.T, p.s, p.samples, p.seed, C=C)
    deg = np.diff(g.indptr).astype(np.float64)
    K = np.asarray(cnt, dtype=np.float64) * (2.0 ** -32 if C > 0 else 1.0)
    off = np.flatnonzero(x != y)
    j = off[len(off) // 2]
    vol = float(g.n_arcs)
    p.b = float(K[j] * vol * vol / (2.0 * p.samples) / (deg[x[j]] * deg[y[j]]))
    sp = oracle.sparsifier(g.indptr, g.indices, p.T, p.s, p.samples, p.seed, p.b, C=C)
    near = np.abs(sp["v"] - 1.0) < 1e-12
    assert near.sum() >= 1
    out = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    assert np.array_equal(to_np(out["indptr"]), sp["indptr"])
    assert np.array_equal(to_np(out["indices"]).astype(np.int64), sp["indices"])
    np.testing.assert_allclose(to_np(out["data"]), sp["data"], rtol=VAL_RTOL, atol=VAL_ATOL)
