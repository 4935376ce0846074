"""Weighted graphs (positive integer arc weights) on the GPU against the
oracle: arc a draws S A_a / vol samples in expectation, a walk step takes
arc j of x by the inverse CDF of A_x. / d_x, and Eq. 1, edge downsampling and
the propagation use the weighted degrees and volume.

* raw draws bit-exact (every arc range, several weight ranges and T);
* pair counts bit-exact on every aggregation method, downsampled weight sums
  bit-exact, window-stratified entries bit-exact;
* the CSR: structure and keep decisions exact, values within 1e-6;
* the weighted propagation (D^-1 A with weights) against the oracle's;
* the whole method, and batched tuning against one-candidate runs;
* zero weights and weighted degrees of 2^31 are refused.
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


@pytest.fixture(scope="module", params=["table", "bucket", "sort"])
def ctx(request):
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    c.set_option(lne.OPT_AGGREGATION, {"table": lne.AGG_TABLE, "bucket": lne.AGG_BUCKET,
                                       "sort": lne.AGG_SORT}[request.param])
    c.agg_name = request.param
    yield c
    c.close()


def _cases():
    a = synth.sbm(600, 3, 0.05, 0.005, seed=3)
    b = synth.chung_lu(2000, 12000, 2.1, seed=4, n_labels=5)
    c = synth.lollipop_tiny()
    return {
        "sbm600_w9": (a, synth.edge_weights(a, 1, 9, 1)),
        "chunglu2k_w1000": (b, synth.edge_weights(b, 1, 1000, 2)),
        "lollipop_w5": (c, synth.edge_weights(c, 1, 5, 3)),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("T,rate", [(10, 3.0), (1, 2.0), (5, 2.5)])
def test_sample_pairs_bit_exact(ctx, name, T, rate):
    g, w = CASES[name]
    s = synth.dirichlet_weights(T, seed=T)
    p = make_params(T, s, rate * g.n_arcs, seed=77)
    dg = lne.DeviceGraph.from_graph(g, weights=w)
    for a0, a1 in [(0, g.n_arcs), (g.n_arcs // 3, g.n_arcs - 1)]:
        u1, v1 = ctx.sample_pairs(dg, p, a0, a1)
        tr = oracle.sample_trace(g.indptr, g.indices, T, s, p.samples, p.seed, a0, a1, fields=("u1", "v1"),
                                 weights=w)
        assert np.array_equal(to_np(u1).astype(np.int64), tr["u1"])
        assert np.array_equal(to_np(v1).astype(np.int64), tr["v1"])


@pytest.mark.parametrize("name", list(CASES))
def test_counts_bit_exact(ctx, name):
    g, w = CASES[name]
    p = make_params(10, synth.dirichlet_weights(10, 5), 20.0 * g.n_arcs, seed=9)
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g, weights=w), p)
    x, y, c = oracle.sparsifier_counts(g.indptr, g.indices, 10, p.s, p.samples, p.seed, weights=w)
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed, weights=w)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["y"]).astype(np.int64), y)
    assert np.array_equal(to_np(res["count"]).astype(np.int64), c)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("rate", [1.0, 20.0])
def test_csr_matches_oracle(ctx, name, rate):
    g, w = CASES[name]
    p = make_params(10, np.full(10, 0.1), rate * g.n_arcs, seed=4, b=1.3)
    out = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g, weights=w), p)
    sp = oracle.sparsifier(g.indptr, g.indices, 10, p.s, p.samples, p.seed, p.b, weights=w)
    assert np.array_equal(to_np(out["indptr"]), sp["indptr"])
    assert np.array_equal(to_np(out["indices"]).astype(np.int64), sp["indices"])
    np.testing.assert_allclose(to_np(out["data"]), sp["data"], rtol=VAL_RTOL, atol=VAL_ATOL)


@pytest.mark.parametrize("name", list(CASES))
def test_downsampled_weights_bit_exact(ctx, name):
    if ctx.agg_name == "bucket":
        pytest.skip("the bucket aggregation has no downsampling")
    g, w = CASES[name]
    p = make_params(6, synth.dirichlet_weights(6, 2), 15.0 * g.n_arcs, seed=13)
    p.downsample_C = 0.4
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g, weights=w), p)
    x, y, ws_ = oracle.sparsifier_counts(g.indptr, g.indices, 6, p.s, p.samples, p.seed, C=0.4, weights=w)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["weight"]).view(np.uint64), ws_)


def test_stratified_entries_bit_exact():
    g, w = CASES["chunglu2k_w1000"]
    c = lne.Context(0)
    try:
        c.set_option(lne.OPT_STRATIFIED, 1)
        p = make_params(7, np.ones(7), 8.0 * g.n_arcs, seed=3)
        res = c.sparsifier_counts(lne.DeviceGraph.from_graph(g, weights=w), p)
        x, y, r, cnt = oracle.stratified_counts(g.indptr, g.indices, 7, p.samples, p.seed, weights=w)
        assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
        assert np.array_equal(to_np(res["window"]).astype(np.int64), r)
        assert np.array_equal(to_np(res["count"]).astype(np.int64), cnt)
    finally:
        c.close()


@pytest.mark.parametrize("k,theta,mu", [(10, 0.5, 0.2), (3, 1.0, 0.0)])
def test_weighted_propagation_matches_oracle(k, theta, mu):
    g = synth.sbm(2000, 4, 0.02, 0.002, seed=8)
    w = synth.edge_weights(g, 1, 50, 4)
    d = 32
    X0 = np.random.default_rng(1).standard_normal((g.n, d))
    ref = oracle.spectral_propagation(g.indptr, g.indices, X0, k, theta, mu, weights=w)
    c = lne.Context(0)
    try:
        p = make_params(1, [1.0], 1.0, d=d, k=k, theta=theta, mu=mu)
        out = c.propagate(lne.DeviceGraph.from_graph(g, weights=w), p, torch.as_tensor(X0.astype(np.float32)).cuda(),
                          want_intermediates=True)
    finally:
        c.close()
    F, P = to_np(out["F"]), to_np(out["P"])
    assert np.max(np.abs(F - ref["F"])) <= 1e-4 * np.abs(ref["F"]).max()
    assert np.max(np.abs(P - ref["P"])) <= 1e-4 * np.abs(ref["P"]).max()
    assert oracle.subspace_sin(to_np(out["X"]).astype(np.float64), ref["X"]) <= 1e-3


def test_weighted_embed_sbm_small():
    g = synth.sbm_small()
    w = synth.edge_weights(g, 1, 20, 6)
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    ref = oracle.embed(g.indptr, g.indices, 10, p.s, p.samples, 32, 1, 10, 0.5, 0.2, 1, weights=w)
    c = lne.Context(0)
    try:
        X = to_np(c.embed(lne.DeviceGraph.from_graph(g, weights=w), p)).astype(np.float64)
    finally:
        c.close()
    assert_subspace(X, ref["X"], tag="weighted embed")


def test_weighted_tune_batch_equals_single_runs():
    g = synth.chung_lu(3000, 30000, 2.1, seed=9, n_labels=12)
    w = synth.edge_weights(g, 1, 30, 7)
    idx = np.random.default_rng(5).permutation(g.n)
    dg = lne.DeviceGraph.from_graph(g, weights=w)
    lab = torch.as_tensor(g.labels).cuda()
    tr, te = torch.as_tensor(idx[: g.n // 2]).cuda(), torch.as_tensor(idx[g.n // 2:]).cuda()
    cands = [make_params(10, np.full(10, 0.1), 50.0 * g.m, d=32, q=1, k=k, theta=th, mu=mu, seed=3)
             for (k, th, mu) in [(10, 0.5, 0.2), (5, 1.0, 0.5), (0, 0.5, 0.2)]]
    c = lne.Context(0)
    try:
        ma, mi, X = c.tune_batch(dg, cands, lab, tr, te, want_embeddings=True)
        for j, p in enumerate(cands):
            Xs = to_np(c.embed(dg, p))
            err = np.max(np.abs(to_np(X[j]) - Xs)) / np.max(np.abs(Xs))
            assert err <= 1e-5, (j, err)
    finally:
        c.close()


def test_bad_weights_refused():
    g = synth.sbm(200, 2, 0.1, 0.02, seed=1)
    p = make_params(10, np.ones(10), 10.0 * g.n_arcs)
    c = lne.Context(0)
    try:
        w = synth.edge_weights(g, 1, 5, 1)
        w[3] = 0
        with pytest.raises(lne.LneError) as e:
            c.sparsifier_csr(lne.DeviceGraph.from_graph(g, weights=w), p)
        assert e.value.code == -1
        big = np.full(g.n_arcs, 2 ** 30, dtype=np.uint32)
        with pytest.raises(lne.LneError) as e:
            c.sparsifier_csr(lne.DeviceGraph.from_graph(g, weights=big), p)
        assert e.value.code == -5
        # the context stays usable
        assert c.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)["nnz"] > 0
    finally:
        c.close()
