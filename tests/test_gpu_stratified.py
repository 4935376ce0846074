"""Window-stratified sampling (LNE_OPT_STRATIFIED) on the GPU against the
oracle. Draws take r ~ U{1..T}; counts are kept per (pair, r); a weighting s
becomes K_s = sum_r w_r C_r (2^-24 units). Not a procedure of the paper: the
oracle restates it and pins its unbiasedness against the exact law.

* (x, y, r, count) entries bit-exact, every T;
* the CSR for several weightings (uniform, Dirichlet, a single window):
  structure and keep decisions exact, values within 1e-6;
* uniform s gives the plain sampler's matrix (uniform s) exactly in structure;
* batched tuning with shared strata equals one-candidate stratified runs;
* edge downsampling is refused in this mode.
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


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    c.set_option(lne.OPT_STRATIFIED, 1)
    yield c
    c.close()


GRAPHS = {
    "sbm600": synth.sbm(600, 3, 0.05, 0.005, seed=3),
    "chunglu2k": synth.chung_lu(2000, 12000, 2.1, seed=4, n_labels=5),
    "lollipop": synth.lollipop_tiny(),
    "ring97": synth.ring(97),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("T,rate", [(10, 10.0), (1, 3.0), (5, 6.5), (16, 2.0)])
def test_strata_bit_exact(ctx, name, T, rate):
    g = GRAPHS[name]
    p = make_params(T, synth.dirichlet_weights(T, 3), rate * g.n_arcs, seed=17)
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    x, y, r, c = oracle.stratified_counts(g.indptr, g.indices, T, p.samples, p.seed)
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["y"]).astype(np.int64), y)
    assert np.array_equal(to_np(res["window"]).astype(np.int64), r)
    assert np.array_equal(to_np(res["count"]).astype(np.int64), c)


def _weightings(T):
    one = np.zeros(T)
    one[min(2, T - 1)] = 1.0
    return {"uniform": np.ones(T), "dirichlet": synth.dirichlet_weights(T, 7), "single": one}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("kind", ["uniform", "dirichlet", "single"])
def test_csr_matches_oracle(ctx, name, kind):
    g = GRAPHS[name]
    T = 6
    s = _weightings(T)[kind]
    p = make_params(T, s, 20.0 * g.n_arcs, seed=5, b=1.5)
    out = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    sp = oracle.stratified_sparsifier(g.indptr, g.indices, T, s, p.samples, p.seed, p.b)
    assert np.array_equal(to_np(out["indptr"]), sp["indptr"])
    assert np.array_equal(to_np(out["indices"]).astype(np.int64), sp["indices"])
    np.testing.assert_allclose(to_np(out["data"]), sp["data"], rtol=VAL_RTOL, atol=VAL_ATOL)


def test_uniform_s_is_the_plain_sampler(ctx):
    g = GRAPHS["chunglu2k"]
    p = make_params(8, np.ones(8), 15.0 * g.n_arcs, seed=9)
    a = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    plain = lne.Context(0)
    try:
        b = plain.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
        assert np.array_equal(to_np(a["indptr"]), to_np(b["indptr"]))
        assert np.array_equal(to_np(a["indices"]), to_np(b["indices"]))
        np.testing.assert_allclose(to_np(a["data"]), to_np(b["data"]), rtol=VAL_RTOL, atol=VAL_ATOL)
    finally:
        plain.close()


def test_tune_batch_shares_strata(ctx):
    """Candidates with different s (same T, S, seed) from one sampling pass:
    each equals its one-candidate stratified run."""
    g = synth.chung_lu(3000, 30000, 2.1, seed=9, n_labels=12)
    idx = np.random.default_rng(5).permutation(g.n)
    tr, te = idx[: g.n // 2], idx[g.n // 2:]
    dg = lne.DeviceGraph.from_graph(g)
    lab, trd, ted = torch.as_tensor(g.labels).cuda(), torch.as_tensor(tr).cuda(), torch.as_tensor(te).cuda()
    cands = [make_params(10, synth.dirichlet_weights(10, j), 50.0 * g.m, d=32, q=1, k=k, theta=0.5, mu=0.2, seed=3)
             for j, k in enumerate([10, 5, 0, 10])]
    ma, mi, X = ctx.tune_batch(dg, cands, lab, trd, ted, want_embeddings=True)
    for j, p in enumerate(cands):
        Xs = to_np(ctx.embed(dg, p))
        Xb = to_np(X[j])
        err = np.max(np.abs(Xb - Xs)) / np.max(np.abs(Xs))
        assert err <= 1e-5, (j, err)
        mas, mis = ctx.macro_f1(torch.as_tensor(Xs).cuda(), lab, trd, ted)
        tol = 0.0 if np.array_equal(Xb, Xs) else 0.005
        assert abs(ma[j] - mas) <= tol and abs(mi[j] - mis) <= tol


def test_embed_matches_oracle(ctx):
    g = synth.sbm_small()
    s = synth.dirichlet_weights(10, 2)
    p = make_params(10, s, 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    sp = oracle.stratified_sparsifier(g.indptr, g.indices, 10, s, p.samples, p.seed)
    rs = oracle.fast_randomized_svd(sp["indptr"], sp["indices"], sp["data"], 32, 1, 16, 1)
    X0 = oracle.embedding_from_svd(rs["U"], rs["sigma"])
    ref = oracle.spectral_propagation(g.indptr, g.indices, X0, 10, 0.5, 0.2)["X"]
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    assert_subspace(X, ref, tag="stratified embed")


def test_downsampling_refused(ctx):
    g = GRAPHS["sbm600"]
    p = make_params(10, np.ones(10), 10.0 * g.n_arcs)
    p.downsample_C = 1.0
    with pytest.raises(lne.LneError) as e:
        ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    assert e.value.code == -5
