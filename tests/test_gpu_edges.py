"""Degenerate and boundary cases of the GPU path against the oracle:

* the smallest graph (one edge), a star, self-loops and parallel arcs: exact
  counts on every aggregation method;
* fewer samples than arcs (rate 0.3 per arc) and all weight on the longest
  window (T = 16, r = 16);
* an empty arc range;
* the randomized SVD at its largest width (c = d + oversample = 160) and the
  whole method on a tiny graph with d + oversample = n.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["table", "bucket", "sort"])
def ctx(request):
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    c.set_option(lne.OPT_AGGREGATION, {"table": lne.AGG_TABLE, "bucket": lne.AGG_BUCKET,
                                       "sort": lne.AGG_SORT}[request.param])
    yield c
    c.close()


def _graph(n, edges, name):
    u = np.array([a for a, _ in edges], dtype=np.int64)
    v = np.array([b for _, b in edges], dtype=np.int64)
    # symmetric CSR with every listed edge in both rows (a self-loop once per listing)
    rows = np.concatenate([u, v[u != v]])
    cols = np.concatenate([v, u[u != v]])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    return synth.Graph(n, indptr, cols.astype(np.int32), None, name)


GRAPHS = {
    "one_edge": _graph(2, [(0, 1)], "one_edge"),
    "star": _graph(31, [(0, i) for i in range(1, 31)], "star"),
    "loops_and_parallel": _graph(6, [(0, 1), (0, 1), (1, 2), (2, 2), (2, 3), (3, 4), (4, 5), (5, 5), (5, 0)],
                                 "loops"),
}


def _check_counts(ctx, g, p):
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    x, y, c = oracle.sparsifier_counts(g.indptr, g.indices, p.T, p.s, p.samples, p.seed)
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["y"]).astype(np.int64), y)
    assert np.array_equal(to_np(res["count"]).astype(np.int64), c)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("T,rate", [(10, 40.0), (3, 0.3)])
def test_small_graph_counts(ctx, name, T, rate):
    g = GRAPHS[name]
    _check_counts(ctx, g, make_params(T, synth.dirichlet_weights(T, 4), rate * g.n_arcs, seed=6))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_small_graph_csr(ctx, name):
    g = GRAPHS[name]
    p = make_params(5, np.ones(5), 50.0 * g.n_arcs, seed=2)
    out = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    ref = oracle.sparsifier(g.indptr, g.indices, 5, p.s, p.samples, p.seed)
    assert np.array_equal(to_np(out["indptr"]), ref["indptr"])
    assert np.array_equal(to_np(out["indices"]).astype(np.int64), ref["indices"])
    np.testing.assert_allclose(to_np(out["data"]), ref["data"], rtol=1e-6, atol=1e-7)


def test_longest_window_only(ctx):
    g = synth.sbm(600, 3, 0.05, 0.005, seed=3)
    s = np.zeros(16)
    s[15] = 1.0
    p = make_params(16, s, 2.0 * g.n_arcs, seed=8)
    _check_counts(ctx, g, p)
    u1, v1 = ctx.sample_pairs(lne.DeviceGraph.from_graph(g), p, 100, 400)
    tr = oracle.sample_trace(g.indptr, g.indices, 16, s, p.samples, p.seed, 100, 400, fields=("r", "u1", "v1"))
    assert np.all(tr["r"] == 16)
    assert np.array_equal(to_np(u1).astype(np.int64), tr["u1"])
    assert np.array_equal(to_np(v1).astype(np.int64), tr["v1"])


def test_empty_arc_range(ctx):
    g = GRAPHS["star"]
    u1, v1 = ctx.sample_pairs(lne.DeviceGraph.from_graph(g), make_params(4, np.ones(4), 10.0 * g.n_arcs), 7, 7)
    assert u1.numel() == 0 and v1.numel() == 0


def test_rsvd_widest_sketch():
    """c = d + oversample = 160, the small SVD's limit."""
    rng = np.random.default_rng(4)
    n, d = 700, 144
    lam = np.concatenate([np.geomspace(60, 20, d), rng.uniform(-1, 1, n - d)])
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = sp.csr_matrix(((Qm * lam) @ Qm.T))
    ref = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, 2, 16, 5)
    c = lne.Context(0)
    try:
        csr = dict(n=n, nnz=M.nnz, indptr=torch.as_tensor(M.indptr.astype(np.int64)).cuda(),
                   indices=torch.as_tensor(M.indices.astype(np.int32)).cuda(),
                   data=torch.as_tensor(M.data.astype(np.float32)).cuda())
        out = c.rsvd(csr, make_params(1, [1.0], 1.0, d=d, oversample=16, q=2, seed=5))
        np.testing.assert_allclose(to_np(out["sigma"]), ref["sigma"], rtol=1e-4)
        U = to_np(out["U"]).astype(np.float64)
        assert oracle.subspace_sin(U, ref["U"]) <= 1e-3
        assert np.max(np.abs(U.T @ U - np.eye(d))) <= 1e-5
        with pytest.raises(lne.LneError):
            c.rsvd(csr, make_params(1, [1.0], 1.0, d=d, oversample=17, q=1, seed=5))   # c = 161
    finally:
        c.close()


def test_embed_tiny_graph_full_width():
    """n = 31, d + oversample = n: the sketch spans the whole space."""
    g = synth.erdos_renyi(31, 0.25, seed=5)
    p = make_params(4, [0.4, 0.3, 0.2, 0.1], 200.0 * g.n_arcs, d=8, oversample=23, q=1, k=3, seed=3)
    ref = oracle.embed(g.indptr, g.indices, 4, p.s, p.samples, 8, 1, 3, 0.5, 0.2, 3, oversample=23)
    c = lne.Context(0)
    try:
        X = to_np(c.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    finally:
        c.close()
    assert X.shape == (31, 8) and np.all(np.isfinite(X))
    # compare the leading directions that are separated from the next one
    sig = ref["prop"]["sigma"]
    gaps = (sig[:-1] - sig[1:]) / sig[:-1]
    sep = np.nonzero(gaps[:7] > 1e-2)[0]
    if len(sep):
        k = int(sep.max()) + 1
        assert oracle.subspace_sin(X[:, :k], ref["X"][:, :k]) <= 1e-2
