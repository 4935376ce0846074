"""Graphs beyond the dense pair table (n > 65536): 64-bit pair keys, radix
sort and run lengths, and the symmetric CSR assembled from the sorted pairs.
Counts must equal the oracle's bit for bit and the CSR its structure (values
within the trunc_log tolerance of the small cases)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def big():
    # 150,000 vertices: 36-bit pair keys, past the 65,536-vertex table limit
    return synth.chung_lu(150_000, 1_200_000, 2.2, seed=4)


def test_large_counts_bit_exact(ctx, big):
    g = big
    s = np.full(5, 0.2)
    p = make_params(5, s, 5.0 * g.n_arcs, seed=11)
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    x, y, c = oracle.sparsifier_counts(g.indptr, g.indices, 5, s, p.samples, p.seed)
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed)
    assert np.array_equal(to_np(res["x"]).astype(np.int64), x)
    assert np.array_equal(to_np(res["y"]).astype(np.int64), y)
    assert np.array_equal(to_np(res["count"]).astype(np.int64), c)


def test_large_csr_matches_oracle(ctx, big):
    g = big
    s = synth.dirichlet_weights(5, seed=6)
    p = make_params(5, s, 3.0 * g.n_arcs, seed=12)
    csr = ctx.sparsifier_csr(lne.DeviceGraph.from_graph(g), p)
    ref = oracle.sparsifier(g.indptr, g.indices, 5, s, p.samples, p.seed)
    assert np.array_equal(to_np(csr["indptr"]), ref["indptr"])
    assert np.array_equal(to_np(csr["indices"]).astype(np.int64), ref["indices"])
    np.testing.assert_allclose(to_np(csr["data"]).astype(np.float64), ref["data"], rtol=1e-6, atol=1e-7)


def test_large_embedding_runs(ctx, big):
    g = big
    p = make_params(5, np.full(5, 0.2), 3.0 * g.n_arcs, d=32, q=1, k=5, seed=13)
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    assert X.shape == (g.n, 32) and np.all(np.isfinite(X))
    # X = U Sigma^1/2 with orthonormal U: X^T X is diagonal (the singular values)
    G = X.T @ X
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-4 * np.abs(np.diag(G)).max()
    assert np.all(np.diff(np.diag(G)) <= 1e-6 * np.diag(G)[0])


def test_auto_uses_the_sort_path_beyond_the_table(ctx, big):
    g = big
    p = make_params(1, [1.0], 1.0 * g.n_arcs, seed=14)
    ctx.set_option(lne.OPT_AGGREGATION, lne.AGG_TABLE)
    with pytest.raises(lne.LneError) as e:
        ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    assert e.value.code == -5
    ctx.set_option(lne.OPT_AGGREGATION, lne.AGG_AUTO)
    res = ctx.sparsifier_counts(lne.DeviceGraph.from_graph(g), p)
    assert res["total_samples"] == oracle.count_samples(g.n_arcs, p.samples, p.seed)


def test_10m_vertex_graph_sampled_draws(ctx):
    """The 10M-vertex, 200M-edge Chung-Lu graph of the large precision run
    (generated on the GPU): three ranges of 2000 arcs (start, middle, end) are
    drawn by the library and by the oracle, bit for bit, at that run's rate
    (S = 5 T m, T = 5)."""
    n, m = 10_000_000, 200_000_000
    indptr, indices = synth.chung_lu_device(n, m, 2.2, seed=4)
    torch.cuda.empty_cache()
    g = lne.DeviceGraph.from_tensors(indptr, indices)
    s = [0.2] * 5
    p = make_params(5, s, 5.0 * 5 * m, seed=4)
    hp, hi = indptr.cpu().numpy(), indices.cpu().numpy().astype(np.int32)
    drawn = 0
    for a0 in (0, g.nnz // 2, g.nnz - 2000):
        u1, v1 = ctx.sample_pairs(g, p, a0, a0 + 2000)
        tr = oracle.sample_trace(hp, hi, 5, s, p.samples, p.seed, a0, a0 + 2000, fields=("u1", "v1"))
        assert np.array_equal(to_np(u1).astype(np.int64), tr["u1"])
        assert np.array_equal(to_np(v1).astype(np.int64), tr["v1"])
        drawn += int(u1.numel())
    assert drawn > 70_000
    del g, indptr, indices
    ctx.trim()
    torch.cuda.empty_cache()
