"""The surrogate's graph statistics on graphs whose values are known in closed
form (complete graph, star, cycle, two components), and the candidate feature
layout, without a GPU: the spectrum (the one statistic the library's
randomized SVD computes) is replaced by fixed values here."""
import numpy as np
import pytest

from paper_2302_07084_gb300 import lne, search


def _csr(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    indptr = np.zeros(n + 1, np.int64)
    indptr[1:] = np.cumsum([len(r) for r in adj])
    indices = np.array([v for r in adj for v in sorted(r)], np.int64)
    return indptr, indices


@pytest.fixture
def stats(monkeypatch):
    monkeypatch.setattr(search, "_normalized_adjacency_spectrum",
                        lambda ctx, indptr, indices, deg, count, seed: np.array([1.0, 0.5, 0.25, 0.125]))
    return lambda g: search.graph_statistics(None, *g, seed=0, sample=10_000)


NAMES = ["log_n", "log_m", "deg_mean", "deg_std", "deg_max", "skew", "gini", "blocks", "assort", "clustering",
         "lam2", "lam3", "lam4", "density", "growth", "giant"]


def _named(v):
    assert v.shape == (search.N_STATS,)
    return dict(zip(NAMES, v))


def test_complete_graph(stats):
    n = 6
    s = _named(stats(_csr(n, [(a, b) for a in range(n) for b in range(a + 1, n)])))
    assert s["log_n"] == pytest.approx(np.log(6)) and s["log_m"] == pytest.approx(np.log(15))
    assert s["deg_mean"] == 5 and s["deg_std"] == 0 and s["deg_max"] == 5 and s["gini"] == pytest.approx(0)
    assert s["clustering"] == pytest.approx(1.0) and s["density"] == pytest.approx(1.0)
    assert s["growth"] == 0.0 and s["giant"] == 1.0
    assert (s["lam2"], s["lam3"], s["lam4"]) == (0.5, 0.25, 0.125)


def test_star(stats):
    n = 9   # hub 0 and 8 leaves
    s = _named(stats(_csr(n, [(0, i) for i in range(1, n)])))
    assert s["clustering"] == 0.0
    assert s["assort"] == pytest.approx(-1.0)           # every arc joins degree 8 and degree 1
    # hub: no two-hop vertex beyond its leaves; a leaf reaches the 7 other leaves
    assert s["growth"] == pytest.approx((0.0 + 8 * 7.0) / 9)
    deg = np.array([8] + [1] * 8, float)
    gini = np.abs(deg[:, None] - deg[None, :]).sum() / (2 * n * n * deg.mean())
    assert s["gini"] == pytest.approx(gini)
    assert s["deg_max"] == 8 and s["skew"] > 0


def test_cycle_and_components(stats):
    c = [(i, (i + 1) % 8) for i in range(8)]           # an 8-cycle
    s = _named(stats(_csr(8, c)))
    assert s["growth"] == pytest.approx(1.0) and s["clustering"] == 0.0 and s["deg_std"] == 0.0
    two = c + [(8 + i, 8 + (i + 1) % 4) for i in range(4)]   # plus a separate 4-cycle
    s = _named(stats(_csr(12, two)))
    assert s["giant"] == pytest.approx(8 / 12)


def test_candidate_features_layout():
    p = lne.Params(T=4, s=[1.0, 1.0, 2.0, 0.0], samples=1.0, k=7, theta=0.6, mu=0.3, q=2)
    st = np.arange(search.N_STATS, dtype=np.float64)
    f = search.candidate_features(p, st)
    assert f.shape == (lne.SURROGATE_INPUTS,) and f.dtype == np.float32
    np.testing.assert_allclose(f[:10], [0.25, 0.25, 0.5, 0.0] + [0.0] * 6)
    np.testing.assert_allclose(f[10:14], [7, 0.6, 0.3, 2], rtol=1e-6)
    np.testing.assert_array_equal(f[14:], st.astype(np.float32))


def test_training_rows_center_scores_per_graph():
    p = [[lne.Params(T=1, s=[1.0], k=k) for k in (3, 5)], [lne.Params(T=1, s=[1.0], k=k) for k in (4, 6)]]
    st = [np.zeros(search.N_STATS), np.ones(search.N_STATS)]
    X, y = search.training_rows(p, st, np.array([[0.5, 0.7], [0.2, 0.2]]))
    assert X.shape == (4, lne.SURROGATE_INPUTS)
    np.testing.assert_allclose(y, [-0.1, 0.1, 0.0, 0.0], atol=1e-7)
