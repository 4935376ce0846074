"""Pins of the oracle on weighted graphs (positive integer arc weights A_uv,
symmetric), against the mathematics of the weighted method:

* the weighted walk step is the inverse CDF of A_x. / d_x with thresholds
  floor(2^32 P_j / d) (closed-form boundaries, exact law when d divides 2^32);
* unit weights reproduce the unweighted draws' arcs, windows, splits and
  coins bit for bit (the step maps words to neighbours by the inverse CDF);
* per-arc sample counts follow S A_a / vol;
* pair counts match the exact expectation S / vol sum_r s_r D (D^-1 A)^r of
  the weighted walk (z-scores), and Eq. 1 at that expectation is the dense
  weighted NetMF matrix;
* edge downsampling follows p_e = min(1, C A_uv (1/d_u + 1/d_v)) (Sec. 4.1);
* the propagation equals the spectral filter of the weighted normalised
  Laplacian.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2302_07084_gb300 import synth


def test_weighted_choice_boundaries():
    w = [1, 2, 5]                      # d = 8: thresholds 2^29, 3 2^29
    t0, t1 = 2 ** 29, 3 * 2 ** 29
    for word, j in [(0, 0), (t0 - 1, 0), (t0, 1), (t1 - 1, 1), (t1, 2), (2 ** 32 - 1, 2)]:
        assert oracle.weighted_choice(w, word) == j
    # a weight not dividing 2^32: threshold floor(2^32 * 1 / 3)
    t = (2 ** 32) // 3
    assert oracle.weighted_choice([1, 2], t - 1) == 0 and oracle.weighted_choice([1, 2], t) == 1
    assert oracle.weighted_choice([7], 123) == 0


def test_weighted_choice_exact_law():
    """d = 16 divides 2^32: word counts per arc are exactly w_j 2^28 (checked on
    every 2^20-th word, with the exact boundaries)."""
    w = np.array([3, 1, 4, 1, 7], dtype=np.uint32)
    words = np.arange(0, 2 ** 32, 2 ** 20, dtype=np.uint64)
    picks = np.array([oracle.weighted_choice(w, int(x)) for x in words])
    counts = np.bincount(picks, minlength=len(w))
    np.testing.assert_array_equal(counts, w.astype(np.int64) * 2 ** 28 // 2 ** 20)


def _weighted(g, seed=3, lo=1, hi=9):
    return synth.edge_weights(g, lo, hi, seed)


def test_unit_weights_reproduce_unweighted_draw_heads():
    """Unit weights: the same per-arc counts, windows, splits and coins; a step
    then picks neighbour j for words in [floor(2^32 j / deg), floor(2^32 (j+1)
    / deg)) -- uniform like the unweighted w mod deg, but another word-to-
    neighbour map, so the endpoints agree in law, not draw by draw."""
    g = synth.sbm(200, 2, 0.1, 0.02, seed=4)
    S = 7.5 * g.n_arcs
    f = ("arc", "r", "sigma", "coin")
    a = oracle.sample_trace(g.indptr, g.indices, 6, np.ones(6), S, 5, fields=f)
    b = oracle.sample_trace(g.indptr, g.indices, 6, np.ones(6), S, 5, fields=f, weights=np.ones(g.n_arcs, np.uint32))
    for k in f:
        np.testing.assert_array_equal(a[k], b[k])
    for deg in (1, 3, 7, 100):
        for j in range(deg):
            lo = (2 ** 32 * j) // deg
            assert oracle.weighted_choice(np.ones(deg), lo) == j
            if lo > 0:
                assert oracle.weighted_choice(np.ones(deg), lo - 1) == j - 1


def test_edge_weights_are_symmetric():
    g = synth.sbm(100, 2, 0.2, 0.05, seed=1)
    w = _weighted(g)
    src = np.repeat(np.arange(g.n), np.diff(g.indptr))
    A = sp.csr_matrix((w.astype(float), g.indices, g.indptr), shape=(g.n, g.n)).toarray()
    np.testing.assert_array_equal(A, A.T)
    assert w.min() >= 1 and w.max() <= 9 and len(np.unique(w)) > 3
    assert np.all(A[src, g.indices] == w)


def test_per_arc_samples_follow_weights():
    g = synth.sbm(100, 2, 0.2, 0.05, seed=1)
    w = _weighted(g, hi=20)
    S = 37.3 * g.n_arcs
    n_a = oracle.arc_samples(g.n_arcs, S, 3, weights=w)
    rate = S * w.astype(np.float64) / w.sum()
    assert np.all((n_a == np.floor(rate)) | (n_a == np.floor(rate) + 1))
    # the Bernoulli parts add up to the fractional parts (z-score)
    frac = rate - np.floor(rate)
    z = ((n_a - np.floor(rate)).sum() - frac.sum()) / np.sqrt(np.sum(frac * (1 - frac)))
    assert abs(z) < 6
    assert oracle.count_samples(g.n_arcs, S, 3, weights=w) == int(n_a.sum())


def _expected_counts_weighted(g, w, T, s, S):
    A = sp.csr_matrix((w.astype(np.float64), g.indices, g.indptr), shape=(g.n, g.n)).toarray()
    d = A.sum(1)
    P = A / d[:, None]
    s = np.asarray(s, float) / np.sum(s)
    acc = np.zeros((g.n, g.n))
    Pr = np.eye(g.n)
    for r in range(1, T + 1):
        Pr = Pr @ P
        acc += s[r - 1] * (d[:, None] * Pr)
    EC = S / d.sum() * acc
    EK = EC + EC.T
    EK[np.diag_indices(g.n)] = np.diag(EC)
    return EK


def test_weighted_counts_match_exact_expectation():
    g = synth.lollipop_tiny()
    w = _weighted(g, seed=5, hi=6)
    T = 4
    s = [0.2, 0.4, 0.1, 0.3]
    S = 40000.0 * g.n_arcs
    x, y, cnt = oracle.sparsifier_counts(g.indptr, g.indices, T, s, S, seed=29, weights=w)
    K = np.zeros((g.n, g.n))
    K[x, y] = cnt
    EK = _expected_counts_weighted(g, w, T, s, S)
    iu = np.triu_indices(g.n)
    assert np.all(K[iu][EK[iu] == 0] == 0)
    m = EK[iu] > 0
    z = (K[iu][m] - EK[iu][m]) / np.sqrt(EK[iu][m])
    assert np.max(np.abs(z)) < 6


def test_weighted_eq1_reproduces_dense_netmf():
    g = synth.sbm(40, 2, 0.4, 0.1, seed=8)
    w = _weighted(g, seed=2, hi=7)
    T, s, S = 3, [0.5, 0.3, 0.2], 1.0e6
    EK = _expected_counts_weighted(g, w, T, s, S)
    iu = np.triu_indices(g.n)
    deg = oracle.weighted_degrees(g.indptr, w)
    v, keep, val = oracle.netmf_values(iu[0], iu[1], EK[iu], deg, S)
    W = oracle.netmf_dense(g.indptr, g.indices, T, s, weights=w)
    np.testing.assert_allclose(v, W[iu], rtol=1e-12, atol=1e-14)
    assert np.array_equal(keep, W[iu] > 1.0)
    # unit weights: the unweighted matrix
    np.testing.assert_allclose(oracle.netmf_dense(g.indptr, g.indices, T, s, weights=np.ones(g.n_arcs)),
                               oracle.netmf_dense(g.indptr, g.indices, T, s), rtol=1e-14)


def test_weighted_downsampling_rule():
    g = synth.sbm(60, 2, 0.3, 0.05, seed=3)
    w = _weighted(g, hi=5)
    thr, wt = oracle.arc_downsample(g.indptr, g.indices, 0.3, weights=w)
    deg = oracle.weighted_degrees(g.indptr, w)
    src = np.repeat(np.arange(g.n), np.diff(g.indptr))
    p = np.minimum(1.0, w * (0.3 * (1.0 / deg[src] + 1.0 / deg[g.indices])))   # A (C (1/d_u + 1/d_v))
    np.testing.assert_array_equal(thr, np.where(p >= 1.0, 2.0 ** 32, np.floor(p * 2.0 ** 32)).astype(np.uint64))
    np.testing.assert_array_equal(wt, np.floor(2.0 ** 32 / p + 0.5).astype(np.uint64))


@pytest.mark.parametrize("k,theta,mu", [(10, 0.5, 0.2), (3, 1.0, 0.0)])
def test_weighted_propagation_matches_spectral_filter(k, theta, mu):
    g = synth.sbm(60, 3, 0.3, 0.05, seed=12)
    w = _weighted(g, hi=9)
    X0 = np.random.default_rng(3).standard_normal((g.n, 8))
    out = oracle.spectral_propagation(g.indptr, g.indices, X0, k, theta, mu, weights=w)
    A = sp.csr_matrix((w.astype(np.float64), g.indices, g.indptr), shape=(g.n, g.n)).toarray()
    d = A.sum(1)
    Dm = np.diag(d ** -0.5)
    lam, V = np.linalg.eigh(np.eye(g.n) - Dm @ A @ Dm)
    y = np.clip(0.5 * (lam - mu) ** 2 - 1.0, -1.0, 1.0)
    c = oracle.chebyshev_coefficients(k, theta)
    g_lam = np.cos(np.outer(np.arange(k), np.arccos(y))).T @ c
    F = np.diag(d ** -0.5) @ (V * g_lam) @ V.T @ np.diag(d ** 0.5) @ X0
    P = (A / d[:, None]) @ (X0 - F)
    np.testing.assert_allclose(out["F"], F, atol=1e-10 * np.abs(F).max())
    np.testing.assert_allclose(out["P"], P, atol=1e-10 * np.abs(P).max())
