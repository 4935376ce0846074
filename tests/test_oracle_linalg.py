"""Pins of the oracle's linear-algebra stages against closed forms.

* eigSVD (Algorithm 2) recovers planted singular triplets.
* Fast randomized SVD (Algorithm 4) recovers a planted spectrum with a gap,
  and its mean error respects the Eq. 2 bound.
* Gaussian sketch moments and normality (Algorithm 4).
* Sparse sign sketch: Floyd's subset sampling exhaustively uniform on a small
  case, exact row structure, uniform columns, fair signs, E[Omega^T Omega];
  Algorithm 4 with it recovers a planted spectrum.
* The Chebyshev coefficients expand exp(-theta y) (Bessel generating function).
* Spectral propagation equals the filter evaluated on the eigenvalues of the
  normalised Laplacian (Sec. 4.3), computed independently from a dense
  eigendecomposition and cos(i arccos y).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats as st

import oracle
from paper_2302_07084_gb300 import synth


def _orth(rng, n, k):
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return Q


def test_eig_svd_planted_triplets():
    rng = np.random.default_rng(0)
    n, k = 500, 24
    Ua, Vb = _orth(rng, n, k), _orth(rng, k, k)
    s = np.geomspace(100.0, 0.5, k)
    X = (Ua * s) @ Vb.T
    U, S, V = oracle.eig_svd(X)
    np.testing.assert_allclose(S, s, rtol=1e-9)
    np.testing.assert_allclose(np.abs(np.sum(U * Ua, axis=0)), 1.0, atol=1e-9)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-9)
    np.testing.assert_allclose((U * S) @ V.T, X, atol=1e-9 * s[0])
    # sign convention: largest-magnitude entry of each column is positive
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(k)] > 0)


def _planted_symmetric(rng, n, lam):
    Q = _orth(rng, n, n)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    Ms = sp.csr_matrix(M)
    return Q, Ms


def test_frsvd_recovers_planted_spectrum():
    rng = np.random.default_rng(1)
    n, d = 300, 12
    lam = np.concatenate([np.linspace(50, 20, d) * np.where(np.arange(d) % 3 == 0, -1, 1),
                          rng.uniform(-1, 1, n - d)])
    Q, M = _planted_symmetric(rng, n, lam)
    order = np.argsort(-np.abs(lam))
    top = Q[:, order[:d]]
    # the error of the range shrinks like (|lam_{d+1}| / |lam_d|)^(q+1) = 20^-(q+1)
    out = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, q=8,
                                     oversample=8, seed=5)
    np.testing.assert_allclose(out["sigma"], np.abs(lam[order[:d]]), rtol=1e-10)
    assert oracle.subspace_sin(out["U"], top) < 1e-9
    # more power iterations shrink the subspace error
    e = [oracle.subspace_sin(oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data,
                                                         d, q=q, oversample=8, seed=5)["U"], top)
         for q in (0, 1, 2)]
    assert e[0] > e[1] > e[2]


def test_frsvd_eq2_bound_mean():
    rng = np.random.default_rng(2)
    n, d, p = 200, 10, 6
    lam = 1.0 / np.arange(1, n + 1) ** 0.7
    Q, M = _planted_symmetric(rng, n, lam * np.where(rng.random(n) < 0.5, -1, 1))
    Md = M.toarray()
    sig_d1 = np.sort(lam)[::-1][d]
    for q in (0, 1, 2):
        errs = []
        for seed in range(20):
            out = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, q=q,
                                             oversample=p, seed=100 + seed)
            Qb = out["Q"]
            errs.append(np.linalg.norm(Md - Qb @ (Qb.T @ Md), 2))
        factor = (1 + np.sqrt(d / (p - 1)) + np.e * np.sqrt(d + p) / p * np.sqrt(n - d)) ** (1.0 / (q + 1))
        assert np.mean(errs) <= factor * sig_d1
        # no basis of d+p columns does better than sigma_{d+p+1} (Eckart-Young)
        assert min(errs) >= np.sort(lam)[::-1][d + p] * (1 - 1e-9)


def test_gaussian_sketch_law():
    n, c = 20000, 12
    Om = oracle.gaussian_sketch(n, c, seed=9)
    z = Om.ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert st.kstest(z, "norm").pvalue > 1e-4
    C = np.corrcoef(Om.T)
    assert np.max(np.abs(C - np.eye(c))) < 5 / np.sqrt(n)
    # narrower sketches are column prefixes of wider ones; same seed, same matrix
    np.testing.assert_array_equal(oracle.gaussian_sketch(50, 7, 9), Om[:50, :7])
    assert not np.array_equal(oracle.gaussian_sketch(50, 7, 10), Om[:50, :7])


@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_chebyshev_coefficients_expand_exponential(theta):
    y = np.linspace(-1, 1, 201)
    k = 25
    c = oracle.chebyshev_coefficients(k, theta)
    Tk = np.cos(np.outer(np.arange(k), np.arccos(y)))
    np.testing.assert_allclose(c @ Tk, np.exp(-theta * y), atol=1e-14, rtol=1e-13)
    # truncation at k = 10 stays within twice the Bessel tail
    c10 = oracle.chebyshev_coefficients(10, theta)
    err = np.max(np.abs(c10 @ Tk[:10] - np.exp(-theta * y)))
    assert err <= 2.0 * np.sum(np.abs(c[10:])) + 1e-15


def _spectral_filter(g, X0, k, theta, mu):
    A = sp.csr_matrix((np.ones(g.n_arcs), g.indices, g.indptr), shape=(g.n, g.n)).toarray()
    d = A.sum(1)
    Dm = np.diag(d ** -0.5)
    Nsym = np.eye(g.n) - Dm @ A @ Dm          # symmetric normalised Laplacian
    lam, V = np.linalg.eigh(Nsym)
    y = np.clip(0.5 * (lam - mu) ** 2 - 1.0, -1.0, 1.0)
    c = oracle.chebyshev_coefficients(k, theta)
    g_lam = np.cos(np.outer(np.arange(k), np.arccos(y))).T @ c
    # I - D^-1 A = D^-1/2 Nsym D^1/2
    G = np.diag(d ** -0.5) @ (V * g_lam) @ V.T @ np.diag(d ** 0.5)
    F = G @ X0
    P = (A / d[:, None]) @ (X0 - F)
    return F, P


@pytest.mark.parametrize("k,theta,mu", [(10, 0.5, 0.2), (3, 1.0, 0.0), (15, 0.3, 0.5), (1, 0.5, 0.2), (2, 0.7, 0.4)])
def test_propagation_matches_spectral_filter(k, theta, mu):
    g = synth.sbm(60, 3, 0.3, 0.05, seed=12)
    X0 = np.random.default_rng(3).standard_normal((g.n, 8))
    out = oracle.spectral_propagation(g.indptr, g.indices, X0, k, theta, mu)
    F, P = _spectral_filter(g, X0, k, theta, mu)
    np.testing.assert_allclose(out["F"], F, atol=1e-10 * np.abs(F).max())
    np.testing.assert_allclose(out["P"], P, atol=1e-10 * np.abs(P).max())
    # final stage: embedding from the SVD of P
    U, S, Vt = np.linalg.svd(P, full_matrices=False)
    np.testing.assert_allclose(out["sigma"], S, rtol=1e-8, atol=1e-12 * S[0])
    assert oracle.subspace_sin(out["U"], U) < 1e-7


def test_propagation_off_is_identity():
    g = synth.ring(10)
    X0 = np.arange(30, dtype=float).reshape(10, 3)
    out = oracle.spectral_propagation(g.indptr, g.indices, X0, 0, 0.5, 0.2)
    np.testing.assert_array_equal(out["X"], X0)


def test_embedding_recovers_blocks():
    g = synth.sbm(800, 4, 0.06, 0.004, seed=21)
    out = oracle.embed(g.indptr, g.indices, T=10, s=np.ones(10), S=100.0 * g.m, d=16, q=1, k=10,
                       theta=0.5, mu=0.2, seed=1)
    X = out["X"]
    y = np.argmax(g.labels, axis=1)
    rng = np.random.default_rng(0)
    idx = rng.permutation(g.n)
    tr, te = idx[: g.n // 2], idx[g.n // 2:]
    Y = np.eye(4)[y]
    Xa = np.hstack([X, np.ones((g.n, 1))])
    W, *_ = np.linalg.lstsq(Xa[tr], Y[tr], rcond=None)
    acc = np.mean(np.argmax(Xa[te] @ W, 1) == y[te])
    assert acc > 0.9


# sparse sign test matrix (the alternative Omega of Sec. 4.2; Tropp et al. 2019)

def test_floyd_subset_exhaustive():
    """Every word combination of Floyd's steps for c = 6, zeta = 3: each of the
    C(6, 3) = 20 subsets comes out equally often (4 x 5 x 6 / 20 = 6 times),
    always as distinct columns; words act modulo j + 1."""
    import itertools
    c, zeta = 6, 3
    combos = np.array(list(itertools.product(range(4), range(5), range(6))), dtype=np.uint64)
    out = oracle.floyd_subset(combos, c)
    assert np.all([len(set(r)) == zeta for r in out.tolist()])
    assert out.min() >= 0 and out.max() < c
    sets, counts = np.unique(np.sort(out, axis=1), axis=0, return_counts=True)
    assert len(sets) == 20 and np.all(counts == 6)
    shifted = combos + np.array([4, 5, 6], dtype=np.uint64) * np.uint64(977)
    np.testing.assert_array_equal(oracle.floyd_subset(shifted, c), out)


def test_sparse_sign_sketch_law():
    n, c, zeta = 20000, 48, 8
    Om = oracle.sparse_sign_sketch(n, c, zeta, seed=9)
    nz = Om != 0
    assert np.all(nz.sum(axis=1) == zeta)
    assert set(np.unique(Om[nz])) == {-1.0, 1.0}
    # columns uniform: each is chosen with probability zeta / c
    colcnt = nz.sum(axis=0)
    assert st.chisquare(colcnt).pvalue > 1e-4
    # signs fair and independent of the column
    neg = (Om < 0).sum()
    tot = n * zeta
    assert abs(neg - tot / 2) < 5 * np.sqrt(tot / 4)
    negc = (Om < 0).sum(axis=0)
    assert np.all(np.abs(negc - colcnt / 2) < 5 * np.sqrt(colcnt / 4) + 1)
    # E[Omega^T Omega] / n = (zeta / c) I
    G = Om.T @ Om / n
    np.testing.assert_allclose(np.diag(G), zeta / c, atol=6 * np.sqrt(zeta / c / n))
    pboth = zeta * (zeta - 1) / (c * (c - 1))
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 6 * np.sqrt(pboth / n)
    # deterministic in the seed; another seed gives another matrix
    np.testing.assert_array_equal(oracle.sparse_sign_sketch(40, c, zeta, 9), Om[:40])
    assert not np.array_equal(oracle.sparse_sign_sketch(40, c, zeta, 10), Om[:40])


def test_very_sparse_words_follow_the_stream_layout():
    """Entry (i, j) of the very sparse projection is decided by word j mod 4 of
    Philox counter (i, j // 4, 0, 0x56535250) under the sketch key (the
    known-answer-pinned Philox), against the threshold floor(2^32 / (2 s))."""
    n, c, s, seed = 5, 10, 2.5, 0x1234567890ABCDEF
    thr = oracle.very_sparse_threshold(n, s)
    assert thr == int(np.floor(4294967296.0 / 5.0))
    key = [(seed & 0xFFFFFFFF) ^ 0x4F4D4547, seed >> 32]
    Om = oracle.very_sparse_sketch(n, c, s, seed)
    for i in range(n):
        for j in range(c):
            w = int(oracle.philox4x32_10([i, j // 4, 0, 0x56535250], key)[j % 4])
            want = 1.0 if w < thr else (-1.0 if w < 2 * thr else 0.0)
            assert Om[i, j] == want
    assert oracle.very_sparse_threshold(10000, 0.0) == int(np.floor(4294967296.0 / 200.0))
    with pytest.raises(ValueError):
        oracle.very_sparse_threshold(10, 0.5)


def test_very_sparse_sketch_law():
    """Li, Hastie and Church's law: +1 and -1 with probability 1/(2s) each,
    independently per entry; E[Omega^T Omega] / n = (1/s) I."""
    n, c, s = 40000, 32, 6.0
    Om = oracle.very_sparse_sketch(n, c, s, seed=9)
    p = oracle.very_sparse_threshold(n, s) / 4294967296.0
    assert abs(p - 1.0 / (2 * s)) < 1e-9
    tot = n * c
    for v in (1.0, -1.0):
        k = int((Om == v).sum())
        assert abs(k - tot * p) < 5 * np.sqrt(tot * p * (1 - p))
    # per column the same law
    colnz = (Om != 0).sum(axis=0)
    assert st.chisquare(colnz).pvalue > 1e-4
    # nonzeros per row ~ Binomial(c, 2p)
    rownz = (Om != 0).sum(axis=1)
    assert abs(rownz.mean() - 2 * p * c) < 5 * np.sqrt(2 * p * c / n)
    assert abs(rownz.var() - c * 2 * p * (1 - 2 * p)) < 0.05 * c * 2 * p
    G = Om.T @ Om / n
    np.testing.assert_allclose(np.diag(G), 2 * p, atol=6 * np.sqrt(2 * p / n))
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 6 * np.sqrt(4 * p * p / n) + 6 / n
    np.testing.assert_array_equal(oracle.very_sparse_sketch(40, c, s, 9), Om[:40])
    assert not np.array_equal(oracle.very_sparse_sketch(40, c, s, 10), Om[:40])


def test_frsvd_very_sparse_recovers_planted_spectrum():
    rng = np.random.default_rng(1)
    n, d = 400, 12
    lam = np.concatenate([np.linspace(50, 20, d) * np.where(np.arange(d) % 3 == 0, -1, 1),
                          rng.uniform(-1, 1, n - d)])
    Q, M = _planted_symmetric(rng, n, lam)
    order = np.argsort(-np.abs(lam))
    out = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, q=8,
                                     oversample=8, seed=5, sketch="very_sparse", sparsity=4.0)
    np.testing.assert_allclose(out["sigma"], np.abs(lam[order[:d]]), rtol=1e-10)
    assert oracle.subspace_sin(out["U"], Q[:, order[:d]]) < 1e-9


@pytest.mark.parametrize("zeta", [1, 4, 8])
def test_frsvd_sparse_sign_recovers_planted_spectrum(zeta):
    rng = np.random.default_rng(1)
    n, d = 300, 12
    lam = np.concatenate([np.linspace(50, 20, d) * np.where(np.arange(d) % 3 == 0, -1, 1),
                          rng.uniform(-1, 1, n - d)])
    Q, M = _planted_symmetric(rng, n, lam)
    order = np.argsort(-np.abs(lam))
    out = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, q=8,
                                     oversample=8, seed=5, sketch="sparse_sign", zeta=zeta)
    assert np.count_nonzero(out["Omega"]) == n * zeta
    np.testing.assert_allclose(out["sigma"], np.abs(lam[order[:d]]), rtol=1e-10)
    assert oracle.subspace_sin(out["U"], Q[:, order[:d]]) < 1e-9
