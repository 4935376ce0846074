"""Pins of the oracle's small helpers, each against something other than
itself: brute-force loops on tiny inputs (the CSR product, the symmetric CSR
assembly), invariants (the sign convention, X = U Sigma^{1/2} giving
X^T X = Sigma), and the weighted per-arc rates summing to S."""
import numpy as np
import pytest

import oracle


def _tiny_csr(rng, n, m, density=0.3):
    dense = np.where(rng.random((n, m)) < density, rng.standard_normal((n, m)), 0.0)
    dense[n // 2] = 0.0                          # an empty row
    indptr = [0]
    indices, data = [], []
    for i in range(n):
        for j in range(m):
            if dense[i, j] != 0.0:
                indices.append(j)
                data.append(dense[i, j])
        indptr.append(len(indices))
    return dense, np.array(indptr, np.int64), np.array(indices, np.int32), np.array(data)


def test_spmm_equals_the_brute_force_product():
    rng = np.random.default_rng(1)
    dense, ip, ix, dv = _tiny_csr(rng, 9, 9)
    X = rng.standard_normal((9, 4))
    Y = oracle.spmm(ip, ix, dv, X)
    want = np.zeros((9, 4))
    for i in range(9):
        for j in range(9):
            for c in range(4):
                want[i, c] += dense[i, j] * X[j, c]
    np.testing.assert_allclose(Y, want, rtol=1e-14, atol=1e-14)
    assert np.all(Y[9 // 2] == 0.0)


def test_sparsifier_csr_is_the_symmetric_matrix_of_the_entries():
    rng = np.random.default_rng(2)
    n = 12
    pairs = sorted({(int(a), int(b)) for a, b in rng.integers(0, n, (40, 2)) if a <= b})
    x = np.array([p[0] for p in pairs], np.int64)
    y = np.array([p[1] for p in pairs], np.int64)
    val = rng.random(len(pairs)) + 0.5
    ip, ix, dv = oracle.sparsifier_csr(n, x, y, val)
    dense = np.zeros((n, n))
    for a, b, v in zip(x, y, val):
        dense[a, b] = v
        dense[b, a] = v
    got = np.zeros((n, n))
    for i in range(n):
        row = ix[ip[i]:ip[i + 1]]
        assert np.all(np.diff(row) > 0), "columns strictly increasing within a row"
        got[i, row] = dv[ip[i]:ip[i + 1]]
    np.testing.assert_array_equal(got, dense.astype(np.float32))
    assert ip[-1] == 2 * len(pairs) - int(np.sum(x == y))   # off-diagonal twice, diagonal once


def test_fix_signs_convention():
    U = np.array([[0.1, -0.9, 0.0, 0.5],
                  [-0.7, 0.2, 0.0, -0.5],
                  [0.3, 0.1, 0.0, 0.2]])
    V = np.arange(8.0).reshape(2, 4) + 1.0
    Uf, Vf = oracle.fix_signs(U, V)
    # column 0: largest |entry| -0.7 -> flipped; column 1: -0.9 -> flipped;
    # column 2: all zero -> kept; column 3: tie 0.5 / -0.5, first index wins -> kept
    sg = np.array([-1.0, -1.0, 1.0, 1.0])
    np.testing.assert_array_equal(Uf, U * sg)
    np.testing.assert_array_equal(Vf, V * sg)
    for j in range(4):
        k = int(np.argmax(np.abs(Uf[:, j])))
        assert Uf[k, j] >= 0.0


def test_embedding_from_svd_gives_sigma_as_gram():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((30, 5)))
    sigma = np.array([9.0, 4.0, 2.25, 1.0, 0.25])
    X = oracle.embedding_from_svd(U, sigma)
    np.testing.assert_allclose(X.T @ X, np.diag(sigma), atol=1e-12)
    for j in range(5):
        np.testing.assert_allclose(X[:, j], U[:, j] * np.sqrt(sigma[j]), rtol=1e-15)


@pytest.mark.parametrize("S", [1e3, 12345.678, 2.5e7])
def test_weighted_arc_rates_sum_to_S(S):
    """The per-arc rates S A_a / vol over all arcs add up to S (each split into
    floor and a 2^-32 fraction, so within one unit per arc of rounding)."""
    rng = np.random.default_rng(4)
    w = rng.integers(1, 50, 200)
    vol = float(w.sum())
    total = 0.0
    for a in w:
        base, thr = oracle.arc_rate_w(S, int(a), vol)
        rate = S * a / vol
        assert base == int(np.floor(rate)) or abs(rate - round(rate)) < 1e-9 * max(rate, 1.0)
        assert 0 <= thr < 2 ** 32
        total += base + thr / 2.0 ** 32
    assert abs(total - S) <= len(w) * 2.0 ** -31 + 1e-9 * S
