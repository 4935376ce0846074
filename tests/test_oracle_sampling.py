"""Pins of the CPU oracle's sampling stage against facts fixed by the paper and
by probability, not against the oracle itself.

* Philox4x32-10 against the published known-answer vectors.
* The window length r follows Multinomial(s) (Algorithm 3), the split is
  uniform on [0, r-1] (Algorithm 1), n_e = floor(S/2m) + Bernoulli (Alg. 3).
* T = 1 (the LINE special case of Eq. 1): every sample returns its own arc.
* Endpoint law: u' ~ row u of P^sigma, v' ~ row v of P^(r-1-sigma),
  independently (Algorithm 1 with P = D^-1 A).
* Expectation: the counts estimate S/vol * sum_r s_r D P^r, and the Eq. 1
  scaling applied to the exact expectation reproduces the dense NetMF matrix.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats as st

import oracle
from paper_2302_07084_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert list(map(int, out)) == r[6:10]


def test_window_thresholds_closed_form():
    thr = oracle.window_thresholds([0.25, 0.25, 0.25, 0.25])
    assert list(map(int, thr)) == [1 << 30, 1 << 31, 3 << 30]
    # all weight on r = 1: no word reaches a threshold of 2^32
    assert list(map(int, oracle.window_thresholds([1.0, 0.0, 0.0]))) == [1 << 32, 1 << 32]
    # all weight on r = T: every word passes a threshold of 0
    assert list(map(int, oracle.window_thresholds([0.0, 0.0, 2.0]))) == [0, 0]
    # unnormalised weights are normalised
    assert list(map(int, oracle.window_thresholds([2.0, 2.0]))) == [1 << 31]


def test_arc_rate_closed_form():
    assert oracle.arc_rate(1000.0, 10) == (100, 0)
    assert oracle.arc_rate(125.0, 10) == (12, 1 << 31)
    assert oracle.arc_rate(3.0, 4) == (0, 3 << 30)


@pytest.fixture(scope="module")
def small_graph():
    return synth.sbm(300, 3, 0.08, 0.01, seed=5)


def test_samples_per_arc(small_graph):
    g = small_graph
    S = 12.5 * g.n_arcs
    na = oracle.arc_samples(g.n_arcs, S, seed=7)
    assert set(np.unique(na)) <= {12, 13}
    # mean 12.5: Binomial(n_arcs, 1/2) extra samples
    extra = int((na - 12).sum())
    z = (extra - g.n_arcs / 2) / np.sqrt(g.n_arcs / 4)
    assert abs(z) < 5
    assert oracle.count_samples(g.n_arcs, S, 7) == int(na.sum())
    # arc ranges partition the total
    h = g.n_arcs // 3
    assert (oracle.count_samples(g.n_arcs, S, 7, 0, h) + oracle.count_samples(g.n_arcs, S, 7, h, g.n_arcs)
            == int(na.sum()))


def test_window_and_split_laws(small_graph):
    g = small_graph
    T = 10
    s = synth.dirichlet_weights(T, seed=3)
    tr = oracle.sample_trace(g.indptr, g.indices, T, s, 40.0 * g.n_arcs, seed=11)
    N = tr["r"].size
    obs = np.bincount(tr["r"], minlength=T + 1)[1:]
    exp = s / s.sum() * N
    keep = exp > 5
    chi = st.chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum())
    assert chi.pvalue > 1e-4
    for r in range(2, T + 1):
        sig = tr["sigma"][tr["r"] == r]
        if sig.size < 50 * r:
            continue
        cnt = np.bincount(sig, minlength=r)
        assert cnt.size == r
        assert st.chisquare(cnt).pvalue > 1e-4


def test_T1_returns_own_arc(small_graph):
    g = small_graph
    S = 5.0 * g.n_arcs            # integer rate: exactly 5 samples per arc
    tr = oracle.sample_trace(g.indptr, g.indices, 1, [1.0], S, seed=2)
    assert np.all(tr["r"] == 1) and np.all(tr["sigma"] == 0)
    src = np.repeat(np.arange(g.n), np.diff(g.indptr))
    assert np.array_equal(tr["u1"], np.repeat(src, 5))
    assert np.array_equal(tr["v1"], np.repeat(g.indices.astype(np.int64), 5))
    x, y, cnt = oracle.sparsifier_counts(g.indptr, g.indices, 1, [1.0], S, seed=2)
    # every edge {u, v} is counted n_{u->v} + n_{v->u} = 10 times, nothing else
    assert np.all(cnt == 10)
    assert x.size == g.m
    A = sp.csr_matrix((np.ones(g.n_arcs), g.indices, g.indptr), shape=(g.n, g.n))
    assert np.all(np.asarray(A[x, y]).ravel() == 1)


def test_chunked_dense_counts_T1_closed_form(small_graph):
    """The chunked dense-table count (for sample counts too large to hold at
    once): with T = 1 every edge is counted exactly n_{u->v} + n_{v->u} times,
    however the arcs are split into chunks."""
    g = small_graph
    S = 5.0 * g.n_arcs
    x, y, cnt = oracle.sparsifier_counts_dense(g.indptr, g.indices, 1, [1.0], S, seed=2,
                                               chunk_samples=7 * 5)   # 7 arcs per chunk
    assert np.all(cnt == 10) and x.size == g.m
    assert np.all(x <= y) and np.all(np.diff(x * g.n + y) > 0)
    A = sp.csr_matrix((np.ones(g.n_arcs), g.indices, g.indptr), shape=(g.n, g.n))
    assert np.all(np.asarray(A[x, y]).ravel() == 1)


def test_chunked_dense_counts_match_exact_expectation():
    """The chunked count against the exact expectation S/vol sum_r s_r D P^r
    (z-scores), with a chunk size that splits the arcs unevenly."""
    g = synth.lollipop_tiny()
    T = 5
    s = [0.1, 0.3, 0.2, 0.25, 0.15]
    S = 20000.0 * g.n_arcs
    x, y, cnt = oracle.sparsifier_counts_dense(g.indptr, g.indices, T, s, S, seed=23, chunk_samples=3 * 20000.0)
    K = np.zeros((g.n, g.n))
    K[x, y] = cnt
    EK = _expected_counts(g, T, s, S)
    iu = np.triu_indices(g.n)
    assert np.all(K[iu][EK[iu] == 0] == 0)
    m = EK[iu] > 0
    z = (K[iu][m] - EK[iu][m]) / np.sqrt(EK[iu][m])
    assert np.max(np.abs(z)) < 6
    assert int(cnt.sum()) == oracle.count_samples(g.n_arcs, S, 23)


def _dense_P(g):
    A = sp.csr_matrix((np.ones(g.n_arcs), g.indices, g.indptr), shape=(g.n, g.n)).toarray()
    d = A.sum(1)
    return A, d, A / d[:, None]


def test_endpoint_law_exhaustive_tiny():
    g = synth.lollipop_tiny()
    A, d, P = _dense_P(g)
    T = 6
    s = np.ones(T)
    tr = oracle.sample_trace(g.indptr, g.indices, T, s, 30000.0 * g.n_arcs, seed=19)
    src = np.repeat(np.arange(g.n), np.diff(g.indptr))
    checked = 0
    for a in [0, 5, 9, 15]:
        u, v = src[a], g.indices[a]
        for r in range(1, T + 1):
            for sig in range(r):
                sel = (tr["arc"] == a) & (tr["r"] == r) & (tr["sigma"] == sig)
                if sel.sum() < 300:
                    continue
                pu = np.linalg.matrix_power(P, sig)[u]
                pv = np.linalg.matrix_power(P, r - 1 - sig)[v]
                joint = np.outer(pu, pv).ravel()
                obs = np.bincount(tr["u1"][sel] * g.n + tr["v1"][sel], minlength=g.n * g.n)
                # impossible endpoints never occur
                assert obs[joint == 0].sum() == 0
                nz = joint > 0
                e = joint[nz] * sel.sum()
                if nz.sum() == 1:
                    assert obs[nz][0] == sel.sum()
                elif e.min() >= 5:
                    assert st.chisquare(obs[nz], e).pvalue > 1e-5
                else:
                    # pooled test on the marginals when cells are small
                    ou = np.bincount(tr["u1"][sel], minlength=g.n)
                    m = pu > 0
                    assert st.chisquare(ou[m], pu[m] * sel.sum()).pvalue > 1e-5
                checked += 1
    assert checked >= 20


def _expected_counts(g, T, s, S):
    """E[K_xy] for the unordered counts (x <= y) from the exact law."""
    A, d, P = _dense_P(g)
    s = np.asarray(s, float) / np.sum(s)
    acc = np.zeros((g.n, g.n))
    Pr = np.eye(g.n)
    for r in range(1, T + 1):
        Pr = Pr @ P
        acc += s[r - 1] * (d[:, None] * Pr)          # D P^r
    EC = S / d.sum() * acc                            # E[ordered count C_xy]
    EK = EC + EC.T
    EK[np.diag_indices(g.n)] = np.diag(EC)
    return EK


def test_counts_match_exact_expectation():
    g = synth.lollipop_tiny()
    T = 5
    s = [0.1, 0.3, 0.2, 0.25, 0.15]
    S = 20000.0 * g.n_arcs
    x, y, cnt = oracle.sparsifier_counts(g.indptr, g.indices, T, s, S, seed=23)
    K = np.zeros((g.n, g.n))
    K[x, y] = cnt
    EK = _expected_counts(g, T, s, S)
    iu = np.triu_indices(g.n)
    assert np.all(K[iu][EK[iu] == 0] == 0)
    m = EK[iu] > 0
    z = (K[iu][m] - EK[iu][m]) / np.sqrt(EK[iu][m])
    assert np.max(np.abs(z)) < 6
    # total equals the number of samples drawn
    assert int(cnt.sum()) == oracle.count_samples(g.n_arcs, S, 23)


def test_eq1_scaling_reproduces_dense_netmf():
    g = synth.sbm(40, 2, 0.4, 0.1, seed=8)
    T = 4
    s = [0.4, 0.3, 0.2, 0.1]
    S = 1.0e6
    EK = _expected_counts(g, T, s, S)
    iu = np.triu_indices(g.n)
    x, y = iu[0], iu[1]
    v, keep, val = oracle.netmf_values(x, y, EK[iu], g.degrees(), S, b=1.0)
    W = oracle.netmf_dense(g.indptr, g.indices, T, s, b=1.0)
    np.testing.assert_allclose(v, W[iu], rtol=1e-12, atol=1e-14)
    # trunc_log of Eq. 1: max(0, log W), zero entries dropped
    assert np.array_equal(keep, W[iu] > 1.0)
    np.testing.assert_allclose(val[keep], np.log(W[iu][keep]), rtol=2e-7)
    # b scales the whole matrix by 1/b
    v2, _, _ = oracle.netmf_values(x, y, EK[iu], g.degrees(), S, b=2.0)
    np.testing.assert_allclose(v2, W[iu] / 2.0, rtol=1e-12, atol=1e-14)


def test_netmf_dense_T1_is_line_matrix():
    g = synth.lollipop_tiny()
    A, d, P = _dense_P(g)
    W = oracle.netmf_dense(g.indptr, g.indices, 1, [1.0])
    np.testing.assert_allclose(W, d.sum() * A / np.outer(d, d), rtol=1e-14)


def test_sparsifier_csr_structure():
    g = synth.sbm(200, 2, 0.1, 0.02, seed=4)
    sp_ = oracle.sparsifier(g.indptr, g.indices, 10, np.ones(10), 50.0 * g.n_arcs, seed=3)
    n = g.n
    M = sp.csr_matrix((sp_["data"], sp_["indices"], sp_["indptr"]), shape=(n, n))
    assert abs(M - M.T).max() == 0
    for i in range(n):
        cols = sp_["indices"][sp_["indptr"][i]:sp_["indptr"][i + 1]]
        assert np.all(np.diff(cols) > 0)
    assert np.all(sp_["data"] > 0)
    # diagonal entries appear once, off-diagonal ones twice
    keep = sp_["keep"]
    ndiag = int((sp_["x"][keep] == sp_["y"][keep]).sum())
    assert M.nnz == 2 * int(keep.sum()) - ndiag


# ----------------------------------------------------------------------------
# edge downsampling (Sec. 4.1; Algorithm 3)
# ----------------------------------------------------------------------------

def _star_path():
    """0 -- 1, 2, 3, 4 and 1 -- 2: degrees 4, 2, 2, 1, 1."""
    e = [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2)]
    u = np.array([a for a, b in e])
    v = np.array([b for a, b in e])
    indptr, indices = synth.csr_from_edges(5, u, v)
    return indptr, indices


def test_downsample_rule_closed_form():
    indptr, indices = _star_path()
    thr, w = oracle.arc_downsample(indptr, indices, 0.5)
    arcs = {(int(a), int(indices[k])): k for a in range(5) for k in range(indptr[a], indptr[a + 1])}
    # arc 0 -> 1: p = 0.5 (1/4 + 1/2) = 0.375
    k = arcs[(0, 1)]
    assert thr[k] == int(0.375 * 2 ** 32) == 1610612736
    assert w[k] == 11453246123            # floor(2^32 / 0.375 + 1/2) = floor(11453246122.67 + 0.5)
    # arc 3 -> 0: p = 0.5 (1 + 1/4) = 0.625
    k = arcs[(3, 0)]
    assert thr[k] == 2684354560 and w[k] == 6871947674
    # C = 2: p = min(1, 2 * 0.75) = 1 -> the coin always keeps, weight exactly 1
    thr, w = oracle.arc_downsample(indptr, indices, 2.0)
    k = arcs[(0, 1)]
    assert thr[k] == 2 ** 32 and w[k] == 2 ** 32


def test_downsampling_with_certain_coins_is_the_plain_count():
    g = synth.sbm(600, 3, 0.05, 0.005, seed=3)
    s = np.full(10, 0.1)
    x, y, c = oracle.sparsifier_counts(g.indptr, g.indices, 10, s, 4.0 * g.n_arcs, 7)
    xw, yw, w = oracle.sparsifier_counts(g.indptr, g.indices, 10, s, 4.0 * g.n_arcs, 7, C=1e6)
    assert np.array_equal(x, xw) and np.array_equal(y, yw)
    assert np.array_equal(w, c.astype(np.uint64) * np.uint64(2 ** 32))


def test_downsampled_counts_are_unbiased():
    """Theorem 1's reweighting: E[sum of 1/p_e over kept draws] = E[count]."""
    g = synth.lollipop_tiny()
    T = 5
    s = [0.1, 0.3, 0.2, 0.25, 0.15]
    S = 20000.0 * g.n_arcs
    C = 0.5
    thr, wts = oracle.arc_downsample(g.indptr, g.indices, C)
    assert np.all(thr < 2 ** 32)             # every arc is really downsampled here
    x, y, w = oracle.sparsifier_counts(g.indptr, g.indices, T, s, S, seed=31, C=C)
    K = np.zeros((g.n, g.n))
    K[x, y] = w.astype(np.float64) * 2.0 ** -32
    EK = _expected_counts(g, T, s, S)
    iu = np.triu_indices(g.n)
    assert np.all(K[iu][EK[iu] == 0] == 0)
    m = EK[iu] > 0
    wmax = float(wts.max()) * 2.0 ** -32      # a draw adds at most 1/min p_e
    z = (K[iu][m] - EK[iu][m]) / np.sqrt(EK[iu][m] * wmax)
    assert np.max(np.abs(z)) < 6


def test_kept_draws_follow_the_coin_law():
    g = synth.sbm(400, 2, 0.06, 0.01, seed=5)
    S = 30.0 * g.n_arcs
    C = 2.0
    tr = oracle.sample_trace(g.indptr, g.indices, 4, [0.25] * 4, S, 9, fields=("arc", "coin"))
    thr, _ = oracle.arc_downsample(g.indptr, g.indices, C)
    p = thr[tr["arc"]].astype(np.float64) / 2.0 ** 32
    kept = tr["coin"].astype(np.uint64) < thr[tr["arc"]]
    z = (kept.sum() - p.sum()) / np.sqrt(np.sum(p * (1 - p)))
    assert abs(z) < 5 and 0 < kept.sum() < len(kept)


# window-stratified counts (one sampling pass shared by many weightings s)

def test_stratified_weights_closed_form():
    w = oracle.stratified_weights([1.0, 1.0, 2.0], 3)
    assert w.tolist() == [round(3 * 0.25 * 2 ** 24), round(3 * 0.25 * 2 ** 24), round(3 * 0.5 * 2 ** 24)]
    assert oracle.stratified_weights(np.ones(10), 10).tolist() == [2 ** 24] * 10
    assert oracle.stratified_weights([0.0, 1.0], 2).tolist() == [0, 2 ** 25]


def test_stratified_uniform_s_is_the_plain_count():
    """With s uniform every weight is exactly 2^24: K = 2^24 x the count of
    the plain sampler with uniform s."""
    g = synth.sbm(300, 3, 0.06, 0.01, seed=2)
    T, S = 6, 30.0 * g.n_arcs
    x, y, r, c = oracle.stratified_counts(g.indptr, g.indices, T, S, 8)
    assert np.all((r >= 1) & (r <= T))
    px, py, K = oracle.stratified_estimate(x, y, r, c, np.ones(T), T)
    qx, qy, qc = oracle.sparsifier_counts(g.indptr, g.indices, T, np.ones(T), S, 8)
    assert np.array_equal(px, qx) and np.array_equal(py, qy)
    assert np.array_equal(K, qc.astype(np.uint64) << np.uint64(24))
    assert int(c.sum()) == oracle.count_samples(g.n_arcs, S, 8)


def test_stratified_estimate_is_unbiased():
    """E[K_s] = S / vol sum_r s~_r [D P^r] (unordered) with s~_r = w_r 2^-24 / T,
    for a weighting far from uniform; z-scores against the exact law with the
    variance sum_r (w_r 2^-24)^2 E[C_r]."""
    g = synth.lollipop_tiny()
    T = 5
    s = [0.05, 0.6, 0.0, 0.3, 0.05]
    S = 40000.0 * g.n_arcs
    x, y, r, c = oracle.stratified_counts(g.indptr, g.indices, T, S, 31)
    px, py, K = oracle.stratified_estimate(x, y, r, c, s, T)
    w = oracle.stratified_weights(s, T).astype(np.float64) * 2.0 ** -24
    EK = np.zeros((g.n, g.n))
    VK = np.zeros((g.n, g.n))
    for rr in range(1, T + 1):
        e = np.zeros(T)
        e[rr - 1] = 1.0
        Er = _expected_counts(g, T, e, S / T)      # E[C_r] (unordered)
        EK += w[rr - 1] * Er
        VK += w[rr - 1] ** 2 * Er
    Kd = np.zeros((g.n, g.n))
    Kd[px, py] = K.astype(np.float64) * 2.0 ** -24
    iu = np.triu_indices(g.n)
    m = VK[iu] > 0
    z = (Kd[iu][m] - EK[iu][m]) / np.sqrt(VK[iu][m])
    assert np.max(np.abs(z)) < 6
    assert np.all(Kd[iu][~m] == 0)
    # the expectation is the plain sampler's with weights s~ (= s up to rounding)
    np.testing.assert_allclose(EK[iu], _expected_counts(g, T, s, S)[iu], rtol=1e-6, atol=1e-9)


def test_stratified_sparsifier_structure():
    g = synth.sbm(300, 3, 0.06, 0.01, seed=2)
    T, S = 6, 30.0 * g.n_arcs
    sp = oracle.stratified_sparsifier(g.indptr, g.indices, T, [0.5, 0.1, 0.1, 0.1, 0.1, 0.1], S, 8)
    # the keep rule of Eq. 1 on K = K_s 2^-24
    deg = np.diff(g.indptr).astype(np.float64)
    a_off, a_diag = oracle.netmf_scale(deg.sum(), S)
    alpha = np.where(sp["x"] == sp["y"], a_diag, a_off)
    v = (sp["K"].astype(np.float64) * 2.0 ** -24 * alpha) / (deg[sp["x"]] * deg[sp["y"]])
    assert np.array_equal(sp["keep"], v > 1.0)
    n = g.n
    M = np.zeros((n, n))
    for i in range(n):
        M[i, sp["indices"][sp["indptr"][i]:sp["indptr"][i + 1]]] = sp["data"][sp["indptr"][i]:sp["indptr"][i + 1]]
    np.testing.assert_array_equal(M, M.T)
