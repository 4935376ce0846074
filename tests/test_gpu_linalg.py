"""GPU randomized SVD and spectral propagation against the CPU oracle.

Floating-point tolerances (FP32 kernels vs FP64 oracle):
* sketch: |dz| <= 1e-5 (1 + |z|)  (FP32 Box-Muller of the same Philox words);
* SpMM: |dY| <= 1e-5 (|M| |X|) + 1e-6, the FP32 accumulation bound for rows
  of a few thousand terms;
* CholeskyQR2: ||Q^T Q - I||_max <= 1e-5, ||Y - Q R|| / ||Y|| <= 1e-5;
* randomized SVD: sin(max principal angle) between the GPU and oracle U
  <= 1e-3 (with the oracle's relative spectral gap at d reported), singular
  values within 1e-4 relative;
* propagation (fed the oracle's X0): F and P within 1e-4 of max|.|, X within
  a subspace angle of 1e-3.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import assert_subspace, col_align, make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


def _csr_dict(indptr, indices, data):
    return dict(n=len(indptr) - 1, nnz=len(indices),
                indptr=torch.as_tensor(np.asarray(indptr, np.int64)).cuda(),
                indices=torch.as_tensor(np.asarray(indices, np.int32)).cuda(),
                data=torch.as_tensor(np.asarray(data, np.float32)).cuda())


@pytest.mark.parametrize("n,c", [(1000, 48), (777, 144), (5, 7), (3000, 1)])
def test_sketch_matches_oracle(ctx, n, c):
    Om = to_np(ctx.gaussian_sketch(n, c, seed=123))
    ref = oracle.gaussian_sketch(n, c, seed=123)
    assert np.all(np.abs(Om - ref) <= 1e-5 * (1 + np.abs(ref)))


@pytest.fixture(scope="module")
def sparse_case():
    g = synth.sbm(1500, 3, 0.03, 0.003, seed=6)
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 50.0 * g.n_arcs, seed=5)
    return g, spx


@pytest.mark.parametrize("c", [1, 33, 48, 144, 200])
def test_spmm_matches_fp64(ctx, sparse_case, c):
    g, spx = sparse_case
    X = np.random.default_rng(c).standard_normal((g.n, c)).astype(np.float32)
    Y = to_np(ctx.spmm(_csr_dict(spx["indptr"], spx["indices"], spx["data"]), torch.as_tensor(X).cuda()))
    M = sp.csr_matrix((spx["data"].astype(np.float64), spx["indices"], spx["indptr"]), shape=(g.n, g.n))
    ref = M @ X.astype(np.float64)
    bound = 1e-5 * (abs(M) @ np.abs(X.astype(np.float64))) + 1e-6
    assert np.all(np.abs(Y - ref) <= bound)


@pytest.mark.parametrize("n,c", [(4000, 48), (2048, 144), (300, 128), (200, 200), (17, 16)])
def test_cholqr2(ctx, n, c):
    rng = np.random.default_rng(n + c)
    # a tall matrix with condition number 1e4
    U, _ = np.linalg.qr(rng.standard_normal((n, c)))
    V, _ = np.linalg.qr(rng.standard_normal((c, c)))
    Y = ((U * np.geomspace(1.0, 1e-4, c)) @ V.T).astype(np.float32)
    Q, R = ctx.cholqr2(torch.as_tensor(Y).cuda())
    Q, R = to_np(Q).astype(np.float64), to_np(R)
    assert np.max(np.abs(Q.T @ Q - np.eye(c))) <= 1e-5
    assert np.linalg.norm(Y - Q @ R) / np.linalg.norm(Y) <= 1e-5
    assert np.allclose(np.tril(R, -1), 0.0)


def test_cholqr2_rank_deficient_reports_numeric_error(ctx):
    Y = np.zeros((100, 8), np.float32)
    Y[:, 0] = 1.0
    with pytest.raises(lne.LneError) as e:
        ctx.cholqr2(torch.as_tensor(Y).cuda())
    assert e.value.code == -6


@pytest.mark.parametrize("c,cond", [(144, 1e4), (128, 1e2), (48, 1e6), (16, 10.0), (7, 3.0), (160, 1e3),
                                    (1, 1.0), (2, 5.0), (33, 1e3), (99, 1e5), (130, 1e4), (145, 1e2)])
def test_svd_small_fp64_accuracy(ctx, c, cond):
    """The small SVD is FP64-accurate at any conditioning: singular values to
    1e-12 relative, U orthonormal to 1e-12, U^T R R^T U diagonal to
    1e-12 sigma_1^2 (refinement of the SVD of R itself, no squaring)."""
    rng = np.random.default_rng(c)
    Ua, _ = np.linalg.qr(rng.standard_normal((c, c)))
    Vb, _ = np.linalg.qr(rng.standard_normal((c, c)))
    s = np.geomspace(1.0, 1.0 / cond, c)
    R = np.triu(np.linalg.qr((Ua * s) @ Vb.T)[1])
    U, sig = ctx.svd_small(torch.as_tensor(R).cuda())
    U, sig = to_np(U), to_np(sig)
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.all(np.diff(sig) <= 0)
    np.testing.assert_allclose(sig, ref, rtol=1e-12)
    orth = np.max(np.abs(U.T @ U - np.eye(c)))
    assert orth <= 1e-12, orth
    B = U.T @ R @ R.T @ U
    off = B - np.diag(np.diag(B))
    assert np.max(np.abs(off)) <= 1e-12 * ref[0] ** 2, np.max(np.abs(off)) / ref[0] ** 2


def _spectrum_case(kind, c, seed):
    """Upper-triangular factors whose spectra have the structure of a
    randomized SVD's factor on a NetMF matrix: a few large values over a dense
    tail (relative gaps down to 1e-6), or tight clusters."""
    rng = np.random.default_rng(seed)
    if kind == "dense_tail":
        s = np.concatenate([np.geomspace(1500.0, 100.0, 16), rng.uniform(40.0, 100.0, c - 16)])
    elif kind == "cluster":   # half the values within 1e-3 of one another
        s = np.concatenate([np.geomspace(10.0, 2.0, c // 2), 1.0 + 1e-3 * rng.random(c - c // 2)])
    else:                     # equal values in three groups, some within 1e-9
        s = np.repeat([3.0, 2.0, 1.0], c // 3 + 1)[:c] * (1.0 + 1e-9 * rng.random(c))
    s = np.sort(s)[::-1]
    Ua, _ = np.linalg.qr(rng.standard_normal((c, c)))
    Vb, _ = np.linalg.qr(rng.standard_normal((c, c)))
    return np.triu(np.linalg.qr((Ua * s) @ Vb.T)[1])


@pytest.mark.parametrize("kind,c,seed", [("dense_tail", 144, 0), ("dense_tail", 144, 2), ("dense_tail", 128, 0),
                                         ("dense_tail", 160, 1), ("cluster", 64, 1), ("cluster", 144, 3),
                                         ("groups", 48, 4)])
def test_svd_small_dense_and_clustered_spectra(ctx, kind, c, seed):
    """The same FP64 bar where singular values are dense or clustered: the
    first-order refinement steps are guarded by each pair's relative gap, and
    the pairs they leave are resolved by the exact FP64 two-sided Jacobi on
    T = U^T R V."""
    R = _spectrum_case(kind, c, seed)
    U, sig = ctx.svd_small(torch.as_tensor(R).cuda())
    U, sig = to_np(U), to_np(sig)
    ref = np.linalg.svd(R, compute_uv=False)
    assert np.all(np.diff(sig) <= 0)
    np.testing.assert_allclose(sig, ref, rtol=1e-12)
    orth = np.max(np.abs(U.T @ U - np.eye(c)))
    assert orth <= 1e-12, orth
    B = U.T @ R @ R.T @ U
    off = B - np.diag(np.diag(B))
    assert np.max(np.abs(off)) <= 1e-12 * ref[0] ** 2, np.max(np.abs(off)) / ref[0] ** 2


def _rsvd_compare(ctx, indptr, indices, data, d, p_os, q, seed):
    ref = oracle.fast_randomized_svd(indptr, indices, data, d, q, p_os, seed)
    p = make_params(1, [1.0], 1.0, d=d, oversample=p_os, q=q, seed=seed)
    out = ctx.rsvd(_csr_dict(indptr, indices, data), p)
    U = to_np(out["U"]).astype(np.float64)
    sig = to_np(out["sigma"])
    gap = (ref["sigma_all"][d - 1] - ref["sigma_all"][d]) / ref["sigma_all"][d - 1]
    ang = oracle.subspace_sin(U, ref["U"])
    return U, sig, ref, gap, ang, out


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_matches_oracle_planted(ctx, q):
    rng = np.random.default_rng(q)
    n, d = 600, 16
    lam = np.concatenate([np.geomspace(40, 10, d), rng.uniform(-1, 1, n - d)])
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = sp.csr_matrix(((Qm * lam) @ Qm.T))
    U, sig, ref, gap, ang, out = _rsvd_compare(ctx, M.indptr.astype(np.int64), M.indices, M.data, d, 16, q, 7)
    assert ang <= 1e-3, (ang, gap)
    np.testing.assert_allclose(sig, ref["sigma"], rtol=1e-4)
    X0 = oracle.embedding_from_svd(ref["U"], ref["sigma"])
    assert np.max(np.abs(col_align(to_np(out["X0"]), X0) - X0)) <= 1e-3 * np.abs(X0).max()
    # columns orthonormal, sign convention honoured
    assert np.max(np.abs(U.T @ U - np.eye(d))) <= 1e-5
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(d)] > 0)


def test_rsvd_on_sparsifier_workload(ctx):
    """SBM sparsifier (10k nodes, S = 10 T m), d = 32, oversample 16, q = 1."""
    g = synth.sbm_small()
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 100.0 * g.m, seed=1)
    U, sig, ref, gap, ang, out = _rsvd_compare(ctx, spx["indptr"], spx["indices"], spx["data"], 32, 16, 1, 1)
    print(f"sbm10k rsvd: sin angle {ang:.3e}, relative gap at d {gap:.3e}")
    np.testing.assert_allclose(sig, ref["sigma"], rtol=1e-4)
    # the leading columns (with a gap to the rest) agree to the gate
    k = 4   # the four block directions
    assert_subspace(U, ref["U"], k, tag="sbm10k rsvd")


@pytest.mark.parametrize("k,theta,mu", [(10, 0.5, 0.2), (1, 0.5, 0.2), (2, 0.7, 0.4), (15, 0.3, 0.5), (0, 0.5, 0.2)])
def test_propagation_matches_oracle(ctx, k, theta, mu):
    g = synth.sbm(2000, 4, 0.02, 0.002, seed=8)
    d = 32
    X0 = np.random.default_rng(1).standard_normal((g.n, d))
    ref = oracle.spectral_propagation(g.indptr, g.indices, X0, k, theta, mu)
    p = make_params(1, [1.0], 1.0, d=d, k=k, theta=theta, mu=mu)
    out = ctx.propagate(lne.DeviceGraph.from_graph(g), p, torch.as_tensor(X0.astype(np.float32)).cuda(),
                        want_intermediates=True)
    X = to_np(out["X"]).astype(np.float64)
    if k == 0:
        np.testing.assert_array_equal(X, X0.astype(np.float32))
        return
    F, P = to_np(out["F"]), to_np(out["P"])
    assert np.max(np.abs(F - ref["F"])) <= 1e-4 * np.abs(ref["F"]).max()
    assert np.max(np.abs(P - ref["P"])) <= 1e-4 * np.abs(ref["P"]).max()
    assert oracle.subspace_sin(X, ref["X"]) <= 1e-3


def test_propagation_isolated_vertices(ctx):
    g0 = synth.sbm(500, 2, 0.05, 0.005, seed=3)
    indptr = np.concatenate([g0.indptr, np.full(4, g0.indptr[-1])])
    g = synth.Graph(504, indptr, g0.indices, None, "iso")
    X0 = np.random.default_rng(2).standard_normal((g.n, 16))
    ref = oracle.spectral_propagation(g.indptr, g.indices, X0, 10, 0.5, 0.2)
    out = ctx.propagate(lne.DeviceGraph.from_graph(g), make_params(1, [1.0], 1.0, d=16, k=10),
                        torch.as_tensor(X0.astype(np.float32)).cuda(), want_intermediates=True)
    P = to_np(out["P"])
    assert np.all(P[500:] == 0)
    assert np.max(np.abs(P - ref["P"])) <= 1e-4 * np.abs(ref["P"]).max()


def test_embed_end_to_end_sbm_small(ctx):
    """Whole method on the 10k-node SBM workload against the oracle."""
    g = synth.sbm_small()
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    ref = oracle.embed(g.indptr, g.indices, 10, p.s, p.samples, 32, 1, 10, 0.5, 0.2, 1)
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    ang = oracle.subspace_sin(X, ref["X"])
    print(f"sbm10k embed: sin angle {ang:.3e}")
    # the planted block structure is recovered identically
    y = np.argmax(g.labels, axis=1)
    def acc(E):
        idx = np.random.default_rng(0).permutation(g.n)
        tr, te = idx[: g.n // 2], idx[g.n // 2:]
        Ea = np.hstack([E, np.ones((g.n, 1))])
        W, *_ = np.linalg.lstsq(Ea[tr], np.eye(4)[y[tr]], rcond=None)
        return np.mean(np.argmax(Ea[te] @ W, 1) == y[te])
    assert abs(acc(X) - acc(ref["X"])) <= 0.005
    assert_subspace(X, ref["X"], tag="sbm10k embed")


def test_embed_rejects_bad_sizes(ctx):
    g = synth.sbm(60, 2, 0.3, 0.05, seed=1)
    p = make_params(10, np.ones(10), 10.0 * g.n_arcs, d=50, oversample=16)
    with pytest.raises(lne.LneError) as e:
        ctx.embed(lne.DeviceGraph.from_graph(g), p)
    assert e.value.code == -1
