"""The sparse sign test matrix of the randomized SVD (the alternative to the
Gaussian Omega named in Sec. 4.2; Tropp et al. 2019) on the GPU against the
oracle:

* the matrix itself bit-exact (every +-1 at the oracle's place), including
  zeta = c (every column) and zeta = 1;
* Y = M Omega, never forming Omega: every entry within one FP32 rounding of
  the FP64 product plus 2^-33 per term (64-bit fixed-point sums), and
  bit-identical from run to run;
* Algorithm 4 with this sketch matches the oracle's (sigma, leading subspace),
  and so does the whole method;
* bad sizes are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import assert_subspace, make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


def _csr_dict(indptr, indices, data):
    n = len(indptr) - 1
    return dict(n=n, nnz=len(indices), indptr=torch.as_tensor(np.asarray(indptr, np.int64)).cuda(),
                indices=torch.as_tensor(np.asarray(indices, np.int32)).cuda(),
                data=torch.as_tensor(np.asarray(data, np.float32)).cuda())


@pytest.mark.parametrize("n,c,zeta,seed", [(1000, 48, 8, 3), (777, 144, 12, 4), (50, 5, 5, 5),
                                           (300, 160, 1, 6), (64, 255, 3, 2 ** 40 + 7)])
def test_sketch_bit_exact(ctx, n, c, zeta, seed):
    got = to_np(ctx.sparse_sign_sketch(n, c, zeta, seed)).astype(np.float64)
    ref = oracle.sparse_sign_sketch(n, c, zeta, seed)
    assert np.array_equal(got, ref)


def _random_sparse(n, density, seed, signed=True):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr", dtype=np.float64)
    M.data = (M.data * 8.0 - (4.0 if signed else 0.0)).astype(np.float32).astype(np.float64)
    M.sort_indices()
    return M


def _check_product(ctx, M, c, zeta, seed):
    Y = to_np(ctx.sparse_sign_spmm(_csr_dict(M.indptr, M.indices, M.data), c, zeta, seed)).astype(np.float64)
    Om = oracle.sparse_sign_sketch(M.shape[0], c, zeta, seed)
    ref = oracle.spmm(M.indptr.astype(np.int64), M.indices, M.data, Om)
    terms = np.diff(M.indptr)[:, None] * zeta
    bound = 2.0 ** -24 * np.abs(ref) + terms * 2.0 ** -33 + 1e-30
    assert np.all(np.abs(Y - ref) <= bound)
    return Y


@pytest.mark.parametrize("n,density,c,zeta", [(3000, 0.01, 48, 8), (2000, 0.05, 144, 8), (517, 0.2, 37, 12),
                                              (1200, 0.002, 16, 1)])
def test_product_matches_oracle(ctx, n, density, c, zeta):
    M = _random_sparse(n, density, seed=n)
    Y1 = _check_product(ctx, M, c, zeta, seed=11)
    Y2 = to_np(ctx.sparse_sign_spmm(_csr_dict(M.indptr, M.indices, M.data), c, zeta, 11)).astype(np.float64)
    assert np.array_equal(Y1, Y2)


def test_product_on_sparsifier_with_empty_rows(ctx):
    """The 10k-node SBM sparsifier plus 20 isolated vertices (empty rows)."""
    g = synth.sbm_small()
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 100.0 * g.m, seed=1)
    n = g.n + 20
    indptr = np.concatenate([spx["indptr"], np.full(20, spx["indptr"][-1])])
    M = sp.csr_matrix((spx["data"].astype(np.float64), spx["indices"], indptr), shape=(n, n))
    Y = _check_product(ctx, M, 48, 8, seed=1)
    assert np.all(Y[g.n:] == 0.0)


def test_rsvd_sparse_sign_on_sparsifier(ctx):
    """Algorithm 4 with the sparse sign sketch on the SBM sparsifier (d = 32,
    oversample 16, q = 1) against the oracle's run with the same sketch."""
    g = synth.sbm_small()
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 100.0 * g.m, seed=1)
    ref = oracle.fast_randomized_svd(spx["indptr"], spx["indices"], spx["data"], 32, 1, 16, 1,
                                     sketch="sparse_sign", zeta=8)
    p = make_params(1, [1.0], 1.0, d=32, oversample=16, q=1, seed=1)
    p.sketch = lne.SKETCH_SPARSE_SIGN
    out = ctx.rsvd(_csr_dict(spx["indptr"], spx["indices"], spx["data"]), p)
    np.testing.assert_allclose(to_np(out["sigma"]), ref["sigma"], rtol=1e-4)
    U = to_np(out["U"]).astype(np.float64)
    assert_subspace(U[:, :32], ref["U"][:, :32], tag="sparse-sign rsvd")


@pytest.mark.parametrize("q", [0, 2])
def test_rsvd_sparse_sign_planted(ctx, q):
    rng = np.random.default_rng(q + 10)
    n, d = 600, 16
    lam = np.concatenate([np.geomspace(40, 10, d), rng.uniform(-1, 1, n - d)])
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = sp.csr_matrix(((Qm * lam) @ Qm.T))
    ref = oracle.fast_randomized_svd(M.indptr.astype(np.int64), M.indices, M.data, d, q, 16, 7,
                                     sketch="sparse_sign", zeta=4)
    p = make_params(1, [1.0], 1.0, d=d, oversample=16, q=q, seed=7)
    p.sketch, p.sketch_zeta = lne.SKETCH_SPARSE_SIGN, 4
    out = ctx.rsvd(_csr_dict(M.indptr, M.indices, M.data), p)
    np.testing.assert_allclose(to_np(out["sigma"]), ref["sigma"], rtol=1e-4)
    assert oracle.subspace_sin(to_np(out["U"]).astype(np.float64), ref["U"]) <= 1e-3


def test_embed_sparse_sign_sbm_small(ctx):
    g = synth.sbm_small()
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    p.sketch = lne.SKETCH_SPARSE_SIGN
    ref = oracle.embed(g.indptr, g.indices, 10, p.s, p.samples, 32, 1, 10, 0.5, 0.2, 1, sketch="sparse_sign")
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    assert_subspace(X, ref["X"], tag="sparse-sign embed")


def test_bad_sizes_refused(ctx):
    for n, c, zeta in [(10, 8, 0), (10, 8, 9), (10, 20, 13), (10, 256, 4)]:
        with pytest.raises(lne.LneError) as e:
            ctx.sparse_sign_sketch(n, c, zeta, 1)
        assert e.value.code == -1
    g = synth.sbm(200, 2, 0.1, 0.01, seed=1)
    p = make_params(10, np.ones(10), 10.0 * g.n_arcs, d=16, oversample=8)
    p.sketch, p.sketch_zeta = lne.SKETCH_SPARSE_SIGN, 13
    with pytest.raises(lne.LneError):
        ctx.embed(lne.DeviceGraph.from_graph(g), p)
    p.sketch, p.sketch_zeta = 7, 0
    with pytest.raises(lne.LneError):
        ctx.embed(lne.DeviceGraph.from_graph(g), p)
