"""The very sparse random projection (the other cheaper Omega of Algorithm 4
that Sec. 4.2 names; Li, Hastie and Church 2006, at scale 1) on the GPU
against the oracle:

* the matrix itself bit-exact (every +-1 at the oracle's place) for s = sqrt(n)
  and for a denser s;
* Y = M Omega, never forming Omega: every entry within one FP32 rounding of
  the FP64 product plus 2^-33 per term, bit-identical from run to run, rows of
  Omega without nonzeros giving exact zeros;
* Algorithm 4 with this sketch matches the oracle's (sigma, subspace), and so
  does the whole method;
* rows with more than 12 nonzeros and s < 1 are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import assert_subspace, full_span_bound, make_params, to_np

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


@pytest.mark.parametrize("n,c,s,seed", [(10000, 48, 0.0, 3), (4000, 144, 0.0, 4), (500, 37, 20.0, 5),
                                        (2000, 160, 0.0, 2 ** 40 + 7)])
def test_sketch_bit_exact(ctx, n, c, s, seed):
    got = to_np(ctx.very_sparse_sketch(n, c, s, seed)).astype(np.float64)
    ref = oracle.very_sparse_sketch(n, c, s, seed)
    assert np.array_equal(got, ref)
    assert (ref == 0).all(axis=1).any()   # rows without any nonzero occur at these sizes


def _random_sparse(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr", dtype=np.float64)
    M.data = (M.data * 8.0 - 4.0).astype(np.float32).astype(np.float64)
    M.sort_indices()
    return M


@pytest.mark.parametrize("n,density,c,s", [(3000, 0.01, 48, 0.0), (2000, 0.05, 144, 0.0), (517, 0.2, 37, 10.0)])
def test_product_matches_oracle(ctx, n, density, c, s):
    M = _random_sparse(n, density, seed=n)
    csr = _csr_dict(M.indptr, M.indices, M.data)
    Y = to_np(ctx.very_sparse_spmm(csr, c, s, 11)).astype(np.float64)
    Om = oracle.very_sparse_sketch(n, c, s, 11)
    ref = oracle.spmm(M.indptr.astype(np.int64), M.indices, M.data, Om)
    terms = np.diff(M.indptr)[:, None] * (Om != 0).sum(axis=1).max()
    bound = 2.0 ** -24 * np.abs(ref) + terms * 2.0 ** -33 + 1e-30
    assert np.all(np.abs(Y - ref) <= bound)
    Y2 = to_np(ctx.very_sparse_spmm(csr, c, s, 11)).astype(np.float64)
    assert np.array_equal(Y, Y2)


def test_rsvd_very_sparse_on_sparsifier(ctx):
    """Algorithm 4 with the very sparse sketch (s = sqrt(n)) on the SBM
    sparsifier (d = 32, oversample 16, q = 1) against the oracle's run with
    the same sketch."""
    g = synth.sbm_small()
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 100.0 * g.m, seed=1)
    ref = oracle.fast_randomized_svd(spx["indptr"], spx["indices"], spx["data"], 32, 1, 16, 1,
                                     sketch="very_sparse", sparsity=0.0)
    p = make_params(1, [1.0], 1.0, d=32, oversample=16, q=1, seed=1)
    p.sketch = lne.SKETCH_VERY_SPARSE
    out = ctx.rsvd(_csr_dict(spx["indptr"], spx["indices"], spx["data"]), p)
    np.testing.assert_allclose(to_np(out["sigma"]), ref["sigma"], rtol=1e-4)
    bound, gap = full_span_bound(ref["sigma_all"], 32)
    assert_subspace(to_np(out["U"]).astype(np.float64), ref["U"], full_bound=bound, tag="very-sparse rsvd")


def test_embed_very_sparse_sbm_small(ctx):
    g = synth.sbm_small()
    p = make_params(10, np.full(10, 0.1), 100.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=1)
    p.sketch, p.sketch_zeta = lne.SKETCH_VERY_SPARSE, 0
    ref = oracle.embed(g.indptr, g.indices, 10, p.s, p.samples, 32, 1, 10, 0.5, 0.2, 1, sketch="very_sparse")
    X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
    bound, gap = full_span_bound(ref["rsvd"]["sigma_all"], 32)
    assert_subspace(X, ref["X"], full_bound=bound, tag="very-sparse embed")


def test_refusals(ctx):
    # s = 1: every entry is +-1, so rows of 20 columns exceed 12 nonzeros
    with pytest.raises(lne.LneError) as e:
        ctx.very_sparse_sketch(50, 20, 1.0, 1)
    assert e.value.code == -5
    with pytest.raises(lne.LneError) as e:
        ctx.very_sparse_sketch(50, 20, 0.5, 1)
    assert e.value.code == -1
    with pytest.raises(lne.LneError) as e:
        ctx.very_sparse_sketch(50, 256, 0.0, 1)
    assert e.value.code == -1
    # the context stays usable after the refusal
    got = to_np(ctx.very_sparse_sketch(400, 20, 0.0, 2)).astype(np.float64)
    assert np.array_equal(got, oracle.very_sparse_sketch(400, 20, 0.0, 2))
