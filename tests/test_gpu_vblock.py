"""Column-blocked CSR products (LNE_OPT_SPMM_VBLOCK): the columns taken in
vertex blocks [b 2^s, (b + 1) 2^s), each block's partial product added to Y in
block order. Forced to small blocks here so that matrices the oracle handles
in seconds span many blocks, rows that cross warp slices, empty rows and rows
with no entry in some blocks.

Tolerances: the FP32 accumulation bound |dY| <= 1e-5 (|M| |X|) + 1e-6 against
FP64 (the blocked sum order differs from the unblocked one); the randomized
SVD against the oracle at the subspace gate of the other tests."""
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


def _csr_dict(M):
    M = M.tocsr()
    M.sort_indices()   # the blocked path needs columns sorted within rows
    return dict(n=M.shape[0], nnz=M.nnz, indptr=torch.as_tensor(M.indptr.astype(np.int64)).cuda(),
                indices=torch.as_tensor(M.indices.astype(np.int32)).cuda(),
                data=torch.as_tensor(M.data.astype(np.float32)).cuda())


def _matrix(n, seed):
    """Symmetric, a power-law row length mix: hub rows of thousands of
    entries (across many warp slices), rows of a few, and empty rows."""
    rng = np.random.default_rng(seed)
    deg = np.minimum((rng.pareto(1.2, n) + 1) * 3, n // 2).astype(np.int64)
    deg[rng.random(n) < 0.05] = 0
    rows = np.repeat(np.arange(n), deg)
    cols = rng.integers(0, n, rows.size)
    keep = deg[cols] > 0
    A = sp.coo_matrix((rng.random(keep.sum()) + 0.1, (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    A = (A + A.T).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def _check(Y, M, X):
    X64 = X.astype(np.float64)
    ref = M @ X64
    bound = 1e-5 * (abs(M) @ np.abs(X64)) + 1e-6
    err = np.abs(Y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("n,c,shift", [(3000, 144, 6), (3000, 48, 9), (2500, 4, 4), (1024, 128, 7)])
def test_blocked_spmm_matches_fp64(ctx, n, c, shift):
    M = _matrix(n, seed=n + c)
    X = np.random.default_rng(c).standard_normal((n, c)).astype(np.float32)
    Mc = _csr_dict(M)
    ctx.set_option(lne.OPT_SPMM_VBLOCK, shift)
    try:
        Y = to_np(ctx.spmm(Mc, torch.as_tensor(X).cuda()))
        Y2 = to_np(ctx.spmm(Mc, torch.as_tensor(X).cuda()))
    finally:
        ctx.set_option(lne.OPT_SPMM_VBLOCK, 0)
    _check(Y, M, X)
    assert np.array_equal(Y, Y2)   # fixed block order: the same bits every run
    ctx.set_option(lne.OPT_SPMM_VBLOCK, -1)
    try:
        Yu = to_np(ctx.spmm(Mc, torch.as_tensor(X).cuda()))
    finally:
        ctx.set_option(lne.OPT_SPMM_VBLOCK, 0)
    _check(Yu, M, X)


def test_blocked_spmm_bf16_operand(ctx):
    n, c = 3000, 144
    M = _matrix(n, seed=11)
    X = torch.randn((n, c), generator=torch.Generator().manual_seed(3)).to(torch.bfloat16)
    Xf = X.float().numpy()   # the operand values the kernel reads
    ctx.set_option(lne.OPT_SPMM_VBLOCK, 7)
    try:
        Y = to_np(ctx.spmm(_csr_dict(M), X.cuda()))
    finally:
        ctx.set_option(lne.OPT_SPMM_VBLOCK, 0)
    _check(Y, M, Xf)


def test_unsorted_rows_fall_back_unblocked(ctx):
    n, c = 800, 48
    M = _matrix(n, seed=5)
    X = np.random.default_rng(1).standard_normal((n, c)).astype(np.float32)
    # reverse the column order inside every row
    ind = M.indices.copy()
    dat = M.data.copy()
    for i in range(n):
        a, b = M.indptr[i], M.indptr[i + 1]
        ind[a:b] = ind[a:b][::-1]
        dat[a:b] = dat[a:b][::-1]
    Mu = dict(n=n, nnz=M.nnz, indptr=torch.as_tensor(M.indptr.astype(np.int64)).cuda(),
              indices=torch.as_tensor(ind.astype(np.int32)).cuda(), data=torch.as_tensor(dat.astype(np.float32)).cuda())
    ctx.set_option(lne.OPT_SPMM_VBLOCK, 5)
    try:
        Y = to_np(ctx.spmm(Mu, torch.as_tensor(X).cuda()))
    finally:
        ctx.set_option(lne.OPT_SPMM_VBLOCK, 0)
    _check(Y, M, X)


def test_vblock_option_is_validated(ctx):
    for bad in (-2, 31):
        with pytest.raises(lne.LneError):
            ctx.set_option(lne.OPT_SPMM_VBLOCK, bad)


def test_blocked_rsvd_matches_oracle(ctx):
    """The randomized SVD with every product column-blocked (blocks of 256
    vertices) against the oracle."""
    g = synth.sbm(3000, 4, 0.02, 0.002, seed=9)
    spx = oracle.sparsifier(g.indptr, g.indices, 10, np.full(10, 0.1), 40.0 * g.n_arcs, seed=4)
    d, os_, q = 16, 16, 1
    ref = oracle.fast_randomized_svd(spx["indptr"], spx["indices"], spx["data"], d, q, os_, 7)
    p = make_params(1, [1.0], 1.0, d=d, oversample=os_, q=q, seed=7)
    M = sp.csr_matrix((spx["data"], spx["indices"], spx["indptr"]), shape=(g.n, g.n))
    ctx.set_option(lne.OPT_SPMM_VBLOCK, 8)
    try:
        out = ctx.rsvd(_csr_dict(M), p)
    finally:
        ctx.set_option(lne.OPT_SPMM_VBLOCK, 0)
    U = to_np(out["U"]).astype(np.float64)
    assert_subspace(U, ref["U"], lead=4, bound=1e-3, full_bound=1e-3, tag="blocked rsvd")
    np.testing.assert_allclose(to_np(out["sigma"]), ref["sigma"], rtol=1e-4)
