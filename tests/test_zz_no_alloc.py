"""lne_svd_small_noalloc: the small SVD for callers that must not allocate
device memory when they call in. Its scratch is a fixed array in device memory
shared by all calls, so two calls in a row must each give the same result as
the allocating entry point (lne_svd_small). This file is collected last."""
import numpy as np
import pytest
import torch

from paper_2302_07084_gb300 import lne

pytestmark = pytest.mark.gpu


def _triangular(c, cond, seed):
    rng = np.random.default_rng(seed)
    Ua, _ = np.linalg.qr(rng.standard_normal((c, c)))
    Vb, _ = np.linalg.qr(rng.standard_normal((c, c)))
    if cond == "dense_tail":   # a dense tail of singular values: the exact cluster step runs
        s = np.sort(np.concatenate([np.geomspace(1500.0, 100.0, 16), rng.uniform(40.0, 100.0, c - 16)]))[::-1]
    else:
        s = np.geomspace(1.0, 1.0 / cond, c)
    return np.triu(np.linalg.qr((Ua * s) @ Vb.T)[1])


def test_noalloc_small_svd_matches_allocating_entry_point():
    from paper_2302_07084_gb300 import build
    build.build()
    ctx = lne.Context(0)
    try:
        # 144 and 48: the register-resident Jacobi; 33 (odd): its padding
        # column; 151 and 160 (the top of the fixed array): the FP32
        # shared-memory Jacobi taken above 144 columns; a dense tail of
        # singular values: the refinement's exact cluster step
        for c, cond, seed in [(144, 1e4, 1), (48, 1e2, 2), (33, 1e2, 4), (151, 1e3, 3), (160, 1e3, 5),
                              (144, "dense_tail", 0)]:
            R = torch.as_tensor(_triangular(c, cond, seed)).cuda()
            U_ref, s_ref = ctx.svd_small(R)
            U_ref, s_ref = U_ref.cpu().numpy(), s_ref.cpu().numpy()
            for _ in range(2):   # the second call reuses what the first left in the scratch
                U = torch.full((c, c), float("nan"), dtype=torch.float64, device="cuda")
                s = torch.full((c,), float("nan"), dtype=torch.float64, device="cuda")
                assert lne.svd_small_noalloc(R, U, s) == 0
                torch.cuda.synchronize()
                U, s = U.cpu().numpy(), s.cpu().numpy()
                np.testing.assert_allclose(s, s_ref, rtol=1e-12)
                sg = np.sign(np.sum(U * U_ref, axis=0))
                assert np.max(np.abs(U * sg - U_ref)) <= 1e-12
                assert np.max(np.abs(U.T @ U - np.eye(c))) <= 1e-12
        # beyond the scratch's capacity: a clear error, nothing written
        big = torch.zeros((161, 161), dtype=torch.float64, device="cuda")
        out = torch.full((161, 161), 7.0, dtype=torch.float64, device="cuda")
        sig = torch.full((161,), 7.0, dtype=torch.float64, device="cuda")
        assert lne.svd_small_noalloc(big, out, sig) == -1
        torch.cuda.synchronize()
        assert bool((out == 7.0).all()) and bool((sig == 7.0).all())
        # wrong dtype or shape: refused in the binding before any launch
        c = R.shape[0]
        U = torch.empty((c, c), dtype=torch.float64, device="cuda")
        s = torch.empty(c, dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError):
            lne.svd_small_noalloc(R.float(), U, s)
        with pytest.raises(ValueError):
            lne.svd_small_noalloc(R, U[:, : c - 1].contiguous(), s)
        with pytest.raises(ValueError):
            lne.svd_small_noalloc(R, U, s[: c - 1])
    finally:
        ctx.close()
