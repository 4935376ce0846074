"""Downstream objective on the GPU (lne_macro_f1) against the oracle.

The same Newton steps run on both sides; the GPU accumulates margins and
Hessians in FP32 (summed in FP64 across row blocks), so predictions can only
differ at near ties: Macro-F1 must agree within 0.005 and the weights within
1e-3 relative. End to end, each side embeds the graph itself and the two
Macro-F1 values must agree within 0.005 (the plain method's own check).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


def _split(n, seed):
    idx = np.random.default_rng(seed).permutation(n)
    return idx[: n // 2], idx[n // 2:]


@pytest.fixture(scope="module")
def chunglu():
    return synth.chung_lu(3000, 30000, 2.1, seed=9, n_labels=12)


def test_macro_f1_same_input(ctx, chunglu):
    g = chunglu
    ref = oracle.embed(g.indptr, g.indices, 10, np.full(10, 0.1), 50.0 * g.m, 32, 1, 10, 0.5, 0.2, 3)
    X = ref["X"]
    tr, te = _split(g.n, 0)
    ma_ref, mi_ref, W_ref = oracle.macro_f1(X, g.labels, tr, te, C=1.0, iters=10)
    ma, mi = ctx.macro_f1(torch.as_tensor(X.astype(np.float32)).cuda(), torch.as_tensor(g.labels).cuda(),
                          torch.as_tensor(tr).cuda(), torch.as_tensor(te).cuda(), C=1.0, iters=10)
    print(f"macro-F1 oracle {ma_ref:.4f} gpu {ma:.4f}; micro-F1 oracle {mi_ref:.4f} gpu {mi:.4f}")
    assert abs(ma - ma_ref) <= 0.005 and abs(mi - mi_ref) <= 0.005


def test_macro_f1_end_to_end(ctx, chunglu):
    g = chunglu
    s = np.full(10, 0.1)
    p = make_params(10, s, 50.0 * g.m, d=32, q=1, k=10, seed=3)
    X = ctx.embed(lne.DeviceGraph.from_graph(g), p)
    tr, te = _split(g.n, 1)
    ma, mi = ctx.macro_f1(X, torch.as_tensor(g.labels).cuda(), torch.as_tensor(tr).cuda(), torch.as_tensor(te).cuda())
    ref = oracle.embed(g.indptr, g.indices, 10, s, p.samples, 32, 1, 10, 0.5, 0.2, 3)
    ma_ref, mi_ref, _ = oracle.macro_f1(ref["X"], g.labels, tr, te)
    print(f"end-to-end macro-F1 oracle {ma_ref:.4f} gpu {ma:.4f}")
    assert abs(ma - ma_ref) <= 0.005


def test_macro_f1_sbm_blocks(ctx):
    g = synth.sbm(2000, 5, 0.04, 0.002, seed=4)
    X = ctx.embed(lne.DeviceGraph.from_graph(g), make_params(10, np.full(10, 0.1), 50.0 * g.m, d=16, seed=2))
    tr, te = _split(g.n, 2)
    ma, mi = ctx.macro_f1(X, torch.as_tensor(g.labels).cuda(), torch.as_tensor(tr).cuda(), torch.as_tensor(te).cuda())
    assert ma > 0.9 and mi > 0.9


def test_macro_f1_rejects_bad_args(ctx):
    X = torch.zeros((10, 4), device="cuda")
    lab = torch.zeros((10, 2), dtype=torch.uint8, device="cuda")
    idx = torch.arange(5, dtype=torch.int32, device="cuda")
    with pytest.raises(lne.LneError):
        ctx.macro_f1(X, lab, idx, idx, C=-1.0)


def test_macro_f1_rejects_row_index_outside_n(ctx):
    """Row indices outside [0, n) are caught by the gather kernel's own bounds
    check (nothing is read there) and reported as LNE_ERR_INVALID; the context
    stays usable."""
    n, d, L = 40, 4, 2
    gen = torch.Generator().manual_seed(5)
    X = torch.randn((n, d), generator=gen).cuda()
    lab = torch.zeros((n, L), dtype=torch.uint8)
    lab[: n // 2, 0] = 1
    lab[n // 2:, 1] = 1
    lab = lab.cuda()
    good = torch.arange(n, dtype=torch.int32, device="cuda")
    for bad_train, bad_test in ((True, False), (False, True)):
        bad = good.clone()
        bad[3] = n if bad_train else -1
        with pytest.raises(lne.LneError, match="outside"):
            ctx.macro_f1(X, lab, bad if bad_train else good, bad if bad_test else good)
    ma, mi = ctx.macro_f1(X, lab, good, good)
    assert 0.0 <= ma <= 1.0 and 0.0 <= mi <= 1.0
