"""Precision plan: error against the FP64 oracle, stage by stage, for the FP32
path and for the BF16-operand path (LNE_PREC_BF16_MIXED: the dense operand of
every sparse product is gathered as bfloat16, accumulation stays FP32, the
Gram / Cholesky / small SVD stay FP64).

Bounds: bfloat16 keeps 8 significant bits (7 stored), so a rounded operand
carries a relative error of at most u = 2^-8 (round to nearest); a product of
FP32 accumulations of such operands stays within a few u in norm. The subspace and
singular-value bounds are set from the leading, well-separated directions.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth
from gpu_common import col_align, make_params, to_np

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def case():
    g = synth.sbm_small()
    s = np.full(10, 0.1)
    S = 100.0 * g.m
    spx = oracle.sparsifier(g.indptr, g.indices, 10, s, S, seed=1)
    return g, s, S, spx


def _csr(spx, n):
    return dict(n=n, nnz=len(spx["indices"]),
                indptr=torch.as_tensor(spx["indptr"]).cuda(),
                indices=torch.as_tensor(spx["indices"].astype(np.int32)).cuda(),
                data=torch.as_tensor(spx["data"]).cuda())


def test_stage_errors(ctx, case, capsys):
    g, s, S, spx = case
    d, p_os, c = 32, 16, 48
    report = {}
    M = sp.csr_matrix((spx["data"].astype(np.float64), spx["indices"], spx["indptr"]), shape=(g.n, g.n))
    Om = oracle.gaussian_sketch(g.n, c, seed=1)
    Om_gpu = ctx.gaussian_sketch(g.n, c, seed=1)
    # stage 1: sketch (FP32 output, then the BF16 operand copy)
    e_fp32 = np.max(np.abs(to_np(Om_gpu) - Om) / (1 + np.abs(Om)))
    Om_h = Om_gpu.to(torch.bfloat16)
    e_bf16 = np.max(np.abs(to_np(Om_h.float()) - Om) / np.maximum(np.abs(Om), 1e-3))
    report["sketch"] = (e_fp32, e_bf16)
    assert e_fp32 <= 1e-5 and e_bf16 <= U_BF16 * 1.01
    # stage 2: Y = M Omega
    Y_ref = M @ Om
    for mode, X in (("fp32", Om_gpu), ("bf16", Om_h)):
        Y = to_np(ctx.spmm(_csr(spx, g.n), X)).astype(np.float64)
        report.setdefault("Y0", []).append(np.linalg.norm(Y - Y_ref) / np.linalg.norm(Y_ref))
    assert report["Y0"][0] <= 1e-6 and report["Y0"][1] <= 2 * U_BF16
    # stage 3: randomized SVD (Sigma, U) and X0 = U Sigma^1/2
    ref = oracle.fast_randomized_svd(spx["indptr"], spx["indices"], spx["data"], d, 1, p_os, 1)
    X0_ref = oracle.embedding_from_svd(ref["U"], ref["sigma"])
    lead = 4   # the planted block directions (well separated)
    for prec in (lne.PREC_FP32, lne.PREC_BF16_MIXED):
        p = make_params(1, [1.0], 1.0, d=d, oversample=p_os, q=1, seed=1)
        p.precision = prec
        out = ctx.rsvd(_csr(spx, g.n), p)
        sig = to_np(out["sigma"])
        U = to_np(out["U"]).astype(np.float64)
        X0 = to_np(out["X0"]).astype(np.float64)
        report.setdefault("sigma", []).append(np.max(np.abs(sig - ref["sigma"]) / ref["sigma"]))
        report.setdefault("U_lead_angle", []).append(oracle.subspace_sin(U[:, :lead], ref["U"][:, :lead]))
        report.setdefault("U_angle", []).append(oracle.subspace_sin(U, ref["U"]))
        report.setdefault("X0_lead", []).append(
            np.max(np.abs(col_align(X0[:, :lead], X0_ref[:, :lead]) - X0_ref[:, :lead])) / np.abs(X0_ref).max())
    assert report["sigma"][0] <= 1e-4 and report["sigma"][1] <= 4 * U_BF16
    assert report["U_lead_angle"][0] <= 1e-3 and report["U_lead_angle"][1] <= 1e-2
    # stage 4: propagation fed the oracle's X0
    prop_ref = oracle.spectral_propagation(g.indptr, g.indices, X0_ref, 10, 0.5, 0.2)
    for prec in (lne.PREC_FP32, lne.PREC_BF16_MIXED):
        p = make_params(1, [1.0], 1.0, d=d, k=10, theta=0.5, mu=0.2)
        p.precision = prec
        out = ctx.propagate(lne.DeviceGraph.from_graph(g), p, torch.as_tensor(X0_ref.astype(np.float32)).cuda(),
                            want_intermediates=True)
        F, P, X = (to_np(out[k]).astype(np.float64) for k in ("F", "P", "X"))
        report.setdefault("F", []).append(np.linalg.norm(F - prop_ref["F"]) / np.linalg.norm(prop_ref["F"]))
        report.setdefault("P", []).append(np.linalg.norm(P - prop_ref["P"]) / np.linalg.norm(prop_ref["P"]))
        report.setdefault("X_lead_angle", []).append(oracle.subspace_sin(X[:, :lead], prop_ref["X"][:, :lead]))
    assert report["F"][0] <= 1e-5 and report["F"][1] <= 4 * U_BF16
    assert report["P"][0] <= 1e-5 and report["P"][1] <= 4 * U_BF16
    # stage 5: whole method
    emb_ref = oracle.embed(g.indptr, g.indices, 10, s, S, d, 1, 10, 0.5, 0.2, 1)
    for prec in (lne.PREC_FP32, lne.PREC_BF16_MIXED):
        p = make_params(10, s, S, d=d, q=1, k=10, seed=1)
        p.precision = prec
        X = to_np(ctx.embed(lne.DeviceGraph.from_graph(g), p)).astype(np.float64)
        report.setdefault("embed_lead_angle", []).append(oracle.subspace_sin(X[:, :lead], emb_ref["X"][:, :lead]))
    assert report["embed_lead_angle"][0] <= 1e-3 and report["embed_lead_angle"][1] <= 1e-2
    with capsys.disabled():
        print("\nper-stage error vs FP64 oracle (fp32, bf16-operand):")
        for k, v in report.items():
            print(f"  {k:18s} {v[0]:.3e}  {v[1]:.3e}")


def test_bf16_rejects_unaligned_width(ctx, case):
    g, s, S, spx = case
    p = make_params(1, [1.0], 1.0, d=30, oversample=15, q=1, seed=1)
    p.precision = lne.PREC_BF16_MIXED
    with pytest.raises(lne.LneError) as e:
        ctx.rsvd(_csr(spx, g.n), p)
    assert e.value.code == -5
