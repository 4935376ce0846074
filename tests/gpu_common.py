"""Shared helpers of the GPU parity tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_07084_gb300 import lne, synth


def make_params(T, s, S, d=32, oversample=16, q=1, k=10, theta=0.5, mu=0.2, seed=1, b=1.0):
    return lne.Params(T=T, s=list(np.asarray(s, dtype=np.float64)), samples=float(S), b=b, d=d,
                      oversample=oversample, q=q, k=k, theta=theta, mu=mu, seed=seed)


def oracle_counts(g, p):
    return oracle.sparsifier_counts(g.indptr, g.indices, p.T, p.s, p.samples, p.seed)


def to_np(t):
    return t.detach().cpu().numpy()


def col_align(A, B):
    """Flip the columns of A to best match B (singular vectors are unique up to sign)."""
    sg = np.sign(np.sum(A * B, axis=0))
    sg[sg == 0] = 1
    return A * sg


def assert_subspace(X, Xref, lead=4, bound=1e-3, full_bound=1e-3, tag=""):
    """The subspace gate of the whole method: the sine of the largest principal
    angle between the GPU's and the oracle's column spans, both on the `lead`
    well-separated leading columns and on all d columns, each <= its bound.
    Returns (leading angle, full angle), which are also printed."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    a_lead = oracle.subspace_sin(X[:, :lead], Xref[:, :lead])
    a_full = oracle.subspace_sin(X, Xref)
    print(f"{tag} subspace sin: leading {lead} {a_lead:.3e}, all {X.shape[1]} {a_full:.3e}")
    assert a_lead <= bound, (a_lead, bound)
    assert a_full <= full_bound, (a_full, full_bound)
    return a_lead, a_full


def leading_gap_index(sigma, kmax=32):
    """The k (2..kmax) with the largest relative gap (sigma_k - sigma_{k+1}) / sigma_k
    among the singular values `sigma` (descending): the leading directions that
    are well separated from the rest. Returns (k, that gap)."""
    s = np.asarray(sigma, dtype=np.float64)
    kmax = min(kmax, s.size - 1)
    gaps = (s[1:kmax] - s[2:kmax + 1]) / s[1:kmax]
    k = int(np.argmax(gaps)) + 2
    return k, float(gaps[k - 2])


def full_span_bound(sigma_all, d):
    """Bound on the sine of the angle between the GPU's and the oracle's d-column
    spans: 1e-3 when the relative gap at d is at least 1e-2, else 1e-5 / gap
    (FP32 rounding of the products moves the span by about that much).
    Returns (bound, relative gap at d)."""
    s = np.asarray(sigma_all, dtype=np.float64)
    gap = (s[d - 1] - s[d]) / s[d - 1]
    return max(1e-3, 1e-5 / max(gap, 1e-12)), float(gap)
