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
