"""Surrogate-guided hyper-parameter search.

The paper tunes T-window weights s_r, the filter (k, theta, mu) and q per data
set with an AutoML search in which every trial is a full run scored by the
downstream Macro-F1 (Sec. 4.4, Sec. 6.1). Here a small regression network
(the surrogate, trained on the GPU by the library's own kernels) predicts that
score from 30 features -- the candidate's parameters and 16 statistics of the
graph -- so a search can rank a large pool of candidates and run the method
only on the few it ranks highest; those full runs make the choice.

Features of a candidate (30): s_1..s_10, k, theta, mu, q, then the graph's
statistics (``graph_statistics``): log n, log m, degree mean / std / max /
skewness / Gini, block-count estimate, degree assortativity, sampled
clustering coefficient, the 2nd..4th eigenvalues of D^-1/2 A D^-1/2 (from a
randomized SVD run by the library), edge density, two-hop growth, giant
component fraction.
"""
from __future__ import annotations

import time
from typing import Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph
import torch

from . import lne

N_STATS = 16


def _normalized_adjacency_spectrum(ctx: lne.Context, indptr, indices, deg, count: int, seed: int):
    """Largest singular values of D^-1/2 A D^-1/2 (= |eigenvalues|), by the
    library's randomized SVD with two power iterations."""
    n = len(deg)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    dinv = 1.0 / np.sqrt(np.maximum(deg, 1))
    data = (dinv[rows] * dinv[indices]).astype(np.float32)
    d = min(count, n - 16)
    csr = dict(n=n, nnz=len(indices), indptr=torch.as_tensor(np.asarray(indptr, np.int64)).cuda(),
               indices=torch.as_tensor(np.asarray(indices, np.int32)).cuda(), data=torch.as_tensor(data).cuda())
    p = lne.Params(T=1, s=[1.0], samples=1.0, d=d, oversample=16, q=2, k=0, seed=seed)
    return ctx.rsvd(csr, p)["sigma"].cpu().numpy()


def graph_statistics(ctx: lne.Context, indptr, indices, seed: int = 0, sample: int = 512) -> np.ndarray:
    """The 16 graph statistics of the surrogate's input (see the module doc)."""
    indptr = np.asarray(indptr, np.int64)
    indices = np.asarray(indices, np.int64)
    n = len(indptr) - 1
    m = len(indices) / 2.0
    deg = np.diff(indptr).astype(np.float64)
    mean, std = deg.mean(), deg.std()
    skew = float(np.mean((deg - mean) ** 3) / std ** 3) if std > 0 else 0.0
    ds = np.sort(deg)
    gini = float((2.0 * np.sum(np.arange(1, n + 1) * ds) / (n * ds.sum()) - (n + 1.0) / n)) if ds.sum() > 0 else 0.0
    rows = np.repeat(np.arange(n), np.diff(indptr))
    du, dv = deg[rows], deg[indices]
    assort = float(np.corrcoef(du, dv)[0, 1]) if du.std() > 0 and dv.std() > 0 else 0.0
    rng = np.random.default_rng(seed)
    nodes = rng.choice(n, size=min(sample, n), replace=False)
    clus, growth = [], []
    for v in nodes:
        nb = indices[indptr[v]:indptr[v + 1]]
        k = len(nb)
        if k == 0:
            continue
        two = np.concatenate([indices[indptr[u]:indptr[u + 1]] for u in nb])
        if k >= 2:
            links = np.count_nonzero(np.isin(two, nb)) / 2.0
            clus.append(links / (k * (k - 1) / 2.0))
        reach = np.setdiff1d(np.unique(two), np.append(nb, v))
        growth.append(len(reach) / k)
    A = sp.csr_matrix((np.ones(len(indices)), indices, indptr), shape=(n, n))
    _, comp = csgraph.connected_components(A, directed=False)
    giant = np.bincount(comp).max() / n
    sig = np.sort(_normalized_adjacency_spectrum(ctx, indptr, indices, deg, 24, seed))[::-1]
    bulk = 2.0 / np.sqrt(max(mean - 1.0, 1.0))            # edge of the random-graph part of the spectrum
    blocks = float(np.count_nonzero(sig > 1.1 * bulk))
    lam = np.concatenate([sig[1:4], np.zeros(3)])[:3]
    return np.array([np.log(n), np.log(max(m, 1.0)), mean, std, deg.max(), skew, gini, blocks, assort,
                     float(np.mean(clus)) if clus else 0.0, lam[0], lam[1], lam[2],
                     2.0 * m / (n * (n - 1.0)), float(np.mean(growth)) if growth else 0.0, giant])


def candidate_features(p: lne.Params, stats: np.ndarray) -> np.ndarray:
    """30 inputs of the surrogate for candidate p on a graph with `stats`."""
    s = np.zeros(10)
    s[:min(10, len(p.s))] = np.asarray(p.s, np.float64)[:10] / np.sum(p.s)
    return np.concatenate([s, [p.k, p.theta, p.mu, p.q], stats]).astype(np.float32)


def training_rows(cands: Sequence[Sequence[lne.Params]], stats: Sequence[np.ndarray], scores: np.ndarray):
    """Surrogate training rows from full runs: features of every candidate of
    every graph, and as target its Macro-F1 minus the mean Macro-F1 of its
    graph's candidates -- the search only ranks candidates within one graph,
    so the network need not learn how hard each graph is."""
    scores = np.asarray(scores, np.float64)
    X = np.stack([candidate_features(p, st) for row, st in zip(cands, stats) for p in row])
    y = (scores - scores.mean(axis=1, keepdims=True)).ravel().astype(np.float32)
    return X, y


def fit_surrogate(ctx: lne.Context, X: np.ndarray, y: np.ndarray, epochs: int = 100, seed: int = 1,
                  batch: int = 256, lr: float = 1e-3) -> float:
    """Initialise, scale the features and train the context's surrogate on the
    GPU; returns the final mean squared error on the training rows."""
    Xd = torch.as_tensor(np.asarray(X, np.float32)).cuda()
    yd = torch.as_tensor(np.asarray(y, np.float32)).cuda()
    ctx.surrogate_init(seed)
    ctx.surrogate_fit_scaling(Xd)
    return ctx.surrogate_train(Xd, yd, epochs=epochs, batch=batch, lr=lr, seed=seed + 1)


def plain_search(ctx: lne.Context, task, cands: Sequence[lne.Params]):
    """Every candidate is a full run (lne_tune_batch); returns (best index,
    scores, seconds)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ma, _ = ctx.tune_batch(task[0], cands, task[1], task[2], task[3])
    return int(np.argmax(ma)), ma, time.perf_counter() - t0


def surrogate_search(ctx: lne.Context, task, stats: np.ndarray, pool: Sequence[lne.Params], top: int):
    """Rank the pool by the surrogate's predicted score, run the `top` best
    with the method, keep the best of those by its measured score. Returns
    (chosen candidate, its measured Macro-F1, predicted scores, seconds)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = torch.as_tensor(np.stack([candidate_features(p, stats) for p in pool])).cuda()
    pred = ctx.surrogate_predict(F).cpu().numpy()
    order = np.argsort(-pred, kind="stable")[:top]
    chosen = [pool[i] for i in order]
    ma, _ = ctx.tune_batch(task[0], chosen, task[1], task[2], task[3])
    j = int(np.argmax(ma))
    return chosen[j], float(ma[j]), pred, time.perf_counter() - t0
