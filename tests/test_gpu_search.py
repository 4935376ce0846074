"""Surrogate-guided search against the plain search (the method scored by
itself): on held-out graphs of the SBM tuning suite, ranking a pool of 256
candidates by the trained network and running only its top 8 must reach the
plain search's best Macro-F1 over 32 full runs within 0.01, and must beat
running 8 candidates chosen without the network on most graphs -- the gain
the network brings. Everything is seeded, so the outcome is deterministic."""
import numpy as np
import pytest
import torch
from scipy.stats import spearmanr

from paper_2302_07084_gb300 import lne, search, synth

pytestmark = pytest.mark.gpu

N_MAX, N_TRAIN, N_TEST, POOL, TOP = 6000, 96, 12, 256, 8


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


def _task(seed):
    g = synth.tuning_graph(seed, n_max=N_MAX)
    idx = np.random.default_rng(seed).permutation(g.n)
    return g, (lne.DeviceGraph(g.indptr, g.indices), torch.as_tensor(g.labels).cuda(),
               torch.as_tensor(idx[: g.n // 2]).cuda(), torch.as_tensor(idx[g.n // 2:]).cuda())


def _cands(g, seed, count, off):
    return [lne.Params(T=10, s=list(c["s"]), samples=100.0 * g.m, d=32, oversample=16, q=1, k=c["k"],
                       theta=c["theta"], mu=c["mu"], seed=seed) for c in synth.tuning_candidates(seed + off, count)]


def test_surrogate_search_reaches_plain_search(ctx, capsys):
    graphs = [_task(2000 + i) for i in range(N_TRAIN)]
    stats = [search.graph_statistics(ctx, g.indptr, g.indices, seed=1) for g, _ in graphs]
    cands = [_cands(g, 2000 + i, 32, 1000) for i, (g, _) in enumerate(graphs)]
    scores, _ = ctx.tune_tasks([t for _, t in graphs], cands)
    X, y = search.training_rows(cands, stats, scores)
    loss = search.fit_surrogate(ctx, X, y, epochs=100, seed=1)
    rows = []
    for i in range(N_TEST):
        g, t = _task(9000 + i)
        st = search.graph_statistics(ctx, g.indptr, g.indices, seed=1)
        plain = _cands(g, 9000 + i, 32, 1000)
        _, sc, _ = search.plain_search(ctx, t, plain)
        pool = plain + _cands(g, 9000 + i, POOL - 32, 3000)
        _, best, pred, _ = search.surrogate_search(ctx, t, st, pool, TOP)
        rows.append((sc.max(), best, sc[:TOP].max(), spearmanr(pred[:32], sc).correlation))
    r = np.array(rows)
    gap = float(np.mean(r[:, 0] - r[:, 1]))
    wins, losses = int((r[:, 1] > r[:, 2]).sum()), int((r[:, 1] < r[:, 2]).sum())
    with capsys.disabled():
        print(f"\ntrain MSE {loss:.5f} (target var {y.var():.5f}); held-out mean Macro-F1: plain-32 {r[:, 0].mean():.4f}"
              f" surrogate top-{TOP} of {POOL} {r[:, 1].mean():.4f} first-{TOP} {r[:, 2].mean():.4f};"
              f" gap {gap:+.4f}; wins/losses vs first-{TOP} {wins}/{losses}; rank corr {np.nanmean(r[:, 3]):.3f}")
    assert gap <= 0.01
    assert wins > 2 * losses and r[:, 1].mean() > r[:, 2].mean()
