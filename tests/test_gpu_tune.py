"""Batched tuning (lne_tune_batch, lne_tune_tasks) against the CPU oracle and
against one-candidate runs.

Every batched candidate's embedding and Macro-F1 must match the oracle's
(oracle.embed + oracle.macro_f1) for that candidate: the subspace gate on the
embedding and 0.005 on the score.

Every candidate's embedding and scores must equal what lne_embed followed by
lne_macro_f1 gives for that candidate alone: the batch shares the sparsifier
and the randomized SVD between candidates with the same sampling inputs and
runs all propagations as column blocks of one product, which changes no
arithmetic of any column. The captured CUDA graph (second call of a shape) and
its replays (later calls, new coefficients) must give the same results, and so
must every CTA size of the merge SpMM.
"""
import numpy as np
import pytest
import torch

from paper_2302_07084_gb300 import lne, synth
import oracle
from gpu_common import full_span_bound, leading_gap_index, make_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def case():
    g = synth.chung_lu(3000, 30000, 2.1, seed=9, n_labels=12)
    idx = np.random.default_rng(5).permutation(g.n)
    tr, te = idx[: g.n // 2], idx[g.n // 2:]
    dev = dict(g=lne.DeviceGraph.from_graph(g), labels=torch.as_tensor(g.labels).cuda(),
               tr=torch.as_tensor(tr).cuda(), te=torch.as_tensor(te).cuda())
    return g, dev


def _cands(g, d, spec):
    return [make_params(10, np.full(10, 0.1), 50.0 * g.m, d=d, q=1, k=k, theta=th, mu=mu, seed=seed)
            for (k, th, mu, seed) in spec]


def _single(ctx, dev, p):
    X = ctx.embed(dev["g"], p)
    ma, mi = ctx.macro_f1(X, dev["labels"], dev["tr"], dev["te"])
    return to_np(X), ma, mi


def _check_against_single(ctx, dev, cands, ma, mi, X):
    for j, p in enumerate(cands):
        Xs, mas, mis = _single(ctx, dev, p)
        Xb = to_np(X[j])
        err = np.max(np.abs(Xb - Xs)) / np.max(np.abs(Xs))
        assert err <= 1e-5, (j, err)
        # the same embedding gives the same scores; a last-bit difference may move a near tie
        tol = 0.0 if np.array_equal(Xb, Xs) else 0.005
        assert abs(ma[j] - mas) <= tol and abs(mi[j] - mis) <= tol, (j, ma[j], mas)


SPEC = [(10, 0.5, 0.2, 3), (5, 1.0, 0.5, 3), (1, 0.5, 0.2, 3), (0, 0.5, 0.2, 3), (2, 0.3, 0.1, 3),
        (10, 0.5, 0.2, 4), (7, 2.0, -0.3, 4)]


def test_batch_equals_single_runs(ctx, case):
    g, dev = case
    cands = _cands(g, 32, SPEC)
    ma, mi, X = ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"], want_embeddings=True)
    _check_against_single(ctx, dev, cands, ma, mi, X)
    exact = [bool(np.array_equal(to_np(X[j]), to_np(ctx.embed(dev["g"], p)))) for j, p in enumerate(cands)]
    print("bit-identical to one-candidate runs:", exact)


def test_graph_capture_and_replay(ctx, case):
    g, dev = case
    # same shape (k values) three times: eager, captured, replayed with new theta / mu
    specs = [[(10, 0.5, 0.2, 3), (6, 1.0, 0.5, 3)],
             [(10, 0.7, 0.3, 3), (6, 0.4, 0.0, 3)],
             [(10, 1.5, -0.2, 3), (6, 0.2, 0.9, 3)]]
    for spec in specs:
        cands = _cands(g, 32, spec)
        ma, mi, X = ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"], want_embeddings=True)
        _check_against_single(ctx, dev, cands, ma, mi, X)
    ctx.trace(True)
    cands = _cands(g, 32, specs[0])
    ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"])
    names = [r["name"] for r in ctx.trace_read()]
    ctx.trace(False)
    assert "propagate_batch_graph" in names and "graph_spmm" not in names


def test_cta_size_does_not_change_results(ctx, case):
    g, dev = case
    cands = _cands(g, 32, SPEC[:3])
    outs = []
    for t in (64, 128, 256, 0):
        ctx.set_option(lne.OPT_SPMM_THREADS, t)
        outs.append(ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"], want_embeddings=True))
    ctx.set_option(lne.OPT_SPMM_THREADS, 0)
    for o in outs[1:]:
        assert torch.equal(o[2], outs[0][2])
        assert np.array_equal(o[0], outs[0][0])


def test_column_block_does_not_change_results(ctx, case):
    """The autotuner's column-block widths (and no blocking) give bit-identical
    batched results: every column gets the same terms in the same order."""
    g, dev = case
    spec = [(3 + j, 0.5 + 0.1 * j, 0.1 * j, 3) for j in range(4)]   # 4 x d = 128: 512 columns
    cands = _cands(g, 128, spec)
    outs = []
    for b in (-1, 128, 256, 0):
        ctx.set_option(lne.OPT_SPMM_COLBLOCK, b)
        outs.append(ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"], want_embeddings=True))
    ctx.set_option(lne.OPT_SPMM_COLBLOCK, 0)
    for o in outs[1:]:
        assert torch.equal(o[2], outs[0][2])
        assert np.array_equal(o[0], outs[0][0])
    with pytest.raises(lne.LneError):
        ctx.set_option(lne.OPT_SPMM_COLBLOCK, 130)


def test_several_column_blocks(ctx, case):
    g, dev = case
    # d = 128: 8 candidates per block, so 9 propagating candidates need two blocks
    spec = [(3 + (j % 4), 0.5 + 0.1 * j, 0.1 * (j % 3), 3) for j in range(9)]
    cands = _cands(g, 128, spec)
    ma, mi, X = ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"], want_embeddings=True)
    picks = [0, 7, 8]
    _check_against_single(ctx, dev, [cands[j] for j in picks], ma[picks], mi[picks], X[picks])


def test_rejects_bad_candidates(ctx, case):
    g, dev = case
    cands = _cands(g, 32, SPEC[:2])
    cands[1].d = 16
    with pytest.raises(lne.LneError) as e:
        ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"])
    assert e.value.code == -1
    cands = _cands(g, 32, SPEC[:2])
    cands[0].precision = lne.PREC_BF16_MIXED
    with pytest.raises(lne.LneError) as e:
        ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"])
    assert e.value.code == -5
    cands = _cands(g, 30, SPEC[:2])
    with pytest.raises(lne.LneError) as e:
        ctx.tune_batch(dev["g"], cands, dev["labels"], dev["tr"], dev["te"])
    assert e.value.code == -5
    with pytest.raises(lne.LneError):
        ctx.set_option(lne.OPT_SPMM_THREADS, 96)


def _task(seed, n, blocks):
    g = synth.sbm(n, blocks, 12.0 / (n / blocks), 3.0 / n, seed)
    idx = np.random.default_rng(seed).permutation(g.n)
    tr, te = idx[: g.n // 2], idx[g.n // 2:]
    dev = (lne.DeviceGraph.from_graph(g), torch.as_tensor(g.labels).cuda(), torch.as_tensor(tr).cuda(),
           torch.as_tensor(te).cuda())
    return g, dev


def _suite_cands(g, seed, count):
    out = []
    for c in synth.tuning_candidates(seed, count):
        out.append(make_params(10, c["s"], 20.0 * g.m, d=32, q=1, k=c["k"], theta=c["theta"], mu=c["mu"],
                               seed=seed))
    return out


def test_tasks_equal_per_task_batches(ctx):
    tasks = [_task(200 + t, n, b) for t, (n, b) in enumerate([(1500, 3), (2600, 5), (900, 2), (2000, 4)])]
    cands = [_suite_cands(g, 300 + t, 5) for t, (g, _) in enumerate(tasks)]
    ctx.set_option(lne.OPT_TUNE_WORKERS, 3)
    ma, mi = ctx.tune_tasks([dev for _, dev in tasks], cands)
    for t, (g, (dg, lab, tr, te)) in enumerate(tasks):
        ma1, mi1 = ctx.tune_batch(dg, cands[t], lab, tr, te)
        assert np.array_equal(ma[t], ma1) and np.array_equal(mi[t], mi1), t
    # the planted blocks are recovered far above chance by the best candidate
    assert ma.max(axis=1).min() > 0.5
    ctx.set_option(lne.OPT_TUNE_WORKERS, 1)
    ma2, mi2 = ctx.tune_tasks([dev for _, dev in tasks], cands)
    assert np.array_equal(ma, ma2) and np.array_equal(mi, mi2)
    ctx.set_option(lne.OPT_TUNE_WORKERS, 4)


def test_tasks_report_the_failing_task(ctx):
    tasks = [_task(210 + t, 1200, 3) for t in range(3)]
    cands = [_suite_cands(g, 310 + t, 2) for t, (g, _) in enumerate(tasks)]
    cands[2][1].d = 16
    with pytest.raises(lne.LneError) as e:
        ctx.tune_tasks([dev for _, dev in tasks], cands)
    assert e.value.code == -1 and "dimension" in str(e.value)
    with pytest.raises(lne.LneError):
        ctx.set_option(lne.OPT_TUNE_WORKERS, 0)


def _oracle_candidate(g, p, tr, te):
    ref = oracle.embed(g.indptr, g.indices, p.T, p.s, p.samples, p.d, p.q, p.k, p.theta, p.mu, p.seed,
                       oversample=p.oversample)
    f_ref = oracle.macro_f1(ref["X"], g.labels, tr, te)[0]
    return ref, f_ref


def _check_against_oracle(g, p, X, f_gpu, ref, f_ref, tag):
    X = np.asarray(X, dtype=np.float64)
    bound, gap = full_span_bound(ref["rsvd"]["sigma_all"], p.d)
    sig_x = ref["prop"]["sigma"] if ref["prop"]["P"] is not None else ref["rsvd"]["sigma"]
    k, _ = leading_gap_index(sig_x, kmax=min(16, p.d - 1))
    a_lead = oracle.subspace_sin(X[:, :k], ref["X"][:, :k])
    a_full = oracle.subspace_sin(X, ref["X"])
    print(f"{tag}: leading {k} sin {a_lead:.2e}, all {p.d} sin {a_full:.2e} (gap at d {gap:.2e}); "
          f"Macro-F1 {f_gpu:.4f} vs oracle {f_ref:.4f}")
    assert a_lead <= 1e-3 and a_full <= bound, (a_lead, a_full, bound)
    assert abs(f_gpu - f_ref) <= 0.005


def test_batch_matches_oracle(ctx):
    """Four candidates with distinct (k, theta, mu), two window weightings s
    (so two sparsifiers and randomized SVDs are shared), against the oracle."""
    g, (dg, lab, tr_t, te_t) = _task(230, 2400, 4)
    tr, te = to_np(tr_t), to_np(te_t)
    s_dir = synth.dirichlet_weights(10, seed=5)
    cands = [make_params(10, np.full(10, 0.1), 20.0 * g.m, d=32, q=1, k=10, theta=0.5, mu=0.2, seed=7),
             make_params(10, np.full(10, 0.1), 20.0 * g.m, d=32, q=1, k=4, theta=0.9, mu=0.4, seed=7),
             make_params(10, s_dir, 20.0 * g.m, d=32, q=1, k=15, theta=0.3, mu=0.0, seed=7),
             make_params(10, s_dir, 20.0 * g.m, d=32, q=1, k=1, theta=0.7, mu=0.3, seed=7)]
    ma, mi, X = ctx.tune_batch(dg, cands, lab, tr_t, te_t, want_embeddings=True)
    for j, p in enumerate(cands):
        ref, f_ref = _oracle_candidate(g, p, tr, te)
        _check_against_oracle(g, p, to_np(X[j]), ma[j], ref, f_ref, f"tune_batch candidate {j}")


def test_tasks_match_oracle(ctx):
    """lne_tune_tasks over two graphs of different sizes, two candidates each,
    against the oracle."""
    tasks = [_task(240 + t, n, b) for t, (n, b) in enumerate([(1800, 3), (2600, 5)])]
    cands = [[make_params(10, synth.dirichlet_weights(10, seed=11 + t), 20.0 * g.m, d=32, q=1, k=k, theta=th,
                          mu=mu, seed=9 + t) for (k, th, mu) in [(10, 0.5, 0.2), (6, 0.8, 0.45)]]
             for t, (g, _) in enumerate(tasks)]
    ctx.set_option(lne.OPT_TUNE_WORKERS, 2)
    ma, _ = ctx.tune_tasks([dev for _, dev in tasks], cands)
    ctx.set_option(lne.OPT_TUNE_WORKERS, 4)
    for t, (g, (dg, lab, tr_t, te_t)) in enumerate(tasks):
        tr, te = to_np(tr_t), to_np(te_t)
        for j, p in enumerate(cands[t]):
            ref, f_ref = _oracle_candidate(g, p, tr, te)
            X = to_np(ctx.embed(dg, p))
            _check_against_oracle(g, p, X, ma[t, j], ref, f_ref, f"tune_tasks graph {t} candidate {j}")
