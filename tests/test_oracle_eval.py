"""Pins of the oracle's downstream objective (Sec. 6.1: one-vs-rest logistic
regression, Micro/Macro-F1) against scikit-learn, an implementation the oracle
does not use, and against hand-counted cases."""
import numpy as np
import pytest

import oracle


def test_f1_hand_counted():
    Yt = np.array([[1, 0], [1, 1], [0, 1], [0, 0]], bool)
    Yp = np.array([[1, 1], [0, 1], [0, 1], [1, 0]], bool)
    # label 0: tp=1 fp=1 fn=1 -> 2/4; label 1: tp=2 fp=1 fn=0 -> 4/5
    ma, mi = oracle.f1_scores(Yt, Yp)
    assert ma == pytest.approx((0.5 + 0.8) / 2)
    assert mi == pytest.approx(2 * 3 / (2 * 3 + 2 + 1))


def test_topk_rule():
    sc = np.array([[0.1, 0.9, 0.5], [2.0, 2.0, -1.0]])
    pred = oracle.predict_topk(sc, np.array([2, 1]))
    assert pred.tolist() == [[False, True, True], [True, False, False]]


def test_f1_matches_sklearn():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    Yt = rng.random((300, 7)) < 0.3
    Yp = rng.random((300, 7)) < 0.3
    ma, mi = oracle.f1_scores(Yt, Yp)
    assert ma == pytest.approx(sk.f1_score(Yt, Yp, average="macro", zero_division=0))
    assert mi == pytest.approx(sk.f1_score(Yt, Yp, average="micro", zero_division=0))


def test_logreg_matches_sklearn_optimum():
    lm = pytest.importorskip("sklearn.linear_model")
    rng = np.random.default_rng(1)
    n, d, L = 400, 6, 3
    X = rng.standard_normal((n, d))
    Wt = rng.standard_normal((d, L))
    Y = (X @ Wt + 0.5 * rng.standard_normal((n, L))) > 0.3
    W = oracle.logreg_ovr(X, Y, C=1.0, iters=15)
    Xa = np.hstack([X, np.ones((n, 1))])
    for l in range(L):
        clf = lm.LogisticRegression(C=1.0, fit_intercept=False, tol=1e-12, max_iter=10000)
        clf.fit(Xa, Y[:, l])
        np.testing.assert_allclose(W[:, l], clf.coef_.ravel(), rtol=1e-5, atol=1e-6)


def test_macro_f1_separable_blocks():
    rng = np.random.default_rng(2)
    y = rng.integers(0, 4, 600)
    X = np.eye(4)[y] * 3 + 0.3 * rng.standard_normal((600, 4))
    labels = np.eye(4, dtype=bool)[y]
    idx = rng.permutation(600)
    ma, mi, _ = oracle.macro_f1(X, labels, idx[:300], idx[300:])
    assert ma > 0.95 and mi > 0.95
