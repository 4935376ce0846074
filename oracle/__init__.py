"""CPU oracle of the LightNE 2.0 hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. The product path (the CUDA
library and its binding) never imports, links or runs anything here, and this
package never imports the product.

Plain, slow, obviously checkable restatement of what the method computes, in
FP64, each function citing the passage it follows:

* sampling (C, ``lne_oracle.c``): Algorithm 1 (PathSampling), Algorithm 3
  (per-edge sampling, Sec. 5.2) and the walk-step rule of Sec. 5.2, on
  unweighted graphs and on graphs with positive integer arc weights (walks
  on D^-1 A with weighted D, samples per arc proportional to its weight);
* ``netmf_values`` / ``sparsifier_csr``: Eq. 1 (the NetMF matrix with the
  truncated logarithm) estimated from the sample counts;
* ``stratified_*``: window-stratified counts shared by many weightings s
  (an unbiased importance-weighted estimate, not in the paper);
* ``gaussian_sketch``: the Gaussian test matrix of Algorithm 4;
* ``sparse_sign_sketch``: the sparse sign test matrix that Sec. 4.2 names as
  an alternative to the Gaussian one (Tropp et al., SISC 2019): zeta
  nonzeros +-1 per row at distinct columns (Floyd's subset sampling);
* ``very_sparse_sketch``: the very sparse random projection named beside it
  (Li, Hastie and Church, KDD 2006): entries +-1 with probability 1/(2s)
  each, 0 otherwise;
* ``eig_svd``: Algorithm 2 (eigSVD);
* ``fast_randomized_svd``: Algorithm 4;
* ``embedding_from_svd``: X = U Sigma^{1/2} (Sec. 4.2);
* ``spectral_propagation``: Sec. 4.3 (Chebyshev filter in the normalised
  Laplacian, then the economic SVD of the last stage, Sec. 6.3);
* ``netmf_dense``: Eq. 1 evaluated densely, for tiny graphs.

Library primitives used as single steps: numpy sort/unique, scipy sparse
matrix products, ``numpy.linalg.eigh`` (the eig of Algorithm 2) and
``scipy.special.iv`` (Bessel coefficients). Each is pinned by tests against
closed forms, not against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp
import scipy.special

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lne_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblne_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_window_thresholds.argtypes = [ctypes.c_int, f64p, u64p]
        L.oracle_arc_rate.argtypes = [ctypes.c_double, ctypes.c_int64, u64p, u64p]
        L.oracle_arc_samples.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_arc_samples.restype = ctypes.c_uint64
        L.oracle_count_samples.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_uint64]
        L.oracle_count_samples.restype = ctypes.c_int64
        L.oracle_sample_trace.argtypes = [ctypes.c_int64, i64p, i32p, u32p, ctypes.c_int, f64p,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_int64, i64p, i32p, i32p, i64p, i64p, u32p]
        L.oracle_sample_trace.restype = ctypes.c_int64
        L.oracle_sketch_words.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, u32p]
        L.oracle_weighted_choice.argtypes = [u32p, ctypes.c_int64, ctypes.c_uint32]
        L.oracle_weighted_choice.restype = ctypes.c_int64
        L.oracle_count_samples_w.argtypes = [u32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                             ctypes.c_uint64]
        L.oracle_count_samples_w.restype = ctypes.c_int64
        L.oracle_arc_rate_w.argtypes = [ctypes.c_double, ctypes.c_uint32, ctypes.c_double, u64p, u64p]
        L.oracle_sparse_sign_words.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, u32p]
        L.oracle_very_sparse_words.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, u32p]
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None, ctype):
    if a is None:
        return ctypes.POINTER(ctype)()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ----------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                               _ptr(out, ctypes.c_uint32))
    return out


def window_thresholds(s) -> np.ndarray:
    """thr_1..thr_{T-1} for drawing r ~ Multinomial(s_1..s_T) (Algorithm 3)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    thr = np.zeros(max(len(s) - 1, 1), dtype=np.uint64)
    lib().oracle_window_thresholds(len(s), _ptr(s, ctypes.c_double), _ptr(thr, ctypes.c_uint64))
    return thr[: len(s) - 1]


def arc_rate(S: float, n_arcs: int) -> tuple[int, int]:
    """(floor(S/2m), floor(frac(S/2m) * 2^32)) -- Algorithm 3."""
    b = ctypes.c_uint64()
    f = ctypes.c_uint64()
    lib().oracle_arc_rate(float(S), int(n_arcs), ctypes.byref(b), ctypes.byref(f))
    return int(b.value), int(f.value)


def _weights(weights, n_arcs=None):
    if weights is None:
        return None
    w = np.ascontiguousarray(weights, dtype=np.uint32)
    assert n_arcs is None or len(w) == n_arcs
    assert np.all(w > 0), "arc weights are positive integers"
    return w


def weighted_degrees(indptr, weights) -> np.ndarray:
    """d_u = sum of the weights of u's arcs (float64, exact below 2^53)."""
    indptr = np.asarray(indptr, dtype=np.int64)
    n = len(indptr) - 1
    if weights is None:
        return np.diff(indptr).astype(np.float64)
    src = np.repeat(np.arange(n), np.diff(indptr))
    return np.bincount(src, weights=np.asarray(weights, dtype=np.float64), minlength=n)


def arc_rate_w(S: float, weight: int, vol: float) -> tuple[int, int]:
    """Weighted graphs: (floor(rate), floor(frac(rate) 2^32)) of
    rate = fl(fl(S A_a) / vol), the arc's share S A_a / vol of the samples."""
    b = ctypes.c_uint64()
    f = ctypes.c_uint64()
    lib().oracle_arc_rate_w(float(S), int(weight), float(vol), ctypes.byref(b), ctypes.byref(f))
    return b.value, f.value


def weighted_choice(w, word: int) -> int:
    """The weighted walk step's arc for a 32-bit word (inverse CDF with
    thresholds floor(2^32 P_j / d))."""
    w = np.ascontiguousarray(w, dtype=np.uint32)
    return int(lib().oracle_weighted_choice(_ptr(w, ctypes.c_uint32), len(w), int(word)))


def arc_samples(n_arcs: int, S: float, seed: int, a0: int = 0, a1: int | None = None, weights=None) -> np.ndarray:
    """n_a for arcs [a0, a1)."""
    a1 = n_arcs if a1 is None else a1
    L = lib()
    w = _weights(weights, n_arcs)
    if w is not None:
        vol = float(np.sum(w, dtype=np.uint64))
        out = []
        for a in range(a0, a1):
            base, thr = arc_rate_w(S, int(w[a]), vol)
            out.append(L.oracle_arc_samples(a, base, thr, seed))
        return np.array(out, dtype=np.int64)
    base, thr = arc_rate(S, n_arcs)
    return np.array([L.oracle_arc_samples(a, base, thr, seed) for a in range(a0, a1)], dtype=np.int64)


def count_samples(n_arcs: int, S: float, seed: int, a0: int = 0, a1: int | None = None, weights=None) -> int:
    a1 = n_arcs if a1 is None else a1
    w = _weights(weights, n_arcs)
    if w is not None:
        return int(lib().oracle_count_samples_w(_ptr(w, ctypes.c_uint32), n_arcs, a0, a1, float(S), seed))
    return int(lib().oracle_count_samples(n_arcs, a0, a1, float(S), seed))


def sample_trace(indptr, indices, T, s, S, seed, a0=0, a1=None, fields=("arc", "r", "sigma", "u1", "v1"),
                 weights=None):
    """Every PathSampling draw of arcs [a0, a1) in (arc, sample) order.

    Returns a dict with the requested fields: ``arc``, window ``r``, split
    ``sigma``, the ordered endpoints ``u1`` (walked from the arc's source)
    and ``v1`` (walked from its target), and the downsampling ``coin`` word.
    With ``weights`` (positive integer arc weights, symmetric) arc a draws
    S A_a / vol samples in expectation and a walk step takes an arc with
    probability proportional to its weight (``weighted_choice``).
    """
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = indptr.shape[0] - 1
    n_arcs = int(indptr[-1])
    a1 = n_arcs if a1 is None else a1
    w = _weights(weights, n_arcs)
    total = count_samples(n_arcs, S, seed, a0, a1, weights=w)
    out = {
        "arc": np.zeros(total, np.int64) if "arc" in fields else None,
        "r": np.zeros(total, np.int32) if "r" in fields else None,
        "sigma": np.zeros(total, np.int32) if "sigma" in fields else None,
        "u1": np.zeros(total, np.int64) if "u1" in fields else None,
        "v1": np.zeros(total, np.int64) if "v1" in fields else None,
        "coin": np.zeros(total, np.uint32) if "coin" in fields else None,
    }
    got = lib().oracle_sample_trace(
        n, _ptr(indptr, ctypes.c_int64), _ptr(indices, ctypes.c_int32), _ptr(w, ctypes.c_uint32), len(s),
        _ptr(s, ctypes.c_double), float(S), int(seed), int(a0), int(a1),
        _ptr(out["arc"], ctypes.c_int64), _ptr(out["r"], ctypes.c_int32),
        _ptr(out["sigma"], ctypes.c_int32), _ptr(out["u1"], ctypes.c_int64),
        _ptr(out["v1"], ctypes.c_int64), _ptr(out["coin"], ctypes.c_uint32))
    assert got == total
    return {k: v for k, v in out.items() if v is not None}


def sample_pairs(indptr, indices, T, s, S, seed, a0=0, a1=None, weights=None):
    """Canonical endpoint pairs (x = min, y = max) of every draw of arcs [a0, a1)."""
    tr = sample_trace(indptr, indices, T, s, S, seed, a0, a1, fields=("u1", "v1"), weights=weights)
    return np.minimum(tr["u1"], tr["v1"]), np.maximum(tr["u1"], tr["v1"])


def arc_downsample(indptr, indices, C: float, weights=None):
    """Edge downsampling (Sec. 4.1, Algorithm 3) per CSR arc u -> v:
    p_e = min(1, C (1/d_u + 1/d_v)); the coin keeps a draw iff its word is below
    thr_e = min(2^32, floor(p_e 2^32)); a kept draw adds the weight 1/p_e, held
    in fixed point with 2^-32 units, w_e = floor(2^32 / p_e + 1/2), so that
    sums are exact and independent of their order. Returns (thr_e, w_e) as
    uint64 arrays over the arcs."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    n = len(indptr) - 1
    deg = weighted_degrees(indptr, weights)
    src = np.repeat(np.arange(n), np.diff(indptr))
    du, dv = deg[src], deg[indices]
    p = C * (1.0 / du + 1.0 / dv)
    if weights is not None:           # p_e = min(1, A_uv (C (1/d_u + 1/d_v))), Sec. 4.1
        p = np.asarray(weights, dtype=np.float64) * p
    p = np.minimum(1.0, p)
    thr = np.where(p >= 1.0, 2.0 ** 32, np.floor(p * 4294967296.0)).astype(np.uint64)
    w = np.floor(4294967296.0 / p + 0.5).astype(np.uint64)
    return thr, w


def sparsifier_counts(indptr, indices, T, s, S, seed, C: float = 0.0, weights=None):
    """Exact multiplicity K_xy of every sampled unordered pair (x <= y).

    The aggregation of Sec. 5.2 (hash table with atomic counts) computes the
    multiset of sampled pairs; here it is a sort and a run-length count.
    Returns (x, y, count) sorted by (x, y). With edge downsampling (C > 0) the
    third array is the pair's summed weight in 2^-32 units (uint64, exact):
    only draws whose coin comes up heads count, each with weight 1/p_e of its
    arc (``arc_downsample``).
    """
    n = len(indptr) - 1
    if C <= 0.0:
        x, y = sample_pairs(indptr, indices, T, s, S, seed, weights=weights)
        keys, cnt = np.unique(x * n + y, return_counts=True)
        return keys // n, keys % n, cnt.astype(np.int64)
    tr = sample_trace(indptr, indices, T, s, S, seed, fields=("arc", "u1", "v1", "coin"), weights=weights)
    thr, w = arc_downsample(indptr, indices, C, weights)
    kept = tr["coin"].astype(np.uint64) < thr[tr["arc"]]
    x = np.minimum(tr["u1"], tr["v1"])[kept]
    y = np.maximum(tr["u1"], tr["v1"])[kept]
    keys, inv = np.unique(x * n + y, return_inverse=True)
    wsum = np.zeros(len(keys), dtype=np.uint64)
    np.add.at(wsum, inv, w[tr["arc"][kept]])
    return keys // n, keys % n, wsum


def sparsifier_counts_dense(indptr, indices, T, s, S, seed, chunk_samples: float = 5.0e7):
    """The same (x, y, count) as ``sparsifier_counts`` (C = 0), for graphs whose
    n x n pair space fits host memory (n up to a few ten thousand) and sample
    counts too large to hold at once: the draws of consecutive arc ranges of
    about ``chunk_samples`` draws each are counted into one dense table of
    unordered pairs (index x n + y, x <= y), which is then read out in (x, y)
    order. Counting is order-independent, so the result is the multiset of
    all draws however the arcs are split."""
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    n = len(indptr) - 1
    n_arcs = int(indptr[-1])
    per_arc = max(float(S) / max(n_arcs, 1), 1e-9)
    step = max(1, int(chunk_samples / per_arc))
    table = np.zeros(n * n, dtype=np.int64)
    for a0 in range(0, n_arcs, step):
        a1 = min(n_arcs, a0 + step)
        x, y = sample_pairs(indptr, indices, T, s, S, seed, a0, a1)
        table += np.bincount(x * n + y, minlength=n * n)
        del x, y
    keys = np.flatnonzero(table)
    return keys // n, keys % n, table[keys]


def stratified_counts(indptr, indices, T, S, seed, weights=None):
    """Window-stratified counts for sharing one sampling pass among many
    window weightings s (a proposal for candidate batching, not a procedure of
    the paper): every draw takes r ~ U{1..T} (Algorithm 3 with
    s uniform) and the pair counts are kept per window length.
    Returns (x, y, r, count) sorted by (x, y, r)."""
    n = len(indptr) - 1
    tr = sample_trace(indptr, indices, T, np.ones(T), S, seed, fields=("r", "u1", "v1"), weights=weights)
    x = np.minimum(tr["u1"], tr["v1"])
    y = np.maximum(tr["u1"], tr["v1"])
    keys, cnt = np.unique((x * n + y) * T + (tr["r"].astype(np.int64) - 1), return_counts=True)
    pair, r = keys // T, keys % T + 1
    return pair // n, pair % n, r, cnt.astype(np.int64)


def stratified_weights(s, T) -> np.ndarray:
    """w_r = floor(T (s_r / sum(s)) 2^24 + 1/2), each step one FP64 rounding and
    the sum taken left to right: the importance weight of window
    r (its probability under s over its probability 1/T under the uniform
    draw) in 2^-24 units, exact integers (w_r < 2^28 for T <= 16)."""
    s = np.asarray(s, dtype=np.float64)[:T]
    tot = 0.0
    for v in s:              # left to right, as the window thresholds sum
        tot += float(v)
    return np.floor(T * (s / tot) * 16777216.0 + 0.5).astype(np.uint64)


def stratified_estimate(x, y, r, cnt, s, T):
    """K_s(x, y) = sum_r w_r C_r(x, y) in 2^-24 units (uint64, exact): an
    unbiased estimate of the pair count a run with weights s would draw
    (E[C_r] = (S / T) P_r and w_r 2^-24 / T = s_r up to the rounding of w_r).
    Returns (x, y, K) over the distinct pairs, sorted by (x, y)."""
    w = stratified_weights(s, T)
    n = int(max(np.max(x, initial=0), np.max(y, initial=0))) + 1
    pair = np.asarray(x, np.int64) * n + np.asarray(y, np.int64)
    up, inv = np.unique(pair, return_inverse=True)
    K = np.zeros(len(up), dtype=np.uint64)
    np.add.at(K, inv, w[np.asarray(r) - 1] * np.asarray(cnt, dtype=np.uint64))
    return up // n, up % n, K


def stratified_sparsifier(indptr, indices, T, s, S, seed, b=1.0, weights=None):
    """Eq. 1 from the stratified estimate K_s (K = fl(double(K_s)) 2^-24)."""
    n = len(indptr) - 1
    deg = weighted_degrees(indptr, weights)
    x, y, r, c = stratified_counts(indptr, indices, T, S, seed, weights=weights)
    px, py, K = stratified_estimate(x, y, r, c, s, T)
    v, keep, val = netmf_values(px, py, K, deg, S, b, unit=2.0 ** -24)
    mp, mc, mv = sparsifier_csr(n, px[keep], py[keep], val[keep])
    return dict(x=px, y=py, K=K, v=v, keep=keep, val=val, indptr=mp, indices=mc, data=mv)


# ----------------------------------------------------------------------------
# Eq. 1: from counts to the truncated-log NetMF estimate
# ----------------------------------------------------------------------------

def netmf_scale(vol: float, S: float, b: float = 1.0) -> tuple[float, float]:
    """(alpha_off, alpha_diag) with entry = alpha * K_xy / (d_x d_y).

    E[ordered count C_xy] = S/vol * [sum_r s_r D (D^-1 A)^r]_xy, so the Eq. 1
    entry vol/b * [sum_r s_r (D^-1 A)^r D^-1]_xy equals vol^2/(S b) * E[C_xy] /
    (d_x d_y). An unordered off-diagonal count K_xy = C_xy + C_yx estimates
    2 E[C_xy]; a diagonal count estimates E[C_xx].
    """
    vv = vol * vol
    return vv / ((2.0 * S) * b), vv / (S * b)


def netmf_values(x, y, cnt, deg, S, b=1.0, weighted=False, unit=None):
    """Pre-log entries v, keep mask (v > 1) and float32 trunc_log values (Eq. 1).

    v = fl(fl(K * alpha) / fl(d_x * d_y)); trunc_log(v) = max(0, log v) is zero
    unless v > 1, and zero entries are dropped from the sparse matrix. With
    ``weighted`` the counts are downsampling weight sums in 2^-32 units and
    K = fl(double(cnt)) * 2^-32; ``unit`` gives another power-of-two unit.
    """
    deg = np.asarray(deg, dtype=np.float64)
    vol = float(deg.sum())
    a_off, a_diag = netmf_scale(vol, float(S), float(b))
    alpha = np.where(x == y, a_diag, a_off)
    K = np.asarray(cnt, dtype=np.float64)
    if weighted:
        unit = 2.0 ** -32
    if unit is not None:
        K = K * unit
    v = (K * alpha) / (deg[x] * deg[y])
    keep = v > 1.0
    val = np.zeros(v.shape, dtype=np.float32)
    val[keep] = np.log(v[keep]).astype(np.float32)
    return v, keep, val


def sparsifier_csr(n, x, y, val):
    """Symmetric CSR of the kept entries: both triangles, rows sorted by column."""
    off = x != y
    rows = np.concatenate([x, y[off]])
    cols = np.concatenate([y, x[off]])
    data = np.concatenate([val, val[off]]).astype(np.float32)
    order = np.lexsort((cols, rows))
    rows, cols, data = rows[order], cols[order], data[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    return indptr, cols.astype(np.int32), data


def sparsifier(indptr, indices, T, s, S, seed, b=1.0, C=0.0, weights=None):
    """Counts -> trunc_log -> CSR. Returns a dict with every intermediate
    (with edge downsampling, C > 0, ``cnt`` holds the weight sums). On a
    weighted graph vol and the degrees of Eq. 1 are the weighted ones."""
    n = len(indptr) - 1
    deg = weighted_degrees(indptr, weights)
    x, y, cnt = sparsifier_counts(indptr, indices, T, s, S, seed, C, weights=weights)
    v, keep, val = netmf_values(x, y, cnt, deg, S, b, weighted=C > 0.0)
    mp, mc, mv = sparsifier_csr(n, x[keep], y[keep], val[keep])
    return dict(x=x, y=y, cnt=cnt, v=v, keep=keep, val=val, indptr=mp, indices=mc, data=mv)


def netmf_dense(indptr, indices, T, s, b=1.0, weights=None):
    """Eq. 1 inside the truncated log, densely: vol/b * sum_r s_r (D^-1 A)^r D^-1.

    For tiny graphs only (n <= a few hundred). ``s`` is normalised to sum 1.
    """
    n = len(indptr) - 1
    vals = np.ones(len(indices)) if weights is None else np.asarray(weights, dtype=np.float64)
    A = sp.csr_matrix((vals, indices, indptr), shape=(n, n)).toarray()
    d = A.sum(1)
    vol = d.sum()
    P = A / d[:, None]
    s = np.asarray(s, dtype=np.float64)
    s = s / s.sum()
    acc = np.zeros((n, n))
    Pr = np.eye(n)
    for r in range(1, T + 1):
        Pr = Pr @ P
        acc += s[r - 1] * Pr
    return vol / b * acc / d[None, :]


# ----------------------------------------------------------------------------
# randomized SVD (Algorithms 2 and 4)
# ----------------------------------------------------------------------------

def gaussian_sketch(n: int, c: int, seed: int) -> np.ndarray:
    """Omega = randn(n, c) (Algorithm 4) by Box-Muller from Philox words.

    Row i, column block cb = col // 4 uses the 4 words of counter (i, cb, 0, 0),
    key (seed_lo ^ 0x4f4d4547, seed_hi); words (w0, w1) give columns 4cb, 4cb+1
    and (w2, w3) give 4cb+2, 4cb+3 with u = (w + 0.5) / 2^32 and
    z = sqrt(-2 ln u_a) * (cos, sin)(2 pi u_b).
    """
    nblk = (c + 3) // 4
    words = np.zeros((n, nblk, 4), dtype=np.uint32)
    lib().oracle_sketch_words(n, nblk, int(seed), _ptr(words, ctypes.c_uint32))
    u = (words.astype(np.float64) + 0.5) / 4294967296.0
    rad = np.sqrt(-2.0 * np.log(u[:, :, 0::2]))
    ang = 2.0 * np.pi * u[:, :, 1::2]
    z = np.empty((n, nblk, 4))
    z[:, :, 0] = rad[:, :, 0] * np.cos(ang[:, :, 0])
    z[:, :, 1] = rad[:, :, 0] * np.sin(ang[:, :, 0])
    z[:, :, 2] = rad[:, :, 1] * np.cos(ang[:, :, 1])
    z[:, :, 3] = rad[:, :, 1] * np.sin(ang[:, :, 1])
    return z.reshape(n, nblk * 4)[:, :c].copy()


def floyd_subset(t_words: np.ndarray, c: int) -> np.ndarray:
    """Floyd's algorithm (Bentley & Floyd, CACM 1987) for a uniform zeta-subset
    of {0..c-1}, row-wise: step k = 0..zeta-1 takes j = c - zeta + k and
    t = word_k mod (j + 1); it adds t unless t was chosen already, else j.
    Returns the chosen columns in the order they were added ([rows, zeta])."""
    t_words = np.asarray(t_words, dtype=np.uint64)
    rows, zeta = t_words.shape
    out = np.zeros((rows, zeta), dtype=np.int64)
    for k in range(zeta):
        j = c - zeta + k
        t = (t_words[:, k] % np.uint64(j + 1)).astype(np.int64)
        taken = (out[:, :k] == t[:, None]).any(axis=1)
        out[:, k] = np.where(taken, j, t)
    return out


def sparse_sign_sketch(n: int, c: int, zeta: int, seed: int) -> np.ndarray:
    """Sparse sign test matrix Omega (n x c): row i has exactly zeta nonzeros,
    +1 or -1, at distinct columns (Sec. 4.2 names it as an alternative to
    the Gaussian Omega of Algorithm 4; the construction is that of Tropp et
    al., SISC 2019, applied to the rows of Omega so that M Omega costs zeta
    terms per nonzero of M).

    Row i reads the words of counters (i, b, 0, 0x53505253), b = 0, 1, ..., key
    (seed_lo ^ 0x4f4d4547, seed_hi), in order: words 0..zeta-1 drive Floyd's
    subset sampling (``floyd_subset``), word zeta holds the signs: the k-th
    chosen column is negative iff bit k is set. Scale 1 (the range of M Omega
    does not depend on it)."""
    nblk = (zeta + 1 + 3) // 4
    words = np.zeros((n, nblk, 4), dtype=np.uint32)
    lib().oracle_sparse_sign_words(n, nblk, int(seed), _ptr(words, ctypes.c_uint32))
    w = words.reshape(n, nblk * 4)
    cols = floyd_subset(w[:, :zeta], c)
    neg = (w[:, zeta:zeta + 1].astype(np.int64) >> np.arange(zeta)[None, :]) & 1
    Om = np.zeros((n, c))
    Om[np.arange(n)[:, None], cols] = 1.0 - 2.0 * neg
    return Om


def very_sparse_threshold(n: int, s: float = 0.0) -> int:
    """thr = floor(2^32 / (2 s)) in FP64 for the very sparse projection, s the
    sparsity (s = sqrt(n) when s <= 0, the "very sparse" choice of Li, Hastie
    and Church, KDD 2006); each entry is +1 with probability thr / 2^32 and -1
    with the same probability. Needs s >= 1."""
    s = float(s) if s > 0 else float(np.sqrt(float(n)))
    if s < 1.0:
        raise ValueError("very sparse projection needs s >= 1")
    return int(np.floor(4294967296.0 / (2.0 * s)))


def very_sparse_sketch(n: int, c: int, s: float, seed: int) -> np.ndarray:
    """Very sparse random projection Omega (n x c), Sec. 4.2's other
    alternative to the Gaussian Omega of Algorithm 4 (Li, Hastie and Church,
    KDD 2006): every entry is independently +1, 0 or -1 with probabilities
    1/(2s), 1 - 1/s, 1/(2s) (scale 1: the range of M Omega does not depend on
    the scale sqrt(s) of the original construction).

    Entry (i, j) reads word j mod 4 of counter (i, j // 4, 0, 0x56535250), key
    (seed_lo ^ 0x4f4d4547, seed_hi): +1 if word < thr, -1 if thr <= word <
    2 thr, else 0, with thr = ``very_sparse_threshold(n, s)``."""
    thr = very_sparse_threshold(n, s)
    nblk = (c + 3) // 4
    words = np.zeros((n, nblk, 4), dtype=np.uint32)
    lib().oracle_very_sparse_words(n, nblk, int(seed), _ptr(words, ctypes.c_uint32))
    w = words.reshape(n, nblk * 4)[:, :c].astype(np.int64)
    return np.where(w < thr, 1.0, np.where(w < 2 * thr, -1.0, 0.0))


def fix_signs(U: np.ndarray, *others: np.ndarray):
    """Make the largest-magnitude entry of every column of U positive (first
    index on ties) and flip the matching columns of ``others``."""
    idx = np.argmax(np.abs(U), axis=0)
    sg = np.sign(U[idx, np.arange(U.shape[1])])
    sg[sg == 0] = 1.0
    return (U * sg,) + tuple(o * sg for o in others)


def eig_svd(X: np.ndarray):
    """Algorithm 2 (eigSVD): C = X^T X; [V, D] = eig(C); S = sqrt(D); U = X V S^-1.

    Columns are returned by decreasing singular value (the algorithm's callers
    take the leading d), with the sign convention of ``fix_signs`` on U.
    """
    C = X.T @ X
    D, V = np.linalg.eigh(C)
    order = np.argsort(D)[::-1]
    D = np.maximum(D[order], 0.0)
    V = V[:, order]
    S = np.sqrt(D)
    with np.errstate(divide="ignore", invalid="ignore"):
        U = (X @ V) / S[None, :]
    U[:, S == 0] = 0.0
    U, V = fix_signs(U, V)
    return U, S, V


def spmm(indptr, indices, data, X):
    n = len(indptr) - 1
    M = sp.csr_matrix((np.asarray(data, np.float64), indices, indptr), shape=(n, X.shape[0]))
    return M @ X


def fast_randomized_svd(indptr, indices, data, d: int, q: int, oversample: int, seed: int,
                        Omega: np.ndarray | None = None, sketch: str = "gaussian", zeta: int = 8,
                        sparsity: float = 0.0):
    """Algorithm 4 (Fast Randomized SVD) on the symmetric sparse M.

    Omega = randn(n, d+s) (or, with sketch="sparse_sign", the sparse sign
    matrix with zeta nonzeros per row; with sketch="very_sparse", the very
    sparse projection of sparsity ``sparsity``, 0 = sqrt(n)); Y = M Omega; Q = eigSVD(Y).U; q times:
    Y = M Q, T = Q, [Q, Sigma, V] = eigSVD(Y); return U = Q(:, 1:d),
    Sigma(1:d), V = T V(:, 1:d). With q = 0 the eigSVD of M Omega supplies
    Sigma and V.
    """
    n = len(indptr) - 1
    c = d + oversample
    if Omega is None:
        if sketch == "sparse_sign":
            Omega = sparse_sign_sketch(n, c, zeta, seed)
        elif sketch == "very_sparse":
            Omega = very_sparse_sketch(n, c, sparsity, seed)
        else:
            Omega = gaussian_sketch(n, c, seed)
    Y = spmm(indptr, indices, data, Omega)
    Q, Sig, V = eig_svd(Y)
    T = Omega
    for _ in range(q):
        Y = spmm(indptr, indices, data, Q)
        T = Q
        Q, Sig, V = eig_svd(Y)
    U = Q[:, :d]
    Vout = T @ V[:, :d]
    return dict(U=U, sigma=Sig[:d], V=Vout, sigma_all=Sig, Q=Q, Omega=Omega)


def embedding_from_svd(U: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """X = U Sigma^{1/2} (Sec. 4.2)."""
    return U * np.sqrt(sigma)[None, :]


# ----------------------------------------------------------------------------
# spectral propagation (Sec. 4.3)
# ----------------------------------------------------------------------------

def chebyshev_coefficients(k: int, theta: float) -> np.ndarray:
    """c_0 = I_0(theta), c_i = 2 (-1)^i I_i(theta): the first k Chebyshev
    coefficients of exp(-theta y) on [-1, 1] (generating function of the
    modified Bessel functions)."""
    i = np.arange(k)
    c = 2.0 * ((-1.0) ** i) * scipy.special.iv(i, theta)
    if k > 0:
        c[0] = scipy.special.iv(0, theta)
    return c


def spectral_propagation(indptr, indices, X0: np.ndarray, k: int, theta: float, mu: float, weights=None):
    """Chebyshev spectral propagation of X0 on the graph.

    With Lap = I - D^-1 A (the paper's normalised Laplacian, Sec. 4.3) and
    Yop = 1/2 (Lap - mu I)^2 - I (spectrum inside [-1, 1]):
      F = sum_{i<k} c_i T_i(Yop) X0,  T_0 = X0, T_1 = Yop X0,
      T_{i+1} = 2 Yop T_i - T_{i-1};
      P = D^-1 A (X0 - F);  X = U_P Sigma_P^{1/2} from eigSVD(P) (Sec. 6.3).
    k = 0 turns propagation off (X = X0). Degree-0 rows of D^-1 A are zero.
    """
    n = len(indptr) - 1
    if k <= 0:
        return dict(F=None, P=None, X=X0.copy())
    vals = np.ones(len(indices)) if weights is None else np.asarray(weights, dtype=np.float64)
    A = sp.csr_matrix((vals, indices, indptr), shape=(n, n))
    deg = np.asarray(A.sum(1)).ravel()
    dinv = np.where(deg > 0, 1.0 / np.where(deg > 0, deg, 1.0), 0.0)
    DA = sp.diags(dinv) @ A

    def Lmu(X):
        return X - DA @ X - mu * X

    def Yop(X):
        return 0.5 * Lmu(Lmu(X)) - X

    c = chebyshev_coefficients(k, theta)
    T0 = X0
    F = c[0] * T0
    if k >= 2:
        T1 = Yop(X0)
        F = F + c[1] * T1
        for i in range(2, k):
            T2 = 2.0 * Yop(T1) - T0
            F = F + c[i] * T2
            T0, T1 = T1, T2
    P = DA @ (X0 - F)
    U, S, _ = eig_svd(P)
    return dict(F=F, P=P, U=U, sigma=S, X=embedding_from_svd(U, S))


# ----------------------------------------------------------------------------
# whole method
# ----------------------------------------------------------------------------

def embed(indptr, indices, T, s, S, d, q, k, theta, mu, seed, oversample=16, b=1.0, C=0.0,
          sketch="gaussian", zeta=8, weights=None, sparsity=0.0):
    """Sparsifier (edge-downsampled when C > 0, Sec. 4.1) -> randomized SVD
    (Gaussian or sparse sign test matrix, Sec. 4.2) -> X0 -> spectral
    propagation -> X."""
    sparse = sparsifier(indptr, indices, T, s, S, seed, b, C, weights=weights)
    rs = fast_randomized_svd(sparse["indptr"], sparse["indices"], sparse["data"], d, q,
                             oversample, seed, sketch=sketch, zeta=zeta, sparsity=sparsity)
    X0 = embedding_from_svd(rs["U"], rs["sigma"])
    prop = spectral_propagation(indptr, indices, X0, k, theta, mu, weights=weights)
    return dict(sparse=sparse, rsvd=rs, X0=X0, prop=prop, X=prop["X"])


def subspace_sin(U1: np.ndarray, U2: np.ndarray) -> float:
    """sin of the largest principal angle between span(U1) and span(U2)."""
    Q1, _ = np.linalg.qr(np.asarray(U1, dtype=np.float64))
    Q2, _ = np.linalg.qr(np.asarray(U2, dtype=np.float64))
    # ||(I - Q1 Q1^T) Q2||_2 is accurate for tiny angles (no 1 - cos^2 cancellation)
    R = Q2 - Q1 @ (Q1.T @ Q2)
    return float(min(1.0, np.linalg.norm(R, 2)))


# ----------------------------------------------------------------------------
# downstream objective: one-vs-rest logistic regression, Macro-F1 (Sec. 6.1)
# ----------------------------------------------------------------------------

def logreg_ovr(X: np.ndarray, Y: np.ndarray, C: float = 1.0, iters: int = 10) -> np.ndarray:
    """One-vs-rest L2-regularised logistic regression (the LIBLINEAR model of
    Sec. 6.1): for each label l, minimise 1/2 |w|^2 + C sum_i log(1 + exp(-y_il w.x_i))
    with y in {-1, +1} and a constant-1 bias feature appended to x. Solved by
    `iters` Newton steps from w = 0 (a library solve per step). Returns W of
    shape (d + 1, L)."""
    n, d = X.shape
    Xa = np.hstack([X, np.ones((n, 1))])
    L = Y.shape[1]
    W = np.zeros((d + 1, L))
    S = np.where(Y, 1.0, -1.0)
    for _ in range(iters):
        Z = Xa @ W                                   # margins
        sg = 1.0 / (1.0 + np.exp(-S * Z))            # sigma(y z)
        R = C * (sg - 1.0) * S                       # d loss / d z
        Dw = C * sg * (1.0 - sg)                     # d^2 loss / d z^2
        G = W + Xa.T @ R
        for l in range(L):
            H = np.eye(d + 1) + Xa.T @ (Xa * Dw[:, l:l + 1])
            W[:, l] -= np.linalg.solve(H, G[:, l])
    return W


def predict_topk(scores: np.ndarray, k_per_row: np.ndarray) -> np.ndarray:
    """Each row predicts its k highest-scoring labels (k = its number of true
    labels; ties broken by the lower label index)."""
    n, L = scores.shape
    order = np.lexsort((np.tile(np.arange(L), (n, 1)), -scores), axis=1)
    pred = np.zeros((n, L), dtype=bool)
    for i in range(n):
        pred[i, order[i, :k_per_row[i]]] = True
    return pred


def f1_scores(Y_true: np.ndarray, Y_pred: np.ndarray):
    """(Macro-F1, Micro-F1): F1 = 2 TP / (2 TP + FP + FN) per label (0 when the
    denominator is 0), averaged over labels; Micro-F1 pools the counts."""
    tp = np.sum(Y_true & Y_pred, axis=0).astype(np.float64)
    fp = np.sum(~Y_true & Y_pred, axis=0).astype(np.float64)
    fn = np.sum(Y_true & ~Y_pred, axis=0).astype(np.float64)
    den = 2 * tp + fp + fn
    f1 = np.where(den > 0, 2 * tp / np.where(den > 0, den, 1.0), 0.0)
    micro_den = 2 * tp.sum() + fp.sum() + fn.sum()
    micro = 2 * tp.sum() / micro_den if micro_den > 0 else 0.0
    return float(f1.mean()), float(micro)


def macro_f1(X, labels, train_idx, test_idx, C=1.0, iters=10):
    """Train on train_idx, predict test_idx with the top-k rule, return
    (Macro-F1, Micro-F1, W)."""
    labels = np.asarray(labels, dtype=bool)
    W = logreg_ovr(np.asarray(X, np.float64)[train_idx], labels[train_idx], C, iters)
    Xt = np.asarray(X, np.float64)[test_idx]
    scores = np.hstack([Xt, np.ones((len(test_idx), 1))]) @ W
    pred = predict_topk(scores, labels[test_idx].sum(1))
    ma, mi = f1_scores(labels[test_idx], pred)
    return ma, mi, W
