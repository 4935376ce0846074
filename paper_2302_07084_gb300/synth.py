"""Seeded synthetic graphs shaped like the paper's workloads.

This module only builds inputs: undirected, unweighted graphs in CSR form plus
planted labels. It holds none of the embedding method's arithmetic, so both the
CUDA path and the CPU oracle can be fed from it.

Graph families (the paper's datasets are not available, Table "Datasets
statistics" in Sec. 6.1 gives their shapes):

* ``sbm``            -- stochastic block model with equal or given block sizes.
* ``chung_lu``       -- power-law expected-degree graph (Chung-Lu), optionally with
                        overlapping planted communities that attract a fixed share
                        of the edges (a BlogCatalog-shaped graph: n=10,312,
                        m=333,983, 39 labels).

All graphs are simple: symmetric, no self-loops, no duplicate edges. CSR uses
``int64`` row pointers and ``int32`` column indices with every row sorted.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    indptr: np.ndarray          # int64 [n+1]
    indices: np.ndarray         # int32 [2m]
    labels: np.ndarray | None   # bool [n, L] multi-hot, or None
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.indices.shape[0] // 2)

    @property
    def n_arcs(self) -> int:
        return int(self.indices.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.indptr)


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR from an undirected edge list (u != v, no duplicates)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return indptr, cols.astype(np.int32)


def _unique_first(keys: np.ndarray) -> np.ndarray:
    """Distinct values of ``keys`` in order of first appearance."""
    _, first = np.unique(keys, return_index=True)
    return keys[np.sort(first)]


def _tri_index_to_pair(t: np.ndarray, s: int) -> tuple[np.ndarray, np.ndarray]:
    """Map t in [0, s(s-1)/2) to (i, j) with 0 <= j < i < s (row-major lower triangle)."""
    t = t.astype(np.int64)
    i = ((np.sqrt(8.0 * t.astype(np.float64) + 1.0) + 1.0) // 2).astype(np.int64)
    # fix rounding of the float square root
    i = np.where(i * (i - 1) // 2 > t, i - 1, i)
    i = np.where((i + 1) * i // 2 <= t, i + 1, i)
    j = t - i * (i - 1) // 2
    return i, j


def _sample_distinct(rng: np.random.Generator, population: int, k: int) -> np.ndarray:
    """k distinct integers from [0, population), in draw order."""
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    if k * 4 >= population:
        return rng.permutation(population)[:k].astype(np.int64)
    out = np.zeros(0, dtype=np.int64)
    while out.size < k:
        draw = rng.integers(0, population, size=int((k - out.size) * 1.1) + 16, dtype=np.int64)
        out = _unique_first(np.concatenate([out, draw]))
    return out[:k]


def sbm(n: int, blocks, p_in: float, p_out: float, seed: int, name: str = "sbm") -> Graph:
    """Stochastic block model.

    ``blocks`` is either a block count (equal sizes, the remainder spread over the
    first blocks) or a list of block sizes summing to n. Every unordered node pair
    within a block is an edge with probability ``p_in``, across blocks ``p_out``.
    The number of edges per block pair is drawn from the binomial law, then that
    many distinct pairs are drawn uniformly.
    """
    rng = np.random.default_rng(seed)
    if isinstance(blocks, (int, np.integer)):
        nb = int(blocks)
        sizes = [n // nb + (1 if b < n % nb else 0) for b in range(nb)]
    else:
        sizes = [int(b) for b in blocks]
    assert sum(sizes) == n
    starts = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    us, vs = [], []
    for bi in range(len(sizes)):
        for bj in range(bi, len(sizes)):
            if bi == bj:
                npairs = sizes[bi] * (sizes[bi] - 1) // 2
                p = p_in
            else:
                npairs = sizes[bi] * sizes[bj]
                p = p_out
            if npairs == 0 or p <= 0.0:
                continue
            k = int(rng.binomial(npairs, min(p, 1.0)))
            t = _sample_distinct(rng, npairs, k)
            if bi == bj:
                i, j = _tri_index_to_pair(t, sizes[bi])
                us.append(starts[bi] + i)
                vs.append(starts[bi] + j)
            else:
                us.append(starts[bi] + t // sizes[bj])
                vs.append(starts[bj] + t % sizes[bj])
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    indptr, indices = csr_from_edges(n, u, v)
    labels = np.zeros((n, len(sizes)), dtype=bool)
    for b in range(len(sizes)):
        labels[starts[b]:starts[b + 1], b] = True
    return Graph(n, indptr, indices, labels, name)


def chung_lu(n: int, m: int, gamma: float, seed: int, n_labels: int = 0,
             intra_fraction: float = 0.7, second_label_p: float = 0.3,
             i0: float = 20.0, name: str = "chung_lu") -> Graph:
    """Power-law expected-degree graph with exactly m distinct undirected edges.

    Node weights follow w_i = (i + i0)^(-1/(gamma-1)) (degree exponent gamma),
    assigned to nodes in a random order. Candidate edges pick both endpoints with
    probability proportional to w. With ``n_labels > 0`` every node gets one
    primary community drawn from Zipf(1) sizes and, with probability
    ``second_label_p``, a second distinct one; a share ``intra_fraction`` of the
    candidate edges is drawn inside a community (community chosen by its total
    weight, endpoints by w within it). Self-loops and repeats are discarded and
    candidates are drawn in batches until m distinct edges exist; the first m in
    draw order are kept.
    """
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    w = w[rng.permutation(n)]
    cum_all = np.cumsum(w)
    total_w = cum_all[-1]

    labels = None
    if n_labels > 0:
        pz = 1.0 / np.arange(1, n_labels + 1, dtype=np.float64)
        pz /= pz.sum()
        primary = rng.choice(n_labels, size=n, p=pz)
        labels = np.zeros((n, n_labels), dtype=bool)
        labels[np.arange(n), primary] = True
        has2 = rng.random(n) < second_label_p
        second = rng.choice(n_labels, size=n, p=pz)
        clash = second == primary
        second[clash] = (second[clash] + 1 + rng.integers(0, n_labels - 1, size=int(clash.sum()))) % n_labels
        labels[np.nonzero(has2)[0], second[has2]] = True
        # members of each community, concatenated, with their cumulative weights
        members = [np.nonzero(labels[:, c])[0] for c in range(n_labels)]
        seg_start = np.concatenate([[0], np.cumsum([len(x) for x in members])]).astype(np.int64)
        flat = np.concatenate(members).astype(np.int64)
        flat_cum = np.cumsum(w[flat])
        comm_w = np.array([w[x].sum() for x in members])
        comm_p = comm_w / comm_w.sum()
        comm_cum_start = np.concatenate([[0.0], flat_cum])[seg_start[:-1]]

    def draw_global(k):
        t = rng.random(k) * total_w
        return np.minimum(np.searchsorted(cum_all, t, side="right"), n - 1)

    def draw_in_comm(c):
        t = comm_cum_start[c] + rng.random(c.size) * comm_w[c]
        idx = np.searchsorted(flat_cum, t, side="right")
        idx = np.clip(idx, seg_start[c], seg_start[c + 1] - 1)
        return flat[idx]

    keys = np.zeros(0, dtype=np.int64)
    while keys.size < m:
        k = int((m - keys.size) * 1.3) + 1024
        if n_labels > 0:
            intra = rng.random(k) < intra_fraction
            u = np.empty(k, dtype=np.int64)
            v = np.empty(k, dtype=np.int64)
            ng = int((~intra).sum())
            u[~intra] = draw_global(ng)
            v[~intra] = draw_global(ng)
            c = rng.choice(n_labels, size=int(intra.sum()), p=comm_p)
            u[intra] = draw_in_comm(c)
            v[intra] = draw_in_comm(c)
        else:
            u = draw_global(k)
            v = draw_global(k)
        ok = u != v
        a = np.minimum(u[ok], v[ok])
        b = np.maximum(u[ok], v[ok])
        keys = _unique_first(np.concatenate([keys, a * n + b]))
    keys = keys[:m]
    indptr, indices = csr_from_edges(n, keys // n, keys % n)
    return Graph(n, indptr, indices, labels, name)


def ring(n: int) -> Graph:
    """Cycle graph on n >= 3 nodes (every degree 2)."""
    u = np.arange(n, dtype=np.int64)
    v = (u + 1) % n
    indptr, indices = csr_from_edges(n, u, v)
    return Graph(n, indptr, indices, None, f"ring{n}")


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    """G(n, p) as a one-block SBM."""
    g = sbm(n, 1, p, 0.0, seed, name=f"er{n}")
    g.labels = None
    return g


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

def sbm_small(seed: int = 1) -> Graph:
    """SBM, n=10,000, 4 equal blocks, p_in=0.008, p_out=0.0005 (~1.19e5 edges)."""
    return sbm(10_000, 4, 0.008, 0.0005, seed, name="sbm10k")


def blogcatalog_like(seed: int = 2) -> Graph:
    """Chung-Lu, n=10,312, m=333,983, exponent 2.1, 39 overlapping labels."""
    return chung_lu(10_312, 333_983, 2.1, seed, n_labels=39, name="blogcatalog_like")


def edge_weights(g: Graph, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integer arc weights in [lo, hi], equal on both arcs of an edge (a
    seeded hash of the unordered pair), in the graph's CSR arc order."""
    src = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(g.indptr))
    dst = np.asarray(g.indices, dtype=np.uint64)
    key = np.minimum(src, dst) * np.uint64(g.n) + np.maximum(src, dst)
    z = key + np.uint64((0x9E3779B97F4A7C15 * (seed + 1)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):   # splitmix64 finaliser, mod 2^64
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (np.uint64(lo) + z % np.uint64(hi - lo + 1)).astype(np.uint32)


def dirichlet_weights(T: int, seed: int) -> np.ndarray:
    """Window weights s_1..s_T drawn from Dirichlet(1,...,1)."""
    return np.random.default_rng(seed).dirichlet(np.ones(T))


def lollipop_tiny() -> Graph:
    """A 7-node graph with a triangle, a path and a leaf (distinct degrees)."""
    e = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 5), (4, 6), (5, 6)]
    u = np.array([a for a, _ in e]); v = np.array([b for _, b in e])
    indptr, indices = csr_from_edges(7, u, v)
    return Graph(7, indptr, indices, None, "lollipop7")


def tuning_graph(seed: int, n_max: int = 50000, blocks_max: int = 20, frac=(0.35, 0.6)) -> Graph:
    """One graph of the many-graph tuning workload: an SBM with
    n ~ U{1000..n_max}, blocks ~ U{2..blocks_max}, average degree ~ U[10, 40]
    and intra-block edge fraction ~ U[frac], all drawn from ``seed``; the
    block is each vertex's label."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1000, n_max + 1))
    nb = int(rng.integers(2, blocks_max + 1))
    deg = float(rng.uniform(10.0, 40.0))
    frac = float(rng.uniform(frac[0], frac[1]))
    size = n / nb
    p_in = min(1.0, frac * deg / max(size - 1.0, 1.0))
    p_out = min(1.0, (1.0 - frac) * deg / max(n - size, 1.0))
    return sbm(n, nb, p_in, p_out, seed, name=f"tune_sbm{seed}")


def tuning_candidates(seed: int, count: int, T: int = 10) -> list[dict]:
    """Candidate parameter sets of the tuning workload: s ~ Dirichlet(1) over T
    windows, k ~ U{3..20}, theta ~ U[0.3, 1], mu ~ U[0, 0.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(dict(s=rng.dirichlet(np.ones(T)), k=int(rng.integers(3, 21)),
                        theta=float(rng.uniform(0.3, 1.0)), mu=float(rng.uniform(0.0, 0.5))))
    return out


def chung_lu_device(n: int, m: int, gamma: float, seed: int, device="cuda", i0: float = 20.0,
                    name: str = "chung_lu_device"):
    """The Chung-Lu graph of ``chung_lu`` (no communities) generated with torch
    on a GPU, for sizes where numpy takes minutes (10M vertices, 200M edges):
    weights (i + i0)^(-1/(gamma-1)) in a seeded random order, candidate
    endpoints drawn proportionally to the weights, self-loops and repeats
    discarded, the first m distinct edges in draw order kept. Returns
    (indptr int64, indices int32) as device tensors. Seeded, but a different
    random stream from ``chung_lu``."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    w = (torch.arange(n, dtype=torch.float64, device=device) + i0) ** (-1.0 / (gamma - 1.0))
    w = w[torch.randperm(n, generator=gen, device=device)]
    cum = torch.cumsum(w, 0)
    total = float(cum[-1])
    keys = torch.zeros(0, dtype=torch.int64, device=device)
    order = torch.zeros(0, dtype=torch.int64, device=device)      # draw index of each kept key
    drawn = 0
    while keys.numel() < m:
        k = int((m - keys.numel()) * 1.3) + 1024
        u = torch.searchsorted(cum, torch.rand(k, dtype=torch.float64, generator=gen, device=device) * total,
                               right=True).clamp_(max=n - 1)
        v = torch.searchsorted(cum, torch.rand(k, dtype=torch.float64, generator=gen, device=device) * total,
                               right=True).clamp_(max=n - 1)
        ok = u != v
        a = torch.minimum(u[ok], v[ok])
        b = torch.maximum(u[ok], v[ok])
        new_keys = a * n + b
        new_order = drawn + torch.nonzero(ok).squeeze(1)
        drawn += k
        allk = torch.cat([keys, new_keys])
        allo = torch.cat([order, new_order])
        uk, inv = torch.unique(allk, return_inverse=True)
        first = torch.full((uk.numel(),), drawn, dtype=torch.int64, device=device)
        first.scatter_reduce_(0, inv, allo, reduce="amin")
        sel = torch.argsort(first)
        keys, order = uk[sel], first[sel]
        del allk, allo, uk, inv, first, sel, u, v, a, b
    keys = keys[:m]
    a, b = keys // n, keys % n
    del keys, order
    rows = torch.cat([a, b])
    cols = torch.cat([b, a])
    del a, b
    key2 = rows * n + cols
    del rows, cols
    key2 = torch.sort(key2).values
    rows = key2 // n
    indices = (key2 % n).to(torch.int32)
    del key2
    counts = torch.bincount(rows, minlength=n)
    del rows
    indptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=indptr[1:])
    return indptr, indices
