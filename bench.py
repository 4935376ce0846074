"""Benchmark of the LightNE 2.0 hot path on GB300.

One step = the whole method on one graph: per-edge PathSampling -> exact pair
counts -> trunc_log CSR (Eq. 1) -> fast randomized SVD (Algorithm 4) ->
spectral propagation (Sec. 4.3). Workload: the BlogCatalog-shaped Chung-Lu
graph (n=10,312, m=333,983, exponent 2.1, 39 labels), T=10 with Dirichlet
window weights, S = 200 T m = 6.68e8 samples, d=128, q=1, k=10.

Metric: sparsifier samples per second of the whole embedding step (S divided
by the end-to-end embed time). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank embeds its own copy of the graph
(replicas; the method needs no exchange between independent problems) and
value is the total samples of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "samples/s (end-to-end embed, S=200Tm)"
WORKLOAD = "blogcatalog_like_chunglu_n10312_m333983_T10_S200Tm_d128_q1_k10"


# DRAM bytes (read + write) per launch of a kernel from one ncu capture on
# this workload, with the SHA-256 (first 16 hex digits) of the source files
# that define the kernel at the time of the capture. The figure is reported
# only while those files are unchanged; otherwise traffic is null.
RECORDED_TRAFFIC = {
    "walk_count": {"bytes": 78.70e6 + 754.08e6, "sources": ("csrc/sampler.cu", "csrc/common.cuh"),
                   "sha16": "e6d222c4b30065fe"},
}


def source_sha16(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, "paper_2302_07084_gb300", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(name):
    rec = RECORDED_TRAFFIC.get(name)
    if not rec or rec["bytes"] is None or source_sha16(rec["sources"]) != rec["sha16"]:
        return None
    return rec["bytes"]


def workload():
    from paper_2302_07084_gb300 import synth
    g = synth.blogcatalog_like(seed=2)
    s = synth.dirichlet_weights(10, seed=3)
    params = dict(T=10, s=list(s), samples=200.0 * 10 * g.m, b=1.0, d=128, oversample=16, q=1, k=10,
                  theta=0.5, mu=0.2, seed=2)
    return g, params


# ---------------------------------------------------------------------------
# per-kernel algorithmic work (bytes or flops per launch), for the roofline
# ---------------------------------------------------------------------------

def walk_ops_per_sample(params):
    """Integer lane-operations one PathSampling draw needs (algorithmic count).

    A Philox4x32-10 block is 10 rounds of 2 wide multiplies and 2 three-input
    XORs (40 ops); a draw with window r needs ceil((r + 2) / 4) blocks (words:
    r, split, coin, r - 1 steps). A walk step is a degree reduction by
    multiply-shift (4 multiplies + 1 add = 5 ops); the window lookup, split,
    pair ordering and the counter address take 12 ops per draw.
    """
    s = np.asarray(params["s"], dtype=np.float64)
    s = s / s.sum()
    r = np.arange(1, len(s) + 1)
    blocks = np.ceil((r + 2) / 4.0)
    return float(np.sum(s * (40.0 * blocks + 5.0 * (r - 1) + 12.0)))


def kernel_model(name, g, params, counts):
    """(bound, algorithmic amount per launch, unit, per-unit description) of a
    kernel, or None. The byte models count the algorithmic (compulsory) bytes:

    walk_count / walk_emit (sampling into the pair table): HBM -- 8 B per
        sample (4 B key write + 4 B key read of the aggregation; the walk's
        record reads hit L2 on this graph).
    spmm (CSR product Y = M X): HBM -- 8 B per nonzero of M (index + value)
        + one read of the dense operand row and one write of Y's row
        (c x (operand bytes + 4)) per row.
    graph_spmm: HBM -- 8 B per arc + d x 8 B per row.
    """
    S = counts["total_samples"]
    n, m2 = g.n, g.n_arcs
    c = params["d"] + params["oversample"]
    if name in ("walk_count", "walk_emit"):
        kept = counts.get("kept_draws", S)
        return "hbm", 8.0 * kept, "GB/s", "8 B per sample x samples"
    if name == "spmm":
        xb = 2 if params.get("precision", 0) == 1 else 4
        return ("hbm", 8.0 * counts.get("nnz_M", 0) + n * c * (xb + 4.0), "GB/s",
                "8 B per nonzero of M + c (operand + 4) B per row")
    if name == "graph_spmm":
        return "hbm", 8.0 * m2 + n * params["d"] * 8.0, "GB/s", "8 B per arc + 8 d B per row"
    return None


def walk_lane_ops(params, counts):
    """Integer lane-operations of the walk (a secondary, ALU view): per draw
    walk_ops_per_sample; a draw that the downsampling coin drops costs its
    head block and bookkeeping only (52)."""
    S = counts["total_samples"]
    kept = counts.get("kept_draws", S)
    return walk_ops_per_sample(params) * kept + 52.0 * (S - kept)


def expected_kept_draws(g, params):
    """Expected number of draws that survive edge downsampling: sum over arcs of
    (S / 2m) p_e, p_e = min(1, C (1/d_u + 1/d_v)) (Sec. 4.1); S without it."""
    C = params.get("downsample_C", 0.0)
    if not C:
        return params["samples"]
    deg = np.diff(g.indptr).astype(np.float64)
    src = np.repeat(np.arange(g.n), np.diff(g.indptr))
    pe = np.minimum(1.0, C * (1.0 / deg[src] + 1.0 / deg[g.indices]))
    return float(params["samples"] / g.n_arcs * pe.sum())


def alu_peak_gops(sm_count, sm_mhz):
    """Integer lane-operations per second if every one of the 4 x 32 lanes of
    each SM issued one per clock (an upper bound: the 32 x 32 -> 64 multiplies
    of Philox issue at a lower rate)."""
    return sm_count * 128 * sm_mhz * 1e6 / 1e9


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = sorted(sm)[len(sm) // 2:]   # upper half: samples under load
        return {"sm_mhz": float(statistics.median(load)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CPU oracle, timed (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

class OracleBaseline:
    """The CPU oracle timed on the workload, on the host's cores.

    Set-up (once, before any timed share) runs the oracle's sparsifier of the
    whole workload: all S draws sampled and counted (``sparsifier_counts_dense``),
    Eq. 1 values and the CSR of M; each of those stages is timed at full size.
    A timed share k of F is then a bounded, proportional piece of the whole
    workload, every part measured on the full-size data:
      * sampling + aggregation (sample_pairs + the sort-and-count of
        ``sparsifier_counts``) of the k-th of F arc ranges;
      * Eq. 1 values + CSR (netmf_values, sparsifier_csr) of the k-th of F
        ranges of the full pair list;
      * the randomized SVD's q + 1 products (oracle.spmm) of the k-th of F row
        blocks of the full M with the n x c dense operand, that block's share of
        the Gram and of U = Y V S^-1, plus the whole c x c eigensolves;
      * propagation's 2k - 1 products of the k-th row block of D^-1 A and its
        share of the last Gram.
    Shares are processed S / F samples' worth of the workload each, so a share's
    rate in samples/s is (S / F) / its time; F shares make the whole workload.
    """

    def __init__(self, g, params, F: int = 64):
        import oracle
        self.oracle = oracle
        self.g, self.p, self.F = g, params, F
        S = params["samples"]
        t0 = time.perf_counter()
        x, y, cnt = oracle.sparsifier_counts_dense(g.indptr, g.indices, params["T"], params["s"], S,
                                                   params["seed"])
        t1 = time.perf_counter()
        self.deg = g.degrees()
        v, keep, val = oracle.netmf_values(x, y, cnt, self.deg, S, params["b"])
        self.M = oracle.sparsifier_csr(g.n, x[keep], y[keep], val[keep])
        t2 = time.perf_counter()
        self.pairs = (x, y, cnt)
        self.setup = {"sampling_aggregation_s": t1 - t0, "values_csr_s": t2 - t1, "nnz_M": int(self.M[0][-1]),
                      "nnz_pairs": int(x.size)}
        c = params["d"] + params["oversample"]
        rng = np.random.default_rng(0)
        self.Xc = rng.standard_normal((g.n, c))           # stands for Omega / Q (same shape)
        self.Xd = rng.standard_normal((g.n, params["d"]))  # stands for X0 / T_i
        self.cores = oracle.num_threads()

    def share(self, k: int) -> float:
        """Run share k mod F; returns its wall time in seconds."""
        oracle, g, p, F = self.oracle, self.g, self.p, self.F
        k %= F
        n, S = g.n, p["samples"]
        t0 = time.perf_counter()
        # sampling + aggregation of arc range k
        a0, a1 = k * g.n_arcs // F, (k + 1) * g.n_arcs // F
        x, y = oracle.sample_pairs(g.indptr, g.indices, p["T"], p["s"], S, p["seed"], a0, a1)
        np.unique(x * n + y, return_counts=True)
        del x, y
        # Eq. 1 values + CSR of pair range k
        px, py, pc = self.pairs
        b0, b1 = k * px.size // F, (k + 1) * px.size // F
        v, keep, val = oracle.netmf_values(px[b0:b1], py[b0:b1], pc[b0:b1], self.deg, S, p["b"])
        oracle.sparsifier_csr(n, px[b0:b1][keep], py[b0:b1][keep], val[keep])
        # randomized SVD: q + 1 products of row block k of M, its Gram share, the eigensolves
        r0, r1 = k * n // F, (k + 1) * n // F
        ip, ix, dv = self.M
        blk_ip = ip[r0:r1 + 1] - ip[r0]
        blk_ix, blk_dv = ix[ip[r0]:ip[r1]], dv[ip[r0]:ip[r1]]
        for _ in range(p["q"] + 1):
            Yb = oracle.spmm(blk_ip, blk_ix, blk_dv, self.Xc)
            C = Yb.T @ Yb
            D, V = np.linalg.eigh(C)
            Yb @ (V / np.sqrt(np.maximum(D, 1e-300)))
        # propagation: 2k - 1 products of row block k of D^-1 A, the last Gram share
        gp = g.indptr[r0:r1 + 1] - g.indptr[r0]
        gi = g.indices[g.indptr[r0]:g.indptr[r1]]
        gv = np.repeat(1.0 / np.maximum(self.deg[r0:r1], 1), np.diff(g.indptr[r0:r1 + 1]))
        for _ in range(max(0, 2 * p["k"] - 1)):
            oracle.spmm(gp, gi, gv, self.Xd)
        Pb = oracle.spmm(gp, gi, gv, self.Xd)
        np.linalg.eigh(Pb.T @ Pb)
        return time.perf_counter() - t0

    def describe(self) -> str:
        return (f"{self.F} proportional shares of the whole workload (each: sampling+aggregation of 1/{self.F} "
                f"of the arcs, Eq. 1 values+CSR of 1/{self.F} of the pairs, the randomized SVD's products and "
                f"propagation's products on 1/{self.F} of the rows of the full-size M (nnz "
                f"{self.setup['nnz_M']}) and of D^-1 A); the full-size M was built by the oracle at set-up "
                f"(sampling+aggregation of all S draws {self.setup['sampling_aggregation_s']:.1f} s, values+CSR "
                f"{self.setup['values_csr_s']:.1f} s, measured)")


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def bench_config(g, params, world):
    """The workload's config dict, identical on both arms."""
    return {"workload": WORKLOAD, "n": g.n, "m": g.m, "samples": params["samples"], "T": params["T"],
            "d": params["d"], "q": params["q"], "k": params["k"],
            "l2": "flushed (256 MB write) between steps", "parallelism": f"replicas{world}"}


def run_reference(args):
    """The oracle on the host's cores: set-up builds the full-size sparsifier,
    then W untimed and K timed proportional shares (OracleBaseline)."""
    world, rank, _ = dist_setup(args.gpus) if int(os.environ.get("WORLD_SIZE", "1")) > 1 else (1, 0, 0)
    if rank != 0:
        return
    g, params = workload()
    t0 = time.perf_counter()
    ob = OracleBaseline(g, params)
    setup_s = time.perf_counter() - t0
    for w in range(args.warmup):
        ob.share(w)
    times = [ob.share(args.warmup + k) for k in range(args.steps)]
    ms = 1e3 * float(np.mean(times))
    v = (params["samples"] / ob.F) / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(g, params, world),
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": ob.cores, "kind": "oracle",
                             "sample": ob.describe()},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "samples_per_step": params["samples"] / ob.F, "setup_s": setup_s, "setup": ob.setup}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args.gpus)
    from paper_2302_07084_gb300 import lne
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    g, params = workload()
    params = dict(params)
    params["seed"] = params["seed"] + rank
    if args.downsample:
        params["downsample_C"] = lne.default_downsample_C(g.n)
    if args.sketch == "sparse_sign":
        params["sketch"] = lne.SKETCH_SPARSE_SIGN
    elif args.sketch == "very_sparse":
        params["sketch"] = lne.SKETCH_VERY_SPARSE
    P = lne.Params(**params)
    ctx = lne.Context(local)
    weights = None
    if args.weighted:   # integer weights 1..9 on both arcs of every edge (seeded)
        from paper_2302_07084_gb300 import synth
        weights = synth.edge_weights(g, 1, 9, seed=2)
    dg = lne.DeviceGraph(g.indptr, g.indices, device=dev, weights=weights)
    X = torch.empty((g.n, P.d), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        ctx.embed(dg, P, out=X)
    torch.cuda.synchronize()
    counts = ctx.sparsifier_counts(dg, P)
    csr = ctx.sparsifier_csr(dg, P)
    info = dict(total_samples=counts["total_samples"], nnz_c=int(counts["x"].numel()), nnz_M=int(csr["nnz"]),
                kept_draws=expected_kept_draws(g, params))
    del counts, csr
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(local)
    clocks.start()
    ctx.trace(True)
    launches0 = ctx.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.embed(dg, P, out=X)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    launches = ctx.kernel_launches() - launches0
    trace = ctx.trace_read()
    ctx.trace(False)
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)
    value = whole_job_rate(world, params["samples"], ms)

    # ---- e2e: host buffers, copies inside the timed region ----
    indptr_h = torch.from_numpy(g.indptr.astype(np.int64)).pin_memory()
    indices_h = torch.from_numpy(g.indices.astype(np.int32)).pin_memory()
    weights_h = torch.from_numpy(weights.view(np.int32)).pin_memory() if weights is not None else None
    X_h = torch.empty((g.n, P.d), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dg.indptr.copy_(indptr_h, non_blocking=True)
        dg.indices.copy_(indices_h, non_blocking=True)
        if weights_h is not None:
            dg.weights.copy_(weights_h, non_blocking=True)
        ctx.embed(dg, P, out=X)
        X_h.copy_(X, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e = max_over_ranks(float(np.mean(e2e_ms)), world, dev)

    # ---- roofline of the dominant kernel (CUDA events on the launching stream) ----
    hbm, bf16, src = read_peaks()
    dom = max(trace, key=lambda t: t["ms"])
    model = kernel_model(dom["name"], g, params, info)
    sm_mhz = clk.get("sm_mhz") or 2070.0
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    avg_s = dom["ms"] / max(1, dom["regions"]) / 1e3
    traffic = recorded_traffic(dom["name"])
    roof = {"kernel": dom["name"], "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": traffic, "avg_launch_ms": avg_s * 1e3}
    if traffic is None:
        roof["traffic_note"] = "no ncu capture of the current source of this kernel"
    if model is not None:
        bound, amount, unit, per_unit = model
        achieved = amount / avg_s / 1e9
        roof.update({"bound": bound, "achieved": achieved, "peak": hbm, "unit": unit, "frac": achieved / hbm,
                     "peak_source": f"{src}: MEASURED_PEAKS hbm_gbs (copy, burst)" if src == "measured"
                     else "fallback 6.8 TB/s", "work_per_launch": amount, "work_model": per_unit})
        if traffic is not None:
            roof["traffic_over_algorithmic"] = traffic / amount
    if dom["name"] in ("walk_count", "walk_emit"):
        ops = walk_lane_ops(params, info)
        peak_alu = alu_peak_gops(sm_count, sm_mhz)
        roof["alu"] = {"achieved": ops / avg_s / 1e9, "peak": peak_alu, "unit": "Gop/s",
                       "frac": ops / avg_s / 1e9 / peak_alu,
                       "peak_source": f"derived: {sm_count} SMs (queried) x 128 lanes x median SM clock"}
    step_total = sum(t["ms"] for t in trace if t["name"] not in ("scan_exclusive",)) / max(1, args.steps)
    breakdown = {t["name"]: round(t["ms"] / max(1, args.steps), 4) for t in trace}

    cfg = bench_config(g, params, world)
    if args.downsample or args.sketch != "gaussian" or args.weighted:
        cfg["workload"] = (WORKLOAD + ("_downsampled_C=ln_n" if args.downsample else "")
                           + ("_sparse_sign_sketch" if args.sketch == "sparse_sign" else "")
                           + ("_very_sparse_sketch" if args.sketch == "very_sparse" else "")
                           + ("_weighted_1to9" if args.weighted else ""))
        if args.downsample:
            cfg["downsample_C"] = params["downsample_C"]
    if rank == 0:
        cpu = None
        if (world == 1 and not args.no_cpu_baseline and not args.downsample and args.sketch == "gaussian"
                and not args.weighted):
            ob = OracleBaseline(g, params)
            times = [ob.share(k) for k in range(args.cpu_shares)]
            v = (params["samples"] / ob.F) / float(np.mean(times))
            cpu = {"value": v, "unit": "samples/s", "cores": ob.cores, "kind": "oracle",
                   "sample": f"{args.cpu_shares} of " + ob.describe()}
        line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg,
                "workload_stats": {"nnz_pairs": info["nnz_c"], "nnz_M": info["nnz_M"]},
                "e2e": {"value": whole_job_rate(world, params["samples"], e2e), "unit": "samples/s",
                        "h2d_bytes_per_step": int(g.indptr.nbytes + g.indices.astype(np.int32).nbytes
                                                  + (weights.nbytes if weights is not None else 0)),
                        "d2h_bytes_per_step": int(g.n * P.d * 4), "ms_per_step": e2e},
                "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "kernel_ms_per_step": breakdown}
        if world == 1 and not args.no_extras and not (args.downsample or args.weighted or args.sketch != "gaussian"):
            line.update(run_extras(args, ctx))
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_extras(args, ctx):
    """The other figures of the metric, measured after the timed region (their
    own clocks, CUDA events or wall time as stated in each): the 10M-vertex
    BF16 embedding, batched tuning against the plain loop, and the
    surrogate-guided search against the plain search. A failure is reported
    in the figure's place."""
    import copy
    import torch
    extras = {}
    jobs = [("large_graph", run_large, dict(scale=1.0, warmup=1, steps=1)),
            ("tuning", run_tune, dict(tune=16)),
            ("surrogate_search", run_surrogate, dict(surrogate=256))]
    for key, fn, over in jobs:
        a = copy.copy(args)
        for k, v in over.items():
            setattr(a, k, v)
        t0 = time.perf_counter()
        try:
            extras[key] = fn(a)
        except Exception as e:   # reported, the benchmark line still prints
            extras[key] = {"error": f"{type(e).__name__}: {e}"}
        extras[key]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return extras


def run_case(args):
    """A small, repeatable run of one stage for profilers (ncu): the bench graph
    with S / --scale samples (the dense count table keeps the footprint under
    1 GB at any S); each stage runs `--steps` times."""
    import torch
    from paper_2302_07084_gb300 import lne
    g, params = workload()
    params = dict(params)
    params["samples"] = params["samples"] / args.scale
    if args.sketch == "sparse_sign":
        params["sketch"] = lne.SKETCH_SPARSE_SIGN
    P = lne.Params(**params)
    ctx = lne.Context(0)
    dg = lne.DeviceGraph(g.indptr, g.indices)
    csr = ctx.sparsifier_csr(dg, P)
    X0 = torch.randn((g.n, P.d), device="cuda")
    for _ in range(args.steps):
        if args.case == "sparsifier":
            ctx.sparsifier_csr(dg, P)
        elif args.case == "rsvd":
            ctx.rsvd(csr, P)
        elif args.case == "propagate":
            ctx.propagate(dg, P, X0)
        elif args.case == "embed":
            ctx.embed(dg, P)
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps({"case": args.case, "steps": args.steps, "samples": params["samples"]}))


def run_tune(args):
    """Tuning throughput on the many-graph SBM suite (graph seeds 100.., 32
    candidates per graph: s ~ Dirichlet(1), k ~ U{3..20}, theta ~ U[0.3, 1],
    mu ~ U[0, 0.5], q = 1, d = 32, S = 100 m): candidates scored per second by
    lne_tune_tasks against the plain loop (lne_embed + lne_macro_f1 per
    candidate, on the first graphs only, to bound its time)."""
    import torch
    from paper_2302_07084_gb300 import lne, synth
    G, per = args.tune, 32
    graphs = [synth.tuning_graph(100 + i) for i in range(G)]
    ctx = lne.Context(0)
    tasks, cands = [], []
    for i, g in enumerate(graphs):
        idx = np.random.default_rng(100 + i).permutation(g.n)
        tasks.append((lne.DeviceGraph(g.indptr, g.indices), torch.as_tensor(g.labels).cuda(),
                      torch.as_tensor(idx[: g.n // 2]).cuda(), torch.as_tensor(idx[g.n // 2:]).cuda()))
        cands.append([lne.Params(T=10, s=list(c["s"]), samples=100.0 * g.m, b=1.0, d=32, oversample=16, q=1,
                                 k=c["k"], theta=c["theta"], mu=c["mu"], seed=100 + i)
                      for c in synth.tuning_candidates(1000 + i, per)])
    out = {"metric": "candidates/s (tuning, SBM suite, 32 candidates per graph)", "unit": "candidates/s",
           "graphs": G, "sum_n": int(sum(g.n for g in graphs)), "sum_m": int(sum(g.m for g in graphs))}
    ctx.tune_tasks(tasks[:2], cands[:2])          # warm-up: workspaces, SpMM CTA sizes
    workers = (1, 4, 8) if G <= 32 else (8,)      # large suites: the best worker count only
    for w in workers:
        ctx.set_option(lne.OPT_TUNE_WORKERS, w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ma, _ = ctx.tune_tasks(tasks, cands)
        dt = time.perf_counter() - t0
        out[f"batched_workers{w}"] = G * per / dt
    out["value"] = max(out[f"batched_workers{w}"] for w in workers)
    out["best_macro_f1_mean"] = float(ma.max(axis=1).mean())
    # window-stratified sampling: one sampling pass per graph for all 32 s
    ctx.set_option(lne.OPT_STRATIFIED, 1)
    ctx.tune_tasks(tasks[:2], cands[:2])
    for w in ((4, 8) if G <= 32 else (8,)):
        ctx.set_option(lne.OPT_TUNE_WORKERS, w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ma_s, _ = ctx.tune_tasks(tasks, cands)
        dt = time.perf_counter() - t0
        out[f"stratified_workers{w}"] = G * per / dt
    out["stratified_best_macro_f1_mean"] = float(ma_s.max(axis=1).mean())
    ctx.set_option(lne.OPT_STRATIFIED, 0)
    Gp = min(G, 2)
    for j in range(2):                             # warm-up of the plain path
        X = ctx.embed(tasks[0][0], cands[0][j])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(Gp):
        dg, lab, tr, te = tasks[i]
        for j in range(per):
            X = ctx.embed(dg, cands[i][j])
            ctx.macro_f1(X, lab, tr, te)
    dt = time.perf_counter() - t0
    out["plain"] = Gp * per / dt
    out["speedup_vs_plain"] = out["value"] / out["plain"]
    ctx.close()
    return out


def run_surrogate(args):
    """Surrogate-guided search on the SBM tuning suite (n <= 8000): the
    network is trained on the full runs of `--surrogate` graphs (32 candidates
    each), then on 16 held-out graphs the plain search (32 full runs) is timed
    against the surrogate search (rank a pool of 256 by the network, run the
    top 8); both report candidates considered per second and Macro-F1."""
    import torch
    from paper_2302_07084_gb300 import lne, search, synth
    from scipy.stats import spearmanr
    G, n_max, pool_n, top = args.surrogate, 8000, 256, 8

    def task(seed):
        g = synth.tuning_graph(seed, n_max=n_max)
        idx = np.random.default_rng(seed).permutation(g.n)
        return g, (lne.DeviceGraph(g.indptr, g.indices), torch.as_tensor(g.labels).cuda(),
                   torch.as_tensor(idx[: g.n // 2]).cuda(), torch.as_tensor(idx[g.n // 2:]).cuda())

    def cands(g, seed, count, off):
        return [lne.Params(T=10, s=list(c["s"]), samples=100.0 * g.m, d=32, oversample=16, q=1, k=c["k"],
                           theta=c["theta"], mu=c["mu"], seed=seed) for c in synth.tuning_candidates(seed + off, count)]

    ctx = lne.Context(0)
    graphs = [task(2000 + i) for i in range(G)]
    stats = [search.graph_statistics(ctx, g.indptr, g.indices, seed=1) for g, _ in graphs]
    cs = [cands(g, 2000 + i, 32, 1000) for i, (g, _) in enumerate(graphs)]
    t0 = time.perf_counter()
    scores, _ = ctx.tune_tasks([t for _, t in graphs], cs)
    t_data = time.perf_counter() - t0
    X, y = search.training_rows(cs, stats, scores)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = search.fit_surrogate(ctx, X, y, epochs=100, seed=1)
    t_train = time.perf_counter() - t0
    rows = []
    for i in range(16):
        g, t = task(9000 + i)
        st = search.graph_statistics(ctx, g.indptr, g.indices, seed=1)
        plain = cands(g, 9000 + i, 32, 1000)
        _, sc, tp = search.plain_search(ctx, t, plain)
        pool = plain + cands(g, 9000 + i, pool_n - 32, 3000)
        _, best, pred, ts = search.surrogate_search(ctx, t, st, pool, top)
        rows.append((sc.max(), best, sc[:top].max(), spearmanr(pred[:32], sc).correlation, tp, ts))
    r = np.array(rows)
    out = {"metric": "candidates/s (surrogate-guided search, SBM suite n<=8000)", "unit": "candidates/s",
           "value": 16 * pool_n / r[:, 5].sum(), "plain": 16 * 32 / r[:, 4].sum(),
           "macro_f1_plain32": float(r[:, 0].mean()), "macro_f1_surrogate": float(r[:, 1].mean()),
           f"macro_f1_first{top}": float(r[:, 2].mean()), "gap_vs_plain": float(np.mean(r[:, 0] - r[:, 1])),
           "wins_losses_vs_unguided": [int((r[:, 1] > r[:, 2]).sum()), int((r[:, 1] < r[:, 2]).sum())],
           "rank_corr": float(np.nanmean(r[:, 3])), "train_rows": int(len(y)), "train_mse": loss,
           "train_s": t_train, "data_s": t_data, "pool": pool_n, "top": top}
    out["speedup_vs_plain"] = out["value"] / out["plain"]
    ctx.close()
    return out


def _sin_angle(torch, U1, U2, lead=None):
    """sin of the largest principal angle between span(U1) and span(U2) (GPU, FP64)."""
    if lead:
        U1, U2 = U1[:, :lead], U2[:, :lead]
    Q1 = torch.linalg.qr(U1.double()).Q
    Q2 = torch.linalg.qr(U2.double()).Q
    R = Q2 - Q1 @ (Q1.T @ Q2)
    lam = torch.linalg.eigvalsh(R.T @ R)
    return float(torch.sqrt(torch.clamp(lam[-1], min=0.0)).item())


def run_large(args):
    """Large-graph precision run: Chung-Lu with 10M vertices and 200M edges
    (exponent 2.2, generated on the GPU), T = 5, s_r = 0.2, S = 5 T m = 5e9,
    d = 128, q = 2, k = 10, BF16 dense operand (FP32 accumulation, FP64-accurate
    Gram / Cholesky / small SVD). Times whole embeddings and reports per stage
    how far the BF16 operand path lands from the FP32 path at full size (the
    FP32 path's own distance to the FP64 oracle is pinned on the 10k-vertex
    SBM by the tests, and this graph's sampled draws by
    tests/test_gpu_large.py). `--scale` divides n and m."""
    import torch
    from paper_2302_07084_gb300 import lne, synth
    n, m = int(10_000_000 / args.scale), int(200_000_000 / args.scale)
    indptr, indices = synth.chung_lu_device(n, m, 2.2, seed=4)
    torch.cuda.empty_cache()      # the generator's temporaries go back to the device
    g = lne.DeviceGraph.from_tensors(indptr, indices)
    base = dict(T=5, s=[0.2] * 5, samples=5.0 * 5 * m, b=1.0, d=128, oversample=16, q=2, k=10, theta=0.5, mu=0.2,
                seed=4)
    p16 = lne.Params(**base, precision=lne.PREC_BF16_MIXED)
    p32 = lne.Params(**base, precision=lne.PREC_FP32)
    ctx = lne.Context(0)
    out = {"metric": "samples/s (large-graph embed, BF16 operand)", "unit": "samples/s",
           "config": {"workload": f"chunglu_n{n}_m{m}_gamma2.2_T5_S5Tm_d128_q2_k10_bf16", "n": n, "m": m,
                      "samples": base["samples"]}}
    for _ in range(max(1, args.warmup)):
        X = ctx.embed(g, p16)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        X = ctx.embed(g, p16)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    out.update(value=base["samples"] / (ms / 1e3), ms_per_step=ms, steps=args.steps,
               workspace_gb=ctx.workspace_bytes() / 1e9)
    ctx.trace(True)
    ctx.embed(g, p16)
    out["stage_ms"] = {r["name"]: round(r["ms"], 2) for r in ctx.trace_read()}
    ctx.trace(False)
    # per-stage distance of the BF16 path from the FP32 path
    csr = ctx.sparsifier_csr(g, p32, copy=False)
    out["config"]["nnz_M"] = csr["nnz"]
    # roofline of the products with M (q + 1 per embedding): the compulsory
    # bytes (8 B per nonzero, the BF16 operand row once,
    # the FP32 result row), and the row gathers (2 c B per nonzero) separately
    if "spmm" in out["stage_ms"]:
        hbm, _, src = read_peaks()
        c = base["d"] + base["oversample"]
        per_ms = out["stage_ms"]["spmm"] / (base["q"] + 1)
        comp = 8.0 * csr["nnz"] + n * c * (2 + 4)
        gath = 2.0 * c * csr["nnz"]
        out["spmm_roofline"] = {"bound": "hbm", "ms_per_product": per_ms, "compulsory_bytes": comp,
                                "achieved": comp / per_ms / 1e6, "peak": hbm, "unit": "GB/s",
                                "frac": comp / per_ms / 1e6 / hbm, "gather_bytes": gath,
                                "gather_gbs": gath / per_ms / 1e6, "peak_source": src}
    r32 = ctx.rsvd(csr, p32)
    r16 = ctx.rsvd(csr, p16)
    dev = {"sigma_max_rel": float(((r16["sigma"] - r32["sigma"]).abs() / r32["sigma"]).max()),
           "U_lead16_sin": _sin_angle(torch, r16["U"], r32["U"], 16),
           "U_all_sin": _sin_angle(torch, r16["U"], r32["U"])}
    X0 = r32["X0"]
    del r16, csr
    a = ctx.propagate(g, p32, X0, want_intermediates=True)
    b = ctx.propagate(g, p16, X0, want_intermediates=True)
    for k in ("F", "P"):
        dev[k + "_rel_fro"] = float(torch.linalg.norm(b[k] - a[k]) / torch.linalg.norm(a[k]))
    dev["X_lead16_sin"] = _sin_angle(torch, b["X"], a["X"], 16)
    out["bf16_vs_fp32"] = dev
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-shares", type=int, default=4, help="oracle shares timed for cpu_baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 10M-vertex, tuning and surrogate figures added to the benchmark line")
    ap.add_argument("--scale", type=float, default=10.0, help="sample-count divisor of --case runs")
    ap.add_argument("--case", choices=["sparsifier", "rsvd", "propagate", "embed"], default=None,
                    help="run one stage on a reduced workload (for profilers) instead of the benchmark")
    ap.add_argument("--tune", type=int, default=0, metavar="G",
                    help="measure tuning throughput on G graphs of the SBM suite instead of the benchmark")
    ap.add_argument("--surrogate", type=int, default=0, metavar="G",
                    help="measure surrogate-guided search after training on G graphs of the SBM suite")
    ap.add_argument("--downsample", action="store_true",
                    help="the benchmark with edge downsampling at C = ln n (draws per second; no CPU baseline)")
    ap.add_argument("--sketch", choices=["gaussian", "sparse_sign", "very_sparse"], default="gaussian",
                    help="test matrix of the randomized SVD (sparse sign: zeta = 8 nonzeros per row; "
                         "very sparse: s = sqrt(n))")
    ap.add_argument("--weighted", action="store_true",
                    help="the benchmark graph with integer edge weights 1..9 (draws per second; no CPU baseline)")
    ap.add_argument("--large", action="store_true",
                    help="the 10M-vertex BF16 precision run instead of the benchmark (--scale divides its size)")
    args = ap.parse_args()
    if args.large:
        if args.scale == 10.0 and "--scale" not in sys.argv:
            args.scale = 1.0
        print(json.dumps(run_large(args)))
    elif args.surrogate:
        print(json.dumps(run_surrogate(args)))
    elif args.tune:
        print(json.dumps(run_tune(args)))
    elif args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
