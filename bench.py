"""Benchmark: verified perturbation points per second on the 784-512-512-10 ReLU
workload (s = 6 pixels, k = 7, 15^6 = 11,390,625 points per query).

One step = one full verification of a query (prologue, screen over every point,
rechecks, FP64 pass, coverage and verdict). `value` is measured with the query
already in device memory (vbmc_verify_query_device, CUDA events on the
launching stream); `e2e` through vbmc_verify_query with host buffers plus the
device-to-host copies of the verdict bitmap and coverage masks.

The same step on the plain FP32 GPU path (no tensor cores) is timed in the same
run for the tensor precisions: `fp32_path` and the ratio `vs_fp32_path`, with a
check that both paths give identical results.

Multi-GPU (--partition): `range` (the default) splits the query's index space
into contiguous slices, one per rank, and merges the slices' results in one
exchange step (paper_1907_12933_gb300.partition: sums, min, bitwise or, joined
tie lists): strong scaling. `queries` gives each rank its own query of the same
net (independent problems, no collective on the data path): weak scaling.

--impl reference times the FP64 CPU oracle (the slow reference program) on
bounded samples of the same workload on the host cores: each step checks one
contiguous sample of the query, and the line reports those steps' own times.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "mlp784x512x512_relu_s6k7"
METRIC = "verified perturbation points/sec"
UNIT = "points/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("VBMC_BENCH_PRECISION", "bf16"))
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nq", type=int, default=512,
                    help="batched workload: number of queries (the full workload has 4096)")
    ap.add_argument("--graph", action="store_true", help="batched workload: CUDA-graph launch")
    ap.add_argument("--schedule", default="small_first", choices=["given", "small_first"],
                    help="batched workload: tile order over the queries")
    ap.add_argument("--no-coverage", action="store_true",
                    help="skip the coverage masks (verdicts only; not the headline workload)")
    ap.add_argument("--s", type=int, default=None,
                    help="override the workload's pixel count (smaller cases for profiling)")
    ap.add_argument("--k", type=int, default=None, help="override the workload's step bound")
    ap.add_argument("--queue-cap", type=int, default=1 << 27,
                    help="batched workload: capacity of each shared recheck queue (entries)")
    ap.add_argument("--train-queries", type=int, default=1500,
                    help="tile-proposal workload: selected training queries (exact labels)")
    ap.add_argument("--test-queries", type=int, default=200,
                    help="tile-proposal workload: selected held-out queries")
    ap.add_argument("--threshold", type=float, default=None,
                    help="check the misclassified literal of Eq. 11 with this reference value V "
                         "instead of the argmax property of Eq. 10")
    ap.add_argument("--filter", default="none", choices=["none", "l2", "shell", "l2+shell"],
                    help="restrict the checked points: the Euclidean ball of Eq. 9 on the grid "
                         "(--l2-max) and/or the outer k-shell")
    ap.add_argument("--l2-max", type=int, default=0,
                    help="--filter l2: largest sum of squared grey-level changes")
    ap.add_argument("--pairs", type=int, default=None,
                    help="pair-coverage workload: number of image pairs (default: the workload's)")
    ap.add_argument("--enum-covers", action="store_true",
                    help="every cover (SS, SV, DS, DV, sign changes) over the pairs (unperturbed image, "
                         "point) of the workload's box, FP64 (vbmc_enum_coverage)")
    ap.add_argument("--cover-g", type=float, default=2.0, help="value-change ratio g of the covers")
    ap.add_argument("--cover-d", type=float, default=1.0, help="distance-change bound d of the covers")
    ap.add_argument("--partition", default="range", choices=["range", "queries"],
                    help="several GPUs: split one query's index space across the ranks and merge "
                         "(range), or give each rank its own query (queries)")
    ap.add_argument("--no-fp32-arm", action="store_true",
                    help="skip timing the plain FP32 GPU path next to a tensor precision")
    return ap.parse_args()


FILTERS = {"none": 0, "l2": 1, "shell": 2, "l2+shell": 3}


def job_throughput(ms_local: float, points_local: int, world: int, device=None) -> tuple[float, int, float]:
    """Whole-job figures of a step over all ranks: the slowest rank's time (max),
    the points all ranks checked (sum) and points per second. Each rank works on
    its own query, so nothing else crosses ranks."""
    if world <= 1:
        return ms_local, points_local, points_local / (ms_local / 1000.0)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([points_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms_max, n_all = float(t.item()), int(n.item())
    return ms_max, n_all, n_all / (ms_max / 1000.0)


def rank_query(w, rank):
    cfg = w["cfg"]
    if rank == 0:
        return w["query"]
    return synth.make_query(cfg["seed"], rank, cfg["dims"][0], cfg["s"], cfg["k"])


# ---------------------------------------------------------------- CPU oracle

def oracle_rate(net, q, seconds):
    """Oracle points/s on a contiguous sample of the workload (all host cores)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = oracle.space_size(len(q["pixels"]), q["k"])
    probe = min(n, 64 * cores)
    t0 = time.perf_counter()
    oracle.verify(net, q, lo=0, hi=probe, bitmap=False)
    dt = time.perf_counter() - t0
    m = int(min(n, max(probe, probe * seconds / max(dt, 1e-6))))
    lo = (n - m) // 2
    t0 = time.perf_counter()
    oracle.verify(net, q, lo=lo, hi=lo + m, bitmap=False)
    dt = time.perf_counter() - t0
    return m / dt, cores, f"points [{lo}, {lo + m}) of query 0 ({m} of {n}), coverage on"


def oracle_steps(net, q, steps, warmup, seconds_total):
    """The reference arm: `warmup` untimed and `steps` timed steps of the FP64
    oracle on all host cores, each step one contiguous sample of the query
    (coverage on), sized so the timed steps take about seconds_total together.
    Returns (points/s, ms per step, points per step, cores, sample text)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = oracle.space_size(len(q["pixels"]), q["k"])
    probe = min(n, 64 * cores)
    for _ in range(max(1, warmup)):
        t0 = time.perf_counter()
        oracle.verify(net, q, lo=0, hi=probe, bitmap=False)
        dt = time.perf_counter() - t0
    per_step = seconds_total / max(1, steps)
    m = int(min(n, max(probe, probe * per_step / max(dt, 1e-6))))
    times, los = [], []
    for i in range(steps):
        lo = ((n - m) * (2 * i + 1)) // (2 * steps)  # samples spread over the space
        t0 = time.perf_counter()
        oracle.verify(net, q, lo=lo, hi=lo + m, bitmap=False)
        times.append(time.perf_counter() - t0)
        los.append(lo)
    rate = steps * m / sum(times)
    sample = (f"{steps} steps of {m} contiguous points of query 0 ({n} points), first at "
              f"{los[0]}, last at {los[-1]}, coverage on")
    return rate, 1000.0 * sum(times) / steps, m, cores, sample


# ------------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, device_index=0):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != device_index:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ roofline inputs

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of each pass
# of the timed step, from one ncu capture of this configuration on a GB300
# (profiles/traffic_mlp784x512x512_s6k7_bf16.md, one kernel per capture; ncu replays
# each kernel from a cold L2, so queue entries a normal step keeps in L2 count as reads).
# Keyed by (workload, precision, coverage, s, k); other configurations report null.
PROFILED_TRAFFIC = {
    ("mlp784x512x512_relu_s6k7", "bf16", True, 6, 7): {
        "screen (first pass over every point)": 1509632 + 1111808,
        "split tensor pass": 50135040 + 103168,
        "FP32 pass": 22624000 + 96000,
        "double-float pass": 2200576 + 1536,
    },
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def screen_flops_per_point(dims, s):
    """Algorithmic FLOPs of the screen per point: 2 * sum_{l>=2} H_{l-1} H_l
    (dense layers) + s * H_1 table adds (incremental layer 1)."""
    dense = sum(dims[l - 1] * dims[l] for l in range(2, len(dims)))
    return 2 * dense + s * dims[1]


def launches_per_step(precision, L, batch=False, n_points=0):
    """Kernels of the library per verify call (cudaMemset/cudaMemcpy not counted)."""
    pro = 1 + L + 1 + 1  # init, L base layers, tables, finish
    if precision == "fp8":
        # per chunk of 2^20 points: layer 1, GEMM + stats per hidden layer >= 2, output
        # layer, FP32, double-float and FP64 passes; then the final work count, stamps
        chunks = max(1, -(-n_points // (1 << 20)))
        return pro + chunks * (1 + 2 * (L - 2) + 1 + 3) + 2
    if precision == "fp64":
        return pro + 1 + 1  # FP64 range pass per query (1 here), time stamps
    if precision == "fp32":
        return pro + 4  # FP32 screen, double-float pass, FP64 pass, time stamps
    # column classes, tensor screen, [split tensor pass], FP32, double-float, FP64, stamps
    return pro + (6 if batch else 7)


def pass_rooflines(precision, dims, s, n_pts, sums, pk, pk_kind, traffic=None):
    """Roofline of each pass of a verify call (CUDA-event times from the library,
    medians over the timed steps) and, at the top level, the pass that took
    longest. Algorithmic work: 2 sum_{l>=2} H_{l-1} H_l + s H_1 FLOP per point
    that the pass evaluates, one evaluation per point in every pass (the split
    tensor pass issues three products per layer; that hardware work is reported
    beside it as hardware_flops_per_launch, not counted as the method's). Peaks: the
    measured BF16 tensor peak (FP16 the same, E4M3 twice: nominal ratios); the
    FP32 ALU peak 152 SM x 128 lanes x 2 FLOP x sm_max_mhz; double-float costs
    11 FP32 instructions per multiply-add, so its peak is the FP32 one x 2/11;
    FP64 the nominal 1.25 TFLOP/s (no measured FP64 peak)."""
    fpp = screen_flops_per_point(dims, s)
    mhz = pk.get("sm_max_mhz", 2070.0)
    alu = 152 * 128 * 2 * mhz * 1e6 / 1e12
    tensor = pk.get("bf16_tflops", 1900.0) * (2.0 if precision == "fp8" else 1.0)
    tkind = pk_kind + (" bf16 x2 (fp8 nominal ratio)" if precision == "fp8" else " bf16 burst")
    med = lambda xs: statistics.median(xs)  # noqa: E731
    last = sums[-1]
    nq = last["n_recheck"]
    first = {"fp64": ("alu", 1.25, "nominal FP64 ALU"), "fp32": ("alu", alu, "derived FP32 ALU")}.get(
        precision, ("tensor", tensor, tkind))
    rows = [("screen (first pass over every point)", med([x["ms_screen"] for x in sums]), fpp * n_pts) + first,
            ("split tensor pass", med([x["ms_pass"][0] for x in sums]), fpp * nq[0], "tensor", tensor, tkind),
            ("FP32 pass", med([x["ms_pass"][1] for x in sums]), fpp * nq[1], "alu", alu, "derived FP32 ALU"),
            ("double-float pass", med([x["ms_pass"][2] for x in sums]), fpp * nq[2], "alu", alu * 2 / 11,
             "derived FP32 ALU x 2/11"),
            ("FP64 pass", med([x["ms_pass"][3] for x in sums]), fpp * nq[3], "alu", 1.25, "nominal FP64 ALU")]
    passes, inside = [], []
    for name, ms, flops, bound, peak, kind in rows:
        if ms <= 0.0:
            continue
        if name != rows[0][0] and flops > 0 and ms < 0.01:
            # no separate time: the pass ran inside the first pass's timed region
            # (the wide-layer path rechecks each chunk's points before the next chunk)
            inside.append(name)
            continue
        ach = flops / (ms / 1000.0) / 1e12
        passes.append({"kernel": name, "launch_ms": ms, "flops_per_launch": flops, "bound": bound,
                       "achieved": ach, "peak": peak, "peak_kind": kind, "frac": ach / peak,
                       "traffic": (traffic or {}).get(name)})
        if name == "split tensor pass":
            passes[-1]["hardware_flops_per_launch"] = 3 * flops
    top = max(passes, key=lambda x: x["launch_ms"])
    roof = {"bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"], "unit": "TFLOP/s",
            "frac": top["frac"], "traffic": top["traffic"], "kernel": top["kernel"], "peak_kind": top["peak_kind"],
            "flops_per_launch": top["flops_per_launch"], "launch_ms": top["launch_ms"], "passes": passes}
    if inside:
        roof["passes_timed_in_screen"] = inside
    return roof


# -------------------------------------------------------------------- main

def main_batch(a):
    """Batched uneven queries (784-256-256-10 ReLU): one vbmc_verify_batch call per
    step over nq queries; value = all queries' points / step time; p50/p99 of the
    per-query time to a final verdict."""
    import torch
    import paper_1907_12933_gb300 as vb
    from paper_1907_12933_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    w = synth.workload(a.workload, nq=a.nq)
    net_d, cfg, qs = w["net"], w["cfg"], w["queries"]
    pts = sum((2 * q["k"] + 1) ** len(q["pixels"]) for q in qs)
    vnet = vb.Net(net_d)
    # one-time launch-shape tuning, cached next to the build (not part of a step)
    tuning = vb.autotune(vnet, os.path.join(ROOT, "paper_1907_12933_gb300", "_build", "tuning.jsonl"))
    res = vb.result_create_batch(vnet, len(qs), max_points=0, max_s=max(len(q["pixels"]) for q in qs),
                                 max_k=max(q["k"] for q in qs), queue_cap=a.queue_cap)
    for _ in range(a.warmup):
        vb.verify_batch(vnet, res, qs, precision=a.precision, coverage=True, bitmap=False,
                        graph=a.graph, schedule=a.schedule)
    clocks = Clocks()
    clocks.start()
    times, ttv = [], []
    for _ in range(a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sums = vb.verify_batch(vnet, res, qs, precision=a.precision, coverage=True, bitmap=False,
                               graph=a.graph, schedule=a.schedule)
        times.append(time.perf_counter() - t0)
        ttv = [x["ms_to_verdict"] for x in sums]
    ck = clocks.stop(torch.cuda.current_device())
    ms = 1000.0 * statistics.median(times)
    dev_ms = sums[0]["ms_device"]
    line = {"metric": METRIC, "value": pts / (dev_ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dev_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "fp16": "f16"}[a.precision],
            "data": "synthetic",
            "config": {"workload": a.workload, "dims": cfg["dims"], "queries": len(qs),
                       "points_total": pts, "s_range": cfg["s_range"], "k_range": cfg["k_range"],
                       "graph": a.graph, "precision": a.precision, "schedule": a.schedule,
                       "tuning": {k: tuning[k] for k in ("simt_range", "simt_range_ctas", "simt_gather",
                                                         "simt_gather_ctas", "df_ctas", "from_cache")}},
            "e2e": {"value": pts / (ms / 1000.0), "unit": UNIT,
                    "h2d_bytes_per_step": len(qs) * (cfg["dims"][0] + 24),
                    "d2h_bytes_per_step": len(qs) * 96},
            "time_to_verdict_ms": {"p50": float(np.percentile(ttv, 50)),
                                   "p99": float(np.percentile(ttv, 99)), "max": float(max(ttv))},
            "verdicts": {"unsafe": sum(x["verdict"] == "UNSAFE" for x in sums),
                         "safe": sum(x["verdict"] == "SAFE" for x in sums),
                         "ties_only": sum(x["verdict"] == "TIES_ONLY" for x in sums),
                         "n_recheck": [sum(x["n_recheck"][i] for x in sums) for i in range(4)]},
            # the smallest-first schedule runs min(8, queries) waves, each a full chain of passes
            "gpu_launches": a.steps * launches_per_step(a.precision, len(cfg["dims"]) - 1, batch=True)
            * (min(8, len(qs)) if a.schedule == "small_first" else 1)}
    if ck:
        line["clocks"] = ck
    print(json.dumps(line))


def main_proposal(a):
    """Learned tile proposal (784-512-512-10 ReLU net, s = 6, k = 7, 64 tiles of
    177,979 points): exact per-tile labels for the training queries, GPU training
    with early stopping, then on held-out queries that hold a witness the device
    time to the first witness with the learned tile order and with plain index
    order (vbmc_search_query; a SAFE verdict needs every tile either way)."""
    import torch
    import paper_1907_12933_gb300 as vb
    from paper_1907_12933_gb300 import build
    from paper_1907_12933_gb300 import proposal as P
    build.build()
    torch.cuda.set_device(0)
    w = synth.workload(a.workload)
    net_d, cfg = w["net"], w["cfg"]
    vnet = vb.Net(net_d)
    H0, T = cfg["dims"][0], cfg["n_tiles"]
    t0 = time.perf_counter()

    def pick(split, want):
        # candidates are drawn until `want` pass the reach filter (about 1 in 50 does)
        got_q, got_x, start = [], [], 0
        while len(got_q) < want and start < 200 * want:
            c = synth.proposal_candidates(split, 20 * want, start=start)
            X, reach, _ = P.features(vnet, c, H0)
            idx = P.select_by_reach(reach)[:want - len(got_q)]
            got_q += [c[i] for i in idx]
            got_x.append(X[torch.from_numpy(idx).cuda()].contiguous())
            start += len(c)
        return got_q, torch.cat(got_x).contiguous(), start

    qtr, Xtr, ntr_c = pick("train", a.train_queries)
    qte, Xte, nte_c = pick("test", a.test_queries)
    Ttr, ctr, lab_s = P.labels(vnet, qtr, T, precision=a.precision)
    _, cte, lab_te_s = P.labels(vnet, qte, T, precision=a.precision)
    nv = len(qtr) // 5
    prop = vb.Proposal((3 * H0, 256, 256, T), max_batch=256, seed=1)
    tt = time.perf_counter()
    hist = P.train(prop, Xtr[nv:].contiguous(), Ttr[nv:].contiguous(), Xtr[:nv].contiguous(),
                   ctr[:nv], max_epochs=24, lr=1e-3, weight_decay=1e-4, patience=4)
    train_s = time.perf_counter() - tt
    learned = P.orders(prop, Xte)
    plain = np.tile(np.arange(T), (len(qte), 1))
    unsafe = np.nonzero(cte.sum(axis=1) > 0)[0]
    sel = unsafe
    qs = [qte[i] for i in sel]
    P.search_all(vnet, qs[:a.warmup], learned[sel[:a.warmup]], precision=a.precision)
    clocks = Clocks()
    clocks.start()
    wall = {}
    res = {}
    for name, od in (("plain", plain), ("learned", learned)):
        tw = time.perf_counter()
        res[name] = P.search_all(vnet, qs, od[sel], precision=a.precision)
        wall[name] = time.perf_counter() - tw
    ck = clocks.stop(torch.cuda.current_device())

    def dist_(v):
        v = np.asarray(v, dtype=np.float64)
        return {"mean": float(v.mean()), "p50": float(np.percentile(v, 50)),
                "p90": float(np.percentile(v, 90)), "p99": float(np.percentile(v, 99))}

    ms = {n: [r["ms_to_witness"] for r in res[n]] for n in res}
    tiles = {n: [r["tiles_checked"] for r in res[n]] for n in res}
    for n in res:
        for r, i in zip(res[n], sel):
            assert r["verdict"] == "UNSAFE" and cte[i, r["witness_tile"]] > 0
    line = {"metric": "time to first witness (learned tile order)", "value": dist_(ms["learned"])["mean"],
            "unit": "ms", "n_gpus": 1, "steps": len(qs), "warmup": a.warmup,
            "ms_per_step": dist_(ms["learned"])["mean"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp64": "f64"}[a.precision],
            "data": "synthetic",
            "config": {"workload": a.workload, "dims": cfg["dims"], "s": cfg["s"], "k": cfg["k"],
                       "n_tiles": T, "proposal": [3 * H0, 256, 256, T],
                       "train_queries": len(qtr), "train_candidates": ntr_c,
                       "test_queries": len(qte), "test_candidates": nte_c,
                       "filter": "first-order reach >= 0.5",
                       "l2": "not flushed: every query's points are new work"},
            "time_to_first_witness_ms": {"learned": dist_(ms["learned"]), "plain": dist_(ms["plain"])},
            "tiles_to_first_witness": {"learned": dist_(tiles["learned"]), "plain": dist_(tiles["plain"])},
            "speedup_mean": float(np.mean(ms["plain"]) / np.mean(ms["learned"])),
            "e2e": {"value": 1000.0 * wall["learned"] / len(qs), "unit": "ms",
                    "plain": 1000.0 * wall["plain"] / len(qs),
                    "h2d_bytes_per_step": H0 + 4 * cfg["s"] + 4 * T, "d2h_bytes_per_step": 256},
            "labels": {"train_s": lab_s, "test_s": lab_te_s,
                       "train_unsafe_frac": float((ctr.sum(1) > 0).mean()),
                       "witness_tiles_mean": float((ctr > 0).sum(1).mean())},
            "training": {"seconds": train_s, "best_epoch": hist["best_epoch"],
                         "val_rank": hist["val_rank"]},
            # per search: set-up (init, L base layers, tables, finish, column classes)
            # plus 6 per checked tile (screen, split pass, FP32, double-float, FP64, stamps)
            "gpu_launches": int(sum(len(cfg["dims"]) + 3 + 6 * t for n in tiles for t in tiles[n])),
            "wall_s": time.perf_counter() - t0}
    if ck:
        line["clocks"] = ck
    print(json.dumps(line))
    prop.free()


def main_pairs(a):
    """Coverage over a dataset of image pairs (784-512-512-10 ReLU, 65,536 pairs of an
    image and a noisy copy): one vbmc_pair_coverage call per step computes every
    cover (sign change, SS, SV, DS, DV and their tie masks) ORed over all pairs.
    value: pairs/s with the pairs resident on the device; e2e: through the host
    API (pairs copied in, masks copied out, inside the timed region)."""
    over = {"n_pairs": a.pairs} if a.pairs else {}
    w = synth.workload(a.workload, **over)
    net_d, cfg = w["net"], w["cfg"]
    x1, x2 = w["pairs"]
    n = x1.shape[0]
    dims = cfg["dims"]
    fma = sum(dims[l - 1] * dims[l] for l in range(1, len(dims)))
    flops_pair = 2 * 2 * fma  # two FP64 forward passes per pair
    if a.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        rate, cores, sample = oracle_pairs_rate(net_d, x1, x2, cfg, a.cpu_seconds * max(1, a.steps) / 10.0)
        line = {"impl": "reference", "metric": "image pairs/sec (all covers)", "value": rate,
                "unit": "pairs/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": 1000.0 * n / rate, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": a.workload, "dims": dims, "pairs": n, "g": cfg["g"], "d": cfg["d"]},
                "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": rate,
                                 "unit": "pairs/s"},
                "e2e": {"value": rate, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    import torch
    import paper_1907_12933_gb300 as vb
    from paper_1907_12933_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    vnet = vb.Net(net_d)
    da = torch.from_numpy(x1).cuda()
    db = torch.from_numpy(x2).cuda()
    masks = vb.pair_masks_device(vnet)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device="cuda")
    for _ in range(a.warmup):
        vb.pair_coverage_device(vnet, da, db, masks, cfg["g"], cfg["d"])
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    for i in range(a.steps):
        flush.zero_()
        ev[i][0].record(stream)
        vb.pair_coverage_device(vnet, da, db, masks, cfg["g"], cfg["d"])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop(torch.cuda.current_device())
    ms = statistics.median([e0.elapsed_time(e1) for e0, e1 in ev])
    e2e = []
    for _ in range(max(1, min(a.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = vb.pair_coverage(vnet, x1, x2, cfg["g"], cfg["d"])
        e2e.append(time.perf_counter() - t0)
    fw, sw = vnet.mask_words()
    pk, pk_kind = peaks()
    ach = flops_pair * n / (ms / 1000.0) / 1e12
    line = {"metric": "image pairs/sec (all covers)", "value": n / (ms / 1000.0), "unit": "pairs/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "dims": dims, "pairs": n, "noise": cfg["noise"],
                       "g": cfg["g"], "d": cfg["d"], "l2": "flushed between timed steps (256 MB write)"},
            "e2e": {"value": n / statistics.median(e2e), "unit": "pairs/s",
                    "h2d_bytes_per_step": int(2 * x1.size), "d2h_bytes_per_step": int(4 * (6 * fw + 4 * sw))},
            "gpu_launches": a.steps,
            "roofline": {"bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s", "frac": ach / 1.25,
                         "traffic": None, "kernel": "k_pairs (two FP64 forward passes per pair)",
                         "peak_kind": "nominal FP64 ALU", "flops_per_launch": flops_pair * n,
                         "launch_ms": ms},
            "covers": {k: out[k + "_fraction"] for k in ("ss", "sv", "ds", "dv")}}
    if ck:
        line["clocks"] = ck
    if not a.no_cpu_baseline:
        rate, cores, sample = oracle_pairs_rate(net_d, x1, x2, cfg, a.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line))


def main_enum_covers(a):
    """Covers over the enumeration: one vbmc_enum_coverage call per step over the
    workload's query (its box, or --s/--k), every cover in FP64. value: points/s."""
    over = {key: val for key, val in (("s", a.s), ("k", a.k)) if val is not None}
    w = synth.workload(a.workload, **over)
    net_d, cfg, q = w["net"], w["cfg"], w["query"]
    s, k = len(q["pixels"]), q["k"]
    n_pts = (2 * k + 1) ** s
    dims = cfg["dims"]
    flops = 2 * sum(dims[l - 1] * dims[l] for l in range(2, len(dims))) + 2 * s * dims[1]
    if a.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        rate, cores, sample = oracle_enum_rate(net_d, q, a)
        print(json.dumps({"impl": "reference", "metric": "points/sec (all covers over the enumeration)",
                          "value": rate, "unit": "points/s", "n_gpus": a.gpus, "steps": a.steps,
                          "warmup": a.warmup, "ms_per_step": 1000.0 * n_pts / rate, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": a.workload, "dims": dims, "s": s, "k": k, "g": a.cover_g,
                                     "d": a.cover_d},
                          "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": rate,
                                           "unit": "points/s"},
                          "e2e": {"value": rate, "unit": "points/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    import torch
    import paper_1907_12933_gb300 as vb
    from paper_1907_12933_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    vnet = vb.Net(net_d)
    res = vb.Result(vnet, max_points=0, max_s=s, max_k=k)
    for _ in range(a.warmup):
        vb.enum_coverage(vnet, res, q["image"], q["pixels"], k, a.cover_g, a.cover_d)
    clocks = Clocks()
    clocks.start()
    times = []
    for _ in range(a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = vb.enum_coverage(vnet, res, q["image"], q["pixels"], k, a.cover_g, a.cover_d)
        times.append(time.perf_counter() - t0)
    ck = clocks.stop(torch.cuda.current_device())
    ms = 1000.0 * statistics.median(times)
    ach = flops * n_pts / (ms / 1000.0) / 1e12
    fw, sw = vnet.mask_words()
    line = {"metric": "points/sec (all covers over the enumeration)", "value": n_pts / (ms / 1000.0),
            "unit": "points/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "dims": dims, "s": s, "k": k, "points": n_pts, "g": a.cover_g,
                       "d": a.cover_d, "timing": "host clock around the blocking call (masks copied back)"},
            "e2e": {"value": n_pts / (ms / 1000.0), "unit": "points/s", "h2d_bytes_per_step": dims[0] + 4 * s,
                    "d2h_bytes_per_step": int(4 * (6 * fw + 4 * sw))},
            "gpu_launches": a.steps,
            "roofline": {"bound": "alu", "achieved": ach, "peak": 1.25, "unit": "TFLOP/s", "frac": ach / 1.25,
                         "traffic": None, "kernel": "k_enum_pairs (FP64 forward of each point)",
                         "peak_kind": "nominal FP64 ALU", "flops_per_launch": flops * n_pts, "launch_ms": ms},
            "covers": {key: out[key + "_fraction"] for key in ("ss", "sv", "ds", "dv")}}
    if ck:
        line["clocks"] = ck
    if not a.no_cpu_baseline:
        rate, cores, sample = oracle_enum_rate(net_d, q, a)
        line["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line))


def oracle_enum_rate(net, q, a):
    """Oracle points/s of the enumeration covers on the box's first points (one host
    thread: the oracle's pair path is sequential)."""
    import oracle
    oracle.build()
    s, k = len(q["pixels"]), q["k"]
    n = (2 * k + 1) ** s
    img = np.asarray(q["image"], np.int64)

    def pairs(lo, hi):
        xs = []
        for t in range(lo, hi):
            x = img.copy()
            for p, d in zip(q["pixels"], oracle.digits(t, s, k)):
                x[p] = min(255, max(0, x[p] + d - k))
            xs.append(x.astype(np.uint8))
        return np.repeat(img.astype(np.uint8)[None], hi - lo, 0), np.array(xs)

    x1, x2 = pairs(0, min(n, 8))
    t0 = time.perf_counter()
    oracle.pairs_coverage(net, x1, x2, a.cover_g, a.cover_d)
    dt = (time.perf_counter() - t0) / len(x1)
    m = int(min(n, max(8, a.cpu_seconds / max(dt, 1e-6))))
    x1, x2 = pairs(0, m)
    t0 = time.perf_counter()
    oracle.pairs_coverage(net, x1, x2, a.cover_g, a.cover_d)
    return m / (time.perf_counter() - t0), 1, f"points [0, {m}) of {n}, all covers"


def oracle_pairs_rate(net, x1, x2, cfg, seconds):
    """Oracle pairs/s on the first pairs of the workload (one host thread per
    forward pass: the oracle's pair path is sequential)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.pairs_coverage(net, x1[:8], x2[:8], cfg["g"], cfg["d"])
    dt = (time.perf_counter() - t0) / 8
    m = int(min(x1.shape[0], max(8, seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.pairs_coverage(net, x1[:m], x2[:m], cfg["g"], cfg["d"])
    dt = time.perf_counter() - t0
    return m / dt, 1, f"pairs [0, {m}) of {x1.shape[0]}, all covers"


def main():
    a = parse()
    if a.workload.startswith("pairs"):
        return main_pairs(a)
    if a.enum_covers:
        return main_enum_covers(a)
    if "batch" in a.workload and a.impl == "ours":
        return main_batch(a)
    if a.workload.startswith("proposal") and a.impl == "ours":
        return main_proposal(a)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    over = {key: val for key, val in (("s", a.s), ("k", a.k)) if val is not None}
    w = synth.workload(a.workload, **over)
    net_d, cfg = w["net"], w["cfg"]
    q = rank_query(w, rank)
    s, k = len(q["pixels"]), q["k"]
    n_pts = (2 * k + 1) ** s

    if a.impl == "reference":
        if rank != 0:
            return
        rate, ms_step, m, cores, sample = oracle_steps(net_d, q, a.steps, a.warmup,
                                                       a.cpu_seconds * max(1, a.steps) / 10.0)
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
                "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": ms_step, "points_per_step": m, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": a.workload, "dims": cfg["dims"], "s": s, "k": k,
                           "points_per_query": n_pts, "parallelism": "host threads",
                           "step": "one bounded contiguous sample of the query (points_per_step)"},
                "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample,
                                 "value": rate, "unit": UNIT},
                "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    else:
        torch.cuda.set_device(0)
    import paper_1907_12933_gb300 as vb
    from paper_1907_12933_gb300 import build, partition
    build.build()

    # range partition: every rank takes a contiguous slice of the same query
    split = world > 1 and a.partition == "range"
    if split:
        q = w["query"]
        lo, hi = partition.rank_range(n_pts, rank, world)
    else:
        lo, hi = 0, n_pts
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    vnet = vb.Net(net_d)
    # one-time launch-shape tuning, cached next to the build (not part of a step)
    tuning = vb.autotune(vnet, os.path.join(ROOT, "paper_1907_12933_gb300", "_build", "tuning.jsonl"))
    res = vb.Result(vnet, max_points=n_pts, max_s=s, max_k=k, ties_cap=1 << 16,
                    queue_cap=n_pts)
    d_img = torch.tensor(q["image"], dtype=torch.uint8, device=dev)
    d_pix = torch.tensor(q["pixels"], dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            dist.barrier()

    # a filter or the threshold literal needs the full query struct: those steps go
    # through vbmc_verify_query (image and pixel list, H_0 + 4 s bytes, copied in
    # on the stream inside the step)
    plain = a.threshold is None and a.filter == "none"

    def step(precision):
        if plain:
            vb.verify_query_device(vnet, res, d_img, d_pix, k, lo=lo, hi=hi, precision=precision,
                                   coverage=not a.no_coverage)
        else:
            vb.verify_query(vnet, res, q["image"], q["pixels"], k, lo=lo, hi=hi, precision=precision,
                            coverage=not a.no_coverage, filter=FILTERS[a.filter], l2_max=a.l2_max,
                            threshold=a.threshold, wait=False)

    def partial():
        """This rank's result of its slice, for the exchange step."""
        sm = vb.result_summary(res)
        out = {"n_points": sm["n_points"], "n_adv": sm["n_adversarial"], "n_ties": sm["n_ties"],
               "first_witness": sm["first_witness"], "D": sm["D"], "base_margin": sm["base_margin"],
               "bitmap": vb.get_verdict_bitmap(res, n_pts), "ties": vb.get_ties(res)}
        if not a.no_coverage:
            out.update({key: val for key, val in vb.get_coverage(res).items()
                        if key in ("flip", "flip_tie", "ss", "ss_tie")})
        return out

    def timed_steps(precision, steps):
        """CUDA-event time of each step on the launching stream (L2 flushed between
        steps), the summaries, and for a split query the exchange step's time."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        sums, merge_ms, merged = [], [], None
        barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(precision)
            ev[i][1].record(stream)
            sums.append(vb.result_summary(res))
            if split:
                t0 = time.perf_counter()
                merged = partition.merge_partials(partial(), device=dev)
                merge_ms.append(1000.0 * (time.perf_counter() - t0))
        torch.cuda.synchronize()
        barrier()
        step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        return step_ms, sums, merge_ms, merged

    # ---- device-resident steps (value)
    for _ in range(a.warmup):
        step(a.precision)
        vb.result_summary(res)
    clocks = Clocks()
    clocks.start()
    t_wall = time.perf_counter()
    step_ms, sums, merge_ms, merged = timed_steps(a.precision, a.steps)
    wall = time.perf_counter() - t_wall
    ck = clocks.stop(torch.cuda.current_device())
    ms = sum(step_ms) / len(step_ms)
    if split:  # the exchange step is part of a step of a split query
        ms += statistics.median(merge_ms)
    # points checked per step by this rank: its slice, or those that pass the filter
    n_chk = hi - lo if plain or a.filter == "none" else int(sums[-1]["n_points"])
    ms_max, n_all, value = job_throughput(ms, n_chk, world, dev)

    # ---- the plain FP32 GPU path on the same query, same timing (the metric's
    # comparison arm); its results must be identical
    fp32_arm = None
    if a.precision in ("bf16", "fp16", "fp8") and not a.no_fp32_arm:
        ref_cov = None if a.no_coverage else vb.get_coverage(res)
        ref_bm = vb.get_verdict_bitmap(res, n_pts)
        step("fp32")
        vb.result_summary(res)
        k32 = max(3, min(a.steps, 5))
        ms32, sums32, merge32, _ = timed_steps("fp32", k32)
        m32 = sum(ms32) / len(ms32) + (statistics.median(merge32) if split else 0.0)
        ms32_max, _, value32 = job_throughput(m32, n_chk, world, dev)
        a0, b0 = sums[-1], sums32[-1]
        same = all(a0[f] == b0[f] for f in ("n_adversarial", "first_witness", "n_ties", "D", "n_points"))
        same = same and np.array_equal(vb.get_verdict_bitmap(res, n_pts), ref_bm)
        if ref_cov is not None:
            cov32 = vb.get_coverage(res)
            same = same and all(np.array_equal(cov32[f], ref_cov[f]) for f in ("flip", "flip_tie", "ss", "ss_tie"))
        fp32_arm = {"value": value32, "unit": UNIT, "ms_per_step": ms32_max, "steps": k32,
                    "call": "vbmc_verify_query_device, precision fp32 (no tensor cores)",
                    "identical_results": bool(same),
                    "ms_pass": dict(zip(("split", "fp32", "double_float", "fp64"), b0["ms_pass"])),
                    "ms_screen": b0["ms_screen"], "n_recheck": b0["n_recheck"]}

    # ---- end-to-end through the host API (copies inside the timed region)
    fw, sw = vnet.mask_words()
    e2e_ms = []
    for i in range(max(1, min(a.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vb.verify_query(vnet, res, q["image"], q["pixels"], k, lo=lo, hi=hi, precision=a.precision,
                        coverage=not a.no_coverage, filter=FILTERS[a.filter], l2_max=a.l2_max,
                        threshold=a.threshold)
        if split:
            partition.merge_partials(partial(), device=dev)
        else:
            vb.get_verdict_bitmap(res, n_pts)
            if not a.no_coverage:
                vb.get_coverage(res)
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    _, _, e2e_value = job_throughput(statistics.median(e2e_ms), n_chk, world, dev)

    if rank == 0:
        last = sums[-1]
        pk, pk_kind = peaks()
        L = len(cfg["dims"]) - 1
        traffic = PROFILED_TRAFFIC.get((a.workload, a.precision, not a.no_coverage, s, k)) \
            if plain and not split else None
        roof = pass_rooflines(a.precision, cfg["dims"], s, n_chk, sums, pk, pk_kind, traffic)
        verdict = {"verdict": last["verdict"], "n_adversarial": last["n_adversarial"],
                   "first_witness": last["first_witness"], "n_ties": last["n_ties"],
                   "n_recheck": last["n_recheck"], "ms_prologue": last["ms_prologue"],
                   "ms_screen": last["ms_screen"], "ms_recheck": last["ms_recheck"],
                   "ms_pass": dict(zip(("split", "fp32", "double_float", "fp64"), last["ms_pass"]))}
        if split:  # the whole query's result after the exchange step
            verdict.update({"verdict": partition.merged_verdict(merged), "n_adversarial": merged["n_adv"],
                            "first_witness": merged["first_witness"], "n_ties": merged["n_ties"],
                            "rank0_slice": [lo, hi], "ms_exchange": statistics.median(merge_ms)})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max,
                "higher_is_better": True, "scaling": "strong" if split else "weak",
                "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "fp16": "f16",
                          "fp8": "e4m3"}[a.precision],
                "data": "synthetic",
                "config": {"workload": a.workload, "dims": cfg["dims"], "act": cfg["act"],
                           "s": s, "k": k, "points_per_query": n_pts, "precision": a.precision,
                           "coverage": not a.no_coverage,
                           "property": "Eq. 10 (argmax)" if a.threshold is None
                           else f"Eq. 11 (threshold literal, V = {a.threshold!r})",
                           "filter": a.filter, "l2_max": a.l2_max if "l2" in a.filter else None,
                           "points_checked": n_chk, "points_checked_all_ranks": n_all,
                           "value_call": "vbmc_verify_query_device" if plain
                           else "vbmc_verify_query (image and pixels copied in inside the step)",
                           "tuning": {key: tuning[key] for key in ("simt_range", "simt_range_ctas", "simt_gather",
                                                                   "simt_gather_ctas", "df_ctas", "from_cache")},
                           "queries": ("one query split into contiguous slices, one per rank, merged "
                                       "by one exchange step") if split
                           else "one per rank (rank r: query r of the workload seed)",
                           "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": (f"range split over {world} ranks" if split else f"dp{world}")
                           if world > 1 else "single GPU"},
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": int(cfg["dims"][0] + 4 * s),
                        "d2h_bytes_per_step": int(4 * ((n_pts + 31) // 32) + 8 * fw + 8 * sw + 128)},
                "gpu_launches": a.steps * launches_per_step(a.precision, L, n_points=n_pts),
                "roofline": roof,
                "verdict": verdict,
                "wall_s": wall}
        if fp32_arm:
            line["fp32_path"] = fp32_arm
            line["vs_fp32_path"] = value / fp32_arm["value"]
        if ck:
            line["clocks"] = ck
        if world == 1 and not a.no_cpu_baseline:
            rate, cores, sample = oracle_rate(net_d, q, a.cpu_seconds)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": sample}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
