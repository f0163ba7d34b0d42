#!/usr/bin/env python
"""Throughput of the particle-filter resampling step on GB300 (one JSON line on stdout).

Workload (the paper's synthetic weight sets, Section 4.1): N = 2^20 particles, x ~ N(0,1),
log-weight -(x - y)^2/2 with y = 2; Metropolis B from Eq. (B) with eps = 1/100 and
beta = E(w)/w_max (B = 16); rejection bound log w_max = 0. One step = every resampler
(multinomial, stratified, systematic, Metropolis, rejection) in binary32 and binary64, each
followed by Permute (the paper's timing convention: until an ancestry vector satisfying the
in-place predicate is delivered, Section 4.4), plus the offspring conversions (Codes 11,
12, prefix sum and adjacent difference) of the systematic output. The metric is ancestors
delivered per second over the step.

Inputs: a pool of weight vectors per dtype, larger than L2 in total, resident in HBM; step k
uses the next five vectors of each pool, so no input is re-read from L2 across steps.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun with N > 1 ranks, each rank runs an independent replica on its own GPU
(resampling one filter does not shard); the value is the total over ranks divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workload  # noqa: E402

METRIC = "G ancestors/s per resampler at N=2^20 (FP32 vs FP64, % HBM roof); batched filters/s"
UNIT = "G ancestors/s"
SCHEME_NAMES = ["multinomial", "stratified", "systematic", "metropolis", "rejection"]
SEED = 20130115
L2_BYTES = 129 * 2**20
LAUNCH_MODES = {"auto": 0, "fused": 1, "separate": 2}  # rs_set_launch_mode


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--log2n", type=int, default=20)
    p.add_argument("--y", type=float, default=2.0)
    p.add_argument("--pool", type=int, default=40, help="weight vectors per dtype")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-filters", type=int, default=4096)
    p.add_argument("--launch-mode", choices=["auto", "fused", "separate"], default="auto",
                   help="launch structure of the scan-based schemes (results are identical)")
    p.add_argument("--sweep", action="store_true",
                   help="per-call times of the five resamplers (with Permute) for N = 2^10 .. "
                        "2^24, binary32 and binary64, L2 flushed before every call; one JSON "
                        "line")
    p.add_argument("--sweep-reps", type=int, default=21)
    p.add_argument("--sweep-y", default="0,1,2,3,4",
                   help="comma-separated y values of the sweep (weight skew)")
    p.add_argument("--precision", action="store_true",
                   help="offspring bias of the scan schemes: binary32 plain vs compensated vs "
                        "binary64, N = 2^16 .. 2^24, y in {0, 2, 4}; one JSON line")
    p.add_argument("--precision-reps", type=int, default=1000)
    p.add_argument("--metropolis-b-reps", type=int, default=400)
    p.add_argument("--smc", action="store_true",
                   help="full bootstrap SMC loop (Code 1) on the linear-Gaussian model, "
                        "N = 2^20, T = 100, systematic / Metropolis / rejection; one JSON line")
    p.add_argument("--prc", action="store_true",
                   help="partial rejection control: time, trials and outcome ESS over v_max")
    p.add_argument("--metropolis-b", action="store_true",
                   help="Metropolis time and offspring bias over B (fractions of B*)")
    p.add_argument("--accuracy", action="store_true",
                   help="the paper's accuracy experiment (Section 4.2): bias share of the MSE "
                   "and MSE / N of the five resamplers over N and y, binary32 and binary64")
    p.add_argument("--accuracy-sizes", default="4,8,12,16,18,20,22",
                   help="log2 N of the accuracy experiment")
    p.add_argument("--philox-peak", action="store_true",
                   help="measure the Philox4x32-10 throughput (rs_philox_throughput)")
    p.add_argument("--single", default=None,
                   help="profile one call: scheme:dtype[:prec], e.g. metropolis:f32 "
                        "(runs warmup + steps calls with Permute, prints one JSON line)")
    return p.parse_args()


def workload_params(args, metropolis_B=None):
    """N and the Metropolis step count of Eq. (B) (eps = 0.01, beta = E(w)/w_max). Our arm
    passes the library's rs_metropolis_B; the reference arm the oracle's."""
    if metropolis_B is None:
        import paper_1301_4019_gb300 as rs
        metropolis_B = rs.rs_metropolis_B
    N = 1 << args.log2n
    B = metropolis_B(0.01, workload.beta_estimate(args.y))
    return N, B


# ---------------------------------------------------------------------------------------
# distributed helpers (replicas; only timing is reduced)
# ---------------------------------------------------------------------------------------
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29531")
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value: float, world: int, device) -> float:
    """Maximum of a per-rank scalar over all ranks (timing only, not the data path)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_replicas(ms_local: float, units_per_rank: float, world: int, device):
    """Whole-job throughput of `world` independent replicas: every rank processed
    units_per_rank units per step; the job's step time is the slowest rank's. Returns
    (ms_per_step of the job, units per second of the job)."""
    ms = reduce_max(ms_local, world, device)
    return ms, world * units_per_rank / (ms * 1e-3)


def workload_config(args, N, B):
    """The workload both arms are measured on (the reference arm reports the same dict)."""
    return {"workload": f"N=2^{args.log2n} single filter, y={args.y}, B={B}, "
                        "5 resamplers x {f32, f64} + Permute + offspring conversions",
            "N": N, "y": args.y, "metropolis_B": B, "log_wmax": 0.0,
            "f32_prefix_sum": "plain binary32",
            "f64_prefix_sum": "double-float (two binary32, about 2^-43 per rounding) over "
                              "binary64 inputs; IEEE binary64 sums are the f64n rows",
            "parallelism": f"replicas x{max(1, args.gpus)}",
            "l2": (f"inputs rotate through a pool of {args.pool} weight vectors per dtype "
                   f"({args.pool * N * 12 / 2**20:.0f} MiB, "
                   f"{'>' if args.pool * N * 12 > L2_BYTES else '<='} L2 {L2_BYTES // 2**20} MiB)"
                   "; no flush"),
            "timing": "CUDA-graph replay of K steps, CUDA events",
            "launch_mode": args.launch_mode}


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.path = None
        self.proc = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax),
                       reasons=sorted(reasons), samples=len(sm))
        return out


# ---------------------------------------------------------------------------------------
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu launch
# capture summarised in profiles/bench_step_N2e20_launches.md (N = 2^20; ncu replays with cold
# caches). Each figure holds for the sources it was taken with: the kernel's .cu file and the
# headers it includes, hashed; `traffic` is null once any of them has changed.
# ---------------------------------------------------------------------------------------
NCU_TRAFFIC = {  # label: (bytes per launch, source hash)
    "permute": (8397926, "e733186968d7e6df"),
    "metropolis_f64": (16800695, "c46523a1c822c284"),
    "metropolis_f32": (8404544, "c46523a1c822c284"),
    "fused_multinomial_f64": (8527008, "97e0f268cecd64bc"),
    "rejection_f64": (8419657, "c46523a1c822c284"),
    "rejection_f32": (4212192, "c46523a1c822c284"),
    "fused_stratified_f64": (8512987, "97e0f268cecd64bc"),
    "permute_sorted": (4333500, "e733186968d7e6df"),
    "fused_systematic_f64": (8506295, "97e0f268cecd64bc"),
    "fused_multinomial_f32": (4351392, "97e0f268cecd64bc"),
    "fused_stratified_f32": (4331552, "97e0f268cecd64bc"),
    "iscan": (4214240, "e733186968d7e6df"),
    "fused_systematic_f32": (4326752, "97e0f268cecd64bc"),
    "search_f32": (12592032, "88475038523181d3"),
    "search_f64": (16783872, "88475038523181d3"),
    "cumoff_to_ancestors": (4204688, "e733186968d7e6df"),
    "offspring": (8391520, "e733186968d7e6df"),
    "fill": (8437, "e733186968d7e6df"),
    "adjacent_difference": (4198432, "e733186968d7e6df"),
    "sidecar": (8394167, "c46523a1c822c284")}

_LABEL_FILES = (("fused_", "fused.cu"), ("permute", "aux.cu"), ("iscan", "aux.cu"),
                ("fill", "aux.cu"), ("offspring", "aux.cu"), ("adjacent", "aux.cu"),
                ("cumoff", "aux.cu"), ("metropolis", "mcmc.cu"), ("rejection", "mcmc.cu"),
                ("prc_", "mcmc.cu"), ("sidecar", "mcmc.cu"), ("max_", "scan.cu"), ("tile_sum", "scan.cu"),
                ("emit_", "scan.cu"), ("search_", "scan.cu"))


def kernel_source_hash(label: str):
    """Hash of the .cu file that defines the kernel behind a traced label and of every
    header it includes (transitively)."""
    import hashlib
    import re
    src = next((f for pre, f in _LABEL_FILES if label.startswith(pre)), None)
    if src is None:
        return None
    csrc = os.path.join(ROOT, "paper_1301_4019_gb300", "csrc")
    seen, todo = set(), [os.path.join(csrc, src)]
    while todo:
        path = os.path.normpath(todo.pop())
        if path in seen or not os.path.exists(path):
            continue
        seen.add(path)
        text = open(path, "rb").read()
        for inc in re.findall(rb'#include "([^"]+)"', text):
            todo.append(os.path.join(os.path.dirname(path), inc.decode()))
    h = hashlib.sha256()
    for path in sorted(seen):
        h.update(os.path.basename(path).encode())
        h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(label: str, N: int):
    entry = NCU_TRAFFIC.get(label)
    if N != 1 << 20 or entry is None or kernel_source_hash(label) != entry[1]:
        return None
    return entry[0]


# ---------------------------------------------------------------------------------------
# algorithmic bytes / operations per kernel launch (roofline numerators)
# ---------------------------------------------------------------------------------------
def rejection_expected_draws(w):
    """Expected attempts and binary32 Philox blocks of one rejection call with weights w
    (w_max = 1): particle i's attempt count T is 1 with probability w_i (attempt 0 proposes
    i itself), else 1 + a geometric count of attempts that accept with p = mean(w). Binary32
    attempts 2m, 2m + 1 share one block, so a particle draws ceil(T / 2) blocks:
    E ceil(T / 2) = w_i + (1 - w_i) (1 + q / (1 - q^2)), q = 1 - p."""
    w = np.asarray(w, dtype=np.float64)
    p = w.mean()
    q = 1.0 - p
    attempts = int(len(w) + np.sum(1.0 - w) / p)
    blocks = int(np.sum(w + (1.0 - w) * (1.0 + q / (1.0 - q * q))))
    return attempts, blocks


def kernel_roofline_units(label: str, N: int, B: int):
    """(bound, algorithmic amount per launch, unit) for a traced kernel label."""
    S = 8 if ("_f64" in label) else 4
    V = 8 if ("_f64" in label or label.endswith("_f32c")) else 4
    # the per-particle figures of the path (2S + 4, + 16 for Permute) split over its kernels
    if label.startswith("fused_systematic_") or label.startswith("fused_stratified_"):
        return "hbm", (2 * S + 4) * N, "B"        # two reads of logw, write a
    if label.startswith("fused_multinomial_"):
        return "hbm", (2 * S + V) * N, "B"        # two reads of logw, write W
    if label.startswith("max_") or label.startswith("tile_sum_"):
        return "hbm", S * N, "B"
    if label.startswith("emit_systematic_") or label.startswith("emit_stratified_"):
        return "hbm", S * N + 8 * N, "B"           # read logw, write a and the claims d
    if label.startswith("emit_W_"):
        return "hbm", S * N + V * N, "B"           # read logw, write W
    if label.startswith("search_"):
        return "hbm", V * N + 4 * N, "B"           # read W once, write a
    if label.startswith("metropolis_f32"):
        return "alu", (B + 1) // 2 * N, "Philox"   # one Philox4x32-10 block per two steps
    if label.startswith("metropolis_"):
        return "alu", B * N, "Philox"              # one Philox4x32-10 block per step
    if label.startswith("rejection_"):
        return "alu", None, "Philox"
    if label in ("permute", "permute_sorted"):
        return "hbm", 16 * N, "B"                  # the claims d written and read, read a, write c
    if label == "fill":
        return "hbm", 4 * N, "B"
    if label == "offspring":
        return "hbm", 12 * N, "B"                  # read a, read-modify-write o
    if label.startswith("iscan"):
        return "hbm", 8 * N, "B"                   # read o, write O
    if label == "adjacent_difference":
        return "hbm", 8 * N, "B"                   # read O, write o
    if label == "cumoff_to_ancestors":
        return "hbm", 12 * N, "B"                  # read O, write a (and the neighbour read)
    return "hbm", None, "B"


# ---------------------------------------------------------------------------------------
# boundary mismatches of the scan-based resamplers against the oracle (after the timed
# regions, on rank 0; the oracle is the checker, never on the measured path)
# ---------------------------------------------------------------------------------------
SCAN_MODES = (("f32", "f32", 0, (0, 1)), ("f32c", "f32", 1, (1,)), ("f64", "f64", 0, (0, 1)),
              ("f64n", "f64", 2, (0, 1)))


def scan_mismatches(rs, h, lw_by_name, N, seed=SEED):
    """For every scan-based scheme and accumulation mode, one call's ancestors at the bench's
    N against the oracle: positions that differ, how many of them lie within the rounding
    bound of a cumulative-weight boundary (counted) and how many do not (must be 0), against
    the sequential oracle in the call's own precision and the double-double one; for plain
    binary32 also the largest offset of the cumulative offspring from the double-double
    oracle's and the bound it must stay within (the boundary rule alone accepts every position
    from about N = 2^18 in binary32)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_tools import cumulative_mismatches, multinomial_mismatches, truth_offset
    oracle.build()
    out = {}
    for kind, pname, prec, oprecs in SCAN_MODES:
        lw_t = lw_by_name[pname]
        lw = lw_t.cpu().numpy()
        for s in (0, 1, 2):  # multinomial, stratified, systematic
            a = rs.rs_resample(h, s, lw_t, seed=seed, prec=prec).cpu().numpy()
            entry = {}
            O_k = None if s == 0 else np.cumsum(np.bincount(a, minlength=N))
            for op in oprecs:
                if s == 0:
                    _, a_o = oracle.multinomial(lw, seed, prec=op)
                    n, bad = multinomial_mismatches(kind, lw, a, a_o, seed,
                                                    oracle_is_sequential=(op == 0))
                else:
                    f = oracle.stratified if s == 1 else oracle.systematic
                    _, O_o, _ = f(lw, seed, prec=op)
                    n, bad = cumulative_mismatches(kind, s, lw, O_k, O_o, seed,
                                                   oracle_is_sequential=(op == 0))
                entry["vs_sequential" if op == 0 else "vs_exact"] = {
                    "differ": int(n), "near_boundary": int(n - bad), "unexplained": int(bad)}
            if s != 0 and kind == "f32":
                dev, bound = truth_offset(kind, s, lw, O_k, seed)
                entry["max_offset_vs_exact"] = dev
                entry["offset_bound"] = bound
            out[f"{SCHEME_NAMES[s]}_{kind}"] = entry
    st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after the mismatch calls: {rs.rs_strerror(st)}")
    return out


def precision_mode_rows(rs, h, pools, N, hbm_peak, reps=21):
    """Per-call time (with Permute) of the scan-based schemes in the compensated binary32 and
    IEEE binary64 modes, which the timed step does not contain; inputs rotate through the
    pools as in the step; median of `reps` calls, each between CUDA events on the stream."""
    import torch
    rows = {}
    out = torch.empty(N, dtype=torch.int32, device=pools["f32"][0].device)
    for kind, pname, prec in (("f32c", "f32", 1), ("f64n", "f64", 2)):
        S = 4 if pname == "f32" else 8
        for s in (0, 1, 2):
            ts = []
            for k in range(reps + 3):
                lw = pools[pname][k % len(pools[pname])]
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                rs.rs_resample(h, s, lw, seed=SEED, step=k, out=out, permute=True, prec=prec)
                e1.record()
                torch.cuda.synchronize()
                if k >= 3:
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            rows[f"{SCHEME_NAMES[s]}_{kind}"] = {
                "ms": round(ms, 5), "G_ancestors_per_s": round(N / (ms * 1e-3) / 1e9, 3),
                "hbm_frac": round(sweep_hbm_bytes(s, S, N) / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                "timing": "single call between events (not in the timed step)"}
    return rows


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def measure_philox_peak(rs, h, draws_per_thread: int = 1024, reps: int = 5) -> dict:
    """The Philox4x32-10 throughput of this GPU (rs_philox_throughput: 2048 threads per SM,
    each drawing `draws_per_thread` blocks; median of `reps` launches timed with CUDA events),
    the peak of the Philox-bound kernels (Metropolis, rejection), beside the figure derived
    from unit counts (SMs x maximum SM clock x 32 IMAD.WIDE per clock / 20 per draw; the
    clock from MEASURED_PEAKS.json, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(h.device).multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    ghz = (float(json.load(open(peaks_path)).get("sm_max_mhz", 2070.0))
           if os.path.exists(peaks_path) else 2070.0) / 1000.0
    threads = sms * 2048
    out = torch.empty(1, dtype=torch.int32, device=torch.device("cuda", h.device))
    for _ in range(2):
        rs.rs_philox_throughput(h, threads, draws_per_thread, seed=1, out=out)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rs.rs_philox_throughput(h, threads, draws_per_thread, seed=1, out=out)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    return {"measured_G_per_s": round(threads * draws_per_thread / (ms * 1e-3) / 1e9, 1),
            "derived_G_per_s": round(sms * ghz * 32 / 20, 1), "sms": sms,
            "threads": threads, "draws_per_thread": draws_per_thread,
            "ms_per_launch": round(ms, 4)}


def run_ours(args):
    import torch
    import paper_1301_4019_gb300 as rs

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    N, B = workload_params(args)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    R = max(5, args.pool - args.pool % 5)
    dtypes = [("f32", np.float32, torch.float32), ("f64", np.float64, torch.float64)]
    pools = {}
    for name, npdt, _ in dtypes:
        pools[name] = [torch.from_numpy(workload.synthetic_logw(N, args.y, seed=SEED + 1000 * r,
                                                                dtype=npdt)).to(dev)
                       for r in range(R)]
    pool_bytes = sum(t.numel() * t.element_size() for p in pools.values() for t in p)
    outs = {name: [torch.empty(N, dtype=torch.int32, device=dev) for _ in range(5)]
            for name, _, _ in dtypes}
    conv = {name: [torch.empty(N, dtype=torch.int32, device=dev) for _ in range(4)]
            for name, _, _ in dtypes}
    h = rs.Handle(N)
    philox = measure_philox_peak(rs, h)
    rs.rs_set_launch_mode(h, LAUNCH_MODES[args.launch_mode])

    def step(k):
        for name, _, _ in dtypes:
            for s in range(5):
                lw = pools[name][(5 * k + s) % R]
                rs.rs_resample(h, s, lw, B=B, seed=SEED, step=k, out=outs[name][s],
                               permute=True, log_wmax=0.0)
        for name, _, _ in dtypes:
            o, O, o2, a2 = conv[name]
            rs.rs_offspring(h, outs[name][rs.SYSTEMATIC], o)
            rs.rs_cumulative_offspring(h, o, O)
            rs.rs_adjacent_difference(h, O, o2)
            rs.rs_cumulative_offspring_to_ancestors(h, O, a2)

    ancestors_per_step = 2 * 5 * N
    stream = torch.cuda.current_stream()

    # --- warm-up (direct launches), status check --------------------------------------
    for k in range(args.warmup):
        step(k)
    st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after warm-up: {rs.rs_strerror(st)}")

    # --- capture one CUDA graph per distinct pool position -----------------------------
    period = R // 5
    graphs = []
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(stream)
    with torch.cuda.stream(cap_stream):
        for p in range(period):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap_stream):
                step(p)
            graphs.append(g)
    stream.wait_stream(cap_stream)
    for g in graphs:
        g.replay()
    torch.cuda.synchronize()

    # --- timed region: K graph replays back to back ------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    e0.record()
    for k in range(args.steps):
        graphs[k % period].replay()
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    ms_total = e0.elapsed_time(e1)
    st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after timed region: {rs.rs_strerror(st)}")
    # a timed region shorter than a second gives the 100 ms clock sampler few samples: the
    # same graphs keep replaying (untimed) until the sampled window covers a second of work
    extra = 0
    while time.perf_counter() - wall0 < 1.0 and extra < 100000:
        for k in range(args.steps):
            graphs[k % period].replay()
        torch.cuda.synchronize()
        extra += args.steps
    clock_window_s = time.perf_counter() - wall0

    # --- traced steps: per-kernel durations on the launching stream ---------------------
    n_ev = 256
    ev_sets = []
    for k in range(args.steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        for e in evs:
            e.record()
        ev_sets.append(evs)
    torch.cuda.synchronize()
    labels_per_step = None
    durations = {}
    t_traced0 = torch.cuda.Event(enable_timing=True)
    t_traced1 = torch.cuda.Event(enable_timing=True)
    t_traced0.record()
    for k in range(args.steps):
        rs.rs_trace(h, ev_sets[k])
        step(k)
        labels = rs.rs_trace_labels(h)
        rs.rs_trace(h, [])
        if labels_per_step is None:
            labels_per_step = labels
    t_traced1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_traced_total = t_traced0.elapsed_time(t_traced1)
    # kernel order inside a step is the same for every step
    call_of = []
    call_idx = 0
    for lab in labels_per_step:
        call_of.append(call_idx)
        if lab == "end":
            call_idx += 1
    for k in range(args.steps):
        evs = ev_sets[k]
        for i, lab in enumerate(labels_per_step[:-1]):
            if lab == "end":
                continue
            durations.setdefault((call_of[i], lab), []).append(evs[i].elapsed_time(evs[i + 1]))
    gpu_launches_per_step = sum(1 for lab in labels_per_step if lab != "end")

    # per kernel label totals
    by_label = {}
    for (_, lab), ds in durations.items():
        by_label.setdefault(lab, []).extend(ds)
    total_kernel_ms = sum(sum(v) for v in by_label.values())
    dom_label = max(by_label, key=lambda lab: sum(by_label[lab]))
    dom_ms = statistics.mean(by_label[dom_label])
    launches_per_step_dom = len(by_label[dom_label]) / args.steps
    bound, amount, unit = kernel_roofline_units(dom_label, N, B)
    # rejection: expected attempts per call N + sum_i (1 - w_i/w_max) / p, p = mean(w)/w_max
    # (w_max = 1: log w_max = 0), one Philox draw each
    w = np.exp(pools["f64"][0].double().cpu().numpy())
    rej_attempts, rej_blocks_f32 = rejection_expected_draws(w)
    if dom_label.startswith("rejection_"):
        amount = rej_blocks_f32 if dom_label.startswith("rejection_f32") else rej_attempts
    if bound == "hbm":
        achieved = amount / (dom_ms * 1e-3) / 1e9 if amount is not None else None
        roof = {"bound": "hbm", "kernel": dom_label,
                "achieved": round(achieved, 1) if achieved is not None else None,
                "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4) if achieved is not None else None,
                "peak_source": peak_src, "traffic": ncu_traffic(dom_label, N),
                "traffic_note": "ncu dram bytes per launch, cold-cache replay (profiles/)",
                "algorithmic_bytes_per_launch": amount}
    else:
        achieved = (amount or 0) / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": dom_label, "achieved": round(achieved, 1),
                "peak": philox["measured_G_per_s"], "unit": "G Philox/s",
                "frac": round(achieved / philox["measured_G_per_s"], 4),
                "peak_source": "measured (rs_philox_throughput)",
                "traffic": ncu_traffic(dom_label, N),
                "traffic_note": "ncu dram bytes per launch, cold-cache replay (profiles/)"}
    roof["share_of_step"] = round(sum(by_label[dom_label]) / total_kernel_ms, 4)
    roof["avg_launch_ms"] = round(dom_ms, 5)

    per_kernel = {lab: {"mean_us": round(1e3 * statistics.mean(ds), 2),
                        "launches_per_step": round(len(ds) / args.steps, 2),
                        "share": round(sum(ds) / total_kernel_ms, 4)}
                  for lab, ds in sorted(by_label.items(), key=lambda kv: -sum(kv[1]))}
    for lab, v in per_kernel.items():  # the Philox-bound kernels against the measured peak
        b, amt, _ = kernel_roofline_units(lab, N, B)
        if lab.startswith("rejection_"):
            amt = rej_blocks_f32 if lab.startswith("rejection_f32") else rej_attempts
            v["expected_trials_per_particle"] = round(rej_attempts / N, 3)
        if b == "alu" and amt:
            v["philox_frac"] = round(amt / (v["mean_us"] * 1e-6) / 1e9
                                     / philox["measured_G_per_s"], 4)

    # per resampler breakdown: sum of the kernels of each resample call
    per_call = {}
    for (ci, lab), ds in durations.items():
        per_call.setdefault(ci, {})[lab] = statistics.mean(ds)
    per_scheme = {}
    ci = 0
    for name, _, _ in dtypes:
        for s in range(5):
            t_ms = sum(per_call.get(ci, {}).values())
            S = 4 if name == "f32" else 8
            per_scheme[f"{SCHEME_NAMES[s]}_{name}"] = {
                "ms": round(t_ms, 5), "G_ancestors_per_s": round(N / (t_ms * 1e-3) / 1e9, 3),
                "hbm_frac": round(sweep_hbm_bytes(s, S, N) / (t_ms * 1e-3) / 1e9 / hbm_peak, 4)}
            ci += 1

    ms_per_step, value = aggregate_replicas(ms_total / args.steps, ancestors_per_step, world,
                                            dev)
    value /= 1e9

    # --- end-to-end through the public API with pinned host buffers ---------------------
    # Every call's log-weights are copied in from pinned host memory and its ancestors
    # copied back, each step. The copies run on their own streams and overlap the kernels of
    # neighbouring calls (two device buffers per dtype; events order every buffer reuse).
    host_in = {name: [torch.from_numpy(workload.synthetic_logw(
        N, args.y, seed=SEED + 7 + s, dtype=npdt)).pin_memory() for s in range(5)]
        for name, npdt, _ in dtypes}
    host_out = {name: [torch.empty(N, dtype=torch.int32).pin_memory() for _ in range(5)]
                for name, _, _ in dtypes}
    dev_in = {name: [torch.empty(N, dtype=tdt, device=dev) for _ in range(2)]
              for name, _, tdt in dtypes}
    dev_out = {name: [torch.empty(N, dtype=torch.int32, device=dev) for _ in range(2)]
               for name, _, _ in dtypes}
    s_h2d, s_cmp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = {(kind, name, b): torch.cuda.Event() for kind in ("h2d", "cmp", "d2h")
          for name, _, _ in dtypes for b in range(2)}
    slot = {name: 0 for name, _, _ in dtypes}

    def e2e_step(k):
        for name, _, _ in dtypes:
            for s in range(5):
                b = slot[name]
                slot[name] ^= 1
                s_h2d.wait_event(ev[("cmp", name, b)])      # the buffer's last reader is done
                with torch.cuda.stream(s_h2d):
                    dev_in[name][b].copy_(host_in[name][s], non_blocking=True)
                ev[("h2d", name, b)].record(s_h2d)
                s_cmp.wait_event(ev[("h2d", name, b)])
                s_cmp.wait_event(ev[("d2h", name, b)])      # the output buffer was copied out
                rs.rs_resample(h, s, dev_in[name][b], B=B, seed=SEED, step=k,
                               out=dev_out[name][b], permute=True, log_wmax=0.0, stream=s_cmp)
                if s == rs.SYSTEMATIC:  # the step's conversions, as in the timed graph
                    o, O, o2, a2 = conv[name]
                    rs.rs_offspring(h, dev_out[name][b], o, stream=s_cmp)
                    rs.rs_cumulative_offspring(h, o, O, stream=s_cmp)
                    rs.rs_adjacent_difference(h, O, o2, stream=s_cmp)
                    rs.rs_cumulative_offspring_to_ancestors(h, O, a2, stream=s_cmp)
                ev[("cmp", name, b)].record(s_cmp)
                s_d2h.wait_event(ev[("cmp", name, b)])
                with torch.cuda.stream(s_d2h):
                    host_out[name][s].copy_(dev_out[name][b], non_blocking=True)
                ev[("d2h", name, b)].record(s_d2h)

    def e2e_drain():
        for key, e in ev.items():
            if key[0] == "d2h":
                s_cmp.wait_event(e)

    for k in range(max(1, args.warmup)):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier(world)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(s_cmp)
    s_h2d.wait_event(f0)
    s_d2h.wait_event(f0)
    for k in range(args.steps):
        e2e_step(k)
    e2e_drain()
    f1.record(s_cmp)
    torch.cuda.synchronize()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / args.steps, world, dev)
    barrier(world)
    st = rs.rs_last_error(h, s_cmp)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after e2e: {rs.rs_strerror(st)}")
    h2d = sum(t.numel() * t.element_size() for p in host_in.values() for t in p)
    d2h = sum(t.numel() * t.element_size() for p in host_out.values() for t in p)

    batched = None if args.no_batched else run_batched(args, dev, world)
    per_scheme.update(precision_mode_rows(rs, h, pools, N, hbm_peak))

    cpu = None
    mism = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(N, B, args.y, budget_s=20.0)
        cpu["all_cores"] = cpu_all_cores(N, B, args.y)
        mism = scan_mismatches(rs, h, {"f32": pools["f32"][0], "f64": pools["f64"][0]}, N)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(args, N, B),
            "l2_pool_mib": round(pool_bytes / 2**20),
            "e2e": {"value": round(world * ancestors_per_step / (ms_e2e * 1e-3) / 1e9, 3),
                    "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(ms_e2e, 5),
                    "copies": "pinned host buffers; H2D and D2H on their own streams, "
                              "overlapping the kernels of neighbouring calls"},
            "roofline": roof,
            "per_scheme": per_scheme,
            "per_scheme_note": "one call with Permute, traced (kernel-to-kernel events); "
                               "hbm_frac = algorithmic bytes (sweep_hbm_bytes) / time / peak; "
                               "f32 = plain binary32 sums, f64 = double-float sums over "
                               "binary64 inputs, f32c = compensated two-float sums, f64n = "
                               "IEEE binary64 sums",
            "per_kernel": per_kernel,
            "philox_peak": philox,
            "gpu_launches": gpu_launches_per_step * args.steps,
            "gpu_launches_per_step": gpu_launches_per_step,
            "traced_ms_per_step": round(ms_traced_total / args.steps, 5),
            "wall_s_timed_region": round(wall, 4),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"], "samples": clk["samples"],
                       "window_s": round(clock_window_s, 3),
                       "window": "nvidia-smi every 100 ms over the timed replays, untimed "
                                 "replays of the same graphs that extend them to 1 s, and "
                                 "the traced steps"},
            "cpu_baseline": cpu,
            "mismatches": mism,
            "mismatches_note": ("one call per scan-based scheme and mode on the first pool "
                                "vector, against the oracle (tests/parity_tools.py rules); "
                                "unexplained must be 0"),
            "batched": batched,
        }
        print(json.dumps(line))
    h.close()


# ---------------------------------------------------------------------------------------
# batched workload: many filters of uneven size in one launch
# ---------------------------------------------------------------------------------------
def run_batched(args, dev, world):
    """F filters, sizes log-uniform in [256, 65536], y_f ~ U[0,4], binary32; systematic and
    Metropolis (per-filter B from Eq. B) each with Permute, one call per scheme per step (nine
    kernels in all), replayed from a CUDA graph, first with the default launch shapes and then
    with those the library's autotuner picks on this batch (rs_tune_batched). Returns
    filters/s, particles/s and the aggregate algorithmic HBM bandwidth at the tuned shapes."""
    import torch
    import paper_1301_4019_gb300 as rs
    F = args.batched_filters
    sizes = workload.ragged_sizes(F, 256, 65536, seed=SEED)
    offsets, lw, y = workload.ragged_logw(sizes, seed=SEED, dtype=np.float32)
    total = int(offsets[-1])
    Bs = np.array([rs.rs_metropolis_B(0.01, workload.beta_estimate(v)) for v in y], np.int32)
    t = torch.from_numpy(lw).to(dev)
    off = torch.from_numpy(offsets).to(dev)
    Bt = torch.from_numpy(Bs).to(dev)
    outs = [torch.empty(total, dtype=torch.int32, device=dev) for _ in range(2)]
    h = rs.Handle(total)

    def step(k):
        rs.rs_resample_batched(h, rs.SYSTEMATIC, t, off, seed=SEED, step=k, out=outs[0],
                               permute=True)
        rs.rs_resample_batched(h, rs.METROPOLIS, t, off, B_per_filter=Bt, seed=SEED, step=k,
                               out=outs[1], permute=True)

    for k in range(args.warmup):
        step(k)
    st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"batched device status: {rs.rs_strerror(st)}")
    # per-kernel durations of one traced step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(16)]
    for e in evs:
        e.record()
    torch.cuda.synchronize()
    rs.rs_trace(h, evs)
    step(0)
    labels = rs.rs_trace_labels(h)
    rs.rs_trace(h, [])
    torch.cuda.synchronize()
    kern = {}
    call = 0
    for i, lab in enumerate(labels[:-1]):
        if lab == "end":
            call += 1
            continue
        name = f"{lab}:{['systematic', 'metropolis'][call]}"
        kern[name] = round(evs[i].elapsed_time(evs[i + 1]) * 1e3, 2)
    def graph_ms():
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                step(0)
        torch.cuda.current_stream().wait_stream(cs)
        g.replay()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return reduce_max(e0.elapsed_time(e1) / args.steps, world, dev)

    ms_default = graph_ms()
    # the library's autotuner on this batch (launch shapes of the Metropolis kernel and of
    # Permute; the ancestors do not depend on them), then the same graph again
    shapes = rs.rs_tune_batched(h, t, off, B_per_filter=Bt, reps=2)
    ms = graph_ms()
    st = rs.rs_last_error(h)
    h.close()
    if st != rs.RS_OK:
        raise SystemExit(f"batched device status: {rs.rs_strerror(st)}")
    return {"workload": f"{F} filters, N_f log-uniform in [256, 65536] ({total} particles), "
                        "y_f ~ U[0,4], binary32; systematic + Metropolis (B from Eq. B per "
                        "filter), each with Permute",
            "filters_per_s": round(world * 2 * F / (ms * 1e-3), 1),
            "G_particles_per_s": round(world * 2 * total / (ms * 1e-3) / 1e9, 3),
            "hbm_GB_per_s": round(world * (sweep_hbm_bytes(2, 4, total)
                                           + sweep_hbm_bytes(3, 4, total)) / (ms * 1e-3) / 1e9,
                                  1),
            "hbm_bytes_note": "algorithmic bytes of both calls with Permute (sweep_hbm_bytes: "
                              "systematic 28 B, Metropolis 24 B per particle; the Metropolis "
                              "gathers hit L2 and are not counted)",
            "ms_per_step": round(ms, 4), "particles": total, "kernel_us": kern,
            "launches_per_step": len(kern),
            "autotuned": {"metropolis_block_ipt": list(shapes["metropolis"]),
                          "permute_block_ipt": list(shapes["permute"]),
                          "ms_per_step_default_256x1": round(ms_default, 4)}}


# ---------------------------------------------------------------------------------------
# the oracle on the host cores: CPU baseline and reference arm
# ---------------------------------------------------------------------------------------
def oracle_step(lw_by_dtype, B, seed, step):
    import oracle
    n = 0
    for lw in lw_by_dtype:
        for s in range(5):
            st, a = oracle.resample(s, lw, B=B, seed=seed, step=step, log_wmax=0.0,
                                    permuted=True)
            assert st == oracle.OK
            n += len(a)
    return n


def host_info() -> dict:
    """The host the CPU legs ran on: logical CPUs and the CPU model (from /proc/cpuinfo)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
                if key == "cpu part" and model is None and ":" in line:
                    model = "cpu part " + line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu": model, "arch": platform.machine()}


def cpu_baseline(N, B, y, budget_s=20.0):
    """The oracle as it stands, single-threaded, on a bounded sample of the workload."""
    import oracle
    oracle.build()
    lws = [workload.synthetic_logw(N, y, seed=SEED + 99, dtype=np.float32),
           workload.synthetic_logw(N, y, seed=SEED + 99, dtype=np.float64)]
    done, t0, reps = 0, time.perf_counter(), 0
    while True:
        done += oracle_step(lws, B, SEED, reps)
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 3:
            break
    el = time.perf_counter() - t0
    return {"value": round(done / el / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} pass(es) of the full step workload at N=2^{int(math.log2(N))} "
                      f"(5 resamplers x 2 dtypes + Permute), single thread, {el:.1f} s",
            "host": host_info()}


_CPU_LW = {}


def _cpu_worker_init(N, y):
    """Process-pool initialiser: the step's two weight vectors, generated once per worker."""
    _CPU_LW[4] = workload.synthetic_logw(N, y, seed=SEED + 99, dtype=np.float32)
    _CPU_LW[8] = workload.synthetic_logw(N, y, seed=SEED + 99, dtype=np.float64)


def _cpu_task(task):
    """One resample with Permute by the oracle, single-threaded (scheme < 0: warm-up)."""
    scheme, S, B, step = task
    if scheme < 0:
        return 0
    import oracle
    st, a = oracle.resample(scheme, _CPU_LW[S], B=B, seed=SEED, step=step, log_wmax=0.0,
                            permuted=True)
    if st != oracle.OK:
        raise RuntimeError(f"oracle status {st}")
    return len(a)


def cpu_all_cores(N, B, y, steps=3):
    """The oracle as it stands on every host core: the step's ten resamples are independent,
    so `steps` steps' calls are spread over one spawned process per core (each call single-
    threaded). Throughput = ancestors / wall time of the calls, pool start excluded."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    tasks = [(s, S, B, k) for k in range(steps) for S in (8, 4) for s in (3, 4, 0, 1, 2)]
    ctx = mp.get_context("spawn")  # never fork a process that has used the GPU
    with ctx.Pool(cores, initializer=_cpu_worker_init, initargs=(N, y)) as pool:
        pool.map(_cpu_task, [(-1, 4, B, 0)] * (2 * cores), chunksize=1)
        t0 = time.perf_counter()
        done = sum(pool.map(_cpu_task, tasks, chunksize=1))
        el = time.perf_counter() - t0
    return {"value": round(done / el / 1e9, 6), "unit": UNIT, "cores": cores,
            "sample": f"{steps} steps of the full step workload at N=2^{int(math.log2(N))} "
                      f"({len(tasks)} independent oracle calls) over {cores} processes, "
                      f"{el:.1f} s wall"}


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    N, B = workload_params(args, oracle.metropolis_B)
    # the config's N when the whole run fits about three minutes (timed from one step),
    # else a 2^18-particle sample; the N used is stated in the config either way
    n_sample = N
    lws = [workload.synthetic_logw(N, args.y, seed=SEED + 5, dtype=np.float32),
           workload.synthetic_logw(N, args.y, seed=SEED + 5, dtype=np.float64)]
    t_one = time.perf_counter()
    oracle_step(lws, B, SEED, 0)
    t_one = time.perf_counter() - t_one
    if t_one * (args.steps + args.warmup) > 180.0 and N > (1 << 18):
        n_sample = 1 << 18
        lws = [workload.synthetic_logw(n_sample, args.y, seed=SEED + 5, dtype=np.float32),
               workload.synthetic_logw(n_sample, args.y, seed=SEED + 5, dtype=np.float64)]
    for k in range(1, args.warmup):
        oracle_step(lws, B, SEED, k)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        done += oracle_step(lws, B, SEED, k)
    el = time.perf_counter() - t0
    value = done / el / 1e9
    sample = (f"each step: 5 resamplers x 2 dtypes + Permute on a 2^{int(math.log2(n_sample))}-"
              f"particle sample of the workload (y={args.y}, B={B}), single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(args, N, B), reference_N=n_sample),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def sweep_hbm_bytes(scheme: int, S: int, N: int) -> int:
    """Algorithmic HBM bytes of one call with Permute: scan schemes read the log-weights twice
    and write the ancestors (the multinomial also writes and re-reads its cumulative weights,
    S bytes each), Metropolis / rejection read each particle's own log-weight and write its
    ancestor; Permute writes and reads the claims, reads the ancestors, writes the result."""
    per = {0: 3 * S + 4, 1: 2 * S + 4, 2: 2 * S + 4, 3: S + 4, 4: S + 4}[scheme]
    return (per + 16) * N


GRAPH_CALLS = 20


def _graph_call_us(call) -> float:
    """Microseconds per call of `call(k, stream)` when GRAPH_CALLS of them (k = 0, 1, ...) are
    captured in one CUDA graph and replayed (median of 5 replays)."""
    import statistics
    import torch
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        for k in range(GRAPH_CALLS):
            call(k, cs)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            for k in range(GRAPH_CALLS):
                call(k, cs)
    torch.cuda.current_stream().wait_stream(cs)
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts) * 1e3 / GRAPH_CALLS


def run_sweep(args):
    import statistics
    import torch
    import paper_1301_4019_gb300 as rs
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ys = [float(v) for v in args.sweep_y.split(",")]
    with rs.Handle(1 << 24) as h:
        rs.rs_set_launch_mode(h, LAUNCH_MODES[args.launch_mode])
        for y, log2n in ((y, n) for y in ys for n in range(10, 25)):
            N = 1 << log2n
            B = workload_params(argparse.Namespace(log2n=log2n, y=y))[1]
            out = torch.empty(N, dtype=torch.int32, device="cuda")
            for name, npdt, prec in (("f32", np.float32, 0), ("f32c", np.float32, 1),
                                     ("f64", np.float64, 0), ("f64n", np.float64, 2)):
                lw = torch.from_numpy(workload.synthetic_logw(N, y, seed=SEED + log2n,
                                                              dtype=npdt)).cuda()
                S = 4 if npdt == np.float32 else 8
                # the compensated and IEEE binary64 modes change only the scan-based schemes
                for scheme in (range(5) if prec == 0 else range(3)):
                    for k in range(3):
                        rs.rs_resample(h, scheme, lw, B=B, seed=SEED, step=k, out=out,
                                       permute=True, log_wmax=0.0, prec=prec)
                    ts = []
                    for k in range(args.sweep_reps):
                        flush.fill_(float(k))
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        rs.rs_resample(h, scheme, lw, B=B, seed=SEED, step=k, out=out,
                                       permute=True, log_wmax=0.0, prec=prec)
                        e1.record()
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    ms = statistics.median(ts)
                    gbs = sweep_hbm_bytes(scheme, S, N) / (ms * 1e-3) / 1e9
                    row = {"y": y, "B": B, "log2n": log2n, "dtype": name,
                           "scheme": SCHEME_NAMES[scheme], "us": round(ms * 1e3, 2),
                           "G_ancestors_per_s": round(N / (ms * 1e-3) / 1e9, 3),
                           "hbm_frac": round(gbs / hbm_peak, 4)}
                    if log2n <= 16:  # launch-bound sizes: also per call inside a CUDA graph
                        row["us_graph"] = round(_graph_call_us(
                            lambda k, st: rs.rs_resample(h, scheme, lw, B=B, seed=SEED, step=k,
                                                         out=out, permute=True, log_wmax=0.0,
                                                         prec=prec, stream=st)), 2)
                    rows.append(row)
                del lw
        st = rs.rs_last_error(h)
    clk = clocks.stop()
    if st != rs.RS_OK:
        raise SystemExit(f"device status after sweep: {rs.rs_strerror(st)}")
    print(json.dumps({"sweep": "N = 2^10 .. 2^24, y in {%s}, B from Eq. B, log_wmax = 0, with "
                      "Permute; dtype f32 = plain binary32 sums, f32c = compensated, f64 = "
                      "double-float over binary64 inputs, f64n = IEEE binary64 (the last "
                      "three for the scan-based schemes); median of %d calls, each after "
                      "writing %d MiB (L2 flush); "
                      "hbm_frac = algorithmic bytes (sweep_hbm_bytes) / time / %.1f GB/s "
                      "(measured); us_graph (N <= 2^16): %d calls captured in one CUDA graph, "
                      "replayed, time / calls (no flush: the inputs stay in L2)"
                      % (args.sweep_y, args.sweep_reps, 2 * L2_BYTES // 2**20, hbm_peak,
                         GRAPH_CALLS),
                      "launch_mode": args.launch_mode, "clocks": clk, "rows": rows}))


def run_precision(args):
    """Mean absolute offspring bias mean_i |mean_r o_i - N pi_i| over R repeats (seeds differ
    by the step counter) of one weight set, against the Monte Carlo noise floor
    sqrt(mean_i Var(o_i) / R), and the squared bias's share of the MSE (bias_mse); pi from
    the input log-weights in binary64 (numpy). The scan-based schemes run in every precision
    mode, Metropolis (B* of Eq. B) and rejection (log w_max = 0) in binary32. The offspring
    are counted on the GPU (rs_offspring) and summed there."""
    import torch
    import paper_1301_4019_gb300 as rs
    R = args.precision_reps
    modes = [("f32 plain", np.float32, rs.PREC_PLAIN), ("f32 compensated", np.float32,
              rs.PREC_COMPENSATED), ("f64", np.float64, rs.PREC_PLAIN)]
    rows = []
    with rs.Handle(1 << 26) as h:
        for log2n in (16, 18, 20, 22, 24, 26):
            N = 1 << log2n
            out = torch.empty(N, dtype=torch.int32, device="cuda")
            o = torch.empty(N, dtype=torch.int32, device="cuda")
            for y in (0.0, 2.0, 4.0):
                lw64 = workload.synthetic_logw(N, y, seed=SEED + 300 + log2n, dtype=np.float64)
                for label, npdt, prec in modes:
                    lw_in = lw64.astype(npdt)
                    w = np.exp(lw_in.astype(np.float64) - lw_in.max())
                    Npi = torch.from_numpy(N * w / math.fsum(w)).cuda()
                    lw = torch.from_numpy(lw_in).cuda()
                    schemes = [rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC]
                    if label == "f32 plain":
                        schemes += [rs.METROPOLIS, rs.REJECTION]
                    B = rs.rs_metropolis_B(0.01, workload.beta_estimate(y))
                    for scheme in schemes:
                        s1 = torch.zeros(N, dtype=torch.float64, device="cuda")
                        s2 = torch.zeros(N, dtype=torch.float64, device="cuda")
                        for r in range(R):
                            rs.rs_resample(h, scheme, lw, B=B, seed=SEED + 7, step=r, out=out,
                                           prec=prec, log_wmax=0.0)
                            rs.rs_offspring(h, out, o)
                            od = o.double()
                            s1 += od
                            s2 += od * od
                        mean = s1 / R
                        var = (s2 / R - mean * mean).clamp_min(0) * R / max(R - 1, 1)
                        b2, mse = bias_mse(s1, s2, Npi, R)
                        rows.append({"log2n": log2n, "y": y, "mode": label,
                                     "scheme": SCHEME_NAMES[scheme],
                                     "B": B if scheme == rs.METROPOLIS else None,
                                     "mean_abs_bias": float((mean - Npi).abs().mean()),
                                     "noise_floor": float(torch.sqrt(var.mean() / R)),
                                     "bias_share": b2 / mse if mse > 0 else 0.0})
                    del lw, Npi
        # deterministic part: the expected offspring given the kernel's own cumulative
        # weights, E_u[o_i] = r_i - r_{i-1} with r_i = N W_i / W_N (Section 4.2's measure without
        # Monte Carlo noise), from the accumulators written out exactly in binary64
        det = []
        for log2n in (16, 18, 20, 22, 24, 26):
            N = 1 << log2n
            for y in (0.0, 2.0, 4.0):
                lw64 = workload.synthetic_logw(N, y, seed=SEED + 300 + log2n, dtype=np.float64)
                w = np.exp(lw64 - lw64.max())
                Npi = torch.from_numpy(N * w / math.fsum(w)).cuda()
                for label, npdt, prec in modes + [("f64 binary64", np.float64,
                                                   rs.PREC_BINARY64)]:
                    lw = torch.from_numpy(lw64.astype(npdt)).cuda()
                    W, _ = rs.rs_cumulative_weights_f64(h, lw, prec=prec)
                    r = W * (N / W[-1])
                    e = torch.diff(r, prepend=torch.zeros(1, dtype=r.dtype, device=r.device))
                    dev = (e - Npi).abs()
                    det.append({"log2n": log2n, "y": y, "mode": label,
                                "mean_abs": float(dev.mean()), "max_abs": float(dev.max())})
                    del lw, W, r, e, dev
                del Npi
        st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after precision study: {rs.rs_strerror(st)}")
    print(json.dumps({"precision": f"{R} repeats per row (seed fixed, step = repeat index); "
                      "bias = mean_i |mean o_i - N pi_i|, pi from the input log-weights in "
                      "binary64; noise floor = sqrt(mean_i Var(o_i) / R); bias_share = "
                      "||Bias||^2 / MSE (Section 4.2; about 1/R for an unbiased scheme); "
                      "Metropolis B = B* (Eq. B), rejection log w_max = 0, both binary32",
                      "rows": rows,
                      "deterministic": "E_u[o_i] - N pi_i from the kernel's cumulative weights "
                      "(rs_cumulative_weights_f64): r_i = N W_i / W_N in binary64; mean and max "
                      "over i of |r_i - r_{i-1} - N pi_i|", "det_rows": det}))


def run_smc(args):
    """Time the bootstrap filter (resample with Permute, in-place copy, propagate + weight,
    log-sum of the weights) over T = 100 observations of the linear-Gaussian model, captured
    as one CUDA graph per scheme and replayed; also report the filter's log-likelihood
    estimates over a few seeds (the tests check them against the Kalman filter)."""
    import statistics
    import torch
    import paper_1301_4019_gb300 as rs
    from paper_1301_4019_gb300 import smc
    N, T, reps = 1 << args.log2n, 100, 5
    phi, sx, sy = workload.LGSSM_PHI, workload.LGSSM_SIGMA_X, workload.LGSSM_SIGMA_Y
    _, y = workload.lgssm_simulate(T, phi, sx, sy, seed=SEED)
    rows = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    with rs.Handle(N) as h:
        rs.rs_set_launch_mode(h, LAUNCH_MODES[args.launch_mode])
        for scheme in (rs.SYSTEMATIC, rs.METROPOLIS, rs.REJECTION):
            lls = [smc.lgssm_bootstrap(h, y, N, scheme, phi, sx, sy, seed=s, B=64)
                   for s in range(4)]
            bufs = smc.LgssmBuffers(N, T)
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                smc.lgssm_bootstrap_launch(h, y, N, scheme, phi, sx, sy, seed=7, bufs=bufs,
                                           stream=cs)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cs):
                    smc.lgssm_bootstrap_launch(h, y, N, scheme, phi, sx, sy, seed=7,
                                               bufs=bufs, stream=cs)
            torch.cuda.current_stream().wait_stream(cs)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rows.append({"scheme": SCHEME_NAMES[scheme], "ms_per_filter": round(ms, 3),
                         "us_per_step": round(1e3 * ms / T, 2),
                         "G_particle_steps_per_s": round(N * T / (ms * 1e-3) / 1e9, 3),
                         "loglik_mean": round(statistics.mean(lls), 4),
                         "loglik_sd": round(statistics.stdev(lls), 4)})
        for scheme in (rs.SYSTEMATIC, rs.REJECTION):  # resampling on demand (ESS < N/2)
            smc.lgssm_adaptive(h, y, N, scheme, phi, sx, sy, 0.5, seed=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            runs = [smc.lgssm_adaptive(h, y, N, scheme, phi, sx, sy, 0.5, seed=s)
                    for s in range(4)]
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / len(runs)
            lls = [r[0] for r in runs]
            rows.append({"scheme": SCHEME_NAMES[scheme] + " (ESS < N/2)",
                         "ms_per_filter": round(ms, 3), "us_per_step": round(1e3 * ms / T, 2),
                         "G_particle_steps_per_s": round(N * T / (ms * 1e-3) / 1e9, 3),
                         "resamplings": [r[1] for r in runs],
                         "loglik_mean": round(statistics.mean(lls), 4),
                         "loglik_sd": round(statistics.stdev(lls), 4),
                         "timing": "host clock; the host reads the ESS every step"})
        for scheme in (rs.SYSTEMATIC, rs.REJECTION):  # the same, decided on the device
            ag = smc.AdaptiveGraph(h, y, N, scheme, phi, sx, sy, 0.5, seed=1)
            ag.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ag.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ll, n_res = ag.result()
            rows.append({"scheme": SCHEME_NAMES[scheme] + " (ESS < N/2, one graph)",
                         "ms_per_filter": round(ms, 3), "us_per_step": round(1e3 * ms / T, 2),
                         "G_particle_steps_per_s": round(N * T / (ms * 1e-3) / 1e9, 3),
                         "resamplings": [n_res], "loglik_mean": round(ll, 4),
                         "timing": "CUDA-graph replay; conditional nodes decide on the device"})
            del ag
        st = rs.rs_last_error(h)
    # many filters: 256 filters of N_f log-uniform on [2^14, 2^18], one graph per run
    rng = np.random.default_rng(SEED + 256)
    sizes = np.floor(np.exp(rng.uniform(math.log(2 ** 14), math.log(2 ** 18), 256)))
    sizes = sizes.astype(np.int64)
    total = int(sizes.sum())
    with rs.Handle(total) as hb:
        for scheme in (rs.SYSTEMATIC, rs.METROPOLIS):
            bufs = smc.BatchedLgssmBuffers(sizes, np.repeat(np.asarray(y)[:, None], 256, axis=1))
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                smc.lgssm_batched_launch(hb, bufs, scheme, phi, sx, sy, seed=3, B=64, stream=cs)
                torch.cuda.synchronize()
                lls = smc.lgssm_batched_loglik_from(bufs, sy)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cs):
                    smc.lgssm_batched_launch(hb, bufs, scheme, phi, sx, sy, seed=3, B=64,
                                             stream=cs)
            torch.cuda.current_stream().wait_stream(cs)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rows.append({"scheme": SCHEME_NAMES[scheme] + " (256 filters, batched)",
                         "filters": 256, "particles": total,
                         "ms_per_filter": round(ms, 3), "us_per_step": round(1e3 * ms / T, 2),
                         "G_particle_steps_per_s": round(total * T / (ms * 1e-3) / 1e9, 3),
                         "loglik_mean": round(float(np.mean(lls)), 4),
                         "loglik_sd": round(float(np.std(lls, ddof=1)), 4)})
        # resampling on demand for every filter of the batch, decided on the device
        for scheme in (rs.SYSTEMATIC,):
            bufs = smc.BatchedLgssmBuffers(sizes, np.repeat(np.asarray(y)[:, None], 256, axis=1))
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                flags = smc.lgssm_batched_adaptive_launch(hb, bufs, scheme, phi, sx, sy, 0.5,
                                                          seed=3, B=64, stream=cs)
                torch.cuda.synchronize()
                lls = smc.lgssm_batched_adaptive_loglik_from(bufs, flags, sy)
                n_res = flags[1:].sum(dim=0).cpu().numpy()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cs):
                    smc.lgssm_batched_adaptive_launch(hb, bufs, scheme, phi, sx, sy, 0.5,
                                                      seed=3, B=64, stream=cs)
            torch.cuda.current_stream().wait_stream(cs)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rows.append({"scheme": SCHEME_NAMES[scheme] + " (256 filters, batched, ESS < N/2 "
                                                            "per filter)",
                         "filters": 256, "particles": total,
                         "ms_per_filter": round(ms, 3), "us_per_step": round(1e3 * ms / T, 2),
                         "G_particle_steps_per_s": round(total * T / (ms * 1e-3) / 1e9, 3),
                         "resamplings_mean": round(float(n_res.mean()), 2),
                         "loglik_mean": round(float(np.mean(lls)), 4),
                         "loglik_sd": round(float(np.std(lls, ddof=1)), 4)})
        st2 = rs.rs_last_error(hb)
    st = st if st != rs.RS_OK else st2
    clk = clocks.stop()
    if st != rs.RS_OK:
        raise SystemExit(f"device status after SMC study: {rs.rs_strerror(st)}")
    print(json.dumps({"smc": f"bootstrap filter, N = 2^{args.log2n}, T = {T}, model "
                      f"x_t = {phi} x_t-1 + N(0, {sx}^2), y_t = x_t + N(0, {sy}^2); per step: "
                      "resample (compensated binary32, Permute), in-place copy, propagate + "
                      "weight, log-sum of the weights; Metropolis B = 64; one CUDA graph per "
                      f"filter run, {reps} replays; batched rows: 256 filters, N_f "
                      "log-uniform on [2^14, 2^18], all on the same observations "
                      "(log-likelihood mean / sd over the filters)", "clocks": clk,
                      "rows": rows}))


def _median_call_ms(fn, reps, flush):
    import statistics
    import torch
    for k in range(3):
        fn(k)
    ts = []
    for k in range(reps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn(k)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def run_prc(args):
    """Partial rejection control (Section 2.2): per-call time with Permute and the outcome
    weights, the expected trials per particle 1 + (1 - v_i/v_max)/p with p = mean(v)/v_max
    (closed form from the weights), and the ESS of the weighted outcome (rs_ess on the
    outcome log-weights), for v_max at quantiles of the weights; "bound" is v_max = 1, the
    a-priori bound of the workload, where the call equals the rejection resampler."""
    import torch
    import paper_1301_4019_gb300 as rs
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    with rs.Handle(1 << 24) as h:
        ess = torch.empty(1, dtype=torch.float64, device="cuda")
        for log2n in (20, 24):
            N = 1 << log2n
            out = torch.empty(N, dtype=torch.int32, device="cuda")
            for y in (2.0, 3.0, 4.0):
                lw64 = workload.synthetic_logw(N, y, seed=SEED + 500 + log2n, dtype=np.float64)
                for name, npdt in (("f32", np.float32), ("f64", np.float64)):
                    lw_np = lw64.astype(npdt)
                    lw = torch.from_numpy(lw_np).cuda()
                    lo = torch.empty_like(lw)
                    for q in ("bound", 0.999, 0.99, 0.9, 0.5):
                        lvmax = 0.0 if q == "bound" else float(np.quantile(lw_np, q))
                        ms = _median_call_ms(
                            lambda k: rs.rs_resample_prc(h, lw, lvmax, seed=SEED, step=k,
                                                         permute=True, out=out, logw_out=lo),
                            args.sweep_reps, flush)
                        rs.rs_ess(h, lo, out=ess)
                        v = np.minimum(np.exp(lw_np.astype(np.float64) - lvmax), 1.0)
                        p = v.mean()
                        rows.append({"log2n": log2n, "y": y, "dtype": name, "v_max": q,
                                     "log_vmax": round(lvmax, 4), "us": round(ms * 1e3, 2),
                                     "G_ancestors_per_s": round(N / (ms * 1e-3) / 1e9, 3),
                                     "expected_trials": round(float(np.mean(1 + (1 - v) / p)),
                                                              3),
                                     "outcome_ess_frac": round(float(ess.item()) / N, 4)})
                    del lw, lo
        st = rs.rs_last_error(h)
    clk = clocks.stop()
    if st != rs.RS_OK:
        raise SystemExit(f"device status after PRC study: {rs.rs_strerror(st)}")
    print(json.dumps({"prc": "partial rejection control with Permute and outcome weights; "
                      f"median of {args.sweep_reps} calls, each after writing "
                      f"{2 * L2_BYTES // 2**20} MiB (L2 flush); v_max at quantiles of the "
                      "weights", "clocks": clk, "rows": rows}))


def run_metropolis_b(args):
    """Metropolis resampler over B (Section 4.4, the time / bias trade-off of Eq. B): per-call
    time with Permute, and the offspring bias mean_i |mean_r o_i - N pi_i| over R repeats
    against the Monte Carlo noise floor sqrt(mean_i Var(o_i) / R), with the TV bound
    (1 - beta)^B of Section 2.1 beside it."""
    import torch
    import paper_1301_4019_gb300 as rs
    R = args.metropolis_b_reps
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    N = 1 << 20
    with rs.Handle(N) as h:
        out = torch.empty(N, dtype=torch.int32, device="cuda")
        o = torch.empty(N, dtype=torch.int32, device="cuda")
        for y in (1.0, 2.0, 3.0):
            beta = workload.beta_estimate(y)
            Bstar = rs.rs_metropolis_B(0.01, beta)
            lw64 = workload.synthetic_logw(N, y, seed=SEED + 600, dtype=np.float64)
            w = np.exp(lw64 - lw64.max())
            Npi = torch.from_numpy(N * w / math.fsum(w)).cuda()
            lw = torch.from_numpy(lw64.astype(np.float32)).cuda()
            for frac in (0.125, 0.25, 0.5, 1.0, 2.0, 4.0):
                B = max(1, int(round(Bstar * frac)))
                ms = _median_call_ms(
                    lambda k: rs.rs_resample(h, rs.METROPOLIS, lw, B=B, seed=SEED, step=k,
                                             out=out, permute=True),
                    args.sweep_reps, flush)
                s1 = torch.zeros(N, dtype=torch.float64, device="cuda")
                s2 = torch.zeros(N, dtype=torch.float64, device="cuda")
                for r in range(R):
                    rs.rs_resample(h, rs.METROPOLIS, lw, B=B, seed=SEED + 9, step=r, out=out)
                    rs.rs_offspring(h, out, o)
                    od = o.double()
                    s1 += od
                    s2 += od * od
                mean = s1 / R
                var = (s2 / R - mean * mean).clamp_min(0) * R / max(R - 1, 1)
                rows.append({"y": y, "B_star": Bstar, "B": B, "us": round(ms * 1e3, 2),
                             "tv_bound": float((1 - beta) ** B),
                             "mean_abs_bias": float((mean - Npi).abs().mean()),
                             "noise_floor": float(torch.sqrt(var.mean() / R))})
            del lw, Npi
        st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after Metropolis B study: {rs.rs_strerror(st)}")
    print(json.dumps({"metropolis_b": f"N = 2^20, binary32, with Permute; time: median of "
                      f"{args.sweep_reps} calls after an L2 flush; bias over {R} repeats "
                      "(step = repeat index); B* from Eq. B with eps = 0.01 and the closed-form "
                      "beta of the workload", "rows": rows}))


def bias_mse(s1, s2, Npi, R: int):
    """The accuracy measures of Section 4.2 from R offspring vectors o_1..o_R of one weight
    vector, given their sums s1_i = sum_r o_ri and s2_i = sum_r o_ri^2 (binary64 tensors or
    arrays of integers) and N pi_i: ||Bias||^2 = sum_i (mean_r o_ri - N pi_i)^2, tr Var =
    sum_i of the sample variance of o_i (divisor R), MSE = tr Var + ||Bias||^2 (= the mean
    over r of sum_i (o_ri - N pi_i)^2). Returns (||Bias||^2, MSE). The variance numerator
    R s2 - s1^2 is exact while it stays below 2^53."""
    mean = s1 / R
    bias2 = float(((mean - Npi) ** 2).sum())
    trvar = float((R * s2 - s1 * s1).sum()) / (R * R)
    return bias2, bias2 + trvar


def run_accuracy(args):
    """The accuracy experiment of Section 4.2 (the bias and MSE figures): for each N and y,
    16 weight vectors, 256 offspring vectors of each resampler per vector; reports the squared
    bias's share of the MSE and MSE / N, averaged over the 16 vectors, in binary32 (plain and
    compensated sums) and binary64. Metropolis runs B* of Eq. B (eps = 0.01); the paper's
    study of B = B*/C (y = 4, C = 1, 2, 4, 8) adds the per-call time (with Permute, L2
    flushed). Offspring are counted with torch.bincount (statistics only)."""
    import torch
    import paper_1301_4019_gb300 as rs
    V, K = 16, 256
    sizes = [int(v) for v in args.accuracy_sizes.split(",")]
    scan = (rs.MULTINOMIAL, rs.STRATIFIED, rs.SYSTEMATIC)
    every = scan + (rs.METROPOLIS, rs.REJECTION)
    modes = [("f32", np.float32, rs.PREC_PLAIN, every),
             ("f32 compensated", np.float32, rs.PREC_COMPENSATED, scan),
             ("f64", np.float64, rs.PREC_PLAIN, every)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    rows, brows = [], []
    t_start = time.perf_counter()
    with rs.Handle(1 << max(sizes)) as h:
        for log2n in sizes:
            N = 1 << log2n
            CH = max(1, min(K, (1 << 24) // N))  # offspring vectors per counting chunk
            A = torch.empty((CH, N), dtype=torch.int32, device="cuda")
            offs = (torch.arange(CH, device="cuda", dtype=torch.int64) * N)[:, None]

            def measure(lw, Npi, scheme, B, prec, v):
                s1 = torch.zeros(N, dtype=torch.int64, device="cuda")
                s2 = torch.zeros(N, dtype=torch.int64, device="cuda")
                for r0 in range(0, K, CH):
                    m = min(CH, K - r0)
                    for r in range(m):
                        rs.rs_resample(h, scheme, lw, B=B, seed=SEED + 13 + v, step=r0 + r,
                                       out=A[r], prec=prec, log_wmax=0.0)
                    cnt = torch.bincount((A[:m].long() + offs[:m]).view(-1),
                                         minlength=m * N).view(m, N)
                    s1 += cnt.sum(0)
                    s2 += (cnt * cnt).sum(0)
                return bias_mse(s1.double(), s2.double(), Npi, K)

            for y in (0.0, 1.0, 2.0, 3.0, 4.0):
                Bstar = rs.rs_metropolis_B(0.01, workload.beta_estimate(y))
                Cs = (1, 2, 4, 8) if y == 4.0 else (1,)
                acc = {}
                for v in range(V):
                    lw64 = workload.synthetic_logw(N, y, seed=SEED + 5000 + 131 * log2n
                                                   + 17 * int(y) + v, dtype=np.float64)
                    for label, npdt, prec, schemes in modes:
                        lw = torch.from_numpy(lw64.astype(npdt)).cuda()
                        lwd = lw.double()
                        w = torch.exp(lwd - lwd.max())
                        Npi = N * w / w.sum()
                        for scheme in schemes:
                            for Cdiv in (Cs if scheme == rs.METROPOLIS and label == "f32"
                                         else (1,)):
                                B = max(1, -(-Bstar // Cdiv))
                                b2, mse = measure(lw, Npi, scheme, B, prec, v)
                                acc.setdefault((label, scheme, Cdiv, B), []).append(
                                    (b2 / mse if mse > 0 else 0.0, mse / N))
                        del lw, lwd, w, Npi
                for (label, scheme, Cdiv, B), vals in acc.items():
                    fr = [a for a, _ in vals]
                    row = {"log2n": log2n, "y": y, "mode": label,
                           "scheme": SCHEME_NAMES[scheme], "B": B if scheme == rs.METROPOLIS
                           else None, "bias_share": float(np.mean(fr)),
                           "bias_share_max": float(np.max(fr)),
                           "mse_per_n": float(np.mean([m for _, m in vals]))}
                    if Cdiv == 1:
                        rows.append(row)
                    if scheme == rs.METROPOLIS and label == "f32" and y == 4.0:
                        lw = torch.from_numpy(workload.synthetic_logw(
                            N, y, seed=SEED + 5000 + 131 * log2n + 68,
                            dtype=np.float64).astype(np.float32)).cuda()
                        ms = _median_call_ms(
                            lambda k: rs.rs_resample(h, rs.METROPOLIS, lw, B=B, seed=SEED,
                                                     step=k, out=A[0], permute=True),
                            11, flush)
                        brows.append(dict(row, C=Cdiv, us=round(ms * 1e3, 2)))
                        del lw
            del A, offs
        st = rs.rs_last_error(h)
    if st != rs.RS_OK:
        raise SystemExit(f"device status after the accuracy study: {rs.rs_strerror(st)}")
    print(json.dumps({"accuracy": f"{V} weight vectors x {K} offspring vectors per (N, y, "
                      "scheme, mode); bias_share = ||Bias||^2 / MSE and mse_per_n = MSE / N, "
                      "means over the weight vectors (bias_share_max: the largest); "
                      "Metropolis B = B* (Eq. B, eps = 0.01), rejection log w_max = 0",
                      "seconds": round(time.perf_counter() - t_start, 1),
                      "rows": rows, "metropolis_b_over_c": brows}))


def run_single(args):
    """One resample configuration on one input, for profilers: warmup + steps calls."""
    import torch
    import paper_1301_4019_gb300 as rs
    parts = args.single.split(":")
    scheme = rs.SCHEMES[parts[0]]
    npdt = {"f32": np.float32, "f64": np.float64}[parts[1]]
    prec = int(parts[2]) if len(parts) > 2 else 0
    N, B = workload_params(args)
    lw = torch.from_numpy(workload.synthetic_logw(N, args.y, seed=SEED, dtype=npdt)).cuda()
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    with rs.Handle(N) as h:
        rs.rs_set_launch_mode(h, LAUNCH_MODES[args.launch_mode])
        for k in range(args.warmup):
            rs.rs_resample(h, scheme, lw, B=B, seed=SEED, step=k, out=out, permute=True, prec=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(args.steps):
            rs.rs_resample(h, scheme, lw, B=B, seed=SEED, step=k, out=out, permute=True, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        st = rs.rs_last_error(h)
    if st != 0:
        raise SystemExit(f"device status {st}")
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"single": args.single, "N": N, "ms_per_call": round(ms, 5),
                      "G_ancestors_per_s": round(N / (ms * 1e-3) / 1e9, 3)}))


def main():
    args = parse_args()
    if args.single:
        run_single(args)
    elif args.sweep:
        run_sweep(args)
    elif args.precision:
        run_precision(args)
    elif args.smc:
        run_smc(args)
    elif args.prc:
        run_prc(args)
    elif args.metropolis_b:
        run_metropolis_b(args)
    elif args.accuracy:
        run_accuracy(args)
    elif args.philox_peak:
        import paper_1301_4019_gb300 as rs
        with rs.Handle(1024) as h:
            print(json.dumps({"philox_peak": measure_philox_peak(rs, h, reps=21)}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
