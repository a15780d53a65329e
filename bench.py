#!/usr/bin/env python3
"""Throughput of the MG-MLQMC hot path on one GB300 (samples/s, KL + FMG).

Workload (default): MLQMC with sample recycling in FP64, 6 levels of 8x8 ..
256x256 cells, s = 100 KL modes (separable exponential covariance, sigma = 1,
correlation length 0.3), rank-1 lattice (CBC, gamma_j = j^-2) with R = 16
random shifts, N_l = 1024, 512, 256, 128, 64, 32 points per shift on levels
0..5 (32,256 FMG solves per step), mean-of-u QoI. One step = normals, fields on
every level of every sample, FMG with two V(2,2)-cycles per level, F_t and the
reuse sums of every level, and the estimator from those sums.

The same step in the mixed form (FP32 V-cycles inside FP64 refinement) is
reported under "mixed". `--impl reference` times the CPU oracle as it stands
on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank runs an independent replica (its own seed);
no data-path collective; value = all ranks' samples / max time ("weak").
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "samples/s (KL+FMG) and time-to-RMSE ε: mixed-precision vs FP64, one GB300"
UNIT = "samples/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed_tf32"],
                    help="form of the main measurement (the other form is reported under 'mixed')")
    ap.add_argument("--no-precision", action="store_true", help="skip the 1024x1024 precision-form comparison")
    ap.add_argument("--no-tte", action="store_true", help="skip the time-to-epsilon runs of Algorithm 1")
    ap.add_argument("--no-matern", action="store_true",
                    help="skip the Matern-covariance step (Nystrom eigenpairs) in both forms")
    ap.add_argument("--smoother", default="auto", choices=["auto", "stream", "tma", "tile"],
                    help="mixed form: force this smoother on every level it handles (default: the autotuner's pick)")
    ap.add_argument("--smoother-plan", default="",
                    help="mixed form: pin smoothers per level, e.g. 1:whole,2:whole,4:tma (profiler runs, where "
                         "the autotuner's timings are not representative)")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernel by kernel instead of replaying a CUDA graph")
    ap.add_argument("--traffic-from", default="",
                    help="ncu CSV of one timed step (DRAM bytes, durations): summarise into profiles/")
    ap.add_argument("--traffic-line", default="", help="the bench JSON line of the same command without ncu")
    ap.add_argument("--counts-div", type=int, default=1,
                    help="divide the per-level counts (small cases for profiler captures only)")
    return ap.parse_args()


def workload_config(rank: int, counts_div: int = 1):
    cfg = dict(W.LATTICE_6LEVEL)
    cfg["seed"] = cfg["seed"] + 1000 * rank
    cfg["counts"] = [max(1, c // counts_div) for c in cfg["counts"]]
    return cfg


def work_list(cfg):
    return W.fixed_count_work(cfg["counts"], cfg["R"])


def n_samples(work):
    return sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)


# --------------------------------------------------------------------------- #
# Roofline denominators                                                         #
# --------------------------------------------------------------------------- #
# fallbacks when MEASURED_PEAKS.json is absent (one earlier GB300 measurement);
# measured_peaks_override replaces them with this machine's figures
HBM_GBS = 6800.0
BF16_TFLOPS = 1900.0
HBM_SRC = "fallback 6.8 TB/s (no measured copy bandwidth on this machine)"
TC_SRC = "fallback bf16 1.9 PFLOP/s x nominal tf32/bf16 ratio"
TF32_TFLOPS = BF16_TFLOPS * 1.1 / 2.25   # measured bf16 x nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s dense)
FP64_TFLOPS = 1.25        # nominal GB300 FP64 (an FMA probe measured 1.20)
FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz = 80.5


def measured_peaks_override():
    global HBM_GBS, BF16_TFLOPS, TF32_TFLOPS, HBM_SRC, TC_SRC
    pk = measured_peaks()
    if pk.get("hbm_gbs"):
        HBM_GBS = float(pk["hbm_gbs"])
        HBM_SRC = "measured copy bandwidth (MEASURED_PEAKS.json)"
    if pk.get("bf16_tflops"):
        BF16_TFLOPS = float(pk["bf16_tflops"])
        TF32_TFLOPS = BF16_TFLOPS * 1.1 / 2.25
        TC_SRC = "measured bf16 burst x nominal tf32/bf16 ratio"


KIND_KERNELS = {
    "points": "k_points (lattice points and normals)",
    "level0": "kb_level0 (banded Cholesky and exact level-0 solve, one thread per sample)",
    "synth": "kb_synth_G/kb_synth_z (separable KL), kb_faces, kb_idiag",
    "smooth": "red-black sweeps (kb_rbgs_whole up to 64x64 with residual/correction fused, kb_rbgs_tma tiles "
              "above; FP64 form: kb_rbgs_whole up to 64x64, kb_gs above)",
    "transfer": "kb_resid_restrict, kb_prolong, kb_resid64, kb_update64",
    "coarse": "kb_coarse_fixed (V-cycle level-0 solves)",
    "reduce": "kb_qoi, kb_resnorm, k_sums, outputs",
    "kl_tc": "kl_tc_kernel (tcgen05 TF32 KL contraction) and its C operand",
}


# kernel name -> the library's timing kind (the same grouping as its event brackets)
KIND_PATTERNS = [
    ("points", r"k_points"), ("level0", r"kb_level0"), ("synth", r"kb_synth_|kb_faces|kb_idiag"),
    ("smooth", r"kb_gs|kb_rbgs_"), ("transfer", r"kb_resid_restrict|kb_prolong|kb_resid64|kb_update64"),
    ("coarse", r"kb_coarse"), ("reduce", r"kb_qoi|kb_resnorm|kb_flags|k_sums|k_fout|kb_u_out|kb_k_out"),
    ("kl_tc", r"kl_tc_kernel|kl_build_c|kl_build_psi"),
]
TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "dram_traffic_mlqmc6.json")


def kernel_kind(name):
    for kind, pat in KIND_PATTERNS:
        if re.search(pat, name):
            return kind
    return None


def sources_digest():
    """SHA-256 over the library's CUDA/C++ sources and header: DRAM counters
    taken on other sources no longer describe these kernels."""
    import glob
    import hashlib

    root = os.path.dirname(os.path.abspath(__file__))
    files = sorted(glob.glob(os.path.join(root, "paper_1806_05619_gb300", "csrc", "*")))
    files = [f for f in files if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    files.append(os.path.join(root, "include", "mlqmc.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.relpath(f, root).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def summarize_traffic(csv_path, form, smoothers):
    """Per-kind DRAM bytes and launches of one captured timed step (ncu CSV of
    dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum in
    base units), merged into the traffic file under `form`."""
    import collections
    import csv

    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    per_launch = collections.defaultdict(dict)
    names = {}
    for row in csv.DictReader(lines):
        v = float(row["Metric Value"].replace(",", ""))
        per_launch[row["ID"]][row["Metric Name"]] = v
        names[row["ID"]] = row["Kernel Name"]
    kinds = collections.defaultdict(lambda: {"launches": 0, "dram_bytes": 0.0, "ns": 0.0})
    for i, m in per_launch.items():
        k = kernel_kind(names[i])
        if k is None:
            continue
        d = kinds[k]
        d["launches"] += 1
        d["dram_bytes"] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
        d["ns"] += m.get("gpu__time_duration.sum", 0.0)
    for d in kinds.values():
        d["dram_bytes_per_launch"] = d["dram_bytes"] / d["launches"]
    data = {}
    if os.path.exists(TRAFFIC_FILE):
        with open(TRAFFIC_FILE) as f:
            data = json.load(f)
    data.setdefault("forms", {})[form] = {"sources_sha256": sources_digest(), "smoothers": smoothers,
                                         "kinds": dict(kinds)}
    with open(TRAFFIC_FILE, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return data["forms"][form]


def measured_traffic(form, kind, smoothers):
    """DRAM bytes per launch of `kind` from the committed ncu capture of this
    form's timed step, or None when there is none, the sources changed since,
    or the smoothers differ from the captured ones."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)["forms"][form]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("sources_sha256") != sources_digest() or rec.get("smoothers") != smoothers:
        return None
    d = rec["kinds"].get(kind)
    return d["dram_bytes_per_launch"] if d else None


def kind_roofline(ms, work):
    """Roofline of one kernel kind from its device time and algorithmic work:
    the bound is the resource whose model time (bytes / HBM, FLOPs / pipe peak)
    is longest; frac = that model time / measured time."""
    t = ms * 1e-3
    t_hbm = work["bytes"] / (HBM_GBS * 1e9)
    t64, t32 = work["f64"] / (FP64_TFLOPS * 1e12), work["f32"] / (FP32_TFLOPS * 1e12)
    t_tc = work["ftc"] / (TF32_TFLOPS * 1e12)
    best = max(("hbm", t_hbm), ("alu64", t64), ("alu32", t32), ("tensor", t_tc), key=lambda x: x[1])
    if t <= 0 or best[1] <= 0:
        return None
    r = {"ms": ms, "gbs": work["bytes"] / t / 1e9, "fp64_tflops": work["f64"] / t / 1e12,
         "fp32_tflops": work["f32"] / t / 1e12, "tc_tflops": work["ftc"] / t / 1e12,
         "algorithmic_bytes": work["bytes"]}
    if best[0] == "hbm":
        r.update(bound="hbm", achieved=r["gbs"], peak=HBM_GBS, unit="GB/s", peak_source=HBM_SRC)
    elif best[0] == "tensor":
        r.update(bound="tensor", achieved=r["tc_tflops"], peak=TF32_TFLOPS, unit="TFLOP/s", peak_source=TC_SRC)
    elif best[0] == "alu64":
        r.update(bound="alu", achieved=r["fp64_tflops"], peak=FP64_TFLOPS, unit="TFLOP/s",
                 peak_source="FP64 1.25 TFLOP/s (nominal GB300 figure; FMA probe 1.20)")
    else:
        r.update(bound="alu", achieved=r["fp32_tflops"], peak=FP32_TFLOPS, unit="TFLOP/s",
                 peak_source="FP32 152 SMs x 128 lanes x 2 x 2070 MHz")
    r["frac"] = r["achieved"] / r["peak"]
    return r


def roofline_report(prof, work, steps, form=None, smoothers=None):
    """Dominant kind's roofline (the bench line's `roofline`) plus every kind's.
    traffic: DRAM bytes per launch of that kind from the committed ncu capture
    of the same form's timed step (None when stale or absent)."""
    kinds = {}
    for k, (ms, n) in prof.items():
        if n == 0:
            continue
        r = kind_roofline(ms, work[k])
        if r:
            r["launches_per_step"] = n / steps
            r["ms_per_step"] = ms / steps
            kinds[k] = r
    tot = sum(v[0] for v in prof.values())
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    roof = {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["frac"], "traffic": measured_traffic(form, dom, smoothers) if form else None,
            "kernel": KIND_KERNELS.get(dom, dom), "kernel_kind": dom,
            "peak_source": d["peak_source"], "share_of_step": d["ms"] / max(1e-9, tot),
            "launches_per_step": d["launches_per_step"], "ms_per_step": d["ms_per_step"],
            "algorithmic_bytes_per_launch": d["algorithmic_bytes"] / max(1, prof[dom][1])}
    by_kind = {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()
                   if kk in ("ms_per_step", "bound", "achieved", "unit", "frac", "gbs", "launches_per_step")}
               for k, v in kinds.items()}
    return roof, by_kind


def clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def clocks_stop(handle, path, device_index=0):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    rows = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(device_index):
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
        except ValueError:
            continue
    if not rows:
        return None
    mx = max(r[1] for r in rows)
    loaded = [r for r in rows if r[0] > 0.5 * mx] or rows
    reasons = set()
    for r in rows:
        for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], r[2:]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------------------- #
# CPU oracle timing (baseline and reference arm)                              #
# --------------------------------------------------------------------------- #
def oracle_rate(cfg, counts, shift=0, n_shifts=1):
    """Time the oracle as it stands (serial, one core) on counts[l] samples of level l
    for shifts shift..shift+n_shifts-1."""
    import oracle as O

    z, _ = O.cbc(cfg["s"], cfg["log2_nmax"])
    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"], corr_len=cfg["corr_len"],
                   qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"], sampler=cfg["sampler"],
                   seed=cfg["seed"], R=cfg["R"], genvec=z, log2_nmax=cfg["log2_nmax"], reuse=cfg["reuse"])
    work = [(lv, 0, int(c), shift, shift + n_shifts) for lv, c in enumerate(counts) if c > 0]
    t0 = time.perf_counter()
    orc.sample_levels(work)
    dt = time.perf_counter() - t0
    return n_samples(work), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload_config(0)
    counts = list(cfg["counts"])
    times = []
    for i in range(args.warmup + args.steps):
        ns, dt = oracle_rate(cfg, counts, shift=i % cfg["R"])
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = ns * len(times) / total
    sample = (f"per step: one shift (of 16), N_l = {counts} samples of levels 0..5 "
              f"({ns} FMG solves, 1/16 of the step, same level mix)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "MLQMC with reuse, FP64, 6 levels 8x8..256x256, s=100, R=16, "
                                   "N_l=1024..32 (bounded sample on CPU)", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# GPU arm                                                                    #
# --------------------------------------------------------------------------- #
def timed_steps(step, K, stream, flush):
    """K steps, each bracketed by CUDA events on the launch stream, L2 flushed
    (512 MiB write) before each outside the events; per-step milliseconds."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def profiled_pass(ctx, step, args, stream, flush):
    """K more steps with the library's per-kernel event brackets on (two
    untimed calls first: the graph is captured again with its brackets):
    per-kind (ms, launches), algorithmic work, and the mean step time of
    the pass. Profiling is off again afterwards (two more untimed calls
    restore the plain graph)."""
    ctx.profile(True)
    for _ in range(2):
        step()
    ctx.profile(True)  # clear the totals of those two calls
    ms = timed_steps(step, args.steps, stream, flush)
    prof = ctx.profile_read()
    work = ctx.profile_work()
    ctx.profile(False)
    for _ in range(2):
        step()
    return prof, work, sum(ms) / len(ms)


def force_smoother(ctx, name, plan=""):
    if ctx.precision == "fp64":
        return
    import paper_1806_05619_gb300 as M
    if name != "auto":
        for t in range(1, ctx.n_levels):
            try:
                ctx.set_smoother(t, name)
            except M.MlqmcError:
                pass
    for item in filter(None, plan.split(",")):
        lv, kind = item.split(":")
        ctx.set_smoother(int(lv), kind)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1806_05619_gb300 as M

    measured_peaks_override()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(M.LIB_PATH):
        raise RuntimeError("libmlqmc.so is not built; run __graft_entry__.build()")

    cfg = workload_config(rank, args.counts_div)
    cfg["precision"] = args.precision
    work = work_list(cfg)
    ns = n_samples(work)
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    ctx = M.Context.from_config(cfg, genvec=genvec, max_samples=ns)
    force_smoother(ctx, args.smoother, args.smoother_plan)
    ctx.set_graphs(not args.no_graphs)
    nl, R = cfg["n_levels"], cfg["R"]
    sums = torch.zeros(nl * R * 2, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        sums.zero_()
        ctx.sample_levels(work, sums, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up: the repeated step is captured as one CUDA graph on its second call
    for _ in range(args.warmup):
        step()
    ctx.check_device(stream)
    barrier()

    # device-timed steps (L2 flushed between steps, outside the events)
    clk_path = os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")
    clk = clocks_start(clk_path)
    launches0 = ctx.launch_count()
    replays0 = ctx.graph_replays()
    barrier()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees these steps only
    step_ms = timed_steps(step, args.steps, stream, flush)
    torch.cuda.profiler.stop()
    barrier()
    launches = ctx.launch_count() - launches0
    replays = ctx.graph_replays() - replays0
    clocks = clocks_stop(clk, clk_path, device_index=local)
    tot_ms = sum(step_ms)
    t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot_ms = float(t.item())
    ctx.check_device(stream)
    value = ns * world * args.steps / (tot_ms * 1e-3)

    # the same K steps again with every kernel bracketed by events (the
    # library's per-kind timing and algorithmic work): roofline per kind
    prof, pwork, prof_ms = profiled_pass(ctx, step, args, stream, flush)

    # end to end through the public API from the host: work list in, estimate out
    e2e_times = []
    host_sums = torch.empty(nl * R * 2, dtype=torch.float64, pin_memory=True)
    for i in range(args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        step()
        host_sums.copy_(sums, non_blocking=True)
        torch.cuda.synchronize(dev)
        S = host_sums.numpy().reshape(nl, R, 2)
        # estimator from the sums (eqs. Upsilon-reuse, MGMLQMC, var_of_mgmlqmc)
        cnt = np.cumsum(np.array(cfg["counts"][::-1]))[::-1]
        Ups = S[:, :, 0] / cnt[:, None]
        Qr = Ups.sum(axis=0)
        est = (Qr.mean(), Qr.var(ddof=1) / R)
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = torch.tensor([sum(e2e_times)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = ns * world * args.steps / float(e2e_t.item())
    h2d = len(work) * 32 + ns * (24 + 8)  # work list + the library's per-sample descriptors
    d2h = nl * R * 2 * 8

    # roofline of the dominant kernel kind: the library's event timing of each
    # launch inside the timed region and the algorithmic work it recorded
    smoothers = [k for k, _ in ctx.smoother_info()]
    roof, by_kind = roofline_report(prof, pwork, args.steps, form=cfg["precision"], smoothers=smoothers)

    mixed = None
    if not args.no_mixed and cfg["precision"] == "fp64":
        mixed = run_mixed_same_workload(args, cfg, work, genvec, dev, stream, flush, M)
    precision_form = None
    if not args.no_precision and rank == 0 and args.counts_div == 1:
        precision_form = run_precision_form(dev, stream, flush, M)
    tte = None
    if not args.no_tte and rank == 0 and args.counts_div == 1:
        tte = run_time_to_eps(M)

    matern = None
    if not args.no_matern and rank == 0 and args.counts_div == 1:
        try:
            matern = run_matern(cfg, work, genvec, dev, stream, flush, M)
        except Exception as e:  # reported in the line; the main measurement stands
            matern = {"error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = [max(1, c // 2) for c in cfg["counts"]]
        nsc, dt = oracle_rate(cfg, counts, shift=0, n_shifts=cfg["R"])
        cpu = {"value": nsc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"all 16 shifts, N_l/2 = {counts} samples of levels 0..5 ({nsc} FMG solves, "
                         f"half the step, same level mix), serial oracle, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if cfg["precision"] == "fp64" else "f32 V-cycles in f64 refinement",
            "data": "synthetic",
            "config": {"workload": "MLQMC with reuse, FP64, 6 levels 8x8..256x256 cells, s=100 KL modes "
                                   "(sep. exponential, sigma=1, lambda=0.3), lattice 2^10 points halving per "
                                   "level, R=16 shifts, N_l=1024,512,256,128,64,32 per shift, FMG mu0=2 V(2,2) "
                                   "RB-GS, mean-of-u QoI",
                       "precision": cfg["precision"], "smoothers": smoothers,
                       "samples_per_step": ns * world, "counts_div": args.counts_div,
                       "l2": "flushed between timed steps (512 MiB write)",
                       "parallelism": f"independent replicas x{world}"},
            "gpu_launches": launches,
            "graph_replays": replays,
            "profiled_pass_ms_per_step": prof_ms,
            "roofline": roof,
            "roofline_by_kind": by_kind,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "estimate": {"Q": float(est[0]), "varQ": float(est[1])}},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        if mixed:
            line["mixed"] = mixed
        if precision_form:
            line["precision_form"] = precision_form
        if tte:
            line["time_to_eps"] = tte
        if matern:
            line["matern"] = matern
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_matern(cfg, work, genvec, dev, stream, flush, M, steps=5, warmup=3):
    """The same 6-level step with the Matern covariance (eq. matern, nu = 1,
    the main step's lambda and sigma) whose KL modes are Nystrom eigenpairs on
    16 x 16 nodes (Sec. 5): the eigensolve and create times (the per-level
    Nystrom interpolation runs at create) and device-timed steps in the FP64
    and mixed TF32 forms, L2 flushed between steps."""
    import torch

    nu, m = 1.0, 16
    t0 = time.perf_counter()
    th, ps = M.nystrom_modes(nu, cfg["corr_len"], cfg["sigma"], m, cfg["s"])
    out = {"workload": f"6 levels 8x8..256x256, s={cfg['s']} Nystrom modes of the Matern covariance "
                       f"(nu={nu}, lambda={cfg['corr_len']}, sigma={cfg['sigma']}) on {m}x{m} nodes; the main "
                       "step's counts, shifts and FMG",
           "eigensolve_seconds": time.perf_counter() - t0}
    ns = n_samples(work)
    sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device=dev)
    for prec in ("fp64", "mixed_tf32"):
        c = dict(cfg)
        c["precision"] = prec
        t0 = time.perf_counter()
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=ns, covariance="matern", matern_nu=nu,
                                    nystrom_m=m, nystrom_theta=th, nystrom_psi=ps)
        torch.cuda.synchronize(dev)  # the per-level interpolation it queued
        create_s = time.perf_counter() - t0

        def step():
            sums.zero_()
            ctx.sample_levels(work, sums, stream=stream)

        for _ in range(warmup):
            step()
        ctx.check_device(stream)
        torch.cuda.synchronize(dev)
        ms = float(np.mean(timed_steps(step, steps, stream, flush)))
        ctx.check_device(stream)
        out[prec] = {"create_seconds": create_s, "ms_per_step": ms, "samples_per_s": ns / (ms * 1e-3)}
        ctx.close()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed_tf32"]["ms_per_step"]
    return out


def run_mixed_same_workload(args, cfg64, work, genvec, dev, stream, flush, M):
    """The same step with FP32 V-cycles inside FP64 refinement (mu0 refinement
    steps per level, each one FP32 V(2,2)-cycle on the FP64 residual)."""
    import torch

    cfg = dict(cfg64)
    cfg["precision"] = "mixed_tf32"
    ns = n_samples(work)
    ctx = M.Context.from_config(cfg, genvec=genvec, max_samples=ns)
    force_smoother(ctx, args.smoother, args.smoother_plan)
    ctx.set_graphs(not args.no_graphs)
    nl, R = cfg["n_levels"], cfg["R"]
    sums = torch.zeros(nl * R * 2, dtype=torch.float64, device=dev)

    def step():
        sums.zero_()
        ctx.sample_levels(work, sums, stream=stream)

    for _ in range(args.warmup):
        step()
    ctx.check_device(stream)
    torch.cuda.synchronize(dev)
    ms = timed_steps(step, args.steps, stream, flush)
    tot = sum(ms)
    prof, pwork, prof_ms = profiled_pass(ctx, step, args, stream, flush)
    ctx.check_device(stream)
    roof, by_kind = roofline_report(prof, pwork, args.steps, form="mixed_tf32",
                                    smoothers=[k for k, _ in ctx.smoother_info()])
    return {"value": ns * args.steps / (tot * 1e-3), "unit": UNIT, "ms_per_step": tot / args.steps,
            "dtype": "f32 V-cycles in f64 refinement, TF32 tensor-core KL, f32 field",
            "roofline": roof, "roofline_by_kind": by_kind, "profiled_pass_ms_per_step": prof_ms,
            "graph_replays": ctx.graph_replays(),
            "smoothers": [{"level": t, "kind": k, "tuned_ms": ms} for t, (k, ms) in enumerate(ctx.smoother_info())]}


def run_precision_form(dev, stream, flush, M):
    """Precision form: one batch of 256 samples whose FMG ends on the 1024x1024
    level (8 levels from 8x8), s = 400 KL modes (lambda = 0.1), 16 shifts x 16
    lattice points, every level refined to ||r||_2/||b||_2 <= 1e-10: the mixed
    forms (TF32 or split-BF16 tensor-core KL, FP32 V-cycles, FP64 residual and
    correction) against the all-FP64 GPU form, timing per batch and the mixed
    results' deviation from the FP64 ones (field, solution, F on every level)."""
    import torch

    cfg = dict(W.PRECISION_1024)
    cfg["log2_nmax"] = 10
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    top = cfg["n_levels"] - 1
    work = [(top, 0, 16, 0, 16)]
    ns = n_samples(work)
    nl, R = cfg["n_levels"], cfg["R"]
    out = {"workload": "256 samples (16 shifts x 16 points) on 8 levels 8x8..1024x1024, s=400, lambda=0.1, "
                       "refined to relative residual 1e-10 on every level"}
    res = {}
    for prec in ["mixed_tf32", "mixed_bf16x3", "fp64"]:
        c = dict(cfg)
        c["precision"] = prec
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=ns)
        sums = torch.zeros(nl * R * 2, dtype=torch.float64, device=dev)
        F = torch.zeros(ns * nl, dtype=torch.float64, device=dev)
        ctx.sample_levels(work, sums, F, stream=stream)  # warm-up (pools)
        ctx.check_device(stream)
        times = []
        for _ in range(2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sums.zero_()
            e0.record(stream)
            ctx.sample_levels(work, sums, F, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        ctx.check_device(stream)
        y = ctx.normals(top, 3, 5, 4)
        kf = ctx.fields(top, y)
        u, Fs = ctx.sample_solution(top, 3, 5)
        res[prec] = dict(ms=min(times), F=F.cpu().numpy().reshape(ns, nl), k=kf.cpu().numpy(),
                         u=u[top].cpu().numpy())
        out[prec] = {"ms_per_batch": min(times), "samples_per_s": ns / (min(times) * 1e-3)}
        del ctx
        torch.cuda.empty_cache()
    b = res["fp64"]
    for prec in ["mixed_tf32", "mixed_bf16x3"]:
        a = res[prec]
        out[prec]["speedup_over_fp64"] = b["ms"] / a["ms"]
        out[prec]["err_vs_fp64"] = {
            "field_max_abs_log_ratio": float(np.max(np.abs(np.log(a["k"] / b["k"])))),
            "solution_max_rel": float(np.max(np.abs(a["u"] - b["u"])) / np.max(np.abs(b["u"]))),
            "F_max_rel_per_level": [float(np.max(np.abs(a["F"][:, t] / b["F"][:, t] - 1))) for t in range(nl)],
        }
    return out


def run_time_to_eps(M):
    """Time to RMSE eps of Algorithm 1 (exact one-level-per-round form,
    deterministic cost model) on the 7-level adaptive problem (8x8..512x512,
    s = 200, lambda = 0.3, 16 shifts, mean-of-u QoI, every level refined to
    1e-10), mixed form against the FP64 form, for eps in {1e-2, 3e-3, 1e-3}
    and two smaller tolerances (3e-4, 1e-4) where the runs take longer."""
    from paper_1806_05619_gb300 import rates

    cfg = dict(W.ADAPTIVE_7LEVEL)
    cfg["log2_nmax"] = 12
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    out = {"workload": "Algorithm 1 on 7 levels 8x8..512x512, s=200, lambda=0.3, R=16, rtol 1e-10",
           "variants": "mixed_tf32 / fp64: reuse (MG-MLQMC), one level per round; mixed_tf32_no_reuse: plain "
                       "MLQMC (each difference from its own samples); mixed_tf32_batched: every level with "
                       "V_l/C_l >= max/2 doubles in one round; mlmc_mixed_tf32: plain MLMC (Monte Carlo "
                       "normals, one replicate, eq. nopt counts)"}
    variants = [("mixed_tf32", "mixed_tf32", True, False), ("fp64", "fp64", True, False),
                ("mixed_tf32_no_reuse", "mixed_tf32", False, False), ("mixed_tf32_batched", "mixed_tf32", True, True)]
    for name, prec, reuse, batched in variants:
        c = dict(cfg)
        c["precision"] = prec
        c["reuse"] = reuse
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=1 << 17)
        rows = []
        for eps in cfg["eps"] + [3e-4, 1e-4]:
            r = ctx.estimate(eps, batched=batched)
            rows.append({"eps": eps, "seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                         "rmse_bound": float(np.sqrt(r["varQ"] + r["bias"] ** 2)), "L": r["L"],
                         "rounds": r["rounds"], "N": r["N"][:r["L"] + 1], "run_status": r["run_status"],
                         "alpha": r["alpha"], "Ybar": r["Ybar"][:r["L"] + 1], "Vell": r["Vell"][:r["L"] + 1]})
        out[name] = rows
        if name == "mixed_tf32":
            # rates of (A1)-(A4) on the same problem, and Proposition 1 against
            # the recycling runs: the predicted factor, the factor the run's own
            # counts give with the measured per-sample costs, and the measured
            # device-time ratio to the run without recycling
            out["rates"] = rates.measure(ctx, n_points=256, lambda_level=2, gamma_levels=3)
        del ctx
    rt = out["rates"]
    prop = {"predicted": rt["prop1_ratio"], "from_counts": [], "measured_gpu_time": []}
    for a, b in zip(out["mixed_tf32"], out["mixed_tf32_no_reuse"]):
        L = a["L"]
        used = np.cumsum(np.array(a["N"][:L + 1], dtype=np.float64)[::-1])[::-1]  # samples on level l
        prop["from_counts"].append({"eps": a["eps"],
                                    "ratio": rates.reuse_cost_ratio(used, rt["ms_per_sample"][:L + 1])})
        prop["measured_gpu_time"].append({"eps": a["eps"], "ratio": a["gpu_seconds"] / b["gpu_seconds"]})
    out["prop1"] = prop
    # plain MLMC (Monte Carlo normals, no recycling, eq. nopt counts) on the same
    # problem, and the paper's speed-ups (Tab. speedup) in device time:
    # S1 = MLMC / MLQMC, S2 = MLMC / MG-MLQMC, S3 = MLQMC / MG-MLQMC
    c = dict(cfg)
    c.update(precision="mixed_tf32", sampler="mc", R=1, reuse=False)
    ctx = M.Context.from_config(c, max_samples=1 << 17)
    rows = []
    for eps in cfg["eps"] + [3e-4, 1e-4]:
        r = ctx.estimate_mlmc(eps)
        rows.append({"eps": eps, "seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                     "rmse_bound": float(np.sqrt(r["varQ"] + r["bias"] ** 2)), "L": r["L"],
                     "rounds": r["rounds"], "N": r["N"][:r["L"] + 1], "run_status": r["run_status"]})
    del ctx
    out["mlmc_mixed_tf32"] = rows
    # also in work (cells of the FMG hierarchy per sample, sum_{t<=l} n_t^2, times samples
    # and replicates): the paper's one-sample-per-core cost, which device time on a
    # latency-bound GPU does not follow
    model = np.cumsum([(cfg["n0"] << t) ** 2 for t in range(cfg["n_levels"])])

    def work(row, R):
        return R * float(np.dot(row["N"], model[:len(row["N"])]))

    sp = []
    for m, q, g in zip(rows, out["mixed_tf32_no_reuse"], out["mixed_tf32"]):
        wm, wq, wg = work(m, 1), work(q, cfg["R"]), work(g, cfg["R"])
        sp.append({"eps": m["eps"], "S1": m["gpu_seconds"] / q["gpu_seconds"],
                   "S2": m["gpu_seconds"] / g["gpu_seconds"], "S3": q["gpu_seconds"] / g["gpu_seconds"],
                   "S1_work": wm / wq, "S2_work": wm / wg, "S3_work": wq / wg})
    keys = ("S1", "S2", "S3", "S1_work", "S2_work", "S3_work")
    out["speedups"] = {"per_eps": sp, "mean": {k: float(np.mean([x[k] for x in sp])) for k in keys}}
    out["mimc"] = run_mimc(M, cfg, genvec, model)
    return out


def run_mimc(M, cfg, genvec, model):
    """Multi-index variant (grid level x V-cycle count, the outlook of Sec. 7)
    on the same 7-level problem in the fixed-cycle mixed form: contexts with
    mu0 = 1, 2, 3 (levels adaptive, every cycle count at each level), against
    Algorithm 1 with mu0 = 3 (the mean both converge to), in device time and in
    work (cells of the FMG hierarchy x V-cycles per level, times samples and
    shifts)."""
    mus = (1, 2, 3)
    c = dict(cfg)
    c.update(precision="mixed_tf32", rtol=0.0)
    ctxs = [M.Context.from_config(c, genvec=genvec, mu0=mu, max_samples=1 << 17) for mu in mus]
    rows = []
    for eps in cfg["eps"] + [3e-4]:
        r = M.estimate_mimc(ctxs, eps)
        a = ctxs[-1].estimate(eps)
        w_mimc = float(cfg["R"] * sum(r["N"][m][t] * float(model[t]) * (mus[m] + (mus[m - 1] if m else 0))
                                      for m in range(len(mus)) for t in range(len(r["N"][m]))))
        w_alg1 = cfg["R"] * mus[-1] * float(np.dot(a["N"][:a["L"] + 1], model[:a["L"] + 1]))
        rows.append({"eps": eps, "mimc": {"seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                                          "varQ": r["varQ"], "bias": r["bias"], "bias_cycles": r["bias_cycles"],
                                          "L": r["L"], "N": r["N"], "rounds": r["rounds"],
                                          "run_status": r["run_status"], "work": w_mimc},
                     "alg1_mu3": {"seconds": a["wall_seconds"], "gpu_seconds": a["gpu_seconds"], "Q": a["Q"],
                                  "varQ": a["varQ"], "bias": a["bias"], "L": a["L"], "N": a["N"][:a["L"] + 1],
                                  "rounds": a["rounds"], "run_status": a["run_status"], "work": w_alg1},
                     "gpu_time_ratio": a["gpu_seconds"] / r["gpu_seconds"], "work_ratio": w_alg1 / w_mimc})
    for x in ctxs:
        x.close()
    return {"workload": "7 levels 8x8..512x512, s=200, lambda=0.3, R=16, mixed_tf32 with fixed cycles, "
                        "mu0 in {1,2,3}, levels adaptive; ratios are Algorithm 1 (mu0=3) over the multi-index run",
            "rows": rows}


def main():
    args = parse()
    if args.traffic_from:
        # fold an ncu capture of one timed step (see profiles/) into the traffic file
        with open(args.traffic_line) as f:
            line = json.loads([ln for ln in f if ln.startswith("{")][-1])
        form = line["config"]["precision"]
        rec = summarize_traffic(args.traffic_from, form, line["config"]["smoothers"])
        print(json.dumps({form: rec}, indent=1))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
