#!/usr/bin/env python3
"""Throughput of the MG-MLQMC hot path on one GB300 (samples/s, KL + FMG).

Workload (default): the 9-level problem, 8x8 .. 2048x2048 cells, s = 1000 KL
modes of the separable exponential covariance (sigma = 1, correlation length
0.05), rank-1 lattice (CBC, gamma_j = j^-2, 2^12 points) with R = 16 random
shifts, FMG with mu0 = 2 V(2,2)-cycles per level, mean-of-u QoI, recycling.
One step = one call of mlqmc_sample_levels on 16 points per shift on the
finest level doubling per coarser level (N_l = 4096 .. 16 per shift on levels
0..8: 256 finest fields, 130,816 samples): normals, fields on every level of
every sample, FMG, F_t and the reuse sums of every level.

The headline `value` is the mixed-precision form (TF32 tensor-core KL, FP32
V-cycles inside FP64 refinement, FP64 sums); the all-FP64 form of the same
step is reported beside it (`fp64`), and Algorithm 1's time to RMSE eps for
both forms under `time_to_eps`. The last stdout line is the compact record;
side studies (`--extras`: the 6-level step in both forms, the 1024x1024
precision form, Algorithm 1 on the 7-level problem with rates, Prop. 1,
speed-ups and the multi-index variant, the Matern step) go to earlier lines
and to `--details-out`.

`--impl reference` times the CPU oracle as it stands on bounded samples of
the same workload, spread over the host cores.

Multi-GPU (torchrun): each rank runs an independent replica (its own seed);
no data-path collective; value = all ranks' samples / max time ("weak").
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import multiprocessing as mp
import os
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
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 form of the step")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 form (one warm-up)")
    ap.add_argument("--no-tte", action="store_true", help="skip Algorithm 1's time to eps on the 9-level problem")
    ap.add_argument("--no-per-level", action="store_true", help="skip the samples/s per finest level")
    ap.add_argument("--tte-profile", action="store_true",
                    help="only Algorithm 1 (mixed, one level per round) to --tte-eps on the 9-level problem, "
                         "inside a profiler range, for a launch list")
    ap.add_argument("--tte-eps", type=float, default=1e-4)
    ap.add_argument("--extras", action="store_true",
                    help="side studies: 6-level step, 1024x1024 precision form, 7-level Algorithm 1 runs, Matern")
    ap.add_argument("--details-out", default="", help="write the side results (JSON) to this file")
    ap.add_argument("--workload", default="mlqmc9", choices=["mlqmc9", "mlqmc6"])
    ap.add_argument("--smoother", default="auto", choices=["auto", "stream", "tma", "tile"],
                    help="mixed form: force this smoother on every level it handles (default: the autotuner's pick)")
    ap.add_argument("--smoother-plan", default="",
                    help="mixed form: pin smoothers per level, e.g. 1:whole,2:whole,4:tma")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernel by kernel instead of replaying a CUDA graph")
    ap.add_argument("--counts-div", type=int, default=1,
                    help="divide the per-level counts (small cases for profiler captures only)")
    ap.add_argument("--cpu-workers", type=int, default=0, help="oracle processes (0: every host core)")
    ap.add_argument("--shifts", type=int, default=0,
                    help="override R (profiler captures only, to keep the device footprint small)")
    ap.add_argument("--modes", type=int, default=0,
                    help="override s (profiler captures of the grid kernels only, to keep the KL tables small)")
    ap.add_argument("--kl-shape", default="",
                    help="N,S,B: time only the tensor-core KL contraction of B samples on an N x N level with S modes")
    return ap.parse_args(argv)


WORKLOADS = {
    "mlqmc9": (W.ADAPTIVE_9LEVEL,
               "MG-MLQMC with reuse, 9 levels 8x8..2048x2048, s=1000 (sep. exp., sigma=1, lambda=0.05), lattice "
               "2^12 pts, R=16, N_l=4096..16 per shift (130,816 samples, 256 finest), FMG mu0=2 V(2,2) RB-GS, "
               "mean-of-u QoI"),
    "mlqmc6": (W.LATTICE_6LEVEL,
               "MG-MLQMC with reuse, 6 levels 8x8..256x256, s=100 (sep. exp., sigma=1, lambda=0.3), lattice 2^10 "
               "pts, R=16, N_l=1024..32 per shift (32,256 samples), FMG mu0=2 V(2,2) RB-GS, mean-of-u QoI"),
}


def workload_config(name, rank=0, counts_div=1, precision=None, modes=0, shifts=0):
    cfg = dict(WORKLOADS[name][0])
    if shifts:
        cfg["R"] = shifts
    cfg["seed"] = cfg["seed"] + 1000 * rank
    cfg["counts"] = [max(1, c // counts_div) for c in cfg["counts"]]
    if precision:
        cfg["precision"] = precision
    if modes:
        cfg["s"] = modes
    return cfg


def n_samples(work):
    return sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in work)


# --------------------------------------------------------------------------- #
# Roofline denominators                                                       #
# --------------------------------------------------------------------------- #
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def peaks():
    """Denominators of the roofline fractions: the measured copy bandwidth and
    cuBLAS bf16 rates of the GB300s (MEASURED_PEAKS.json), else the
    fallback figures; TF32 = bf16 x the nominal TF32/BF16 ratio 1.1/2.25;
    FP64 = 1.20 TFLOP/s from an FMA probe on this machine's GB300 (nominal 1.25);
    FP32 = 152 SMs x 128 lanes x 2 x 2070 MHz."""
    pk = measured_peaks()
    P = {"hbm": 6800.0, "hbm_src": "fallback 6.8 TB/s", "bf16": 1900.0, "bf16_sust": 1700.0,
         "tc_src": "fallback bf16 1.9 / 1.7 PFLOP/s"}
    if pk.get("hbm_gbs"):
        P["hbm"], P["hbm_src"] = float(pk["hbm_gbs"]), "measured copy bandwidth"
    if pk.get("bf16_tflops"):
        P["bf16"] = float(pk["bf16_tflops"])
        P["bf16_sust"] = float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"]))
        P["tc_src"] = "measured bf16 (sustained) x nominal tf32/bf16 1.1/2.25"
    P["tf32_sust"] = P["bf16_sust"] * 1.1 / 2.25
    P["fp64"] = 1.20
    P["fp32"] = 152 * 128 * 2 * 2.070e9 / 1e12
    return P


KIND_KERNELS = {
    "points": "k_points", "level0": "kb_level0_fixed", "synth": "kb_synth_G/z, kb_faces",
    "transfer": "kb_prolong_resid_tma, kb_resid_restrict, kb_prolong(_resid64)", "coarse": "kb_coarse_fixed",
    "reduce": "kb_qoi(_part), k_sums", "kl_tc": "kl_tc_kernel (tcgen05)",
}
SMOOTHER_KERNELS = {"whole": "kb_rbgs_whole", "tma": "kb_rbgs_tma", "stream": "kb_rbgs_stream", "tile": "kb_rbgs_tile",
                    "gs": "kb_gs"}


def kernel_name(kind, level, smoothers):
    if kind == "smooth" and level is not None:
        return SMOOTHER_KERNELS[smoothers[level]]
    return KIND_KERNELS.get(kind, kind)


def bucket_roofline(cell, P):
    """Roofline of one (kind, level) bucket from its event time and algorithmic
    work: the bound is the resource whose model time (bytes / HBM; FLOPs / the
    pipe's peak) is longest; achieved = work / time; frac = achieved / peak."""
    t = cell["ms"] * 1e-3
    cand = [("hbm", cell["bytes"] / (P["hbm"] * 1e9)), ("alu64", cell["f64"] / (P["fp64"] * 1e12)),
            ("alu32", cell["f32"] / (P["fp32"] * 1e12)), ("tensor", cell["ftc"] / (P["tf32_sust"] * 1e12))]
    bound, tm = max(cand, key=lambda x: x[1])
    if t <= 0 or tm <= 0:
        return None
    if bound == "hbm":
        r = dict(bound="hbm", achieved=cell["bytes"] / t / 1e9, peak=P["hbm"], unit="GB/s", peak_src=P["hbm_src"])
    elif bound == "tensor":
        r = dict(bound="tensor", achieved=cell["ftc"] / t / 1e12, peak=P["tf32_sust"], unit="TFLOP/s",
                 peak_src=P["tc_src"])
    elif bound == "alu64":
        r = dict(bound="alu", achieved=cell["f64"] / t / 1e12, peak=P["fp64"], unit="TFLOP/s",
                 peak_src="FP64 1.20 TFLOP/s (FMA probe)")
    else:
        r = dict(bound="alu", achieved=cell["f32"] / t / 1e12, peak=P["fp32"], unit="TFLOP/s",
                 peak_src="FP32 152x128x2x2070 MHz")
    r["frac"] = r["achieved"] / r["peak"]
    return r


def sources_digest(files=None):
    """SHA-256 over source files (paths relative to the repository; default:
    the library's CUDA/C++ sources and header): DRAM counters taken on other
    sources no longer describe these kernels."""
    if files is None:
        files = sorted(os.path.relpath(f, ROOT) for f in glob.glob(os.path.join(ROOT, "paper_1806_05619_gb300", "csrc", "*"))
                       if f.endswith((".cu", ".cuh", ".h", ".cpp")))
        files.append("include/mlqmc.h")
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(form, kernel, n):
    """DRAM bytes per algorithmic byte of `kernel` on an n x n level in `form`:
    the ratio over one-kernel ncu captures on a small case (the capture
    commands and the algorithmic bytes of each captured launch are in the
    record, profiles/dram_traffic.json); the traffic of a launch in the timed
    step is that ratio times its algorithmic bytes, i.e. the captured traffic
    scaled by the cells processed. None when absent or when the kernel's
    source files differ from those the record was taken on."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    e = rec.get("kernels", {}).get(f"{form}|{kernel}|{n}")
    if not e or sources_digest(e.get("sources")) != e.get("sources_sha256"):
        return None
    return e.get("dram_per_alg_byte")


def roofline_report(ctx, levels_prof, P, form, steps):
    """The dominant (kernel kind, level) bucket of the profiled steps as the
    bench line's `roofline`, and every bucket with at least 1 % of the time."""
    smoothers = [k for k, _ in ctx.smoother_info()]
    tot = sum(v["ms"] for v in levels_prof.values())
    rows = []
    for (kind, lv), cell in levels_prof.items():
        r = bucket_roofline(cell, P)
        if r is None:
            continue
        r.update(kind=kind, level=lv, kernel=kernel_name(kind, lv, smoothers), share=cell["ms"] / max(tot, 1e-12),
                 ms_per_step=cell["ms"] / steps, launches_per_step=cell["n"] / steps,
                 n=(ctx.n(lv) if lv is not None else None))
        rows.append(r)
    rows.sort(key=lambda r: -r["share"])
    dom = next(r for r in rows if r["level"] is not None)
    per_launch_bytes = levels_prof[(dom["kind"], dom["level"])]["bytes"] / max(1, levels_prof[(dom["kind"], dom["level"])]["n"])
    ratio = measured_traffic(form, dom["kernel"], dom["n"])
    traffic = round(ratio * per_launch_bytes) if ratio is not None else None
    roof = {"bound": dom["bound"], "achieved": round(dom["achieved"], 1), "peak": dom["peak"], "unit": dom["unit"],
            "frac": round(dom["frac"], 3), "traffic": traffic,
            "kernel": f"{dom['kernel']} on {dom['n']}x{dom['n']}", "share": round(dom["share"], 3),
            "alg_bytes_per_launch": per_launch_bytes, "peak_src": dom["peak_src"] + " (of measured)"
            if "measured" in dom["peak_src"] else dom["peak_src"]}
    table = [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()
              if k in ("kernel", "level", "bound", "achieved", "unit", "frac", "share", "ms_per_step",
                       "launches_per_step")} for r in rows if r["share"] >= 0.01]
    return roof, table


# --------------------------------------------------------------------------- #
# Clocks during the timed region                                              #
# --------------------------------------------------------------------------- #
def clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except OSError:
        return None, None


def clocks_summary(lines, device_index=0):
    """Median SM clock under load, the maximum, and every throttle reason seen."""
    rows = []
    for line in lines:
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


def clocks_stop(handle, path, device_index=0):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.close()
    with open(path) as fh:
        return clocks_summary(fh.readlines(), device_index)


# --------------------------------------------------------------------------- #
# CPU oracle timing (baseline and reference arm), one process per core        #
# --------------------------------------------------------------------------- #
def _oracle_job(job):
    """One oracle process: the samples of `work` as the oracle computes them
    (serial, as it stands); returns (samples, seconds)."""
    cfg, genvec, work = job
    import oracle as O

    orc = O.Oracle(n_levels=cfg["n_levels"], n0=cfg["n0"], s=cfg["s"], sigma=cfg["sigma"], corr_len=cfg["corr_len"],
                   qoi=cfg["qoi"], mu0=cfg["mu0"], nu1=cfg["nu1"], nu2=cfg["nu2"], rtol=cfg["rtol"],
                   sampler=cfg["sampler"], seed=cfg["seed"], R=cfg["R"], genvec=genvec,
                   log2_nmax=cfg["cpu_log2_nmax"], reuse=cfg["reuse"])
    t0 = time.perf_counter()
    orc.sample_levels(work)
    return n_samples(work), time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample_setup(cfg, div):
    """The oracle's own generating vector for the points a CPU sample uses and
    the per-shift counts of that sample (the step's counts / div, same level mix)."""
    import oracle as O

    counts = [max(1, c // div) for c in cfg["counts"]]
    m = max(1, int(np.ceil(np.log2(max(counts)))))
    c = dict(cfg)
    c["cpu_log2_nmax"] = m
    z, _ = O.cbc(cfg["s"], m)
    return c, [int(v) for v in z], counts


def oracle_pool_run(jobs, workers):
    """Run oracle jobs on `workers` spawned processes; wall seconds and per-job results."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=workers) as pool:
        pool.map(_oracle_job, [(jobs[0][0], jobs[0][1], [(0, 0, 1, 0, 1)])] * workers)  # load the oracle everywhere
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    return wall, res


def cpu_baseline(cfg, workers, div=16):
    """The oracle on every host core: the step's counts / div on all R shifts,
    one shift per job; value = samples / wall time. single_core = the mean
    per-process rate measured during the same run (all cores busy)."""
    c, z, counts = cpu_sample_setup(cfg, div)
    jobs = [(c, z, [(lv, 0, n, r, r + 1) for lv, n in enumerate(counts)]) for r in range(cfg["R"])]
    wall, res = oracle_pool_run(jobs, workers)
    ns = sum(r[0] for r in res)
    return {"value": ns / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "single_core": float(np.mean([r[0] / r[1] for r in res])),
            "sample": f"N_l/{div}={counts} per shift x {cfg['R']} shifts ({ns} samples), one shift per process, "
                      f"{wall:.1f} s wall; oracle lattice 2^{c['cpu_log2_nmax']} pts"}


def run_reference(args):
    """The oracle as it stands, spread over the host cores: each step is one
    shift's samples at the step's counts / 16 (same level mix, 511 samples);
    W warm-up steps, then K timed steps run concurrently, one per process."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload_config(args.workload)
    workers = args.cpu_workers or host_cores()
    c, z, counts = cpu_sample_setup(cfg, 16)

    def jobs(k, off):
        return [(c, z, [(lv, 0, n, (off + i) % cfg["R"], (off + i) % cfg["R"] + 1) for lv, n in enumerate(counts)])
                for i in range(k)]

    if args.warmup:
        oracle_pool_run(jobs(args.warmup, 0), min(workers, args.warmup))
    wall, res = oracle_pool_run(jobs(args.steps, args.warmup), min(workers, args.steps))
    ns = sum(r[0] for r in res)
    value = ns / wall
    sample = (f"per step one shift, N_l/16={counts} ({res[0][0]} samples); {args.steps} steps on "
              f"{min(workers, args.steps)} processes, {wall:.1f} s wall")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1] + " (bounded sample on the host cores)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(workers, args.steps), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# GPU arm                                                                     #
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


def per_level_rates(step, stream, flush, K, warm=2):
    """Samples/s per finest level: for each level l, a call with only the
    step's level-l samples (N_l points x R shifts; FMG on levels 0..l of each),
    `warm` untimed calls (the repeat is replayed as a graph, as in the step),
    then K calls device-timed with the L2 flushed before each."""
    cfg = step.cfg
    out = []
    for lv, n in enumerate(cfg["counts"]):
        if n <= 0:
            continue
        work = [(lv, 0, n, 0, cfg["R"])]

        def call():
            step.sums.zero_()
            step.ctx.sample_levels(work, step.sums, stream=stream)

        for _ in range(warm):
            call()
        ms = float(np.mean(timed_steps(call, K, stream, flush)))
        ns = n * cfg["R"]
        out.append({"level": lv, "n": step.ctx.n(lv), "samples": ns, "ms": round(ms, 4),
                    "samples_per_s": round(ns / (ms * 1e-3), 1)})
    step.ctx.check_device(stream)
    return out


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


class Step:
    """One context and the fixed-count step on it."""

    def __init__(self, M, cfg, genvec, dev, args, ns):
        import torch

        self.cfg = cfg
        self.work = W.fixed_count_work(cfg["counts"], cfg["R"])
        t0 = time.perf_counter()
        self.ctx = M.Context.from_config(cfg, genvec=genvec, max_samples=ns)
        torch.cuda.synchronize(dev)
        self.create_s = time.perf_counter() - t0
        force_smoother(self.ctx, args.smoother, args.smoother_plan)
        self.ctx.set_graphs(not args.no_graphs)
        self.sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device=dev)

    def __call__(self, stream):
        self.sums.zero_()
        self.ctx.sample_levels(self.work, self.sums, stream=stream)

    def profiled(self, stream, flush, K, warm=2, restore=True):
        """K steps with the library's per-launch event brackets (`warm`
        untimed calls first: the graph is captured again with its brackets);
        the per-(kind, level) times and work; plain replay restored afterwards
        when `restore`."""
        self.ctx.profile(True)
        for _ in range(warm):
            self(stream)
        self.ctx.profile(True)
        ms = timed_steps(lambda: self(stream), K, stream, flush)
        prof = self.ctx.profile_read_levels()
        self.ctx.profile(False)
        for _ in range(2 if restore else 0):
            self(stream)
        return prof, float(np.mean(ms))

    def close(self):
        self.ctx.close()


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1806_05619_gb300 as M

    P = peaks()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(M.LIB_PATH):
        raise RuntimeError("libmlqmc.so is not built; run __graft_entry__.build()")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    details = {}
    cfg = workload_config(args.workload, rank, args.counts_div, precision="mixed_tf32", modes=args.modes,
                          shifts=args.shifts)
    ns = n_samples(W.fixed_count_work(cfg["counts"], cfg["R"]))
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # ---- headline: the mixed form ------------------------------------------
    step = Step(M, cfg, genvec, dev, args, ns)
    for _ in range(args.warmup):  # the repeated step is captured as one CUDA graph on its second call
        step(stream)
    step.ctx.check_device(stream)
    barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")
    clk = clocks_start(clk_path)
    launches0, replays0 = step.ctx.launch_count(), step.ctx.graph_replays()
    barrier()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees these steps only
    step_ms = timed_steps(lambda: step(stream), args.steps, stream, flush)
    torch.cuda.profiler.stop()
    barrier()
    launches = step.ctx.launch_count() - launches0
    replays = step.ctx.graph_replays() - replays0
    clocks = clocks_stop(clk, clk_path, device_index=local)
    step.ctx.check_device(stream)
    tot_ms = max_over_ranks(sum(step_ms))
    value = ns * world * args.steps / (tot_ms * 1e-3)

    # per-(kernel, level) event timing of K more steps: the roofline
    prof, prof_ms = step.profiled(stream, flush, args.steps)
    roof, table = roofline_report(step.ctx, prof, P, "mixed_tf32", args.steps)
    details["roofline_table_mixed"] = table
    details["profiled_pass_ms_per_step"] = prof_ms

    # end to end through the public API from host memory: the host work list in
    # (the library uploads one 32-byte descriptor per sample), the reuse sums
    # back to pinned host memory, the estimator by mlqmc_estimator_from_sums
    nl, R = cfg["n_levels"], cfg["R"]
    host_sums = torch.empty(nl * R * 2, dtype=torch.float64, pin_memory=True)
    Nl = list(cfg["counts"])
    e2e_times = []
    est = None
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        step(stream)
        host_sums.copy_(step.sums, non_blocking=True)
        torch.cuda.synchronize(dev)
        est = M.estimator_from_sums(Nl, host_sums.numpy().reshape(nl, R, 2), R, reuse=cfg["reuse"])
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = ns * world * args.steps / max_over_ranks(sum(e2e_times))
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": ns * 32, "d2h_bytes_per_step": nl * R * 2 * 8}
    details["estimate_mixed"] = {"Q": est["Q"], "varQ": est["varQ"]}
    smoothers = [k for k, _ in step.ctx.smoother_info()]
    details["autotuner"] = {"smoothers": step.ctx.smoother_info(), "schedule": step.ctx.schedule_info()}
    if not args.no_per_level:
        details["per_finest_level"] = {"mixed_tf32": per_level_rates(step, stream, flush, args.steps)}
    create_mixed = step.create_s
    step.close()
    del step
    torch.cuda.empty_cache()

    # ---- the all-FP64 form of the same step --------------------------------
    fp64 = None
    if not args.no_fp64:
        c64 = dict(cfg)
        c64["precision"] = "fp64"
        s64 = Step(M, c64, genvec, dev, args, ns)
        s64(stream)
        s64.ctx.check_device(stream)
        torch.cuda.synchronize(dev)
        ms64 = timed_steps(lambda: s64(stream), args.fp64_steps, stream, flush)
        s64.ctx.check_device(stream)
        t64 = max_over_ranks(sum(ms64))
        fp64 = {"value": round(ns * world * args.fp64_steps / (t64 * 1e-3), 1),
                "ms_per_step": round(t64 / args.fp64_steps, 2), "steps": args.fp64_steps}
        host_sums.copy_(s64.sums)
        e64 = M.estimator_from_sums(Nl, host_sums.numpy().reshape(nl, R, 2), R, reuse=cfg["reuse"])
        details["estimate_fp64"] = {"Q": e64["Q"], "varQ": e64["varQ"]}
        prof64, _ = s64.profiled(stream, flush, 1, warm=0, restore=False)
        _, details["roofline_table_fp64"] = roofline_report(s64.ctx, prof64, P, "fp64", 1)
        fp64["speedup_mixed"] = round((t64 / args.fp64_steps) / (tot_ms / args.steps), 2)
        if not args.no_per_level:
            details.setdefault("per_finest_level", {})["fp64"] = per_level_rates(s64, stream, flush, 1, warm=1)
        s64.close()
        del s64
        torch.cuda.empty_cache()

    # ---- Algorithm 1 to eps on the same problem, both forms ----------------
    tte = None
    if not args.no_tte and rank == 0 and args.counts_div == 1 and args.workload == "mlqmc9":
        tte = run_tte9(M, cfg, args.tte_eps, dev)
        details["time_to_eps_9level"] = tte

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg, args.cpu_workers or host_cores())

    if rank == 0 and args.extras and args.counts_div == 1:
        details.update(run_extras(args, dev, stream, flush, M, P))

    if rank == 0:
        details_line = {"details": details}
        print(json.dumps(details_line, default=float), flush=True)
        if args.details_out:
            with open(args.details_out, "w") as f:
                json.dump(details, f, indent=1, default=float)
        line = make_line(args, world, value, tot_ms, ns, smoothers, create_mixed, launches, replays, roof, e2e,
                         clocks, cpu, fp64, tte)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def make_line(args, world, value, tot_ms, ns, smoothers, create_s, launches, replays, roof, e2e, clocks, cpu, fp64,
              tte):
    """The compact record printed last (well under 2 KB)."""
    if cpu:
        cpu = dict(cpu, value=round(cpu["value"], 2), single_core=round(cpu["single_core"], 2))
    return {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(tot_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycles in f64 refinement, tf32 KL", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][1], "precision": "mixed_tf32", "samples_per_step": ns * world,
                   "counts_div": args.counts_div, "smoothers": "".join(x[0] for x in smoothers),
                   "l2": "flushed (512 MiB write) between steps", "parallelism": f"independent replicas x{world}",
                   "create_s": round(create_s, 1)},
        "gpu_launches": launches, "graph_replays": replays, "roofline": roof,
        "e2e": {k: (round(v, 1) if isinstance(v, float) else v) for k, v in e2e.items()},
        "clocks": clocks, "cpu_baseline": cpu, "fp64": fp64,
        "time_to_eps": ({"eps": tte["eps"], "mixed_s": round(tte["mixed_tf32"]["seconds"], 3),
                         "fp64_s": round(tte["fp64"]["seconds"], 3) if "fp64" in tte else None,
                         "mixed_round_graphs_s": (round(tte["mixed_tf32_round_graphs"]["seconds"], 3)
                                                  if "mixed_tf32_round_graphs" in tte else None),
                         "mixed_batched_s": (round(tte["mixed_tf32_batched"]["seconds"], 3)
                                             if "mixed_tf32_batched" in tte else None),
                         "mixed_batched_rounds": (tte["mixed_tf32_batched"]["rounds"]
                                                  if "mixed_tf32_batched" in tte else None),
                         "fp64_batched_s": (round(tte["fp64_batched"]["seconds"], 3)
                                            if "fp64_batched" in tte else None),
                         "mixed_L": tte["mixed_tf32"]["L"], "mixed_rounds": tte["mixed_tf32"]["rounds"]}
                        if tte else None),
    }


def run_tte9(M, cfg, eps, dev):
    """Algorithm 1 (one level per round, deterministic cost model) to RMSE eps on
    the 9-level problem, mixed TF32 against FP64, wall and device seconds."""
    import torch

    out = {"eps": eps, "workload": "Algorithm 1 on the 9-level problem (s=1000, lambda=0.05, R=16), FMG mu0=2"}
    c = dict(cfg)
    c["log2_nmax"] = 14
    genvec, _ = M.cbc_genvec(c["s"], c["log2_nmax"])
    # the default policy launches a fixed-cycle round kernel by kernel; the
    # third run forces one graph launch per round for comparison; the batched
    # runs double every level whose V/C is within half of the largest in the
    # same round (all those levels' samples in one call, one graph launch)
    for name, prec, rounds, batched in (("mixed_tf32", "mixed_tf32", "converged", False),
                                        ("fp64", "fp64", "converged", False),
                                        ("mixed_tf32_round_graphs", "mixed_tf32", "on", False),
                                        ("mixed_tf32_batched", "mixed_tf32", "converged", True),
                                        ("mixed_tf32_batched_round_graphs", "mixed_tf32", "on", True),
                                        ("fp64_batched", "fp64", "converged", True)):
        c["precision"] = prec
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=1 << 16)
        ctx.set_round_graphs(rounds)
        r = ctx.estimate(eps, batched=batched)
        out[name] = {"seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                     "rmse_bound": float(np.sqrt(r["varQ"] + r["bias"] ** 2)), "L": r["L"], "rounds": r["rounds"],
                     "N": r["N"][:r["L"] + 1], "run_status": r["run_status"], "graphs": ctx.graph_stats()}
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------------------- #
# Side studies (--extras)                                                     #
# --------------------------------------------------------------------------- #
def run_extras(args, dev, stream, flush, M, P):
    out = {}
    out["mlqmc6"] = run_step6(args, dev, stream, flush, M, P)
    out["precision_form"] = run_precision_form(dev, stream, flush, M)
    out["time_to_eps_7level"] = run_time_to_eps(M)
    try:
        cfg = workload_config("mlqmc6")
        genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
        out["matern"] = run_matern(cfg, W.fixed_count_work(cfg["counts"], cfg["R"]), genvec, dev, stream, flush, M)
    except Exception as e:  # reported; the other results stand
        out["matern"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_step6(args, dev, stream, flush, M, P, steps=10, warmup=3):
    """The 6-level step in both forms, device-timed, with its roofline table."""
    res = {}
    for prec in ("fp64", "mixed_tf32"):
        cfg = workload_config("mlqmc6", precision=prec)
        genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
        ns = n_samples(W.fixed_count_work(cfg["counts"], cfg["R"]))
        st = Step(M, cfg, genvec, dev, args, ns)
        for _ in range(warmup):
            st(stream)
        st.ctx.check_device(stream)
        ms = float(np.mean(timed_steps(lambda: st(stream), steps, stream, flush)))
        prof, _ = st.profiled(stream, flush, steps)
        roof, table = roofline_report(st.ctx, prof, P, prec, steps)
        res[prec] = {"ms_per_step": ms, "samples_per_s": ns / (ms * 1e-3), "roofline": roof, "table": table}
        st.close()
    res["mixed_speedup"] = res["fp64"]["ms_per_step"] / res["mixed_tf32"]["ms_per_step"]
    return res


def run_matern(cfg, work, genvec, dev, stream, flush, M, steps=5, warmup=3):
    """The 6-level step with the Matern covariance (eq. matern, nu = 1) whose KL
    modes are Nystrom eigenpairs on 16 x 16 nodes (Sec. 5), in both forms."""
    import torch

    nu, m = 1.0, 16
    t0 = time.perf_counter()
    th, ps = M.nystrom_modes(nu, cfg["corr_len"], cfg["sigma"], m, cfg["s"])
    out = {"eigensolve_seconds": time.perf_counter() - t0}
    ns = n_samples(work)
    sums = torch.zeros(cfg["n_levels"] * cfg["R"] * 2, dtype=torch.float64, device=dev)
    for prec in ("fp64", "mixed_tf32"):
        c = dict(cfg)
        c["precision"] = prec
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=ns, covariance="matern", matern_nu=nu,
                                    nystrom_m=m, nystrom_theta=th, nystrom_psi=ps)

        def step():
            sums.zero_()
            ctx.sample_levels(work, sums, stream=stream)

        for _ in range(warmup):
            step()
        ctx.check_device(stream)
        ms = float(np.mean(timed_steps(step, steps, stream, flush)))
        out[prec] = {"ms_per_step": ms, "samples_per_s": ns / (ms * 1e-3)}
        ctx.close()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed_tf32"]["ms_per_step"]
    return out


def run_precision_form(dev, stream, flush, M):
    """One batch of 256 samples whose FMG ends on 1024x1024 (8 levels, s = 400,
    lambda = 0.1), every level refined to a relative residual of 1e-10: the
    mixed forms against the all-FP64 form, time per batch and the mixed
    results' deviation from the FP64 ones (field, solution, F per level)."""
    import torch

    cfg = dict(W.PRECISION_1024)
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    top = cfg["n_levels"] - 1
    work = [(top, 0, 16, 0, 16)]
    ns = n_samples(work)
    nl, R = cfg["n_levels"], cfg["R"]
    out, res = {}, {}
    for prec in ["mixed_tf32", "mixed_bf16x3", "fp64"]:
        c = dict(cfg)
        c["precision"] = prec
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=ns)
        sums = torch.zeros(nl * R * 2, dtype=torch.float64, device=dev)
        F = torch.zeros(ns * nl, dtype=torch.float64, device=dev)
        ctx.sample_levels(work, sums, F, stream=stream)
        ctx.check_device(stream)
        ctx.profile(True)
        times = []
        for _ in range(2):
            sums.zero_()
            times.append(timed_steps(lambda: ctx.sample_levels(work, sums, F, stream=stream), 1, stream, flush)[0])
        kl = {k: v for k, v in ctx.profile_read_levels().items() if k[0] == "kl_tc" and k[1] == top}
        ctx.profile(False)
        ctx.check_device(stream)
        y = ctx.normals(top, 3, 5, 4)
        kf = ctx.fields(top, y)
        u, _ = ctx.sample_solution(top, 3, 5)
        res[prec] = dict(ms=min(times), F=F.cpu().numpy().reshape(ns, nl), k=kf.cpu().numpy(), u=u[top].cpu().numpy())
        out[prec] = {"ms_per_batch": min(times), "samples_per_s": ns / (min(times) * 1e-3)}
        if kl:
            cell = next(iter(kl.values()))
            out[prec]["kl_1024"] = {"ms_per_launch": cell["ms"] / cell["n"],
                                    "tflops": cell["ftc"] / (cell["ms"] * 1e-3) / 1e12,
                                    "gbs": cell["bytes"] / (cell["ms"] * 1e-3) / 1e9}
        ctx.close()
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
    """Algorithm 1 on the 7-level adaptive problem (8x8..512x512, s = 200,
    lambda = 0.3, 16 shifts, mean-of-u QoI, every level refined to 1e-10):
    mixed against FP64, without recycling, batched rounds, plain MLMC, the
    rates and Proposition 1, and the multi-index variant."""
    from paper_1806_05619_gb300 import rates

    cfg = dict(W.ADAPTIVE_7LEVEL)
    cfg["log2_nmax"] = 12
    genvec, _ = M.cbc_genvec(cfg["s"], cfg["log2_nmax"])
    out = {}
    variants = [("mixed_tf32", "mixed_tf32", True, False, True), ("fp64", "fp64", True, False, True),
                ("mixed_tf32_no_reuse", "mixed_tf32", False, False, True),
                ("mixed_tf32_batched", "mixed_tf32", True, True, True),
                ("mixed_tf32_launch_by_launch", "mixed_tf32", True, False, False)]
    eps_list = cfg["eps"] + [3e-4, 1e-4]
    for name, prec, reuse, batched, graphs in variants:
        c = dict(cfg)
        c["precision"] = prec
        c["reuse"] = reuse
        ctx = M.Context.from_config(c, genvec=genvec, max_samples=1 << 17)
        ctx.set_graphs(graphs)
        rows = []
        for eps in eps_list:
            r = ctx.estimate(eps, batched=batched)
            rows.append({"eps": eps, "seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                         "L": r["L"], "rounds": r["rounds"], "N": r["N"][:r["L"] + 1], "run_status": r["run_status"]})
        out[name] = rows
        if name == "mixed_tf32":
            out["rates"] = rates.measure(ctx, n_points=256, lambda_level=2, gamma_levels=3)
        ctx.close()
    rt = out["rates"]
    prop = {"predicted": rt["prop1_ratio"], "from_counts": [], "measured_gpu_time": []}
    for a, b in zip(out["mixed_tf32"], out["mixed_tf32_no_reuse"]):
        L = a["L"]
        used = np.cumsum(np.array(a["N"][:L + 1], dtype=np.float64)[::-1])[::-1]
        prop["from_counts"].append({"eps": a["eps"], "ratio": rates.reuse_cost_ratio(used, rt["ms_per_sample"][:L + 1])})
        prop["measured_gpu_time"].append({"eps": a["eps"], "ratio": a["gpu_seconds"] / b["gpu_seconds"]})
    out["prop1"] = prop
    c = dict(cfg)
    c.update(precision="mixed_tf32", sampler="mc", R=1, reuse=False)
    ctx = M.Context.from_config(c, max_samples=1 << 17)
    rows = []
    for eps in eps_list:
        r = ctx.estimate_mlmc(eps)
        rows.append({"eps": eps, "seconds": r["wall_seconds"], "gpu_seconds": r["gpu_seconds"], "Q": r["Q"],
                     "L": r["L"], "rounds": r["rounds"], "N": r["N"][:r["L"] + 1], "run_status": r["run_status"]})
    ctx.close()
    out["mlmc_mixed_tf32"] = rows
    model = np.cumsum([(cfg["n0"] << t) ** 2 for t in range(cfg["n_levels"])])

    def work(row, R):
        return R * float(np.dot(row["N"], model[:len(row["N"])]))

    sp = []
    for m, q, g in zip(rows, out["mixed_tf32_no_reuse"], out["mixed_tf32"]):
        wm, wq, wg = work(m, 1), work(q, cfg["R"]), work(g, cfg["R"])
        sp.append({"eps": m["eps"], "S1": m["gpu_seconds"] / q["gpu_seconds"],
                   "S2": m["gpu_seconds"] / g["gpu_seconds"], "S3": q["gpu_seconds"] / g["gpu_seconds"],
                   "S1_work": wm / wq, "S2_work": wm / wg, "S3_work": wq / wg})
    out["speedups"] = sp
    out["mimc"] = run_mimc(M, cfg, genvec, model)
    return out


def run_mimc(M, cfg, genvec, model):
    """Multi-index variant (grid level x V-cycle count, the outlook of Sec. 7)
    on the 7-level problem in the fixed-cycle mixed form, mu0 in {1, 2, 3},
    against Algorithm 1 with mu0 = 3, in device time and in work."""
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
        rows.append({"eps": eps, "mimc_gpu_s": r["gpu_seconds"], "alg1_gpu_s": a["gpu_seconds"],
                     "gpu_time_ratio": a["gpu_seconds"] / r["gpu_seconds"], "work_ratio": w_alg1 / w_mimc,
                     "mimc_L": r["L"], "alg1_L": a["L"]})
    for x in ctxs:
        x.close()
    return rows


def run_kl_shape(args):
    """Only the tensor-core KL contraction (eq. truncatedKL): B samples on the
    n x n level with s modes through mlqmc_fields (TF32, FP32 accumulation,
    exp epilogue), device-timed per launch by the library's event brackets;
    algorithmic work 2 n^2 s B FLOP and 4 (n^2 B + n^2 K + B K) bytes."""
    import torch

    import paper_1806_05619_gb300 as M

    n, s, B = (int(x) for x in args.kl_shape.split(","))
    L = int(round(np.log2(n // 8)))
    cfg = W.scaled(W.PRECISION_1024, n_levels=L + 1, s=s, rtol=0.0)
    genvec, _ = M.cbc_genvec(s, 10)
    ctx = M.Context.from_config(cfg, genvec=genvec, max_samples=B)
    y = torch.from_numpy(W.random_normals(s, B, tag=77)).cuda()
    for _ in range(args.warmup):
        ctx.fields(L, y)
    torch.cuda.synchronize()
    ctx.profile(True)
    torch.cuda.profiler.start()
    for _ in range(args.steps):
        ctx.fields(L, y)
    torch.cuda.profiler.stop()
    cell = ctx.profile_read_levels()[("kl_tc", L)]
    ctx.profile(False)
    ctx.check_device()
    P = peaks()
    t = cell["ms"] * 1e-3 / cell["n"]
    out = {"kl_shape": {"cells": n * n, "modes": s, "samples": B}, "ms_per_launch": t * 1e3,
           "tflops": cell["ftc"] / cell["n"] / t / 1e12, "gbs": cell["bytes"] / cell["n"] / t / 1e9,
           "tf32_peak_sustained": P["tf32_sust"], "hbm_peak": P["hbm"]}
    out["tensor_frac"] = out["tflops"] / P["tf32_sust"]
    out["hbm_frac"] = out["gbs"] / P["hbm"]
    print(json.dumps(out), flush=True)
    ctx.close()


def run_tte_profile(args):
    """Algorithm 1 on the 9-level problem in the mixed form, one level per
    round, with a profiler range around the estimate only (context creation
    and the autotuner stay outside): one summary line."""
    import torch

    import paper_1806_05619_gb300 as M

    c = dict(workload_config("mlqmc9", precision="mixed_tf32"))
    c["log2_nmax"] = 14
    genvec, _ = M.cbc_genvec(c["s"], c["log2_nmax"])
    ctx = M.Context.from_config(c, genvec=genvec, max_samples=1 << 16)
    ctx.set_round_graphs("converged")
    torch.cuda.synchronize()
    n0 = ctx.launch_count()
    torch.cuda.profiler.start()
    r = ctx.estimate(args.tte_eps)
    torch.cuda.profiler.stop()
    print(json.dumps({"tte_profile": {"eps": args.tte_eps, "seconds": r["wall_seconds"], "rounds": r["rounds"],
                                      "L": r["L"], "N": r["N"][:r["L"] + 1], "launches": ctx.launch_count() - n0}}))
    ctx.close()


def main():
    args = parse()
    if args.tte_profile:
        run_tte_profile(args)
        return
    if args.kl_shape:
        run_kl_shape(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
