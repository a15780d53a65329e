"""Host logic of bench.py that the bench line's evidence rests on, on
synthetic inputs (no GPU): the roofline classification and fraction of one
(kernel kind, level) bucket, the choice of the dominant bucket, the DRAM
traffic record and its invalidation when the library sources change, the
clock summary from nvidia-smi samples, and the size of the final line."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _cell(ms, n=1, bytes_=0.0, f64=0.0, f32=0.0, ftc=0.0):
    return {"ms": ms, "n": n, "bytes": bytes_, "f64": f64, "f32": f32, "ftc": ftc}


def test_bucket_roofline_bound_and_fraction(bench):
    P = bench.peaks()
    hbm = P["hbm"]
    # bytes that take 0.5 ms at the HBM peak, measured 1 ms: half the roofline
    r = bench.bucket_roofline(_cell(1.0, bytes_=hbm * 1e9 * 0.5e-3, f32=1e6), P)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
    assert r["frac"] == pytest.approx(0.5, rel=1e-12)
    assert r["achieved"] == pytest.approx(hbm * 0.5, rel=1e-12)
    # FP64 work whose model time exceeds the bytes': FP64-bound, against the FP64 peak
    r = bench.bucket_roofline(_cell(1.0, bytes_=1e3, f64=P["fp64"] * 1e12 * 0.8e-3), P)
    assert r["bound"] == "alu" and r["peak"] == P["fp64"] and r["frac"] == pytest.approx(0.8, rel=1e-12)
    # FP32 work
    r = bench.bucket_roofline(_cell(1.0, bytes_=1e3, f32=P["fp32"] * 1e12 * 0.3e-3), P)
    assert r["bound"] == "alu" and r["peak"] == P["fp32"] and r["frac"] == pytest.approx(0.3, rel=1e-12)
    # tensor work against the sustained TF32 figure (bf16 x 1.1 / 2.25)
    r = bench.bucket_roofline(_cell(1.0, bytes_=1e3, ftc=P["tf32_sust"] * 1e12 * 0.25e-3), P)
    assert r["bound"] == "tensor" and r["frac"] == pytest.approx(0.25, rel=1e-12)
    assert P["tf32_sust"] == pytest.approx(P["bf16_sust"] * 1.1 / 2.25, rel=1e-12)
    assert bench.bucket_roofline(_cell(0.0, ftc=1e9), P) is None


class _Ctx:
    def __init__(self, smoothers):
        self._s = smoothers

    def smoother_info(self):
        return [(k, {}) for k in self._s]

    def n(self, t):
        return 8 << t


def test_roofline_report_takes_the_longest_level_bucket(bench, monkeypatch):
    P = bench.peaks()
    hbm = P["hbm"] * 1e9
    prof = {("smooth", 8): _cell(6.0, 12, bytes_=hbm * 3e-3),
            ("smooth", 2): _cell(1.0, 12, bytes_=hbm * 0.1e-3),
            ("transfer", 8): _cell(2.0, 4, bytes_=hbm * 1e-3),
            ("reduce", None): _cell(7.0, 2, bytes_=1e6)}  # no single level: never the dominant kernel
    monkeypatch.setattr(bench, "measured_traffic", lambda form, kernel, n: 0.95 if n == 2048 else None)
    ctx = _Ctx(["gs", "whole", "whole", "whole", "tma", "tma", "tma", "tma", "tma"])
    roof, table = bench.roofline_report(ctx, prof, P, "mixed_tf32", steps=2)
    assert roof["kernel"] == "kb_rbgs_tma on 2048x2048"
    assert roof["frac"] == pytest.approx(0.5, abs=1e-3)
    assert roof["alg_bytes_per_launch"] == pytest.approx(hbm * 3e-3 / 12, rel=1e-12)
    assert roof["share"] == pytest.approx(6.0 / 16.0, abs=1e-3)
    assert roof["traffic"] == round(0.95 * hbm * 3e-3 / 12)  # DRAM per algorithmic byte x the launch's bytes
    assert {r["kernel"] for r in table} >= {"kb_rbgs_tma", "kb_rbgs_whole", "kb_qoi(_part), k_sums"}


def test_traffic_record_and_its_invalidation(bench, tmp_path, monkeypatch):
    traffic = tmp_path / "dram_traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    assert bench.measured_traffic("mixed_tf32", "kb_rbgs_tma", 2048) is None  # no record
    files = ["paper_1806_05619_gb300/csrc/rbgs_tma.cu", "paper_1806_05619_gb300/csrc/fmg_device.cuh"]
    entry = {"dram_per_alg_byte": 0.93, "sources": files, "sources_sha256": bench.sources_digest(files)}
    rec = {"kernels": {"mixed_tf32|kb_rbgs_tma|2048": entry}}
    traffic.write_text(json.dumps(rec))
    assert bench.measured_traffic("mixed_tf32", "kb_rbgs_tma", 2048) == 0.93
    assert bench.measured_traffic("mixed_tf32", "kb_rbgs_tma", 1024) is None   # another level
    assert bench.measured_traffic("fp64", "kb_rbgs_tma", 2048) is None         # another form
    entry["sources_sha256"] = "0" * 64                                          # other kernel sources
    traffic.write_text(json.dumps(rec))
    assert bench.measured_traffic("mixed_tf32", "kb_rbgs_tma", 2048) is None
    assert bench.sources_digest(files) != bench.sources_digest(files[:1])


def test_clock_summary(bench):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 600, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle sample
            "1, 300, 2070, 80.0, 0x0, Active, Not Active, Not Active, Not Active"]        # another GPU
    c = bench.clocks_summary(rows, device_index=0)
    assert c["sm_max_mhz"] == 2070 and c["samples"] == 4
    assert c["sm_mhz"] == 2070            # median of the loaded samples (idle one excluded)
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.clocks_summary([], 0) is None
    assert bench.clocks_stop((None, None), "unused") is None


def test_final_line_is_compact(bench):
    args = bench.parse([])
    roof = {"bound": "hbm", "achieved": 4321.0, "peak": 6783.1, "unit": "GB/s", "frac": 0.637,
            "traffic": 1.234e10, "kernel": "kb_rbgs_tma on 2048x2048", "share": 0.41,
            "alg_bytes_per_launch": 1.7e10, "peak_src": "measured copy bandwidth (of measured)"}
    e2e = {"value": 512345.6, "unit": "samples/s", "h2d_bytes_per_step": 4186112, "d2h_bytes_per_step": 2304}
    clocks = {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 41}
    cpu = {"value": 12.3456, "unit": "samples/s", "cores": 16, "kind": "oracle", "single_core": 0.77,
           "sample": "N_l/16=[256, 128, 64, 32, 16, 8, 4, 2, 1] per shift x 16 shifts (8176 samples), one shift per "
                     "process, 30.1 s wall; oracle lattice 2^8 pts"}
    fp64 = {"value": 90000.0, "ms_per_step": 1453.2, "steps": 3, "speedup_mixed": 6.1}
    tte = {"eps": 1e-4, "mixed_tf32": {"seconds": 1.234, "L": 5, "rounds": 40}, "fp64": {"seconds": 7.89},
           "mixed_tf32_round_graphs": {"seconds": 1.345}, "mixed_tf32_batched": {"seconds": 1.111, "rounds": 33},
           "fp64_batched": {"seconds": 6.543}}
    line = bench.make_line(args, 1, 654321.5, 2000.0, 130816, ["gs", "whole", "whole", "whole", "tma", "tma", "tma",
                                                                "tma", "tma"], 12.3, 123, 10, roof, e2e, clocks, cpu,
                           fp64, tte)
    text = json.dumps(line)
    assert len(text) < 2048, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
                "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert key in line
    assert line["config"]["workload"].startswith("MG-MLQMC with reuse, 9 levels")
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"]
    for key in ("mixed_s", "fp64_s", "mixed_round_graphs_s", "mixed_batched_s", "mixed_batched_rounds", "fp64_batched_s"):
        assert line["time_to_eps"][key] is not None, key


def test_cpu_sample_keeps_the_level_mix(bench):
    import workloads as W

    cfg = bench.workload_config("mlqmc9")
    assert cfg["counts"] == [4096, 2048, 1024, 512, 256, 128, 64, 32, 16]
    assert bench.n_samples(W.fixed_count_work(cfg["counts"], cfg["R"])) == 130816
