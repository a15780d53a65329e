"""Host logic of bench.py that the bench line's evidence rests on, on
synthetic inputs (no GPU): kernel names to timing kinds, the roofline
classification and fraction, the per-kind DRAM summary of an ncu launch list
and its invalidation when the library sources or smoothers change, and the
clock summary from nvidia-smi samples."""
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


def test_kernel_names_map_to_the_library_kinds(bench):
    k = bench.kernel_kind
    assert k("void <unnamed>::kb_rbgs_tma<32, 2, 1>(mlqmc_dev::FmgArgs, int, int)") == "smooth"
    assert k("void <unnamed>::kb_gs<double>(mlqmc_dev::FmgArgs, int, int, int)") == "smooth"
    assert k("kb_prolong_resid64") == "transfer"
    assert k("kb_resid_restrict<float>") == "transfer"
    assert k("kl_tc_kernel<256, 0>") == "kl_tc"
    assert k("kb_level0_fixed<float, 1, 8>") == "level0"
    assert k("kb_coarse_fixed<float, 8>") == "coarse"
    assert k("k_sums") == "reduce"
    assert k("void at::vectorized_elementwise_kernel<4, at::FillFunctor<float>>") is None  # the L2 flush


def test_roofline_bound_and_fraction(bench):
    hbm = bench.HBM_GBS
    # 1 GB in 0.5 ms of model time at the HBM peak, measured 1 ms: half the roofline
    ms = 1.0
    work = {"bytes": hbm * 1e9 * 0.5e-3, "f64": 0.0, "f32": 1e6, "ftc": 0.0}
    r = bench.kind_roofline(ms, work)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
    assert r["frac"] == pytest.approx(0.5, rel=1e-12)
    assert r["achieved"] == pytest.approx(hbm * 0.5, rel=1e-12)
    # FP64 work whose model time exceeds the bytes': FP64-bound, against the FP64 peak
    work = {"bytes": 1e3, "f64": bench.FP64_TFLOPS * 1e12 * 0.8e-3, "f32": 0.0, "ftc": 0.0}
    r = bench.kind_roofline(ms, work)
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_TFLOPS
    assert r["frac"] == pytest.approx(0.8, rel=1e-12)
    # tensor work
    work = {"bytes": 1e3, "f64": 0.0, "f32": 0.0, "ftc": bench.TF32_TFLOPS * 1e12 * 0.25e-3}
    r = bench.kind_roofline(ms, work)
    assert r["bound"] == "tensor" and r["frac"] == pytest.approx(0.25, rel=1e-12)
    assert bench.kind_roofline(0.0, work) is None


def test_roofline_report_takes_the_longest_kind(bench):
    prof = {"smooth": (6.0, 12), "transfer": (2.0, 4), "points": (0.1, 2)}
    hbm = bench.HBM_GBS * 1e9
    work = {"smooth": {"bytes": hbm * 3e-3, "f64": 0, "f32": 0, "ftc": 0},
            "transfer": {"bytes": hbm * 1e-3, "f64": 0, "f32": 0, "ftc": 0},
            "points": {"bytes": 1e6, "f64": 0, "f32": 0, "ftc": 0}}
    roof, by_kind = bench.roofline_report(prof, work, steps=2)
    assert roof["kernel_kind"] == "smooth"
    assert roof["frac"] == pytest.approx(0.5, rel=1e-12)
    assert roof["launches_per_step"] == 6 and roof["ms_per_step"] == 3.0
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(hbm * 3e-3 / 12, rel=1e-12)
    assert roof["share_of_step"] == pytest.approx(6.0 / 8.1, rel=1e-12)
    assert roof["traffic"] is None  # no form given: no capture to consult
    assert set(by_kind) == {"smooth", "transfer", "points"}


def _ncu_rows(rows):
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    out = ["==PROF== a line ncu prints before the table", head]
    for i, name, rd, wr, ns in rows:
        for metric, unit, v in (("dram__bytes_read.sum", "byte", rd), ("dram__bytes_write.sum", "byte", wr),
                                ("gpu__time_duration.sum", "ns", ns)):
            out.append(f'"{i}","1","python3","127.0.0.1","{name}","1","7","(256, 1, 1)","(608, 1, 1)","0",'
                       f'"10.3","Command line profiler metrics","{metric}","{unit}","{v:,}"')
    return "\n".join(out) + "\n"


def test_traffic_summary_and_its_invalidation(bench, tmp_path, monkeypatch):
    csv_path = tmp_path / "launches.csv"
    csv_path.write_text(_ncu_rows([
        (0, "void at::vectorized_elementwise_kernel<4, at::FillFunctor<float>>", 1000, 500_000_000, 70_000),
        (1, "void <unnamed>::kb_gs<double>(mlqmc_dev::FmgArgs, int, int, int)", 300_000_000, 200_000_000, 80_000),
        (2, "void <unnamed>::kb_gs<double>(mlqmc_dev::FmgArgs, int, int, int)", 350_000_000, 250_000_000, 90_000),
        (3, "void <unnamed>::kb_resid_restrict<double>(mlqmc_dev::FmgArgs, int, int)", 40_000_000, 10_000_000, 5_000),
    ]))
    traffic = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    rec = bench.summarize_traffic(str(csv_path), "fp64", ["gs", "whole"])
    sm = rec["kinds"]["smooth"]
    assert sm["launches"] == 2 and sm["dram_bytes"] == 1_100_000_000 and sm["ns"] == 170_000
    assert sm["dram_bytes_per_launch"] == 550_000_000
    assert rec["kinds"]["transfer"]["dram_bytes"] == 50_000_000
    assert "None" not in json.dumps(rec["kinds"])  # the flush kernel belongs to no kind
    assert bench.measured_traffic("fp64", "smooth", ["gs", "whole"]) == 550_000_000
    assert bench.measured_traffic("fp64", "smooth", ["gs", "tma"]) is None      # other smoothers
    assert bench.measured_traffic("mixed_tf32", "smooth", ["gs", "whole"]) is None  # no capture of that form
    data = json.loads(traffic.read_text())
    data["forms"]["fp64"]["sources_sha256"] = "0" * 64                           # other library sources
    traffic.write_text(json.dumps(data))
    assert bench.measured_traffic("fp64", "smooth", ["gs", "whole"]) is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary(bench, tmp_path):
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 600, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle sample
            "1, 300, 2070, 80.0, 0x0, Active, Not Active, Not Active, Not Active"]        # another GPU
    path.write_text("\n".join(rows) + "\n")
    c = bench.clocks_stop((_Proc(), open(tmp_path / "unused", "w")), str(path), device_index=0)
    assert c["sm_max_mhz"] == 2070 and c["samples"] == 4
    assert c["sm_mhz"] == 2070            # median of the loaded samples (idle one excluded)
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.clocks_stop((None, None), str(path)) is None
