"""Host logic of bench.py (no GPU): the kernel-source hash that decides whether
a committed ncu summary still describes the kernels, the reading of DRAM/L2
bytes from such a summary, the integer-issue roofline arithmetic, the HBM
peak's source, and the parsing of nvidia-smi clock samples."""
import os
import shutil
import types

import pytest

import bench

CSRC_FILES = ("decode_int8.cu", "decode_int8.cuh", "decode_persistent.cu", "decode_persistent.cuh", "maxh.cuh",
              "row_update.cuh", "common.cuh")


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1903_10107_gb300", "csrc")
    dst = tmp_path / "paper_1903_10107_gb300" / "csrc"
    dst.mkdir(parents=True)
    for fn in CSRC_FILES:
        shutil.copy(os.path.join(src, fn), dst / fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_kernel_sha_ignores_comments_and_layout_only(fake_root):
    sha = bench.kernel_sources_sha()
    f = fake_root / "paper_1903_10107_gb300" / "csrc" / "common.cuh"
    txt = f.read_text()
    f.write_text("// a new comment\n/* and a block\n comment */\n" + txt.replace(" = ", "  =\n    ", 3))
    assert bench.kernel_sources_sha() == sha
    f.write_text(txt.replace("0x7E7E7E7Eu", "0x7E7E7E7Fu", 1))
    assert bench.kernel_sources_sha() != sha


def test_profiled_bytes_only_for_the_current_kernels(fake_root):
    sha = bench.kernel_sources_sha()
    p = fake_root / "profiles" / "persistent_kernel_wl.md"
    p.write_text(f"# title\n\nkernel_sha: {sha}\ndram_bytes_per_frame_iteration: 1000.5\n"
                 "l2_bytes_per_frame_iteration: 2500\n")
    assert bench.profile_value("persistent_kernel", "wl", "dram_bytes_per_frame_iteration") == pytest.approx(1000.5)
    assert bench.profile_value("persistent_kernel", "wl", "l2_bytes_per_frame_iteration") == pytest.approx(2500.0)
    assert bench.profile_value("decode_kernel", "wl", "dram_bytes_per_frame_iteration") is None  # no summary
    p.write_text("kernel_sha: 0123456789abcdef\ndram_bytes_per_frame_iteration: 1000.5\n")
    assert bench.profile_value("persistent_kernel", "wl", "dram_bytes_per_frame_iteration") is None  # stale


def test_committed_profiles_parse():
    import glob
    paths = [p for p in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")) if "kernel_sha:" in open(p).read()]
    assert paths
    for path in paths:
        txt = open(path).read()
        assert "dram_bytes_per_frame_iteration:" in txt and "--clock-control none" in txt, path


def test_workload_config_is_the_same_for_both_arms():
    args = bench.parse_args([])
    w = bench.inputs.WORKLOADS[bench.DEFAULT_WORKLOAD]
    a = bench.workload_config(args, w, 16384, 1)
    assert a == bench.workload_config(bench.parse_args(["--impl", "reference"]), w, 16384, 1)
    assert a["protocol"].startswith("interactive") and a["f_start"] == 1.1 and a["max_iter"] == 200
    assert "no flush" in a["l2"]
    f = bench.workload_config(bench.parse_args(["--protocol", "fixed"]), w, 16384, 1)
    assert f["target_f"] == w.target_f and "f_start" not in f
    small = bench.workload_config(args, bench.inputs.WORKLOADS["n4096_r075_q02"], 64, 1)
    assert small["l2"].startswith("L2 flushed") and small["protocol"].startswith("single code")


def test_roofline_alu_arithmetic():
    r = bench.roofline_alu(it_sum=1000, edges=192000, seconds=0.01, clk={"sm_mhz": 2000.0}, sms=152)
    assert r["peak"] == pytest.approx(152 * 4 * 32 * 2000e6 * 4 / 1e12)
    assert r["achieved"] == pytest.approx(bench.ALU_OPS_PER_EDGE * 192000 * 1000 / 0.01 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # no clock sample: the maximum SM clock
    assert bench.roofline_alu(1, 1, 1.0, None)["peak"] == pytest.approx(152 * 4 * 32 * 2070e6 * 4 / 1e12)


def test_roofline_hbm_arithmetic(fake_root):
    (fake_root / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6000.0}')
    r = bench.roofline_hbm(3e9, 0.001, "persistent_kernel", None)
    assert r["achieved"] == pytest.approx(3000.0) and r["frac"] == pytest.approx(0.5)
    assert r["peak_kind"].startswith("measured") and r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_peak_source(fake_root):
    assert bench.peaks() == (6800.0, "fallback")
    (fake_root / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6691.8}')
    assert bench.peaks()[0] == 6691.8 and bench.peaks()[1].startswith("measured")


def test_clock_samples_median_and_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    s = bench.ClockSampler(0)
    s.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0)
    s.lines = ["2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    r = s.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]
