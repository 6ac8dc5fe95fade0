"""Host logic of bench.py (no GPU): the kernel-source hash that decides whether
a committed ncu summary still describes the kernels, the reading of DRAM/L2
bytes from such a summary, the integer-issue roofline arithmetic, the HBM
peak's source, and the parsing of nvidia-smi clock samples."""
import os
import shutil
import types

import pytest
import torch

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
    p.write_text(f"# title\n\nkernel_sha: {sha}\ndram_bytes_per_frame: 1000.5\nl2_bytes_per_frame: 2500\n")
    assert bench.profiled_traffic("persistent_kernel", "wl", 4) == pytest.approx(4002.0)
    assert bench.profiled_traffic("persistent_kernel", "wl", 4, "l2_bytes_per_frame") == pytest.approx(10000.0)
    assert bench.profiled_traffic("decode_kernel", "wl", 4) is None  # no summary
    p.write_text("kernel_sha: 0123456789abcdef\ndram_bytes_per_frame: 1000.5\n")
    assert bench.profiled_traffic("persistent_kernel", "wl", 4) is None  # stale summary


def test_committed_profiles_parse():
    for kernel, wl in (("persistent_kernel", "n49152_mixed_q01_08"), ("decode_kernel", "n40960_r080_q03")):
        path = os.path.join(bench.ROOT, "profiles", f"{kernel}_{wl}.md")
        txt = open(path).read()
        assert "kernel_sha:" in txt and "dram_bytes_per_frame:" in txt and "l2_bytes_per_frame:" in txt
        assert "--clock-control none" in txt


def test_roofline_alu_arithmetic(monkeypatch):
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: types.SimpleNamespace(multi_processor_count=152))
    r = bench.roofline_alu(it_sum=1000, edges=192000, seconds=0.01, clk={"sm_mhz": 2000.0})
    assert r["peak"] == pytest.approx(152 * 4 * 32 * 2000e6 * 4 / 1e12)
    assert r["achieved"] == pytest.approx(bench.ALU_OPS_PER_EDGE * 192000 * 1000 / 0.01 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # no clock sample: the maximum SM clock
    assert bench.roofline_alu(1, 1, 1.0, None)["peak"] == pytest.approx(152 * 4 * 32 * 2070e6 * 4 / 1e12)


def test_peak_source(fake_root):
    assert bench.peaks() == (6800.0, "fallback")
    (fake_root / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6691.8}')
    assert bench.peaks() == (6691.8, "measured")


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
