"""Host-side logic of the build: the unroll widths the kernels are compiled
for and the rule that picks one for a code (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_1903_10107_gb300 import build

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1903_10107_gb300", "csrc")


def test_unroll_widths_parse_ascending_and_cover_degree_64():
    ws = build.unroll_widths()
    assert ws == sorted(set(ws)) and ws[0] >= 1
    assert ws[-1] * 2 >= 64  # the code handle accepts rows of up to 64 edges


def test_generated_units_one_per_width(tmp_path, monkeypatch):
    monkeypatch.setattr(build, "GEN_DIR", str(tmp_path))
    paths = build._generated()
    assert [os.path.basename(p) for p in paths] == [f"maxh_{m}.cu" for m in build.unroll_widths()]
    for m, p in zip(build.unroll_widths(), paths):
        txt = open(p).read()
        assert f"decode_launch<{m}>" in txt and f"persist_launch<{m}>" in txt
    mtimes = [os.path.getmtime(p) for p in paths]
    build._generated()  # unchanged content is not rewritten
    assert [os.path.getmtime(p) for p in paths] == mtimes


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_pick_maxh_is_the_smallest_width_holding_half_the_row(tmp_path):
    src = tmp_path / "pick.cpp"
    src.write_text('#include <cstdio>\n#include "maxh.cuh"\n'
                   "int main() { for (int d = 1; d <= 70; ++d) std::printf(\"%d %d\\n\", d, ldpc_dec::pick_maxh(d)); }\n")
    exe = tmp_path / "pick"
    subprocess.run(["g++", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    ws = build.unroll_widths()
    for line in filter(None, out):
        d, m = map(int, line.split())
        need = (d + 1) // 2
        fits = [w for w in ws if w >= need]
        assert m == (fits[0] if fits else 0), (d, m)
