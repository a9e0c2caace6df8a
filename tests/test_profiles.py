"""The committed profile summaries: every one names the kernel and workload
it covers, gives the full command that made it (committed files only, ncu
with --clock-control none), and bench.py takes a summary's DRAM traffic only
for the kernel its title names and only while the device sources are the
ones it was taken on."""
import re
from pathlib import Path

import pytest

import bench

ROOT = Path(__file__).resolve().parent.parent
PROFILES = sorted((ROOT / "profiles").glob("*.md"))


def test_there_are_profiles():
    names = {p.name for p in PROFILES}
    assert {"launches_fp32.md", "objective_fp32.md", "lloyd_fp32.md", "peaks_gb300.md"} <= names


@pytest.mark.parametrize("path", PROFILES, ids=lambda p: p.name)
def test_summary_has_title_and_command(path):
    txt = path.read_text()
    assert re.match(r"# \S+", txt), "title line"
    cmds = [l.strip() for l in txt.splitlines() if l.startswith("    ")]
    assert cmds, "the command that made the summary"
    body = " ".join(cmds)
    assert "bench.py" in body or "paper_2311_04517_gb300.peaks" in body
    assert "_work" not in txt
    if "ncu " in body:
        assert "--clock-control none" in body
    assert len(txt) < 8192, "a short summary, not raw output"


def test_traffic_only_for_the_named_kernel_and_sources():
    for p in (ROOT / "profiles").glob("objective_*.md"):
        txt = p.read_text()
        kernel = re.match(r"#\s+(\w+)", txt).group(1)
        h = bench.kernel_source_hash(kernel)
        workload = p.stem.split("_")[1]
        rec = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        src = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
        assert rec and src, p.name
        got = bench.profiled_traffic("objective", workload, kernel)
        if src.group(1) == h:
            assert got == float(rec.group(1)), p.name
        else:
            assert got is None, p.name
        assert bench.profiled_traffic("objective", workload, "no_such_kernel") is None
