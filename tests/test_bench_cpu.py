"""Host logic of the benchmark: the reference arm's JSON line (the FP64 oracle timed on a bounded
sample of the benchmark workload), the split of timed steps into persistent launches, and the
recorded DRAM traffic being tied to the kernel sources it was measured on."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_chunks():
    assert bench.launch_chunks(20, 8) == [8, 8, 4]
    assert bench.launch_chunks(8, 8) == [8]
    assert bench.launch_chunks(3, 1) == [1, 1, 1]
    assert bench.launch_chunks(0, 8) == []


def test_recorded_traffic_matches_the_sources():
    """The DRAM bytes in the benchmark line belong to the kernel sources they were captured on:
    reported for those sources and the captured launch size, null for any other launch size."""
    spl = bench.STEP_TRAFFIC["steps_per_launch"]
    assert bench.step_traffic(spl) == bench.STEP_TRAFFIC["bytes_per_launch"]
    assert bench.step_traffic(spl + 1) is None
    # below the algorithmic bytes of a launch (14 B x 4M beams x 6 stages per step): the state
    # stays in the L2
    assert bench.STEP_TRAFFIC["bytes_per_launch"] < 14 * 4_000_000 * 6 * spl


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "beam-updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "bulb2f_1000E_2000u_mixed_dp45"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "beam-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_kernel_code_hash_ignores_comments_only(tmp_path):
    """The key of the recorded counters changes with the kernel code, not with its comments."""
    import shutil
    csrc = tmp_path / "paper_1912_10596_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_1912_10596_gb300", "csrc", f), csrc / f)
    saved = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        h0 = bench.kernel_code_hash()
        k = csrc / "kernels_2f.cu"
        k.write_text(k.read_text() + "\n// a comment\n/* and a block\n   comment */\n")
        assert bench.kernel_code_hash() == h0
        k.write_text(k.read_text() + "\nstatic int xflat_unused_symbol = 0;\n")
        assert bench.kernel_code_hash() != h0
    finally:
        bench.ROOT = saved


def test_issue_roofline_uses_the_recorded_instruction_count():
    """The issue-rate figure beside the HBM fraction: the recorded warp instructions per step over
    the step time, against 4 warp instructions per clock per SM; none without a clock reading."""
    r = bench.issue_roofline(0.25, 2000.0, 152)
    assert r is not None
    n = bench.STEP_INSTRUCTIONS["warp_inst_per_step"]
    assert abs(r["frac"] - n / 0.25e-3 / (4 * 152 * 2000e6)) < 1e-12
    assert bench.issue_roofline(0.25, None, 152) is None
    assert bench.STEP_INSTRUCTIONS["code_sha256"] == bench.kernel_code_hash()
