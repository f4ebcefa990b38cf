"""Host-side accounting of bench.py (no GPU): the algorithmic bytes behind the
roofline line, and the ncu-summary reader that supplies its DRAM traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import bench  # noqa: E402


def test_sweep_bytes_of_the_benchmark_workload():
    # boxes3d 243^3 at s = 8: 14,212,390 cells without a surplus, 136,517 with an
    # FP32 record.  Per cell: u read, u written, b read (4 B each), eps_c 4 B and
    # a class byte (17 B); an FP32 surplus adds 28 x 4 B + a 4-byte scale slot.
    cbc = [14212390, 0, 0, 136517]
    n = 243
    expect = n ** 3 * 17 + 136517 * 116
    assert bench.sweep_bytes(3, n, cbc, True, 4) == expect == 259767391
    # the layout adds the vertex boundary ring and the segment bases
    assert bench.sweep_overhead_bytes(3, n, True, 4) == (244 ** 3 - n ** 3) * 12 + n * n * 8 * 12


def test_sweep_bytes_full_storage_and_2d():
    assert bench.sweep_bytes(3, 27, [0, 0, 0, 0], False, 8) == 27 ** 3 * (24 + 28 * 8)
    assert bench.sweep_bytes(2, 81, [6561, 0, 0, 0], True, 4) == 81 ** 2 * 17
    assert bench.sweep_bytes(2, 81, [6000, 300, 200, 61], True, 4) == 81 ** 2 * 17 + 300 * 10 + 200 * 16 + 61 * 28


def test_sweep_traffic_reads_the_committed_summary():
    assert bench.sweep_traffic("fourier3d") is None      # other workloads: no capture
    t = bench.sweep_traffic("boxes3d")
    if t is None:
        pytest.skip("the sweep source changed since the committed ncu summary was taken")
    # a positive byte count within 10% of the algorithmic bytes plus the layout
    # overhead (re-reads would show here)
    ref = bench.sweep_bytes(3, 243, [14212390, 0, 0, 136517], True, 4) + bench.sweep_overhead_bytes(3, 243, True, 4)
    assert abs(t - ref) <= 0.1 * ref


def test_profile_summaries_name_their_commands_on_committed_files():
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith((".md", ".txt"))]
    assert names
    for f in names:
        text = open(os.path.join(prof, f)).read()
        assert "ncu " in text and "--clock-control none" in text, f
        assert "_work" not in text, f            # the commands run committed files only
        assert "python bench.py" in text, f


def test_committed_sources_do_not_use_the_working_folder():
    for top in ("paper_2005_03606_gb300", "oracle", "tests", "include"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, top)):
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                    text = open(os.path.join(dirpath, f), errors="replace").read()
                    assert "_work/" not in text.replace('"_work/"', ""), os.path.join(dirpath, f)
    for f in ("bench.py", "__graft_entry__.py"):
        assert "_work" not in open(os.path.join(ROOT, f)).read(), f
