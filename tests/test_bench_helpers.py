"""Host-side helpers of bench.py: DRAM traffic and the instruction-issue
roofline of the dominant kernel, read from a recorded ncu capture that is only
valid for the kernel sources it was taken from (their hash)."""
import json

import bench


def _record(tmp_path, inst=3.0e9, bytes_=1.2e9, cells=16384 * 16384, sha=None):
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps({"pass1_tile_solve": {
        "source_sha1": sha or bench.source_sha1(), "warp_instructions_per_launch": inst,
        "bytes_per_launch": bytes_, "launch_cells": cells}}))
    return str(p)


def test_issue_roofline_from_a_recorded_capture(tmp_path):
    path = _record(tmp_path)
    r = bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100, path=path,
                             cells=16384 * 16384)
    assert r is not None and r["bound"] == "issue"
    assert abs(r["achieved"] - 3.0e9 / 5e-3) < 1e-6 * r["achieved"]
    assert abs(r["peak"] - 100 * 4 * 2000e6) < 1.0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_issue_roofline_unknown_or_stale(tmp_path):
    path = _record(tmp_path)
    assert bench.issue_roofline("pass1_tile_solve", 0.0, 2000.0, 100, path=path) is None
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 0.0, 100, path=path) is None
    assert bench.issue_roofline("no_such_kernel", 5.0, 2000.0, 100, path=path) is None
    stale = _record(tmp_path, sha="0" * 40)
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100, path=stale) is None
    assert bench.traffic_for("pass1_tile_solve", path=stale) is None
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100,
                                path=str(tmp_path / "none")) is None


def test_recorded_counts_scale_with_the_raster(tmp_path):
    path = _record(tmp_path)
    full = bench.traffic_for("pass1_tile_solve", 16384 * 16384, path=path)
    quarter = bench.traffic_for("pass1_tile_solve", 8192 * 8192, path=path)
    assert full and quarter and abs(4 * quarter - full) <= 4
    a = bench.issue_roofline("pass1_tile_solve", 1.0, 2000.0, 100, path=path,
                             cells=16384 * 16384)
    b = bench.issue_roofline("pass1_tile_solve", 1.0, 2000.0, 100, path=path, cells=8192 * 8192)
    assert abs(a["warp_instructions_per_launch"] - 4 * b["warp_instructions_per_launch"]) < 1.0
