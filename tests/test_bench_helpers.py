"""Host-side helpers of bench.py: the instruction-issue roofline of the
dominant kernel, read from the recorded ncu capture of the same sources."""
import json

import bench


def test_issue_roofline_from_the_recorded_capture():
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    inst = rec["pass1_tile_solve"]["warp_instructions_per_launch"]
    r = bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100)
    assert r is not None and r["bound"] == "issue"
    assert abs(r["achieved"] - inst / 5e-3) < 1e-6 * r["achieved"]
    assert abs(r["peak"] - 100 * 4 * 2000e6) < 1.0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_issue_roofline_unknown_or_stale(tmp_path):
    assert bench.issue_roofline("pass1_tile_solve", 0.0, 2000.0, 100) is None
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 0.0, 100) is None
    assert bench.issue_roofline("no_such_kernel", 5.0, 2000.0, 100) is None
    stale = tmp_path / "traffic.json"
    stale.write_text(json.dumps({"pass1_tile_solve": {"source_sha1": "0" * 40,
                                                      "warp_instructions_per_launch": 1.0}}))
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100, path=str(stale)) is None
    assert bench.issue_roofline("pass1_tile_solve", 5.0, 2000.0, 100, path=str(tmp_path / "none")) is None


def test_recorded_counts_scale_with_the_raster():
    full = bench.traffic_for("pass1_tile_solve", 16384 * 16384)
    quarter = bench.traffic_for("pass1_tile_solve", 8192 * 8192)
    assert full and quarter and abs(4 * quarter - full) <= 4
    a = bench.issue_roofline("pass1_tile_solve", 1.0, 2000.0, 100, cells=16384 * 16384)
    b = bench.issue_roofline("pass1_tile_solve", 1.0, 2000.0, 100, cells=8192 * 8192)
    assert abs(a["warp_instructions_per_launch"] - 4 * b["warp_instructions_per_launch"]) < 1.0
