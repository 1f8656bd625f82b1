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


# ---------------------------------------------------------------------------
# the ncu CSV -> traffic record step, and the parity helpers (oracle-backed)
# ---------------------------------------------------------------------------
def _ncu_csv(path, launches):
    """An ncu --csv log: a preamble, the header, one row per (launch, metric)."""
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"')
    rows = ["==PROF== Connected to process 1", head]
    for i, (name, rd, wr, inst) in enumerate(launches):
        for metric, unit, v in (("dram__bytes_read.sum", "byte", rd),
                                ("dram__bytes_write.sum", "byte", wr),
                                ("smsp__inst_executed.sum", "inst", inst)):
            rows.append(f'"{i}","1","python3","h","{name}(TileArgs)","1","7","(128, 1, 1)",'
                        f'"(912, 1, 1)","0","10.3","m","{metric}","{unit}","{v:,}"')
    path.write_text("\n".join(rows) + "\n")


def test_record_traffic_sums_one_call_per_phase(tmp_path):
    forest = ["void k_forest_init<unsigned long long>", "void k_forest_indeg<unsigned long long>",
              "void k_forest_leaves<unsigned long long>", "void k_forest_walk<unsigned long long>",
              "void k_forest_final<unsigned long long>"]
    call = ([("void k_walk<0, 1, 1>", 100, 400, 800)] + [(k, 10, 1, 3) for k in forest]
            + [("void k_addin<1>", 300, 100, 200)])
    csv = tmp_path / "t.csv"
    _ncu_csv(csv, call + call)  # two calls: only the first counts
    out = tmp_path / "traffic.json"
    rec = bench.record_traffic(str(csv), 1000, "test raster", out_path=str(out))
    assert rec["pass1_tile_solve"]["bytes_per_launch"] == 500
    assert rec["pass1_tile_solve"]["warp_instructions_per_launch"] == 800
    assert rec["perimeter_graph_resolve"]["launches"] == 5
    assert rec["perimeter_graph_resolve"]["bytes_per_launch"] == 55
    assert rec["pass2_tile_finalize"]["bytes_per_launch"] == 400
    assert "f32_pass1_tile_solve" not in rec
    assert all(r["source_sha1"] == bench.source_sha1() and r["launch_cells"] == 1000
               for r in rec.values())
    assert json.loads(out.read_text()) == rec
    assert bench.traffic_for("pass1_tile_solve", 4000, path=str(out)) == 2000


def _acyclic(rows, cols, seed):
    import synth

    return synth.acyclic_random_codes(rows, cols, seed)


def test_parity_helpers_pass_exact_counts_and_catch_a_planted_error():
    import numpy as np

    import oracle

    codes = _acyclic(60, 70, 5)
    good = oracle.counts(codes).values
    r32 = bench.parity_counts_u32(codes, good.astype(np.uint32))
    assert r32["residual_mismatches"] == 0 and r32["vs_oracle"].endswith("exact")
    r64 = bench.parity_counts_u64(codes, good.copy())
    assert r64["residual_mismatches"] == 0 and not r64["vs_oracle"].endswith("MISMATCH")
    bad = good.copy()
    i = int(np.argmax(good))
    bad.flat[i] += 1
    r = bench.parity_counts_u64(codes, bad)
    assert r["residual_mismatches"] > 0 and r["vs_oracle"].endswith("MISMATCH")
    assert r["first_mismatch"] <= i


def test_f32_sampled_parity_passes_the_oracle_and_catches_an_error():
    import numpy as np
    import torch

    import oracle

    codes = _acyclic(50, 64, 6)
    w = np.random.default_rng(7).random(codes.shape, dtype=np.float32)
    ref = oracle.weighted(codes, w).values.astype(np.float32)
    ok = bench.parity_f32_sampled(codes, torch.from_numpy(w), torch.from_numpy(ref.copy()))
    assert ok["vs_oracle"].startswith("within 2e-5") and ok["max_rel_err"] < 1e-6
    worse = ref * np.float32(1.001)
    bad = bench.parity_f32_sampled(codes, torch.from_numpy(w), torch.from_numpy(worse))
    assert bad["vs_oracle"] == "MISMATCH"
