"""Benchmark: D8 flow accumulation on one GB300 (or N replicas under torchrun).

Workload (one step = the whole hot path over one raster: pass 1, the
perimeter-graph resolve and pass 2): a 16384 x 16384 raster (2.7e8 cells) of
uint8 D8 codes from the seeded spectral-DEM generator (1/f^2 spectrum,
priority-flood eps fill, 1% NoData disk; seed 201), unit weights, uint32
counts, with the tile shape picked by the library's autotuner (fa_autotune,
run before the timed region).  Inputs are resident in HBM; they (268 MB codes
+ 1.07 GB output) exceed the 129 MB L2, so no explicit flush runs between
steps.

Printed JSON line: cells/s over all ranks (max-over-ranks time), the roofline
of the dominant kernel (algorithmic bytes / live CUDA-event duration), the
float32 weighted form, an end-to-end number through the public API with host
buffers, the oracle timed on host cores, and SM clocks sampled during the
timed region.  Two more forms are timed on the same GPU against the plain
kernel (their per-cell time over the plain kernel's):
  batched: 64 spectral-DEM rasters, rows U{257..4096} x cols U{311..6000}
    (seeds 301..364), 8 float32 fields each (4 uniform [0,1), 4 lognormal
    sigma=1), one CUDA-graph replay of fa_accumulate_batched with the tile
    shape fa_autotune_batched picks, against the same 512 (raster, field)
    pairs run one fa_accumulate call each with that shape;
  adjoint: an 8192 x 8192 DEM raster (seed 401), dL/dA nonzero at 256 gauge
    cells, fa_accumulate_adjoint against the float32 forward on that raster.

--impl reference: times the CPU oracle (test infrastructure, a deliberately
slow reference) on the same workload and metric on host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

ROWS = COLS = 16384
SEED, WSEED = 201, 202
TILE = (64, 64)
BYTES_PER_CELL_COUNTS = 5  # 1 B code read + 4 B uint32 written (algorithmic minimum)
BYTES_PER_CELL_F32 = 9     # + 4 B float32 weight read
BYTES_PER_CELL_ABSORB = 13  # + 4 B float32 factor read
ASEED = 205                 # absorption factors, U[0.9, 1)
ABS_TILE = (32, 64)         # the absorption default tile
WORKLOAD = "d8_dem_16384x16384"
BATCH_N, BATCH_FIELDS, BATCH_SEED, BATCH_SHAPE_SEED = 64, 8, 301, 300
ADJ_N, ADJ_SEED, ADJ_GAUGES = 8192, 401, 256
D8_N, D8_SEED = 8192, 201
# the scale raster: 6250^2 coarse spectral DEM x16 = 100000^2 (1e10 cells)
SCALE_COARSE, SCALE_F, SCALE_SEED, SCALE_NSEED, SCALE_WSEED = 6250, 16, 501, 502, 503
TUNE_ROWS = 16384        # the autotuner times candidate tiles on this many rows
CPU_SAMPLE_ROWS = 2048   # the oracle's bounded sample of the scale raster


def pass_bytes(cells: int):
    """Algorithmic bytes per launch of each phase (counts): pass 1 reads the
    codes and writes A_loc into the output, the step's whole minimum (5
    B/cell); the perimeter resolve and pass 2 move O(perimeter) and overhead
    bytes, not counted."""
    return {0: cells * BYTES_PER_CELL_COUNTS, 1: 0, 2: 0}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
def dist_setup():
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest of every rank's x (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, ms_max: float, ws: int) -> float:
    """Whole-job units/s: every rank processed units_per_rank in at most ms_max."""
    return ws * units_per_rank / (ms_max / 1e3)


def traffic_for(kernel: str, cells: int = ROWS * COLS, path=None):
    """dram bytes per launch recorded from an ncu capture of this exact kernel
    source (profiles/traffic.json), scaled from the launch it describes to
    `cells` (traffic grows with the number of tiles); None when absent or
    stale."""
    try:
        with open(path or os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except Exception:
        return None
    if not rec:
        return None
    if rec.get("source_sha1") != source_sha1() or "bytes_per_launch" not in rec:
        return None
    return int(round(rec["bytes_per_launch"] * cells / rec.get("launch_cells", cells)))


# forward kernels by phase, as ncu names them ("void fa::k_walk<0, 1, 1>(fa::TileArgs, ...)")
TRAFFIC_PHASES = [
    ("pass1_tile_solve", r"k_walk<0, 1,"),
    ("perimeter_graph_resolve", r"k_forest_\w+<unsigned long long>"),
    ("pass2_tile_finalize", r"k_addin<"),
    ("f32_pass1_tile_solve", r"k_walk<1, 1,"),
    ("f32_perimeter_graph_resolve", r"k_forest_\w+<unsigned __int128>"),
    ("f32_pass2_tile_solve", r"k_walk<1, 2,"),
]


def record_traffic(csv_path: str, cells: int, desc: str, out_path=None) -> dict:
    """profiles/traffic.json from an ncu --csv capture with the metrics
    dram__bytes_read.sum, dram__bytes_write.sum and smsp__inst_executed.sum:
    per phase, the bytes and warp instructions of one call (the first
    captured launches of the phase's kernels), with the hash of the kernel
    sources they belong to."""
    import csv

    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    launches = {}
    for r in csv.DictReader(lines):
        d = launches.setdefault(int(r["ID"]), {"name": r["Kernel Name"]})
        d[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    ids = sorted(launches)
    out = {}
    for phase, key in TRAFFIC_PHASES:
        hit = [i for i in ids if re.search(key, launches[i]["name"])]
        if not hit:
            continue
        # one call: the resolve is five launches, a tile pass one
        first = hit[:5 if "resolve" in phase else 1]
        rd = sum(launches[i].get("dram__bytes_read.sum", 0.0) for i in first)
        wr = sum(launches[i].get("dram__bytes_write.sum", 0.0) for i in first)
        inst = sum(launches[i].get("smsp__inst_executed.sum", 0.0) for i in first)
        out[phase] = {"kernel": "; ".join(sorted({launches[i]["name"].split("(")[0] for i in first})),
                      "launches": len(first), "bytes_per_launch": int(rd + wr),
                      "dram_read": rd, "dram_write": wr,
                      "warp_instructions_per_launch": int(inst), "launch_cells": int(cells),
                      "measured_on": desc, "source_sha1": source_sha1()}
    with open(out_path or os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


def issue_roofline(kernel: str, ms: float, sm_mhz: float, sms: int, path=None,
                   cells: int = ROWS * COLS):
    """The kernel's achieved instruction issue rate against the GPU's ceiling:
    warp instructions per launch (from the same ncu capture as its traffic,
    scaled to the launch, valid only for the hashed kernel sources) over the
    live launch duration, against 4 warp instructions per clock per SM (one
    per scheduler) at the sampled SM clock.  None when unknown or stale."""
    try:
        with open(path or os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        if not rec or rec.get("source_sha1") != source_sha1() or not (ms > 0 and sm_mhz > 0 and sms > 0):
            return None
        inst = float(rec["warp_instructions_per_launch"]) * cells / rec.get("launch_cells", cells)
    except Exception:
        return None
    achieved = inst / (ms / 1e3)
    peak = sms * 4 * sm_mhz * 1e6
    return {"bound": "issue", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_launch": inst}


def source_sha1() -> str:
    """Hash of the sources that define the forward kernels (pass 1, the
    perimeter-graph resolve, pass 2)."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1608_04431_gb300", "csrc")
    for f in ("fa_common.cuh", "fa_forward.cu", "fa_internal.h"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def cpu_oracle_time(codes, sample_rows=None):
    import oracle

    sub = codes if sample_rows is None else codes[:sample_rows]
    oracle.build()
    t0 = time.perf_counter()
    res = oracle.counts(sub)
    dt = time.perf_counter() - t0
    return sub.size / dt, dt, res, sub.shape


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle (Algorithm 1 over a whole raster,
    one host thread) on bounded samples of the headline workload, printed as
    the contract's JSON line.  Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    steps = max(1, min(args.steps, 3))
    if args.workload == "scale":
        n = args.scale_coarse
        R = C = n * SCALE_F
        rows = min(R, CPU_SAMPLE_ROWS)
        codes = scale_sample_codes(args, rows)  # generated on the host, before any timing
        workload = f"d8_scale_{R}x{C}"
        sample = f"rows 0..{rows - 1} of the {R}x{C} scale raster as a raster of their own"
    else:
        import synth

        R, C = ROWS, COLS
        rows = ROWS // 4  # each step: a 4096-row band (~6.7e7 cells, a few seconds on one core)
        codes = synth.dem_codes(ROWS, COLS, SEED)[:rows]
        workload = f"d8_dem_{ROWS}x{COLS}"
        sample = f"first {rows} rows of the {ROWS}x{COLS} raster per step"
    codes = np.ascontiguousarray(codes)
    vals = []
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_time(codes)
    t_all = 0.0
    for _ in range(steps):
        v, dt, _, shape = cpu_oracle_time(codes)
        vals.append(v)
        t_all += dt
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": "cells/s (D8 flow accumulation, uint32 counts)",
        "value": value, "unit": "cells/s", "n_gpus": args.gpus, "steps": steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_all / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "uint64", "data": "synthetic",
        "config": {"workload": workload, "rows": R, "cols": C,
                   "reference": "CPU oracle (Kahn queue over the whole raster, Algorithm 1), 1 thread"},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time(fn, stream, n):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def leg_batched(fa, dev, stream, opts, warmup, reps):
    """64 rasters x 8 fields: one graph replay against the per-pair loop."""
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import synth

    shapes = synth.batch_shapes(BATCH_N, BATCH_SHAPE_SEED)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        codes = list(ex.map(lambda i: synth.dem_codes(*shapes[i], BATCH_SEED + i), range(BATCH_N)))
    items = []
    for i, c in enumerate(codes):
        g = torch.Generator(device=dev)
        g.manual_seed(BATCH_SEED * 1000 + i)
        ws = []
        for k in range(BATCH_FIELDS):
            t = torch.empty(c.shape, dtype=torch.float32, device=dev)
            if k < BATCH_FIELDS // 2:
                t.uniform_(0.0, 1.0, generator=g)
            else:
                t.log_normal_(0.0, 1.0, generator=g)
            ws.append(t)
        items.append({"codes": torch.from_numpy(c).to(dev), "weights": ws})
    cells = int(sum(c.size for c in codes))
    pairs = cells * BATCH_FIELDS
    plan = fa.BatchPlan(items, BATCH_FIELDS, tile="auto", stream=stream)
    opts = fa.options(plan.tile)
    for _ in range(warmup):
        plan.run(stream)
    ms_b = _time(lambda: plan.run(stream), stream, reps)
    st = plan.status_read(stream)[0]

    # the same pairs, one fa_accumulate call each
    rmax = max(r for r, _ in shapes)
    cmax = max(c for _, c in shapes)
    work = torch.empty(fa.fa_workspace_size(rmax, cmax, opts), dtype=torch.uint8, device=dev)
    outs = [[torch.empty(it["codes"].shape, dtype=torch.float32, device=dev)
             for _ in range(BATCH_FIELDS)] for it in items]

    def loop():
        for it, oo in zip(items, outs):
            for k in range(BATCH_FIELDS):
                e = fa.fa_accumulate(it["codes"], it["weights"][k], None, oo[k], fa.FA_OUT_F32,
                                     work, opts, None, stream)
                if e != fa.FA_OK:
                    raise fa.FlowAccError(e, "fa_accumulate (batch loop)")

    loop()
    ms_l = _time(loop, stream, max(2, reps // 2))
    worst = 0.0
    for ob, ol in zip(plan.outs, outs):
        for k in range(BATCH_FIELDS):
            a, b = ob[k].double(), ol[k].double()
            worst = max(worst, float(((a - b).abs() / b.abs().clamp_min(1e-30)).max()))
    plan.close()
    return {"rasters": BATCH_N, "fields": BATCH_FIELDS, "cells": cells, "cell_fields": pairs,
            "ms_graph_replay": ms_b, "cell_fields_per_s": pairs / (ms_b / 1e3),
            "ns_per_cell_field": ms_b * 1e6 / pairs,
            "ms_plain_loop": ms_l, "plain_loop_cell_fields_per_s": pairs / (ms_l / 1e3),
            "time_vs_plain_loop": ms_b / ms_l,
            # algorithmic bytes: 1 B code per cell, 4 B weight + 4 B output per pair
            "hbm_frac_step": (cells + 8 * pairs) / (ms_b / 1e3) / 1e9,  # divided by the peak below
            "tile": list(plan.tile), "status": int(st), "max_rel_diff_vs_plain": worst}


def leg_d8(fa, dev, stream, warmup, reps, peak):
    """D8 codes from the 8192^2 spectral DEM with its 1% NoData disk (the step
    before accumulation): fa_d8_codes time and HBM fraction at its algorithmic
    6 B/cell (4 B elevation + 1 B NoData read, 1 B code written).  Returns the
    record and (elevations, NoData, codes) for the CPU-baseline leg's check."""
    import torch

    import synth

    z = synth.spectral_dem(D8_N, D8_N, D8_SEED)
    nd = synth.nodata_disk(D8_N, D8_N, D8_SEED + 7919).astype(np.uint8)
    zt, ndt = torch.from_numpy(z).to(dev), torch.from_numpy(nd).to(dev)
    out = torch.empty(z.shape, dtype=torch.uint8, device=dev)

    def step():
        e = fa.fa_d8_codes(zt, ndt, out, stream)
        if e != fa.FA_OK:
            raise fa.FlowAccError(e, "fa_d8_codes")

    for _ in range(warmup):
        step()
    ms = _time(step, stream, reps)
    cells = z.size
    gbs = 6 * cells / (ms / 1e3) / 1e9
    rec = {"rows": D8_N, "cols": D8_N, "cells": cells, "ms": ms, "cells_per_s": cells / (ms / 1e3),
           "bytes_per_cell": 6, "achieved_gbs": gbs, "hbm_frac": gbs / peak}
    return rec, (z, nd, out.cpu().numpy())


def leg_adjoint(fa, dev, stream, opts, warmup, reps):
    """8192^2 DEM: fa_accumulate_adjoint (dL/dA nonzero at 256 gauges) against
    the float32 forward on the same raster; checked by <A(w), g> = <w, grad_w>."""
    import torch

    import synth

    codes = synth.dem_codes(ADJ_N, ADJ_N, ADJ_SEED)
    cells = codes.size
    cd = torch.from_numpy(codes).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(ADJ_SEED + 1)
    w = torch.empty(codes.shape, dtype=torch.float32, device=dev).uniform_(0.0, 2.0, generator=g)
    work = torch.empty(fa.fa_workspace_size(ADJ_N, ADJ_N, opts), dtype=torch.uint8, device=dev)
    A = torch.empty(codes.shape, dtype=torch.float32, device=dev)
    cnt = fa.accumulate(cd).view(torch.int32).cpu().numpy().view(np.uint32)
    gidx = synth.gauges(codes != 0, cnt, ADJ_GAUGES, ADJ_SEED + 2)
    gout = torch.zeros(cells, dtype=torch.float32, device=dev)
    gout[torch.from_numpy(gidx).to(dev)] = torch.from_numpy(
        synth.rng(ADJ_SEED + 3).standard_normal(gidx.size).astype(np.float32)).to(dev)
    gout = gout.view(codes.shape)
    gw = torch.empty_like(gout)

    def fwd():
        e = fa.fa_accumulate(cd, w, None, A, fa.FA_OUT_F32, work, opts, None, stream)
        if e != fa.FA_OK:
            raise fa.FlowAccError(e, "fa_accumulate (adjoint leg)")

    def adj():
        e = fa.fa_accumulate_adjoint(cd, None, gout, gw, work, opts, None, stream)
        if e != fa.FA_OK:
            raise fa.FlowAccError(e, "fa_accumulate_adjoint")

    for _ in range(warmup):
        fwd()
        adj()
    ms_f = _time(fwd, stream, reps)
    ms_a = _time(adj, stream, reps)
    st = fa.fa_status_read(None, work, stream)[0]
    lhs = float((A.double() * gout.double()).sum())
    rhs = float((w.double() * gw.double()).sum())
    return {"rows": ADJ_N, "cols": ADJ_N, "cells": cells, "gauges": int(gidx.size),
            "ms_adjoint": ms_a, "cells_per_s": cells / (ms_a / 1e3),
            "ms_forward_f32_same_raster": ms_f, "time_vs_forward_f32": ms_a / ms_f,
            # algorithmic bytes: 1 B code + 4 B dL/dA (dense) + 4 B dL/dw per cell
            "hbm_frac_step": 9 * cells / (ms_a / 1e3) / 1e9,  # divided by the peak below
            "status": int(st), "dot_identity_rel_err": abs(lhs - rhs) / max(abs(lhs), 1e-30)}


def leg_absorb(fa, dev, stream, codes_d, ms_f32, cells, warmup, reps, peak):
    """Accumulation with absorption on the bench raster: weights U[0, 1)
    and factors U[0.9, 1) drawn on the device with seeded generators; time
    per step, phases, and the HBM fraction at 13 B/cell (1 B code, 4 B weight,
    4 B factor read, 4 B float32 written)."""
    import torch

    g = torch.Generator(device=dev)
    g.manual_seed(WSEED)
    w = torch.rand(codes_d.shape, generator=g, device=dev, dtype=torch.float32)
    g.manual_seed(ASEED)
    a = torch.rand(codes_d.shape, generator=g, device=dev, dtype=torch.float32) * 0.1 + 0.9
    a.clamp_(max=1.0)
    out = torch.empty(codes_d.shape, dtype=torch.float32, device=dev)
    opts = fa.options(ABS_TILE)
    work = torch.empty(fa.fa_absorb_workspace_size(*codes_d.shape, opts), dtype=torch.uint8,
                       device=dev)

    def step():
        s = fa.fa_accumulate_absorb(codes_d, w, a, None, out, work, opts, None, stream)
        if s != fa.FA_OK:
            raise fa.FlowAccError(s, "fa_accumulate_absorb")

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    st = fa.fa_status_read(None, work, stream)
    ms = _time(step, stream, reps)
    fa.fa_timing_enable(True)
    ph = []
    for _ in range(3):
        step()
        ph.append(fa.fa_timing_read())
    fa.fa_timing_enable(False)
    ph = np.mean(np.array(ph), axis=0).tolist()
    gbs = cells * BYTES_PER_CELL_ABSORB / (ms / 1e3) / 1e9
    rec = {"ms": ms, "cells_per_s": cells / (ms / 1e3), "tile": list(ABS_TILE),
           "bytes_per_cell": BYTES_PER_CELL_ABSORB, "hbm_frac_step": gbs / peak,
           "phases_ms": dict(zip(["pass1_tile_solve", "perimeter_graph_resolve",
                                  "pass2_tile_resolve"], ph)),
           "time_vs_plain_f32": ms / ms_f32, "status": int(st[0])}
    data = (w.cpu().numpy(), a.cpu().numpy(), out.cpu().numpy())  # for the oracle check
    del w, a, out, work
    return rec, data


def host_available_bytes() -> int:
    """MemAvailable of the host (Linux), 0 if unknown."""
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


class HostPinned:
    """A page-locked host array of exactly the requested size (cudaHostAlloc
    through the CUDA runtime library), so that copies to and from it run at
    the link's rate.  The caching host allocator behind pin_memory() rounds a
    request up to a power of two (80 GB would take 128 GB of a host with 200).
    close() frees it."""

    _rt = None

    @classmethod
    def _runtime(cls):
        if cls._rt is None:
            import ctypes
            import glob

            libs = sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so.*")) or ["libcudart.so"]
            cls._rt = ctypes.CDLL(libs[-1])
        return cls._rt

    def __init__(self, shape, dtype):
        import ctypes

        import torch

        n = int(np.prod(shape)) * np.dtype(dtype).itemsize
        self.p = ctypes.c_void_p()
        err = self._runtime().cudaHostAlloc(ctypes.byref(self.p), ctypes.c_size_t(max(n, 1)), 0)
        if err != 0:
            raise RuntimeError(f"cudaHostAlloc of {n / 1e9:.1f} GB failed ({err})")
        buf = (ctypes.c_uint8 * max(n, 1)).from_address(self.p.value)
        self.a = np.frombuffer(buf, dtype=dtype, count=int(np.prod(shape))).reshape(shape)
        self.t = torch.from_numpy(self.a)

    def close(self):
        if self.p:
            del self.t, self.a
            self._runtime().cudaFreeHost(self.p)
            self.p = None


def parity_counts_u32(codes_h, got_h):
    """The headline's complete check (oracle): the Eq. 1 residual at every
    cell and conservation, over row bands on all host cores."""
    import oracle

    t0 = time.perf_counter()
    v = oracle.verify_counts_u32(codes_h, got_h, threads=os.cpu_count() or 1, band=1024)
    return {"vs_oracle": "Eq. 1 residual at every cell and conservation" + (
                " exact" if v["mismatches"] == 0 and v["conserved"] else
                (" (conserved modulo 2^32)" if v["mismatches"] == 0 and v["conserved_mod_2_32"]
                 else ": MISMATCH")),
            "residual_mismatches": v["mismatches"], "first_mismatch": v["first"],
            "outlet_sum": v["outlet_sum"], "valid_cells": v["n_valid"],
            "check_s": round(time.perf_counter() - t0, 1),
            "note": "the residual check is complete for integer counts on an acyclic raster"}


def parity_counts_u64(codes_h, o64):
    """The same complete check on uint64 counts (no wrap-around)."""
    import oracle

    t0 = time.perf_counter()
    v = oracle.verify_counts_u32(codes_h, o64, threads=os.cpu_count() or 1, band=1024)
    return {"vs_oracle": "uint64 Eq. 1 residual at every cell and exact conservation" + (
                "" if v["mismatches"] == 0 and v["conserved"] else ": MISMATCH"),
            "residual_mismatches": v["mismatches"], "first_mismatch": v["first"],
            "outlet_sum": v["outlet_sum"], "valid_cells": v["n_valid"],
            "check_s": round(time.perf_counter() - t0, 1)}


F32_SAMPLE_SEED, F32_SAMPLE_N, F32_BORDER_N = 504, 4096, 256


def parity_f32_sampled(codes_h, w_d, out_d):
    """Float32 sums at full size on sampled cells: 4096 cells uniform over the
    raster and 256 on its border (outlets), seeded; each cell's FP64 value
    comes from the oracle's search of its upstream area, and the result must
    lie within 2e-5 of it, relatively (weights >= 0)."""
    import torch

    import oracle

    R, C = codes_h.shape
    g = np.random.default_rng(F32_SAMPLE_SEED)
    inner = g.integers(0, R * C, F32_SAMPLE_N)
    side = g.integers(0, 4, F32_BORDER_N)
    t = g.integers(0, max(R, C), F32_BORDER_N)
    br = np.where(side == 0, 0, np.where(side == 1, R - 1, t % R))
    bc = np.where(side == 2, 0, np.where(side == 3, C - 1, t % C))
    cells = np.unique(np.concatenate([inner, br * C + bc])).astype(np.int64)
    got = out_d.view(-1)[torch.from_numpy(cells).to(out_d.device)].double().cpu().numpy()
    t0 = time.perf_counter()
    w_h = w_d.cpu().numpy()
    ref, size = oracle.upstream_sums(codes_h, cells, w_h, threads=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    del w_h
    ok = size > 0
    err = np.abs(got[ok] - ref[ok])
    rel = err / np.maximum(np.abs(ref[ok]), 1e-300)
    return {"vs_oracle": ("within 2e-5 relative on every sampled cell"
                          if bool((err <= 2e-5 * np.abs(ref[ok])).all()) else "MISMATCH"),
            "cells_checked": int(ok.sum()), "sample": f"{F32_SAMPLE_N} uniform + {F32_BORDER_N} "
            f"border cells (seed {F32_SAMPLE_SEED})", "max_rel_err": float(rel.max()),
            "largest_area_cells": int(size.max()), "area_cells_total": int(size[ok].sum()),
            "check_s": round(dt, 1),
            "oracle": "FP64 sum over each cell's upstream area, searched against the flow"}


def leg_ooc(fa, codes_h, reps: int):
    """Out-of-core counts: the headline raster's codes in pinned host memory,
    uint64 counts written to pinned host memory, solved on the device in
    16384 x 16384 outer blocks (two code copies in, one uint64 copy out per
    cell).  Timed on the host clock around the synchronous call.  Returns the
    record and the page-locked uint64 counts for the parity check, or
    (record, None) when the host lacks the memory for the output."""
    import torch

    R, C = codes_h.shape
    need = R * C * 8
    avail = host_available_bytes()
    if avail and avail < need * 1.25 + (8 << 30):
        return {"skipped": f"host memory: {avail / 1e9:.0f} GB available, the uint64 output "
                           f"needs {need / 1e9:.0f} GB"}, None
    c_h = torch.from_numpy(codes_h)
    pinned = HostPinned((R, C), np.int64)
    out64 = pinned.t
    opts = fa.options(None)
    n_ws = fa.fa_ooc_workspace_size(R, C, 0, 0, opts)
    work = torch.empty(n_ws, dtype=torch.uint8, device="cuda")
    st = fa.fa_accumulate_ooc(c_h, out64, 0, 0, work, opts)  # warm-up
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        st = fa.fa_accumulate_ooc(c_h, out64, 0, 0, work, opts)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * min(times)
    nb = -(-R // 16384) * -(-C // 16384)
    rec = {"workload": f"host-resident {R}x{C} headline raster", "blocks": nb,
           "block": [min(R, 16384), min(C, 16384)], "device_workspace_gb": n_ws / 1e9,
           "ms": ms, "ms_all": [1e3 * t for t in times], "cells_per_s": R * C / (ms / 1e3),
           "h2d_bytes": 2 * R * C, "d2h_bytes": 8 * R * C,
           "host_link_gbs": 10 * R * C / (ms / 1e3) / 1e9, "status": int(st),
           "out": "uint64 (exact beyond 2^32)"}
    del work
    torch.cuda.empty_cache()
    return rec, pinned


def headline_codes(args, dev):
    """uint8 codes of the headline raster on `dev`, its workload name and a
    description of its recipe."""
    import torch

    import synth

    if args.workload == "scale":
        n = args.scale_coarse
        codes_d = synth.scale_codes_device(n, n, SCALE_F, SCALE_SEED, SCALE_NSEED, device=dev)
        R, C = codes_d.shape
        return codes_d, f"d8_scale_{R}x{C}", (
            f"coarse {n}x{n} spectral DEM (seed {SCALE_SEED}) eps-filled (4-connected), "
            f"bilinear x{SCALE_F}, noise U[-0.5,0.5] m (seed {SCALE_NSEED}); steepest descent "
            "among neighbours lower in the upsampled surface (acyclic, no NoData)")
    codes = synth.dem_codes(ROWS, COLS, SEED)
    return torch.from_numpy(codes).to(dev), f"d8_dem_{ROWS}x{COLS}", (
        f"spectral DEM (seed {SEED}), 1% NoData disk, priority-flood eps fill, D8")


def scale_sample_codes(args, rows: int):
    """The first `rows` rows of the headline raster, generated on the host
    (bit-identical to the device generator's rows), as its own raster."""
    import synth

    if args.workload != "scale":
        return synth.dem_codes(ROWS, COLS, SEED)[:rows]
    n = args.scale_coarse
    full = synth.scale_codes_rows(n, n, SCALE_F, SCALE_SEED, SCALE_NSEED, 0, rows)
    return full


def main():
    global ROWS, COLS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale", choices=["scale", "dem16384"],
                    help="headline raster: the 1e10-cell scale raster (default) or the "
                         "16384^2 spectral DEM")
    ap.add_argument("--scale-coarse", type=int, default=SCALE_COARSE,
                    help="coarse side of the scale raster (x16 fine); smaller only for "
                         "profiler captures and quick checks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the end-to-end, f32 and 16384^2 legs")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up and timed steps (for ncu): no clock sampling, phase "
                         "timing, extra legs or CPU baseline")
    ap.add_argument("--profile-f32", action="store_true",
                    help="with --profile: after the timed steps, three calls of the float32 "
                         "form (w ~ U[0, 1)) on the same raster")
    ap.add_argument("--record-traffic", metavar="CSV",
                    help="write profiles/traffic.json from an ncu --csv capture of the forward "
                         "kernels (dram bytes, warp instructions) and exit; the capture's "
                         "raster is described by --workload/--scale-coarse/--size")
    ap.add_argument("--profile-absorb", action="store_true",
                    help="with --profile: after the timed steps, three calls of the absorption "
                         "form on the same raster")
    ap.add_argument("--tile", default="auto",
                    help="tile shape HxW for the headline, or 'auto' (fa_autotune; default)")
    ap.add_argument("--size", type=int, default=ROWS,
                    help="side of the 16384^2 DEM; smaller only for profiler captures")
    args = ap.parse_args()
    if args.size != ROWS:
        ROWS = COLS = args.size
    if args.record_traffic:
        if args.workload == "scale":
            n = (args.scale_coarse * SCALE_F) ** 2
            desc = (f"{args.scale_coarse * SCALE_F}^2 band-generated scale raster "
                    f"(coarse {args.scale_coarse}^2 x{SCALE_F}, seeds {SCALE_SEED}/{SCALE_NSEED})")
        else:
            n = ROWS * COLS
            desc = f"{ROWS}^2 spectral DEM seed {SEED}"
        print(json.dumps(record_traffic(args.record_traffic, n, desc), indent=1))
        return
    if args.profile:
        args.no_extra = args.no_cpu_baseline = True
    if args.warmup < 3:
        args.warmup = 3

    ws, rank, local = dist_setup() if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch

    import synth
    import paper_1608_04431_gb300 as fa

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = peaks()
    t_gen = time.perf_counter()
    codes_d, WORKLOAD, recipe = headline_codes(args, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    R, C = codes_d.shape
    cells = R * C
    if args.tile == "auto":
        # tuned on a band of the raster (its first rows) before the timed region
        tile = fa.autotune(codes_d[:min(R, TUNE_ROWS)])
        fa._ws_cache.clear()
        torch.cuda.empty_cache()
    else:
        tile = tuple(int(v) for v in args.tile.lower().split("x"))
    opts = fa.options(tile)
    work = torch.empty(fa.fa_workspace_size(R, C, opts), dtype=torch.uint8, device=dev)
    out_d = torch.empty((R, C), dtype=torch.uint32, device=dev)

    def step_counts():
        st = fa.fa_accumulate(codes_d, None, None, out_d, fa.FA_OUT_U32, work, opts, None, stream)
        if st != fa.FA_OK:
            raise fa.FlowAccError(st, "fa_accumulate")

    for _ in range(args.warmup):
        step_counts()
    torch.cuda.synchronize()
    st = fa.fa_status_read(None, work, stream)
    if st[0] not in (fa.FA_OK, fa.FA_WARN_OVERFLOW):
        raise fa.FlowAccError(st[0], "device status")
    overflow = st[0] == fa.FA_WARN_OVERFLOW

    sampler = ClockSampler(local)
    if not args.profile:
        sampler.start()
        t_pre = time.time()
        while time.time() - t_pre < 0.4:  # keep the GPU busy while the sampler starts
            step_counts()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step_counts()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, ws)
    value = job_throughput(cells, ms_max, ws)

    if args.profile:
        if args.profile_f32:
            g = torch.Generator(device=dev)
            g.manual_seed(WSEED)
            w_d = torch.rand(codes_d.shape, generator=g, device=dev, dtype=torch.float32)
            out_f = torch.empty(codes_d.shape, dtype=torch.float32, device=dev)
            for _ in range(3):
                s = fa.fa_accumulate(codes_d, w_d, None, out_f, fa.FA_OUT_F32, work, opts, None,
                                     stream)
                if s != fa.FA_OK:
                    raise fa.FlowAccError(s, "fa_accumulate f32")
            torch.cuda.synchronize()
            del w_d, out_f
        if args.profile_absorb:
            g = torch.Generator(device=dev)
            g.manual_seed(WSEED)
            w_d = torch.rand(codes_d.shape, generator=g, device=dev, dtype=torch.float32)
            g.manual_seed(ASEED)
            a_d = (torch.rand(codes_d.shape, generator=g, device=dev) * 0.1 + 0.9).clamp_(max=1.0)
            out_a = torch.empty(codes_d.shape, dtype=torch.float32, device=dev)
            opts_a = fa.options(ABS_TILE)
            work_a = torch.empty(fa.fa_absorb_workspace_size(R, C, opts_a),
                                 dtype=torch.uint8, device=dev)
            for _ in range(3):
                s = fa.fa_accumulate_absorb(codes_d, w_d, a_d, None, out_a, work_a, opts_a, None,
                                            stream)
                if s != fa.FA_OK:
                    raise fa.FlowAccError(s, "fa_accumulate_absorb")
            torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "ms_per_step": ms_max, "workload": WORKLOAD}),
              flush=True)
        return

    # per-phase durations, live, on the launching stream
    phases = []
    fa.fa_timing_enable(True)
    for _ in range(3):
        step_counts()
        phases.append(fa.fa_timing_read())
    fa.fa_timing_enable(False)
    ph = np.mean(np.array(phases), axis=0).tolist()
    names = ["pass1_tile_solve", "perimeter_graph_resolve", "pass2_tile_finalize"]
    dom = int(np.argmax(ph))
    alg = pass_bytes(cells)
    ach = alg[dom] / (ph[dom] / 1e3) / 1e9 if alg[dom] else 0.0
    roof = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_kind": peak_kind,
            "bytes_per_launch": alg[dom], "traffic": traffic_for(names[dom], cells)}
    step_ach = cells * BYTES_PER_CELL_COUNTS / (ms / 1e3) / 1e9
    roof_step = {"bound": "hbm", "achieved": step_ach, "peak": peak, "unit": "GB/s",
                 "frac": step_ach / peak, "bytes_per_cell": BYTES_PER_CELL_COUNTS}
    line = {
        "metric": "cells/s (D8 flow accumulation, uint32 counts)", "value": value,
        "unit": "cells/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": R, "cols": C, "recipe": recipe,
                   "tile": list(tile),
                   "tile_choice": ("fa_autotune on the first %d rows" % min(R, TUNE_ROWS))
                   if args.tile == "auto" else "fixed",
                   "weights": "unit", "out": "uint32",
                   "l2": "inputs+outputs %.1f GB > 129 MB L2, no flush" % (cells * 5 / 1e9),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "generation_s": round(t_gen, 1)},
        "roofline": roof, "roofline_step": roof_step,
        "phases_ms": dict(zip(names, ph)),
        "clocks": clocks,
    }
    line["gpu_launches"] = args.steps * fa.fa_kernel_launches(R, C, opts)
    line["roofline_issue"] = issue_roofline(names[dom], ph[dom], clocks.get("sm_mhz") or 0.0,
                                            torch.cuda.get_device_properties(dev).multi_processor_count,
                                            cells=cells)
    if overflow:
        line["status"] = "FA_WARN_OVERFLOW (a count reached 2^32; outputs are mod 2^32)"

    codes_h = None
    forms = {}
    check = not args.no_cpu_baseline and rank == 0  # the oracle's checks run on rank 0
    if not args.no_extra:
        # end to end through the public API from pinned host buffers
        pc = HostPinned((R, C), np.uint8)
        h_codes = pc.t
        h_codes.copy_(codes_d)
        po = HostPinned((R, C), np.int32)
        h_out = po.t
        ke = 3 if cells > 2e9 else max(5, args.steps // 4)

        def step_e2e():
            codes_d.copy_(h_codes, non_blocking=True)
            step_counts()
            h_out.copy_(out_d, non_blocking=True)

        step_e2e()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ke):
            step_e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        mse = max_over_ranks(e0.elapsed_time(e1) / ke, ws)
        line["e2e"] = {"value": job_throughput(cells, mse, ws), "unit": "cells/s",
                       "h2d_bytes_per_step": int(cells), "d2h_bytes_per_step": int(cells * 4),
                       "ms_per_step": mse, "steps": ke}
        codes_h = pc.a
        if check:
            line["parity"] = parity_counts_u32(codes_h, po.a.view(np.uint32))
        del h_out
        po.close()
        del po

        # out of core: the same raster from host memory, uint64 counts to host memory
        ooc_rec, ooc_out = leg_ooc(fa, codes_h, 2)
        if ooc_out is not None:
            if check:
                ooc_rec["parity"] = parity_counts_u64(codes_h, ooc_out.a.view(np.uint64))
            ooc_out.close()
        forms["out_of_core"] = ooc_rec
        del ooc_out

        # float32 weights on the headline raster: w ~ U[0, 1), drawn on the device
        del out_d
        torch.cuda.empty_cache()
        w_d = torch.empty((R, C), dtype=torch.float32, device=dev)
        g = torch.Generator(device=dev)
        g.manual_seed(SCALE_WSEED if args.workload == "scale" else WSEED)
        for r0 in range(0, R, 8192):
            w_d[r0:r0 + 8192].uniform_(0.0, 1.0, generator=g)
        outf = torch.empty((R, C), dtype=torch.float32, device=dev)
        # its own tile shape, tuned like the headline's on the first rows
        tile_f = fa.autotune(codes_d[:min(R, TUNE_ROWS)], w_d[:min(R, TUNE_ROWS)])
        fa._ws_cache.clear()
        torch.cuda.empty_cache()
        opts_f = fa.options(tile_f)
        work_f = torch.empty(fa.fa_workspace_size(R, C, opts_f), dtype=torch.uint8, device=dev)

        def step_f32():
            s = fa.fa_accumulate(codes_d, w_d, None, outf, fa.FA_OUT_F32, work_f, opts_f, None,
                                 stream)
            if s != fa.FA_OK:
                raise fa.FlowAccError(s, "fa_accumulate f32")

        for _ in range(3):
            step_f32()
        kf = 5 if cells > 2e9 else max(10, args.steps // 3)
        msf_h = _time(step_f32, stream, kf)
        stf = fa.fa_status_read(None, work_f, stream)[0]
        forms["headline_f32"] = {
            "workload": WORKLOAD, "ms": msf_h, "cells_per_s": cells / (msf_h / 1e3),
            "tile": list(tile_f), "bytes_per_cell": BYTES_PER_CELL_F32,
            "hbm_frac_step": cells * BYTES_PER_CELL_F32 / (msf_h / 1e3) / 1e9 / peak,
            "status": int(stf)}
        if check:
            forms["headline_f32"]["parity"] = parity_f32_sampled(codes_h, w_d, outf)
        del w_d, outf, work_f
    del codes_d, work
    torch.cuda.empty_cache()

    d8_data = absorb_data = dem_got = None
    if not args.no_extra:
        forms_dem, d8_data, absorb_data, dem_got = legs_dem16384(fa, dev, stream, peak, args,
                                                                 rank, ws)
        forms.update(forms_dem)
    if forms:
        line["forms"] = forms

    if not args.no_cpu_baseline and rank == 0:
        import oracle

        # the oracle on a bounded sample of the headline workload
        rows_s = CPU_SAMPLE_ROWS if args.workload == "scale" else ROWS
        sample = codes_h[:rows_s] if codes_h is not None else scale_sample_codes(args, rows_s)
        oracle.build()
        t0 = time.perf_counter()
        res = oracle.counts(np.ascontiguousarray(sample))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sample.size / dt, "unit": "cells/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"rows 0..{sample.shape[0] - 1} of the {R}x{C} headline "
                                          f"raster as a raster of their own ({sample.size:.3g} "
                                          f"cells, {dt:.1f} s)"}
        del res
        if dem_got is not None:
            dcodes = synth.dem_codes(ROWS, COLS, SEED)
            ref = oracle.counts(dcodes).values.astype(np.uint32)
            forms["plain_u32_dem"]["parity_vs_oracle"] = (
                "bit-exact" if np.array_equal(dem_got, ref) else "MISMATCH")
            del ref
        if d8_data is not None:  # the direction step's oracle, timed on one core too
            z, nd, got_d8 = d8_data
            t0 = time.perf_counter()
            ref_d8 = oracle.d8(z, nd)
            dt8 = time.perf_counter() - t0
            rec = forms["d8_directions"]
            rec["parity_vs_oracle"] = "bit-exact" if np.array_equal(got_d8, ref_d8) else "MISMATCH"
            rec["cpu_oracle_cells_per_s"] = z.size / dt8
        if absorb_data is not None:  # absorption's oracle (FP64), timed on one core
            w_h, a_h, got_a = absorb_data
            dcodes = synth.dem_codes(ROWS, COLS, SEED)
            t0 = time.perf_counter()
            ref_a = oracle.absorb(dcodes, a_h, w_h)
            dta = time.perf_counter() - t0
            ok = ref_a.state == 1
            err = np.abs(got_a[ok].astype(np.float64) - ref_a.values[ok])
            bound = 2e-5 * np.abs(ref_a.values[ok])
            rec = forms["absorb"]
            rec["parity_vs_oracle"] = ("within 2e-5 relative" if bool((err <= bound).all())
                                       else "MISMATCH")
            rec["max_rel_err_vs_oracle"] = float(np.max(err / np.maximum(np.abs(ref_a.values[ok]),
                                                                         1e-300)))
            rec["cpu_oracle_cells_per_s"] = dcodes.size / dta
            del absorb_data, ref_a

    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def legs_dem16384(fa, dev, stream, peak, args, rank, ws):
    """The forms measured on the 16384^2 spectral DEM: plain uint32 counts,
    float32 weights, packed codes, absorption, batches, D8 directions and the
    adjoint (8192^2), each against the plain kernel on the same GPU."""
    import torch

    import synth

    forms = {}
    codes = synth.dem_codes(ROWS, COLS, SEED)
    cells = codes.size
    codes_d = torch.from_numpy(codes).to(dev)
    tile = fa.autotune(codes_d)
    opts = fa.options(tile)
    work = torch.empty(fa.fa_workspace_size(ROWS, COLS, opts), dtype=torch.uint8, device=dev)
    out_d = torch.empty((ROWS, COLS), dtype=torch.uint32, device=dev)

    def step_counts():
        st = fa.fa_accumulate(codes_d, None, None, out_d, fa.FA_OUT_U32, work, opts, None, stream)
        if st != fa.FA_OK:
            raise fa.FlowAccError(st, "fa_accumulate")

    for _ in range(3):
        step_counts()
    k2 = max(10, args.steps)
    ms = _time(step_counts, stream, k2)
    fa.fa_timing_enable(True)
    ph = []
    for _ in range(3):
        step_counts()
        ph.append(fa.fa_timing_read())
    fa.fa_timing_enable(False)
    ph = np.mean(np.array(ph), axis=0).tolist()
    forms["plain_u32_dem"] = {
        "workload": f"d8_dem_{ROWS}x{COLS}", "ms": ms, "cells_per_s": cells / (ms / 1e3),
        "tile": list(tile), "hbm_frac_step": cells * BYTES_PER_CELL_COUNTS / (ms / 1e3) / 1e9 / peak,
        "phases_ms": dict(zip(["pass1_tile_solve", "perimeter_graph_resolve",
                               "pass2_tile_finalize"], ph))}
    dem_got = out_d.view(torch.int32).cpu().numpy().view(np.uint32)

    # float32 weighted form on the same raster
    w_d = torch.from_numpy(synth.uniform_weights(codes.shape, WSEED)).to(dev)
    outf = torch.empty((ROWS, COLS), dtype=torch.float32, device=dev)
    tile_f = fa.autotune(codes_d, w_d)
    opts_f = fa.options(tile_f)
    work_f = torch.empty(fa.fa_workspace_size(ROWS, COLS, opts_f), dtype=torch.uint8, device=dev)

    def step_f32():
        s = fa.fa_accumulate(codes_d, w_d, None, outf, fa.FA_OUT_F32, work_f, opts_f, None, stream)
        if s != fa.FA_OK:
            raise fa.FlowAccError(s, "fa_accumulate f32")

    for _ in range(3):
        step_f32()
    msf = _time(step_f32, stream, k2)
    forms["plain_f32_dem"] = {"workload": f"d8_dem_{ROWS}x{COLS}", "cells_per_s": cells / (msf / 1e3),
                              "ms": msf, "tile": list(tile_f),
                              "hbm_frac_step": cells * BYTES_PER_CELL_F32 / (msf / 1e3) / 1e9 / peak}
    del w_d, outf, work_f

    # packed codes (two per byte, 4.5 B/cell) on the same raster and tile
    pk = fa.pack_codes(codes_d)
    out_p = torch.empty_like(out_d)
    opts_p = fa.options(tile, code_format=fa.FA_CODES_NIBBLE)

    def step_packed():
        s = fa.fa_accumulate(pk, None, None, out_p, fa.FA_OUT_U32, work, opts_p, None, stream)
        if s != fa.FA_OK:
            raise fa.FlowAccError(s, "fa_accumulate packed")

    for _ in range(3):
        step_packed()
    msp = _time(step_packed, stream, k2)
    forms["plain_u32_packed"] = {
        "cells_per_s": cells / (msp / 1e3), "ms": msp, "tile": list(tile), "bytes_per_cell": 4.5,
        "hbm_frac_step": cells * 4.5 / (msp / 1e3) / 1e9 / peak,
        "identical_to_byte_codes": bool(torch.equal(out_p.view(torch.int32),
                                                    out_d.view(torch.int32)))}
    del pk, out_p

    forms["absorb"], absorb_data = leg_absorb(fa, dev, stream, codes_d, msf, cells, 3, k2, peak)
    if rank != 0 or args.no_cpu_baseline:
        absorb_data = None
    del codes_d, work, out_d
    fa._ws_cache.clear()
    torch.cuda.empty_cache()

    d8_data = None
    if rank == 0:
        b = leg_batched(fa, dev, stream, opts, 2, 5)
        b["hbm_frac_step"] = b["hbm_frac_step"] / peak
        b["ns_per_cell_plain_f32"] = msf * 1e6 / cells
        b["time_per_cell_vs_plain_f32"] = b["ns_per_cell_field"] / b["ns_per_cell_plain_f32"]
        forms["batched"] = b
        torch.cuda.empty_cache()
        forms["d8_directions"], d8_data = leg_d8(fa, dev, stream, 3, 50, peak)
        torch.cuda.empty_cache()
        a = leg_adjoint(fa, dev, stream, fa.options(TILE), 3, 20)
        a["hbm_frac_step"] = a["hbm_frac_step"] / peak
        a["time_per_cell_vs_plain_f32"] = (a["ms_adjoint"] / a["cells"]) / (msf / cells)
        forms["adjoint"] = a
        fa._ws_cache.clear()
        torch.cuda.empty_cache()
    return forms, d8_data, absorb_data, dem_got



if __name__ == "__main__":
    main()
