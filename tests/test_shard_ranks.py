"""The shard form's exchange on CPU ranks (gloo): every rank exports the
records of its band of outer blocks, rank 0 gathers them, solves the blocks'
perimeter graph and scatters in(p), every rank finishes its band.  The stages
are the CPU stand-ins of tests/_shard_stages.py (the CUDA stages are covered
by tests/test_gpu_shard.py); the assembled counts must equal the oracle's
counts of the whole raster (Algorithm 1), exactly.  Also the host-side
checks of the C entry points (nothing is launched)."""
import ctypes
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from tests._shard_stages import Grid, OracleStages, perim_cells

fa = pytest.importorskip("paper_1608_04431_gb300")
shard = fa.shard

CASES = {
    # name: (rows, cols, seed, block)
    "ragged": (70, 53, 11, (16, 20)),
    "one_block_row": (12, 90, 12, (16, 32)),
    "thin_blocks": (64, 40, 13, (5, 40)),
}


def _codes(rows, cols, seed):
    return synth.acyclic_random_codes(rows, cols, seed)


def _want(codes):
    return oracle.counts(codes).values


# ---------------------------------------------------------------------------
# pieces
# ---------------------------------------------------------------------------
def test_records_layout_and_put():
    pmax = 7
    a = shard.Records(2, pmax)
    assert a.buf.numel() == shard.Records.nbytes(2, pmax) == 14 * 2 * pmax + 8
    a.nexit(2)[:] = torch.tensor([3, 1], dtype=torch.int32)
    a.link(2)[:] = torch.arange(2 * pmax, dtype=torch.int16)
    a.node_dst(2)[:] = torch.arange(100, 100 + 2 * pmax, dtype=torch.int32)
    a.node_val(2)[:] = torch.arange(2 * pmax, dtype=torch.float64) / 2
    b = shard.Records(5, pmax)
    b.put(3, a, 2)
    assert torch.equal(b.nexit(5), torch.tensor([0, 0, 0, 3, 1], dtype=torch.int32))
    assert torch.equal(b.link(5)[3 * pmax:], a.link(2))
    assert torch.equal(b.node_dst(5)[3 * pmax:], a.node_dst(2))
    assert torch.equal(b.node_val(5)[3 * pmax:], a.node_val(2))
    assert not b.node_val(3).any() and not b.link(3).any()


def test_bands_partition_block_rows():
    for nby in (1, 2, 5, 9):
        for world in (1, 2, 3, 4, 8):
            bs = shard.bands(nby, world)
            assert len(bs) == world and bs[0][0] == 0 and bs[-1][1] == nby
            assert all(bs[i][1] == bs[i + 1][0] for i in range(world - 1))
            sizes = [b1 - b0 for b0, b1 in bs]
            assert max(sizes) - min(sizes) <= 1
    assert shard.band_rows((0, 2), 16, 70) == (0, 33)
    assert shard.band_rows((2, 5), 16, 70) == (31, 70)
    assert shard.band_rows((1, 1), 16, 70) == (0, 0)
    assert shard.out_rows((2, 5), 16, 70) == (32, 70)


def test_geometry_matches_the_block_grid():
    for rows, cols, _, block in CASES.values():
        st, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, *block)
        g = Grid((rows, cols), block)
        assert st == fa.FA_OK and (nby, nbx, pmax) == (g.nby, g.nbx, g.pmax)
    st, nby, nbx, pmax = fa.fa_shard_geometry(100, 100, 0, 0)  # default block: the raster
    assert (st, nby, nbx, pmax) == (fa.FA_OK, 1, 1, 396)
    assert fa.fa_shard_geometry(40000, 40000, 20000, 20000)[0] == fa.FA_ERR_INVALID_ARG


def test_perimeter_order_visits_each_cell_once():
    for h, w in ((1, 1), (1, 6), (5, 1), (2, 2), (3, 4), (6, 5)):
        cells = perim_cells(h, w)
        assert len(cells) == len(set(cells)) == (w if h == 1 else h if w == 1 else 2 * (h + w) - 4)
        assert all(r in (0, h - 1) or c in (0, w - 1) for r, c in cells)


@pytest.mark.parametrize("name", sorted(CASES))
def test_stand_in_stages_in_one_process(name):
    rows, cols, seed, block = CASES[name]
    codes = _codes(rows, cols, seed)
    out = shard.accumulate_sharded(torch.from_numpy(codes), 0, (rows, cols), block,
                                   stages=OracleStages())
    assert np.array_equal(out.numpy().view(np.uint64), _want(codes))


def test_stand_in_resolve_on_a_hand_made_chain():
    # a 1 x 6 raster flowing east in blocks of 1 x 2: every block passes its
    # flow on, so G of the exit of block b is 2 (b + 1) and in(p) at the
    # first cell of block b + 1 is that
    codes = np.full((1, 6), 1, dtype=np.uint8)
    out = shard.accumulate_sharded(torch.from_numpy(codes), 0, (1, 6), (1, 2), stages=OracleStages())
    assert out.numpy().ravel().tolist() == [1, 2, 3, 4, 5, 6]


# ---------------------------------------------------------------------------
# gloo ranks
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, case, res):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        rows, cols, seed, block = case
        codes = _codes(rows, cols, seed)
        nby = Grid((rows, cols), block).nby
        band = shard.bands(nby, ws)[rank]
        ra, rb = shard.band_rows(band, block[0], rows)
        mine = torch.from_numpy(np.ascontiguousarray(codes[ra:rb]))  # only the band and its ring
        out = shard.accumulate_sharded(mine, ra, (rows, cols), block, stages=OracleStages())
        res[rank] = (band, out.numpy().tobytes())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,name", [(2, "ragged"), (3, "thin_blocks"), (3, "one_block_row")])
def test_gloo_ranks_match_the_whole_raster(ws, name):
    rows, cols, seed, block = CASES[name]
    mgr = mp.get_context("spawn").Manager()
    res = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), CASES[name], res), nprocs=ws, join=True,
                       start_method="spawn")
    got = np.zeros((rows, cols), dtype=np.uint64)
    bh = Grid((rows, cols), block).bh
    for r in range(ws):
        band, raw = res[r]
        r0, r1 = shard.out_rows(band, bh, rows)
        got[r0:r1] = np.frombuffer(raw, dtype=np.uint64).reshape(r1 - r0, cols)
    assert np.array_equal(got, _want(_codes(rows, cols, seed)))


# ---------------------------------------------------------------------------
# host-side checks of the C entry points (no device work)
# ---------------------------------------------------------------------------
def _records(nb, pmax):
    r = shard.Records(nb, pmax)
    return r, r.nexit(nb), r.link(nb), r.node_dst(nb), r.node_val(nb)


def test_resolve_rejects_bad_records_before_any_device_work():
    lib = fa._lib.load()
    rows, cols, bh, bw = 32, 32, 16, 16
    _, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, bh, bw)
    nb = nby * nbx
    fake_ws = ctypes.c_void_p(256)  # never dereferenced: the records are checked first

    def resolve(rec):
        _, nexit, link, dst, val = rec
        inflow = torch.zeros(nb * pmax, dtype=torch.int64)
        return lib.fa_shard_resolve(rows, cols, bh, bw, fa._ptr(nexit), fa._ptr(link), fa._ptr(dst),
                                    fa._ptr(val), fa._ptr(inflow), fake_ws, 0, None, None)

    rec = _records(nb, pmax)
    rec[2][:] = -1                       # all links none
    rec[1][0] = pmax + 1                 # more exits than slots
    assert resolve(rec) == fa.FA_ERR_INVALID_ARG
    rec[1][0] = 1
    rec[3][0] = nb * pmax                # target outside the raster
    assert resolve(rec) == fa.FA_ERR_INVALID_ARG
    rec[3][0] = pmax + 3                 # a slot of block 1 ...
    rec[2][pmax + 3] = 5                 # ... linked to rank 5, but block 1 has no exits
    assert resolve(rec) == fa.FA_ERR_INVALID_ARG
    rec[2][pmax + 3] = -1                # link none: valid records, then the workspace is checked
    assert resolve(rec) == fa.FA_ERR_WORKSPACE


def test_export_and_finish_check_bands_and_rows():
    lib = fa._lib.load()
    rows, cols, bh, bw = 70, 53, 16, 20
    codes = torch.zeros((rows, cols), dtype=torch.uint8)
    _, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, bh, bw)
    rec = _records(nbx * nby, pmax)
    fake_ws = ctypes.c_void_p(256)

    def export(band0, band1, row0, nrows):
        return lib.fa_shard_export(fa._ptr(codes), row0, nrows, cols, rows, cols, bh, bw, band0,
                                   band1, fa._ptr(rec[1]), fa._ptr(rec[2]), fa._ptr(rec[3]),
                                   fa._ptr(rec[4]), fake_ws, 0, None, None, None)

    assert export(0, nby + 1, 0, rows) == fa.FA_ERR_INVALID_ARG     # past the last block row
    assert export(2, 1, 0, rows) == fa.FA_ERR_INVALID_ARG           # reversed band
    assert export(1, 2, 16, 16) == fa.FA_ERR_INVALID_ARG            # ring row 15 missing
    assert export(1, 2, 15, 17) == fa.FA_ERR_INVALID_ARG            # ring row 32 missing
    assert export(1, 2, 15, 18) == fa.FA_ERR_WORKSPACE              # rows fine: workspace next
    assert export(2, 2, 0, 0) == fa.FA_ERR_WORKSPACE                # empty band: valid
    inflow = torch.zeros(nbx * pmax, dtype=torch.int64)
    out = torch.zeros((16, cols), dtype=torch.int64)

    def finish(band0, band1, row0, nrows, pitch_out=cols):
        return lib.fa_shard_finish(fa._ptr(codes), row0, nrows, cols, rows, cols, bh, bw, band0,
                                   band1, fa._ptr(inflow), fa._ptr(out), pitch_out, fake_ws, 0,
                                   None, None, None)

    assert finish(1, 2, 16, 16) == fa.FA_ERR_INVALID_ARG
    assert finish(1, 2, 15, 18, pitch_out=cols - 1) == fa.FA_ERR_INVALID_ARG
    assert finish(1, 2, 15, 18) == fa.FA_ERR_WORKSPACE


def test_empty_raster_and_idle_ranks_in_one_process():
    empty = torch.zeros((0, 9), dtype=torch.uint8)
    out = shard.accumulate_sharded(empty, 0, (0, 9), (4, 4), stages=OracleStages())
    assert out.shape == (0, 9)
    st, nby, nbx, pmax = fa.fa_shard_geometry(0, 9, 4, 4)
    assert st == fa.FA_OK and nby == 0
    assert shard.bands(0, 3) == [(0, 0)] * 3


# ---------------------------------------------------------------------------
# failures: no rank is left waiting in a collective
# ---------------------------------------------------------------------------
class _FailingStages(OracleStages):
    """Stand-ins that make one stage fail on one rank: raise (a failed call)
    or report FA_ERR_BAD_CODE (a condition found by the device)."""

    def __init__(self, rank, where, how):
        self.rank, self.where, self.how = rank, where, how

    def _hit(self, stage):
        return dist.get_rank() == self.rank and self.where == stage

    def export(self, *args):
        st = super().export(*args)
        if self._hit("export"):
            if self.how == "raise":
                raise RuntimeError("export broke")
            return fa.FA_ERR_BAD_CODE
        return st

    def resolve(self, *args):
        if self._hit("resolve"):
            raise RuntimeError("resolve broke")
        return super().resolve(*args)

    def finish(self, *args):
        st = super().finish(*args)
        if self._hit("finish"):
            raise RuntimeError("finish broke")
        return st


def _rank_fail(rank, ws, port, case, fail, check, res):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=60))
    try:
        rows, cols, seed, block = case
        codes = torch.from_numpy(_codes(rows, cols, seed))
        try:
            out = shard.accumulate_sharded(codes, 0, (rows, cols), block,
                                           stages=_FailingStages(*fail), check=check)
            res[rank] = ("ok", out.numpy().tobytes())
        except fa.FlowAccError as e:
            res[rank] = ("status", e.status)
        except shard.ShardAborted:
            res[rank] = ("aborted", None)
        except RuntimeError as e:
            res[rank] = ("raised", str(e))
    finally:
        dist.destroy_process_group()


def _run_fail(fail, check=True, ws=2, name="ragged"):
    mgr = mp.get_context("spawn").Manager()
    res = mgr.dict()
    mp.start_processes(_rank_fail, args=(ws, _free_port(), CASES[name], fail, check, res),
                       nprocs=ws, join=True, start_method="spawn")
    return [res[r] for r in range(ws)]


@pytest.mark.parametrize("fail,expect", [
    ((1, "export", "raise"), [("aborted", None), ("raised", "export broke")]),
    ((0, "resolve", "raise"), [("raised", "resolve broke"), ("aborted", None)]),
    ((1, "finish", "raise"), [("aborted", None), ("raised", "finish broke")]),
])
def test_a_failed_stage_stops_every_rank(fail, expect):
    assert _run_fail(fail) == expect


def test_device_conditions_reach_every_rank():
    got = _run_fail((1, "export", "status"), check=True)
    assert got == [("status", fa.FA_ERR_BAD_CODE)] * 2
    got = _run_fail((1, "export", "status"), check=False)
    rows, cols, seed, block = CASES["ragged"]
    whole = np.zeros((rows, cols), dtype=np.uint64)
    bh = Grid((rows, cols), block).bh
    for r, (kind, raw) in enumerate(got):
        assert kind == "ok"
        band = shard.bands(Grid((rows, cols), block).nby, 2)[r]
        r0, r1 = shard.out_rows(band, bh, rows)
        whole[r0:r1] = np.frombuffer(raw, dtype=np.uint64).reshape(r1 - r0, cols)
    assert np.array_equal(whole, _want(_codes(rows, cols, seed)))


# ---------------------------------------------------------------------------
# checkpoint and resume: records kept after pass A, in(p) after the resolve
# ---------------------------------------------------------------------------
class _CountingStages(OracleStages):
    def __init__(self, fail_finish_rank=None):
        self.calls = {"export": 0, "resolve": 0, "finish": 0}
        self.fail_finish_rank = fail_finish_rank

    def export(self, *args):
        self.calls["export"] += 1
        return super().export(*args)

    def resolve(self, *args):
        self.calls["resolve"] += 1
        return super().resolve(*args)

    def finish(self, *args):
        self.calls["finish"] += 1
        rank = dist.get_rank() if dist.is_initialized() else 0
        if self.fail_finish_rank == rank:
            raise RuntimeError("crash during the finish")
        return super().finish(*args)


def test_checkpoint_resumes_at_the_finish(tmp_path):
    rows, cols, seed, block = CASES["ragged"]
    codes = torch.from_numpy(_codes(rows, cols, seed))
    want = _want(codes.numpy())
    first = _CountingStages(fail_finish_rank=0)
    with pytest.raises(RuntimeError, match="crash"):
        shard.accumulate_sharded(codes, 0, (rows, cols), block, stages=first, checkpoint=str(tmp_path))
    assert first.calls == {"export": 1, "resolve": 1, "finish": 1}
    again = _CountingStages()
    out = shard.accumulate_sharded(codes, 0, (rows, cols), block, stages=again, checkpoint=str(tmp_path))
    assert again.calls == {"export": 0, "resolve": 0, "finish": 1}
    assert np.array_equal(out.numpy().view(np.uint64), want)
    # files of another block shape do not apply; a damaged file is redone
    other = _CountingStages()
    out = shard.accumulate_sharded(codes, 0, (rows, cols), (8, 20), stages=other, checkpoint=str(tmp_path))
    assert other.calls == {"export": 1, "resolve": 1, "finish": 1}
    assert np.array_equal(out.numpy().view(np.uint64), want)
    (tmp_path / "records_0_of_1.npz").write_bytes(b"not an npz file")
    redo = _CountingStages()
    out = shard.accumulate_sharded(codes, 0, (rows, cols), (8, 20), stages=redo, checkpoint=str(tmp_path))
    assert redo.calls == {"export": 1, "resolve": 0, "finish": 1}
    assert np.array_equal(out.numpy().view(np.uint64), want)
    whole = (tmp_path / "inflow_of_1.npz").read_bytes()
    (tmp_path / "inflow_of_1.npz").write_bytes(whole[: len(whole) // 2])  # cut short
    redo = _CountingStages()
    out = shard.accumulate_sharded(codes, 0, (rows, cols), (8, 20), stages=redo, checkpoint=str(tmp_path))
    assert redo.calls == {"export": 0, "resolve": 1, "finish": 1}
    assert np.array_equal(out.numpy().view(np.uint64), want)


def _rank_ckpt(rank, ws, port, case, ckpt, fail_rank, res):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=60))
    try:
        rows, cols, seed, block = case
        codes = torch.from_numpy(_codes(rows, cols, seed))
        st = _CountingStages(fail_finish_rank=fail_rank)
        try:
            out = shard.accumulate_sharded(codes, 0, (rows, cols), block, stages=st, checkpoint=ckpt)
            res[rank] = ("ok", dict(st.calls), out.numpy().tobytes())
        except (RuntimeError, shard.ShardAborted) as e:
            res[rank] = (type(e).__name__, dict(st.calls), None)
    finally:
        dist.destroy_process_group()


def test_checkpoint_resume_on_gloo_ranks(tmp_path):
    ws, name = 2, "ragged"
    rows, cols, seed, block = CASES[name]

    def run(fail_rank):
        mgr = mp.get_context("spawn").Manager()
        res = mgr.dict()
        mp.start_processes(_rank_ckpt, args=(ws, _free_port(), CASES[name], str(tmp_path), fail_rank,
                                             res), nprocs=ws, join=True, start_method="spawn")
        return [res[r] for r in range(ws)]

    first = run(fail_rank=1)
    assert [k for k, _, _ in first] == ["ShardAborted", "RuntimeError"]
    assert [c["export"] for _, c, _ in first] == [1, 1] and first[0][1]["resolve"] == 1
    again = run(fail_rank=None)
    assert all(k == "ok" for k, _, _ in again)
    assert [c for _, c, _ in again] == [{"export": 0, "resolve": 0, "finish": 1}] * 2
    got = np.zeros((rows, cols), dtype=np.uint64)
    g = Grid((rows, cols), block)
    for r, (_, _, raw) in enumerate(again):
        r0, r1 = shard.out_rows(shard.bands(g.nby, ws)[r], g.bh, rows)
        got[r0:r1] = np.frombuffer(raw, dtype=np.uint64).reshape(r1 - r0, cols)
    assert np.array_equal(got, _want(_codes(rows, cols, seed)))


# ---------------------------------------------------------------------------
# rank loss, injected on the host: a rank that exits mid-solve
# ---------------------------------------------------------------------------
class _DiesInExport(OracleStages):
    def export(self, *args):
        if dist.get_rank() == 1:
            os._exit(3)  # the process is gone, with nothing in flight
        return super().export(*args)


def _rank_lost(rank, ws, port, case, res):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=30))
    rows, cols, seed, block = case
    codes = torch.from_numpy(_codes(rows, cols, seed))
    try:
        shard.accumulate_sharded(codes, 0, (rows, cols), block, stages=_DiesInExport())
        res[rank] = "finished"
    except Exception as e:  # noqa: BLE001  (whatever the backend raises for a lost peer)
        res[rank] = "raised " + type(e).__name__
    try:
        dist.destroy_process_group()
    except Exception:  # noqa: BLE001
        pass


def test_a_lost_rank_makes_the_others_raise_not_hang():
    mgr = mp.get_context("spawn").Manager()
    res = mgr.dict()
    ctx = mp.start_processes(_rank_lost, args=(2, _free_port(), CASES["ragged"], res), nprocs=2,
                             join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(timeout=120)
    alive = [p for p in ctx.processes if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank was still waiting after its peer exited"
    assert ctx.processes[1].exitcode == 3
    assert ctx.processes[0].exitcode == 0 and res[0].startswith("raised")
