"""GPU parity of the shard form (fa_shard_export / fa_shard_resolve /
fa_shard_finish) against the oracle.

Ranks are emulated in one process, one after another (their kernels never
wait on one another: the exchange is on the host), each given only its
band's rows of codes.  Counts must equal the oracle's counts of the whole
raster (Algorithm 1) bit for bit.  The device records are compared with the
CPU stand-in stages of tests/_shard_stages.py on what is unique about them:
per perimeter slot, the target and A_loc of the exit it links to, and in(p).
The multi-process exchange itself is tested on gloo ranks in
tests/test_shard_ranks.py.
"""
import numpy as np
import pytest
import torch

import synth
from tests._shard_stages import OracleStages

pytestmark = pytest.mark.gpu

fa = pytest.importorskip("paper_1608_04431_gb300")
shard = fa.shard


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def emulate(codes, block, world, stages, tile=None):
    """The protocol of shard.accumulate_sharded with `world` ranks run one
    after another; returns (uint64 counts, records of all blocks, in(p))."""
    rows, cols = codes.shape
    st, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, *block)
    assert st == fa.FA_OK
    bh = min(block[0], rows)
    bands = shard.bands(nby, world)
    cap = max(b1 - b0 for b0, b1 in bands) * nbx
    parts = []
    for band in bands:
        rec = shard.Records(cap, pmax)
        if band[1] > band[0]:
            ra, rb = shard.band_rows(band, bh, rows)
            assert stages.export(torch.from_numpy(np.ascontiguousarray(codes[ra:rb])), ra,
                                 (rows, cols), block, band, rec) == fa.FA_OK
        parts.append(rec)
    full = shard.Records(nby * nbx, pmax)
    for (b0, b1), rec in zip(bands, parts):
        if b1 > b0:
            full.put(b0 * nbx, rec, (b1 - b0) * nbx)
    inflow, st = stages.resolve((rows, cols), block, full)
    assert st == fa.FA_OK
    out = np.zeros((rows, cols), dtype=np.uint64)
    for band in bands:
        if band[1] == band[0]:
            continue
        ra, rb = shard.band_rows(band, bh, rows)
        r0, r1 = shard.out_rows(band, bh, rows)
        o = torch.zeros((r1 - r0, cols), dtype=torch.int64)
        part = inflow[band[0] * nbx * pmax: band[1] * nbx * pmax].clone()
        assert stages.finish(torch.from_numpy(np.ascontiguousarray(codes[ra:rb])), ra, (rows, cols),
                             block, band, part, o) == fa.FA_OK
        out[r0:r1] = o.numpy().view(np.uint64)
    return out, full, inflow.numpy().view(np.uint64)


def canonical(rec, nb):
    """Per block perimeter slot: (target slot, A_loc) of the exit its link
    names, or None; independent of the order of the exit ranks."""
    pmax = rec.pmax
    link = rec.link(nb).numpy().view(np.uint16)
    dst = rec.node_dst(nb).numpy().view(np.uint32)
    val = rec.node_val(nb).numpy()
    nexit = rec.nexit(nb).numpy().view(np.uint32)
    out = []
    for b in range(nb):
        for s in range(pmax):
            lk = int(link[b * pmax + s])
            if lk == 0xFFFF:
                out.append(None)
            else:
                assert lk < nexit[b]
                out.append((int(dst[b * pmax + lk]), float(val[b * pmax + lk])))
    return out


@pytest.mark.parametrize("shape,seed,block,world,tile", [
    ((300, 410), 401, (64, 80), 2, None),
    ((300, 410), 401, (40, 56), 3, (16, 16)),
    ((300, 410), 401, (17, 23), 4, (8, 8)),
    ((700, 530), 451, (128, 200), 5, (32, 64)),
    ((700, 530), 451, (700, 100), 2, None),      # one block row: one rank idle
    ((64, 900), 452, (1, 900), 8, None),         # one-row blocks
])
def test_device_stages_match_oracle(oracle_mod, shape, seed, block, world, tile):
    codes = synth.dem_codes(*shape, seed)
    got, _, _ = emulate(codes, block, world, shard.DeviceStages(tile=tile), tile)
    ref = oracle_mod.counts(codes)
    assert ref.n_cycle == 0 and ref.n_bad == 0
    np.testing.assert_array_equal(got, ref.values.astype(np.uint64))


@pytest.mark.parametrize("shape,seed,block", [((150, 170), 461, (32, 40)), ((90, 77), 462, (16, 20))])
def test_device_records_and_inflow_match_stand_in(shape, seed, block):
    codes = synth.dem_codes(*shape, seed)
    dev_out, dev_rec, dev_in = emulate(codes, block, 2, shard.DeviceStages())
    ref_out, ref_rec, ref_in = emulate(codes, block, 2, OracleStages())
    nb = dev_rec.cap
    assert canonical(dev_rec, nb) == canonical(ref_rec, nb)
    np.testing.assert_array_equal(dev_in, ref_in)
    np.testing.assert_array_equal(dev_out, ref_out)


def test_device_resolve_takes_records_made_elsewhere(oracle_mod):
    """The C resolve on records exported by the stand-in (another rank order
    and another implementation) gives the same in(p) and counts."""
    codes = synth.acyclic_random_codes(70, 53, 11)
    block = (16, 20)
    _, ref_rec, ref_in = emulate(codes, block, 3, OracleStages())
    inflow, st = shard.DeviceStages().resolve((70, 53), block, ref_rec)
    assert st == fa.FA_OK
    np.testing.assert_array_equal(inflow.numpy().view(np.uint64), ref_in)


def test_accumulate_sharded_single_process(oracle_mod):
    codes = synth.dem_codes(1000, 1300, 441)
    out = shard.accumulate_sharded(torch.from_numpy(codes), 0, codes.shape, (256, 384))
    ref = oracle_mod.counts(codes)
    np.testing.assert_array_equal(out.numpy().view(np.uint64), ref.values.astype(np.uint64))


def test_cycle_through_blocks_is_reported_by_resolve():
    # cells (7, 7) and (8, 7) point at each other across the border of
    # 8-row blocks: a cycle of two outer exits
    codes = np.full((16, 16), 1, np.uint8)
    codes[7, 7], codes[8, 7] = 7, 3  # S, N
    st = shard.DeviceStages()
    rows, cols = codes.shape
    _, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, 8, 16)
    rec = shard.Records(nby * nbx, pmax)
    assert st.export(torch.from_numpy(codes), 0, (rows, cols), (8, 16), (0, nby), rec) == fa.FA_OK
    inflow = torch.zeros(nby * nbx * pmax, dtype=torch.int64)
    ws = fa.workspace(fa.fa_ooc_workspace_size(rows, cols, 8, 16), "cuda")
    s = fa.fa_shard_resolve(rows, cols, 8, 16, rec.nexit(2), rec.link(2), rec.node_dst(2),
                            rec.node_val(2), inflow, ws)
    assert s == fa.FA_ERR_CYCLE


def test_bad_code_reported_by_export_in_raster_numbering():
    codes = np.full((50, 70), 1, np.uint8)
    codes[40, 5] = 200
    rows, cols = codes.shape
    _, nby, nbx, pmax = fa.fa_shard_geometry(rows, cols, 16, 16)
    band = (2, 4)
    ra, rb = shard.band_rows(band, 16, rows)
    n = (band[1] - band[0]) * nbx
    rec = shard.Records(n, pmax)
    ws = fa.workspace(fa.fa_ooc_workspace_size(rows, cols, 16, 16), "cuda")
    d_status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device="cuda")
    s = fa.fa_shard_export(torch.from_numpy(np.ascontiguousarray(codes[ra:rb])), ra, rows, cols, 16,
                           16, band[0], band[1], rec.nexit(n), rec.link(n), rec.node_dst(n),
                           rec.node_val(n), ws, None, d_status)
    assert s == fa.FA_ERR_BAD_CODE
    s2, cnt, first = fa.fa_status_read(d_status)
    assert s2 == fa.FA_ERR_BAD_CODE and cnt == 1 and first == 40 * 70 + 5
