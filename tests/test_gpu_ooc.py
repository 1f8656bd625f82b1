"""GPU parity of fa_accumulate_ooc (codes and counts in host memory, solved
block by block) against the CPU oracle.

Counts are integers: every exact cell must match the oracle bit for bit,
NoData cells read 0, and cells on cycles (unspecified) are skipped while the
status reports the cycle.  Small forced outer blocks make every path cross
many block borders, so the block-level perimeter graph (Section 3.2) and the
inflow walks (Algorithm 3) carry most of the result.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

fa = pytest.importorskip("paper_1608_04431_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(codes, block, tile=None, check=False):
    """Returns (uint64 counts, status)."""
    c = torch.from_numpy(np.ascontiguousarray(codes))
    out = torch.empty(codes.shape, dtype=torch.int64)
    opts = fa.options(tile)
    bh, bw = block
    n = fa.fa_ooc_workspace_size(codes.shape[0], codes.shape[1], bh, bw, opts)
    assert n > 0
    ws = fa.workspace(n, "cuda")
    st = fa.fa_accumulate_ooc(c, out, bh, bw, ws, opts)
    return out.numpy().view(np.uint64), st


def check(oracle_mod, codes, block, tile=None, mask_free=True):
    ref = oracle_mod.counts(codes)
    got, st = run(codes, block, tile)
    ok = ref.state == 1
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint64))
    assert (got[ref.state == 0] == 0).all()
    if ref.n_cycle == 0 and ref.n_bad == 0:
        assert st == fa.FA_OK, st
    return ref, got, st


@pytest.mark.parametrize("block,tile", [
    ((40, 56), (16, 16)), ((17, 23), None), ((300, 410), None), ((1, 64), (8, 8)),
    ((64, 1), (8, 8)), ((128, 200), (32, 64)), ((299, 409), (64, 64)), ((2, 2), (1, 1)),
])
def test_dem_blocks(oracle_mod, block, tile):
    codes = synth.dem_codes(300, 410, 401)
    check(oracle_mod, codes, block, tile)


@pytest.mark.parametrize("R,C,block", [(37, 41, (7, 9)), (64, 64, (8, 8)), (20, 101, (3, 10)),
                                       (1, 500, (1, 33)), (500, 1, (33, 1))])
def test_serpentine_closed_form(R, C, block):
    """One path through every cell: the cell k steps along it counts k + 1.
    The path leaves and re-enters blocks on every row."""
    codes = synth.serpentine_codes(R, C)
    got, st = run(codes, block)
    assert st == fa.FA_OK
    np.testing.assert_array_equal(got, (synth.serpentine_index(R, C) + 1).astype(np.uint64))


@pytest.mark.parametrize("seed,R,C,block,tile", [
    (411, 200, 333, (50, 60), None), (412, 400, 128, (33, 128), (32, 32)),
    (413, 97, 1000, (97, 77), (16, 128)),
])
def test_acyclic_random(oracle_mod, seed, R, C, block, tile):
    codes = synth.acyclic_random_codes(R, C, seed)
    ref, _, st = check(oracle_mod, codes, block, tile)
    assert ref.n_cycle == 0 and st == fa.FA_OK


@pytest.mark.parametrize("seed,R,C,block", [(421, 100, 77, (20, 20)), (422, 129, 200, (64, 33)),
                                            (423, 50, 50, (7, 5))])
def test_random_with_cycles(oracle_mod, seed, R, C, block):
    codes = synth.random_codes(R, C, seed)
    ref, _, st = check(oracle_mod, codes, block, (16, 16))
    if ref.n_cycle:
        assert st == fa.FA_ERR_CYCLE


def test_cycle_across_blocks_reported():
    """A 2 x 2 cycle split over four 1 x 1 blocks is seen only by the
    block-level resolve."""
    four = np.array([[1, 7], [3, 5]], np.uint8)
    _, st = run(four, (1, 1))
    assert st == fa.FA_ERR_CYCLE


def test_bad_code_index_in_raster_numbering():
    codes = np.full((50, 70), 1, np.uint8)
    codes[10, 20] = 77
    codes[40, 5] = 200
    c = torch.from_numpy(codes)
    out = torch.empty(codes.shape, dtype=torch.int64)
    ws = fa.workspace(fa.fa_ooc_workspace_size(50, 70, 16, 16), "cuda")
    d_status = torch.zeros(fa.FA_STATUS_WORDS, dtype=torch.int32, device="cuda")
    st = fa.fa_accumulate_ooc(c, out, 16, 16, ws, None, d_status)
    assert st == fa.FA_ERR_BAD_CODE
    st2, cnt, first = fa.fa_status_read(d_status)
    assert st2 == fa.FA_ERR_BAD_CODE and cnt == 2 and first == 10 * 70 + 20
    got = out.numpy()
    assert got[10, 20] == 0 and got[10, 21] == 1 and got[10, 19] == 20


def test_pitched_host_views(oracle_mod):
    codes = synth.dem_codes(150, 170, 431)
    big = np.zeros((150, 203), np.uint8)
    big[:, 5:175] = codes
    c = torch.from_numpy(big)[:, 5:175]
    out_big = torch.full((150, 190), -7, dtype=torch.int64)
    out = out_big[:, 3:173]
    ws = fa.workspace(fa.fa_ooc_workspace_size(150, 170, 64, 48), "cuda")
    st = fa.fa_accumulate_ooc(c, out, 64, 48, ws)
    assert st == fa.FA_OK
    ref = oracle_mod.counts(codes)
    got = out.numpy().view(np.uint64)
    ok = ref.state == 1
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint64))
    assert (out_big[:, :3] == -7).all() and (out_big[:, 173:] == -7).all()


def test_pinned_matches_device_path():
    """Pinned host buffers (copies overlap the block solves) and the default
    block shape give the in-core result."""
    codes = synth.dem_codes(1000, 1300, 441)
    c = torch.from_numpy(codes).pin_memory()
    out = torch.empty(codes.shape, dtype=torch.int64).pin_memory()
    fa.accumulate_ooc(c, block=(256, 384), out=out)
    dev = fa.accumulate(torch.from_numpy(codes).cuda(), check=True)
    d = dev.view(torch.int32).cpu().numpy().view(np.uint32).astype(np.uint64)
    np.testing.assert_array_equal(out.numpy().view(np.uint64), d)
    whole = fa.accumulate_ooc(codes)
    np.testing.assert_array_equal(whole.numpy().view(np.uint64), d)


def test_empty_and_invalid():
    e = np.zeros((0, 5), np.uint8)
    got, st = run(e, (4, 4))
    assert st == fa.FA_OK and got.size == 0
    assert fa.fa_ooc_workspace_size(40000, 40000, 20000, 20000) == 0  # perimeter > 65534 slots
    assert fa.fa_ooc_workspace_size(40000, 40000, 16384, 16384) > 0
    # a block longer than the raster is cut to it
    assert fa.fa_ooc_workspace_size(100, 100, 30000, 30000) == fa.fa_ooc_workspace_size(100, 100)
    nib = fa.options(None, 0, fa.FA_CODES_NIBBLE)
    assert fa.fa_ooc_workspace_size(100, 100, 10, 10, nib) == 0
    with pytest.raises(fa.FlowAccError):
        fa.accumulate_ooc(np.zeros((10, 10), np.uint8), block=(-1, 5))
