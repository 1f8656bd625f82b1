"""GPU parity of fa_accumulate (through the C ABI) against the CPU oracle.

Counts must match bit for bit on every exact cell; float32 weighted sums must
satisfy |gpu - ref| <= 2e-5 * |ref| (weights >= 0, so ref = 0 forces gpu = 0).
Cells on cycles are unspecified and skipped; the status block must flag them.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _golden

pytestmark = pytest.mark.gpu

RTOL = 2e-5

fa = pytest.importorskip("paper_1608_04431_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def to_np(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def run(codes, weights=None, mask=None, tile=None, out_dtype=None):
    """Returns (values, (status, count, first_index))."""
    c = dev(codes)
    w = None if weights is None else dev(weights)
    m = None if mask is None else dev(mask)
    out = fa.accumulate(c, w, m, out_dtype=out_dtype, tile=tile)
    st = fa.fa_status_read(None, fa.workspace(0, c.device))
    torch.cuda.synchronize()
    return to_np(out), st


def check_counts(oracle_mod, codes, mask=None, tile=None):
    ref = oracle_mod.counts(codes, mask)
    got, st = run(codes, None, mask, tile)
    ok = ref.state == 1
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint32))
    assert (got[ref.state == 0] == 0).all()
    if ref.n_cycle == 0 and ref.n_bad == 0:
        assert st[0] in (fa.FA_OK, fa.FA_WARN_OVERFLOW), st
    return ref, got, st


def check_weighted(oracle_mod, codes, w, mask=None, tile=None):
    ref = oracle_mod.weighted(codes, w, mask)
    got, st = run(codes, w, mask, tile)
    ok = ref.state == 1
    err = np.abs(got[ok].astype(np.float64) - ref.values[ok])
    bound = RTOL * np.abs(ref.values[ok])
    assert (err <= bound).all(), f"max rel err {np.max(err / np.maximum(np.abs(ref.values[ok]), 1e-300))}"
    assert (got[ref.state == 0] == 0).all()
    return ref, got, st


# ---------------------------------------------------------------------------
# hand-worked examples
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", _golden.names())
@pytest.mark.parametrize("tile", [None, (1, 1), (2, 2), (1, 3), (3, 1)])
def test_golden(oracle_mod, name, tile):
    fx = _golden.load(name)
    got, st = run(fx["codes"], None, fx.get("mask"), tile)
    state = fx.get("state")
    exact = (state == 1) if state is not None else np.ones(got.shape, bool)
    if "counts" in fx:
        np.testing.assert_array_equal(got[exact], fx["counts"][exact].astype(np.uint32))
    if "weighted" in fx:
        gw, _ = run(fx["codes"], fx["weights"], fx.get("mask"), tile)
        np.testing.assert_array_equal(gw, fx["weighted"].astype(np.float32))
    if fx.get("n_bad"):
        assert st[0] == fa.FA_ERR_BAD_CODE
    if fx.get("n_cycle"):
        assert st[0] == fa.FA_ERR_CYCLE


# ---------------------------------------------------------------------------
# closed forms, edge shapes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("R,C", [(1, 1), (1, 200), (200, 1), (65, 64), (64, 65), (130, 257)])
def test_closed_forms(R, C):
    rr, cc = np.indices((R, C))
    for code, expect in ((1, cc + 1), (5, C - cc), (7, rr + 1), (3, R - rr),
                         (8, np.minimum(rr, cc) + 1)):
        got, st = run(np.full((R, C), code, np.uint8))
        np.testing.assert_array_equal(got, expect.astype(np.uint32))
        assert st[0] == fa.FA_OK


def test_empty_raster():
    for R, C in ((0, 0), (0, 5), (7, 0)):
        c = torch.zeros((R, C), dtype=torch.uint8, device="cuda")
        out = fa.accumulate(c)
        st = fa.fa_status_read(None, fa.workspace(0, c.device))
        assert out.shape == (R, C) and st[0] == fa.FA_OK


@pytest.mark.parametrize("R,C,tile", [(257, 311, None), (300, 300, (16, 16)), (1000, 37, (64, 8)),
                                      (64, 64, (64, 64)), (129, 129, (96, 80))])
def test_serpentine(oracle_mod, R, C, tile):
    codes = synth.serpentine_codes(R, C)
    k = synth.serpentine_index(R, C)
    got, st = run(codes, tile=tile)
    np.testing.assert_array_equal(got, (k + 1).astype(np.uint32))
    w = synth.uniform_weights((R, C), 3)
    check_weighted(oracle_mod, codes, w, tile=tile)


# ---------------------------------------------------------------------------
# random rasters: NoData, NoFlow, masks, cycles, ragged tiles
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,R,C,tile", [
    (1, 64, 64, None), (2, 100, 77, (8, 8)), (3, 129, 200, (16, 32)), (4, 33, 500, (4, 64)),
    (5, 300, 301, None), (6, 50, 50, (1, 1)), (7, 31, 17, (5, 3)), (8, 200, 90, (96, 80)),
])
def test_random_with_cycles(oracle_mod, seed, R, C, tile):
    codes = synth.random_codes(R, C, seed)
    mask = (synth.rng(seed + 50).random((R, C)) < 0.02).astype(np.uint8)
    ref, got, st = check_counts(oracle_mod, codes, mask, tile)
    if ref.n_cycle:
        assert st[0] == fa.FA_ERR_CYCLE
    w = synth.lognormal_weights((R, C), seed + 60)
    check_weighted(oracle_mod, codes, w, mask, tile)


@pytest.mark.parametrize("seed,R,C,tile", [(11, 200, 333, None), (12, 400, 128, (32, 32)),
                                           (13, 97, 1000, (16, 128))])
def test_acyclic_random(oracle_mod, seed, R, C, tile):
    codes = synth.acyclic_random_codes(R, C, seed)
    ref, got, st = check_counts(oracle_mod, codes, None, tile)
    assert ref.n_cycle == 0 and st[0] == fa.FA_OK
    w = synth.uniform_weights((R, C), seed + 1)
    check_weighted(oracle_mod, codes, w, None, tile)


def test_tile_shape_invariance():
    """Integer results are identical for every tile shape (the paper's own
    correctness check compares the tiled run with the untiled one)."""
    codes = synth.dem_codes(257, 311, 99)
    base, _ = run(codes, tile=(127, 63))
    for tile in [(1, 1), (2, 5), (8, 8), (16, 64), (64, 64), (64, 128), (32, 256), (1, 2048),
                 (512, 1), (256, 32)]:
        got, st = run(codes, tile=tile)
        np.testing.assert_array_equal(got, base, err_msg=str(tile))


def test_unsupported_tile_shapes_rejected():
    c = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    w = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(fa.FlowAccError):
        fa.accumulate(c, tile=(4096, 1))  # 16-bit cell index space exceeded
    with pytest.raises(fa.FlowAccError):
        fa.accumulate(c, tile=(257, 63))  # 257 x 63 cells > 8192
    with pytest.raises(fa.FlowAccError):
        fa.accumulate(c, w, tile=(128, 128))  # 16384 cells > 8192


def test_bad_code_status():
    codes = np.full((50, 70), 1, np.uint8)
    codes[10, 20] = 77
    codes[40, 5] = 200
    got, (st, cnt, first) = run(codes)
    assert st == fa.FA_ERR_BAD_CODE and cnt == 2 and first == 10 * 70 + 20
    assert got[10, 20] == 0 and got[10, 21] == 1 and got[10, 19] == 20


def test_cycle_status_cross_tile():
    four = np.array([[1, 7], [3, 5]], np.uint8)
    for tile in [(1, 1), (2, 2), (1, 2)]:
        _, (st, cnt, _) = run(four, tile=tile)
        assert st == fa.FA_ERR_CYCLE


def test_determinism_f32():
    codes = synth.dem_codes(600, 700, 21)
    w = synth.lognormal_weights(codes.shape, 22)
    a, _ = run(codes, w)
    b, _ = run(codes, w)
    assert a.tobytes() == b.tobytes()


def test_pitched_views(oracle_mod):
    codes = synth.dem_codes(150, 170, 31)
    w = synth.uniform_weights(codes.shape, 32)
    big_c = torch.zeros((150, 200), dtype=torch.uint8, device="cuda")
    big_c[:, :170] = dev(codes)
    big_w = torch.zeros((150, 256), dtype=torch.float32, device="cuda")
    big_w[:, :170] = dev(w)
    big_o = torch.zeros((150, 180), dtype=torch.float32, device="cuda")
    fa.accumulate(big_c[:, :170], big_w[:, :170], out=big_o[:, :170])
    torch.cuda.synchronize()
    ref = oracle_mod.weighted(codes, w)
    got = big_o[:, :170].cpu().numpy()
    np.testing.assert_allclose(got, ref.values, rtol=RTOL, atol=0)
    assert (big_o[:, 170:] == 0).all()


def test_unit_weights_f32_output(oracle_mod):
    codes = synth.dem_codes(300, 200, 41)
    ref = oracle_mod.counts(codes)
    got, _ = run(codes, None, None, None, out_dtype=fa.FA_OUT_F32)
    np.testing.assert_array_equal(got, ref.values.astype(np.float32))


# ---------------------------------------------------------------------------
# workload shapes: 500x500 DEM with a NoData disk; 16384^2 DEM; 8192^2 serpentine
# ---------------------------------------------------------------------------
def test_dem_500(oracle_mod):
    codes = synth.dem_codes(500, 500, 101, nodata_radius=28)
    ref, got, st = check_counts(oracle_mod, codes)
    assert ref.n_cycle == 0 and st[0] == fa.FA_OK
    bad, _ = oracle_mod.residual_u32(codes, got)
    assert bad == 0


@pytest.mark.slow
def test_dem_16384_counts_and_weights(oracle_mod):
    codes = synth.dem_codes(16384, 16384, 201)
    ref, got, st = check_counts(oracle_mod, codes)
    assert st[0] == fa.FA_OK
    del ref, got
    w = synth.uniform_weights(codes.shape, 202)
    check_weighted(oracle_mod, codes, w)


@pytest.mark.slow
def test_serpentine_8192():
    R = C = 8192
    codes = synth.serpentine_codes(R, C)
    got, st = run(codes)
    k = synth.serpentine_index(R, C)
    np.testing.assert_array_equal(got, (k + 1).astype(np.uint32))
    assert st[0] == fa.FA_OK


@pytest.mark.parametrize("R,C,pitch,tile", [(1024, 2048, 2048, None), (1000, 1000, 1008, (64, 64)),
                                            (333, 517, 528, (32, 48)), (129, 260, 272, (16, 16)),
                                            (700, 300, 304, (96, 80))])
def test_tma_and_plain_loads_agree(oracle_mod, R, C, pitch, tile):
    """The TMA-staged and the plain-load tile paths give identical results
    (rasters with 16-byte aligned pitch and tile widths that are multiples of
    16 take the TMA path by default)."""
    codes = synth.dem_codes(R, C, 71)
    big = torch.zeros((R, pitch), dtype=torch.uint8, device="cuda")
    big[:, :C] = dev(codes)
    view = big[:, :C]
    a = fa.accumulate(view, tile=tile)
    b = fa.accumulate(view, tile=tile, flags=fa.FA_OPT_NO_TMA)
    torch.cuda.synchronize()
    ga, gb = to_np(a), to_np(b)
    np.testing.assert_array_equal(ga, gb)
    ref = oracle_mod.counts(codes)
    np.testing.assert_array_equal(ga, ref.values.astype(np.uint32))
    w = synth.uniform_weights((R, C), 72)
    bw = torch.zeros((R, pitch), dtype=torch.float32, device="cuda")
    bw[:, :C] = dev(w)
    fw = fa.accumulate(view, bw[:, :C], tile=tile)
    fw2 = fa.accumulate(view, bw[:, :C], tile=tile, flags=fa.FA_OPT_NO_TMA)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fw.cpu().numpy(), fw2.cpu().numpy())
