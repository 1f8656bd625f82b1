"""GPU checks of the tile-shape autotuner: it picks one of its candidates,
leaves that shape's (correct) result in the output, and the shapes it picks
give the same counts as the default tile."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
fa = pytest.importorskip("paper_1608_04431_gb300")
CANDIDATES = {(64, 64), (64, 128), (128, 64), (96, 64), (64, 96), (32, 128), (128, 32), (48, 64),
              (32, 64), (64, 32), (32, 256), (48, 128)}
RTOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


def test_autotune_counts_result_and_choice(oracle_mod):
    codes = synth.dem_codes(700, 900, 61)
    cd = torch.from_numpy(codes).cuda()
    out = torch.full(codes.shape, 7, dtype=torch.uint32, device="cuda")
    ws = torch.empty(fa.fa_autotune_workspace_size(*codes.shape), dtype=torch.uint8, device="cuda")
    st, best = fa.fa_autotune(cd, None, None, out, fa.FA_OUT_U32, ws)
    assert st == fa.FA_OK
    assert (best.tile_h, best.tile_w) in CANDIDATES
    ref = oracle_mod.counts(codes).values.astype(np.uint32)
    np.testing.assert_array_equal(u32(out), ref)
    again = fa.accumulate(cd, tile=(best.tile_h, best.tile_w))
    np.testing.assert_array_equal(u32(again), ref)


def test_autotune_weighted_and_auto_tile(oracle_mod):
    codes = synth.dem_codes(600, 640, 62)
    w = synth.lognormal_weights(codes.shape, 63)
    cd, wd = torch.from_numpy(codes).cuda(), torch.from_numpy(w).cuda()
    got = fa.accumulate(cd, wd, tile="auto").cpu().numpy().astype(np.float64)
    ref = oracle_mod.weighted(codes, w).values
    assert (np.abs(got - ref) <= RTOL * np.abs(ref)).all()
    tile = fa.autotune(cd, wd)  # cached: the same answer without re-timing
    assert tuple(tile) in CANDIDATES and fa.autotune(cd, wd) == tile


def test_autotune_batched_plan(oracle_mod):
    shapes = [(300, 420), (257, 311), (520, 200)]
    batch = [(synth.dem_codes(r, c, 70 + i), [synth.uniform_weights((r, c), 80 + i)])
             for i, (r, c) in enumerate(shapes)]
    items = [{"codes": torch.from_numpy(c).cuda(), "weights": [torch.from_numpy(w[0]).cuda()]}
             for c, w in batch]
    plan = fa.BatchPlan(items, 1, tile="auto")
    assert tuple(plan.tile) in CANDIDATES
    outs = plan.run()
    torch.cuda.synchronize()
    assert plan.status_read()[0] == fa.FA_OK
    for (c, w), o in zip(batch, outs):
        ref = oracle_mod.weighted(c, w[0]).values
        got = o[0].cpu().numpy().astype(np.float64)
        assert (np.abs(got - ref) <= RTOL * np.abs(ref)).all()
    plan.close()
