"""GPU parity of fa_accumulate_batched and the CUDA-graph batch plan.

A batch must give, for every (raster, field), what fa_accumulate gives for it
alone: bit-identical uint32 counts, and float32 sums within the parity
tolerance (the cross-tile fixed-point scale is set by the largest raster of
the batch, so the last bit of a float sum may differ), and the oracle's values.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
fa = pytest.importorskip("paper_1608_04431_gb300")
RTOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t):
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


def close(got, ref):
    got = got.astype(np.float64)
    return (np.abs(got - ref) <= RTOL * np.abs(ref)).all()


def make_items(shapes, seed, n_fields, masks=False):
    items, host = [], []
    for i, (R, C) in enumerate(shapes):
        codes = synth.dem_codes(R, C, seed + i)
        ws = [synth.uniform_weights((R, C), seed * 100 + i * 10 + k) if k % 2 == 0
              else synth.lognormal_weights((R, C), seed * 100 + i * 10 + k)
              for k in range(n_fields)]
        m = (synth.rng(seed + 50 + i).random((R, C)) < 0.01).astype(np.uint8) if masks else None
        item = {"codes": dev(codes)}
        if n_fields:
            item["weights"] = [dev(w) for w in ws]
        if masks:
            item["mask"] = dev(m)
        items.append(item)
        host.append((codes, ws, m))
    return items, host


@pytest.mark.parametrize("tile", [None, (32, 48), (16, 16)])
def test_batched_counts_equal_plain(oracle_mod, tile):
    shapes = [(257, 311), (100, 900), (1, 50), (640, 64), (333, 333)]
    items, host = make_items(shapes, 11, 0, masks=True)
    outs = fa.accumulate_batched(items, 0, tile=tile, check=True)
    torch.cuda.synchronize()
    for it, (codes, _, m), o in zip(items, host, outs):
        plain = u32(fa.accumulate(it["codes"], None, it["mask"], tile=tile))
        np.testing.assert_array_equal(u32(o[0]), plain)
        ref = oracle_mod.counts(codes, m)
        np.testing.assert_array_equal(u32(o[0]), ref.values.astype(np.uint32))


@pytest.mark.parametrize("tile", [None, (64, 32)])
def test_batched_fields_match_oracle(oracle_mod, tile):
    shapes = [(300, 410), (129, 777), (512, 96)]
    items, host = make_items(shapes, 21, 3)
    outs = fa.accumulate_batched(items, 3, tile=tile, check=True)
    torch.cuda.synchronize()
    for it, (codes, ws, _), o in zip(items, host, outs):
        for k in range(3):
            ref = oracle_mod.weighted(codes, ws[k]).values
            assert close(o[k].cpu().numpy(), ref)
            plain = fa.accumulate(it["codes"], it["weights"][k], tile=tile).cpu().numpy()
            assert close(o[k].cpu().numpy(), plain.astype(np.float64))


def test_batched_with_empty_raster_and_cycles(oracle_mod):
    cyc = synth.random_codes(60, 70, 5)
    items = [{"codes": dev(cyc)}, {"codes": torch.zeros((0, 9), dtype=torch.uint8, device="cuda")},
             {"codes": dev(synth.dem_codes(90, 80, 6))}]
    outs = fa.accumulate_batched(items, 0)
    st = fa.fa_status_read(None, fa.workspace(0, torch.device("cuda")))
    assert st[0] == fa.FA_ERR_CYCLE
    ref = oracle_mod.counts(cyc)
    ok = ref.state == 1
    np.testing.assert_array_equal(u32(outs[0][0])[ok], ref.values[ok].astype(np.uint32))
    assert outs[1][0].shape == (0, 9)
    np.testing.assert_array_equal(u32(outs[2][0]),
                                  oracle_mod.counts(synth.dem_codes(90, 80, 6)).values.astype(np.uint32))


def test_plan_replay(oracle_mod):
    shapes = [(200, 300), (150, 450), (64, 64)]
    items, host = make_items(shapes, 31, 2)
    plan = fa.BatchPlan(items, 2)
    a = [[t.clone() for t in o] for o in plan.run()]
    b = plan.run()
    torch.cuda.synchronize()
    assert plan.status_read()[0] == fa.FA_OK
    for oa, ob, (codes, ws, _) in zip(a, b, host):
        for k in range(2):
            assert oa[k].cpu().numpy().tobytes() == ob[k].cpu().numpy().tobytes()
            assert close(ob[k].cpu().numpy(), oracle_mod.weighted(codes, ws[k]).values)
    # the graph reads the buffers at replay time: new weights in place, new result
    new_w = synth.uniform_weights(shapes[0], 999)
    items[0]["weights"][0].copy_(dev(new_w))
    c = plan.run()
    torch.cuda.synchronize()
    assert close(c[0][0].cpu().numpy(), oracle_mod.weighted(host[0][0], new_w).values)
    plan.close()


@pytest.mark.slow
def test_batch_of_64_uneven_rasters_8_fields(oracle_mod):
    """64 rasters with sizes U{257..4096} x U{311..6000} and 8 fields (4 uniform
    [0,1), 4 lognormal sigma=1), one batch; every field of every raster against
    the same field run alone, and a sample of rasters against the oracle."""
    batch = synth.batch_rasters(64, 301, 300, 8)
    items = [{"codes": dev(c), "weights": [dev(w) for w in ws]} for c, ws in batch]
    plan = fa.BatchPlan(items, 8)
    outs = plan.run()
    torch.cuda.synchronize()
    assert plan.status_read()[0] == fa.FA_OK
    for i, (it, o) in enumerate(zip(items, outs)):
        for k in range(8):
            plain = fa.accumulate(it["codes"], it["weights"][k]).cpu().numpy().astype(np.float64)
            assert close(o[k].cpu().numpy(), plain), (i, k)
    for i in (0, 17, 63):
        codes, ws = batch[i]
        for k in (0, 7):
            assert close(outs[i][k].cpu().numpy(), oracle_mod.weighted(codes, ws[k]).values)
    plan.close()
