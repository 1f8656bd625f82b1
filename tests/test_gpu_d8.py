"""GPU parity of fa_d8_codes (D8 directions from elevations) with the oracle's
fa_oracle_d8: bit-exact codes, since both decide slopes in float32 with the
same correctly rounded operations."""
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


def gpu_d8(z, nd=None):
    zt = torch.from_numpy(np.ascontiguousarray(z, np.float32)).cuda()
    ndt = None if nd is None else torch.from_numpy(np.ascontiguousarray(nd, np.uint8)).cuda()
    return fa.d8_codes(zt, ndt).cpu().numpy()


@pytest.mark.parametrize("R,C", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 3), (4, 5), (37, 45),
                                 (257, 300), (130, 1029)])
def test_random_dems(oracle_mod, R, C):
    g = np.random.default_rng(R * 1000 + C)
    z = g.random((R, C), dtype=np.float32) * 100
    nd = (g.random((R, C)) < 0.05).astype(np.uint8)
    np.testing.assert_array_equal(gpu_d8(z), oracle_mod.d8(z))
    np.testing.assert_array_equal(gpu_d8(z, nd), oracle_mod.d8(z, nd))


def test_spectral_dem_and_integer_ties(oracle_mod):
    z = synth.spectral_dem(300, 420, 11)
    nd = synth.nodata_disk(300, 420, 12)
    np.testing.assert_array_equal(gpu_d8(z, nd), oracle_mod.d8(z, nd))
    zi = np.random.default_rng(5).integers(0, 4, size=(200, 211)).astype(np.float32)  # many ties
    np.testing.assert_array_equal(gpu_d8(zi), oracle_mod.d8(zi))


def test_pitched_views(oracle_mod):
    g = np.random.default_rng(9)
    big = torch.from_numpy(g.random((90, 140), dtype=np.float32)).cuda()
    z = big[3:80, 5:121]  # pitch 140, unaligned start
    out_big = torch.zeros((100, 150), dtype=torch.uint8, device="cuda")
    out = out_big[2:79, 1:117]
    assert fa.fa_d8_codes(z, None, out) == fa.FA_OK
    np.testing.assert_array_equal(out.cpu().numpy(), oracle_mod.d8(z.cpu().numpy()))


def test_directions_then_accumulation(oracle_mod):
    z = synth.spectral_dem(256, 300, 21)
    nd = synth.nodata_disk(256, 300, 22)
    zt, ndt = torch.from_numpy(z).cuda(), torch.from_numpy(nd.astype(np.uint8)).cuda()
    codes = fa.d8_codes(zt, ndt)
    acc = fa.accumulate(codes, check=False)
    ref_codes = oracle_mod.d8(z, nd)
    ref = oracle_mod.counts(ref_codes)
    ok = ref.state == 1
    got = acc.view(torch.int32).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint32))
