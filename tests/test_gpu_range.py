"""Float32 weights whose magnitudes differ by many powers of two, against the
FP64 oracle.

The paper lets each cell carry "any other user-specified weighting value"
(Section 3.1).  Inside a tile the library adds a cell's inflows in a fixed
neighbour order as compensated float pairs (about 48 bits), so a small weight
keeps its relative precision next to a large one in the same tile; across
tiles the sums are 128-bit fixed point scaled to cells * max|w|, which
resolves 2^-(124 - ceil(log2(cells * max|w|))) absolutely.  The bound checked
here is the plain one, |gpu - ref| <= 2e-5 |ref| for weights of one sign (a
cell whose true sum is 0 must read exactly 0), and for mixed signs
|gpu - ref| <= 2e-5 * (the same sum over |w|), the adjoint's bound.
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


def run(codes, w, tile):
    c = torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
    got = fa.accumulate(c, wt, tile=tile, check=True)
    return got.cpu().numpy().astype(np.float64)


def check_one_sign(oracle_mod, codes, w, tile):
    ref = oracle_mod.weighted(codes, w)
    got = run(codes, w, tile)
    ok = ref.state == 1
    err = np.abs(got[ok] - ref.values[ok])
    bound = RTOL * np.abs(ref.values[ok])
    assert (err <= bound).all(), f"max err/|ref| {np.max(err / np.maximum(np.abs(ref.values[ok]), 1e-300))}"
    assert (got[ref.state == 0] == 0).all()
    return ref, got


def log_uniform(shape, seed, lo_exp, hi_exp):
    """|w| = 2^u with u uniform in [lo_exp, hi_exp)."""
    g = synth.rng(seed)
    return np.exp2(g.uniform(lo_exp, hi_exp, size=shape)).astype(np.float32)


@pytest.mark.parametrize("tile", [(32, 64), (64, 64), (16, 16)])
def test_weights_from_2_to_minus_60_up_to_1(oracle_mod, tile):
    codes = synth.dem_codes(300, 410, 71)
    w = log_uniform(codes.shape, 72, -60.0, 0.0)
    check_one_sign(oracle_mod, codes, w, tile)


@pytest.mark.parametrize("tile", [(32, 64), (64, 64)])
def test_tiny_weights_next_to_one_huge_weight(oracle_mod, tile):
    """Every tile has one weight of 1 and the rest 2^-50 or 2^-40: the
    cells upstream of the big one only see tiny weights, and must keep them
    to the relative bound."""
    codes = synth.dem_codes(256, 320, 73)
    w = np.where(synth.rng(74).random(codes.shape) < 0.5, np.float32(2.0 ** -50),
                 np.float32(2.0 ** -40)).astype(np.float32)
    th, tw = tile
    w[th // 2::th, tw // 2::tw] = 1.0
    check_one_sign(oracle_mod, codes, w, tile)


def test_zero_weights_give_exact_zeros(oracle_mod):
    """Cells whose whole upstream area weighs 0 must read exactly 0, also
    where the rest of the tile carries large weights."""
    codes = synth.dem_codes(200, 260, 75)
    w = np.zeros(codes.shape, np.float32)
    g = synth.rng(76)
    hot = g.random(codes.shape) < 0.3
    w[hot] = g.random(int(hot.sum())).astype(np.float32) * np.float32(1e6)
    ref, got = check_one_sign(oracle_mod, codes, w, (32, 64))
    zero = (ref.state == 1) & (ref.values == 0.0)
    assert zero.any()
    assert (got[zero] == 0.0).all()


def test_single_tile_keeps_relative_precision_far_below_the_maximum(oracle_mod):
    """Inside one tile nothing is fixed point: weights 2^-120 .. 1 in a
    raster that is a single 64 x 128 tile stay within the relative bound."""
    codes = synth.dem_codes(64, 128, 77)
    w = log_uniform(codes.shape, 78, -120.0, 0.0)
    check_one_sign(oracle_mod, codes, w, (64, 128))


@pytest.mark.parametrize("tile", [(32, 64), (64, 64)])
def test_mixed_signs_against_the_absolute_sum(oracle_mod, tile):
    """Negative weights are allowed (the operator is linear); the error is
    measured against the sum of |w| along the same upstream area."""
    codes = synth.dem_codes(300, 333, 79)
    g = synth.rng(80)
    w = (log_uniform(codes.shape, 81, -30.0, 0.0) *
         np.where(g.random(codes.shape) < 0.5, -1.0, 1.0)).astype(np.float32)
    ref = oracle_mod.weighted(codes, w)
    absref = oracle_mod.weighted(codes, np.abs(w))
    got = run(codes, w, tile)
    ok = ref.state == 1
    err = np.abs(got[ok] - ref.values[ok])
    assert (err <= RTOL * absref.values[ok]).all()


def test_results_are_bitwise_reproducible():
    """Fixed summation order: two runs give the same bits."""
    codes = synth.dem_codes(300, 300, 82)
    w = log_uniform(codes.shape, 83, -60.0, 10.0)
    a = run(codes, w, (32, 64))
    b = run(codes, w, (32, 64))
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
