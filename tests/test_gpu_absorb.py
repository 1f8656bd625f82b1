"""GPU parity of fa_accumulate_absorb against the oracle's FP64 absorption.

Eq. 1 with one factor a(n) in [0, 1] per cell.  Weights and factors are
nonnegative here, so every term of a sum is nonnegative and the float32 result
must satisfy |gpu - ref| <= 2e-5 |ref|, the relative bound of the plain forms.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def status():
    st = fa.fa_status_read(None, fa.workspace(0, "cuda"))
    torch.cuda.synchronize()
    return st


def check(oracle_mod, codes, a, w=None, mask=None, tile=None):
    ref = oracle_mod.absorb(codes, a, w, mask)
    got = fa.absorb(dev(codes), dev(a), None if w is None else dev(w),
                    None if mask is None else dev(mask), tile=tile).cpu().numpy()
    st = status()
    ok = ref.state == 1
    bound = RTOL * np.abs(ref.values[ok])
    err = np.abs(got[ok].astype(np.float64) - ref.values[ok])
    assert (err <= bound).all(), f"max err/bound {np.max(err / np.maximum(bound, 1e-300))}"
    assert (got[ref.state == 0] == 0).all()
    if ref.n_cycle:
        assert st[0] == fa.FA_ERR_CYCLE
    elif ref.n_bad == 0:
        assert st[0] == fa.FA_OK, st
    return ref, got, st


@pytest.mark.parametrize("tile", [None, (1, 1), (2, 2), (1, 3), (3, 1)])
def test_hand_example(oracle_mod, tile):
    g = _golden.load("hand_3x3.txt")
    half = np.full((3, 3), 0.5, np.float32)
    got = fa.absorb(dev(g["codes"]), dev(half), tile=tile).cpu().numpy()
    np.testing.assert_array_equal(got, [[1, 1, 1], [1, 3.5, 1], [1, 3.75, 1]])
    got = fa.absorb(dev(g["codes"]), dev(half), dev(g["weights"]), tile=tile).cpu().numpy()
    np.testing.assert_array_equal(got, [[1, 2, 3], [4, 13, 6], [7, 22.5, 9]])


@pytest.mark.parametrize("a,C,tile", [(0.999, 5000, None), (0.5, 700, (1, 64)), (0.9, 333, (1, 7))])
def test_geometric_row(a, C, tile):
    codes = np.ones((1, C), np.uint8)
    got = fa.absorb(dev(codes), dev(np.full((1, C), a, np.float32)), tile=tile).cpu().numpy()[0]
    af = float(np.float32(a))
    want = (1.0 - af ** (np.arange(C) + 1.0)) / (1.0 - af)
    np.testing.assert_allclose(got, want, rtol=RTOL)


def test_special_factors(oracle_mod):
    R, C = 300, 257
    codes = synth.dem_codes(R, C, 141)
    w = synth.uniform_weights((R, C), 142)
    ones = np.ones((R, C), np.float32)
    # nothing absorbed: the plain float sums, and counts with unit weights
    a1 = fa.absorb(dev(codes), dev(ones), dev(w)).cpu().numpy()
    ref = oracle_mod.weighted(codes, w)
    np.testing.assert_allclose(a1, ref.values, rtol=RTOL)
    c1 = fa.absorb(dev(codes), dev(ones)).cpu().numpy()
    np.testing.assert_array_equal(c1, oracle_mod.counts(codes).values.astype(np.float32))
    # everything absorbed: each cell keeps its own weight
    a0 = fa.absorb(dev(codes), dev(np.zeros((R, C), np.float32)), dev(w)).cpu().numpy()
    valid = codes != 0
    np.testing.assert_array_equal(a0[valid], w[valid])
    assert (a0[~valid] == 0).all()


@pytest.mark.parametrize("seed,R,C,tile", [
    (1, 64, 64, None), (2, 100, 77, (8, 8)), (3, 129, 200, (16, 32)), (4, 33, 500, (4, 64)),
    (5, 300, 301, None), (6, 50, 50, (1, 1)), (7, 31, 17, (5, 3)), (8, 200, 90, (32, 96)),
])
def test_random_with_cycles(oracle_mod, seed, R, C, tile):
    codes = synth.random_codes(R, C, seed)
    mask = (synth.rng(seed + 50).random((R, C)) < 0.02).astype(np.uint8)
    a = synth.uniform_weights((R, C), seed + 70)
    w = synth.lognormal_weights((R, C), seed + 60)
    check(oracle_mod, codes, a, w, mask, tile)
    check(oracle_mod, codes, a, None, mask, tile)


@pytest.mark.parametrize("R,C,tile", [(1000, 1000, None), (777, 1301, (32, 128)), (513, 640, (64, 32))])
def test_dem(oracle_mod, R, C, tile):
    codes = synth.dem_codes(R, C, 151)
    a = synth.uniform_weights((R, C), 152, 0.9, 1.0)
    w = synth.uniform_weights((R, C), 153)
    check(oracle_mod, codes, a, w, None, tile)


def test_packed_codes_and_determinism(oracle_mod):
    R, C = 600, 901
    codes = synth.dem_codes(R, C, 161)
    a = synth.uniform_weights((R, C), 162, 0.5, 1.0)
    w = synth.uniform_weights((R, C), 163)
    x = fa.absorb(dev(codes), dev(a), dev(w))
    y = fa.absorb(dev(codes), dev(a), dev(w))
    pk = fa.pack_codes(dev(codes))
    z = fa.absorb(pk, dev(a), dev(w))
    torch.cuda.synchronize()
    assert torch.equal(x, y) and torch.equal(x, z)


@pytest.mark.parametrize("codes,tile", [([[1, 5]], None), ([[1, 7], [3, 5]], (2, 2)),
                                        ([[1, 7], [3, 5]], (1, 1)), ([[1, 1, 6], [9, 3, 5]], None)])
def test_cycles_flagged(oracle_mod, codes, tile):
    # in-tile cycles of length 2 and 4 (pointer doubling comes back to the
    # cell itself on those), a cross-tile 4-cycle, and a 3-cycle fed by a cell
    codes = np.array(codes, np.uint8)
    a = np.full(codes.shape, 0.75, np.float32)
    ref = oracle_mod.absorb(codes, a)
    assert ref.n_cycle > 0
    got = fa.absorb(dev(codes), dev(a), tile=tile).cpu().numpy()
    st, count, _ = status()
    assert st == fa.FA_ERR_CYCLE and count > 0
    ok = ref.state == 1
    np.testing.assert_allclose(got[ok], ref.values[ok], rtol=RTOL)


def test_bad_factors_flagged():
    R, C = 40, 50
    codes = synth.dem_codes(R, C, 171)
    r, c = (int(v) for v in np.argwhere(codes[7:] != 0)[0] + [7, 0])  # a valid cell
    for bad in (1.5, -0.25, float("nan")):
        a = np.full((R, C), 0.9, np.float32)
        a[r, c] = bad
        fa.absorb(dev(codes), dev(a))
        st, _, first = status()
        assert st == fa.FA_ERR_NONFINITE
        assert first == r * C + c


@pytest.mark.slow
def test_dem_16384(oracle_mod):
    R = C = 16384
    codes = synth.dem_codes(R, C, 201)
    a = synth.uniform_weights((R, C), 204, 0.9, 1.0)
    w = synth.uniform_weights((R, C), 202)
    check(oracle_mod, codes, a, w)
