"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: they use hand-worked examples
(tests/golden), closed forms, conservation of flow, a brute-force path walker
written here in plain Python, the structure of cycles, and for the adjoint the
dot-product identity and central finite differences.
"""
import numpy as np
import pytest

import synth
from tests import _golden

# code -> (dr, dc), written out from the encoding: E NE N NW W SW S SE
STEP = {1: (0, 1), 2: (-1, 1), 3: (-1, 0), 4: (-1, -1), 5: (0, -1), 6: (1, -1), 7: (1, 0),
        8: (1, 1)}


def _valid(codes, mask, r, c):
    R, C = codes.shape
    if not (0 <= r < R and 0 <= c < C):
        return False
    k = int(codes[r, c])
    if k == 0 or k > 9:
        return False
    return mask is None or mask[r, c] == 0


def _down(codes, mask, r, c):
    k = int(codes[r, c])
    if k not in STEP:
        return None
    rr, cc = r + STEP[k][0], c + STEP[k][1]
    return (rr, cc) if _valid(codes, mask, rr, cc) else None


def py_walk(codes, w=None, mask=None):
    """Definition of flow accumulation by path walking (pure Python): each
    valid cell adds its weight to every cell on its downstream path.  Returns
    (values, on_cycle) where on_cycle marks cells whose walk never ends."""
    R, C = codes.shape
    out = np.zeros((R, C))
    cyc = np.zeros((R, C), dtype=bool)
    for r in range(R):
        for c in range(C):
            if not _valid(codes, mask, r, c):
                continue
            wy = 1.0 if w is None else float(w[r, c])
            cur, seen = (r, c), set()
            while cur is not None and cur not in seen:
                seen.add(cur)
                out[cur] += wy
                cur = _down(codes, mask, *cur)
            if cur is not None:  # re-entered a visited cell: the cycle
                s = cur
                while True:
                    cyc[s] = True
                    s = _down(codes, mask, *s)
                    if s == cur:
                        break
    return out, cyc


def py_path_sum(codes, g, mask=None):
    """sum of g over each valid cell's downstream path (itself included)."""
    R, C = codes.shape
    lam = np.zeros((R, C))
    for r in range(R):
        for c in range(C):
            if not _valid(codes, mask, r, c):
                continue
            cur, n = (r, c), 0
            while cur is not None and n <= R * C:
                lam[r, c] += float(g[cur])
                cur = _down(codes, mask, *cur)
                n += 1
    return lam


# ---------------------------------------------------------------------------
# hand-worked examples
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", _golden.names())
def test_golden(oracle_mod, name):
    fx = _golden.load(name)
    codes = fx["codes"]
    mask = fx.get("mask")
    res = oracle_mod.counts(codes, mask)
    state = fx.get("state")
    exact = (state == 1) if state is not None else np.ones(codes.shape, bool)
    if "counts" in fx:
        np.testing.assert_array_equal(res.values[exact].astype(np.int64), fx["counts"][exact])
    if state is not None:
        np.testing.assert_array_equal(res.state, state)
    if "n_cycle" in fx:
        assert res.n_cycle == fx["n_cycle"]
    if "n_bad" in fx:
        assert res.n_bad == fx["n_bad"]
    if "weighted" in fx:
        rw = oracle_mod.weighted(codes, fx["weights"], mask)
        np.testing.assert_array_equal(rw.values, fx["weighted"])
    if "adjoint" in fx:
        ra = oracle_mod.adjoint(codes, fx["g"], mask)
        np.testing.assert_array_equal(ra.values, fx["adjoint"])


def test_nodata_outputs_zero(oracle_mod):
    fx = _golden.load("hand_5x5.txt")
    res = oracle_mod.counts(fx["codes"])
    assert res.values[2, 2] == 0 and res.state[2, 2] == 0


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("R,C", [(1, 1), (1, 7), (5, 1), (13, 29)])
def test_all_east_west_north_south(oracle_mod, R, C):
    rr, cc = np.indices((R, C))
    for code, expect in ((1, cc + 1), (5, C - cc), (7, rr + 1), (3, R - rr)):
        res = oracle_mod.counts(np.full((R, C), code, np.uint8))
        np.testing.assert_array_equal(res.values, expect.astype(np.uint64))


@pytest.mark.parametrize("R,C", [(6, 6), (4, 9), (9, 4)])
def test_all_diagonal(oracle_mod, R, C):
    rr, cc = np.indices((R, C))
    # SE: each cell's upslope cells are (r-t, c-t), t >= 0
    res = oracle_mod.counts(np.full((R, C), 8, np.uint8))
    np.testing.assert_array_equal(res.values, (np.minimum(rr, cc) + 1).astype(np.uint64))
    # NW: mirrored
    res = oracle_mod.counts(np.full((R, C), 4, np.uint8))
    np.testing.assert_array_equal(res.values,
                                  (np.minimum(R - 1 - rr, C - 1 - cc) + 1).astype(np.uint64))


@pytest.mark.parametrize("R,C", [(1, 9), (2, 5), (7, 11), (64, 33)])
def test_serpentine(oracle_mod, R, C):
    codes = synth.serpentine_codes(R, C)
    k = synth.serpentine_index(R, C)
    res = oracle_mod.counts(codes)
    np.testing.assert_array_equal(res.values, (k + 1).astype(np.uint64))
    w = synth.uniform_weights((R, C), 7)
    order = np.argsort(k.ravel())
    prefix = np.cumsum(w.ravel()[order].astype(np.float64))
    expect = np.empty(R * C)
    expect[order] = prefix
    rw = oracle_mod.weighted(codes, w)
    np.testing.assert_allclose(rw.values.ravel(), expect, rtol=1e-13)


# ---------------------------------------------------------------------------
# conservation and brute force
# ---------------------------------------------------------------------------
def _terminal(codes, mask=None):
    R, C = codes.shape
    t = np.zeros((R, C), dtype=bool)
    for r in range(R):
        for c in range(C):
            t[r, c] = _valid(codes, mask, r, c) and _down(codes, mask, r, c) is None
    return t


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_conservation(oracle_mod, seed):
    codes = synth.acyclic_random_codes(37, 23, seed)
    w = synth.lognormal_weights(codes.shape, seed + 10)
    valid = (codes > 0) & (codes <= 9)
    term = _terminal(codes)
    rc = oracle_mod.counts(codes)
    assert rc.n_cycle == 0
    assert int(rc.values[term].sum()) == int(valid.sum())
    rw = oracle_mod.weighted(codes, w)
    assert rw.values[term].sum() == pytest.approx(w[valid].astype(np.float64).sum(), rel=1e-12)


def test_conservation_dem(oracle_mod):
    codes = synth.dem_codes(120, 150, 11)
    valid = (codes > 0) & (codes <= 9)
    rc = oracle_mod.counts(codes)
    assert rc.n_cycle == 0 and rc.n_bad == 0
    assert int(rc.values[_terminal(codes)].sum()) == int(valid.sum())


@pytest.mark.parametrize("seed,R,C", [(5, 1, 40), (6, 17, 19), (7, 64, 64), (8, 31, 57)])
def test_bruteforce_random_with_cycles(oracle_mod, seed, R, C):
    codes = synth.random_codes(R, C, seed)
    mask = (synth.rng(seed + 99).random((R, C)) < 0.03).astype(np.uint8)
    w = synth.uniform_weights((R, C), seed + 1)
    expect, cyc = py_walk(codes, w, mask)
    res = oracle_mod.weighted(codes, w, mask)
    np.testing.assert_array_equal(res.state == 2, cyc)
    ok = res.state == 1
    np.testing.assert_allclose(res.values[ok], expect[ok], rtol=1e-12, atol=1e-12)
    cnt_expect, _ = py_walk(codes, None, mask)
    rc = oracle_mod.counts(codes, mask)
    np.testing.assert_array_equal(rc.values[ok], cnt_expect[ok].astype(np.uint64))
    # the C brute-force walker agrees with the Python one on exact cells, with
    # weights and with unit weights, and finds the same cycle cells
    bf = oracle_mod.bruteforce(codes, w, mask)
    np.testing.assert_allclose(bf.values[ok], expect[ok], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(bf.state == 2, cyc)
    bfc = oracle_mod.bruteforce(codes, None, mask)
    np.testing.assert_array_equal(bfc.values[ok], cnt_expect[ok])


def test_mask_equals_nodata_code(oracle_mod):
    codes = synth.random_codes(30, 40, 21)
    mask = (synth.rng(22).random(codes.shape) < 0.1).astype(np.uint8)
    c2 = codes.copy()
    c2[mask != 0] = 0
    a = oracle_mod.counts(codes, mask)
    b = oracle_mod.counts(c2)
    np.testing.assert_array_equal(a.values, b.values)
    np.testing.assert_array_equal(a.state, b.state)


def test_cycles(oracle_mod):
    two = np.array([[1, 5]], np.uint8)
    r = oracle_mod.counts(two)
    assert r.n_cycle == 2 and (r.state == 2).all()
    four = np.array([[1, 7], [3, 5]], np.uint8)
    r = oracle_mod.counts(four)
    assert r.n_cycle == 4


def test_bad_codes_counted(oracle_mod):
    codes = np.array([[1, 10, 255], [9, 0, 3]], np.uint8)
    r = oracle_mod.counts(codes)
    assert r.n_bad == 2
    assert r.state[0, 1] == 0 and r.state[0, 2] == 0


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [31, 32])
def test_adjoint_dot_product_identity(oracle_mod, seed):
    codes = synth.acyclic_random_codes(29, 41, seed)
    g = synth.rng(seed).standard_normal(codes.shape).astype(np.float32)
    w = synth.uniform_weights(codes.shape, seed + 3)
    A = oracle_mod.weighted(codes, w).values
    lam = oracle_mod.adjoint(codes, g).values
    lhs = float((A * g.astype(np.float64)).sum())
    rhs = float((w.astype(np.float64) * lam).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-9)


def test_adjoint_path_sum_bruteforce(oracle_mod):
    codes = synth.random_codes(23, 27, 41)
    g = synth.rng(42).standard_normal(codes.shape).astype(np.float32)
    res = oracle_mod.adjoint(codes, g)
    expect = py_path_sum(codes, g)
    ok = res.state == 1
    assert ok.sum() > 100
    np.testing.assert_allclose(res.values[ok], expect[ok], rtol=1e-12, atol=1e-12)
    # cells on cycles or upstream of one are marked unspecified
    _, cyc = py_walk(codes)
    assert (res.state[cyc] == 2).all()


def test_adjoint_central_fd(oracle_mod):
    """L(w) = sum_g (A[g] - t[g])^2 is quadratic in w, so central differences
    are exact up to rounding; dL/dw = adjoint of 2 (A - t) on the gauges."""
    codes = synth.dem_codes(40, 50, 51)
    valid = (codes > 0) & (codes <= 9)
    w = synth.uniform_weights(codes.shape, 52, 0.0, 2.0).astype(np.float64)
    cnt = oracle_mod.counts(codes).values
    gauges = synth.gauges(valid, cnt, 12, 53, min_count=5)
    A0 = oracle_mod.weighted(codes, w.astype(np.float32)).values
    tgt = A0.ravel()[gauges] * 0.9

    def loss(wv):
        A = oracle_mod.weighted(codes, wv.astype(np.float32)).values
        return float(((A.ravel()[gauges] - tgt) ** 2).sum())

    wf = w.astype(np.float32)
    A = oracle_mod.weighted(codes, wf).values
    gA = np.zeros(codes.size)
    gA[gauges] = 2.0 * (A.ravel()[gauges] - tgt)
    grad = oracle_mod.adjoint(codes, gA.reshape(codes.shape).astype(np.float32)).values
    cells = synth.rng(54).choice(np.flatnonzero(valid.ravel()), 16, replace=False)
    h = 0.5
    for i in cells:
        wp = wf.astype(np.float64).copy().ravel()
        wm = wp.copy()
        wp[i] += h
        wm[i] -= h
        fd = (loss(wp.reshape(codes.shape)) - loss(wm.reshape(codes.shape))) / (2 * h)
        assert fd == pytest.approx(grad.ravel()[i], rel=1e-5, abs=1e-4)


# ---------------------------------------------------------------------------
# streaming residual verifier
# ---------------------------------------------------------------------------
def test_residual_verifier(oracle_mod):
    codes = synth.dem_codes(64, 80, 61)
    A = oracle_mod.counts(codes).values.astype(np.uint32)
    bad, first = oracle_mod.residual_u32(codes, A)
    assert bad == 0 and first == -1
    B = A.copy()
    B[10, 20] += 1  # planted mistake: the cell and its downstream cell disagree
    bad, first = oracle_mod.residual_u32(codes, B)
    assert bad >= 1 and first <= 10 * 80 + 20 + 80 + 1


def test_residual_rows_partition_the_raster(oracle_mod):
    """The band form of the residual check: disjoint bands that cover the
    raster find exactly the mismatches of the whole-raster check, each in the
    band holding the planted cell (Eq. 1 is checked cell by cell, so a band
    needs no other band's verdict)."""
    codes = synth.dem_codes(90, 70, 62)
    A = oracle_mod.counts(codes).values.astype(np.uint32)
    B = A.copy()
    B[47, 33] += 5
    whole = oracle_mod.residual_u32(codes, B)
    bands = [oracle_mod.residual_u32_rows(codes, B, r, min(90, r + 16)) for r in range(0, 90, 16)]
    assert sum(b for b, _ in bands) == whole[0] >= 1
    assert min(f for _, f in bands if f >= 0) == whole[1]
    hit = [i for i, (b, _) in enumerate(bands) if b]
    assert 47 // 16 in hit and all(abs(i * 16 - 47) <= 17 for i in hit)
    assert all(oracle_mod.residual_u32_rows(codes, A, r, r + 16)[0] == 0 for r in range(0, 90, 16))


def test_outlet_sum_hand_5x5(oracle_mod):
    """Conservation on the hand-worked 5x5 raster: its terminal cells hold
    19 (off the grid at (0,0)), 2 (into NoData at (2,3)) and 3 (NoFlow at
    (4,2)), 24 in all, one per valid cell.  The counts come from the golden
    file, not from the oracle's solver."""
    g = _golden.load("hand_5x5.txt")
    A = g["counts"].astype(np.uint32)
    s, nv = oracle_mod.outlet_sum_u32(g["codes"], A)
    assert (s, nv) == (24, 24)
    # bands add up; a wrong terminal value breaks it, a wrong inner value does not
    parts = [oracle_mod.outlet_sum_u32(g["codes"], A, r, r + 2) for r in range(0, 5, 2)]
    assert sum(p[0] for p in parts) == 24 and sum(p[1] for p in parts) == 24
    B = A.copy()
    B[4, 2] += 1
    assert oracle_mod.outlet_sum_u32(g["codes"], B)[0] == 25
    B = A.copy()
    B[1, 1] += 1
    assert oracle_mod.outlet_sum_u32(g["codes"], B)[0] == 24


def test_outlet_sum_closed_form_and_mask(oracle_mod):
    """All-east raster, A(r, c) = c + 1 (closed form): the terminal cells are
    the last column, each holding cols; with a masked column the cells west
    of it end there instead."""
    rows, cols = 7, 9
    codes = np.full((rows, cols), 1, np.uint8)
    A = np.tile(np.arange(1, cols + 1, dtype=np.uint32), (rows, 1))
    assert oracle_mod.outlet_sum_u32(codes, A) == (rows * cols, rows * cols)
    mask = np.zeros((rows, cols), np.uint8)
    mask[:, 4] = 1
    Am = np.where(np.arange(cols) < 4, np.arange(1, cols + 1), np.arange(cols) - 4)
    Am = np.tile(Am.astype(np.uint32), (rows, 1))
    Am[:, 4] = 0
    assert oracle_mod.outlet_sum_u32(codes, Am, mask=mask) == (rows * 8, rows * 8)
    v = oracle_mod.verify_counts_u32(codes, Am, threads=2, band=3, mask=mask)
    assert v["mismatches"] == 0 and v["conserved"]


def test_verify_counts_finds_a_planted_error(oracle_mod):
    codes = synth.dem_codes(120, 64, 63)
    A = oracle_mod.counts(codes).values.astype(np.uint32)
    v = oracle_mod.verify_counts_u32(codes, A, threads=3, band=10)
    assert v["mismatches"] == 0 and v["first"] == -1 and v["conserved"]
    assert v["n_valid"] == int(((codes >= 1) & (codes <= 9)).sum())
    B = A.copy()
    B[77, 5] -= 1
    v = oracle_mod.verify_counts_u32(codes, B, threads=3, band=10)
    assert v["mismatches"] >= 1 and v["first"] <= 77 * 64 + 5


def test_synth_dem_is_drained(oracle_mod):
    codes = synth.dem_codes(200, 173, 71)
    r = oracle_mod.counts(codes)
    assert r.n_cycle == 0 and r.n_bad == 0
    assert not (codes == 9).any()
    nd = (codes == 0).mean()
    assert 0.005 < nd < 0.02


# ---------------------------------------------------------------------------
# D8 directions (the step before accumulation)
# ---------------------------------------------------------------------------
def test_d8_hand_example(oracle_mod):
    # worked by hand: border cells drain outward (corners diagonal); (1,1)=5
    # drops 4 to its SE neighbour (slope 4/sqrt2 = 2.83 > 1 to the E); (1,2)=4
    # drops 3 to the S; (2,1)=6 drops 5 to the E; (2,2)=1 is a pit: NoFlow
    z = np.array([[9, 9, 9, 9], [9, 5, 4, 9], [9, 6, 1, 9], [9, 9, 9, 9]], np.float32)
    want = np.array([[4, 3, 3, 2], [5, 8, 7, 1], [5, 1, 9, 1], [6, 7, 7, 8]], np.uint8)
    np.testing.assert_array_equal(oracle_mod.d8(z), want)


def test_d8_ties_go_to_the_first_direction(oracle_mod):
    z = np.full((3, 3), 5.0, np.float32)
    z[1, 1] = 3.0
    z[1, 2] = 1.0  # E, drop 2
    z[2, 1] = 1.0  # S, drop 2: equal, E comes first
    assert oracle_mod.d8(z)[1, 1] == 1
    z[2, 1] = 0.9999  # S now strictly steeper
    assert oracle_mod.d8(z)[1, 1] == 7


def test_d8_nodata_and_flats(oracle_mod):
    z = np.full((5, 5), 2.0, np.float32)
    nd = np.zeros((5, 5), np.uint8)
    assert oracle_mod.d8(z)[2, 2] == 9  # a flat interior cell: NoFlow
    nd[1, 2] = 1  # N of the centre
    nd[3, 2] = 1  # S of the centre
    got = oracle_mod.d8(z, nd)
    assert got[2, 2] == 3  # no lower neighbour: the first NoData one (N before S)
    assert got[1, 2] == 0 and got[3, 2] == 0


def test_d8_tilted_plane(oracle_mod):
    R, C = 6, 9
    z = -np.tile(np.arange(C, dtype=np.float32), (R, 1))  # falls to the east
    got = oracle_mod.d8(z)
    assert (got[1:-1, 1:-1] == 1).all()
    assert (got[0, 1:-1] == 3).all() and (got[-1, 1:-1] == 7).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_d8_matches_the_generator_on_integer_dems(oracle_mod, seed):
    # the input generator's D8 (synth, double precision, its own code) decides
    # the same on integer elevations: drops are exact and no cardinal slope can
    # come within float rounding of a diagonal one at these magnitudes
    g = np.random.default_rng(seed)
    z = g.integers(0, 60, size=(40, 57)).astype(np.float32)
    nd = (g.random(z.shape) < 0.05).astype(np.uint8)
    np.testing.assert_array_equal(oracle_mod.d8(z, nd), synth.d8_codes(z, nd.astype(bool)))


# ---------------------------------------------------------------------------
# Packed and foreign codes (input decoding in front of Eq. 1)
# ---------------------------------------------------------------------------
def test_unpack_nibbles_hand_example(oracle_mod):
    # the 3x3 hand example with its codes packed by hand: row "8 7 6" is byte
    # 0x78 (8 low, 7 high) then 0x06; rows "1 7 5" are 0x71, 0x05
    g = _golden.load("hand_3x3.txt")
    packed = np.array([[0x78, 0x06], [0x71, 0x05], [0x71, 0x05]], np.uint8)
    codes = oracle_mod.unpack_nibbles(packed, 3)
    np.testing.assert_array_equal(codes, g["codes"])
    np.testing.assert_array_equal(oracle_mod.counts(codes).values, g["counts"])


def test_unpack_nibble_order(oracle_mod):
    # byte 0x91: cell 0 = 1 (E) into cell 1 = 9 (NoFlow), counts 1 and 2;
    # swapped nibbles would read 9 then 1 and give 1 and 1
    codes = oracle_mod.unpack_nibbles(np.array([[0x91]], np.uint8), 2)
    np.testing.assert_array_equal(codes, [[1, 9]])
    np.testing.assert_array_equal(oracle_mod.counts(codes).values, [[1, 2]])
    # odd width: the last byte's high nibble lies beyond the row and is ignored
    codes = oracle_mod.unpack_nibbles(np.array([[0x91, 0xF5]], np.uint8), 3)
    np.testing.assert_array_equal(codes, [[1, 9, 5]])


def test_unpacked_bad_nibbles_are_counted(oracle_mod):
    # nibbles 10..15 are invalid codes, counted like invalid bytes
    codes = oracle_mod.unpack_nibbles(np.array([[0xA1, 0x9F]], np.uint8), 4)
    np.testing.assert_array_equal(codes, [[1, 10, 15, 9]])
    assert oracle_mod.counts(codes).n_bad == 2


def test_recode_power_of_two_hand_example(oracle_mod):
    # the 3x3 hand example in the one-bit-per-direction scheme (E 1, SE 2, S 4,
    # SW 8, W 16, NW 32, N 64, NE 128), with its table typed from that scheme
    g = _golden.load("hand_3x3.txt")
    foreign = np.array([[2, 4, 8], [1, 4, 16], [1, 4, 16]], np.uint8)
    table = bytearray(256)
    for bit, code in {1: 1, 2: 8, 4: 7, 8: 6, 16: 5, 32: 4, 64: 3, 128: 2}.items():
        table[bit] = code
    codes = oracle_mod.recode(foreign, table)
    np.testing.assert_array_equal(codes, g["codes"])
    np.testing.assert_array_equal(oracle_mod.counts(codes).values, g["counts"])


# ---------------------------------------------------------------------------
# Absorption (Eq. 1 with alpha(n, d(n)) = a(n) in [0, 1])
# ---------------------------------------------------------------------------
def py_walk_absorb(codes, a, w=None, mask=None):
    """Definition by path walking (pure Python): each valid cell y adds w(y)
    times the product of a over the cells it has left behind to every cell on
    its downstream path.  Returns (values, on_cycle)."""
    R, C = codes.shape
    out = np.zeros((R, C))
    _, cyc = py_walk(codes, None, mask)
    for r in range(R):
        for c in range(C):
            if not _valid(codes, mask, r, c) or cyc[r, c]:
                continue
            share = 1.0 if w is None else float(w[r, c])
            cur, steps = (r, c), 0
            while cur is not None and steps <= R * C:
                out[cur] += share
                share *= float(a[cur])
                cur = _down(codes, mask, *cur)
                steps += 1
    return out, cyc


def test_absorb_hand_example(oracle_mod):
    # the 3x3 hand example with half of every cell's flow passed on: the centre
    # gets 1 + 0.5 * (five unit cells) = 3.5; the bottom centre gets
    # 1 + 0.5 * (3.5 + 1 + 1) = 3.75.  With weights 1..9 the centre gets
    # 5 + 0.5 * (1 + 2 + 3 + 4 + 6) = 13 and the bottom centre
    # 8 + 0.5 * (13 + 7 + 9) = 22.5
    g = _golden.load("hand_3x3.txt")
    half = np.full((3, 3), 0.5, np.float32)
    np.testing.assert_array_equal(oracle_mod.absorb(g["codes"], half).values,
                                  [[1, 1, 1], [1, 3.5, 1], [1, 3.75, 1]])
    np.testing.assert_array_equal(oracle_mod.absorb(g["codes"], half, g["weights"]).values,
                                  [[1, 2, 3], [4, 13, 6], [7, 22.5, 9]])


def test_absorb_special_factors(oracle_mod):
    codes = synth.random_codes(40, 53, 61)
    mask = (synth.rng(62).random(codes.shape) < 0.03).astype(np.uint8)
    w = synth.uniform_weights(codes.shape, 63)
    # nothing absorbed: plain accumulation
    one = oracle_mod.absorb(codes, np.ones(codes.shape, np.float32), w, mask)
    ref = oracle_mod.weighted(codes, w, mask)
    ok = ref.state == 1
    np.testing.assert_array_equal(one.state, ref.state)
    np.testing.assert_array_equal(one.values[ok], ref.values[ok])
    cnt = oracle_mod.absorb(codes, np.ones(codes.shape, np.float32), None, mask)
    np.testing.assert_array_equal(cnt.values[ok], oracle_mod.counts(codes, mask).values[ok])
    # everything absorbed: each cell keeps its own weight
    zero = oracle_mod.absorb(codes, np.zeros(codes.shape, np.float32), w, mask)
    np.testing.assert_array_equal(zero.values[ok], w[ok].astype(np.float64))
    assert (zero.values[ref.state == 0] == 0).all()


@pytest.mark.parametrize("a", [0.25, 0.9, 0.999])
def test_absorb_geometric_row(oracle_mod, a):
    # one row draining east with a constant factor: A(c) = 1 + a + ... + a^c
    C = 300
    codes = np.ones((1, C), np.uint8)
    got = oracle_mod.absorb(codes, np.full((1, C), a, np.float32)).values[0]
    af = float(np.float32(a))
    want = (1.0 - af ** (np.arange(C) + 1.0)) / (1.0 - af)
    np.testing.assert_allclose(got, want, rtol=1e-12)


@pytest.mark.parametrize("seed,R,C", [(71, 17, 23), (72, 40, 40), (73, 1, 60), (74, 33, 9)])
def test_absorb_bruteforce(oracle_mod, seed, R, C):
    codes = synth.random_codes(R, C, seed)
    mask = (synth.rng(seed + 5).random((R, C)) < 0.03).astype(np.uint8)
    a = synth.uniform_weights((R, C), seed + 6)
    w = synth.lognormal_weights((R, C), seed + 7)
    expect, cyc = py_walk_absorb(codes, a, w, mask)
    res = oracle_mod.absorb(codes, a, w, mask)
    np.testing.assert_array_equal(res.state == 2, cyc)
    ok = res.state == 1
    np.testing.assert_allclose(res.values[ok], expect[ok], rtol=1e-12, atol=1e-300)


def test_absorb_residual_on_a_dem(oracle_mod):
    # Eq. 1 cell by cell: A(p) - w(p) - sum of a(n) A(n) over n draining into p
    codes = synth.dem_codes(120, 97, 75)
    a = synth.uniform_weights(codes.shape, 76, 0.5, 1.0)
    w = synth.uniform_weights(codes.shape, 77)
    A = oracle_mod.absorb(codes, a, w).values
    R, C = codes.shape
    resid = np.zeros((R, C))
    for r in range(R):
        for c in range(C):
            if not _valid(codes, None, r, c):
                continue
            s = A[r, c] - w[r, c]
            for k, (dr, dc) in STEP.items():
                rr, cc = r - dr, c - dc  # the neighbour that would step onto (r, c)
                if _valid(codes, None, rr, cc) and int(codes[rr, cc]) == k:
                    s -= float(a[rr, cc]) * A[rr, cc]
            resid[r, c] = abs(s) / max(A[r, c], 1.0)
    assert resid.max() < 1e-12


def test_uint64_checks_do_not_wrap(oracle_mod):
    """The uint64 forms of the residual and conservation checks: zero
    mismatches on the oracle's own counts and on the all-east closed form, and
    a count off by exactly 2^32, invisible to the uint32 forms, is found."""
    codes = synth.dem_codes(80, 96, 64)
    A = oracle_mod.counts(codes).values.astype(np.uint64)
    assert oracle_mod.residual_u64_rows(codes, A, 0, 80) == (0, -1)
    v = oracle_mod.verify_counts_u32(codes, A, threads=2, band=7)
    assert v["mismatches"] == 0 and v["conserved"]
    B = A.copy()
    B[30, 40] += np.uint64(1 << 32)
    assert oracle_mod.residual_u32(codes, B.astype(np.uint32))[0] == 0
    bad, first = oracle_mod.residual_u64_rows(codes, B, 0, 80)
    assert bad >= 1 and first <= 30 * 96 + 40
    rows, cols = 5, 11
    east = np.full((rows, cols), 1, np.uint8)
    Ae = np.tile(np.arange(1, cols + 1, dtype=np.uint64), (rows, 1))
    assert oracle_mod.residual_u64_rows(east, Ae, 0, rows) == (0, -1)
    assert oracle_mod.outlet_sum_u64(east, Ae) == (rows * cols, rows * cols)
    Ai = Ae.copy()
    Ai[2, 3] += np.uint64(1 << 32)  # an inner cell: it and its downstream cell disagree
    assert oracle_mod.residual_u64_rows(east, Ai, 0, rows) == (2, 2 * cols + 3)
    Ae[2, cols - 1] += np.uint64(1 << 32)  # a terminal cell: conservation breaks by 2^32
    s, nv = oracle_mod.outlet_sum_u64(east, Ae)
    assert s - nv == 1 << 32
    v = oracle_mod.verify_counts_u32(east, Ae.astype(np.int64))
    assert not v["conserved"] and v["conserved_mod_2_32"] and v["mismatches"] == 1


# ---------------------------------------------------------------------------
# upstream-area sums at chosen cells (the per-cell definition of Eq. 1's solution)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", _golden.names())
def test_upstream_sums_golden(oracle_mod, name):
    """Every exact cell of each hand-worked fixture, queried one by one, gives
    the fixture's count and, where it has weights, its weighted sum; cycle
    cells report size -1; NoData cells 0."""
    fx = _golden.load(name)
    codes = fx["codes"]
    mask = fx.get("mask")
    cells = np.arange(codes.size)
    if "counts" in fx:
        v, n = oracle_mod.upstream_sums(codes, cells, None, mask)
        state = fx.get("state")
        exact = (state == 1).ravel() if state is not None else np.ones(codes.size, bool)
        np.testing.assert_array_equal(v[exact], fx["counts"].ravel()[exact].astype(np.float64))
        np.testing.assert_array_equal(n[exact], fx["counts"].ravel()[exact])
        if state is not None:
            assert (n[(state == 2).ravel()] == -1).all()
    if "weighted" in fx:
        v, _ = oracle_mod.upstream_sums(codes, cells, fx["weights"], mask)
        np.testing.assert_array_equal(v, fx["weighted"].ravel())


@pytest.mark.parametrize("R,C", [(1, 9), (6, 7), (11, 5)])
def test_upstream_sums_serpentine(oracle_mod, R, C):
    """One path through every cell: the cell k steps along it has k + 1 cells
    upstream, and with weights w their prefix sum."""
    codes = synth.serpentine_codes(R, C)
    k = synth.serpentine_index(R, C).ravel()
    v, n = oracle_mod.upstream_sums(codes, np.arange(R * C), threads=3)
    np.testing.assert_array_equal(n, k + 1)
    w = synth.uniform_weights((R, C), 71)
    order = np.argsort(k)
    prefix = np.cumsum(w.ravel()[order].astype(np.float64))
    v, _ = oracle_mod.upstream_sums(codes, np.arange(R * C), w)
    np.testing.assert_allclose(v[order], prefix, rtol=1e-12)


def test_upstream_sums_match_the_queue_solution(oracle_mod):
    """Two formulations of Eq. 1, the search against the flow per cell and
    the queue order over the raster, agree on a DEM with NoData, a mask and
    weights (FP64; sums in different orders)."""
    codes = synth.dem_codes(70, 90, 72)
    mask = (synth.rng(73).random(codes.shape) < 0.02).astype(np.uint8)
    w = synth.lognormal_weights(codes.shape, 74)
    ref = oracle_mod.weighted(codes, w, mask)
    cells = synth.rng(75).choice(codes.size, 500, replace=False)
    v, n = oracle_mod.upstream_sums(codes, cells, w, mask, threads=4)
    np.testing.assert_allclose(v, ref.values.ravel()[cells], rtol=1e-12)
    cnt = oracle_mod.counts(codes, mask)
    np.testing.assert_array_equal(n, cnt.values.ravel()[cells].astype(np.int64))
