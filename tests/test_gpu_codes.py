"""GPU parity for packed codes (two per byte) and code translation.

Packed rasters are built here with numpy; the oracle unpacks the same bytes
with its own decoder and accumulates the result, so the comparison runs from
identical stored bytes through two independent decoders.  Counts must match
bit for bit; float sums as in the plain forward tests.  Packed and byte codes
must also give identical results on the GPU for the same tile shape, since
only the loading of the codes differs.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

RTOL = 2e-5

fa = pytest.importorskip("paper_1608_04431_gb300")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t):
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def pack(codes, pitch=None):
    """Two codes per byte: cell c in byte c // 2, low nibble for even c."""
    R, C = codes.shape
    nb = (C + 1) // 2
    out = np.zeros((R, nb if pitch is None else pitch), np.uint8)
    lo = codes[:, 0::2].astype(np.uint8) & 15
    hi = codes[:, 1::2].astype(np.uint8) & 15
    out[:, :lo.shape[1]] = lo
    out[:, :hi.shape[1]] |= hi << 4
    return out


def packed_dev(codes, pitch=None):
    """PackedCodes on the device; with a pitch, a view into a wider buffer."""
    R, C = codes.shape
    p = pack(codes, pitch)
    t = dev(p)
    return fa.PackedCodes(t if pitch is None else t[:, :(C + 1) // 2], C)


def status():
    st = fa.fa_status_read(None, fa.workspace(0, "cuda"))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("seed,R,C,tile,pitch", [
    (1, 64, 64, None, None), (2, 100, 77, (8, 8), None), (3, 129, 201, (16, 32), 104),
    (4, 33, 500, (4, 64), 251), (5, 300, 301, None, None), (6, 50, 51, (1, 1), None),
    (7, 31, 17, (5, 3), 9), (8, 200, 90, (96, 80), None), (9, 77, 333, (7, 13), 170),
])
def test_packed_random_with_cycles(oracle_mod, seed, R, C, tile, pitch):
    codes = synth.random_codes(R, C, seed)
    mask = (synth.rng(seed + 50).random((R, C)) < 0.02).astype(np.uint8)
    p = pack(codes, pitch)
    ref = oracle_mod.counts(oracle_mod.unpack_nibbles(p, C), mask)
    pk = packed_dev(codes, pitch)
    m = dev(mask)
    got = to_np(fa.accumulate(pk, None, m, tile=tile))
    st = status()
    ok = ref.state == 1
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint32))
    assert (got[ref.state == 0] == 0).all()
    if ref.n_cycle:
        assert st[0] == fa.FA_ERR_CYCLE
    # byte codes, same tile shape: identical
    byt = to_np(fa.accumulate(dev(codes), None, m, tile=tile))
    np.testing.assert_array_equal(got[ok], byt[ok])
    w = synth.lognormal_weights((R, C), seed + 60)
    refw = oracle_mod.weighted(oracle_mod.unpack_nibbles(p, C), w, mask)
    gw = to_np(fa.accumulate(pk, dev(w), m, tile=tile))
    okw = refw.state == 1
    err = np.abs(gw[okw].astype(np.float64) - refw.values[okw])
    assert (err <= RTOL * np.abs(refw.values[okw])).all()
    bw = to_np(fa.accumulate(dev(codes), dev(w), m, tile=tile))
    np.testing.assert_array_equal(gw[okw], bw[okw])


@pytest.mark.parametrize("R,C,tile", [(1000, 1000, None), (777, 1301, (64, 128)), (513, 640, (32, 64)),
                                      (300, 299, (96, 64))])
def test_packed_dem_matches_bytes_and_oracle(oracle_mod, R, C, tile):
    # either form takes the TMA-staged path where the raster allows it (for
    # packed rows: a 16-byte pitch, here only 640 columns), else plain loads:
    # both must agree with the oracle bit for bit
    codes = synth.dem_codes(R, C, 81)
    ref = oracle_mod.counts(codes)
    pk = packed_dev(codes)
    a = to_np(fa.accumulate(pk, tile=tile))
    b = to_np(fa.accumulate(dev(codes), tile=tile))
    assert status()[0] == fa.FA_OK
    np.testing.assert_array_equal(a, ref.values.astype(np.uint32))
    np.testing.assert_array_equal(a, b)


def test_packed_bad_nibbles_status(oracle_mod):
    R, C = 90, 131
    codes = synth.acyclic_random_codes(R, C, 21)
    g = synth.rng(22)
    bad = g.random((R, C)) < 0.01
    codes = codes.copy()
    codes[bad] = g.integers(10, 16, size=int(bad.sum()))
    p = pack(codes)
    un = oracle_mod.unpack_nibbles(p, C)
    ref = oracle_mod.counts(un)
    got = to_np(fa.accumulate(packed_dev(codes), tile=(32, 32)))
    st, count, first = status()
    assert st == fa.FA_ERR_BAD_CODE
    assert count == ref.n_bad == int(bad.sum())
    assert first == int(np.flatnonzero(un > 9)[0])
    ok = ref.state == 1
    np.testing.assert_array_equal(got[ok], ref.values[ok].astype(np.uint32))


def test_packed_adjoint(oracle_mod):
    R, C = 300, 257
    codes = synth.dem_codes(R, C, 91)
    g = synth.uniform_weights((R, C), 92, -1.0, 1.0)
    p = pack(codes)
    ref = oracle_mod.adjoint(oracle_mod.unpack_nibbles(p, C), g)
    absref = oracle_mod.adjoint(codes, np.abs(g))
    a = to_np(fa.adjoint(packed_dev(codes), dev(g), tile=(64, 64)))
    b = to_np(fa.adjoint(dev(codes), dev(g), tile=(64, 64)))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a, b)
    ok = ref.state == 1
    err = np.abs(a[ok].astype(np.float64) - ref.values[ok])
    assert (err <= RTOL * absref.values[ok] + 1e-30).all()


def test_packed_batched_and_noalloc(oracle_mod):
    shapes = [(257, 311), (300, 129), (64, 1001), (1, 5)]
    items, byte_items, refs = [], [], []
    for i, (R, C) in enumerate(shapes):
        codes = synth.dem_codes(R, C, 100 + i) if min(R, C) > 8 else synth.random_codes(R, C, 100 + i)
        w = synth.uniform_weights((R, C), 200 + i)
        items.append({"codes": packed_dev(codes), "weights": [dev(w)]})
        byte_items.append({"codes": dev(codes), "weights": [dev(w)]})
        refs.append(oracle_mod.counts(codes))
    outs = fa.accumulate_batched([{"codes": it["codes"]} for it in items], 0, tile=(64, 64))
    for o, ref in zip(outs, refs):
        ok = ref.state == 1
        np.testing.assert_array_equal(to_np(o[0])[ok], ref.values[ok].astype(np.uint32))
    fo = fa.accumulate_batched(items, 1, tile=(64, 64))
    fb = fa.accumulate_batched(byte_items, 1, tile=(64, 64))
    for a, b in zip(fo, fb):
        np.testing.assert_array_equal(to_np(a[0]), to_np(b[0]))
    with pytest.raises(ValueError):
        fa.accumulate_batched([items[0], byte_items[1]], 1)
    # the entry point without a workspace reads packed codes too
    R, C = shapes[0]
    out = torch.empty((R, C), dtype=torch.uint32, device="cuda")
    assert fa.fa_accumulate_noalloc(items[0]["codes"], None, None, out, fa.FA_OUT_U32) == fa.FA_OK
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(out), refs[0].values.astype(np.uint32))


def test_packed_autograd():
    R, C = 200, 173
    codes = synth.dem_codes(R, C, 111)
    w = torch.tensor(synth.uniform_weights((R, C), 112), device="cuda", requires_grad=True)
    pk = packed_dev(codes)
    a = fa.FlowAccumulate.apply(w, pk, None, (64, 64))
    (a * a).sum().backward()
    ga = w.grad.clone()
    w.grad = None
    b = fa.FlowAccumulate.apply(w, dev(codes), None, (64, 64))
    (b * b).sum().backward()
    assert torch.equal(a, b) and torch.equal(ga, w.grad)


@pytest.mark.parametrize("R,C,ps,pd", [(1, 1, 1, 1), (37, 101, 101, 101), (64, 1024, 1024, 1024),
                                       (129, 333, 341, 347), (5, 8, 13, 9)])
def test_recode_bytes_and_nibbles(oracle_mod, R, C, ps, pd):
    g = synth.rng(R * 1000 + C)
    src = g.integers(0, 256, size=(R, C)).astype(np.uint8)
    table = g.integers(0, 256, size=256).astype(np.uint8).tobytes()
    sbuf = torch.zeros((R, ps), dtype=torch.uint8, device="cuda")
    sbuf[:, :C] = dev(src)
    s = sbuf[:, :C]
    want = oracle_mod.recode(src, table)
    dbuf = torch.full((R, pd), 0xEE, dtype=torch.uint8, device="cuda")
    d = dbuf[:, :C]
    assert fa.fa_recode(s, table, d, fa.FA_CODES_BYTE) == fa.FA_OK
    got = dbuf.cpu().numpy()
    np.testing.assert_array_equal(got[:, :C], want)
    assert (got[:, C:] == 0xEE).all()  # nothing written past the row
    nb = (C + 1) // 2
    pbuf = torch.full((R, max(pd // 2, nb)), 0xEE, dtype=torch.uint8, device="cuda")
    assert fa.fa_recode(s, table, pbuf[:, :nb], fa.FA_CODES_NIBBLE, C) == fa.FA_OK
    pk = pbuf.cpu().numpy()
    np.testing.assert_array_equal(oracle_mod.unpack_nibbles(pk[:, :nb], C), np.minimum(want, 15))
    if C % 2:
        assert (pk[:, nb - 1] >> 4 == 0).all()  # the unused high nibble is 0
    assert (pk[:, nb:] == 0xEE).all()
    # no table: the values themselves
    assert fa.fa_recode(s, None, d, fa.FA_CODES_BYTE) == fa.FA_OK
    np.testing.assert_array_equal(dbuf.cpu().numpy()[:, :C], src)


def test_power_of_two_codes_end_to_end(oracle_mod):
    R, C = 400, 515
    codes = synth.dem_codes(R, C, 121)
    to_bits = np.array([0, 1, 128, 64, 32, 16, 8, 4, 2, 0], np.uint8)  # our code -> its bit
    foreign = to_bits[codes]  # NoFlow has no bit: this DEM has none
    assert not (codes == 9).any()
    ref = oracle_mod.counts(oracle_mod.recode(foreign, fa.power_of_two_table()))
    np.testing.assert_array_equal(ref.values, oracle_mod.counts(codes).values)
    pk = fa.pack_codes(dev(foreign), fa.power_of_two_table())
    got = to_np(fa.accumulate(pk))
    assert status()[0] == fa.FA_OK
    np.testing.assert_array_equal(got, ref.values.astype(np.uint32))
    byt = fa.recode(dev(foreign), fa.power_of_two_table())
    np.testing.assert_array_equal(to_np(fa.accumulate(byt)), got)


@pytest.mark.slow
def test_packed_dem_16384(oracle_mod):
    codes = synth.dem_codes(16384, 16384, 201)
    pk = fa.pack_codes(dev(codes))
    got = to_np(fa.accumulate(pk, tile=(64, 128)))
    assert status()[0] == fa.FA_OK
    ref = oracle_mod.counts(oracle_mod.unpack_nibbles(pk.data.cpu().numpy(), 16384))
    np.testing.assert_array_equal(got, ref.values.astype(np.uint32))


@pytest.mark.parametrize("R,C,pitch,tile", [(1024, 2048, 1024, None), (1000, 1001, 512, (64, 64)),
                                            (333, 517, 272, (32, 64)), (129, 260, 144, (16, 32)),
                                            (700, 301, 160, (96, 80)), (64, 8191, 4096, (64, 128)),
                                            (97, 63, 48, (128, 32))])
def test_packed_tma_and_plain_loads_agree(oracle_mod, R, C, pitch, tile):
    """Packed rows with a 16-byte pitch and tile widths that are multiples of
    32 are staged by TMA; the result must equal the plain loads, the byte
    codes and the oracle.  The spare high nibble of an odd-width row holds a
    valid code (W, which would flow into the row's last cell) and the pitch
    padding holds garbage: neither may be read as a cell."""
    codes = synth.dem_codes(R, C, 131)
    p = pack(codes, pitch)
    if C % 2:
        p[:, C // 2] |= 5 << 4
    p[:, (C + 1) // 2:] = 0x55
    ref = oracle_mod.counts(oracle_mod.unpack_nibbles(p[:, :(C + 1) // 2], C))
    t = dev(p)
    pk = fa.PackedCodes(t[:, :(C + 1) // 2], C)
    a = to_np(fa.accumulate(pk, tile=tile))
    assert status()[0] == fa.FA_OK
    b = to_np(fa.accumulate(pk, tile=tile, flags=fa.FA_OPT_NO_TMA))
    c = to_np(fa.accumulate(dev(codes), tile=tile))
    np.testing.assert_array_equal(a, ref.values.astype(np.uint32))
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    w = dev(synth.uniform_weights((R, C), 132))
    fw = to_np(fa.accumulate(pk, w, tile=tile))
    gw = to_np(fa.accumulate(pk, w, tile=tile, flags=fa.FA_OPT_NO_TMA))
    np.testing.assert_array_equal(fw, gw)
