"""GPU parity of fa_accumulate_adjoint (and the autograd wrapper) against the
oracle's transpose product, the dot-product identity and central finite
differences.

Tolerance: |gpu - ref| <= 2e-5 * (sum of |g| along the cell's downstream
path), the path-sum analogue of the forward's relative bound (g has mixed
signs, so a relative bound on the result itself would be meaningless).
"""
import numpy as np
import pytest
import torch

import synth
from tests import _golden

pytestmark = pytest.mark.gpu
fa = pytest.importorskip("paper_1608_04431_gb300")
TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_adj(codes, g, mask=None, tile=None):
    c = dev(codes)
    m = None if mask is None else dev(mask)
    out = fa.adjoint(c, dev(g.astype(np.float32)), m, tile=tile)
    st = fa.fa_status_read(None, fa.workspace(0, c.device))
    return out.cpu().numpy(), st


def check_adj(oracle_mod, codes, g, mask=None, tile=None):
    g = g.astype(np.float32)
    ref = oracle_mod.adjoint(codes, g, mask)
    scale = oracle_mod.adjoint(codes, np.abs(g), mask).values
    got, st = run_adj(codes, g, mask, tile)
    ok = ref.state == 1
    err = np.abs(got[ok].astype(np.float64) - ref.values[ok])
    assert (err <= TOL * scale[ok] + 1e-30).all(), float(np.max(err - TOL * scale[ok]))
    assert (got[ref.state == 0] == 0).all()
    return ref, got, st


@pytest.mark.parametrize("name", [n for n in _golden.names()
                                  if "adjoint" in _golden.load(n)])
@pytest.mark.parametrize("tile", [None, (1, 1), (2, 2), (3, 1)])
def test_golden_adjoint(name, tile):
    fx = _golden.load(name)
    got, st = run_adj(fx["codes"], fx["g"], fx.get("mask"), tile)
    np.testing.assert_array_equal(got, fx["adjoint"].astype(np.float32))
    assert st[0] == fa.FA_OK


@pytest.mark.parametrize("seed,R,C,tile", [(1, 64, 64, None), (2, 100, 77, (8, 8)),
                                           (3, 129, 200, (16, 32)), (4, 333, 257, None),
                                           (5, 40, 600, (4, 64)), (6, 31, 17, (5, 3))])
def test_random_acyclic(oracle_mod, seed, R, C, tile):
    codes = synth.acyclic_random_codes(R, C, seed)
    g = synth.rng(seed + 5).standard_normal((R, C))
    ref, got, st = check_adj(oracle_mod, codes, g, None, tile)
    assert st[0] == fa.FA_OK


@pytest.mark.parametrize("seed,tile", [(7, None), (8, (4, 4)), (9, (1, 1))])
def test_random_with_cycles(oracle_mod, seed, tile):
    codes = synth.random_codes(90, 110, seed)
    mask = (synth.rng(seed).random(codes.shape) < 0.02).astype(np.uint8)
    g = synth.rng(seed + 1).standard_normal(codes.shape)
    ref, got, st = check_adj(oracle_mod, codes, g, mask, tile)
    if (ref.state == 2).any():
        assert st[0] == fa.FA_ERR_CYCLE


def test_serpentine_adjoint(oracle_mod):
    codes = synth.serpentine_codes(300, 257)
    g = synth.rng(3).standard_normal(codes.shape)
    check_adj(oracle_mod, codes, g, None, (32, 32))


def test_dot_product_identity():
    codes = synth.dem_codes(700, 650, 17)
    w = synth.uniform_weights(codes.shape, 18, 0.0, 2.0)
    g = synth.rng(19).standard_normal(codes.shape).astype(np.float32)
    c = dev(codes)
    A = fa.accumulate(c, dev(w)).cpu().numpy().astype(np.float64)
    lam = fa.adjoint(c, dev(g)).cpu().numpy().astype(np.float64)
    lhs = float((A * g).sum())
    rhs = float((w.astype(np.float64) * lam).sum())
    assert lhs == pytest.approx(rhs, rel=1e-5)


def test_tile_invariance_adjoint():
    codes = synth.dem_codes(300, 280, 23)
    g = synth.rng(24).standard_normal(codes.shape).astype(np.float32)
    base, _ = run_adj(codes, g, None, (300, 28))
    for tile in [(1, 1), (8, 8), (64, 64), (64, 128), (17, 5)]:
        got, _ = run_adj(codes, g, None, tile)
        np.testing.assert_allclose(got, base, rtol=1e-5, atol=1e-5)


def test_autograd_matches_oracle(oracle_mod):
    codes = synth.dem_codes(200, 230, 33)
    w = synth.uniform_weights(codes.shape, 34, 0.0, 2.0)
    c = dev(codes)
    wt = dev(w).requires_grad_(True)
    A = fa.FlowAccumulate.apply(wt, c)
    coef = dev(synth.rng(35).standard_normal(codes.shape).astype(np.float32))
    (A * coef).sum().backward()
    ref = oracle_mod.adjoint(codes, coef.cpu().numpy())
    scale = oracle_mod.adjoint(codes, np.abs(coef.cpu().numpy())).values
    got = wt.grad.cpu().numpy().astype(np.float64)
    assert (np.abs(got - ref.values) <= TOL * scale + 1e-30).all()


def test_central_fd_small(oracle_mod):
    """Central differences of a quadratic gauge loss evaluated with the FP64
    oracle (exact up to rounding for a quadratic) against the GPU gradient."""
    codes = synth.dem_codes(120, 140, 43)
    valid = (codes > 0) & (codes <= 9)
    w = synth.uniform_weights(codes.shape, 44, 0.0, 2.0)
    cnt = oracle_mod.counts(codes).values
    gauges = synth.gauges(valid, cnt, 16, 45, min_count=20)
    tgt = oracle_mod.weighted(codes, w).values.ravel()[gauges] * 0.95

    def loss64(wv):
        A = oracle_mod.weighted(codes, wv.astype(np.float32)).values.ravel()
        return float(((A[gauges] - tgt) ** 2).sum())

    wt = dev(w).requires_grad_(True)
    A = fa.FlowAccumulate.apply(wt, dev(codes)).flatten()
    idx = torch.from_numpy(gauges).cuda()
    loss = ((A[idx].double() - torch.from_numpy(tgt).cuda()) ** 2).sum()
    loss.backward()
    grad = wt.grad.cpu().numpy().ravel()
    cells = synth.rng(46).choice(np.flatnonzero(valid.ravel()), 12, replace=False)
    h = 0.5
    for i in cells:
        wp, wm = w.astype(np.float64).ravel().copy(), w.astype(np.float64).ravel().copy()
        wp[i] += h
        wm[i] -= h
        fd = (loss64(wp.reshape(codes.shape)) - loss64(wm.reshape(codes.shape))) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-4, abs=1e-3 * max(1.0, abs(fd)))


@pytest.mark.slow
def test_gauge_loss_8192(oracle_mod):
    """8192^2 DEM, w ~ U[0,2), 256 gauges, targets from perturbed weights; the
    gradient against the oracle's transpose product and against central
    differences on 64 cells (32 upstream of gauges, 32 uniform)."""
    R = C = 8192
    codes = synth.dem_codes(R, C, 401)
    valid = (codes > 0) & (codes <= 9)
    w = synth.uniform_weights(codes.shape, 402, 0.0, 2.0)
    cnt = oracle_mod.counts(codes).values
    gauges = synth.gauges(valid, cnt, 256, 403, min_count=100)
    del cnt
    wpert = (w * (1.0 + 0.1 * synth.rng(404).standard_normal(codes.shape))).astype(np.float32)
    tgt = oracle_mod.weighted(codes, wpert).values.ravel()[gauges]
    del wpert
    A64 = oracle_mod.weighted(codes, w).values.ravel()

    wt = dev(w).requires_grad_(True)
    A = fa.FlowAccumulate.apply(wt, dev(codes)).flatten()
    idx = torch.from_numpy(gauges).cuda()
    loss = ((A[idx].double() - torch.from_numpy(tgt).cuda()) ** 2).sum()
    loss.backward()
    grad = wt.grad.cpu().numpy().ravel().astype(np.float64)

    # transpose product: g = 2 (A - t) on the gauges, taken from the GPU forward
    gA = np.zeros(R * C, dtype=np.float64)
    gA[gauges] = 2.0 * (A[idx].detach().double().cpu().numpy() - tgt)
    g32 = gA.astype(np.float32).reshape(R, C)
    ref = oracle_mod.adjoint(codes, g32)
    scale = oracle_mod.adjoint(codes, np.abs(g32)).values.ravel()
    err = np.abs(grad - ref.values.ravel())
    assert (err <= TOL * scale + 1e-30).all()

    # central differences, exact for the quadratic loss: A is linear in w, so
    # A(w +- h e_i) = A(w) +- h on the cells of i's downstream path (walked here)
    def path_of(i):
        out = []
        r, c = divmod(int(i), C)
        for _ in range(R * C):
            out.append(r * C + c)
            k = int(codes[r, c])
            if k < 1 or k > 8:
                break
            dr, dc = synth.DR[k], synth.DC[k]
            rr, cc = r + dr, c + dc
            if not (0 <= rr < R and 0 <= cc < C) or not valid[rr, cc]:
                break
            r, c = rr, cc
        return np.array(out)

    gset = {int(gi): n for n, gi in enumerate(gauges)}
    g2 = synth.rng(405)

    def upstream_of(gi):
        # random walk against the flow from a gauge: each step moves to a
        # random neighbour that drains into the current cell
        cur = int(gi)
        for _ in range(int(g2.integers(1, 200))):
            r, c = divmod(cur, C)
            preds = []
            for k in range(1, 9):
                rr, cc = r + synth.DR[k], c + synth.DC[k]
                if 0 <= rr < R and 0 <= cc < C and valid[rr, cc]:
                    kk = int(codes[rr, cc])
                    if 1 <= kk <= 8 and rr + synth.DR[kk] == r and cc + synth.DC[kk] == c:
                        preds.append(rr * C + cc)
            if not preds:
                break
            cur = preds[int(g2.integers(0, len(preds)))]
        return cur

    up = [upstream_of(gi) for gi in g2.choice(gauges, 32, replace=False)]
    cells = up + [int(x) for x in g2.choice(np.flatnonzero(valid.ravel()), 32, replace=False)]
    base = A64[gauges] - tgt  # FP64 forward
    h = 0.5
    n_on = 0
    for i in cells:
        on = [gset[int(x)] for x in path_of(i) if int(x) in gset]
        n_on += bool(on)
        dp, dm = base.copy(), base.copy()
        dp[on] += h
        dm[on] -= h
        fd = (float((dp ** 2).sum()) - float((dm ** 2).sum())) / (2 * h)
        # dL/dw_i = sum over gauges on the path of 2 (A_g - t_g); the GPU value
        # inherits the forward's 2e-5 relative error on each A_g
        tol = 2.0 * TOL * float(np.abs(A64[gauges][on]).sum()) + 1e-6 * abs(fd) + 1e-9
        assert abs(grad[i] - fd) <= tol, (i, grad[i], fd, tol)
    assert n_on >= 32
