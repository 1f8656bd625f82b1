"""Seeded synthetic inputs for D8 flow accumulation.

This module is input infrastructure shared by the CPU oracle side and the CUDA
side.  It holds none of the flow-accumulation arithmetic: it makes elevation
rasters, fills their depressions, derives one-byte D8 codes, and draws weight
fields, gauges and batch shapes.  The paper evaluates on SRTM, NED and PAMAP
DEMs (Section 5, Table 1); these generators stand in for them with rasters of
the same kind: spectrally synthesised terrain (1/f^2 power spectrum),
depression-filled by priority-flood with an epsilon gradient (Section 2), with
D8 steepest-descent directions and a contiguous NoData blob.

Code encoding: 0 NoData, 1..8 = E, NE, N, NW, W, SW, S, SE, 9 NoFlow.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

CODE_NODATA = 0
CODE_NOFLOW = 9
# (dr, dc) per code 1..8 (index 0 unused)
DR = (0, 0, -1, -1, -1, 0, 1, 1, 1)
DC = (0, 1, 1, 0, -1, -1, -1, 0, 1)


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.synth_priority_flood_eps.argtypes = [p, p, i64, i64, ctypes.c_float]
        lib.synth_priority_flood_eps.restype = ctypes.c_int
        lib.synth_priority_flood_eps4.argtypes = [p, p, i64, i64, ctypes.c_float]
        lib.synth_priority_flood_eps4.restype = ctypes.c_int
        lib.synth_d8.argtypes = [p, p, i64, i64, p]
        lib.synth_d8.restype = None
        lib.synth_bilinear_up.argtypes = [p, i64, i64, i64, p]
        lib.synth_bilinear_up.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# elevation
# ---------------------------------------------------------------------------
def spectral_dem(rows: int, cols: int, seed: int, zmax: float = 1000.0) -> np.ndarray:
    """Gaussian white noise shaped to amplitude ~ 1/|f| (power ~ 1/f^2), DC
    removed, rescaled to [0, zmax] metres, float32."""
    import scipy.fft as sfft

    noise = rng(seed).standard_normal((rows, cols), dtype=np.float32)
    spec = sfft.rfft2(noise, workers=-1)
    del noise
    fy = np.fft.fftfreq(rows).astype(np.float32)
    fx = np.fft.rfftfreq(cols).astype(np.float32)
    fx2 = fx * fx
    for r0 in range(0, rows, 1024):
        blk = fy[r0:r0 + 1024, None]
        f = np.sqrt(blk * blk + fx2[None, :])
        with np.errstate(divide="ignore"):
            amp = np.where(f > 0, 1.0 / f, 0.0).astype(np.float32)
        spec[r0:r0 + 1024] *= amp
    dem = sfft.irfft2(spec, s=(rows, cols), workers=-1).astype(np.float32, copy=False)
    del spec
    lo, hi = float(dem.min()), float(dem.max())
    dem -= np.float32(lo)
    dem *= np.float32(zmax / (hi - lo))
    return dem


def nodata_disk(rows: int, cols: int, seed: int, frac: float = 0.01, radius: float | None = None):
    """Boolean mask of one contiguous disk covering ~frac of the cells, with a
    seeded centre at least radius+2 cells from every edge."""
    if radius is None:
        radius = float(np.sqrt(frac * rows * cols / np.pi))
    g = rng(seed)
    m = int(np.ceil(radius)) + 2
    cr = int(g.integers(m, max(m + 1, rows - m)))
    cc = int(g.integers(m, max(m + 1, cols - m)))
    rr = np.arange(rows)[:, None] - cr
    ccs = np.arange(cols)[None, :] - cc
    return (rr * rr + ccs * ccs) <= radius * radius


def priority_flood_eps(dem: np.ndarray, nodata: np.ndarray, eps: float = 1e-4,
                       edge_only: bool = False) -> np.ndarray:
    """Priority-flood eps fill; edge_only spreads the flood to the four edge
    neighbours only, so that every filled cell is strictly above an edge
    neighbour."""
    z = np.ascontiguousarray(dem, dtype=np.float32).copy()
    nd = np.ascontiguousarray(nodata, dtype=np.uint8)
    fn = _load().synth_priority_flood_eps4 if edge_only else _load().synth_priority_flood_eps
    rc = fn(_ptr(z), _ptr(nd), z.shape[0], z.shape[1], float(eps))
    if rc != 0:
        raise MemoryError("priority flood: allocation failed")
    return z


def d8_codes(z: np.ndarray, nodata: np.ndarray) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float32)
    nd = np.ascontiguousarray(nodata, dtype=np.uint8)
    out = np.empty(z.shape, dtype=np.uint8)
    _load().synth_d8(_ptr(z), _ptr(nd), z.shape[0], z.shape[1], _ptr(out))
    return out


def bilinear_up(a: np.ndarray, f: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty((a.shape[0] * f, a.shape[1] * f), dtype=np.float32)
    _load().synth_bilinear_up(_ptr(a), a.shape[0], a.shape[1], int(f), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# caching
# ---------------------------------------------------------------------------
_CACHE_VERSION = "v1"


def _cache_dir() -> str | None:
    d = os.environ.get("FA_SYNTH_CACHE", "/tmp/fa_synth_cache")
    if d in ("", "0", "off"):
        return None
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, make):
    d = _cache_dir()
    if d is None:
        return make()
    h = hashlib.sha1((_CACHE_VERSION + key).encode()).hexdigest()[:20]
    path = os.path.join(d, f"{h}.npy")
    if os.path.exists(path):
        try:
            return np.load(path, mmap_mode=None)
        except Exception:
            pass
    arr = make()
    tmp = path + f".tmp{os.getpid()}.npy"
    np.save(tmp, arr)
    os.replace(tmp, path)
    return arr


# ---------------------------------------------------------------------------
# D8 rasters
# ---------------------------------------------------------------------------
def dem_codes(rows: int, cols: int, seed: int, nodata_frac: float = 0.01,
              nodata_radius: float | None = None, eps: float = 1e-4) -> np.ndarray:
    """Spectral DEM -> NoData disk -> priority-flood eps fill -> D8 codes (uint8)."""
    key = f"dem_codes/{rows}/{cols}/{seed}/{nodata_frac}/{nodata_radius}/{eps}"

    def make():
        dem = spectral_dem(rows, cols, seed)
        if nodata_frac > 0 or nodata_radius:
            nd = nodata_disk(rows, cols, seed + 7919, nodata_frac, nodata_radius)
        else:
            nd = np.zeros((rows, cols), dtype=bool)
        z = priority_flood_eps(dem, nd, eps)
        del dem
        return d8_codes(z, nd)

    return _cached(key, make)


def serpentine_codes(rows: int, cols: int) -> np.ndarray:
    """Boustrophedon single drainage path covering every cell: row 0 runs east,
    row 1 west, ...; the end of each row steps south; the last cell exits
    off-grid.  Path index k of cell (r, c) is r*cols + (c if r even else cols-1-c)."""
    codes = np.empty((rows, cols), dtype=np.uint8)
    codes[0::2, :] = 1  # E
    codes[1::2, :] = 5  # W
    codes[0::2, cols - 1] = 7  # S at the east end of even rows
    codes[1::2, 0] = 7  # S at the west end of odd rows
    # last cell: keep its row direction, which points off-grid (E on an even
    # last row at the east edge, W on an odd last row at the west edge)
    if (rows - 1) % 2 == 0:
        codes[rows - 1, cols - 1] = 1
    else:
        codes[rows - 1, 0] = 5
    if cols == 1:
        codes[:, 0] = 7
    return codes


def serpentine_index(rows: int, cols: int) -> np.ndarray:
    r = np.arange(rows, dtype=np.int64)[:, None]
    c = np.arange(cols, dtype=np.int64)[None, :]
    cc = np.where(r % 2 == 0, c, cols - 1 - c)
    return r * cols + cc


def random_codes(rows: int, cols: int, seed: int, p_nodata: float = 0.05,
                 p_noflow: float = 0.03) -> np.ndarray:
    """Uniform random directions with scattered NoData and NoFlow cells; may
    contain cycles (2-cycles are common)."""
    g = rng(seed)
    codes = g.integers(1, 9, size=(rows, cols), dtype=np.uint8)
    u = g.random((rows, cols))
    codes[u < p_nodata] = 0
    codes[(u >= p_nodata) & (u < p_nodata + p_noflow)] = 9
    return codes


def acyclic_random_codes(rows: int, cols: int, seed: int, p_nodata: float = 0.05,
                         p_noflow: float = 0.02) -> np.ndarray:
    """Random D8 codes guaranteed acyclic: a random potential field orders the
    cells and each cell points at a random strictly-lower neighbour (or off the
    grid / NoFlow when it has none)."""
    g = rng(seed)
    pot = g.random((rows, cols))
    nd = g.random((rows, cols)) < p_nodata
    codes = np.zeros((rows, cols), dtype=np.uint8)
    for r in range(rows):
        for c in range(cols):
            if nd[r, c]:
                continue
            cands = []
            for k in range(1, 9):
                rr, cc = r + DR[k], c + DC[k]
                if 0 <= rr < rows and 0 <= cc < cols:
                    if not nd[rr, cc] and pot[rr, cc] < pot[r, c]:
                        cands.append(k)
                    elif nd[rr, cc]:
                        cands.append(k)  # into NoData: flow leaves the system
                else:
                    cands.append(k)  # off-grid outlet
            if not cands or g.random() < p_noflow:
                codes[r, c] = 9
            else:
                codes[r, c] = cands[int(g.integers(0, len(cands)))]
    return codes


# ---------------------------------------------------------------------------
# weights, batches, gauges
# ---------------------------------------------------------------------------
def uniform_weights(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    w = rng(seed).random(shape, dtype=np.float32)
    if lo != 0.0 or hi != 1.0:
        w = (w * np.float32(hi - lo) + np.float32(lo)).astype(np.float32)
    return w


def lognormal_weights(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    return rng(seed).lognormal(0.0, sigma, size=shape).astype(np.float32)


def batch_shapes(n: int, seed: int, rmin=257, rmax=4096, cmin=311, cmax=6000):
    """Independent uniform row and column counts for a batch of rasters."""
    g = rng(seed)
    rows = g.integers(rmin, rmax + 1, size=n)
    cols = g.integers(cmin, cmax + 1, size=n)
    return [(int(r), int(c)) for r, c in zip(rows, cols)]


def batch_rasters(n: int = 64, first_seed: int = 301, shape_seed: int = 300,
                  n_fields: int = 8, threads: int | None = None, shapes=None):
    """n spectral-DEM rasters with n_fields f32 weight fields each: the first
    half uniform [0,1), the second half lognormal sigma=1."""
    if shapes is None:
        shapes = batch_shapes(n, shape_seed)
    seeds = [first_seed + i for i in range(n)]

    def one(i):
        r, c = shapes[i]
        codes = dem_codes(r, c, seeds[i])
        fields = []
        for k in range(n_fields):
            fs = seeds[i] * 100 + k
            if k < (n_fields + 1) // 2:
                fields.append(uniform_weights((r, c), fs))
            else:
                fields.append(lognormal_weights((r, c), fs))
        return codes, fields

    threads = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, range(n)))


def scale_codes(coarse_rows: int, coarse_cols: int, factor: int, seed: int,
                noise_seed: int, noise_amp: float = 0.5) -> np.ndarray:
    """Coarse spectral DEM bilinearly upsampled by an integer factor plus
    seeded white noise U[-amp, amp], then filled and converted to D8."""
    key = f"scale_codes/{coarse_rows}/{coarse_cols}/{factor}/{seed}/{noise_seed}/{noise_amp}"

    def make():
        dem = bilinear_up(spectral_dem(coarse_rows, coarse_cols, seed), factor)
        g = rng(noise_seed)
        for r0 in range(0, dem.shape[0], 4096):
            blk = dem[r0:r0 + 4096]
            blk += (g.random(blk.shape, dtype=np.float32) * np.float32(2 * noise_amp)
                    - np.float32(noise_amp))
        nd = np.zeros(dem.shape, dtype=bool)
        z = priority_flood_eps(dem, nd)
        del dem
        return d8_codes(z, nd)

    return _cached(key, make)


def gauges(valid_mask: np.ndarray, counts: np.ndarray, n: int, seed: int, min_count: int = 100):
    """n distinct gauge cells drawn uniformly among valid cells with count >= min_count."""
    cand = np.flatnonzero((counts.ravel() >= min_count) & valid_mask.ravel())
    g = rng(seed)
    return np.sort(g.choice(cand, size=min(n, cand.size), replace=False))


# ---------------------------------------------------------------------------
# the 1e10-cell scale raster, generated on a torch device band by band
# ---------------------------------------------------------------------------
def _fmix32(h, torch):
    """murmur3's 32-bit finaliser on int64 tensors holding values < 2^32."""
    m = 0xFFFFFFFF
    h = h ^ (h >> 16)
    h = (h * 0x85EBCA6B) & m
    h = h ^ (h >> 13)
    h = (h * 0xC2B2AE35) & m
    return h ^ (h >> 16)


def cell_noise(idx, seed: int, amp: float, torch):
    """Counter-based white noise U[-amp, amp) for global cell indices idx
    (int64 tensor): two rounds of murmur3's finaliser over (seed, index), top
    24 bits as a uniform fraction, in float64.  The same cell gets the same
    value whichever band computes it."""
    lo = idx & 0xFFFFFFFF
    hi = idx >> 32
    h = _fmix32(hi ^ (seed & 0xFFFFFFFF), torch)
    h = _fmix32(lo ^ h, torch)
    u = (h >> 8).to(torch.float64) * (1.0 / (1 << 24))
    return (u * 2.0 - 1.0) * amp


def scale_coarse(coarse_rows: int, coarse_cols: int, seed: int, eps: float = 1e-4) -> np.ndarray:
    """The coarse level of the scale raster: spectral DEM, eps-filled by
    priority flood (no NoData), float32."""
    key = f"scale_coarse4/{coarse_rows}/{coarse_cols}/{seed}/{eps}"

    def make():
        dem = spectral_dem(coarse_rows, coarse_cols, seed)
        return priority_flood_eps(dem, np.zeros(dem.shape, dtype=bool), eps, edge_only=True)

    return _cached(key, make)


def _bilinear_axis(n_fine: int, n_coarse: int, f: int, torch, dev):
    """Per fine index along one axis: the lower coarse index of its patch and
    its fraction.  Fine cell i sits at coarse coordinate x = i / f, so every
    coarse cell centre is also a fine cell centre and the fine cells on a line
    between two coarse centres interpolate those two alone; past the last
    coarse centre the last patch is extended linearly (no clamp)."""
    x = torch.arange(n_fine, device=dev, dtype=torch.float64) / f
    x0 = torch.clamp(torch.floor(x), 0, max(n_coarse - 2, 0)).to(torch.int64)
    return x0, x - x0.to(torch.float64)


def scale_codes_device(coarse_rows: int, coarse_cols: int, factor: int, seed: int,
                       noise_seed: int, noise_amp: float = 0.5, band: int = 256,
                       device="cuda", rows=None):
    """uint8 D8 codes of the scale raster, generated on `device` (a torch
    device) band by band; returns a [coarse_rows*factor, coarse_cols*factor]
    uint8 tensor there, or only the rows rows[0] .. rows[1] - 1 of it (the
    same values: every cell is computed from its own neighbourhood).

    S is the eps-filled coarse spectral DEM bilinearly upsampled by `factor`
    (float64, exact for these weights); Z = S + white noise U[-amp, amp)
    (counter-based, cell_noise).  Each interior cell drains to the neighbour
    with the steepest Z descent (drop / distance, diagonal distance sqrt 2,
    ties to the first of E, NE, N, NW, W, SW, S, SE) among the neighbours that
    are strictly lower in S; with none it is NoFlow.  Border cells drain off
    the grid (perpendicular, diagonal at the corners).  Because every step
    goes strictly down in S the codes are acyclic, and because S has no
    depressions flow follows the coarse drainage across the raster; the noise
    only picks among the descending neighbours.  This stands in for filling
    the noisy fine raster itself, whose priority flood over 1e10 cells takes
    tens of minutes on a host."""
    import torch

    dev = torch.device(device)
    F = torch.from_numpy(scale_coarse(coarse_rows, coarse_cols, seed)).to(dev, torch.float64)
    R, C = coarse_rows * factor, coarse_cols * factor
    lo, hi = (0, R) if rows is None else (max(0, int(rows[0])), min(R, int(rows[1])))
    codes = torch.empty((max(0, hi - lo), C), dtype=torch.uint8, device=dev)
    xc0, fx = _bilinear_axis(C, coarse_cols, factor, torch, dev)
    yc0_all, fy_all = _bilinear_axis(R, coarse_rows, factor, torch, dev)
    xc1 = torch.clamp(xc0 + 1, max=coarse_cols - 1)
    colidx = torch.arange(C, device=dev, dtype=torch.int64)
    inv_sqrt2 = 1.0 / np.sqrt(2.0)
    dirs = [(1, 0, 1), (2, -1, 1), (3, -1, 0), (4, -1, -1), (5, 0, -1), (6, 1, -1), (7, 1, 0),
            (8, 1, 1)]
    for r0 in range(lo, hi, band):
        r1 = min(hi, r0 + band)
        ra, rb = max(0, r0 - 1), min(R, r1 + 1)  # rows of S and Z with a halo row
        y0 = yc0_all[ra:rb]
        y1 = torch.clamp(y0 + 1, max=coarse_rows - 1)
        fy = fy_all[ra:rb, None]
        top = F[y0][:, xc0] * (1.0 - fx) + F[y0][:, xc1] * fx
        bot = F[y1][:, xc0] * (1.0 - fx) + F[y1][:, xc1] * fx
        S = top * (1.0 - fy) + bot * fy
        del top, bot
        rows_idx = torch.arange(ra, rb, device=dev, dtype=torch.int64)[:, None]
        Z = S + cell_noise(rows_idx * C + colidx[None, :], noise_seed, noise_amp, torch)
        # a halo row beyond the raster's edge is never lower in S
        if ra == r0:
            S = torch.cat([torch.full((1, C), float("inf"), dtype=torch.float64, device=dev), S])
            Z = torch.cat([torch.zeros((1, C), dtype=torch.float64, device=dev), Z])
        if rb == r1:
            S = torch.cat([S, torch.full((1, C), float("inf"), dtype=torch.float64, device=dev)])
            Z = torch.cat([Z, torch.zeros((1, C), dtype=torch.float64, device=dev)])
        # rows r0..r1-1 sit at 1..r1-r0 of the haloed arrays
        i0, i1 = 1, 1 + (r1 - r0)
        Sc, Zc = S[i0:i1, 1:C - 1], Z[i0:i1, 1:C - 1]
        best = torch.full(Sc.shape, -float("inf"), dtype=torch.float64, device=dev)
        code = torch.full(Sc.shape, 9, dtype=torch.uint8, device=dev)
        for k, dr, dc in dirs:
            Sn = S[i0 + dr:i1 + dr, 1 + dc:C - 1 + dc]
            Zn = Z[i0 + dr:i1 + dr, 1 + dc:C - 1 + dc]
            slope = Zc - Zn
            if dr and dc:
                slope = slope * inv_sqrt2
            take = (Sn < Sc) & (slope > best)
            best = torch.where(take, slope, best)
            code = torch.where(take, torch.full_like(code, k), code)
        out = codes[r0 - lo:r1 - lo]
        out[:, 1:C - 1] = code
        # border cells drain off the grid
        out[:, 0] = 5
        out[:, C - 1] = 1
        if r0 == 0:
            out[0, :] = 3
            out[0, 0], out[0, C - 1] = 4, 2
        if r1 == R:
            out[-1, :] = 7
            out[-1, 0], out[-1, C - 1] = 6, 8
        del S, Z, best, code
    return codes


def scale_codes_rows(coarse_rows: int, coarse_cols: int, factor: int, seed: int,
                     noise_seed: int, r0: int, r1: int, noise_amp: float = 0.5) -> np.ndarray:
    """Rows r0 .. r1 - 1 of the scale raster generated on the host (torch on
    the CPU), the same bytes as scale_codes_device gives for those rows."""
    return scale_codes_device(coarse_rows, coarse_cols, factor, seed, noise_seed, noise_amp,
                              device="cpu", rows=(r0, r1)).numpy()
