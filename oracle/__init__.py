"""CPU oracle for D8 flow accumulation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it, and
the two share no code: the oracle is plain C (``fa_oracle.c``, compiled with
gcc) plus the numpy marshalling below.

Functions (all on numpy arrays, row-major, row 0 = north):
  counts(codes, mask)            -> uint64 upslope counts (Eq. 1, w = 1)
  weighted(codes, w, mask)       -> FP64 weighted accumulation (Eq. 1)
  absorb(codes, a, w, mask)      -> FP64 accumulation with absorption (Eq. 1,
                                    alpha = a(n) in [0, 1] towards d(n))
  adjoint(codes, g, mask)        -> FP64 lam = (I - P)^-T g (downstream path sums)
  bruteforce(codes, w, mask)     -> FP64 path-walking sums straight from the
                                    definition (small rasters only)
  residual_u32(codes, A, mask)   -> number of cells violating Eq. 1 (mod 2^32)
  residual_u32_rows(...)         -> the same on a band of rows
  outlet_sum_u32(codes, A, ...)  -> conservation: sum of A over terminal cells
                                    and the number of valid cells
  verify_counts_u32(codes, A)    -> both over row bands on host threads (any size)
  d8(z, nodata)                  -> uint8 D8 codes from float32 elevations (the
                                    direction step before accumulation)
  unpack_nibbles(packed, cols)   -> uint8 codes from codes stored two per byte
  recode(codes, table)           -> codes translated through a 256-entry table

Each returns the values plus a ``state`` array: 0 NoData, 1 exact,
2 unspecified (on a cycle; for the adjoint, on or upstream of a cycle).

Parity status: every function is pinned by tests/test_oracle.py (hand-worked
examples, closed forms, conservation, brute force, cycle cases, the adjoint
dot-product identity and central finite differences), and
tests/test_oracle_mutants.py shows that planted mistakes in a copy of this
oracle (one-line changes to the C source, or a replaced decoder) each make a
pin fail.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fa_oracle.c")
_LIB = os.path.join(_HERE, "libfa_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile fa_oracle.c with gcc into libfa_oracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declares the argument and result types of the oracle's C functions on a
    loaded copy of the library and returns it."""
    i64, p = ctypes.c_int64, ctypes.c_void_p
    pi64 = ctypes.POINTER(ctypes.c_int64)
    lib.fa_oracle_counts.argtypes = [p, i64, i64, i64, p, i64, p, p, pi64, pi64]
    lib.fa_oracle_counts.restype = ctypes.c_int
    lib.fa_oracle_weighted.argtypes = [p, i64, i64, i64, p, i64, p, i64, p, p, pi64, pi64]
    lib.fa_oracle_weighted.restype = ctypes.c_int
    lib.fa_oracle_adjoint.argtypes = [p, i64, i64, i64, p, i64, p, i64, p, p, pi64, pi64]
    lib.fa_oracle_adjoint.restype = ctypes.c_int
    lib.fa_oracle_absorb.argtypes = [p, i64, i64, i64, p, i64, p, i64, p, i64, p, p, pi64, pi64]
    lib.fa_oracle_absorb.restype = ctypes.c_int
    lib.fa_oracle_d8.argtypes = [p, i64, i64, i64, p, i64, p]
    lib.fa_oracle_d8.restype = ctypes.c_int
    lib.fa_oracle_bruteforce.argtypes = [p, i64, i64, i64, p, i64, p, i64, p, p]
    lib.fa_oracle_bruteforce.restype = ctypes.c_int
    lib.fa_oracle_residual_u32.argtypes = [p, i64, i64, i64, p, i64, p, i64, pi64]
    lib.fa_oracle_residual_u32.restype = ctypes.c_int64
    lib.fa_oracle_residual_u32_rows.argtypes = [p, i64, i64, i64, p, i64, p, i64, i64, i64, pi64]
    lib.fa_oracle_residual_u32_rows.restype = ctypes.c_int64
    lib.fa_oracle_outlet_sum_u32.argtypes = [p, i64, i64, i64, p, i64, p, i64, i64, i64,
                                             ctypes.POINTER(ctypes.c_uint64), pi64]
    lib.fa_oracle_outlet_sum_u32.restype = None
    lib.fa_oracle_residual_u64_rows.argtypes = [p, i64, i64, i64, p, i64, p, i64, i64, i64, pi64]
    lib.fa_oracle_residual_u64_rows.restype = ctypes.c_int64
    lib.fa_oracle_outlet_sum_u64.argtypes = [p, i64, i64, i64, p, i64, p, i64, i64, i64,
                                             ctypes.POINTER(ctypes.c_uint64), pi64]
    lib.fa_oracle_outlet_sum_u64.restype = None
    lib.fa_oracle_upstream_sums.argtypes = [p, i64, i64, i64, p, i64, p, i64, p, i64, p, p]
    lib.fa_oracle_upstream_sums.restype = ctypes.c_int64
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


@dataclass
class Result:
    values: np.ndarray
    state: np.ndarray  # 0 NoData, 1 exact, 2 unspecified (cycle)
    n_cycle: int
    n_bad: int


def _prep(codes, mask):
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    if codes.ndim != 2:
        raise ValueError("codes must be 2-D")
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        if mask.shape != codes.shape:
            raise ValueError("mask shape differs from codes")
    return codes, mask


def _p(a):
    return None if a is None else a.ctypes.data


def counts(codes, mask=None) -> Result:
    """Unit-weight accumulation, uint64 (Algorithm 1 over the whole raster)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    out = np.empty((R, C), dtype=np.uint64)
    st = np.empty((R, C), dtype=np.uint8)
    nc, nb = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = _load().fa_oracle_counts(_p(codes), R, C, C, _p(mask), C, _p(out), _p(st),
                                  ctypes.byref(nc), ctypes.byref(nb))
    if rc:
        raise MemoryError("oracle: allocation failed")
    return Result(out, st, nc.value, nb.value)


def weighted(codes, w, mask=None) -> Result:
    """Weighted accumulation in FP64 from float32 weights."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    w = np.ascontiguousarray(w, dtype=np.float32)
    if w.shape != codes.shape:
        raise ValueError("weights shape differs from codes")
    out = np.empty((R, C), dtype=np.float64)
    st = np.empty((R, C), dtype=np.uint8)
    nc, nb = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = _load().fa_oracle_weighted(_p(codes), R, C, C, _p(mask), C, _p(w), C, _p(out), _p(st),
                                    ctypes.byref(nc), ctypes.byref(nb))
    if rc:
        raise MemoryError("oracle: allocation failed")
    return Result(out, st, nc.value, nb.value)


def absorb(codes, a, w=None, mask=None) -> Result:
    """Accumulation with absorption in FP64: A(p) = w(p) + sum of a(n) A(n)
    over the cells n draining into p; a: float32 factors in [0, 1]; w: float32
    weights or None (unit)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != codes.shape:
        raise ValueError("a shape differs from codes")
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.shape != codes.shape:
            raise ValueError("weights shape differs from codes")
    out = np.empty((R, C), dtype=np.float64)
    st = np.empty((R, C), dtype=np.uint8)
    nc, nb = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = _load().fa_oracle_absorb(_p(codes), R, C, C, _p(mask), C, _p(w), C, _p(a), C, _p(out),
                                  _p(st), ctypes.byref(nc), ctypes.byref(nb))
    if rc:
        raise MemoryError("oracle: allocation failed")
    return Result(out, st, nc.value, nb.value)


def adjoint(codes, g, mask=None) -> Result:
    """lam = (I - P)^-T g: sum of g along each cell's downstream path, FP64."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    g = np.ascontiguousarray(g, dtype=np.float32)
    if g.shape != codes.shape:
        raise ValueError("g shape differs from codes")
    out = np.empty((R, C), dtype=np.float64)
    st = np.empty((R, C), dtype=np.uint8)
    nc, nb = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = _load().fa_oracle_adjoint(_p(codes), R, C, C, _p(mask), C, _p(g), C, _p(out), _p(st),
                                   ctypes.byref(nc), ctypes.byref(nb))
    if rc:
        raise MemoryError("oracle: allocation failed")
    return Result(out, st, nc.value, nb.value)


def bruteforce(codes, w=None, mask=None) -> Result:
    """Every valid cell adds its weight to each cell on its downstream path."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    out = np.empty((R, C), dtype=np.float64)
    st = np.empty((R, C), dtype=np.uint8)
    _load().fa_oracle_bruteforce(_p(codes), R, C, C, _p(mask), C, _p(w), C, _p(out), _p(st))
    return Result(out, st, int((st == 2).sum()), int((codes > 9).sum()))


def residual_u32(codes, A, mask=None):
    """(mismatches, first_index) of the Eq. 1 residual check on uint32 counts."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    A = np.ascontiguousarray(A, dtype=np.uint32)
    first = ctypes.c_int64(-1)
    bad = _load().fa_oracle_residual_u32(_p(codes), R, C, C, _p(mask), C, _p(A), C,
                                         ctypes.byref(first))
    return int(bad), int(first.value)


def residual_u32_rows(codes, A, r_begin: int, r_end: int, mask=None):
    """The Eq. 1 residual check of residual_u32 on rows r_begin..r_end-1 only
    (neighbours read from the whole raster): (mismatches, first_index)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    A = np.ascontiguousarray(A, dtype=np.uint32)
    first = ctypes.c_int64(-1)
    bad = _load().fa_oracle_residual_u32_rows(_p(codes), R, C, C, _p(mask), C, _p(A), C,
                                              int(r_begin), int(r_end), ctypes.byref(first))
    return int(bad), int(first.value)


def outlet_sum_u32(codes, A, r_begin: int = 0, r_end: int | None = None, mask=None):
    """Conservation on rows r_begin..r_end-1: (sum of A over terminal cells,
    number of valid cells).  Over a whole acyclic raster with unit weights
    they are equal (modulo 2^32 if a count wrapped)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    A = np.ascontiguousarray(A, dtype=np.uint32)
    s, nv = ctypes.c_uint64(0), ctypes.c_int64(0)
    _load().fa_oracle_outlet_sum_u32(_p(codes), R, C, C, _p(mask), C, _p(A), C, int(r_begin),
                                     int(R if r_end is None else r_end), ctypes.byref(s),
                                     ctypes.byref(nv))
    return int(s.value), int(nv.value)


def residual_u64_rows(codes, A, r_begin: int, r_end: int, mask=None):
    """The Eq. 1 residual check on uint64 counts (exact, no wrap-around) on
    rows r_begin..r_end-1: (mismatches, first_index)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    A = np.ascontiguousarray(A).view(np.uint64)
    first = ctypes.c_int64(-1)
    bad = _load().fa_oracle_residual_u64_rows(_p(codes), R, C, C, _p(mask), C, _p(A), C,
                                              int(r_begin), int(r_end), ctypes.byref(first))
    return int(bad), int(first.value)


def outlet_sum_u64(codes, A, r_begin: int = 0, r_end: int | None = None, mask=None):
    """Conservation on rows r_begin..r_end-1 for uint64 counts: (sum of A over
    terminal cells, number of valid cells)."""
    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    A = np.ascontiguousarray(A).view(np.uint64)
    s, nv = ctypes.c_uint64(0), ctypes.c_int64(0)
    _load().fa_oracle_outlet_sum_u64(_p(codes), R, C, C, _p(mask), C, _p(A), C, int(r_begin),
                                     int(R if r_end is None else r_end), ctypes.byref(s),
                                     ctypes.byref(nv))
    return int(s.value), int(nv.value)


def upstream_sums(codes, cells, w=None, mask=None, threads: int = 1):
    """Eq. 1's solution at the given flat cell indices (r * cols + c), each
    from its upstream area gathered by a search against the flow: (FP64
    values, area sizes); size -1 (value NaN) marks a cell on a cycle.  Work
    is the total size of the areas, so it suits samples of a raster of any
    size; queries are split over `threads` host threads."""
    from concurrent.futures import ThreadPoolExecutor

    codes, mask = _prep(codes, mask)
    R, C = codes.shape
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float32)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty(cells.size, dtype=np.float64)
    size = np.empty(cells.size, dtype=np.int64)
    lib = _load()
    chunks = np.array_split(np.arange(cells.size), max(1, min(threads, cells.size)))

    def one(ix):
        if ix.size == 0:
            return 0
        lo = int(ix[0])
        n = lib.fa_oracle_upstream_sums(
            _p(codes), R, C, C, _p(mask), C, _p(w), C,
            ctypes.c_void_p(cells.ctypes.data + 8 * lo), int(ix.size),
            ctypes.c_void_p(out.ctypes.data + 8 * lo), ctypes.c_void_p(size.ctypes.data + 8 * lo))
        if n < 0:
            raise MemoryError("upstream_sums: stack allocation failed")
        return n

    with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
        list(ex.map(one, chunks))
    return out, size


def verify_counts_u32(codes, A, threads: int = 1, band: int = 1024, mask=None):
    """Complete check of uint32 counts (uint64 when A holds 64-bit integers)
    on an acyclic raster of any size: the Eq. 1 residual at every cell and
    conservation, over row bands in a pool of host threads (the C calls
    release the interpreter lock).  Returns a dict with mismatches, first
    mismatching index, outlet sum, valid cells and whether conservation holds
    exactly and modulo 2^32."""
    from concurrent.futures import ThreadPoolExecutor

    codes, mask = _prep(codes, mask)
    wide = np.asarray(A).dtype.itemsize == 8
    A = np.ascontiguousarray(A).view(np.uint64) if wide else np.ascontiguousarray(A, dtype=np.uint32)
    res_rows = residual_u64_rows if wide else residual_u32_rows
    osum = outlet_sum_u64 if wide else outlet_sum_u32
    R = codes.shape[0]
    bands = [(r, min(R, r + band)) for r in range(0, R, band)]

    def one(b):
        bad, f = res_rows(codes, A, b[0], b[1], mask)
        s, nv = osum(codes, A, b[0], b[1], mask)
        return bad, f, s, nv

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        res = list(ex.map(one, bands))
    bad = sum(r[0] for r in res)
    firsts = [r[1] for r in res if r[1] >= 0]
    s = sum(r[2] for r in res)
    nv = sum(r[3] for r in res)
    return {"mismatches": bad, "first": min(firsts) if firsts else -1, "outlet_sum": s,
            "n_valid": nv, "conserved": s == nv, "conserved_mod_2_32": (s - nv) % (1 << 32) == 0}


def d8(z, nodata=None) -> np.ndarray:
    """D8 codes (uint8) from float32 elevations z; nodata: bool/uint8 mask or None.
    Rules in fa_oracle.c (fa_oracle_d8)."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.float32)
    rows, cols = z.shape
    out = np.zeros((rows, cols), dtype=np.uint8)
    nd = None if nodata is None else np.ascontiguousarray(nodata, dtype=np.uint8)
    lib.fa_oracle_d8(_p(z), rows, cols, cols, None if nd is None else _p(nd), cols, _p(out))
    return out


def unpack_nibbles(packed, cols: int) -> np.ndarray:
    """One code per cell from codes stored two per byte.  Section 4 notes that
    the ten code values fit in half a byte; the stored layout (the library's
    packed format) puts cell c of a row in byte c // 2, in the low four bits
    when c is even and the high four bits when c is odd."""
    p = np.asarray(packed, dtype=np.uint8)
    rows = p.shape[0]
    out = np.zeros((rows, cols), dtype=np.uint8)
    for c in range(cols):
        byte = p[:, c // 2]
        out[:, c] = (byte & 0x0F) if c % 2 == 0 else (byte >> 4)
    return out


def recode(codes, table) -> np.ndarray:
    """Codes of another scheme translated cell by cell: value v becomes
    table[v] (a 256-entry table)."""
    t = np.frombuffer(bytes(bytearray(table)), dtype=np.uint8)
    if t.size != 256:
        raise ValueError("a code table has 256 entries")
    c = np.asarray(codes, dtype=np.uint8)
    return t[c]
