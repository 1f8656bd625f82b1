"""GB300 (sm_103a) D8 flow accumulation.

Thin binding over the C ABI of libfa.so (include/fa.h).  The ``fa_*``
functions carry the C names and only marshal arguments: torch tensors supply
device memory and the current CUDA stream; every step of the computation runs
in the library's CUDA kernels.  ``accumulate`` is a convenience wrapper that
also allocates the output and a cached workspace.

Flow accumulation (the paper's Eq. 1 with alpha in {0,1}): for every valid
cell p, A(p) = w(p) + sum of A(n) over neighbours n that drain into p.
Besides the plain form: batches (accumulate_batched, BatchPlan), the adjoint
(adjoint, FlowAccumulate), absorption (absorb: Eq. 1 with one factor per
cell), D8 codes from elevations (d8_codes), packed and translated codes
(PackedCodes, pack_codes, recode) and the tile-shape autotuner (autotune).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (FA_ERR_BAD_CODE, FA_ERR_CUDA, FA_ERR_CYCLE, FA_ERR_INVALID_ARG,  # noqa: F401
                   FA_ERR_NONFINITE, FA_ERR_TIMEOUT, FA_ERR_TOO_LARGE, FA_ERR_WORKSPACE,
                   FA_NOALLOC_SCRATCH_BYTES, FA_OK, FA_OPT_NO_TMA, FA_OUT_F32, FA_OUT_U32,
                   FA_CODES_BYTE, FA_CODES_NIBBLE,
                   FA_STATUS_WORDS,
                   FA_WARN_OVERFLOW, STATUS_NAMES, fa_options, fa_raster, FA_MAX_FIELDS)

__all__ = ["fa_version", "fa_workspace_size", "fa_kernel_launches", "fa_accumulate",
           "fa_batched_workspace_size", "fa_accumulate_batched", "fa_batched_plan_create",
           "fa_plan_launch", "fa_plan_destroy", "accumulate_batched", "BatchPlan",
           "fa_accumulate_noalloc", "fa_accumulate_adjoint", "fa_status_read", "adjoint", "FlowAccumulate",
           "fa_timing_enable", "fa_timing_read", "accumulate", "fa_selftest_wait_timeout",
           "fa_autotune_workspace_size", "fa_autotune", "fa_autotune_batched_workspace_size",
           "fa_autotune_batched", "autotune", "autotune_batched", "fa_d8_codes", "d8_codes",
           "fa_recode", "recode", "pack_codes", "PackedCodes", "power_of_two_table",
           "fa_absorb_workspace_size", "fa_accumulate_absorb", "absorb",
           "fa_ooc_workspace_size", "fa_accumulate_ooc", "accumulate_ooc",
           "fa_shard_geometry", "fa_shard_export", "fa_shard_resolve", "fa_shard_finish",
           "FlowAccError", "options"]


class FlowAccError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


def options(tile=None, flags: int = 0, code_format: int = FA_CODES_BYTE) -> fa_options:
    o = fa_options()
    if tile is not None:
        o.tile_h, o.tile_w = int(tile[0]), int(tile[1])
    o.flags = int(flags)
    o.code_format = int(code_format)
    return o


class PackedCodes:
    """D8 codes packed two per byte (FA_CODES_NIBBLE): the code of cell (r, c)
    is in data[r, c // 2], low four bits for even c, high four bits for odd c.
    data: uint8 CUDA tensor [R, >= (cols + 1) // 2] with unit column stride.
    Accepted wherever byte codes are; the calls set code_format themselves."""

    def __init__(self, data: torch.Tensor, cols: int):
        if data.dtype != torch.uint8 or data.dim() != 2:
            raise TypeError("packed codes must be a 2-D uint8 tensor")
        if cols < 0 or data.shape[1] < (cols + 1) // 2:
            raise ValueError("packed codes hold fewer than (cols + 1) // 2 bytes per row")
        self.data = data
        self.cols = int(cols)

    @property
    def shape(self):
        return (self.data.shape[0], self.cols)

    @property
    def device(self):
        return self.data.device

    @property
    def is_cuda(self):
        return self.data.is_cuda

    @property
    def dtype(self):
        return self.data.dtype

    def data_ptr(self):
        return self.data.data_ptr()


def _with_format(codes, opts):
    """A copy of opts whose code_format matches the type of `codes`."""
    o = fa_options()
    if opts is not None:
        o.tile_h, o.tile_w, o.flags, o.code_format = opts.tile_h, opts.tile_w, opts.flags, opts.code_format
    if isinstance(codes, PackedCodes):
        o.code_format = FA_CODES_NIBBLE
    return o


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _pitch(t):
    if t is None:
        return 0
    if isinstance(t, PackedCodes):
        t = t.data
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("rasters must be 2-D with unit column stride")
    return t.stride(0)


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def fa_version() -> int:
    return _lib.load().fa_version()


def fa_workspace_size(rows: int, cols: int, opts: fa_options | None = None) -> int:
    return _lib.load().fa_workspace_size(rows, cols, ctypes.byref(opts or fa_options()))


def fa_kernel_launches(rows: int, cols: int, opts: fa_options | None = None) -> int:
    return _lib.load().fa_kernel_launches(rows, cols, ctypes.byref(opts or fa_options()))


def fa_accumulate(codes, weights, mask, out, out_dtype, workspace, opts=None, d_status=None,
                  stream=None) -> int:
    """Enqueue fa_accumulate on the current (or given) stream; returns the
    host-side status code.  All tensors are CUDA tensors."""
    rows, cols = codes.shape
    return _lib.load().fa_accumulate(
        _ptr(codes), rows, cols, _pitch(codes), _ptr(weights), _pitch(weights), _ptr(mask),
        _pitch(mask), _ptr(out), out_dtype, _pitch(out), _ptr(workspace), workspace.numel(),
        ctypes.byref(_with_format(codes, opts)), _ptr(d_status), _stream_ptr(stream))


def fa_accumulate_noalloc(codes, weights, mask, out, out_dtype, opts=None, d_status=None,
                          stream=None) -> int:
    """Enqueue fa_accumulate_noalloc: fa_accumulate without a workspace, for
    callers that cannot allocate device memory; scratch comes from a fixed
    buffer inside the library (FA_NOALLOC_SCRATCH_BYTES), shared by all calls
    on a device, so overlapping calls race.  Returns the host-side status."""
    rows, cols = codes.shape
    return _lib.load().fa_accumulate_noalloc(
        _ptr(codes), rows, cols, _pitch(codes), _ptr(weights), _pitch(weights), _ptr(mask),
        _pitch(mask), _ptr(out), out_dtype, _pitch(out), ctypes.byref(_with_format(codes, opts)),
        _ptr(d_status), _stream_ptr(stream))


def fa_accumulate_adjoint(codes, mask, grad_out, grad_w, workspace, opts=None, d_status=None,
                          stream=None) -> int:
    """Enqueue fa_accumulate_adjoint: grad_w = (I - P)^-T grad_out."""
    rows, cols = codes.shape
    return _lib.load().fa_accumulate_adjoint(
        _ptr(codes), rows, cols, _pitch(codes), _ptr(mask), _pitch(mask), _ptr(grad_out),
        _pitch(grad_out), _ptr(grad_w), _pitch(grad_w), _ptr(workspace), workspace.numel(),
        ctypes.byref(_with_format(codes, opts)), _ptr(d_status), _stream_ptr(stream))


def fa_ooc_workspace_size(rows: int, cols: int, block_rows: int = 0, block_cols: int = 0,
                          opts: fa_options | None = None) -> int:
    return _lib.load().fa_ooc_workspace_size(rows, cols, block_rows, block_cols,
                                             ctypes.byref(opts or fa_options()))


def fa_accumulate_ooc(codes, out, block_rows, block_cols, workspace, opts=None, d_status=None,
                      stream=None) -> int:
    """fa_accumulate_ooc: uint64 counts of a raster in HOST memory (codes:
    uint8 [R, C] CPU tensor, out: int64/uint64 [R, C] CPU tensor), solved on
    the device block by block; synchronous, returns the decoded status."""
    rows, cols = codes.shape
    if codes.is_cuda or out.is_cuda:
        raise TypeError("fa_accumulate_ooc takes host (CPU) tensors")
    if out.element_size() != 8:
        raise TypeError("out must be a 64-bit integer tensor")
    empty = rows == 0 or cols == 0
    return _lib.load().fa_accumulate_ooc(
        None if empty else _ptr(codes), rows, cols, cols if empty else _pitch(codes),
        None if empty else _ptr(out), cols if empty else _pitch(out), block_rows, block_cols,
        _ptr(workspace), workspace.numel(), ctypes.byref(opts or fa_options()), _ptr(d_status),
        _stream_ptr(stream))


def _host(t, what):
    if t is not None and t.is_cuda:
        raise TypeError(f"{what} must be a host (CPU) tensor")
    return t


def fa_shard_geometry(rows: int, cols: int, block_rows: int = 0, block_cols: int = 0):
    """fa_shard_geometry -> (status, nby, nbx, pmax): the outer block grid of
    the shard form and the record slots per block."""
    grid = (ctypes.c_int64 * 2)()
    pmax = ctypes.c_int32(0)
    st = _lib.load().fa_shard_geometry(rows, cols, block_rows, block_cols, grid, ctypes.byref(pmax))
    return st, grid[0], grid[1], pmax.value


def fa_shard_export(codes, codes_row0, rows, cols, block_rows, block_cols, band0, band1, nexit, link,
                    node_dst, node_val, workspace, opts=None, d_status=None, stream=None) -> int:
    """fa_shard_export: pass A on the blocks of block rows [band0, band1).
    codes: uint8 CPU tensor holding raster rows codes_row0 .. (the band and
    its ring rows); nexit (32-bit), link (16-bit), node_dst (32-bit) and
    node_val (float64): CPU tensors receiving the band's records."""
    for t, what in ((codes, "codes"), (nexit, "nexit"), (link, "link"), (node_dst, "node_dst"),
                    (node_val, "node_val")):
        _host(t, what)
    return _lib.load().fa_shard_export(
        _ptr(codes), codes_row0, codes.shape[0], _pitch(codes), rows, cols, block_rows, block_cols,
        band0, band1, _ptr(nexit), _ptr(link), _ptr(node_dst), _ptr(node_val), _ptr(workspace),
        workspace.numel(), ctypes.byref(opts or fa_options()), _ptr(d_status), _stream_ptr(stream))


def fa_shard_resolve(rows, cols, block_rows, block_cols, nexit, link, node_dst, node_val, inflow,
                     workspace, d_status=None, stream=None) -> int:
    """fa_shard_resolve: the records of all blocks (CPU tensors) -> inflow
    (64-bit CPU tensor, one value per block perimeter slot)."""
    for t, what in ((nexit, "nexit"), (link, "link"), (node_dst, "node_dst"),
                    (node_val, "node_val"), (inflow, "inflow")):
        _host(t, what)
    return _lib.load().fa_shard_resolve(
        rows, cols, block_rows, block_cols, _ptr(nexit), _ptr(link), _ptr(node_dst), _ptr(node_val),
        _ptr(inflow), _ptr(workspace), workspace.numel(), _ptr(d_status), _stream_ptr(stream))


def fa_shard_finish(codes, codes_row0, rows, cols, block_rows, block_cols, band0, band1, inflow,
                    out, workspace, opts=None, d_status=None, stream=None) -> int:
    """fa_shard_finish: pass C on the blocks of block rows [band0, band1) with
    the band's in(p) (64-bit CPU tensor); out: 64-bit CPU tensor of the
    band's raster rows."""
    for t, what in ((codes, "codes"), (inflow, "inflow"), (out, "out")):
        _host(t, what)
    if out.element_size() != 8:
        raise TypeError("out must be a 64-bit integer tensor")
    return _lib.load().fa_shard_finish(
        _ptr(codes), codes_row0, codes.shape[0], _pitch(codes), rows, cols, block_rows, block_cols,
        band0, band1, _ptr(inflow), _ptr(out), _pitch(out), _ptr(workspace), workspace.numel(),
        ctypes.byref(opts or fa_options()), _ptr(d_status), _stream_ptr(stream))


def fa_absorb_workspace_size(rows: int, cols: int, opts: fa_options | None = None) -> int:
    return _lib.load().fa_absorb_workspace_size(rows, cols, ctypes.byref(opts or fa_options()))


def fa_accumulate_absorb(codes, weights, factors, mask, out, workspace, opts=None, d_status=None,
                         stream=None) -> int:
    """Enqueue fa_accumulate_absorb: A(p) = w(p) + sum of a(n) A(n) over the
    cells n draining into p (float32 out)."""
    rows, cols = codes.shape
    return _lib.load().fa_accumulate_absorb(
        _ptr(codes), rows, cols, _pitch(codes), _ptr(weights), _pitch(weights), _ptr(factors),
        _pitch(factors), _ptr(mask), _pitch(mask), _ptr(out), _pitch(out), _ptr(workspace),
        workspace.numel(), ctypes.byref(_with_format(codes, opts)), _ptr(d_status),
        _stream_ptr(stream))


def fa_d8_codes(dem, nodata, codes, stream=None) -> int:
    """Enqueue fa_d8_codes: uint8 D8 codes from float32 elevations."""
    rows, cols = dem.shape
    return _lib.load().fa_d8_codes(_ptr(dem), rows, cols, _pitch(dem), _ptr(nodata), _pitch(nodata),
                                   _ptr(codes), _pitch(codes), _stream_ptr(stream))


def fa_recode(src, table, dst, dst_format: int, cols: int | None = None, stream=None) -> int:
    """Enqueue fa_recode: src uint8 [R, C] codes through a 256-byte table (or
    None) into dst (bytes, or packed codes when dst_format is FA_CODES_NIBBLE;
    cols defaults to src's width)."""
    rows, c = src.shape
    cols = c if cols is None else cols
    tab = None
    if table is not None:
        tb = bytes(bytearray(table))
        if len(tb) != 256:
            raise ValueError("a code table has 256 entries")
        tab = (ctypes.c_uint8 * 256).from_buffer_copy(tb)
    return _lib.load().fa_recode(_ptr(src), rows, cols, _pitch(src), tab, _ptr(dst), _pitch(dst),
                                 int(dst_format), _stream_ptr(stream))


def fa_autotune_workspace_size(rows: int, cols: int, opts: fa_options | None = None) -> int:
    return _lib.load().fa_autotune_workspace_size(rows, cols, ctypes.byref(opts or fa_options()))


def fa_autotune(codes, weights, mask, out, out_dtype, workspace, opts=None, stream=None):
    """Run fa_autotune; returns (status, fa_options of the fastest shape)."""
    rows, cols = codes.shape
    best = fa_options()
    st = _lib.load().fa_autotune(
        _ptr(codes), rows, cols, _pitch(codes), _ptr(weights), _pitch(weights), _ptr(mask),
        _pitch(mask), _ptr(out), out_dtype, _pitch(out), _ptr(workspace), workspace.numel(),
        ctypes.byref(_with_format(codes, opts)), _stream_ptr(stream), ctypes.byref(best))
    return st, best


def fa_autotune_batched_workspace_size(rasters, n_fields: int, opts=None) -> int:
    arr = (fa_raster * max(1, len(rasters)))(*rasters)
    return _lib.load().fa_autotune_batched_workspace_size(arr, len(rasters), n_fields,
                                                          ctypes.byref(opts or fa_options()))


def fa_autotune_batched(rasters, n_fields: int, workspace, opts=None, stream=None):
    """Run fa_autotune_batched; returns (status, fa_options of the fastest shape)."""
    arr = (fa_raster * max(1, len(rasters)))(*rasters)
    best = fa_options()
    st = _lib.load().fa_autotune_batched(arr, len(rasters), n_fields, _ptr(workspace),
                                         workspace.numel(), ctypes.byref(opts or fa_options()),
                                         _stream_ptr(stream), ctypes.byref(best))
    return st, best


def fa_batched_workspace_size(rasters, n_fields: int, opts: fa_options | None = None) -> int:
    arr = (fa_raster * max(1, len(rasters)))(*rasters)
    return _lib.load().fa_batched_workspace_size(arr, len(rasters), n_fields,
                                                 ctypes.byref(opts or fa_options()))


def fa_accumulate_batched(rasters, n_fields: int, workspace, opts=None, d_status=None,
                          stream=None) -> int:
    """Enqueue fa_accumulate_batched over a list of fa_raster descriptors."""
    arr = (fa_raster * max(1, len(rasters)))(*rasters)
    return _lib.load().fa_accumulate_batched(arr, len(rasters), n_fields, _ptr(workspace),
                                             workspace.numel(), ctypes.byref(opts or fa_options()),
                                             _ptr(d_status), _stream_ptr(stream))


def fa_batched_plan_create(rasters, n_fields: int, workspace, opts=None, d_status=None,
                           stream=None):
    """Capture a batch in a CUDA graph; returns (status, plan handle)."""
    arr = (fa_raster * max(1, len(rasters)))(*rasters)
    h = ctypes.c_void_p()
    st = _lib.load().fa_batched_plan_create(arr, len(rasters), n_fields, _ptr(workspace),
                                            workspace.numel(), ctypes.byref(opts or fa_options()),
                                            _ptr(d_status), _stream_ptr(stream), ctypes.byref(h))
    return st, h


def fa_plan_launch(plan, stream=None) -> int:
    return _lib.load().fa_plan_launch(plan, _stream_ptr(stream))


def fa_plan_destroy(plan) -> None:
    _lib.load().fa_plan_destroy(plan)


def fa_status_read(d_status=None, workspace=None, stream=None):
    """Synchronise the stream and read the device status block back:
    returns (status, count, first_index)."""
    cnt, first = ctypes.c_int64(0), ctypes.c_int64(-1)
    st = _lib.load().fa_status_read(_ptr(d_status), _ptr(workspace), _stream_ptr(stream),
                                    ctypes.byref(cnt), ctypes.byref(first))
    return st, cnt.value, first.value


def fa_selftest_wait_timeout(limit_ns: int, d_status, stream=None) -> int:
    """Enqueue the bounded-wait self-test: one device wait that can never
    complete gives up after limit_ns and records FA_FLAG_TIMEOUT in d_status
    (read it back with fa_status_read).  Returns the host-side status."""
    return _lib.load().fa_selftest_wait_timeout(int(limit_ns), _ptr(d_status),
                                                _stream_ptr(stream))


def fa_timing_enable(on: bool) -> None:
    _lib.load().fa_timing_enable(1 if on else 0)


def fa_timing_read(n: int = 8):
    """Phase durations (ms) of the most recent call made while timing was on."""
    buf = (ctypes.c_float * n)()
    m = _lib.load().fa_timing_read(buf, n)
    if m < 0:
        raise FlowAccError(FA_ERR_CUDA, "fa_timing_read")
    return [float(buf[i]) for i in range(m)]


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
_ws_cache: dict = {}


def workspace(nbytes: int, device) -> torch.Tensor:
    """A cached uint8 workspace of at least nbytes on `device` (torch memory).
    accumulate, absorb, adjoint and autotune share this one buffer per device,
    so their calls must not overlap on the GPU: issue them on one stream, or
    give concurrent calls their own workspaces through the fa_* functions."""
    key = torch.device(device)
    if key.type == "cuda" and key.index is None:  # "cuda" and "cuda:N" share one buffer
        key = torch.device("cuda", torch.cuda.current_device())
    ws = _ws_cache.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=key)
        _ws_cache[key] = ws
    return ws


def d8_codes(dem: torch.Tensor, nodata: torch.Tensor | None = None, out=None, stream=None):
    """D8 codes (uint8 [R, C]) from float32 elevations on the device; nodata:
    uint8 [R, C] or None."""
    if dem.dtype != torch.float32 or not dem.is_cuda:
        raise TypeError("dem must be a float32 CUDA tensor")
    if out is None:
        out = torch.empty(dem.shape, dtype=torch.uint8, device=dem.device)
    st = fa_d8_codes(dem, nodata, out, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_d8_codes")
    return out


def power_of_two_table() -> bytes:
    """A code table (for recode / fa_recode) from the one-bit-per-direction
    scheme 1 = E, 2 = SE, 4 = S, 8 = SW, 16 = W, 32 = NW, 64 = N, 128 = NE to
    this library's codes; 0 stays NoData and every other value becomes 10
    (invalid: reported as FA_ERR_BAD_CODE and treated as NoData)."""
    t = bytearray([10] * 256)
    t[0] = 0
    for bit, code in ((1, 1), (2, 8), (4, 7), (8, 6), (16, 5), (32, 4), (64, 3), (128, 2)):
        t[bit] = code
    return bytes(t)


def recode(src: torch.Tensor, table=None, packed: bool = False, out=None, stream=None):
    """src uint8 [R, C] codes translated through a 256-entry table (None keeps
    the values): a uint8 [R, C] tensor, or PackedCodes when packed=True."""
    if src.dtype != torch.uint8 or not src.is_cuda:
        raise TypeError("src must be a uint8 CUDA tensor")
    R, C = src.shape
    if packed:
        if out is None:
            out = PackedCodes(torch.empty((R, (C + 1) // 2), dtype=torch.uint8, device=src.device), C)
        dst, fmt = out.data, FA_CODES_NIBBLE
    else:
        if out is None:
            out = torch.empty((R, C), dtype=torch.uint8, device=src.device)
        dst, fmt = out, FA_CODES_BYTE
    st = fa_recode(src, table, dst, fmt, C, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_recode")
    return out


def pack_codes(codes: torch.Tensor, table=None, stream=None) -> PackedCodes:
    """Byte codes (optionally through a table) packed two per byte."""
    return recode(codes, table, packed=True, stream=stream)


_tile_cache: dict = {}


def autotune(codes: torch.Tensor, weights: torch.Tensor | None = None,
             mask: torch.Tensor | None = None, stream=None):
    """The fastest tile shape for this raster (fa_autotune on the given inputs),
    remembered per (device, shape, weighted, masked) for tile="auto"."""
    R, C = codes.shape
    key = (codes.device, R, C, weights is not None, mask is not None, isinstance(codes, PackedCodes))
    if key not in _tile_cache:
        out_dtype = FA_OUT_U32 if weights is None else FA_OUT_F32
        out = torch.empty((R, C), dtype=torch.uint32 if weights is None else torch.float32,
                          device=codes.device)
        ws = workspace(fa_autotune_workspace_size(R, C), codes.device)
        st, best = fa_autotune(codes, weights, mask, out, out_dtype, ws, None, stream)
        if st != FA_OK:
            raise FlowAccError(st, "fa_autotune")
        _tile_cache[key] = (best.tile_h, best.tile_w)
    return _tile_cache[key]


def accumulate(codes: torch.Tensor, weights: torch.Tensor | None = None,
               mask: torch.Tensor | None = None, out_dtype=None, tile=None,
               out: torch.Tensor | None = None, check: bool = False, stream=None, flags: int = 0):
    """Flow accumulation of one raster.  codes: uint8 [R, C] CUDA tensor or
    PackedCodes; weights: float32 [R, C] or None (counts); mask: uint8 [R, C]
    or None.
    Returns uint32 counts (no weights, default) or float32 sums.  tile: None
    (64 x 64), (h, w), or "auto" (autotune() once per raster shape).
    check=True synchronises and raises FlowAccError on any device-reported
    error."""
    if codes.dtype != torch.uint8 or not codes.is_cuda:
        raise TypeError("codes must be a uint8 CUDA tensor")
    if isinstance(tile, str):
        if tile != "auto":
            raise ValueError("tile must be None, (h, w) or 'auto'")
        tile = autotune(codes, weights, mask, stream)
    if out_dtype is None:
        out_dtype = FA_OUT_U32 if weights is None else FA_OUT_F32
    R, C = codes.shape
    if out is None:
        out = torch.empty((R, C), dtype=torch.uint32 if out_dtype == FA_OUT_U32 else torch.float32,
                          device=codes.device)
    opts = options(tile, flags)
    ws = workspace(fa_workspace_size(R, C, opts), codes.device)
    st = fa_accumulate(codes, weights, mask, out, out_dtype, ws, opts, None, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_accumulate")
    if check:
        st, _, _ = fa_status_read(None, ws, stream)
        if st < 0:
            raise FlowAccError(st, "fa_accumulate (device)")
    return out


def accumulate_ooc(codes, block=None, tile=None, out=None, device=None, stream=None,
                   check: bool = True):
    """Counts of a raster held in host memory (uint8 [R, C] CPU tensor or
    numpy array), solved on `device` one outer block at a time (block: None =
    16384 x 16384, or (h, w)).  Returns uint64 counts as an int64 CPU tensor
    (bit pattern of the uint64; counts stay below 2^63).  check=True raises
    FlowAccError on any device-reported error."""
    if not isinstance(codes, torch.Tensor):
        codes = torch.from_numpy(codes)
    if codes.dtype != torch.uint8 or codes.is_cuda or codes.dim() != 2:
        raise TypeError("codes must be a 2-D uint8 host tensor")
    R, C = codes.shape
    if out is None:
        out = torch.empty((R, C), dtype=torch.int64)
    bh, bw = block if block is not None else (0, 0)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    opts = options(tile)
    n = fa_ooc_workspace_size(R, C, bh, bw, opts)
    if n == 0:
        raise FlowAccError(FA_ERR_INVALID_ARG, "fa_ooc_workspace_size")
    ws = workspace(n, dev)
    st = fa_accumulate_ooc(codes, out, bh, bw, ws, opts, None, stream)
    if st not in (FA_OK, FA_WARN_OVERFLOW) and (check or st in (FA_ERR_INVALID_ARG, FA_ERR_WORKSPACE, FA_ERR_CUDA)):
        raise FlowAccError(st, "fa_accumulate_ooc")
    return out


def adjoint(codes: torch.Tensor, grad_out: torch.Tensor, mask: torch.Tensor | None = None,
            tile=None, out: torch.Tensor | None = None, check: bool = False, stream=None):
    """dL/dw for dL/dA = grad_out: the sum of grad_out along each cell's
    downstream path (float32)."""
    if grad_out.dtype != torch.float32:
        raise TypeError("grad_out must be float32")
    R, C = codes.shape
    if out is None:
        out = torch.empty((R, C), dtype=torch.float32, device=codes.device)
    opts = options(tile)
    ws = workspace(fa_workspace_size(R, C, opts), codes.device)
    st = fa_accumulate_adjoint(codes, mask, grad_out, out, ws, opts, None, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_accumulate_adjoint")
    if check:
        st, _, _ = fa_status_read(None, ws, stream)
        if st < 0:
            raise FlowAccError(st, "fa_accumulate_adjoint (device)")
    return out


def absorb(codes, factors: torch.Tensor, weights: torch.Tensor | None = None,
           mask: torch.Tensor | None = None, tile=None, out: torch.Tensor | None = None,
           check: bool = False, stream=None):
    """Accumulation with absorption: every cell n passes the fraction
    factors[n] (float32 in [0, 1]) of its accumulated flow downstream.
    codes: uint8 [R, C] or PackedCodes; weights: float32 or None (unit).
    Returns float32 [R, C]."""
    if factors.dtype != torch.float32:
        raise TypeError("factors must be float32")
    R, C = codes.shape
    if out is None:
        out = torch.empty((R, C), dtype=torch.float32, device=codes.device)
    opts = options(tile)
    ws = workspace(fa_absorb_workspace_size(R, C, opts), codes.device)
    st = fa_accumulate_absorb(codes, weights, factors, mask, out, ws, opts, None, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_accumulate_absorb")
    if check:
        st, _, _ = fa_status_read(None, ws, stream)
        if st < 0:
            raise FlowAccError(st, "fa_accumulate_absorb (device)")
    return out


class FlowAccumulate(torch.autograd.Function):
    """A = accumulation of weights w over the D8 codes; differentiable in w.
    forward: fa_accumulate (float32); backward: fa_accumulate_adjoint."""

    @staticmethod
    def forward(ctx, weights, codes, mask=None, tile=None):
        raw = codes.data if isinstance(codes, PackedCodes) else codes
        ctx.save_for_backward(raw, mask) if mask is not None else ctx.save_for_backward(raw)
        ctx.packed_cols = codes.cols if isinstance(codes, PackedCodes) else None
        ctx.has_mask = mask is not None
        ctx.tile = tile
        return accumulate(codes, weights.contiguous(), mask, out_dtype=FA_OUT_F32, tile=tile)

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        codes = saved[0] if ctx.packed_cols is None else PackedCodes(saved[0], ctx.packed_cols)
        mask = saved[1] if ctx.has_mask else None
        gw = adjoint(codes, grad_out.contiguous().float(), mask, tile=ctx.tile)
        return gw, None, None, None


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------
def make_raster(codes: torch.Tensor, weights=None, outs=None, mask: torch.Tensor | None = None):
    """fa_raster for one raster: codes uint8 [R, C] (or PackedCodes, with the
    batch's code_format set to FA_CODES_NIBBLE); weights: list of float32
    [R, C] fields (or None for counts); outs: matching output tensors."""
    r = fa_raster()
    R, C = codes.shape
    r.codes, r.rows, r.cols, r.pitch_codes = codes.data_ptr(), R, C, _pitch(codes)
    if mask is not None:
        r.mask, r.pitch_mask = mask.data_ptr(), _pitch(mask)
    if weights:
        if len(weights) > FA_MAX_FIELDS:
            raise ValueError("too many fields")
        for k, w in enumerate(weights):
            r.weights[k] = w.data_ptr()
        r.pitch_w = _pitch(weights[0])
    for k, o in enumerate(outs):
        r.out[k] = o.data_ptr()
    r.pitch_out = _pitch(outs[0])
    return r


def _batch_outputs(items, n_fields):
    outs = []
    for it in items:
        codes = it["codes"]
        R, C = codes.shape
        if n_fields == 0:
            outs.append([torch.empty((R, C), dtype=torch.uint32, device=codes.device)])
        else:
            outs.append([torch.empty((R, C), dtype=torch.float32, device=codes.device)
                         for _ in range(n_fields)])
    return outs


def _batch_format(items) -> int:
    """The code format of a batch: all byte codes or all PackedCodes."""
    packed = {isinstance(it["codes"], PackedCodes) for it in items}
    if len(packed) > 1:
        raise ValueError("a batch holds either byte codes or packed codes, not both")
    return FA_CODES_NIBBLE if packed == {True} else FA_CODES_BYTE


def accumulate_batched(items, n_fields: int = 0, tile=None, check: bool = False, stream=None):
    """Flow accumulation of many rasters in one pass.  items: list of dicts with
    'codes' (uint8 [R, C]), optional 'weights' (list of n_fields float32 [R, C])
    and optional 'mask'.  Returns a list of output lists (uint32 counts when
    n_fields == 0, else n_fields float32 sums per raster)."""
    outs = _batch_outputs(items, n_fields)
    rasters = [make_raster(it["codes"], it.get("weights"), o, it.get("mask"))
               for it, o in zip(items, outs)]
    dev = items[0]["codes"].device if items else torch.device("cuda")
    if isinstance(tile, str):
        tile = autotune_batched(items, n_fields, stream)
    opts = options(tile, code_format=_batch_format(items))
    ws = workspace(fa_batched_workspace_size(rasters, n_fields, opts), dev)
    st = fa_accumulate_batched(rasters, n_fields, ws, opts, None, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_accumulate_batched")
    if check:
        st, _, _ = fa_status_read(None, ws, stream)
        if st < 0:
            raise FlowAccError(st, "fa_accumulate_batched (device)")
    return outs


def autotune_batched(items, n_fields: int = 0, stream=None):
    """The fastest tile shape for this batch (fa_autotune_batched on its inputs;
    outputs go to scratch tensors)."""
    outs = _batch_outputs(items, n_fields)
    rasters = [make_raster(it["codes"], it.get("weights"), o, it.get("mask"))
               for it, o in zip(items, outs)]
    dev = items[0]["codes"].device
    opts = options(code_format=_batch_format(items))
    ws = torch.empty(max(fa_autotune_batched_workspace_size(rasters, n_fields, opts), 1 << 20),
                     dtype=torch.uint8, device=dev)
    st, best = fa_autotune_batched(rasters, n_fields, ws, opts, stream)
    if st != FA_OK:
        raise FlowAccError(st, "fa_autotune_batched")
    return (best.tile_h, best.tile_w)


class BatchPlan:
    """A batch captured once in a CUDA graph; run() replays it.  Holds its
    own workspace, status block and output tensors.  tile: None (64 x 64),
    (h, w), or "auto" (autotune_batched first; the shape is kept in .tile)."""

    def __init__(self, items, n_fields: int = 0, tile=None, stream=None):
        self.items = items  # keep inputs alive
        if isinstance(tile, str):
            tile = autotune_batched(items, n_fields, stream)
        self.tile = tile
        self.outs = _batch_outputs(items, n_fields)
        rasters = [make_raster(it["codes"], it.get("weights"), o, it.get("mask"))
                   for it, o in zip(items, self.outs)]
        opts = options(tile, code_format=_batch_format(items))
        dev = items[0]["codes"].device
        self.ws = torch.empty(max(fa_batched_workspace_size(rasters, n_fields, opts), 1 << 20),
                              dtype=torch.uint8, device=dev)
        self.status = torch.zeros(FA_STATUS_WORDS, dtype=torch.int32, device=dev)
        st, self.handle = fa_batched_plan_create(rasters, n_fields, self.ws, opts, self.status,
                                                 stream)
        if st != FA_OK:
            raise FlowAccError(st, "fa_batched_plan_create")

    def run(self, stream=None):
        st = fa_plan_launch(self.handle, stream)
        if st != FA_OK:
            raise FlowAccError(st, "fa_plan_launch")
        return self.outs

    def status_read(self, stream=None):
        return fa_status_read(self.status, None, stream)

    def close(self):
        if self.handle:
            fa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from . import shard  # noqa: E402  (the multi-process form; uses the functions above)
