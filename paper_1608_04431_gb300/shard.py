"""Shard form across processes: the out-of-core stages split over ranks (one
per GPU), the paper's two MapReduces (Section 3, Algorithm 3; Section 4 on
the data sent).

Every rank owns a band of whole outer block rows.  It exports the perimeter
records of its blocks (pass A), rank 0 gathers the records of all blocks,
solves the blocks' perimeter graph (Section 3.2) and scatters to each rank
the flow entering its blocks, in(p) per block perimeter slot; every rank then
finishes its blocks (pass C) into uint64 counts of its rows.  Only records
and in(p) travel: 14 bytes per perimeter slot plus 4 per block up, 8 per slot
down.  The exchange is torch.distributed gather/scatter on host tensors (gloo,
or any backend that takes CPU tensors).

The stage calls are the C entry points fa_shard_export / fa_shard_resolve /
fa_shard_finish (DeviceStages); another object with the same three methods
can stand in for them, which is how the exchange is tested on CPU ranks.

Failures: a stage that raises on one rank (a bad argument, a CUDA error)
must not leave the others waiting in a collective, so after each stage the
ranks agree whether any of them failed (one small all-reduce or broadcast)
and all raise at the same point.  Conditions the device reports after a
completed stage (invalid codes, cycles) are combined over all ranks at the
end, so every rank returns or raises the same status.  A rank that dies
outright makes the others' next collective fail: at once where the backend
sees the connection close (gloo), at the latest after the process group's
timeout.

Checkpoints: with a checkpoint directory each rank keeps its records after
pass A and rank 0 keeps in(p) after the resolve, so that a solve stopped
later resumes at the finish (accumulate_sharded).
"""
from __future__ import annotations

import os
import zipfile

import numpy as np
import torch
import torch.distributed as dist

from . import (FA_ERR_BAD_CODE, FA_ERR_CYCLE, FA_ERR_INVALID_ARG, FA_ERR_NONFINITE, FA_ERR_TIMEOUT,
               FA_OK, FA_WARN_OVERFLOW, FlowAccError, fa_ooc_workspace_size, fa_shard_export,
               fa_shard_finish, fa_shard_geometry, fa_shard_resolve, options, workspace)

# statuses the device reports after a completed stage, least to most severe
# (the order fa_status_read uses); any other status is a failed call
_DEVICE_STATUS = [FA_OK, FA_WARN_OVERFLOW, FA_ERR_TIMEOUT, FA_ERR_NONFINITE, FA_ERR_CYCLE,
                  FA_ERR_BAD_CODE]


class ShardAborted(RuntimeError):
    """A stage failed on another rank; every rank stops at the same point."""


class Records:
    """Perimeter records of up to `cap` blocks in one uint8 host tensor (the
    unit the gather moves): node_val float64 [cap * pmax], node_dst 32-bit
    [cap * pmax], nexit 32-bit [cap], link 16-bit [cap * pmax], in that
    order.  The first `n` blocks are in use; views of their part are
    nexit(n), link(n), node_dst(n), node_val(n)."""

    def __init__(self, cap: int, pmax: int, buf: torch.Tensor | None = None):
        self.cap, self.pmax = int(cap), int(pmax)
        m = self.cap * self.pmax
        self._o_dst = 8 * m
        self._o_nexit = self._o_dst + 4 * m
        self._o_link = self._o_nexit + 4 * self.cap
        size = self._o_link + 2 * m
        if buf is None:
            buf = torch.zeros(size, dtype=torch.uint8)
        if buf.dtype != torch.uint8 or buf.numel() != size or buf.is_cuda:
            raise ValueError("records buffer must be a host uint8 tensor of the packed size")
        self.buf = buf

    @staticmethod
    def nbytes(cap: int, pmax: int) -> int:
        return 14 * cap * pmax + 4 * cap

    def node_val(self, n: int) -> torch.Tensor:
        return self.buf[: 8 * n * self.pmax].view(torch.float64)

    def node_dst(self, n: int) -> torch.Tensor:
        return self.buf[self._o_dst: self._o_dst + 4 * n * self.pmax].view(torch.int32)

    def nexit(self, n: int) -> torch.Tensor:
        return self.buf[self._o_nexit: self._o_nexit + 4 * n].view(torch.int32)

    def link(self, n: int) -> torch.Tensor:
        return self.buf[self._o_link: self._o_link + 2 * n * self.pmax].view(torch.int16)

    def put(self, at: int, other: "Records", n: int) -> None:
        """Copies the first n blocks of `other` to blocks at .. at + n - 1."""
        p = self.pmax
        self.node_val(at + n)[at * p:].copy_(other.node_val(n))
        self.node_dst(at + n)[at * p:].copy_(other.node_dst(n))
        self.nexit(at + n)[at:].copy_(other.nexit(n))
        self.link(at + n)[at * p:].copy_(other.link(n))


def _ckpt_save(path: str, arrays: dict, meta: dict) -> None:
    """Arrays plus integer metadata to an .npz file, written under another
    name first so that a crash mid-write leaves no file that looks whole."""
    tmp = path + ".part"
    with open(tmp, "wb") as f:
        np.savez(f, **arrays, **{"m_" + k: np.int64(v) for k, v in meta.items()})
    os.replace(tmp, path)


def _ckpt_load(path: str, meta: dict):
    """The arrays of a file written by _ckpt_save with the same metadata, or
    None (absent, unreadable or from another solve)."""
    try:
        with np.load(path) as z:
            if any(int(z["m_" + k]) != int(v) for k, v in meta.items()):
                return None
            return {k: z[k].copy() for k in z.files if not k.startswith("m_")}
    except (OSError, ValueError, KeyError, EOFError, zipfile.BadZipFile):
        return None


def bands(nby: int, world: int):
    """Block rows [band0, band1) of each rank: contiguous, sizes differing by
    at most one (a rank gets an empty band when world > nby)."""
    return [(r * nby // world, (r + 1) * nby // world) for r in range(world)]


def band_rows(band, block_rows: int, rows: int):
    """Raster rows a band's blocks read: its own rows and one ring row above
    and below, inside the raster ([ra, rb); empty band -> (0, 0))."""
    b0, b1 = band
    if b1 <= b0:
        return 0, 0
    return max(b0 * block_rows - 1, 0), min(b1 * block_rows + 1, rows)


def out_rows(band, block_rows: int, rows: int):
    """Raster rows of a band's counts ([r0, r1))."""
    b0, b1 = band
    return min(b0 * block_rows, rows), min(b1 * block_rows, rows)


class DeviceStages:
    """The three stages as calls of the CUDA library on the current device:
    export -> status, resolve -> (in(p), status), finish -> status, where a
    status is what the device reported after the completed stage; a failed
    call raises FlowAccError."""

    def __init__(self, device=None, tile=None):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.opts = options(tile)

    def _ws(self, rows, cols, bh, bw):
        n = fa_ooc_workspace_size(rows, cols, bh, bw, self.opts)
        if n == 0:
            raise FlowAccError(FA_ERR_INVALID_ARG, "fa_ooc_workspace_size")
        return workspace(n, self.device)

    def export(self, codes, codes_row0, shape, block, band, rec: Records) -> int:
        rows, cols = shape
        n = (band[1] - band[0]) * _grid(shape, block)[1]
        st = fa_shard_export(codes, codes_row0, rows, cols, block[0], block[1], band[0], band[1],
                             rec.nexit(n), rec.link(n), rec.node_dst(n), rec.node_val(n),
                             self._ws(rows, cols, *block), self.opts)
        return _device_status(st, "fa_shard_export")

    def resolve(self, shape, block, rec: Records):
        rows, cols = shape
        nb = rec.cap
        inflow = torch.zeros(nb * rec.pmax, dtype=torch.int64)
        st = fa_shard_resolve(rows, cols, block[0], block[1], rec.nexit(nb), rec.link(nb),
                              rec.node_dst(nb), rec.node_val(nb), inflow, self._ws(rows, cols, *block))
        return inflow, _device_status(st, "fa_shard_resolve")

    def finish(self, codes, codes_row0, shape, block, band, inflow, out) -> int:
        rows, cols = shape
        st = fa_shard_finish(codes, codes_row0, rows, cols, block[0], block[1], band[0], band[1],
                             inflow, out, self._ws(rows, cols, *block), self.opts)
        return _device_status(st, "fa_shard_finish")


def _device_status(st, what):
    """A status the device reported after a completed stage, passed on; any
    other (a failed call) raised."""
    if st not in _DEVICE_STATUS:
        raise FlowAccError(st, what)
    return st


def _worse(a, b):
    return a if _DEVICE_STATUS.index(a) >= _DEVICE_STATUS.index(b) else b


def _grid(shape, block):
    st, nby, nbx, pmax = fa_shard_geometry(shape[0], shape[1], block[0], block[1])
    if st != FA_OK:
        raise ValueError(f"no block grid for raster {shape} and blocks {block}")
    return nby, nbx, pmax


def _agree(flag: int, on: bool, group) -> int:
    """The largest of every rank's flag (this rank's alone without a group)."""
    if not on:
        return flag
    t = torch.tensor([flag], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return int(t.item())


def accumulate_sharded(codes: torch.Tensor, codes_row0: int, shape, block=None, group=None,
                       stages=None, tile=None, check: bool = True,
                       checkpoint: str | None = None) -> torch.Tensor:
    """Counts of this rank's band of a raster of `shape` (rows, cols), solved
    with every rank of `group` (torch.distributed, initialised; or a single
    process when it is not).  codes: uint8 CPU tensor holding raster rows
    codes_row0 .. (at least the rows band_rows() names for this rank's band;
    the whole raster with codes_row0 = 0 will do).  block: outer block shape
    (rows, cols); None = 16384 x 16384.  Returns int64 counts (uint64 bit
    patterns) of raster rows out_rows(band) for this rank's band, where band
    = bands(nby, world)[rank].  check=True raises FlowAccError, on every
    rank, when the device reported an error on any rank (the most severe
    one); a stage that fails on some rank raises there and ShardAborted on
    the others, at the same point.

    checkpoint: a directory all ranks can write (shared, or the same path on
    each node for its ranks' files and rank 0's).  Each rank keeps its
    band's records there after pass A and rank 0 keeps in(p) after the
    resolve; a later call on the same raster with the same blocks and number
    of ranks loads them instead of repeating that work, so a solve that
    stopped during the finish resumes at the finish.  (The paper's
    discussion of robustness describes caching the tiles' perimeter data and
    the global solution this way, and leaves it out of its implementation.)
    The files are checked against the raster shape, blocks and ranks, not
    against the codes: a directory serves one raster."""
    rows, cols = int(shape[0]), int(shape[1])
    bh, bw = (block if block is not None else (16384, 16384))
    bh, bw = min(int(bh), max(rows, 1)), min(int(bw), max(cols, 1))
    nby, nbx, pmax = _grid((rows, cols), (bh, bw))
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    stages = stages if stages is not None else DeviceStages(tile=tile)
    all_bands = bands(nby, world)
    band = all_bands[rank]
    cap = max(b1 - b0 for b0, b1 in all_bands) * nbx
    nblk = (band[1] - band[0]) * nbx
    root = 0 if not on or group is None else dist.get_global_rank(group, 0)
    status = FA_OK

    def stop(failed, what):
        # every rank learns whether a stage failed anywhere, then all stop
        if _agree(1 if failed is not None else 0, on, group):
            if failed is not None:
                raise failed
            raise ShardAborted(f"{what} failed on another rank")

    meta = dict(rows=rows, cols=cols, bh=bh, bw=bw, world=world)
    rec_path = os.path.join(checkpoint, f"records_{rank}_of_{world}.npz") if checkpoint else None
    in_path = os.path.join(checkpoint, f"inflow_of_{world}.npz") if checkpoint else None

    # 1. pass A on this rank's blocks (or its records kept by an earlier call)
    mine = Records(cap, pmax)
    failed = None
    try:
        kept = _ckpt_load(rec_path, dict(meta, rank=rank)) if rec_path else None
        if kept is not None and kept["buf"].size == mine.buf.numel():
            mine.buf.copy_(torch.from_numpy(kept["buf"]))
            status = _worse(status, int(kept["status"]))
        elif nblk:
            st = stages.export(codes, codes_row0, (rows, cols), (bh, bw), band, mine)
            status = _worse(status, st)
            if rec_path:
                _ckpt_save(rec_path, {"buf": mine.buf.numpy(), "status": np.int64(st)},
                           dict(meta, rank=rank))
    except Exception as e:  # noqa: BLE001  (re-raised below, after the other ranks know)
        failed = e
    stop(failed, "the export")

    # 2-4. records to rank 0, the blocks' graph solved there, in(p) back
    recv = torch.zeros(cap * pmax, dtype=torch.int64)
    if rank == 0:
        parts = [mine] if world == 1 else [Records(cap, pmax) for _ in range(world)]
        if world > 1:
            dist.gather(mine.buf, [p.buf for p in parts], dst=root, group=group)
        chunks, failed = None, None
        try:
            kept = _ckpt_load(in_path, meta) if in_path else None
            if kept is not None and kept["inflow"].size == nby * nbx * pmax:
                inflow, st = torch.from_numpy(kept["inflow"]), int(kept["status"])
            else:
                full = Records(nby * nbx, pmax)
                for r, (b0, b1) in enumerate(all_bands):
                    if b1 > b0:
                        full.put(b0 * nbx, parts[r], (b1 - b0) * nbx)
                inflow, st = stages.resolve((rows, cols), (bh, bw), full)
                if in_path:
                    _ckpt_save(in_path, {"inflow": inflow.numpy(), "status": np.int64(st)}, meta)
            status = _worse(status, st)
            chunks = []
            for b0, b1 in all_bands:
                c = torch.zeros(cap * pmax, dtype=torch.int64)
                c[: (b1 - b0) * nbx * pmax] = inflow[b0 * nbx * pmax: b1 * nbx * pmax]
                chunks.append(c)
        except Exception as e:  # noqa: BLE001
            failed = e
        flag = torch.tensor([1 if failed is not None else 0], dtype=torch.int64)
        if world > 1:
            dist.broadcast(flag, src=root, group=group)
        if failed is not None:
            raise failed
        if world > 1:
            dist.scatter(recv, chunks, src=root, group=group)
        else:
            recv = chunks[0]
    else:
        dist.gather(mine.buf, None, dst=root, group=group)
        flag = torch.zeros(1, dtype=torch.int64)
        dist.broadcast(flag, src=root, group=group)
        if int(flag.item()):
            raise ShardAborted("the resolve failed on the root rank")
        dist.scatter(recv, None, src=root, group=group)

    # 5. pass C on this rank's blocks
    r0, r1 = out_rows(band, bh, rows)
    out = torch.zeros((r1 - r0, cols), dtype=torch.int64)
    failed = None
    try:
        if nblk:
            status = _worse(status, stages.finish(codes, codes_row0, (rows, cols), (bh, bw), band,
                                                  recv[: nblk * pmax], out))
    except Exception as e:  # noqa: BLE001
        failed = e
    stop(failed, "the finish")

    # the most severe condition any rank's device reported
    status = _DEVICE_STATUS[_agree(_DEVICE_STATUS.index(status), on, group)]
    if check and status < 0:
        raise FlowAccError(status, "accumulate_sharded")
    return out
