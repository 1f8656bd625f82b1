"""The shard form's three stages on the CPU, for tests: the records, in(p)
and counts computed from their definitions with plain loops and the oracle
(Algorithm 1 on each block as a raster of its own).  They stand in for the
CUDA stages so that the exchange between processes runs on CPU ranks, and
they give the unique parts of the device records (in(p), and each perimeter
slot's exit target and A_loc) to compare with.

Definitions (Section 3.2 at the level of outer blocks):
  exit      a block perimeter cell whose flow enters a valid cell (code 1..9)
            of another block; its record is (global slot of that cell, A_loc)
            where A_loc is the cell's accumulation within its block alone;
  link(s)   for an exit, its own rank; for a valid perimeter cell receiving
            flow from another block, the exit its path inside the block
            reaches (none if the path ends inside); else none;
  G(e)      A_loc(e) + the sum of G over the exits whose entry links to e;
  in(p)     the sum of G(e) over the exits e whose target is p;
  counts    A_loc + the sum of in(p) over the entries p upstream in the block.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

TERM = 0xFFFF
# direction offsets of codes 1..8 (E, NE, N, NW, W, SW, S, SE), row 0 = north
DR = (0, 0, -1, -1, -1, 0, 1, 1, 1)
DC = (0, 1, 1, 0, -1, -1, -1, 0, 1)


def perim_count(h, w):
    return w if h == 1 else (h if w == 1 else 2 * h + 2 * w - 4)


def perim_cells(h, w):
    """Perimeter cells in slot order: top row west to east, right column north
    to south, bottom row east to west, left column south to north."""
    if h == 1:
        return [(0, c) for c in range(w)]
    if w == 1:
        return [(r, 0) for r in range(h)]
    return ([(0, c) for c in range(w)] + [(r, w - 1) for r in range(1, h)]
            + [(h - 1, c) for c in range(w - 2, -1, -1)] + [(r, 0) for r in range(h - 2, 0, -1)])


class Grid:
    def __init__(self, shape, block):
        self.rows, self.cols = int(shape[0]), int(shape[1])
        self.bh = min(int(block[0]), max(self.rows, 1))
        self.bw = min(int(block[1]), max(self.cols, 1))
        self.nby = -(-self.rows // self.bh)
        self.nbx = -(-self.cols // self.bw)
        self.pmax = perim_count(self.bh, self.bw)

    def block(self, b):
        by, bx = divmod(b, self.nbx)
        R0, C0 = by * self.bh, bx * self.bw
        return R0, C0, min(self.bh, self.rows - R0), min(self.bw, self.cols - C0)

    def slot_id(self, R, C):
        by, bx = R // self.bh, C // self.bw
        R0, C0, h, w = self.block(by * self.nbx + bx)
        return (by * self.nbx + bx) * self.pmax + perim_cells(h, w).index((R - R0, C - C0))


class OracleStages:
    """export / resolve / finish with the interface of shard.DeviceStages
    (statuses: always FA_OK = 0; a cycle raises)."""

    @staticmethod
    def _codes(codes, codes_row0, g):
        a = codes.numpy() if isinstance(codes, torch.Tensor) else np.asarray(codes)

        def code(R, C):
            if 0 <= R < g.rows and 0 <= C < g.cols:
                return int(a[R - codes_row0, C])
            return 0
        return a, code

    def export(self, codes, codes_row0, shape, block, band, rec):
        g = Grid(shape, block)
        a, code = self._codes(codes, codes_row0, g)
        b0, b1 = band[0] * g.nbx, band[1] * g.nbx
        n = b1 - b0
        nexit = rec.nexit(n).numpy().view(np.uint32)
        link = rec.link(n).numpy().view(np.uint16)
        dst = rec.node_dst(n).numpy().view(np.uint32)
        val = rec.node_val(n).numpy()
        link[:] = TERM
        for b in range(b0, b1):
            i = b - b0
            R0, C0, h, w = g.block(b)
            blk = np.ascontiguousarray(a[R0 - codes_row0: R0 - codes_row0 + h, C0: C0 + w])
            A = oracle.counts(blk).values
            cells = perim_cells(h, w)
            where = {cell: s for s, cell in enumerate(cells)}
            inside = lambda r, c: 0 <= r < h and 0 <= c < w  # noqa: E731
            k = 0
            for s, (r, c) in enumerate(cells):
                d = int(blk[r, c])
                if 1 <= d <= 8:
                    tr, tc = r + DR[d], c + DC[d]
                    if not inside(tr, tc) and 1 <= code(R0 + tr, C0 + tc) <= 9:
                        dst[i * g.pmax + k] = g.slot_id(R0 + tr, C0 + tc)
                        val[i * g.pmax + k] = float(A[r, c])
                        link[i * g.pmax + s] = k
                        k += 1
            nexit[i] = k
            for s, (r, c) in enumerate(cells):
                if link[i * g.pmax + s] != TERM or not 1 <= int(blk[r, c]) <= 9:
                    continue
                fed = False
                for d in range(1, 9):
                    nr, nc = r + DR[d], c + DC[d]
                    if inside(nr, nc):
                        continue
                    e = code(R0 + nr, C0 + nc)
                    fed |= 1 <= e <= 8 and (nr + DR[e], nc + DC[e]) == (r, c)
                if not fed:
                    continue
                rr, cc, end = r, c, None
                for _ in range(h * w + 1):
                    d = int(blk[rr, cc])
                    if not 1 <= d <= 8:
                        break
                    tr, tc = rr + DR[d], cc + DC[d]
                    if not inside(tr, tc):
                        end = (rr, cc)
                        break
                    if not 1 <= int(blk[tr, tc]) <= 9:
                        break
                    rr, cc = tr, tc
                if end is not None:
                    link[i * g.pmax + s] = link[i * g.pmax + where[end]]
        return 0

    def resolve(self, shape, block, rec):
        g = Grid(shape, block)
        nb = rec.cap
        nexit = rec.nexit(nb).numpy().view(np.uint32)
        link = rec.link(nb).numpy().view(np.uint16)
        dst = rec.node_dst(nb).numpy().view(np.uint32)
        val = rec.node_val(nb).numpy()
        nodes = [b * g.pmax + j for b in range(nb) for j in range(int(nexit[b]))]
        succ, indeg, G = {}, {u: 0 for u in nodes}, {u: int(val[u]) for u in nodes}
        for u in nodes:
            t = int(dst[u])
            lk = int(link[t])
            succ[u] = None if lk == TERM else (t // g.pmax) * g.pmax + lk
            if succ[u] is not None:
                indeg[succ[u]] += 1
        todo = [u for u in nodes if indeg[u] == 0]
        while todo:
            u = todo.pop()
            v = succ[u]
            if v is not None:
                G[v] += G[u]
                indeg[v] -= 1
                if indeg[v] == 0:
                    todo.append(v)
        if any(indeg[u] for u in nodes):
            raise ValueError("the blocks' perimeter graph has a cycle")
        inflow = np.zeros(nb * g.pmax, dtype=np.uint64)
        for u in nodes:
            inflow[int(dst[u])] += np.uint64(G[u])
        return torch.from_numpy(inflow.view(np.int64)), 0

    def finish(self, codes, codes_row0, shape, block, band, inflow, out):
        g = Grid(shape, block)
        a, _ = self._codes(codes, codes_row0, g)
        inf = inflow.numpy().view(np.uint64)
        o = out.numpy().view(np.uint64)
        r0 = band[0] * g.bh
        for b in range(band[0] * g.nbx, band[1] * g.nbx):
            i = b - band[0] * g.nbx
            R0, C0, h, w = g.block(b)
            blk = np.ascontiguousarray(a[R0 - codes_row0: R0 - codes_row0 + h, C0: C0 + w])
            wi = np.zeros((h, w), dtype=np.float32)
            for s, (r, c) in enumerate(perim_cells(h, w)):
                v = int(inf[i * g.pmax + s])
                assert v < 1 << 24, "stand-in finish is exact only below 2^24"
                wi[r, c] = v
            extra = oracle.weighted(blk, wi).values
            o[R0 - r0: R0 - r0 + h, C0: C0 + w] = oracle.counts(blk).values + extra.astype(np.uint64)
        return 0
