// Out-of-core accumulation: rasters whose codes and counts stay in host
// memory, processed on the device one outer block at a time.
//
// The paper's stated aim (Section 2) is rasters larger than the memory of
// any one machine, with only one tile and the producer's perimeter data held
// at once (Section 3, EVICT).  Here the raster is split into outer blocks
// (block_rows x block_cols cells); each block is solved on the device by the
// same tile pipeline as fa_accumulate, as if it were a raster of its own, and
// only the outer perimeter graph of the whole raster stays on the device:
//   pass A  per block: its codes (with a one-cell ring) are copied in, the
//           block is accumulated, and its perimeter records are made: A_loc
//           and the target of every cell whose flow enters another block (an
//           outer exit), and for every cell receiving flow from another block
//           (an outer entry) the outer exit its path inside the block reaches
//           (Algorithm 2 at the block level, hopping over the block's own
//           tile links between the first and the last tile of the path);
//   resolve the outer exits' graph (Section 3.2), solved on the device by the
//           walks of the tile resolve, which also give in(p) per block
//           perimeter slot: the sum of G over the outer exits draining into
//           that cell;
//   pass C  per block again (EVICT): codes copied in and the block solved
//           again by the tile pipeline with in(p) handed to it as extra
//           inflow at each outer entry, so that the pipeline's own resolve
//           and finalising pass carry it along the paths (Algorithm 3); the
//           tile-local sums plus the uint64 offsets are the block's counts,
//           copied out.
// The shard form (fa_shard_export / fa_shard_resolve / fa_shard_finish) runs
// the same three stages in separate processes: pass A on a band of block
// rows, the resolve on the gathered records of all blocks, pass C on the band
// with its part of in(p).
// Codes are copied on a second stream into one of two device buffers while
// the other is in use (with pinned host memory the copies overlap the work).
#include <algorithm>
#include <cstring>

#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

// Device copy of a block's codes: row r (-1 .. hb) of the block at byte
// (r + 1) * pd, column c (-1 .. wb) at byte OX + c.  The block's own cells
// start at a 16-byte boundary (OX = 16), so the tile passes can stage them by
// TMA; the ring column left of them sits at byte 15.
constexpr int OX = 16;
__host__ __device__ inline int64_t ooc_pitch(int64_t bw) { return ((OX + bw + 1 + 15) / 16) * 16; }

struct OocBlock {
    const uint8_t *codes;  // the block's code buffer (ring included)
    int64_t pd;            // its row pitch
    int hb, wb;            // the block's size (ragged at the raster's edges)
    int by, bx;            // block coordinates
    int64_t b;             // block number by * nbx + bx
};

struct OocGrid {
    int64_t rows, cols;
    int bh, bw, nby, nbx, pmax;  // nominal block size, blocks, perimeter slots per block
};

__device__ __forceinline__ uint32_t ooc_code(const OocBlock &k, int r, int c) {
    return k.codes[(int64_t)(r + 1) * k.pd + OX + c];
}

// Global slot id of the cell (rr, cc), just outside block k, in its own block.
__device__ __forceinline__ uint32_t ooc_outside_slot(const OocGrid &g, const OocBlock &k, int rr, int cc) {
    const int byd = k.by + (rr < 0 ? -1 : (rr >= k.hb ? 1 : 0));
    const int bxd = k.bx + (cc < 0 ? -1 : (cc >= k.wb ? 1 : 0));
    const int64_t R0 = (int64_t)k.by * g.bh, C0 = (int64_t)k.bx * g.bw;
    const int64_t R0d = (int64_t)byd * g.bh, C0d = (int64_t)bxd * g.bw;
    const int hd = (int)min((int64_t)g.bh, g.rows - R0d), wd = (int)min((int64_t)g.bw, g.cols - C0d);
    const int sd = slot_of((int)(R0 + rr - R0d), (int)(C0 + cc - C0d), hd, wd);
    return (uint32_t)(((int64_t)byd * g.nbx + bxd) * g.pmax + sd);
}

// The outside neighbours (direction bits j = code - 1) of block cell (r, c)
// whose flow enters it.
__device__ __forceinline__ uint32_t ooc_inflow_mask(const OocBlock &k, int r, int c) {
    uint32_t m = 0;
    for (int j = 0; j < 8; ++j) {
        const int nr = r + dir_dr(j + 1), nc = c + dir_dc(j + 1);
        if ((unsigned)nr < (unsigned)k.hb && (unsigned)nc < (unsigned)k.wb) continue;
        const int kh = (int)ooc_code(k, nr, nc);
        if (kh >= 1 && kh <= 8 && nr + dir_dr(kh) == r && nc + dir_dc(kh) == c) m |= 1u << j;
    }
    return m;
}

// Pass A, outer exits: every block-perimeter cell whose flow enters a valid
// cell of another block gets a rank (node id b * pmax + rank), its target's
// global slot id and its block-local accumulation A_loc.
__global__ void k_ooc_exits(OocGrid g, OocBlock k, const uint32_t *A, uint32_t *nexit,
                            uint16_t *link, uint32_t *node_dst, double *node_val) {
    const int P = perim_count(k.hb, k.wb);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P) return;
    int r, c;
    cell_of(s, k.hb, k.wb, r, c);
    const size_t base = (size_t)k.b * g.pmax;
    uint16_t lk = LINK_TERM;
    const uint32_t code = ooc_code(k, r, c);
    if (code >= 1 && code <= 8) {
        const int tr = r + dir_dr((int)code), tc = c + dir_dc((int)code);
        if (((unsigned)tr >= (unsigned)k.hb || (unsigned)tc >= (unsigned)k.wb) &&
            ooc_code(k, tr, tc) - 1u < 9u) {
            const uint32_t rk = atomicAdd(&nexit[k.b], 1u);
            node_dst[base + rk] = ooc_outside_slot(g, k, tr, tc);
            node_val[base + rk] = (double)A[(int64_t)r * k.wb + c];
            lk = (uint16_t)rk;
        }
    }
    link[base + s] = lk;
}

// The inner tiles of a block (the tile pipeline's decomposition of it).
struct InnerGeo {
    int th, tw, tiles_x, pmax;
};

// Inner tile and slot of block cell (r, c), and the tile's extent.
__device__ __forceinline__ void inner_slot(const InnerGeo &ig, const OocBlock &k, int r, int c,
                                           int &T, int &sl) {
    const int ty = r / ig.th, tx = c / ig.tw;
    const int R0 = ty * ig.th, C0 = tx * ig.tw;
    const int ht = min(ig.th, k.hb - R0), wt = min(ig.tw, k.wb - C0);
    T = ty * ig.tiles_x + tx;
    sl = slot_of(r - R0, c - C0, ht, wt);
}

// Follows the path from block cell (r, c) inside its inner tile.  Returns 1
// when the next cell is a valid cell of the block in another inner tile
// ((r, c) is then an exit of its tile), 0 when the path ends in the tile (at
// NoFlow, NoData, a cycle, or a cell whose flow leaves the block); (r, c) is
// the last cell reached in the tile.
__device__ __forceinline__ int follow_in_tile(const InnerGeo &ig, const OocBlock &k, int &r, int &c) {
    const int R0 = (r / ig.th) * ig.th, C0 = (c / ig.tw) * ig.tw;
    for (int s = 0; s <= ig.th * ig.tw; ++s) {
        const uint32_t code = ooc_code(k, r, c);
        if (code < 1 || code > 8) return 0;
        const int tr = r + dir_dr((int)code), tc = c + dir_dc((int)code);
        if ((unsigned)tr >= (unsigned)k.hb || (unsigned)tc >= (unsigned)k.wb) return 0;
        if (ooc_code(k, tr, tc) - 1u >= 9u) return 0;
        if ((unsigned)(tr - R0) >= (unsigned)ig.th || (unsigned)(tc - C0) >= (unsigned)ig.tw) return 1;
        r = tr;
        c = tc;
    }
    return 0;
}

// Pass A, outer entries, by the block's own perimeter graph: the path from an
// outer entry is followed cell by cell only inside the inner tile where it
// starts and the one where it ends; between them it hops from inner exit to
// inner exit (ilink: slot -> exit rank its path reaches, idst: exit -> slot of
// its target), as the tile pipeline linked them (Algorithm 2 inside tiles).
__global__ void k_ooc_links_hop(OocGrid g, OocBlock k, InnerGeo ig, const uint16_t *ilink,
                                const uint32_t *idst, int64_t inodes, uint16_t *link) {
    const int P = perim_count(k.hb, k.wb);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P) return;
    int r, c;
    cell_of(s, k.hb, k.wb, r, c);
    const size_t base = (size_t)k.b * g.pmax;
    if (link[base + s] != LINK_TERM) return;
    if (ooc_code(k, r, c) - 1u >= 9u || !ooc_inflow_mask(k, r, c)) return;
    uint16_t lk = LINK_TERM;
    bool ok = true;
    int64_t hops = 0;
    while (follow_in_tile(ig, k, r, c) == 1) {
        // (r, c) is an inner exit: hop along the exits the path passes
        int T, sl;
        inner_slot(ig, k, r, c, T, sl);
        uint16_t il = ilink[(size_t)T * ig.pmax + sl];  // an exit links to its own rank
        if (il == LINK_TERM) {
            ok = false;
            break;
        }
        uint32_t dst = idst[(size_t)T * ig.pmax + il];
        for (il = ilink[dst]; il != LINK_TERM && hops <= inodes; il = ilink[dst], ++hops)
            dst = idst[(size_t)(dst / ig.pmax) * ig.pmax + il];
        if (++hops > inodes) {  // a cycle of exits
            ok = false;
            break;
        }
        // the path ends in the tile of entry slot dst: its cell
        const int T2 = (int)(dst / ig.pmax), sl2 = (int)(dst - (uint32_t)T2 * ig.pmax);
        const int ty = T2 / ig.tiles_x, tx = T2 - ty * ig.tiles_x;
        const int R0 = ty * ig.th, C0 = tx * ig.tw;
        int lr, lc;
        cell_of(sl2, min(ig.th, k.hb - R0), min(ig.tw, k.wb - C0), lr, lc);
        r = R0 + lr;
        c = C0 + lc;
    }
    if (ok && (r == 0 || c == 0 || r == k.hb - 1 || c == k.wb - 1))
        lk = link[base + slot_of(r, c, k.hb, k.wb)];
    link[base + s] = lk;
}

// Pass C: the flow entering the block at each outer entry (in(p), the sum of
// G over the outer exits draining into it, per perimeter slot of the block),
// handed to the tile pipeline: at the entry's inner slot (added along its
// path in the tile) and at the slot of the inner exit that path reaches
// (added to that exit before the resolve).
__global__ void k_ooc_inject(OocBlock k, InnerGeo ig, const unsigned long long *inb,
                             unsigned long long *inj, unsigned long long *injx) {
    const int P = perim_count(k.hb, k.wb);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P) return;
    const unsigned long long in = inb[s];
    if (!in) return;
    int r, c;
    cell_of(s, k.hb, k.wb, r, c);
    int T, sl;
    inner_slot(ig, k, r, c, T, sl);
    inj[(size_t)T * ig.pmax + sl] = in;
    if (follow_in_tile(ig, k, r, c) == 1) {
        inner_slot(ig, k, r, c, T, sl);
        atomicAdd(&injx[(size_t)T * ig.pmax + sl], in);
    }
}

// Pass C: counts = A_loc + the entering flow, in place in `off`; a count of
// 2^32 or more is reported as FA_FLAG_OVERFLOW only by uint32 outputs, so
// nothing is flagged here.
__global__ void k_ooc_combine(int64_t n, const uint32_t *A, unsigned long long *off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += A[i];
}

// Folds the status block of one inner (block) call into the call's own:
// flags or-ed, counts added, the first index mapped from the block's cell
// numbering (r * wb + c) to the raster's.
__global__ void k_ooc_status_merge(const StatusBlock *inner, StatusBlock *st, int64_t R0, int64_t C0,
                                   int wb, int64_t cols) {
    if (threadIdx.x != 0) return;
    if (!inner->flags) return;
    long long first = NO_INDEX;
    if (inner->first != NO_INDEX) {
        const long long r = inner->first / wb, c = inner->first % wb;
        first = (R0 + r) * cols + (C0 + c);
    }
    status_report(st, inner->flags, inner->count, first);
}

__global__ void k_ooc_status_reset(StatusBlock *st) {
    if (threadIdx.x == 0) {
        st->flags = 0;
        st->count = 0;
        st->first = NO_INDEX;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

constexpr int kDefaultBlock = 16384;

struct OocPlan {
    OocGrid g;
    Geom gi;         // inner geometry of a nominal block
    int64_t nb;      // blocks
    size_t inner_ws; // inner workspace bytes
};

bool ooc_plan(int64_t rows, int64_t cols, int64_t block_rows, int64_t block_cols,
              const fa_options *opts, OocPlan &p) {
    if (rows < 0 || cols < 0 || block_rows < 0 || block_cols < 0) return false;
    if (opts && opts->code_format != FA_CODES_BYTE) return false;
    // a block larger than the raster is the raster
    const int64_t bh = std::min<int64_t>(block_rows ? block_rows : kDefaultBlock, std::max<int64_t>(rows, 1));
    const int64_t bw = std::min<int64_t>(block_cols ? block_cols : kDefaultBlock, std::max<int64_t>(cols, 1));
    if (bh > 65535 || bw > 65535) return false;
    const int64_t pmax = perim_count((int)bh, (int)bw);
    if (pmax > 65534) return false;  // exit ranks and slots must stay below 0xFFFF
    p.g.rows = rows;
    p.g.cols = cols;
    p.g.bh = (int)bh;
    p.g.bw = (int)bw;
    p.g.nby = (int)((rows + bh - 1) / bh);
    p.g.nbx = (int)((cols + bw - 1) / bw);
    p.g.pmax = (int)pmax;
    p.nb = (int64_t)p.g.nby * p.g.nbx;
    if (p.nb * pmax >= 0xFFFFFFFFll) return false;  // node ids are 32-bit
    if (!make_geom(bh, bw, opts, p.gi)) return false;
    if (!forward_tile_ok(p.gi, 0)) return false;
    FwdWork w;
    p.inner_ws = carve_forward(nullptr, 0, p.gi, w, true);
    return true;
}

struct OocWork {
    void *status, *inner_status;
    uint32_t *misc, *nexit;
    uint16_t *link;
    uint32_t *node_dst, *J0, *J1;
    double *node_val;
    unsigned long long *x;    // G per outer exit node
    unsigned long long *inb;  // in(p) per outer perimeter slot
    uint8_t *codes[2];
    uint32_t *A;
    unsigned long long *off[2];
    unsigned long long *inj, *injx;  // per inner perimeter slot of a block
    void *inner;
};

size_t carve_ooc(void *ws, size_t bytes, const OocPlan &p, OocWork &w) {
    Carver c(ws, bytes);
    const size_t nodes = (size_t)p.nb * p.g.pmax;
    const size_t cells = (size_t)p.g.bh * p.g.bw;
    const size_t cbytes = (size_t)(p.g.bh + 2) * ooc_pitch(p.g.bw);
    w.status = c.take<uint8_t>(64);
    w.inner_status = c.take<uint8_t>(64);
    w.misc = c.take<uint32_t>(16);
    w.nexit = c.take<uint32_t>(p.nb);
    w.link = c.take<uint16_t>(nodes);
    w.node_dst = c.take<uint32_t>(nodes);
    w.J0 = c.take<uint32_t>(nodes);
    w.J1 = c.take<uint32_t>(nodes);
    w.node_val = c.take<double>(nodes);
    w.x = c.take<unsigned long long>(nodes);
    w.inb = c.take<unsigned long long>(nodes);
    for (int i = 0; i < 2; ++i) w.codes[i] = c.take<uint8_t>(cbytes);
    w.A = c.take<uint32_t>(cells);
    for (int i = 0; i < 2; ++i) w.off[i] = c.take<unsigned long long>(cells);
    const size_t islots = (size_t)p.gi.tiles() * p.gi.pmax;
    w.inj = c.take<unsigned long long>(islots);
    w.injx = c.take<unsigned long long>(islots);
    w.inner = c.take<uint8_t>(p.inner_ws);
    return c.used();
}

OocBlock block_of(const OocPlan &p, int64_t b, const uint8_t *buf) {
    OocBlock k;
    k.codes = buf;
    k.pd = ooc_pitch(p.g.bw);
    k.by = (int)(b / p.g.nbx);
    k.bx = (int)(b % p.g.nbx);
    k.b = b;
    k.hb = (int)std::min<int64_t>(p.g.bh, p.g.rows - (int64_t)k.by * p.g.bh);
    k.wb = (int)std::min<int64_t>(p.g.bw, p.g.cols - (int64_t)k.bx * p.g.bw);
    return k;
}

// Host rows of the raster: raster row `row0` at `p`, `nrows` rows of `pitch`
// bytes (the whole raster, or one shard's band with its ring rows).
struct HostRows {
    const uint8_t *p;
    int64_t row0, nrows, pitch;
};

// Host uint64 counts: raster row `row0` at `p`, rows of `pitch` elements.
struct HostOut {
    uint64_t *p;
    int64_t row0, pitch;
};

// Raster rows that the blocks of block rows [by0, by1) read: their own rows
// and the ring rows above and below, inside the raster.
void band_rows(const OocPlan &p, int64_t by0, int64_t by1, int64_t &ra, int64_t &rb) {
    ra = std::max<int64_t>(by0 * p.g.bh - 1, 0);
    rb = std::min<int64_t>(by1 * p.g.bh + 1, p.g.rows);
}

// Copies block k's codes with their one-cell ring from the host rows; ring
// cells outside the raster read 0 (NoData).
cudaError_t copy_block_in(const OocPlan &p, const OocBlock &k, uint8_t *buf, const HostRows &h,
                          cudaStream_t cs) {
    const int64_t R0 = (int64_t)k.by * p.g.bh, C0 = (int64_t)k.bx * p.g.bw;
    const int64_t ra = std::max<int64_t>(R0 - 1, 0), rb = std::min<int64_t>(R0 + k.hb + 1, p.g.rows);
    const int64_t ca = std::max<int64_t>(C0 - 1, 0), cb = std::min<int64_t>(C0 + k.wb + 1, p.g.cols);
    const bool edge = ra == R0 || ca == C0 || rb < R0 + k.hb + 1 || cb < C0 + k.wb + 1;
    if (edge) {
        cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)(k.hb + 2) * k.pd, cs);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpy2DAsync(buf + (ra - R0 + 1) * k.pd + OX + (ca - C0), (size_t)k.pd,
                             h.p + (ra - h.row0) * h.pitch + ca, (size_t)h.pitch, (size_t)(cb - ca),
                             (size_t)(rb - ra), cudaMemcpyHostToDevice, cs);
}

unsigned grid_for(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

// The block loop of one call: each block's codes are copied in on stream
// `cin` into one of two device buffers while the other is in use, and its
// counts copied out on stream `cout`; events order the buffers between the
// copy streams and the work stream `s`.
class BlockLoop {
  public:
    BlockLoop(const OocPlan &p, const OocWork &w, StatusBlock *st, const fa_options *opts,
              cudaStream_t s)
        : p_(p), w_(w), st_(st), opts_(opts), s_(s) {}
    BlockLoop(const BlockLoop &) = delete;
    BlockLoop &operator=(const BlockLoop &) = delete;

    // Creates the copy streams and events; the copies start after the work
    // enqueued on `s` so far.
    cudaError_t start() {
        cudaError_t e = cudaStreamCreateWithFlags(&cin_, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cout_, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&ready_[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed_[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done_[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&drained_[i], cudaEventDisableTiming);
        }
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventRecord(freed_[i], s_);
            if (e == cudaSuccess) e = cudaEventRecord(drained_[i], s_);
        }
        return e;
    }

    // Pass A over blocks [b0, b1): solve, outer exits and entry links.
    cudaError_t pass_a(const HostRows &h, int64_t b0, int64_t b1) {
        for (int64_t b = b0; b < b1; ++b) {
            const int i = (int)(b & 1);
            Block x;
            cudaError_t r = stage_in(h, b, x);
            if (r != cudaSuccess) return r;
            r = launch_forward(x.gi, x.k.codes + x.k.pd + OX, x.k.pd, nullptr, 0, nullptr, 0, w_.A,
                               x.k.wb, 0, x.iw, w_.inner_status, s_);
            if (r != cudaSuccess) return r;
            k_ooc_status_merge<<<1, 32, 0, s_>>>(reinterpret_cast<const StatusBlock *>(w_.inner_status),
                                                st_, x.R0, x.C0, x.k.wb, p_.g.cols);
            k_ooc_exits<<<grid_for(x.P, 128), 128, 0, s_>>>(p_.g, x.k, w_.A, w_.nexit, w_.link,
                                                           w_.node_dst, w_.node_val);
            k_ooc_links_hop<<<grid_for(x.P, 128), 128, 0, s_>>>(p_.g, x.k, x.ig, x.iw.link, x.iw.node_dst,
                                                               x.gi.tiles() * x.gi.pmax, w_.link);
            if ((r = cudaGetLastError()) != cudaSuccess) return r;
            if ((r = cudaEventRecord(freed_[i], s_)) != cudaSuccess) return r;
        }
        return cudaSuccess;
    }

    // Pass C over blocks [b0, b1): each block solved again with in(p) (w.inb,
    // per outer slot) injected, its counts copied out to `o`; merge_status
    // also folds the block solves' status into the call's.
    cudaError_t pass_c(const HostRows &h, const HostOut &o, int64_t b0, int64_t b1, bool merge_status) {
        for (int64_t b = b0; b < b1; ++b) {
            const int i = (int)(b & 1);
            Block x;
            cudaError_t r = stage_in(h, b, x);
            if (r != cudaSuccess) return r;
            const size_t islots = (size_t)x.gi.tiles() * x.gi.pmax;
            if ((r = cudaMemsetAsync(w_.inj, 0, islots * 8, s_)) != cudaSuccess) return r;
            if ((r = cudaMemsetAsync(w_.injx, 0, islots * 8, s_)) != cudaSuccess) return r;
            k_ooc_inject<<<grid_for(x.P, 128), 128, 0, s_>>>(x.k, x.ig, w_.inb + (size_t)b * p_.g.pmax,
                                                            w_.inj, w_.injx);
            if ((r = cudaGetLastError()) != cudaSuccess) return r;
            if ((r = cudaStreamWaitEvent(s_, drained_[i], 0)) != cudaSuccess) return r;
            if ((r = cudaMemsetAsync(w_.off[i], 0, (size_t)x.n * 8, s_)) != cudaSuccess) return r;
            const PipeHooks hk{w_.inj, w_.injx, w_.off[i]};
            r = launch_forward_hooked(x.gi, x.k.codes + x.k.pd + OX, x.k.pd, w_.A, x.k.wb, x.iw,
                                      w_.inner_status, hk, s_);
            if (r != cudaSuccess) return r;
            if (merge_status)
                k_ooc_status_merge<<<1, 32, 0, s_>>>(
                    reinterpret_cast<const StatusBlock *>(w_.inner_status), st_, x.R0, x.C0, x.k.wb,
                    p_.g.cols);
            if ((r = cudaEventRecord(freed_[i], s_)) != cudaSuccess) return r;
            k_ooc_combine<<<grid_for(x.n, 256), 256, 0, s_>>>(x.n, w_.A, w_.off[i]);
            if ((r = cudaGetLastError()) != cudaSuccess) return r;
            if ((r = cudaEventRecord(done_[i], s_)) != cudaSuccess) return r;
            if ((r = cudaStreamWaitEvent(cout_, done_[i], 0)) != cudaSuccess) return r;
            r = cudaMemcpy2DAsync(o.p + (x.R0 - o.row0) * o.pitch + x.C0, (size_t)o.pitch * 8, w_.off[i],
                                  (size_t)x.k.wb * 8, (size_t)x.k.wb * 8, (size_t)x.k.hb,
                                  cudaMemcpyDeviceToHost, cout_);
            if (r != cudaSuccess) return r;
            if ((r = cudaEventRecord(drained_[i], cout_)) != cudaSuccess) return r;
        }
        return cudaSuccess;
    }

    // The work stream continues after the last copy out.
    cudaError_t join() {
        cudaError_t r = cudaEventRecord(drained_[0], cout_);
        return r == cudaSuccess ? cudaStreamWaitEvent(s_, drained_[0], 0) : r;
    }

    // Waits for all three streams (the copies read and write host memory, so
    // the calls are synchronous); returns the work stream's error.
    cudaError_t finish() {
        const cudaError_t e = cudaStreamSynchronize(s_);
        if (cin_) cudaStreamSynchronize(cin_);
        if (cout_) cudaStreamSynchronize(cout_);
        return e;
    }

    ~BlockLoop() {
        finish();
        for (int i = 0; i < 2; ++i) {
            if (ready_[i]) cudaEventDestroy(ready_[i]);
            if (freed_[i]) cudaEventDestroy(freed_[i]);
            if (done_[i]) cudaEventDestroy(done_[i]);
            if (drained_[i]) cudaEventDestroy(drained_[i]);
        }
        if (cin_) cudaStreamDestroy(cin_);
        if (cout_) cudaStreamDestroy(cout_);
    }

  private:
    struct Block {
        OocBlock k;
        Geom gi;
        FwdWork iw;
        InnerGeo ig;
        int P;
        int64_t R0, C0, n;
    };

    // Block b's codes copied into buffer b & 1 once that buffer is free; the
    // work stream waits for them.  Fills the block's inner geometry.
    cudaError_t stage_in(const HostRows &h, int64_t b, Block &x) {
        const int i = (int)(b & 1);
        x.k = block_of(p_, b, w_.codes[i]);
        cudaError_t r = cudaStreamWaitEvent(cin_, freed_[i], 0);
        if (r == cudaSuccess) r = copy_block_in(p_, x.k, w_.codes[i], h, cin_);
        if (r == cudaSuccess) r = cudaEventRecord(ready_[i], cin_);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(s_, ready_[i], 0);
        if (r != cudaSuccess) return r;
        if (!make_geom(x.k.hb, x.k.wb, opts_, x.gi)) return cudaErrorInvalidValue;
        if (carve_forward(w_.inner, p_.inner_ws, x.gi, x.iw, false) > p_.inner_ws) return cudaErrorInvalidValue;
        x.ig = InnerGeo{x.gi.th, x.gi.tw, x.gi.tiles_x, x.gi.pmax};
        x.P = perim_count(x.k.hb, x.k.wb);
        x.R0 = (int64_t)x.k.by * p_.g.bh;
        x.C0 = (int64_t)x.k.bx * p_.g.bw;
        x.n = (int64_t)x.k.hb * x.k.wb;
        return cudaSuccess;
    }

    const OocPlan &p_;
    const OocWork &w_;
    StatusBlock *st_;
    const fa_options *opts_;
    cudaStream_t s_;
    cudaStream_t cin_ = nullptr, cout_ = nullptr;
    cudaEvent_t ready_[2] = {}, freed_[2] = {}, done_[2] = {}, drained_[2] = {};
};

// Status reset and cleared perimeter records of blocks [b0, b1) on `s`: no
// exits, every slot's link none (slots past a ragged block's perimeter too).
cudaError_t reset_records(const OocPlan &p, const OocWork &w, StatusBlock *st, int64_t b0, int64_t b1,
                          cudaStream_t s) {
    k_ooc_status_reset<<<1, 32, 0, s>>>(st);
    cudaError_t r = cudaMemsetAsync(w.misc, 0, 16 * sizeof(uint32_t), s);
    if (r == cudaSuccess && b1 > b0) r = cudaMemsetAsync(w.nexit + b0, 0, (size_t)(b1 - b0) * 4, s);
    if (r == cudaSuccess && b1 > b0)
        r = cudaMemsetAsync(w.link + (size_t)b0 * p.g.pmax, 0xFF, (size_t)(b1 - b0) * p.g.pmax * 2, s);
    return r == cudaSuccess ? cudaGetLastError() : r;
}

}  // namespace

}  // namespace fa

using namespace fa;

namespace {

// Workspace and status checks shared by the out-of-core and shard calls.
fa_status ws_setup(const OocPlan &p, void *workspace, size_t ws_bytes, const int32_t *d_status,
                   OocWork &w) {
    if (d_status && ((uintptr_t)d_status & 7)) return FA_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return FA_ERR_WORKSPACE;
    if (carve_ooc(workspace, ws_bytes, p, w) > ws_bytes) return FA_ERR_WORKSPACE;
    return FA_OK;
}

// A shard's band of block rows [band0, band1) and the host rows it was
// given: raster rows [codes_row0, codes_row0 + codes_rows) must hold every
// row its blocks read.
bool band_ok(const OocPlan &p, int64_t band0, int64_t band1, int64_t codes_row0, int64_t codes_rows) {
    if (band0 < 0 || band1 < band0 || band1 > p.g.nby) return false;
    if (band1 == band0) return true;
    int64_t ra, rb;
    band_rows(p, band0, band1, ra, rb);
    return codes_row0 >= 0 && codes_rows >= 0 && codes_row0 <= ra && codes_row0 + codes_rows >= rb;
}

// Records from other processes are checked before they reach the device: at
// most pmax exits per block, every exit's target a slot of the raster, and
// the link of that slot none or an exit of its block.
bool records_ok(const OocPlan &p, const uint32_t *nexit, const uint16_t *link, const uint32_t *node_dst) {
    const uint64_t pmax = (uint64_t)p.g.pmax, nodes = (uint64_t)p.nb * pmax;
    for (int64_t b = 0; b < p.nb; ++b)
        if (nexit[b] > pmax) return false;
    for (int64_t b = 0; b < p.nb; ++b)
        for (uint32_t j = 0; j < nexit[b]; ++j) {
            const uint64_t dst = node_dst[(uint64_t)b * pmax + j];
            if (dst >= nodes) return false;
            const uint16_t l = link[dst];
            if (l != LINK_TERM && l >= nexit[dst / pmax]) return false;
        }
    return true;
}

StatusBlock *status_of(int32_t *d_status, const OocWork &w) {
    return reinterpret_cast<StatusBlock *>(d_status ? (void *)d_status : w.status);
}

}  // namespace

extern "C" size_t fa_ooc_workspace_size(int64_t rows, int64_t cols, int64_t block_rows,
                                        int64_t block_cols, const fa_options *opts) {
    OocPlan p;
    if (!ooc_plan(rows, cols, block_rows, block_cols, opts, p)) return 0;
    OocWork w;
    return carve_ooc(nullptr, 0, p, w);
}

extern "C" fa_status fa_accumulate_ooc(const uint8_t *codes, int64_t rows, int64_t cols,
                                       int64_t pitch_codes, uint64_t *out, int64_t pitch_out,
                                       int64_t block_rows, int64_t block_cols, void *workspace,
                                       size_t ws_bytes, const fa_options *opts, int32_t *d_status,
                                       void *stream) {
    OocPlan p;
    if (!ooc_plan(rows, cols, block_rows, block_cols, opts, p)) return FA_ERR_INVALID_ARG;
    const bool empty = rows == 0 || cols == 0;
    if (!empty && (!codes || !out || pitch_codes < cols || pitch_out < cols)) return FA_ERR_INVALID_ARG;
    OocWork w;
    const fa_status v = ws_setup(p, workspace, ws_bytes, d_status, w);
    if (v != FA_OK) return v;
    cudaStream_t s = (cudaStream_t)stream;
    StatusBlock *st = status_of(d_status, w);
    const bool was = timing_swap(false);  // block calls record no phase events
    cudaError_t e, es;
    {
        BlockLoop loop(p, w, st, opts, s);
        e = reset_records(p, w, st, 0, p.nb, s);
        if (e == cudaSuccess && !empty) {
            const HostRows h{codes, 0, rows, pitch_codes};
            e = loop.start();
            if (e == cudaSuccess) e = loop.pass_a(h, 0, p.nb);
            if (e == cudaSuccess)
                e = resolve_exit_forest_u64(p.nb, p.g.pmax, w.nexit, w.link, w.node_dst, w.node_val, w.x,
                                            w.inb, w.J0, w.J1, w.misc, st, s);
            if (e == cudaSuccess) e = loop.pass_c(h, HostOut{out, 0, pitch_out}, 0, p.nb, false);
            if (e == cudaSuccess) e = loop.join();
        }
        es = loop.finish();
    }
    timing_swap(was);
    if (e != cudaSuccess || es != cudaSuccess) return FA_ERR_CUDA;
    return fa_status_read(d_status, workspace, stream, nullptr, nullptr);
}

extern "C" fa_status fa_shard_geometry(int64_t rows, int64_t cols, int64_t block_rows,
                                       int64_t block_cols, int64_t *block_grid, int32_t *pmax) {
    OocPlan p;
    if (!block_grid || !pmax || !ooc_plan(rows, cols, block_rows, block_cols, nullptr, p))
        return FA_ERR_INVALID_ARG;
    block_grid[0] = p.g.nby;
    block_grid[1] = p.g.nbx;
    *pmax = p.g.pmax;
    return FA_OK;
}

extern "C" fa_status fa_shard_export(const uint8_t *codes, int64_t codes_row0, int64_t codes_rows,
                                     int64_t pitch_codes, int64_t rows, int64_t cols,
                                     int64_t block_rows, int64_t block_cols, int64_t band0,
                                     int64_t band1, uint32_t *nexit, uint16_t *link,
                                     uint32_t *node_dst, double *node_val, void *workspace,
                                     size_t ws_bytes, const fa_options *opts, int32_t *d_status,
                                     void *stream) {
    OocPlan p;
    if (!ooc_plan(rows, cols, block_rows, block_cols, opts, p)) return FA_ERR_INVALID_ARG;
    if (!band_ok(p, band0, band1, codes_row0, codes_rows)) return FA_ERR_INVALID_ARG;
    const int64_t b0 = band0 * p.g.nbx, b1 = band1 * p.g.nbx;
    if (b1 > b0 && (!codes || pitch_codes < cols || !nexit || !link || !node_dst || !node_val))
        return FA_ERR_INVALID_ARG;
    OocWork w;
    const fa_status v = ws_setup(p, workspace, ws_bytes, d_status, w);
    if (v != FA_OK) return v;
    cudaStream_t s = (cudaStream_t)stream;
    StatusBlock *st = status_of(d_status, w);
    const size_t n0 = (size_t)b0 * p.g.pmax, nn = (size_t)(b1 - b0) * p.g.pmax;
    const bool was = timing_swap(false);
    cudaError_t e, es;
    {
        BlockLoop loop(p, w, st, opts, s);
        e = reset_records(p, w, st, b0, b1, s);
        if (e == cudaSuccess && nn) e = cudaMemsetAsync(w.node_dst + n0, 0, nn * 4, s);
        if (e == cudaSuccess && nn) e = cudaMemsetAsync(w.node_val + n0, 0, nn * 8, s);
        if (e == cudaSuccess && nn) {
            e = loop.start();
            if (e == cudaSuccess) e = loop.pass_a(HostRows{codes, codes_row0, codes_rows, pitch_codes}, b0, b1);
            if (e == cudaSuccess) e = loop.join();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(nexit, w.nexit + b0, (size_t)(b1 - b0) * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(link, w.link + n0, nn * 2, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(node_dst, w.node_dst + n0, nn * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(node_val, w.node_val + n0, nn * 8, cudaMemcpyDeviceToHost, s);
        }
        es = loop.finish();
    }
    timing_swap(was);
    if (e != cudaSuccess || es != cudaSuccess) return FA_ERR_CUDA;
    return fa_status_read(d_status, workspace, stream, nullptr, nullptr);
}

extern "C" fa_status fa_shard_resolve(int64_t rows, int64_t cols, int64_t block_rows,
                                      int64_t block_cols, const uint32_t *nexit, const uint16_t *link,
                                      const uint32_t *node_dst, const double *node_val,
                                      uint64_t *inflow, void *workspace, size_t ws_bytes,
                                      int32_t *d_status, void *stream) {
    OocPlan p;
    if (!ooc_plan(rows, cols, block_rows, block_cols, nullptr, p)) return FA_ERR_INVALID_ARG;
    const size_t nodes = (size_t)p.nb * p.g.pmax;
    if (nodes && (!nexit || !link || !node_dst || !node_val || !inflow)) return FA_ERR_INVALID_ARG;
    if (nodes && !records_ok(p, nexit, link, node_dst)) return FA_ERR_INVALID_ARG;
    if (d_status && ((uintptr_t)d_status & 7)) return FA_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return FA_ERR_WORKSPACE;
    OocWork w;
    carve_ooc(workspace, ws_bytes, p, w);
    if ((uintptr_t)(w.inb + nodes) > (uintptr_t)workspace + ws_bytes) return FA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    StatusBlock *st = status_of(d_status, w);
    k_ooc_status_reset<<<1, 32, 0, s>>>(st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(w.misc, 0, 16 * sizeof(uint32_t), s);
    if (e == cudaSuccess && nodes) {
        e = cudaMemcpyAsync(w.nexit, nexit, (size_t)p.nb * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.link, link, nodes * 2, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.node_dst, node_dst, nodes * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.node_val, node_val, nodes * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = resolve_exit_forest_u64(p.nb, p.g.pmax, w.nexit, w.link, w.node_dst, w.node_val, w.x,
                                        w.inb, w.J0, w.J1, w.misc, st, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(inflow, w.inb, nodes * 8, cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e != cudaSuccess || es != cudaSuccess) return FA_ERR_CUDA;
    return fa_status_read(d_status, workspace, stream, nullptr, nullptr);
}

extern "C" fa_status fa_shard_finish(const uint8_t *codes, int64_t codes_row0, int64_t codes_rows,
                                     int64_t pitch_codes, int64_t rows, int64_t cols,
                                     int64_t block_rows, int64_t block_cols, int64_t band0,
                                     int64_t band1, const uint64_t *inflow, uint64_t *out,
                                     int64_t pitch_out, void *workspace, size_t ws_bytes,
                                     const fa_options *opts, int32_t *d_status, void *stream) {
    OocPlan p;
    if (!ooc_plan(rows, cols, block_rows, block_cols, opts, p)) return FA_ERR_INVALID_ARG;
    if (!band_ok(p, band0, band1, codes_row0, codes_rows)) return FA_ERR_INVALID_ARG;
    const int64_t b0 = band0 * p.g.nbx, b1 = band1 * p.g.nbx;
    if (b1 > b0 && (!codes || pitch_codes < cols || !inflow || !out || pitch_out < cols))
        return FA_ERR_INVALID_ARG;
    OocWork w;
    const fa_status v = ws_setup(p, workspace, ws_bytes, d_status, w);
    if (v != FA_OK) return v;
    cudaStream_t s = (cudaStream_t)stream;
    StatusBlock *st = status_of(d_status, w);
    const size_t n0 = (size_t)b0 * p.g.pmax, nn = (size_t)(b1 - b0) * p.g.pmax;
    const bool was = timing_swap(false);
    cudaError_t e, es;
    {
        BlockLoop loop(p, w, st, opts, s);
        e = reset_records(p, w, st, b0, b0, s);
        if (e == cudaSuccess && nn) e = cudaMemcpyAsync(w.inb + n0, inflow, nn * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nn) {
            e = loop.start();
            if (e == cudaSuccess)
                e = loop.pass_c(HostRows{codes, codes_row0, codes_rows, pitch_codes},
                                HostOut{out, band0 * p.g.bh, pitch_out}, b0, b1, true);
            if (e == cudaSuccess) e = loop.join();
        }
        es = loop.finish();
    }
    timing_swap(was);
    if (e != cudaSuccess || es != cudaSuccess) return FA_ERR_CUDA;
    return fa_status_read(d_status, workspace, stream, nullptr, nullptr);
}
