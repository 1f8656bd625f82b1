// Out-of-core accumulation: rasters whose codes and counts stay in host
// memory, processed on the device one outer block at a time.
//
// The paper's stated aim (Section 1) is rasters larger than the memory of
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
//           walks of the tile resolve;
//   pass C  per block again (EVICT): codes copied in and the block solved
//           again by the tile pipeline with the flow entering each outer entry
//           (the sum of G over the outer exits draining into it) handed to it
//           as extra inflow at that entry, so that the pipeline's own resolve
//           and finalising pass carry it along the paths (Algorithm 3); the
//           tile-local sums plus the uint64 offsets are the block's counts,
//           copied out.
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

// Pass C: the flow entering the block at each outer entry (the sum of G over
// the outer exits draining into it), handed to the tile pipeline: at the
// entry's inner slot (added along its path in the tile) and at the slot of
// the inner exit that path reaches (added to that exit before the resolve).
__global__ void k_ooc_inject(OocGrid g, OocBlock k, InnerGeo ig, const uint16_t *link,
                             const unsigned long long *G, unsigned long long *inj,
                             unsigned long long *injx) {
    const int P = perim_count(k.hb, k.wb);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P) return;
    int r, c;
    cell_of(s, k.hb, k.wb, r, c);
    if (ooc_code(k, r, c) - 1u >= 9u) return;
    uint32_t m = ooc_inflow_mask(k, r, c);
    unsigned long long in = 0;
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        const uint32_t src = ooc_outside_slot(g, k, r + dir_dr(j + 1), c + dir_dc(j + 1));
        const uint16_t lk = link[src];  // the outer exit's own rank
        if (lk == LINK_TERM) continue;
        in += G[(size_t)(src - src % (uint32_t)g.pmax) + lk];
    }
    if (!in) return;
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
    unsigned long long *x;
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

// Copies block k's codes with their one-cell ring from the host raster; ring
// cells outside the raster read 0 (NoData).
cudaError_t copy_block_in(const OocPlan &p, const OocBlock &k, uint8_t *buf, const uint8_t *codes,
                          int64_t pitch, cudaStream_t cs) {
    const int64_t R0 = (int64_t)k.by * p.g.bh, C0 = (int64_t)k.bx * p.g.bw;
    const int64_t ra = std::max<int64_t>(R0 - 1, 0), rb = std::min<int64_t>(R0 + k.hb + 1, p.g.rows);
    const int64_t ca = std::max<int64_t>(C0 - 1, 0), cb = std::min<int64_t>(C0 + k.wb + 1, p.g.cols);
    const bool edge = ra == R0 || ca == C0 || rb < R0 + k.hb + 1 || cb < C0 + k.wb + 1;
    if (edge) {
        cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)(k.hb + 2) * k.pd, cs);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpy2DAsync(buf + (ra - R0 + 1) * k.pd + OX + (ca - C0), (size_t)k.pd,
                             codes + ra * pitch + ca, (size_t)pitch, (size_t)(cb - ca),
                             (size_t)(rb - ra), cudaMemcpyHostToDevice, cs);
}

unsigned grid_for(int64_t n, int bs) { return (unsigned)std::max<int64_t>(1, (n + bs - 1) / bs); }

}  // namespace

}  // namespace fa

using namespace fa;

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
    if (d_status && ((uintptr_t)d_status & 7)) return FA_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return FA_ERR_WORKSPACE;
    OocWork w;
    if (carve_ooc(workspace, ws_bytes, p, w) > ws_bytes) return FA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    StatusBlock *st = reinterpret_cast<StatusBlock *>(d_status ? (void *)d_status : w.status);

    // copy streams (host -> device codes, device -> host counts) and the
    // events that order the two buffers of each kind between them and `s`
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t ready[2] = {}, freed[2] = {}, done[2] = {}, drained[2] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&drained[i], cudaEventDisableTiming);
    }
    const bool was = timing_swap(false);  // block calls record no phase events

    auto run = [&]() -> cudaError_t {
        k_ooc_status_reset<<<1, 32, 0, s>>>(st);
        cudaError_t r = cudaMemsetAsync(w.nexit, 0, (size_t)p.nb * sizeof(uint32_t), s);
        if (r == cudaSuccess) r = cudaMemsetAsync(w.misc, 0, 16 * sizeof(uint32_t), s);
        if (r != cudaSuccess || empty) return r;
        // the copy streams start after the resets above
        if ((r = cudaEventRecord(freed[0], s)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(freed[1], s)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(drained[0], s)) != cudaSuccess) return r;
        if ((r = cudaEventRecord(drained[1], s)) != cudaSuccess) return r;
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                r = resolve_exit_forest_u64(p.nb, p.g.pmax, w.nexit, w.link, w.node_dst, w.node_val,
                                            w.x, w.J0, w.J1, w.misc, st, s);
                if (r != cudaSuccess) return r;
            }
            for (int64_t b = 0; b < p.nb; ++b) {
                const int i = (int)(b & 1);
                const OocBlock k = block_of(p, b, w.codes[i]);
                if ((r = cudaStreamWaitEvent(cin, freed[i], 0)) != cudaSuccess) return r;
                if ((r = copy_block_in(p, k, w.codes[i], codes, pitch_codes, cin)) != cudaSuccess) return r;
                if ((r = cudaEventRecord(ready[i], cin)) != cudaSuccess) return r;
                if ((r = cudaStreamWaitEvent(s, ready[i], 0)) != cudaSuccess) return r;

                Geom gi;
                make_geom(k.hb, k.wb, opts, gi);
                FwdWork iw;
                if (carve_forward(w.inner, p.inner_ws, gi, iw, false) > p.inner_ws) return cudaErrorInvalidValue;
                const InnerGeo ig{gi.th, gi.tw, gi.tiles_x, gi.pmax};
                const int P = perim_count(k.hb, k.wb);
                const int64_t R0 = (int64_t)k.by * p.g.bh, C0 = (int64_t)k.bx * p.g.bw;
                const int64_t n = (int64_t)k.hb * k.wb;
                if (pass == 0) {
                    r = launch_forward(gi, k.codes + k.pd + OX, k.pd, nullptr, 0, nullptr, 0, w.A, k.wb,
                                       0, iw, w.inner_status, s);
                    if (r != cudaSuccess) return r;
                    k_ooc_status_merge<<<1, 32, 0, s>>>(
                        reinterpret_cast<const StatusBlock *>(w.inner_status), st, R0, C0, k.wb, p.g.cols);
                    k_ooc_exits<<<grid_for(P, 128), 128, 0, s>>>(p.g, k, w.A, w.nexit, w.link, w.node_dst,
                                                                w.node_val);
                    k_ooc_links_hop<<<grid_for(P, 128), 128, 0, s>>>(p.g, k, ig, iw.link, iw.node_dst,
                                                                    gi.tiles() * gi.pmax, w.link);
                    if ((r = cudaGetLastError()) != cudaSuccess) return r;
                    if ((r = cudaEventRecord(freed[i], s)) != cudaSuccess) return r;
                    continue;
                }
                // pass C: the block solved again with its inflow from other
                // blocks injected, the offsets into off[i] (uint64)
                const size_t islots = (size_t)gi.tiles() * gi.pmax;
                if ((r = cudaMemsetAsync(w.inj, 0, islots * 8, s)) != cudaSuccess) return r;
                if ((r = cudaMemsetAsync(w.injx, 0, islots * 8, s)) != cudaSuccess) return r;
                k_ooc_inject<<<grid_for(P, 128), 128, 0, s>>>(p.g, k, ig, w.link, w.x, w.inj, w.injx);
                if ((r = cudaGetLastError()) != cudaSuccess) return r;
                if ((r = cudaStreamWaitEvent(s, drained[i], 0)) != cudaSuccess) return r;
                if ((r = cudaMemsetAsync(w.off[i], 0, (size_t)n * 8, s)) != cudaSuccess) return r;
                const PipeHooks hk{w.inj, w.injx, w.off[i]};
                r = launch_forward_hooked(gi, k.codes + k.pd + OX, k.pd, w.A, k.wb, iw, w.inner_status,
                                          hk, s);
                if (r != cudaSuccess) return r;
                if ((r = cudaEventRecord(freed[i], s)) != cudaSuccess) return r;
                k_ooc_combine<<<grid_for(n, 256), 256, 0, s>>>(n, w.A, w.off[i]);
                if ((r = cudaGetLastError()) != cudaSuccess) return r;
                if ((r = cudaEventRecord(done[i], s)) != cudaSuccess) return r;
                if ((r = cudaStreamWaitEvent(cout, done[i], 0)) != cudaSuccess) return r;
                r = cudaMemcpy2DAsync(out + R0 * pitch_out + C0, (size_t)pitch_out * 8, w.off[i],
                                      (size_t)k.wb * 8, (size_t)k.wb * 8, (size_t)k.hb,
                                      cudaMemcpyDeviceToHost, cout);
                if (r != cudaSuccess) return r;
                if ((r = cudaEventRecord(drained[i], cout)) != cudaSuccess) return r;
            }
        }
        // the caller's stream ends after the last copy out
        if ((r = cudaEventRecord(drained[0], cout)) != cudaSuccess) return r;
        return cudaStreamWaitEvent(s, drained[0], 0);
    };
    if (e == cudaSuccess) e = run();
    timing_swap(was);
    // the call is synchronous: its copies read and write host memory
    const cudaError_t es = cudaStreamSynchronize(s);
    if (cin) cudaStreamSynchronize(cin);
    if (cout) cudaStreamSynchronize(cout);
    for (int i = 0; i < 2; ++i) {
        if (ready[i]) cudaEventDestroy(ready[i]);
        if (freed[i]) cudaEventDestroy(freed[i]);
        if (done[i]) cudaEventDestroy(done[i]);
        if (drained[i]) cudaEventDestroy(drained[i]);
    }
    if (cin) cudaStreamDestroy(cin);
    if (cout) cudaStreamDestroy(cout);
    if (e != cudaSuccess || es != cudaSuccess) return FA_ERR_CUDA;
    return fa_status_read(d_status, workspace, stream, nullptr, nullptr);
}
