// Forward D8 flow accumulation: tile passes and perimeter-graph resolve.
//
// Pipeline for one raster, or a batch of rasters each carrying up to
// FA_MAX_FIELDS weight fields (Section 3 of the paper):
//   pass 1  k_walk<M, 1>    per tile: Algorithm 1 in shared memory, then the
//                           perimeter data of Section 3.2: A_loc at every exit
//                           cell and the exit cell its flow enters in the
//                           neighbouring tile; Algorithm 2 (the exit each entry
//                           cell's path reaches) by walking the entry paths.
//                           Counts (M = 0) leave A_loc in the output raster.
//   resolve k_forest_*      the global flow graph over exit cells
//                           (Section 3.2): G(e) = A_loc(e) + sum of G over the
//                           exits whose flow enters the tile at a cell linked
//                           to e, by last-arriver walks over the exit nodes
//                           (Algorithm 1 on the perimeter graph).
//   pass 2  counts: k_addin  per tile: the flow entering at each entry cell
//                           added along its in-tile path in the output
//                           (Algorithm 3, Section 3.3; A_loc retained, the
//                           codes staged again, only the entry paths walked);
//           float: k_walk<1, 2>  per tile: Algorithm 1 again with the flow
//                           entering from other tiles added to the weight of
//                           its entry cell, writing A (EVICT).
//
// Algorithm 1 inside a tile: every cell's in-tile dependency count (its
// in-degree) is gathered first; the cells with none start a walk.  A walk
// hands a finished cell's flow to its downstream cell; the walk that brings
// the last missing inflow of a cell continues from it (its flow is then
// complete), every other walk stops there.  Each cell is passed on exactly
// once, so a tile costs O(cells) work, and the lanes of a warp take new
// starting cells from the warp's share of the tile as their walks end.
//   counts: each cell's word packs (pending inflows, successor, sum); one
//           atomic add hands a walk's sum over and returns the downstream
//           cell's successor and partial sum, so a step is one shared-memory
//           operation.  Integer sums: the order of the adds cannot change a
//           bit of the result.
//   float weights: each cell's word packs (pending inflows, which neighbours
//           drain into it, successor); the walk that completes a cell adds
//           its inflows in a fixed neighbour order as compensated float pairs
//           (about 48 bits), so results are run-to-run reproducible and any
//           weight, however small next to the others, keeps its relative
//           precision.
#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

struct TileArgs {
    RasterDesc one;  // the raster of a single-raster call
    int th, tw, pmax;
    int nib;         // codes packed two per byte (FA_CODES_NIBBLE)
    int nf;          // weight fields per raster (1 for counts)
    uint32_t *nexit;
    uint16_t *link;
    uint32_t *node_dst;
    double *node_val;
    const void *G;  // resolved perimeter graph: u64 counts or u128 fixed-point sums, [node * nf + f]
    StatusBlock *st;
    uint32_t *maxw;
    const unsigned long long *infl;  // counts: flow arriving at each perimeter slot (pass 2)
    unsigned long long *off64;       // counts: if set, pass 2 adds into this uint64 raster instead
    // batches: a table of rasters (nullptr for one raster), each with its
    // tiles numbered from its tile_base in one global tile sequence
    const RasterDesc *rtab;
    int nr;
    int64_t T;            // tiles in all
    int64_t fcells;       // cell bound of the perimeter-graph fixed-point scale
    uint64_t wait_ns;     // bound of a staged-load wait
};

// Points the raster fields of `a` at the raster owning global tile t.
__device__ __forceinline__ const RasterDesc &raster_of(const TileArgs &a, int64_t t) {
    if (!a.rtab) return a.one;
    int lo = 0, hi = a.nr - 1;  // last raster with tile_base <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.rtab[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return a.rtab[lo];
}

// global fixed-point scale for the perimeter graph: |sum| <= cells * max|w| < 2^(124 - q)
__device__ __forceinline__ int fix_scale(int64_t cells, uint32_t maxw_bits) {
    float mw = __uint_as_float(maxw_bits);
    if (!(mw > 0.0f) || maxw_bits >= 0x7f800000u) return 0;
    int e;
    frexp((double)cells * (double)mw, &e);  // bound < 2^e
    return 124 - e;
}

// ---------------------------------------------------------------------------
// Shared-memory layout of a tile's codes: halo row hr (0 .. h+1, tile row
// r = hr - 1) starts at hr * S; tile column c sits at byte c + X0 (halo
// columns at bytes X0 - 1 and X0 + w).  A row is exactly the TMA box that
// starts X0 bytes left of the tile (a 16-byte aligned column when the tile
// width is a multiple of 16).  S >= X0 + tw + 16.
// ---------------------------------------------------------------------------
constexpr int X0 = 16;
__host__ __device__ inline int tile_stride(int tw) { return ((tw + 32 + 15) / 16) * 16; }

// bytes of one staged code tile, rounded so that what follows stays 128-aligned
__host__ __device__ inline size_t code_buf_bytes(int th, int tw) {
    return (((size_t)(th + 2) * tile_stride(tw)) + 127) & ~size_t(127);
}

// Packed codes (two per byte) staged by TMA: the box starts PX0 cells (16
// bytes) left of the tile, so that its first byte is a 16-byte column when the
// tile width is a multiple of 32; byte b of a box row holds cells C0 - PX0 +
// 2b and + 1.  A box row covers the S cells of a code-buffer row (which starts
// X0 cells left of the tile): S / 2 + 8 bytes, rounded to 16.
constexpr int PX0 = 32;
__host__ __device__ inline int packed_box_bytes(int tw) { return ((tile_stride(tw) / 2 + 8 + 15) / 16) * 16; }
__host__ __device__ inline size_t packed_buf_bytes(int th, int tw) {
    return (((size_t)(th + 2) * packed_box_bytes(tw)) + 127) & ~size_t(127);
}

// How a tile gets its codes: plain loads, TMA-staged bytes, or TMA-staged
// packed codes spread to bytes in shared memory.
enum { LOAD_PLAIN = 0, LOAD_TMA = 1, LOAD_TMA_PACKED = 2 };

// ---------------------------------------------------------------------------
// Cell words.  The words of a tile and of the one-cell ring around it are
// numbered wi = (r + 1) * W2 + (c + 1), W2 = tw + 2 (tile row r, tile column
// c; the ring at r = -1, r = th, c = -1, c = tw), at most 2^14 - 1 of them,
// so a word index fits 14 bits and SUCC_NONE is never one.  Pending-inflow
// counts sit in the top four bits.  Every word that is not a valid cell of
// the tile (NoData, off the raster, outside a ragged tile, or the ring) holds
// the count SENT_CNT: at most eight cells add one to it and a walk reaching
// it takes one off again, so it never reads as complete (0) or as the last
// inflow (1) and its sums are never used.  A cell's successor is simply the
// word its code points at, so the one-pass init needs neither the target's
// code nor bounds; a walk that reaches a SENT_CNT word stops there.
// ---------------------------------------------------------------------------
constexpr int MAX_TILE_CELLS = 8192;
constexpr int MAX_TILE_WORDS = 16383;
constexpr uint32_t SUCC_NONE = 0x3FFFu;
constexpr uint32_t SENT_CNT = 7;

__host__ __device__ inline int tile_words(int th, int tw) { return (th + 2) * (tw + 2); }

// counts: (pending << CNT) | (successor << SUCC) | partial sum; 32-bit words
// in pass 1 (a tile sum is at most 8192 < 2^14), 64-bit words in pass 2,
// where the flow entering from other tiles (up to 2^46 cells) is added.
// Sums that walks bring to a SENT_CNT word may carry into its successor bits,
// never into its count.
template <class W> struct CountWord;
template <> struct CountWord<uint32_t> {
    static constexpr int SUCC = 14, CNT = 28;
    static constexpr uint32_t ACC = (1u << 14) - 1, ONE = 1u << 28, SENT = SENT_CNT << 28;
};
template <> struct CountWord<unsigned long long> {
    static constexpr int SUCC = 46, CNT = 60;
    static constexpr unsigned long long ACC = (1ull << 46) - 1, ONE = 1ull << 60,
                                        SENT = (unsigned long long)SENT_CNT << 60;
};
// float weights: (pending << GW_CNT) | GW_VALID for a valid cell of the tile
// | (mask of the neighbours draining into the cell << GW_PM) | successor; the
// sums live in a separate array of compensated float pairs.  (A valid cell
// may have up to eight pending inflows, so the flag, not the count, tells it
// from a SENT_CNT word before the walks.)
constexpr int GW_PM = 14, GW_CNT = 28;
constexpr uint32_t GW_ONE = 1u << GW_CNT, GW_SENT = SENT_CNT << GW_CNT, GW_VALID = 1u << 27;

// Threads of a tile block: one per 32 cells, at least a warp, at most 256.
__host__ __device__ inline int walk_threads(int th, int tw) {
    const int n = th * tw;
    const int t = ((n + 32 * 32 - 1) / (32 * 32)) * 32;
    return t < 32 ? 32 : (t > 256 ? 256 : t);
}

// Shared memory of k_walk<MODE, PASS, LOAD> for a tile shape.
__host__ __device__ inline size_t walk_smem_bytes(int th, int tw, int mode, int pass, int load) {
    const size_t nwd = (size_t)tile_words(th, tw), pm = (size_t)(2 * th + 2 * tw);
    size_t b = 128;  // alignment slack of the dynamic window
    b += code_buf_bytes(th, tw) + (load == LOAD_TMA_PACKED ? packed_buf_bytes(th, tw) : 0);
    b += nwd * ((mode == 0 && pass == 2) ? 8 : 4);  // cell words
    b = (b + 15) & ~size_t(15);
    if (mode == 1) b += nwd * 8;                     // float pair sums
    b += nwd * 2;                                    // queued walk starts
    b = (b + 15) & ~size_t(15);
    b += pm * 4 + pm * 2 + pm * 2 + pm;              // exit targets, exit ranks, entry list, inflow masks
    return (b + 15) & ~size_t(15);
}

__host__ __device__ inline bool tile_shape_ok(int th, int tw, int valm) {
    if (th < 1 || tw < 1 || (int64_t)th * tw > MAX_TILE_CELLS) return false;
    if ((int64_t)(th + 2) * (tw + 2) > MAX_TILE_WORDS) return false;
    for (int pass = 1; pass <= 2; ++pass)
        if (walk_smem_bytes(th, tw, valm, pass, LOAD_TMA_PACKED) > 227 * 1024) return false;
    return true;
}

// Code of raster column gc in a row of packed codes: low nibble for even
// columns, high nibble for odd ones.
__device__ __forceinline__ uint32_t nibble_at(const uint8_t *row, int64_t gc) {
    return ((uint32_t)row[gc >> 1] >> ((gc & 1) << 2)) & 15u;
}

// Four packed codes (one 16-bit load) spread to one byte each.
__device__ __forceinline__ uint32_t spread_nibbles(uint32_t hw) {
    return (hw & 0xFu) | ((hw & 0xF0u) << 4) | ((hw & 0xF00u) << 8) | ((hw & 0xF000u) << 12);
}

// Load a tile's codes with a one-cell halo (Algorithm 1's F) into ec: valid
// codes 1..9 as they are, NoData, masked, invalid and off-raster cells as 0,
// bytes beyond the halo ring 0.  Each lane first issues the loads for up to
// four rows (one 32-bit word of interior codes, or the single halo byte its
// word holds), then converts and stores them, so several global loads are in
// flight per lane.  Invalid codes inside the tile are counted.  Packed codes
// (nib) are spread to one byte per cell on the way.
__device__ __forceinline__ void load_codes(const RasterDesc &ras, uint8_t *ec, int64_t R0, int64_t C0,
                                           int h, int w, int S, bool nib, bool count_bad, int &nbad,
                                           long long &fbad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // bytes: 4-byte loads of four codes; packed: 2-byte loads of four codes
    const bool fast =
        nib ? ((reinterpret_cast<uintptr_t>(ras.codes) | (uintptr_t)ras.pc) & 1) == 0 && (C0 & 3) == 0
            : ((reinterpret_cast<uintptr_t>(ras.codes) | (uintptr_t)ras.pc | (uintptr_t)C0) & 3) == 0;
    const int words = S >> 2;
    constexpr int U = 4;
    for (int hr0 = warp; hr0 < h + 2; hr0 += U * nw) {
        for (int wd0 = 0; wd0 < words; wd0 += 32) {
            const int wd = wd0 + lane;
            const int c0 = 4 * wd - X0;  // tile column of the word's first byte
            uint32_t raw[U], mraw[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {  // issue every load first
                const int hr = hr0 + u * nw;
                raw[u] = 0;
                mraw[u] = 0;
                if (hr >= h + 2 || wd >= words) continue;
                const int64_t gr = R0 - 1 + hr;
                if (gr < 0 || gr >= ras.rows) continue;
                const uint8_t *prow = ras.codes + gr * ras.pc;  // packed: indexed by raster column
                const uint8_t *row = prow + C0;
                const uint8_t *mrow = ras.mask ? ras.mask + gr * ras.pm + C0 : nullptr;
                if (c0 >= 0 && c0 + 3 < w) {
                    if (nib) {
                        const int64_t gc = C0 + c0;
                        if (fast) {
                            raw[u] = spread_nibbles(*reinterpret_cast<const uint16_t *>(prow + (gc >> 1)));
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) raw[u] |= nibble_at(prow, gc + j) << (8 * j);
                        }
                    } else if (fast) {
                        raw[u] = *reinterpret_cast<const uint32_t *>(row + c0);
                    } else {
                        raw[u] = (uint32_t)row[c0] | ((uint32_t)row[c0 + 1] << 8) |
                                 ((uint32_t)row[c0 + 2] << 16) | ((uint32_t)row[c0 + 3] << 24);
                    }
                    if (mrow)
                        mraw[u] = (uint32_t)mrow[c0] | ((uint32_t)mrow[c0 + 1] << 8) |
                                  ((uint32_t)mrow[c0 + 2] << 16) | ((uint32_t)mrow[c0 + 3] << 24);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = c0 + j;
                        if (c < -1 || c > w) continue;
                        if (C0 + c < 0 || C0 + c >= ras.cols) continue;
                        raw[u] |= (nib ? nibble_at(prow, C0 + c) : (uint32_t)row[c]) << (8 * j);
                        if (mrow) mraw[u] |= (uint32_t)(mrow[c] ? 1 : 0) << (8 * j);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {  // then convert and store
                const int hr = hr0 + u * nw;
                if (hr >= h + 2 || wd >= words) continue;
                const int64_t gr = R0 - 1 + hr;
                const bool hrow = hr == 0 || hr == h + 1;
                uint32_t v = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = c0 + j;
                    if (c < -1 || c > w) continue;
                    const uint32_t k = (raw[u] >> (8 * j)) & 0xffu;
                    const bool hcell = hrow || c == -1 || c == w;
                    if (k > 9) {
                        if (count_bad && !hcell) {
                            ++nbad;
                            fbad = min(fbad, (long long)(gr * ras.cols + C0 + c));
                        }
                        continue;
                    }
                    if (k == 0 || ((mraw[u] >> (8 * j)) & 0xffu)) continue;
                    v |= k << (8 * j);
                }
                reinterpret_cast<uint32_t *>(ec + hr * S)[wd] = v;
            }
        }
    }
}

// A code byte names a valid cell (1..9: a direction or NoFlow).
__device__ __forceinline__ bool vcode(uint32_t b) { return b - 1u < 9u; }

// acq_rel add on a shared-memory word: the flow a walk stored before it is
// visible to the walk that completes the downstream cell.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "r"(smem_addr(p)), "r"(v)
                 : "memory");
    return old;
}

// Global slot id of the perimeter cell (r + dr, c + dc) just outside the tile
// (ty, tx) of an h x w tile whose cell (r, c) drains there: its tile and its
// slot in that tile.
__device__ __forceinline__ uint32_t outside_slot(const RasterDesc &ras, const TileArgs &a, int ty,
                                                 int tx, int64_t R0, int64_t C0, int h, int w,
                                                 int rr, int cc) {
    const int tyd = ty + (rr < 0 ? -1 : (rr >= h ? 1 : 0));
    const int txd = tx + (cc < 0 ? -1 : (cc >= w ? 1 : 0));
    const int64_t R0d = (int64_t)tyd * a.th, C0d = (int64_t)txd * a.tw;
    const int hd = (int)min((int64_t)a.th, ras.rows - R0d);
    const int wd = (int)min((int64_t)a.tw, ras.cols - C0d);
    const int sd = slot_of((int)(R0 + rr - R0d), (int)(C0 + cc - C0d), hd, wd);
    return (uint32_t)(((size_t)ras.tile_base + (size_t)tyd * ras.tiles_x + txd) * a.pmax + sd);
}

// ---------------------------------------------------------------------------
// The walks of one tile (Algorithm 1).  Warp w holds the queue q[0 .. qn) of
// the cells with no inflow inside the tile from its share of the tile; idle
// lanes take the next queued cells in lane order and walk them downstream.
// ---------------------------------------------------------------------------
template <int MODE, class W>
__device__ __forceinline__ void walk_tile(W *word, FF *val, const uint16_t *q, int qn,
                                          const int *nb) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int pos = 0;              // next queue entry (warp-uniform)
    bool act = false;
    uint32_t sc = SUCC_NONE;  // successor of the lane's cell
    W acc = 0;                // counts: the lane's cell's sum
    // one step of the lane's walk: hand the flow to the successor; go on
    // from it only if this brought its last pending inflow
    auto step = [&]() {
        if (sc == SUCC_NONE) {
            act = false;  // NoFlow: the path ends here
        } else if constexpr (MODE == 0) {
            const W old = atomicAdd(&word[sc], acc - CountWord<W>::ONE);
            act = (old >> CountWord<W>::CNT) == 1;  // the last inflow: continue from sc
            acc += old & CountWord<W>::ACC;
            sc = (uint32_t)(old >> CountWord<W>::SUCC) & SUCC_NONE;
        } else {
            const uint32_t old = atom_add_acq_rel(reinterpret_cast<uint32_t *>(&word[sc]), 0u - GW_ONE);
            act = (old >> GW_CNT) == 1;
            if (act) {  // complete: own weight plus inflows in a fixed order
                const int t = (int)sc;
                FF v = val[t];
                uint32_t pm = (old >> GW_PM) & 0xFFu;
                while (pm) {
                    const int j = __ffs(pm) - 1;
                    pm &= pm - 1u;
                    v = ff_add(v, val[t + nb[j]]);
                }
                val[t] = v;
                sc = old & SUCC_NONE;
            }
        }
    };
    // while the warp's queue lasts, idle lanes take its next cells
    while (pos < qn) {
        const uint32_t idle = __ballot_sync(0xffffffffu, !act);
        if (idle) {
            const int my = pos + __popc(idle & lt);
            if (!act && my < qn) {
                const W wv = word[q[my]];
                if constexpr (MODE == 0) {
                    acc = wv & CountWord<W>::ACC;
                    sc = (uint32_t)(wv >> CountWord<W>::SUCC) & SUCC_NONE;
                } else {
                    sc = (uint32_t)wv & SUCC_NONE;
                }
                act = true;
            }
            pos += __popc(idle);
        }
        if (act) step();
    }
    // then each lane finishes its own walk (the long last walks: no refill
    // bookkeeping per step)
    while (act) step();
}

// ---------------------------------------------------------------------------
// Tile pass.  PASS 1: Algorithm 1 per field, then A_loc at the exits, the
// exit targets and ranks, and the exit each entry cell's path reaches
// (Algorithm 2).  PASS 2: Algorithm 1 per field with the resolved inflow
// added at the entry cells (Algorithm 3), writing the output.  MODE 0: unit
// weights, integer counts; MODE 1: float weights (nf fields).
// Persistent CTAs: each block takes tiles t = blockIdx.x, + gridDim.x, ...
// With TMA the codes of the next tile are staged into shared memory while the
// current one is walked (they are no longer read by then).  The words are
// zero when a tile starts (cleared by the previous tile's last pass), so one
// pass sets every word: each valid cell adds its own (successor, weight) and
// one pending inflow to its successor's word, every other word its SENT_CNT.
// ---------------------------------------------------------------------------
template <int MODE, int PASS, int LOAD>
__global__ void __launch_bounds__(256, MODE == 0 ? 4 : 2) k_walk(const __grid_constant__ TileArgs A,
                                                                const __grid_constant__ CUtensorMap tmap) {
    typedef typename std::conditional<MODE == 0 && PASS == 2, unsigned long long, uint32_t>::type W;
    const TileArgs &a = A;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_warp[33];
    __shared__ int s_flags, s_nent;
    __shared__ int s_nb[8];
    __shared__ __align__(8) uint64_t s_bar;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int th = a.th, tw = a.tw;
    const int S = tile_stride(tw);
    const int W2 = tw + 2, NWD = tile_words(th, tw);
    // wi / W2 as umulhi(wi, rdiv), exact for wi < 2^14 and 3 <= W2 <= 8194
    // (the rounding error wi / 2^32 stays below 1 / W2)
    const uint32_t rdiv = 0xFFFFFFFFu / (uint32_t)W2 + 1u;
    const int64_t T = a.T;
    const int nf = a.nf;
    const W SENT = MODE == 0 ? (W)CountWord<W>::SENT : (W)GW_SENT;
    constexpr int CNT = MODE == 0 ? CountWord<W>::CNT : GW_CNT;
    constexpr int SUCC = MODE == 0 ? CountWord<W>::SUCC : 0;

    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem) + 127) &
                                                ~uintptr_t(127));
    uint8_t *cbuf = base;                                  // byte codes of the tile and its halo
    uint8_t *stage = base + code_buf_bytes(th, tw);        // packed: the TMA stage
    uint8_t *p = stage + (LOAD == LOAD_TMA_PACKED ? packed_buf_bytes(th, tw) : 0);
    W *word = reinterpret_cast<W *>(p);
    p += (size_t)NWD * sizeof(W);
    p = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    FF *val = reinterpret_cast<FF *>(p);
    if (MODE == 1) p += (size_t)NWD * sizeof(FF);
    constexpr bool RETAIN = MODE == 0 && PASS == 1;     // counts: A_loc stays in the output
    uint16_t *queue = reinterpret_cast<uint16_t *>(p);     // walk starts
    p += (size_t)NWD * 2;
    p = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    uint32_t *pexit = reinterpret_cast<uint32_t *>(p);     // slot -> global slot id of its exit target
    p += (size_t)a.pmax * 4;
    uint16_t *prank = reinterpret_cast<uint16_t *>(p);     // slot -> exit rank, LINK_TERM if none
    p += (size_t)a.pmax * 2;
    uint16_t *pent = reinterpret_cast<uint16_t *>(p);      // the entry cells' slots
    p += (size_t)a.pmax * 2;
    uint8_t *pinf = p;                                     // slot -> neighbours outside draining in

    int nbad = 0, ncyc = 0, nonfinite = 0, ovf = 0;
    long long fbad = NO_INDEX;
    uint32_t gmaxw = 0;

    if (tid < 8) s_nb[tid] = dir_dr(tid + 1) * W2 + dir_dc(tid + 1);
    if (tid == 0) {
        s_flags = 0;
        if (LOAD != LOAD_PLAIN) {
            mbar_init(&s_bar, 1);
            mbar_fence_init();
        }
    }
    for (int wi = tid; wi < NWD; wi += nt) word[wi] = 0;
    __syncthreads();
    auto issue = [&](int64_t tn) {  // one thread: stage tile tn's codes (TMA: one raster only)
        const int tyn = (int)(tn / a.one.tiles_x), txn = (int)(tn - (int64_t)tyn * a.one.tiles_x);
        if constexpr (LOAD == LOAD_TMA_PACKED) {  // x in bytes: (C0 - PX0) / 2, a multiple of 16
            mbar_expect_tx(&s_bar, (uint32_t)((th + 2) * packed_box_bytes(tw)));
            tma_load_2d(stage, &tmap, (txn * tw - PX0) / 2, tyn * th - 1, &s_bar);
        } else {
            mbar_expect_tx(&s_bar, (uint32_t)((th + 2) * S));
            tma_load_2d(cbuf, &tmap, txn * tw - X0, tyn * th - 1, &s_bar);
        }
    };
    if (LOAD != LOAD_PLAIN && tid == 0 && blockIdx.x < T) issue(blockIdx.x);

    int it = 0;
    bool timed_out = false;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++it) {
        const RasterDesc &ras = raster_of(a, t);
        const int lt = (int)(t - ras.tile_base);
        const int ty = lt / ras.tiles_x, tx = lt - ty * ras.tiles_x;
        const int64_t R0 = (int64_t)ty * th, C0 = (int64_t)tx * tw;
        const int h = (int)min((int64_t)th, ras.rows - R0);
        const int w = (int)min((int64_t)tw, ras.cols - C0);
        const int P = perim_count(h, w);
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = tid; s < a.pmax; s += nt) {
            pexit[s] = NODE_NONE;
            prank[s] = LINK_TERM;
            pinf[s] = 0;
        }
        if (tid == 0) s_nent = 0;

        // [phase] codes of the tile and its one-cell halo ring
        if constexpr (LOAD != LOAD_PLAIN) {
            if (tid == 0 && !mbar_wait(&s_bar, (uint32_t)(it & 1), a.wait_ns)) s_flags |= FA_FLAG_TIMEOUT;
            __syncthreads();
            if (s_flags & FA_FLAG_TIMEOUT) {
                timed_out = true;
                break;
            }
            if constexpr (LOAD == LOAD_TMA_PACKED) {
                // spread the packed box to one byte per cell: code-buffer word
                // wd (cells C0 - X0 + 4wd ..) is box bytes 2wd + 8 and 2wd + 9.
                // Cells right of the raster are NoData, the spare high nibble of
                // an odd-width row included (left of it and above or below it
                // the box already reads 0).
                const int PB = packed_box_bytes(tw), W4 = S >> 2;
                for (int i = tid; i < (th + 2) * W4; i += nt) {
                    const int hr = i / W4, wd = i - hr * W4;
                    uint32_t v = spread_nibbles(*reinterpret_cast<const uint16_t *>(stage + hr * PB + 2 * wd + 8));
                    const int64_t keep = ras.cols - (C0 - X0 + 4 * wd);  // cells of the word inside
                    if (keep < 4) v = keep <= 0 ? 0u : (v & ((1u << (8 * keep)) - 1u));
                    reinterpret_cast<uint32_t *>(cbuf + hr * S)[wd] = v;
                }
                fence_proxy_async();
                __syncthreads();
                if (tid == 0 && t + gridDim.x < T) issue(t + gridDim.x);  // the stage is free again
            }
        } else {
            load_codes(ras, cbuf, R0, C0, h, w, S, a.nib != 0, PASS == 1, nbad, fbad);
            __syncthreads();
        }

        // [phase] init, one pass over every word (tile and ring): a valid
        // cell adds its own successor and unit weight to its word and one
        // pending inflow (with its direction bit for float weights) to the
        // word its code points at; any other word adds its SENT_CNT
        for (int wi = tid; wi < NWD; wi += nt) {
            const int hr = (int)__umulhi((uint32_t)wi, rdiv), r = hr - 1, c = wi - hr * W2 - 1;
            const bool tile = (unsigned)r < (unsigned)h && (unsigned)c < (unsigned)w;
            const uint32_t k = tile ? cbuf[hr * S + X0 + c] : 0u;
            if constexpr (LOAD != LOAD_PLAIN && PASS == 1) {  // raw staged codes
                if (tile && k > 9u) {
                    ++nbad;
                    fbad = min(fbad, (long long)((R0 + r) * ras.cols + (C0 + c)));
                }
            }
            if (!vcode(k)) {
                atomicAdd(&word[wi], SENT);
                continue;
            }
            uint32_t sc = SUCC_NONE;
            if (k <= 8u) {
                sc = (uint32_t)(wi + dir_dr((int)k) * W2 + dir_dc((int)k));
                if constexpr (MODE == 0) atomicAdd(&word[sc], CountWord<W>::ONE);
                else atomicAdd(&word[sc], GW_ONE | (1u << (GW_PM + dir_rev((int)k) - 1)));
            }
            if constexpr (MODE == 0) atomicAdd(&word[wi], ((W)sc << SUCC) | (W)1);
            else atomicAdd(&word[wi], sc | GW_VALID);
        }
        // the perimeter: exits (flow into a valid cell of another tile) and
        // the outside neighbours draining into each perimeter cell
        for (int s = tid; s < P; s += nt) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int k = cbuf[(r + 1) * S + X0 + c];
            if (!vcode(k)) continue;
            if (PASS == 1 && k <= 8) {
                const int tr = r + dir_dr(k), tc = c + dir_dc(k);
                if (((unsigned)tr >= (unsigned)h || (unsigned)tc >= (unsigned)w) &&
                    vcode(cbuf[(tr + 1) * S + X0 + tc]))
                    pexit[s] = outside_slot(ras, a, ty, tx, R0, C0, h, w, tr, tc);
            }
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int nr = r + dir_dr(j + 1), nc = c + dir_dc(j + 1);
                if ((unsigned)nr < (unsigned)h && (unsigned)nc < (unsigned)w) continue;
                const int kh = cbuf[(nr + 1) * S + X0 + nc];
                if (kh >= 1 && kh <= 8 && nr + dir_dr(kh) == r && nc + dir_dc(kh) == c) m |= 1u << j;
            }
            pinf[s] = (uint8_t)m;
            if (PASS == 1 && m) pent[atomicAdd(&s_nent, 1)] = (uint16_t)s;
        }
        if constexpr (LOAD == LOAD_TMA) fence_proxy_async();  // the code buffer is refilled by TMA
        __syncthreads();
        if constexpr (LOAD == LOAD_TMA) {
            if (tid == 0 && t + gridDim.x < T) issue(t + gridDim.x);
        }

        // the cells with no inflow inside the tile start the walks: warp w
        // queues those of its share of the words (32-word chunks c0 .. c1)
        const int nch = (NWD + 31) >> 5;
        const int c0 = (int)((int64_t)nch * warp / nw), c1 = (int)((int64_t)nch * (warp + 1) / nw);
        uint16_t *wq = queue + c0 * 32;
        int qn = 0;
        for (int ch = c0; ch < c1; ++ch) {
            const int wi = ch * 32 + lane;
            const bool leaf = wi < NWD && (word[wi] >> CNT) == 0;
            const uint32_t b = __ballot_sync(0xffffffffu, leaf);
            if (leaf) wq[qn + __popc(b & ((1u << lane) - 1u))] = (uint16_t)wi;
            qn += __popc(b);
        }
        __syncwarp();

        // exit ranks in slot order (pass 1)
        int nexits = 0;
        if constexpr (PASS == 1) {
            const int chunk = (P + nt - 1) / nt;
            const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
            int mine = 0;
            for (int s = s0; s < s1; ++s) mine += pexit[s] != NODE_NONE;
            int rk = block_exclusive_scan(mine, s_warp, &nexits);
            for (int s = s0; s < s1; ++s) {
                const uint32_t dst = pexit[s];
                if (dst == NODE_NONE) {
                    a.link[tbase + s] = LINK_TERM;
                    continue;
                }
                prank[s] = (uint16_t)rk;
                a.node_dst[tbase + rk] = dst;
                a.link[tbase + s] = (uint16_t)rk;  // an exit's path reaches itself
                ++rk;
            }
        }

        // [phase] walk, once per field
        for (int f = 0; f < nf; ++f) {
            if constexpr (MODE == 1) {
                const float *wp = ras.w[f];
                for (int wi = tid; wi < NWD; wi += nt) {
                    const uint32_t wv = word[wi];
                    if (!(wv & GW_VALID)) {  // not a valid cell of the tile: its sentinel again
                        if (f > 0)
                            word[wi] = (wv & ((1u << GW_CNT) - 1u)) |
                                       ((SENT_CNT + (uint32_t)__popc((wv >> GW_PM) & 0xFFu)) << GW_CNT);
                        continue;
                    }
                    const int hr = (int)__umulhi((uint32_t)wi, rdiv), r = hr - 1, c = wi - hr * W2 - 1;
                    const float wf = wp ? wp[(R0 + r) * ras.pw + (C0 + c)] : 1.0f;
                    if constexpr (PASS == 1) {
                        const uint32_t b = __float_as_uint(wf) & 0x7fffffffu;
                        if (b >= 0x7f800000u) nonfinite = 1;
                        gmaxw = max(gmaxw, b);
                    }
                    val[wi] = FF{wf, 0.0f};
                    if (f > 0)  // the pending counts again, from the inflow mask
                        word[wi] = (wv & ((1u << GW_CNT) - 1u)) |
                                   ((uint32_t)__popc((wv >> GW_PM) & 0xFFu) << GW_CNT);
                }
            }
            if constexpr (PASS == 2) {
                // the flow entering from other tiles, added at its entry cell
                // (Algorithm 3), summed over the outside neighbours in a fixed
                // order (float pairs: after the cell's own weight is in place)
                if constexpr (MODE == 1) __syncthreads();
                const int qf = MODE == 1 ? fix_scale(a.fcells, *a.maxw) : 0;
                for (int s = tid; s < P; s += nt) {
                    uint32_t m = pinf[s];
                    if (!m) continue;
                    int r, c;
                    cell_of(s, h, w, r, c);
                    const int wi = (r + 1) * W2 + c + 1;
                    FF v;
                    if constexpr (MODE == 1) v = val[wi];
                    unsigned long long add = 0;
                    while (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1u;
                        const uint32_t src = outside_slot(ras, a, ty, tx, R0, C0, h, w,
                                                          r + dir_dr(j + 1), c + dir_dc(j + 1));
                        const uint16_t lk = a.link[src];  // the exit's own rank
                        if (lk == LINK_TERM) continue;
                        const size_t node = (size_t)(src - src % (uint32_t)a.pmax) + lk;
                        if constexpr (MODE == 0) {
                            add += reinterpret_cast<const unsigned long long *>(a.G)[node];
                        } else {
                            v = ff_add(v, fix2ff(reinterpret_cast<const u128 *>(a.G)[node * nf + f], qf));
                        }
                    }
                    if constexpr (MODE == 0) word[wi] += (W)add;
                    else val[wi] = v;
                }
            }
            __syncthreads();

            walk_tile<MODE, W>(word, val, wq, qn, s_nb);
            __syncthreads();

            if constexpr (PASS == 1) {
                // A_loc at every exit: the perimeter data of Section 3.2
                for (int s = tid; s < P; s += nt) {
                    const uint16_t rk = prank[s];
                    if (rk == LINK_TERM) continue;
                    int r, c;
                    cell_of(s, h, w, r, c);
                    const int wi = (r + 1) * W2 + c + 1;
                    double v;
                    if constexpr (MODE == 0) v = (double)(word[wi] & CountWord<W>::ACC);
                    else v = (double)val[wi].hi + (double)val[wi].lo;
                    a.node_val[(tbase + rk) * nf + f] = v;
                }
            } else {
                // the output raster of field f: A at complete cells, 0 at
                // NoData (and on cycles); the words are cleared for the next
                // tile after the last field
                const bool last = f == nf - 1;
                for (int wi = tid; wi < NWD; wi += nt) {
                    const W wv = word[wi];
                    if (last) word[wi] = 0;
                    const int hr = (int)__umulhi((uint32_t)wi, rdiv), r = hr - 1, c = wi - hr * W2 - 1;
                    if ((unsigned)r >= (unsigned)h || (unsigned)c >= (unsigned)w) continue;
                    uint32_t o = 0;
                    if ((wv >> CNT) == 0) {
                        if constexpr (MODE == 0) {
                            const unsigned long long s64 = (unsigned long long)(wv & CountWord<W>::ACC);
                            ovf |= (s64 >> 32) != 0;
                            o = (uint32_t)s64;
                        } else {
                            o = __float_as_uint(ff_round(val[wi]));
                        }
                    }
                    reinterpret_cast<uint32_t *>(ras.out[f])[(size_t)(R0 + r) * ras.po + C0 + c] = o;
                }
            }
            if (f + 1 < nf) __syncthreads();
        }

        if constexpr (PASS == 1) {
            // Algorithm 2 for the entry cells: the exit each one's path
            // reaches (the last valid cell of the tile on it, if on the
            // perimeter and an exit); one entry per lane at a time
            for (int e = tid; e < s_nent; e += nt) {
                const int slot = pent[e];
                int r, c;
                cell_of(slot, h, w, r, c);
                int cur = (r + 1) * W2 + c + 1, steps = 0;
                W wc = word[cur];
                for (;;) {
                    const uint32_t sc = (uint32_t)(wc >> SUCC) & SUCC_NONE;
                    if (sc == SUCC_NONE) break;
                    const W wn = word[sc];
                    if ((wn >> CNT) >= SENT_CNT) break;  // leaves the tile or the data
                    if (++steps > h * w) {              // a cycle: the path never ends
                        cur = -1;
                        break;
                    }
                    cur = (int)sc;
                    wc = wn;
                }
                uint16_t lk = LINK_TERM;
                if (cur >= 0) {
                    const int hr = (int)__umulhi((uint32_t)cur, rdiv), rr = hr - 1, cc = cur - hr * W2 - 1;
                    if (rr == 0 || cc == 0 || rr == h - 1 || cc == w - 1) lk = prank[slot_of(rr, cc, h, w)];
                }
                a.link[tbase + slot] = lk;
            }
        }
        if constexpr (PASS == 1) {
            if (tid == 0) a.nexit[t] = (uint32_t)nexits;
            __syncthreads();
            // cells still waiting for an inflow lie on a cycle inside the
            // tile (a cycle cell misses exactly its predecessor on the
            // cycle); counts: A_loc goes to the output raster (0 at NoData
            // and on cycles); the words are cleared for the next tile
            for (int wi = tid; wi < NWD; wi += nt) {
                const W wv = word[wi];
                word[wi] = 0;
                const int hr = (int)__umulhi((uint32_t)wi, rdiv), r = hr - 1, c = wi - hr * W2 - 1;
                if ((wv >> CNT) == 1) {
                    ++ncyc;
                    fbad = min(fbad, (long long)((R0 + r) * ras.cols + (C0 + c)));
                }
                if constexpr (RETAIN) {
                    if ((unsigned)r < (unsigned)h && (unsigned)c < (unsigned)w)
                        reinterpret_cast<uint32_t *>(ras.out[0])[(size_t)(R0 + r) * ras.po + C0 + c] =
                            (wv >> CNT) == 0 ? (uint32_t)(wv & CountWord<W>::ACC) : 0u;
                }
            }
        }
        __syncthreads();
        // [phase] end
    }

    // ---- status -------------------------------------------------------------
    __shared__ int s_cnt_bad, s_cnt_cyc;
    __shared__ long long s_first;
    __shared__ uint32_t s_maxw;
    if (tid == 0) {
        s_cnt_bad = 0;
        s_cnt_cyc = 0;
        s_first = NO_INDEX;
        s_maxw = 0;
    }
    __syncthreads();
    nbad = warp_sum(nbad);
    ncyc = warp_sum(ncyc);
    fbad = warp_min_ll(fbad);
    gmaxw = warp_max_u(gmaxw);
    nonfinite = warp_sum(nonfinite);
    ovf = warp_sum(ovf);
    if (lane == 0) {
        if (nbad) atomicAdd(&s_cnt_bad, nbad);
        if (ncyc) atomicAdd(&s_cnt_cyc, ncyc);
        if (fbad != NO_INDEX) atomicMin(&s_first, fbad);
        if (gmaxw) atomicMax(&s_maxw, gmaxw);
        if (nonfinite) atomicOr(&s_flags, FA_FLAG_NONFINITE);
        if (ovf) atomicOr(&s_flags, FA_FLAG_OVERFLOW);
    }
    __syncthreads();
    if (tid == 0) {
        int fl = s_flags;
        if (s_cnt_bad) fl |= FA_FLAG_BAD_CODE;
        if (s_cnt_cyc) fl |= FA_FLAG_CYCLE;
        if (fl) status_report(a.st, fl, s_cnt_bad + s_cnt_cyc, s_first);
        if (s_maxw) atomicMax(a.maxw, s_maxw);
        // a wait that ran out may leave its copy in flight into this block's
        // shared memory: wait for it once more (bounded) before exiting
        if (LOAD != LOAD_PLAIN && timed_out) mbar_wait(&s_bar, (uint32_t)(it & 1), a.wait_ns);
    }
}

// ---------------------------------------------------------------------------
// Pass 2 for counts (Algorithm 3, Section 3.3).  Pass 1 left A_loc in the
// output.  The flow arriving at entry cell p from outside, in(p), is the sum
// of G over the exits outside the tile that drain into p (the resolve added
// each exit's G to the perimeter slot of the cell it drains into), and it
// reaches every cell on p's path inside the tile; where paths merge, each
// adds its own in(p) below the merge.  So this pass stages the tile's codes
// again (two buffers: the next tile's copy overlaps this tile's walks) and
// walks each entry's path, adding in(p) to the output as reductions in L2.
// Integer adds: their order does not matter.  Whether a count of the tile
// can reach 2^32 is known up front (A_loc plus the tile's whole inflow bounds
// every count); only then are the adds made as atomics that return the old
// value, to flag the overflow.
// ---------------------------------------------------------------------------
constexpr int ADDIN_THREADS = 128;

__host__ __device__ inline size_t addin_smem_bytes(int th, int tw, int load) {
    const size_t cb = code_buf_bytes(th, tw), pb = packed_buf_bytes(th, tw);
    const size_t bufs = load == LOAD_TMA ? 2 * cb : (load == LOAD_TMA_PACKED ? cb + 2 * pb : cb);
    const int pm = 2 * th + 2 * tw;
    return 128 + bufs + (size_t)pm * 8 + (size_t)pm * 2 + 16;
}

template <int LOAD>
__global__ void __launch_bounds__(ADDIN_THREADS, 8) k_addin(const __grid_constant__ TileArgs A,
                                                          const __grid_constant__ CUtensorMap tmap) {
    const TileArgs &a = A;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_n, s_flags;
    __shared__ int s_oc[8];          // code k -> step in the staged codes
    __shared__ long long s_oo[8];    // code k -> step in the output raster (its pitch)
    __shared__ unsigned long long s_tot;
    __shared__ __align__(8) uint64_t s_bar[2];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int th = a.th, tw = a.tw, S = tile_stride(tw);
    const int64_t T = a.T;

    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem) + 127) &
                                                ~uintptr_t(127));
    const size_t cbb = code_buf_bytes(th, tw), pbb = packed_buf_bytes(th, tw);
    // TMA targets: two code buffers (bytes), or two packed stages spread into
    // one code buffer; plain loads fill the one code buffer
    uint8_t *cb0 = base;
    uint8_t *cb1 = LOAD == LOAD_TMA ? base + cbb : base;
    uint8_t *st0 = base + cbb, *st1 = base + cbb + pbb;
    uint8_t *p = base + (LOAD == LOAD_TMA ? 2 * cbb : (LOAD == LOAD_TMA_PACKED ? cbb + 2 * pbb : cbb));
    unsigned long long *pin = reinterpret_cast<unsigned long long *>(p);  // entry -> in(p)
    p += (size_t)a.pmax * 8;
    uint16_t *pent = reinterpret_cast<uint16_t *>(p);                    // entry -> its slot

    // thread 0 keeps the copies' bookkeeping: the parity each buffer's
    // barrier completes next and whether a copy into it is in flight
    uint32_t ph0 = 0, ph1 = 0;
    bool fl0 = false, fl1 = false;
    auto issue = [&](int64_t tn, int b) {  // one thread: stage tile tn's codes into buffer b
        const int tyn = (int)(tn / a.one.tiles_x), txn = (int)(tn - (int64_t)tyn * a.one.tiles_x);
        uint64_t *bar = &s_bar[b];
        if constexpr (LOAD == LOAD_TMA_PACKED) {  // x in bytes: (C0 - PX0) / 2, a multiple of 16
            mbar_expect_tx(bar, (uint32_t)((th + 2) * packed_box_bytes(tw)));
            tma_load_2d(b ? st1 : st0, &tmap, (txn * tw - PX0) / 2, tyn * th - 1, bar);
        } else {
            mbar_expect_tx(bar, (uint32_t)((th + 2) * S));
            tma_load_2d(b ? cb1 : cb0, &tmap, txn * tw - X0, tyn * th - 1, bar);
        }
        if (b) fl1 = true;
        else fl0 = true;
    };
    if (tid == 0) {
        s_flags = 0;
        if (LOAD != LOAD_PLAIN) {
            mbar_init(&s_bar[0], 1);
            mbar_init(&s_bar[1], 1);
            mbar_fence_init();
        }
    }
    __syncthreads();
    if (LOAD != LOAD_PLAIN && tid == 0) {
        if (blockIdx.x < T) issue(blockIdx.x, 0);
        if (blockIdx.x + gridDim.x < T) issue(blockIdx.x + gridDim.x, 1);
    }

    int ovf = 0;
    int it = 0;
    bool timed_out = false;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++it) {
        const int bi = it & 1;
        const RasterDesc &ras = raster_of(a, t);
        const int lt = (int)(t - ras.tile_base);
        const int ty = lt / ras.tiles_x, tx = lt - ty * ras.tiles_x;
        const int64_t R0 = (int64_t)ty * th, C0 = (int64_t)tx * tw;
        const int h = (int)min((int64_t)th, ras.rows - R0);
        const int w = (int)min((int64_t)tw, ras.cols - C0);
        const int P = perim_count(h, w);
        if (tid == 0) {
            s_n = 0;
            s_tot = 0;
        }
        uint8_t *cbuf = LOAD == LOAD_TMA ? (bi ? cb1 : cb0) : cb0;
        __syncthreads();

        // ---- entry cells: the perimeter slots that receive flow from outside
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = tid; s < P; s += nt) {
            const unsigned long long in = a.infl[tbase + s];
            if (!in) continue;
            const int e = atomicAdd(&s_n, 1);
            pent[e] = (uint16_t)s;
            pin[e] = in;
            atomicAdd(&s_tot, in);
        }

        // ---- codes of the tile and its ring
        if constexpr (LOAD != LOAD_PLAIN) {
            if (tid == 0) {
                const bool ok = mbar_wait(&s_bar[bi], bi ? ph1 : ph0, a.wait_ns);
                if (ok) {
                    if (bi) { ph1 ^= 1u; fl1 = false; }
                    else { ph0 ^= 1u; fl0 = false; }
                } else {
                    s_flags |= FA_FLAG_TIMEOUT;
                }
            }
            __syncthreads();
            if (s_flags & FA_FLAG_TIMEOUT) {
                timed_out = true;
                break;
            }
            if constexpr (LOAD == LOAD_TMA_PACKED) {
                const uint8_t *stage = bi ? st1 : st0;
                const int PB = packed_box_bytes(tw), W4 = S >> 2;
                for (int i = tid; i < (th + 2) * W4; i += nt) {
                    const int hr = i / W4, wd = i - hr * W4;
                    uint32_t v = spread_nibbles(*reinterpret_cast<const uint16_t *>(stage + hr * PB + 2 * wd + 8));
                    const int64_t keep = ras.cols - (C0 - X0 + 4 * wd);  // cells of the word inside
                    if (keep < 4) v = keep <= 0 ? 0u : (v & ((1u << (8 * keep)) - 1u));
                    reinterpret_cast<uint32_t *>(cbuf + hr * S)[wd] = v;
                }
                fence_proxy_async();
                __syncthreads();
                if (tid == 0 && t + 2 * (int64_t)gridDim.x < T) issue(t + 2 * (int64_t)gridDim.x, bi);
            }
        } else {
            int nb0 = 0;
            long long fb0 = NO_INDEX;
            load_codes(ras, cbuf, R0, C0, h, w, S, a.nib != 0, false, nb0, fb0);
            __syncthreads();
        }

        // ---- each entry's path inside the tile receives its in(p).  The
        // staged codes outside the tile (the ring, and the frame beyond a
        // ragged tile) get the bit 0x80, so that one test on the next cell's
        // code tells "leaves the tile" and "into NoData" both; a step is then
        // one code read (kept as the next step's code), two table steps and
        // the output update.
        const int W2 = tw + 2;
        for (int i = tid; i < (th + 2 - h) * W2; i += nt) {  // rows -1 and h .. th
            const int q = i / W2, c = i - q * W2 - 1, hr = q == 0 ? 0 : h + q;
            cbuf[hr * S + X0 + c] |= 0x80;
        }
        for (int i = tid; i < h * (tw + 2 - w); i += nt) {   // columns -1 and w .. tw of rows 0 .. h-1
            const int nc = tw + 2 - w, r = i / nc, q = i - r * nc, c = q == 0 ? -1 : w + q - 1;
            cbuf[(r + 1) * S + X0 + c] |= 0x80;
        }
        if (tid < 8) {
            s_oc[tid] = dir_dr(tid + 1) * S + dir_dc(tid + 1);
            s_oo[tid] = (long long)dir_dr(tid + 1) * ras.po + dir_dc(tid + 1);
        }
        __syncthreads();
        const int ne = s_n;
        const bool safe = s_tot + (unsigned long long)h * w < (1ull << 32);  // no count reaches 2^32
        uint32_t *out = reinterpret_cast<uint32_t *>(ras.out[0]);
        unsigned long long *o64 = a.off64;  // uint64 offsets (the out-of-core blocks)
        for (int e = tid; e < ne; e += nt) {
            int r, c;
            cell_of(pent[e], h, w, r, c);
            const unsigned long long v = pin[e];
            int ci = (r + 1) * S + X0 + c;
            size_t oi = (size_t)(R0 + r) * ras.po + (size_t)(C0 + c);
            uint32_t k = cbuf[ci];  // the code of the cell the path is at
            for (int stp = 0; stp < h * w; ++stp) {
                if (o64) {
                    atomicAdd(o64 + oi, v);  // a reduction
                } else if (safe) {
                    atomicAdd(out + oi, (uint32_t)v);  // result unused: a reduction
                } else {
                    const uint32_t old = atomicAdd(out + oi, (uint32_t)v);
                    if ((v >> 32) || (unsigned long long)old + (uint32_t)v >= (1ull << 32)) ovf = 1;
                }
                if (k - 1u >= 8u) break;  // NoFlow: the path ends
                const int nci = ci + s_oc[k - 1];
                const uint32_t kn = cbuf[nci];
                if (kn - 1u >= 9u) break;  // leaves the tile, or into NoData
                ci = nci;
                oi += s_oo[k - 1];
                k = kn;  // one code read per step
            }
        }
        if constexpr (LOAD == LOAD_TMA) fence_proxy_async();  // the buffer is refilled by TMA
        __syncthreads();
        if constexpr (LOAD == LOAD_TMA) {
            if (tid == 0 && t + 2 * (int64_t)gridDim.x < T) issue(t + 2 * (int64_t)gridDim.x, bi);
        }
    }
    ovf = __syncthreads_or(ovf);
    if (tid == 0) {
        int fl = s_flags | (ovf ? FA_FLAG_OVERFLOW : 0);
        if (fl) status_report(a.st, fl, 0, NO_INDEX);
        // a wait that ran out may leave copies in flight into this block's
        // shared memory: wait for them once more (bounded) before exiting
        if (LOAD != LOAD_PLAIN && timed_out) {
            if (fl0) mbar_wait(&s_bar[0], ph0, a.wait_ns);
            if (fl1) mbar_wait(&s_bar[1], ph1, a.wait_ns);
        }
    }
}

// ---------------------------------------------------------------------------
// perimeter-graph (exit forest) resolve; nf values per node, one pointer
// structure shared by all fields
// ---------------------------------------------------------------------------
struct ForestArgs {
    int64_t tiles, nodes;  // nodes: tiles * pmax (bounds a walk)
    int pmax, nf;
    int64_t cells;
    int valm;
    const uint32_t *nexit;
    const uint16_t *link;
    const uint32_t *node_dst;
    const double *node_val;
    void *x;  // u64 (counts) or u128 (fixed-point sums) per node and field
    uint32_t *J0;  // successor node (the exit its target entry cell links to) or NODE_NONE
    uint32_t *J1;  // predecessors still to come
    uint32_t *misc;  // [0] max|w| bits, [1] nodes finished by the walks
    StatusBlock *st;
    unsigned long long *infl;  // counts: per perimeter slot, the flow arriving from outside, or NULL
    const unsigned long long *inj;   // counts: per perimeter slot, flow entering from beyond the raster, or NULL
    const unsigned long long *injx;  // counts: per exit slot, that flow reaching the exit, or NULL
};

// Node values: uint64 counts (unit weights) or 128-bit fixed-point sums.
__device__ __forceinline__ void atomic_add_v(unsigned long long *p, unsigned long long v) {
    atomicAdd(p, v);
}
__device__ __forceinline__ void atomic_add_v(u128 *p, u128 v) { atomic_add_u128(p, v); }

template <class V>
__global__ void k_forest_init(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    V *x = reinterpret_cast<V *>(f.x);
    const uint32_t n = f.nexit[tile];
    const int q = f.valm ? fix_scale(f.cells, f.misc[0]) : 0;
    const size_t base = (size_t)tile * f.pmax;
    if (f.infl)
        for (int j = lane; j < f.pmax; j += 32) f.infl[base + j] = f.inj ? f.inj[base + j] : 0ull;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        for (int k = 0; k < f.nf; ++k) {
            const size_t i = node * f.nf + k;
            const double v = f.node_val[i];
            if constexpr (sizeof(V) == 8) x[i] = (V)v;  // an exact integer count
            else x[i] = f.valm ? d2fix(v, q) : (u128)(unsigned long long)v;
        }
        const uint32_t dst = f.node_dst[node];
        const uint16_t l = f.link[dst];
        f.J0[node] = l == LINK_TERM ? NODE_NONE : (dst / f.pmax) * f.pmax + l;
        f.J1[node] = 0;
    }
    if constexpr (sizeof(V) == 8) {
        // flow entering the tile from beyond the raster (an outer block's
        // inflow) joins the value of the exit its path reaches: injx is
        // keyed by that exit's slot, whose link is the exit's own rank
        if (f.injx) {
            __syncwarp();
            for (int j = lane; j < f.pmax; j += 32) {
                const unsigned long long v = f.injx[base + j];
                const uint16_t l = v ? f.link[base + j] : LINK_TERM;
                if (l != LINK_TERM) atomicAdd(&x[base + l], (V)v);
            }
        }
    }
}

// The exit forest solved the way a tile is (Algorithm 1 on the perimeter
// graph of Section 3.2): J1 counts each node's predecessors (k_forest_indeg);
// the nodes without one are marked (k_forest_leaves) and each starts a walk
// (k_forest_walk) that adds its finished value G into its successor's and
// moves on when it brought the successor's last inflow, so each node is
// passed on once.  Values and counts are separate words in global memory: the
// count goes down by an acquire-release atomic, so a walk's adds are visible
// before it takes one off the count, and the walk that takes the last one
// reads the successor's value after that (loads that bypass L1).  Integer
// adds: the order in which they land does not matter.
template <class V>
__global__ void k_forest_indeg(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32) {
        const uint32_t s = f.J0[base + j];
        if (s != NODE_NONE) atomicAdd(&f.J1[s], 1u);
    }
}

// Marks the nodes without predecessors (the walks start there) before any
// walk runs: a count that the walks bring to zero must not pass for one.
constexpr uint32_t WALK_START = 0x80000000u;
template <class V>
__global__ void k_forest_leaves(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32)
        if (f.J1[base + j] == 0) f.J1[base + j] = WALK_START;
}

__device__ __forceinline__ unsigned long long load_cg(const unsigned long long *p) { return __ldcg(p); }
__device__ __forceinline__ u128 load_cg(const u128 *p) {
    const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
    return (u128)__ldcg(q) | ((u128)__ldcg(q + 1) << 64);
}

// One pending inflow fewer at a node: acquire-release at GPU scope, so the
// value adds a walk made before it are visible to the walk that takes the
// last inflow, which reads the value after it (no separate fences).
__device__ __forceinline__ uint32_t dec_acq_rel_gpu(uint32_t *p) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(0xFFFFFFFFu)
                 : "memory");
    return old;
}

template <class V>
__global__ void k_forest_walk(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    V *x = reinterpret_cast<V *>(f.x);
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int done = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        size_t u = base + j;
        if (f.J1[u] != WALK_START) continue;  // waits for inflow: another walk finishes it
        ++done;
        for (int64_t steps = 0; steps <= f.nodes; ++steps) {
            const uint32_t v = f.J0[u];
            if (v == NODE_NONE) break;  // its path ends inside the target tile
            for (int q = 0; q < f.nf; ++q)
                atomic_add_v(&x[(size_t)v * f.nf + q], load_cg(&x[u * f.nf + q]));
            if (dec_acq_rel_gpu(&f.J1[v]) != 1u) break;  // not the last inflow of v
            u = v;
            ++done;
        }
    }
    done = warp_sum(done);
    if (lane == 0 && done) atomicAdd(&f.misc[1], (uint32_t)done);
}

// Nodes whose count never reached zero lie on a cycle across tiles.
template <class V>
__global__ void k_forest_final(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int ncyc = 0;
    for (uint32_t j = lane; j < n; j += 32) ncyc += f.J1[base + j] != 0 && f.J1[base + j] != WALK_START;
    if constexpr (sizeof(V) == 8) {
        // counts: each exit's G to the perimeter slot of the cell it drains
        // into, for the finalising pass (Algorithm 3's offsets)
        if (f.infl) {
            const V *x = reinterpret_cast<const V *>(f.x);
            for (uint32_t j = lane; j < n; j += 32) atomicAdd(&f.infl[f.node_dst[base + j]], x[base + j]);
        }
    }
    ncyc = warp_sum(ncyc);
    if (lane == 0 && ncyc) status_report(f.st, FA_FLAG_CYCLE, ncyc, NO_INDEX);
}

__global__ void k_init_status(StatusBlock *st, uint32_t *misc, int nmisc) {
    const int i = threadIdx.x;
    if (i == 0) {
        st->flags = 0;
        st->count = 0;
        st->first = NO_INDEX;
    }
    for (int j = i; j < nmisc; j += blockDim.x) misc[j] = 0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool make_geom(int64_t rows, int64_t cols, const fa_options *opts, Geom &g) {
    int th = 64, tw = 64;
    if (opts && opts->tile_h) th = opts->tile_h;
    if (opts && opts->tile_w) tw = opts->tile_w;
    // any form's largest tile (the forward kernels' own limit is tile_shape_ok)
    if (th < 1 || tw < 1 || (int64_t)th * tw > 16384) return false;
    if (rows < 0 || cols < 0) return false;
    g.rows = rows;
    g.cols = cols;
    g.th = th;
    g.tw = tw;
    g.tiles_y = (int)((rows + th - 1) / th);
    g.tiles_x = (int)((cols + tw - 1) / tw);
    g.pmax = 2 * th + 2 * tw;
    g.flags = opts ? opts->flags : 0;
    g.code_format = opts ? opts->code_format : FA_CODES_BYTE;
    g.nf = 1;
    if (g.code_format != FA_CODES_BYTE && g.code_format != FA_CODES_NIBBLE) return false;
    // node ids are tile * pmax + rank in 32 bits
    if ((double)g.tiles() * g.pmax >= 4.0e9) return false;
    return true;
}

bool forward_tile_ok(const Geom &g, int valm) { return tile_shape_ok(g.th, g.tw, valm); }

static int jump_rounds(int64_t max_nodes) {
    int k = 1;
    while (k < 40 && ((int64_t)1 << k) <= max_nodes) ++k;
    return k + 1;
}

size_t carve_forward(void *ws, size_t bytes, const Geom &g, FwdWork &w, bool dry) {
    Carver c(ws, bytes);
    const size_t T = (size_t)g.tiles(), S = T * g.pmax, SV = S * (size_t)std::max(1, g.nf);
    w.kmax = jump_rounds((int64_t)S);
    w.status = c.take<uint8_t>(64);
    w.misc = c.take<uint32_t>(2 + w.kmax);
    w.nexit = c.take<uint32_t>(T);
    w.link = c.take<uint16_t>(S);
    w.node_dst = c.take<uint32_t>(S);
    w.node_val = c.take<double>(SV);
    w.x = c.take<u128>(SV);
    w.J0 = c.take<uint32_t>(S);
    w.J1 = c.take<uint32_t>(S);
    w.infl = c.take<unsigned long long>(S);
    (void)dry;
    return c.used() + 256;
}

template <class K>
static cudaError_t set_smem(K kern, size_t smem, int &configured) {
    if (smem > 48 * 1024 && configured < (int)smem) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = (int)smem;
    }
    return cudaSuccess;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against libcuda); nullptr when unavailable
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// TMA staging of code tiles: a 2-D uint8 map over the raster with a box of
// tile_stride(tw) x (th + 2) bytes.  Needs a 16-byte aligned base and pitch,
// a tile width that is a multiple of 16 (so every box starts on a 16-byte
// column), box sides <= 256 and no separate mask raster.  Packed codes: a map
// over the (cols + 1) / 2 bytes of each row with a box of
// packed_box_bytes(tw) x (th + 2) bytes; the tile width must be a multiple of
// 32 so that every box starts on a 16-byte column ((C0 - PX0) / 2 bytes).
static bool make_code_map(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                          bool packed, CUtensorMap *m) {
    if (mask || !codes) return false;
    if (((uintptr_t)codes & 15) || (pc & 15) || (g.tw & (packed ? 31 : 15))) return false;
    const int S = packed ? packed_box_bytes(g.tw) : tile_stride(g.tw);
    if (S > 256 || g.th + 2 > 256) return false;
    if (g.cols >= (int64_t(1) << 31) || g.rows >= (int64_t(1) << 31)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)code_row_bytes(g.cols, packed ? FA_CODES_NIBBLE : FA_CODES_BYTE),
                          (cuuint64_t)g.rows};
    cuuint64_t strides[1] = {(cuuint64_t)pc};
    cuuint32_t box[2] = {(cuuint32_t)S, (cuuint32_t)(g.th + 2)};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(codes), dims, strides,
               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

// Shared-memory limit and blocks per SM of k_walk<MODE, PASS, LOAD> for a tile
// shape (set once per kernel, occupancy queried once per shape).
template <int MODE, int PASS, int LOAD>
static cudaError_t walk_config(const Geom &g, int &blocks_per_sm) {
    static int configured = 0;
    static int per_sm = 0, per_sm_smem = -1, per_sm_nt = -1;
    const size_t smem = walk_smem_bytes(g.th, g.tw, MODE, PASS, LOAD);
    cudaError_t e = set_smem(k_walk<MODE, PASS, LOAD>, smem, configured);
    if (e != cudaSuccess) return e;
    const int nt = walk_threads(g.th, g.tw);
    if (per_sm_smem != (int)smem || per_sm_nt != nt) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<MODE, PASS, LOAD>, nt, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        per_sm_smem = (int)smem;
        per_sm_nt = nt;
    }
    blocks_per_sm = per_sm;
    return cudaSuccess;
}

template <int MODE, int PASS, int LOAD>
static cudaError_t launch_walk_k(const Geom &g, const TileArgs &ta, const CUtensorMap &m,
                                 cudaStream_t s) {
    int per_sm = 1;
    cudaError_t e = walk_config<MODE, PASS, LOAD>(g, per_sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ta.T, (int64_t)per_sm * sm_count());
    k_walk<MODE, PASS, LOAD><<<grid, walk_threads(g.th, g.tw),
                               walk_smem_bytes(g.th, g.tw, MODE, PASS, LOAD), s>>>(ta, m);
    return cudaGetLastError();
}

// Shared-memory limit and blocks per SM of k_addin<LOAD> (as walk_config).
template <int LOAD>
static cudaError_t addin_config(const Geom &g, int &blocks_per_sm) {
    static int configured = 0;
    static int per_sm = 0, per_sm_smem = -1;
    const size_t smem = addin_smem_bytes(g.th, g.tw, LOAD);
    cudaError_t e = set_smem(k_addin<LOAD>, smem, configured);
    if (e != cudaSuccess) return e;
    if (per_sm_smem != (int)smem) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_addin<LOAD>, ADDIN_THREADS, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        per_sm_smem = (int)smem;
    }
    blocks_per_sm = per_sm;
    return cudaSuccess;
}

template <int LOAD>
static cudaError_t launch_addin_k(const Geom &g, const TileArgs &ta, const CUtensorMap &m,
                                  cudaStream_t s) {
    int per_sm = 1;
    cudaError_t e = addin_config<LOAD>(g, per_sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ta.T, (int64_t)per_sm * sm_count());
    k_addin<LOAD><<<grid, ADDIN_THREADS, addin_smem_bytes(g.th, g.tw, LOAD), s>>>(ta, m);
    return cudaGetLastError();
}

template <int MODE, int PASS>
static cudaError_t launch_walk(const Geom &g, const TileArgs &ta, const uint8_t *codes,
                               int64_t pc, const uint8_t *mask, bool allow_tma, cudaStream_t s) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const bool packed = g.code_format == FA_CODES_NIBBLE;
    if (allow_tma && make_code_map(g, codes, pc, mask, packed, &m))
        return packed ? launch_walk_k<MODE, PASS, LOAD_TMA_PACKED>(g, ta, m, s)
                      : launch_walk_k<MODE, PASS, LOAD_TMA>(g, ta, m, s);
    return launch_walk_k<MODE, PASS, LOAD_PLAIN>(g, ta, m, s);
}

static cudaError_t launch_addin(const Geom &g, const TileArgs &ta, const uint8_t *codes, int64_t pc,
                                const uint8_t *mask, bool allow_tma, cudaStream_t s) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const bool packed = g.code_format == FA_CODES_NIBBLE;
    if (allow_tma && make_code_map(g, codes, pc, mask, packed, &m))
        return packed ? launch_addin_k<LOAD_TMA_PACKED>(g, ta, m, s)
                      : launch_addin_k<LOAD_TMA>(g, ta, m, s);
    return launch_addin_k<LOAD_PLAIN>(g, ta, m, s);
}

// Sets the kernels' shared-memory limits and caches their occupancy and the SM
// count ahead of a stream capture (done on first use otherwise).  Batches
// never stage codes by TMA.
cudaError_t prepare_forward(const Geom &g, int val_mode) {
    int per_sm = 1;
    cudaError_t e = val_mode ? walk_config<1, 1, LOAD_PLAIN>(g, per_sm)
                             : walk_config<0, 1, LOAD_PLAIN>(g, per_sm);
    if (e == cudaSuccess && val_mode) e = walk_config<1, 2, LOAD_PLAIN>(g, per_sm);
    if (e == cudaSuccess && !val_mode) e = addin_config<LOAD_PLAIN>(g, per_sm);
    sm_count();
    return e;
}

// Status reset, pass 1, the perimeter-graph resolve and pass 2 for the tiles
// described by `ta` (one raster, or a batch through ta.rtab).
static cudaError_t run_pipeline(const Geom &g, TileArgs ta, int val_mode, const FwdWork &ws,
                                void *status, const uint8_t *tma_codes, int64_t tma_pc,
                                const uint8_t *tma_mask, cudaStream_t s,
                                const PipeHooks *hooks = nullptr) {
    StatusBlock *st = reinterpret_cast<StatusBlock *>(status ? status : ws.status);
    k_init_status<<<1, 64, 0, s>>>(st, ws.misc, 2 + ws.kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ta.T == 0) return cudaSuccess;

    ta.th = g.th;
    ta.tw = g.tw;
    ta.pmax = g.pmax;
    ta.nib = g.code_format == FA_CODES_NIBBLE;
    ta.nf = val_mode ? std::max(1, g.nf) : 1;
    ta.nexit = ws.nexit;
    ta.link = ws.link;
    ta.node_dst = ws.node_dst;
    ta.node_val = ws.node_val;
    ta.G = ws.x;
    ta.st = st;
    ta.maxw = ws.misc;
    ta.infl = ws.infl;
    ta.off64 = hooks ? hooks->off64 : nullptr;
    ta.wait_ns = kWaitLimitNs;

    timing_mark(0, s);
    const bool tma = !(g.flags & FA_OPT_NO_TMA) && ta.rtab == nullptr;
    e = val_mode ? launch_walk<1, 1>(g, ta, tma_codes, tma_pc, tma_mask, tma, s)
                 : launch_walk<0, 1>(g, ta, tma_codes, tma_pc, tma_mask, tma, s);
    if (e != cudaSuccess) return e;
    timing_mark(1, s);

    ForestArgs f;
    f.tiles = ta.T;
    f.nodes = ta.T * g.pmax;
    f.pmax = g.pmax;
    f.nf = ta.nf;
    f.cells = ta.fcells;
    f.valm = val_mode;
    f.nexit = ws.nexit;
    f.link = ws.link;
    f.node_dst = ws.node_dst;
    f.node_val = ws.node_val;
    f.x = ws.x;
    f.J0 = ws.J0;
    f.J1 = ws.J1;
    f.misc = ws.misc;
    f.st = st;
    f.infl = val_mode ? nullptr : ws.infl;
    f.inj = (hooks && !val_mode) ? hooks->inj : nullptr;
    f.injx = (hooks && !val_mode) ? hooks->injx : nullptr;
    const unsigned fb = (unsigned)((f.tiles * 32 + 255) / 256);
    if (val_mode) {
        k_forest_init<u128><<<fb, 256, 0, s>>>(f);
        k_forest_indeg<u128><<<fb, 256, 0, s>>>(f);
        k_forest_leaves<u128><<<fb, 256, 0, s>>>(f);
        k_forest_walk<u128><<<fb, 256, 0, s>>>(f);
        k_forest_final<u128><<<fb, 256, 0, s>>>(f);
    } else {
        k_forest_init<unsigned long long><<<fb, 256, 0, s>>>(f);
        k_forest_indeg<unsigned long long><<<fb, 256, 0, s>>>(f);
        k_forest_leaves<unsigned long long><<<fb, 256, 0, s>>>(f);
        k_forest_walk<unsigned long long><<<fb, 256, 0, s>>>(f);
        k_forest_final<unsigned long long><<<fb, 256, 0, s>>>(f);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_mark(2, s);
    e = val_mode ? launch_walk<1, 2>(g, ta, tma_codes, tma_pc, tma_mask, tma, s)
                 : launch_addin(g, ta, tma_codes, tma_pc, tma_mask, tma, s);
    timing_mark(3, s);
    timing_set_count(3);
    return e;
}

cudaError_t resolve_exit_forest_u64(int64_t groups, int pmax, const uint32_t *nexit,
                                    const uint16_t *link, const uint32_t *node_dst,
                                    const double *node_val, unsigned long long *x,
                                    unsigned long long *infl, uint32_t *J0, uint32_t *J1,
                                    uint32_t *misc, void *status, cudaStream_t s) {
    if (groups == 0) return cudaSuccess;
    ForestArgs f;
    std::memset(&f, 0, sizeof(f));
    f.tiles = groups;
    f.nodes = groups * pmax;
    f.pmax = pmax;
    f.nf = 1;
    f.cells = 0;
    f.valm = 0;
    f.nexit = nexit;
    f.link = link;
    f.node_dst = node_dst;
    f.node_val = node_val;
    f.x = x;
    f.J0 = J0;
    f.J1 = J1;
    f.misc = misc;
    f.st = reinterpret_cast<StatusBlock *>(status);
    f.infl = infl;
    const unsigned fb = (unsigned)((groups * 32 + 255) / 256);
    k_forest_init<unsigned long long><<<fb, 256, 0, s>>>(f);
    k_forest_indeg<unsigned long long><<<fb, 256, 0, s>>>(f);
    k_forest_leaves<unsigned long long><<<fb, 256, 0, s>>>(f);
    k_forest_walk<unsigned long long><<<fb, 256, 0, s>>>(f);
    k_forest_final<unsigned long long><<<fb, 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_forward(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                           int64_t pm, const float *w, int64_t pw, void *out, int64_t po,
                           int val_mode, const FwdWork &ws, void *status, cudaStream_t s) {
    TileArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    RasterDesc &r = ta.one;
    r.codes = codes;
    r.pc = pc;
    r.mask = mask;
    r.pm = pm;
    r.w[0] = w;
    r.pw = pw;
    r.out[0] = out;
    r.po = po;
    r.rows = g.rows;
    r.cols = g.cols;
    r.tiles_x = g.tiles_x;
    r.tiles_y = g.tiles_y;
    r.tile_base = 0;
    ta.rtab = nullptr;
    ta.nr = 1;
    ta.T = (g.rows == 0 || g.cols == 0) ? 0 : g.tiles();
    ta.fcells = g.rows * g.cols;
    Geom g1 = g;
    g1.nf = 1;
    return run_pipeline(g1, ta, val_mode, ws, status, codes, pc, mask, s);
}

cudaError_t launch_forward_hooked(const Geom &g, const uint8_t *codes, int64_t pc, void *out,
                                  int64_t po, const FwdWork &ws, void *status, const PipeHooks &hooks,
                                  cudaStream_t s) {
    TileArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    RasterDesc &r = ta.one;
    r.codes = codes;
    r.pc = pc;
    r.out[0] = out;
    r.po = po;
    r.rows = g.rows;
    r.cols = g.cols;
    r.tiles_x = g.tiles_x;
    r.tiles_y = g.tiles_y;
    ta.nr = 1;
    ta.T = (g.rows == 0 || g.cols == 0) ? 0 : g.tiles();
    ta.fcells = g.rows * g.cols;
    Geom g1 = g;
    g1.nf = 1;
    return run_pipeline(g1, ta, 0, ws, status, codes, pc, nullptr, s, &hooks);
}

cudaError_t launch_forward_batched(const Geom &g, const RasterDesc *d_tab, int nr, int64_t T,
                                   int64_t cells_bound, int val_mode, const FwdWork &ws,
                                   void *status, cudaStream_t s) {
    TileArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.rtab = d_tab;
    ta.nr = nr;
    ta.T = T;
    ta.fcells = cells_bound;
    return run_pipeline(g, ta, val_mode, ws, status, nullptr, 0, nullptr, s);
}

}  // namespace fa
