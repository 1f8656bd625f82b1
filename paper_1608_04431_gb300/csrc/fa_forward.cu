// Forward D8 flow accumulation: tile passes and perimeter-graph resolve.
//
// Pipeline for one raster (Section 3 of the paper; the tile-local result is
// retained in the output raster between the passes):
//   pass 1  k_solve<V>      per tile: Algorithm 1 (dependency counts, then a
//                           queue-free Kahn loop) writing the tile-local
//                           accumulation A_loc into the output; Algorithm 2
//                           for the cells that receive flow from other tiles;
//                           emits A_loc at every exit cell and the target of
//                           its flow (the perimeter data of Section 3.2).
//   resolve k_forest_*      the global flow graph over exit cells
//                           (Section 3.2): G(e) = A_loc(e) + sum of G over the
//                           exits whose flow enters the tile at a cell linked
//                           to e, by pointer-jumping rounds.
//   pass 2  k_offsets<V>    per tile: the flow in(p) entering each perimeter
//                           cell p from other tiles is added to every cell on
//                           p's downstream path inside the tile (Algorithm 3,
//                           Section 3.3), read-modify-writing only those cells
//                           of the output.
// Inside a tile all sums are integers: uint32 counts, or 64-bit fixed point
// with a per-tile scale for float weights, so the order in which atomics land
// cannot change any bit of the result.
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
    int nib;  // codes packed two per byte (FA_CODES_NIBBLE)
    uint32_t *nexit;
    uint16_t *link;
    uint32_t *node_dst;
    double *node_val;
    const void *G;  // resolved perimeter graph: u64 counts or u128 fixed-point sums
    StatusBlock *st;
    uint32_t *maxw;
    uint32_t *ef_hdr, *ef_cp, *seg_merge, *inf_src;
    uint16_t *ef_seg, *inf_seg;
    // batches: a table of rasters (nullptr for one raster), each with its
    // tiles numbered from its tile_base in one global tile sequence
    const RasterDesc *rtab;
    int nr;
    int64_t T;            // tiles in all
    int64_t fcells;       // cell bound of the perimeter-graph fixed-point scale
};

// Points the raster fields of `a` at the raster owning global tile t.
__device__ __forceinline__ RasterDesc raster_of(const TileArgs &a, int64_t t) {
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

// per-tile 64-bit scale: |sum| <= bound < 2^(62 - q)
__device__ __forceinline__ int tile_scale(double bound) {
    if (!(bound > 0.0) || !(bound < 1e300)) return 0;
    int e;
    frexp(bound, &e);
    return 62 - e;
}

__device__ __forceinline__ long long f2fix64(float x, int q) { return (long long)ldexp((double)x, q); }

// ---------------------------------------------------------------------------
// Shared-memory layout of a tile.  Codes and every per-cell array share one
// byte-index space: halo row hr (0 .. h+1, tile row r = hr - 1) starts at
// hr * S; tile column c sits at byte c + X0 (halo columns at bytes X0 - 1 and
// X0 + w).  Each group of 4 interior cells is one aligned 32-bit word, so the
// in-degree is computed four cells at a time, and a row is exactly the TMA box
// that starts X0 bytes left of the tile (a 16-byte aligned column when the
// tile width is a multiple of 16).  S >= X0 + tw + 16.
// ---------------------------------------------------------------------------
constexpr int X0 = 16;
__host__ __device__ inline int tile_stride(int tw) { return ((tw + 32 + 15) / 16) * 16; }

// bytes of one staged code tile, rounded so a second stage stays 128-aligned
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

// How pass 1 gets its codes: plain loads, TMA-staged bytes, or TMA-staged
// packed codes spread to bytes in shared memory.
enum { LOAD_PLAIN = 0, LOAD_TMA = 1, LOAD_TMA_PACKED = 2 };

// Row stride of the compact per-cell arrays (word, sums, claim tags): a
// multiple of four so that a four-cell group is one 16-byte store.
__host__ __device__ inline int cell_stride(int tw) { return (tw + 3) & ~3; }

// Four-cell groups of the compact arrays owned by one jump thread (their
// pointers live in registers during the rounds).
constexpr int KG = 4;
// Threads of a tile-solve block: one per KG groups of the compact arrays
// (th x cell_stride(tw) cells <= 16384), at least a warp, at most 1024.  All
// of them run the jump rounds, then walk the entry paths.
__host__ __device__ inline int jump_threads(int th, int tw) {
    const int ng = th * cell_stride(tw) / 4;
    const int need = (ng + KG - 1) / KG;
    return min(1024, max(32, ((need + 31) / 32) * 32));
}
__host__ __device__ inline int solve_threads(int th, int tw) { return jump_threads(th, tw); }

__host__ __device__ inline size_t solve_smem_bytes(int th, int tw, int valm, int load) {
    const size_t nc = (size_t)th * cell_stride(tw), pm = (size_t)(2 * th + 2 * tw);
    size_t b = 128;                           // alignment slack of the dynamic window
    // codes: one buffer; two TMA stages; or two packed stages and one buffer
    b += load == LOAD_TMA_PACKED ? 2 * packed_buf_bytes(th, tw) + code_buf_bytes(th, tw)
                                 : code_buf_bytes(th, tw) * (load == LOAD_TMA ? 2 : 1);
    b += nc * (valm ? 16 : 4);                // value and round inflow per cell
    b += nc * 2;                              // successor (jump pointer) per cell
    b += pm * 4;                              // segment -> where it joins another
    b += pm * 2 * 4;                          // exit rank per slot, entry list, segment ends, entry number
    b += (pm + 8) * 2;                        // inflow link -> slot
    return (b + 15) & ~size_t(15);
}

__host__ __device__ inline size_t offsets_smem_bytes(int th, int tw) {
    // segments: at most one per perimeter cell
    const size_t pc = (size_t)perim_count(th, tw);
    size_t b = pc * 16;                       // inflow per segment (graph scale), then prefix sums
    b += pc * 8 * 2;                          // inflow at the tile scale, flow at the end
    b += pc * 4 * 2 + (pc + 1) * 4;           // join target, pending joins / fill, bucket start
    b += pc * 2 * 2;                          // join position, joins grouped by target
    return (b + 15) & ~size_t(15);
}

__host__ __device__ inline bool tile_shape_ok(int th, int tw, int valm) {
    return (int64_t)(th + 2) * tile_stride(tw) <= 65535 && (int64_t)th * tw <= 16384 &&
           (int64_t)th * cell_stride(tw) <= 16384 &&
           solve_smem_bytes(th, tw, valm, LOAD_PLAIN) <= 227 * 1024 &&
           offsets_smem_bytes(th, tw) <= 227 * 1024;
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


// ---------------------------------------------------------------------------
// pass 1: tile solve
// ---------------------------------------------------------------------------
// Persistent CTAs: each block solves tiles t = blockIdx.x, + gridDim.x, ...
// With TMA the codes of tile t + gridDim.x (box of S x (th+2) bytes at column
// C0 - X0, row R0 - 1; outside the raster reads as 0 = NoData) are staged into
// the other shared buffer while tile t is solved.  Packed codes are staged the
// same way (half as many bytes) and spread to one byte per cell when their
// tile begins.
//
// Besides A_loc and the perimeter records (Algorithms 1 and 2) a tile records
// its entry forest for pass 2: the cells on the in-tile paths downstream of
// its entry cells.  The path of every entry is walked once, claiming cells as
// it goes; a walk that reaches a cell already claimed by another entry's walk
// stops there and records the join.  Each walk's claimed run is a segment:
// the cells of segment e at positions 0, 1, ... in path order.
constexpr uint32_t NO_JOIN = 0xFFFFFFFFu;
constexpr uint16_t NO_ENTRY = 0xFFFFu;

// A block of solve_threads(tile) threads (up to 1024), each owning at most KG
// four-cell groups of the compact arrays during the jump rounds.
template <int VALM, int TMA>
__global__ void __launch_bounds__(1024) k_solve(TileArgs A, const __grid_constant__ CUtensorMap tmap) {
    typedef typename std::conditional<VALM == 0, uint32_t, long long>::type PV;
    const TileArgs &a = A;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_warp[33];
    __shared__ int s_nent, s_flags, s_nef, s_ninf;
    __shared__ uint32_t s_maxw;
    __shared__ __align__(8) uint64_t s_bar[2];

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int S = tile_stride(a.tw);
    const int NB = (a.th + 2) * S;
    const int WS = cell_stride(a.tw);  // compact arrays: cell (r, c) at r * WS + c
    const int NC = a.th * WS;
    const int64_t T = a.T;

    // shared layout: code buffers (two TMA stages, each 128-byte aligned for
    // the bulk copies; packed: two packed stages and the spread buffer), then
    // the per-cell arrays
    const size_t CB = code_buf_bytes(a.th, a.tw);
    const size_t STG = TMA == LOAD_TMA_PACKED ? packed_buf_bytes(a.th, a.tw) : CB;
    const int PB = packed_box_bytes(a.tw);
    uint8_t *base128 = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem) + 127) &
                                                   ~uintptr_t(127));
    uint8_t *cbuf0 = base128;
    uint8_t *cbuf1 = base128 + (TMA ? STG : 0);
    uint8_t *spread = base128 + 2 * STG;  // packed: the codes of the current tile, one byte each
    uint8_t *cells = base128 + (TMA == LOAD_TMA_PACKED ? 2 * STG + CB : (TMA ? 2 : 1) * CB);
    // counts: per cell its value x (low 16 bits) and the inflow of the current
    // jump round (high 16 bits); weights: 64-bit fixed-point x and inflow
    uint32_t *xd = reinterpret_cast<uint32_t *>(cells);
    long long *x64 = reinterpret_cast<long long *>(cells);
    long long *d64 = x64 + NC;
    uint16_t *J = reinterpret_cast<uint16_t *>(cells + (VALM ? 16 : 4) * (size_t)NC);
    uint32_t *tagw = xd;  // after the rounds: claiming segment + 1 << 16 | position, 0 = free
    uint32_t *segjoin = reinterpret_cast<uint32_t *>(J + NC);
    uint16_t *rank = reinterpret_cast<uint16_t *>(segjoin + a.pmax);
    uint16_t *entq = rank + a.pmax;
    uint16_t *segend = entq + a.pmax;
    uint16_t *eidx = segend + a.pmax;     // slot -> entry number, NO_ENTRY if not an entry
    uint16_t *lslot = eidx + a.pmax;      // inflow link -> the slot it feeds

    // status, accumulated over this block's tiles
    int nbad = 0, ncyc = 0, nonfinite = 0;
    long long fbad = NO_INDEX;
    uint32_t gmaxw = 0;

    if (tid == 0) {
        s_flags = 0;
        if (TMA) {
            mbar_init(&s_bar[0], 1);
            mbar_init(&s_bar[1], 1);
            mbar_fence_init();
        }
    }
    __syncthreads();
    auto issue = [&](int tn, int bb) {  // one thread: stage tile tn's codes into buffer bb
        const int tyn = tn / A.one.tiles_x, txn = tn - tyn * A.one.tiles_x;  // TMA: one raster only
        if constexpr (TMA == LOAD_TMA_PACKED) {  // x in bytes: (C0 - PX0) / 2, a multiple of 16
            mbar_expect_tx(&s_bar[bb], (uint32_t)((a.th + 2) * PB));
            tma_load_2d(bb ? cbuf1 : cbuf0, &tmap, (txn * a.tw - PX0) / 2, tyn * a.th - 1, &s_bar[bb]);
        } else {
            mbar_expect_tx(&s_bar[bb], (uint32_t)NB);
            tma_load_2d(bb ? cbuf1 : cbuf0, &tmap, txn * a.tw - X0, tyn * a.th - 1, &s_bar[bb]);
        }
    };
    if (TMA && tid == 0 && blockIdx.x < T) issue(blockIdx.x, 0);

    int it = 0, to_it = -1;
    for (int t = blockIdx.x; t < T; t += gridDim.x, ++it) {
        const RasterDesc ras = raster_of(a, t);
        const int lt = (int)(t - ras.tile_base);
        const int ty = lt / ras.tiles_x, tx = lt - ty * ras.tiles_x;
        const int64_t R0 = (int64_t)ty * a.th, C0 = (int64_t)tx * a.tw;
        const int h = (int)min((int64_t)a.th, ras.rows - R0);
        const int w = (int)min((int64_t)a.tw, ras.cols - C0);
        const int n_in = h * w;
        const int P = perim_count(h, w);
        const size_t tbase = (size_t)t * a.pmax;
        const size_t efb = (size_t)t * a.th * a.tw, infb = (size_t)t * (a.pmax + 8);
        uint8_t *ec = TMA == LOAD_TMA_PACKED ? spread : ((TMA && (it & 1)) ? cbuf1 : cbuf0);
        if (tid == 0) {
            s_nent = 0;
            s_maxw = 0;
            s_nef = 0;
            s_ninf = 0;
        }
        for (int q = tid; q < a.pmax; q += nt) eidx[q] = NO_ENTRY;

        // [phase] load
        if constexpr (TMA) {
            const int64_t tn = t + gridDim.x;
            if (tid == 0) {  // one thread waits for the stage; the barrier publishes it
                if (tn < T) issue((int)tn, (it & 1) ^ 1);
                if (!mbar_wait(&s_bar[it & 1], (uint32_t)((it >> 1) & 1))) s_flags |= FA_FLAG_TIMEOUT;
            }
            __syncthreads();
            if (s_flags & FA_FLAG_TIMEOUT) {
                to_it = (t + (int64_t)gridDim.x < T) ? -2 - it : it;  // -2-it: the next stage was issued too
                break;
            }
            // the staged box holds raw codes: readers take bytes 1..9 as
            // valid and tell the halo ring by coordinates; invalid codes of
            // the tile are counted in the init pass
            if constexpr (TMA == LOAD_TMA_PACKED) {
                // spread the packed box to one byte per cell: code-buffer word
                // wd (cells C0 - X0 + 4wd ..) is box bytes 2wd + 8 and 2wd + 9.
                // Cells right of the raster are NoData, the spare high nibble
                // of an odd-width row included (left of it and above or below
                // it the box already reads 0).
                const uint8_t *stg = (it & 1) ? cbuf1 : cbuf0;
                const int W4 = S >> 2;
                for (int i = tid; i < (a.th + 2) * W4; i += nt) {
                    const int hr = i / W4, wd = i - hr * W4;
                    uint32_t v = spread_nibbles(*reinterpret_cast<const uint16_t *>(stg + hr * PB + 2 * wd + 8));
                    const int64_t keep = ras.cols - (C0 - X0 + 4 * wd);  // cells of the word inside
                    if (keep < 4) v = keep <= 0 ? 0u : (v & ((1u << (8 * keep)) - 1u));
                    reinterpret_cast<uint32_t *>(spread + hr * S)[wd] = v;
                }
            }
        } else {
            load_codes(ras, ec, R0, C0, h, w, S, a.nib != 0, true, nbad, fbad);
        }
        __syncthreads();

        // [phase] init
        // ---- the in-tile successor of every cell (Algorithm 1's D, as the
        // jump pointer J_0), four cells per lane from the same neighbour
        // words: byte j of nbr_k is the code of cell j's neighbour in
        // direction k.  A row of g groups uses the next power of two >= g
        // lanes, so one warp iteration covers 32 / lanes-per-row rows.  Cells
        // outside the tile (edge tiles) get no successor and value 0.
        uint32_t maxw = 0;
        const int groups = (w + 3) >> 2;  // groups holding tile cells
        const int gall = WS >> 2;         // groups per row of the compact arrays
        int lpr_log = 0;
        while ((1 << lpr_log) < gall && lpr_log < 5) ++lpr_log;
        const int rows_per_it = 32 >> lpr_log;
        const int sub = lane >> lpr_log, gl = lane & ((1 << lpr_log) - 1);
        for (int r0 = warp * rows_per_it; r0 < a.th; r0 += nw * rows_per_it) {
            for (int g0 = 0; g0 < gall; g0 += (1 << lpr_log)) {
                const int r = r0 + sub, gq = g0 + gl;
                if (r >= a.th || gq >= gall) continue;
                const int c = 4 * gq, wbase = r * WS + c;
                uint32_t jw0 = 0xFFFFFFFFu, jw1 = 0xFFFFFFFFu, valid = 0;
                uint32_t wbits[4] = {0u, 0u, 0u, 0u};  // raw weight bits (weights)
                if (r < h && gq < groups) {
                    const int base = (r + 1) * S + c + X0;
                    // each cell's code names its successor; it counts when the
                    // target is a valid cell of the tile (not the halo ring)
                    const uint32_t me = *reinterpret_cast<const uint32_t *>(ec + base);
                    const int nvalid = min(4, w - c);
                    const uint32_t colmask = nvalid >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nvalid)) - 1u);
                    valid = __vcmpgeu4(me, 0x01010101u) & __vcmpleu4(me, 0x09090909u) & colmask;
                    if constexpr (TMA) {  // raw codes: count the invalid ones of the tile
                        const uint32_t bad = __vcmpgtu4(me, 0x09090909u) & colmask;
                        if (bad) {
                            nbad += __popc(bad) >> 3;
                            fbad = min(fbad, (long long)((R0 + r) * ras.cols + (C0 + c + ((__ffs(bad) - 1) >> 3))));
                        }
                    }
                    uint32_t sc[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = (int)((me >> (8 * q)) & 0xFFu);
                        sc[q] = 0xFFFFu;  // no successor in the tile
                        if (q < nvalid && k >= 1 && k <= 8) {
                            const int tr = r + dir_dr(k), tc = c + q + dir_dc(k);
                            if (tr >= 0 && tr < h && tc >= 0 && tc < w && vcode(ec[base + q + off_of(k, S)]))
                                sc[q] = (uint32_t)(wbase + q + dir_dr(k) * WS + dir_dc(k));
                        }
                    }
                    jw0 = sc[0] | (sc[1] << 16);
                    jw1 = sc[2] | (sc[3] << 16);
                    if constexpr (VALM == 1) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (!((valid >> (8 * q)) & 1u)) continue;
                            const float wf = ras.w ? ras.w[(R0 + r) * ras.pw + (C0 + c + q)] : 1.0f;
                            wbits[q] = __float_as_uint(wf);
                            const uint32_t b = wbits[q] & 0x7fffffffu;
                            if (b >= 0x7f800000u) nonfinite = 1;
                            maxw = max(maxw, b);
                        }
                    }
                }
                *reinterpret_cast<uint2 *>(J + wbase) = make_uint2(jw0, jw1);
                if constexpr (VALM == 0) {
                    *reinterpret_cast<uint4 *>(xd + wbase) =
                        make_uint4(valid & 1u, (valid >> 8) & 1u, (valid >> 16) & 1u, valid >> 24 & 1u);
                } else {
                    // raw weight bits until the tile's scale is known
                    *reinterpret_cast<longlong2 *>(x64 + wbase) = make_longlong2(wbits[0], wbits[1]);
                    *reinterpret_cast<longlong2 *>(x64 + wbase + 2) = make_longlong2(wbits[2], wbits[3]);
                    *reinterpret_cast<longlong2 *>(d64 + wbase) = make_longlong2(0, 0);
                    *reinterpret_cast<longlong2 *>(d64 + wbase + 2) = make_longlong2(0, 0);
                }
            }
        }

        // ---- inflow links: every valid cell of the halo ring draining into the
        // tile (an exit of its own tile) feeds a perimeter cell, which is then
        // an entry cell.  Ring positions: the row above (w + 2 cells, west to
        // east), the row below, then the columns west and east of the tile.
        const int ring = 2 * (h + w) + 4;
        for (int q = tid; q < ring; q += nt) {
            int rr, cc;
            if (q < w + 2) {
                rr = -1;
                cc = q - 1;
            } else if (q < 2 * w + 4) {
                rr = h;
                cc = q - (w + 2) - 1;
            } else if (q < 2 * w + 4 + h) {
                rr = q - (2 * w + 4);
                cc = -1;
            } else {
                rr = q - (2 * w + 4 + h);
                cc = w;
            }
            const int k = ec[(rr + 1) * S + cc + X0];
            if (k < 1 || k > 8) continue;  // NoData, off the raster, NoFlow, invalid
            const int tr = rr + dir_dr(k), tc = cc + dir_dc(k);
            if (tr < 0 || tr >= h || tc < 0 || tc >= w) continue;  // drains elsewhere
            if (!vcode(ec[(tr + 1) * S + tc + X0])) continue;      // into NoData
            const int st = slot_of(tr, tc, h, w);
            eidx[st] = 0;  // an entry cell
            const int tyh = ty + (rr < 0 ? -1 : (rr >= h ? 1 : 0));
            const int txh = tx + (cc < 0 ? -1 : (cc >= w ? 1 : 0));
            const int64_t R0h = (int64_t)tyh * a.th, C0h = (int64_t)txh * a.tw;
            const int hh = (int)min((int64_t)a.th, ras.rows - R0h);
            const int wh = (int)min((int64_t)a.tw, ras.cols - C0h);
            const int sh = slot_of((int)(R0 + rr - R0h), (int)(C0 + cc - C0h), hh, wh);
            const int jl = atomicAdd(&s_ninf, 1);
            a.inf_src[infb + jl] =
                (uint32_t)(((size_t)ras.tile_base + (size_t)tyh * ras.tiles_x + txh) * a.pmax + sh);
            lslot[jl] = (uint16_t)st;
        }

        // ---- exit cells (flow leaves the tile into a valid cell) get ranks in
        // slot order; entry cells are numbered (one entry-forest segment each)
        const int chunk = (P + nt - 1) / nt;
        const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
        int mine = 0;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * S + c + X0;
            const int k = ec[i];
            if (k >= 1 && k <= 8 && vcode(ec[i + off_of(k, S)])) {
                const int tr = r + dir_dr(k), tc = c + dir_dc(k);
                if (tr < 0 || tr >= h || tc < 0 || tc >= w) ++mine;  // a valid cell outside
            }
        }
        int total;
        int rk = block_exclusive_scan(mine, s_warp, &total);  // (its barriers publish eidx)
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * S + c + X0;
            const int k = ec[i];
            const int trx = r + dir_dr(k), tcx = c + dir_dc(k);
            const bool ex = k >= 1 && k <= 8 && (trx < 0 || trx >= h || tcx < 0 || tcx >= w) &&
                            vcode(ec[i + off_of(k, S)]);
            rank[s] = ex ? (uint16_t)rk : LINK_TERM;
            if (ex) {
                // where the exit's flow goes: a perimeter slot of a neighbouring tile
                const int rr = r + dir_dr(k), cc = c + dir_dc(k);  // tile-local, one step outside
                const int tyd = ty + (rr < 0 ? -1 : (rr >= h ? 1 : 0));
                const int txd = tx + (cc < 0 ? -1 : (cc >= w ? 1 : 0));
                const int64_t R0d = (int64_t)tyd * a.th, C0d = (int64_t)txd * a.tw;
                const int hd = (int)min((int64_t)a.th, ras.rows - R0d);
                const int wd = (int)min((int64_t)a.tw, ras.cols - C0d);
                const int sd = slot_of((int)(R0 + rr - R0d), (int)(C0 + cc - C0d), hd, wd);
                a.node_dst[tbase + rk] =
                    (uint32_t)(((size_t)ras.tile_base + (size_t)tyd * ras.tiles_x + txd) * a.pmax + sd);
                a.link[tbase + s] = (uint16_t)rk;  // an exit links to itself
                ++rk;
            }
            if (eidx[s] != NO_ENTRY) {
                const int e = atomicAdd(&s_nent, 1);
                entq[e] = (uint16_t)s;
                eidx[s] = (uint16_t)e;
            } else if (!ex) {
                a.link[tbase + s] = LINK_TERM;
            }
        }
        int qt = 0;
        if constexpr (VALM == 1) {
            gmaxw = max(gmaxw, maxw);
            maxw = warp_max_u(maxw);
            if (lane == 0 && maxw) atomicMax(&s_maxw, maxw);
            __syncthreads();
            qt = (s_maxw >= 0x7f800000u) ? 0
                                         : tile_scale((double)n_in * (double)__uint_as_float(s_maxw));
            for (int r = warp; r < h; r += nw)
                for (int c = lane; c < w; c += 32) {
                    const int i = (r + 1) * S + c + X0;
                    if (ec[i]) x64[r * WS + c] = f2fix64(__uint_as_float((uint32_t)x64[r * WS + c]), qt);
                }
        }
        __syncthreads();

        // [phase] walk
        // ---- A_loc by pointer jumping on the tile's flow forest (Eq. 1 with
        // the tile as the whole raster).  In round k every cell u adds its
        // value to J_k(u), the cell 2^k steps downstream (while the in-tile
        // path is that long), and J_{k+1}(u) = J_k(J_k(u)).  After rounds
        // 0..m-1 a cell holds the sum over the cells at most 2^m - 1 steps
        // upstream of it, which is A_loc once 2^m exceeds the longest path.
        // A round scatters into the inflow half (counts) or array (weights)
        // and gathers J_k o J_k; after a barrier every cell folds its inflow
        // into its value and publishes its new pointer.  Each thread keeps
        // the pointers of its four-cell groups in registers.  Integer sums:
        // the result does not depend on the order of the atomic adds.
        const int NG = NC >> 2;
        const int njt = jump_threads(a.th, a.tw);
        const bool sep = nt > njt;
        if (tid < njt) {
            uint2 jg[KG];
#pragma unroll
            for (int i = 0; i < KG; ++i) {
                const int g = tid + i * njt;
                jg[i] = g < NG ? *reinterpret_cast<const uint2 *>(J + 4 * g)
                               : make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
            }
            for (int round = 0; round < 16; ++round) {  // 2^15 > any in-tile path
                uint2 jn[KG];
#pragma unroll
                for (int i = 0; i < KG; ++i) {
                    jn[i] = jg[i];
                    const int g = tid + i * njt;
                    if (g >= NG || (jg[i].x & jg[i].y) == 0xFFFFFFFFu) continue;  // no pointer left
                    const uint32_t jv[4] = {jg[i].x & 0xFFFFu, jg[i].x >> 16, jg[i].y & 0xFFFFu,
                                            jg[i].y >> 16};
                    uint32_t jj[4];
                    if constexpr (VALM == 0) {
                        const uint4 x4 = *reinterpret_cast<const uint4 *>(xd + 4 * g);
                        const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            jj[q] = 0xFFFFu;
                            if (jv[q] != 0xFFFFu) {
                                jj[q] = J[jv[q]];
                                atomicAdd(&xd[jv[q]], xs[q] << 16);  // into the inflow half
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            jj[q] = 0xFFFFu;
                            if (jv[q] != 0xFFFFu) {
                                jj[q] = J[jv[q]];
                                atomicAdd(reinterpret_cast<unsigned long long *>(&d64[jv[q]]),
                                          (unsigned long long)x64[4 * g + q]);
                            }
                        }
                    }
                    jn[i] = make_uint2(jj[0] | (jj[1] << 16), jj[2] | (jj[3] << 16));
                }
                bar_sync_n(1, njt);
                int act = 0;
#pragma unroll
                for (int i = 0; i < KG; ++i) {
                    const int g = tid + i * njt;
                    if (g >= NG) continue;
                    if (jn[i].x != jg[i].x || jn[i].y != jg[i].y) {
                        *reinterpret_cast<uint2 *>(J + 4 * g) = jn[i];
                        jg[i] = jn[i];
                    }
                    act |= (jg[i].x & jg[i].y) != 0xFFFFFFFFu;
                    if constexpr (VALM == 0) {
                        uint4 v = *reinterpret_cast<const uint4 *>(xd + 4 * g);
                        if ((v.x | v.y | v.z | v.w) >> 16) {
                            v.x = (v.x & 0xFFFFu) + (v.x >> 16);
                            v.y = (v.y & 0xFFFFu) + (v.y >> 16);
                            v.z = (v.z & 0xFFFFu) + (v.z >> 16);
                            v.w = (v.w & 0xFFFFu) + (v.w >> 16);
                            *reinterpret_cast<uint4 *>(xd + 4 * g) = v;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const long long dv = d64[4 * g + q];
                            if (dv) {
                                x64[4 * g + q] += dv;
                                d64[4 * g + q] = 0;
                            }
                        }
                    }
                }
                if (!bar_or_n(1, njt, act)) break;
            }
            // cells whose path never ended lie on a cycle inside the tile or drain
            // into one
#pragma unroll
            for (int i = 0; i < KG; ++i) {
                const int g = tid + i * njt;
                if (g >= NG || (jg[i].x & jg[i].y) == 0xFFFFFFFFu) continue;
                const uint32_t jv[4] = {jg[i].x & 0xFFFFu, jg[i].x >> 16, jg[i].y & 0xFFFFu, jg[i].y >> 16};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (jv[q] == 0xFFFFu) continue;
                    ++ncyc;
                    const int ci = 4 * g + q, rr = ci / WS, cc = ci - rr * WS;
                    fbad = min(fbad, (long long)((R0 + rr) * ras.cols + (C0 + cc)));
                }
            }

        }  // jump threads

        // [phase] output
        // ---- write A_loc (0 for NoData; unspecified on cycles) and the exit
        // records; the value array then holds the entry walks' claim tags ---
        const double inv = ldexp(1.0, -qt);
        // four cells per lane, as in the init loop; whole 16-byte stores when
        // the output row allows them
        const bool vec = ((reinterpret_cast<uintptr_t>(ras.out) |
                           ((uintptr_t)ras.po << 2) | ((uintptr_t)C0 << 2)) & 15) == 0;
        for (int r0 = warp * rows_per_it; r0 < h; r0 += nw * rows_per_it) {
            for (int g0 = 0; g0 < groups; g0 += (1 << lpr_log)) {
                const int r = r0 + sub, gq = g0 + gl;
                if (r >= h || gq >= groups) continue;
                const int c = 4 * gq, wb = r * WS + c;
                const int nvalid = min(4, w - c);
                const uint32_t codes4 = *reinterpret_cast<const uint32_t *>(ec + (r + 1) * S + c + X0);
                uint32_t ov[4];
                if constexpr (VALM == 0) {
                    const uint4 x4 = *reinterpret_cast<const uint4 *>(xd + wb);
                    const uint32_t xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) ov[jj] = xs[jj] & 0xFFFFu;  // NoData holds 0
                } else {
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const bool valid = jj < nvalid && vcode((codes4 >> (8 * jj)) & 0xFFu);
                        ov[jj] = valid ? __float_as_uint((float)((double)x64[wb + jj] * inv)) : 0u;
                    }
                }
                uint32_t *orow = reinterpret_cast<uint32_t *>(ras.out) + (size_t)(R0 + r) * ras.po + C0 + c;
                if (vec && nvalid == 4) {
                    *reinterpret_cast<uint4 *>(orow) = make_uint4(ov[0], ov[1], ov[2], ov[3]);
                } else {
                    for (int jj = 0; jj < nvalid; ++jj) orow[jj] = ov[jj];
                }
            }
        }
        for (int s = tid; s < P; s += nt) {
            const uint16_t rks = rank[s];
            if (rks == LINK_TERM) continue;
            int r, c;
            cell_of(s, h, w, r, c);
            double vv;
            if constexpr (VALM == 0) vv = (double)(xd[r * WS + c] & 0xFFFFu);
            else vv = (double)x64[r * WS + c] * inv;
            a.node_val[tbase + rks] = vv;  // A_loc at the exit (the perimeter data's A)
        }
        __syncthreads();
        for (int q = tid; q < NC; q += nt) tagw[q] = 0u;
        __syncthreads();

        // ---- Algorithm 2 for the entry cells, one segment per entry: claim
        // cells along the path until it leaves the tile, ends, or reaches a
        // cell another segment claimed (the extra warp, during the rounds)
        if (!sep || tid >= njt) {
            const int nent = s_nent;
            uint32_t *efc = a.ef_cp + efb;
            uint16_t *efs = a.ef_seg + efb;
            const int q0 = sep ? tid - njt : tid, qs = sep ? nt - njt : nt;
            for (int q = q0; q < nent; q += qs) {
                int r, c;
                cell_of(entq[q], h, w, r, c);
                int pi = (r + 1) * S + c + X0, ci = r * WS + c;
                uint16_t end = LINK_TERM;
                uint32_t join = NO_JOIN;
                int k = ec[pi];  // this cell's code, carried from step to step
                for (int pos = 0; pos < n_in; ++pos) {
                    // the next cell and its code are read while the claim is in flight
                    const bool dir = k >= 1 && k <= 8;
                    const int np = dir ? pi + off_of(k, S) : pi;
                    const int kn = ec[np];
                    const uint32_t old =
                        atomicCAS(&tagw[ci], 0u, ((uint32_t)(q + 1) << 16) | (uint32_t)pos);
                    if (old != 0) {  // joins segment (old >> 16) - 1 at its position old & 0xFFFF
                        join = old - (1u << 16);
                        break;
                    }
                    const int idx = atomicAdd(&s_nef, 1);
                    efc[idx] = ((uint32_t)ci << 16) | (uint32_t)pos;
                    efs[idx] = (uint16_t)q;
                    if (!dir) break;         // NoFlow: the path ends here
                    if (!vcode(kn)) break;   // into NoData or off the raster
                    const int tr = r + dir_dr(k), tc = c + dir_dc(k);
                    if (tr < 0 || tr >= h || tc < 0 || tc >= w) {  // leaves the tile: an exit
                        end = rank[slot_of(r, c, h, w)];
                        break;
                    }
                    pi = np;
                    ci += dir_dr(k) * WS + dir_dc(k);
                    r = tr;
                    c = tc;
                    k = kn;
                }
                segend[q] = end;
                segjoin[q] = join;
            }
        }
        __syncthreads();

        // ---- links of the entry cells; the entry forest's segment joins
        const int nent = s_nent;
        for (int j = tid; j < s_ninf; j += nt) a.inf_seg[infb + j] = eidx[lslot[j]];
        for (int e = tid; e < nent; e += nt) {
            a.seg_merge[tbase + e] = segjoin[e];
            const int s = entq[e];
            if (rank[s] != LINK_TERM) continue;  // an exit links to itself
            int x = e;
            for (int hop = 0; hop < nent && segjoin[x] != NO_JOIN; ++hop) x = (int)(segjoin[x] >> 16);
            a.link[tbase + s] = segjoin[x] == NO_JOIN ? segend[x] : LINK_TERM;
        }
        if (tid == 0) {
            a.nexit[t] = (uint32_t)total;
            reinterpret_cast<uint4 *>(a.ef_hdr)[t] =
                make_uint4((uint32_t)s_nef, (uint32_t)nent, (uint32_t)s_ninf, 0u);
        }
        if constexpr (TMA) fence_proxy_async();  // this buffer is refilled by TMA later
        __syncthreads();
        // [phase] end
    }

    // ---- status -------------------------------------------------------------
    __shared__ int s_cnt_bad, s_cnt_cyc;
    __shared__ long long s_first;
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
    if (lane == 0) {
        if (nbad) atomicAdd(&s_cnt_bad, nbad);
        if (ncyc) atomicAdd(&s_cnt_cyc, ncyc);
        if (fbad != NO_INDEX) atomicMin(&s_first, fbad);
        if (gmaxw) atomicMax(&s_maxw, gmaxw);
        if (nonfinite) atomicOr(&s_flags, FA_FLAG_NONFINITE);
    }
    __syncthreads();
    if (tid == 0) {
        int fl = s_flags;
        if (s_cnt_bad) fl |= FA_FLAG_BAD_CODE;
        if (s_cnt_cyc) fl |= FA_FLAG_CYCLE;
        if (fl) status_report(a.st, fl, s_cnt_bad + s_cnt_cyc, s_first);
        if (s_maxw) atomicMax(a.maxw, s_maxw);
    }
    if constexpr (TMA) {
        // a timed-out wait may leave copies in flight into this block's
        // shared memory: wait again (bounded) for the stages still pending
        if (to_it != -1 && tid == 0) {
            const int i0 = to_it >= 0 ? to_it : -2 - to_it;
            mbar_wait(&s_bar[i0 & 1], (uint32_t)((i0 >> 1) & 1));
            if (to_it < -1) mbar_wait(&s_bar[(i0 + 1) & 1], (uint32_t)(((i0 + 1) >> 1) & 1));
        }
    }
}

// ---------------------------------------------------------------------------
// pass 2: add the flow entering each tile to the cells downstream of its entry
// cells.  in(e), the flow arriving at entry e from outside, follows e's path:
// every cell of segment e gets in(e), and from the cell where segment q joins
// segment e onwards every cell also gets F(q), the flow at the end of q
// (in(q) plus the F of every segment joining q).  So the offset of the cell at
// position j of segment e is in(e) + sum of F(q) over the segments q joining e
// at positions <= j.  Codes are not needed: pass 1 recorded the segments.
// ---------------------------------------------------------------------------
template <int VALM>
__global__ void __launch_bounds__(128) k_offsets(TileArgs A) {
    typedef typename std::conditional<VALM == 0, unsigned long long, long long>::type OV;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_emax;
    const TileArgs &a = A;
    const int64_t t = blockIdx.x;
    const uint4 hd = reinterpret_cast<const uint4 *>(a.ef_hdr)[t];
    const int nef = (int)hd.x, nseg = (int)hd.y, ninf = (int)hd.z;
    if (nseg == 0 || nef == 0) return;  // no flow enters this tile
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const RasterDesc ras = raster_of(a, t);
    const int lt = (int)(t - ras.tile_base);
    const int ty = lt / ras.tiles_x, tx = lt - ty * ras.tiles_x;
    const int64_t R0 = (int64_t)ty * a.th, C0 = (int64_t)tx * a.tw;
    const int h = (int)min((int64_t)a.th, ras.rows - R0);
    const int w = (int)min((int64_t)a.tw, ras.cols - C0);
    const int WS = cell_stride(a.tw);
    const int P = perim_count(h, w);
    const int pm = a.pmax;
    const size_t tb = (size_t)t * pm, eb = (size_t)t * a.th * a.tw, ib = (size_t)t * (pm + 8);

    // one segment per entry cell: nseg <= perimeter cells of the nominal tile
    const int pc = perim_count(a.th, a.tw);
    u128 *inS = reinterpret_cast<u128 *>(smem);  // [pc] in(e), perimeter-graph scale
    OV *pre = reinterpret_cast<OV *>(inS);       //   later: prefix sums of F over grouped joins
    OV *inT = reinterpret_cast<OV *>(inS + pc);  // [pc] in(e), this tile's scale
    OV *F = inT + pc;                            // [pc] flow at the end of segment e
    int *par = reinterpret_cast<int *>(F + pc);  // [pc] segment e joins, or -1
    int *pend = par + pc;                        // [pc] joins into e not yet summed
    int *mfill = pend;                           //   later: fill counts of the groups
    int *moff = pend + pc;                       // [pc + 1] start of e's joins in mlist
    uint16_t *mpos = reinterpret_cast<uint16_t *>(moff + pc + 1);  // [pc] position e joins at
    uint16_t *mlist = mpos + pc;                 // [pc] joining segments grouped by target

    if (tid == 0) s_emax = INT_MIN;
    for (int e = tid; e < nseg; e += nt) {
        inS[e] = 0;
        pend[e] = 0;
        moff[e] = 0;
    }
    __syncthreads();

    // ---- in(e) = sum of G over the exits outside draining into entry e
    for (int j = tid; j < ninf; j += nt) {
        const uint32_t src = a.inf_src[ib + j];
        const uint16_t lk = a.link[src];
        if (lk == LINK_TERM) continue;  // never: a cell draining into this tile is an exit
        const size_t gi = src - src % (uint32_t)pm + lk;
        if constexpr (VALM == 0)
            atomicAdd(reinterpret_cast<unsigned long long *>(&inS[a.inf_seg[ib + j]]),
                      reinterpret_cast<const unsigned long long *>(a.G)[gi]);
        else
            atomic_add_u128(&inS[a.inf_seg[ib + j]], reinterpret_cast<const u128 *>(a.G)[gi]);
    }
    // ---- the join tree of the segments
    for (int e = tid; e < nseg; e += nt) {
        const uint32_t m = a.seg_merge[tb + e];
        if (m == NO_JOIN) {
            par[e] = -1;
            continue;
        }
        const int p = (int)(m >> 16);
        par[e] = p;
        mpos[e] = (uint16_t)(m & 0xFFFFu);
        atomicAdd(&pend[p], 1);
        atomicAdd(&moff[p], 1);
    }
    __syncthreads();
    const int qf = VALM ? fix_scale(a.fcells, *a.maxw) : 0;
    if constexpr (VALM == 1) {
        int emax = INT_MIN;
        for (int e = tid; e < nseg; e += nt) {
            if (inS[e] == 0) continue;
            int ex;
            frexp(fabs(fix2d(inS[e], qf)), &ex);
            emax = max(emax, ex);
        }
        if (emax != INT_MIN) atomicMax(&s_emax, emax);
        __syncthreads();
        if (s_emax == INT_MIN) return;  // no inflow at all
    }
    // offsets of this tile stay below P * max|in(e)| < 2^(emax + log2 P)
    int qo = 0;
    if constexpr (VALM == 1) {
        int lp = 0;
        while ((1 << lp) < P) ++lp;
        qo = 62 - (s_emax + lp + 1);
    }
    for (int e = tid; e < nseg; e += nt) {
        OV v;
        if constexpr (VALM == 0) {
            v = (OV)inS[e];
        } else {
            const int sh = qf - qo;  // from the graph scale to this tile's scale
            const i128 si = (i128)inS[e];
            v = (OV)(sh >= 0 ? (sh < 127 ? (si >> sh) : (si < 0 ? -1 : 0)) : (si << (-sh)));
        }
        inT[e] = v;
        F[e] = v;
    }
    __syncthreads();

    // ---- F over the join tree, leaves first (one warp; the rounds end when
    // no segment became ready, at the latest after nseg rounds)
    if (warp == 0) {
        for (int round = 0; round <= nseg; ++round) {
            bool any = false;
            for (int e = lane; e < nseg; e += 32)
                if (pend[e] == 0) {
                    pend[e] = -2;  // ready: every join into e is summed
                    any = true;
                }
            if (!__any_sync(0xffffffffu, any)) break;
            __syncwarp();
            for (int e = lane; e < nseg; e += 32) {
                if (pend[e] != -2) continue;
                pend[e] = -1;
                const int p = par[e];
                if (p >= 0) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&F[p]),
                              (unsigned long long)F[e]);
                    atomicSub(&pend[p], 1);
                }
            }
            __syncwarp();
        }
        // group the joins by target: exclusive scan of the counts
        int run = 0;
        for (int b0 = 0; b0 < nseg; b0 += 32) {
            const int e = b0 + lane;
            const int cnt = e < nseg ? moff[e] : 0;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (e < nseg) moff[e] = run + incl - cnt;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) moff[nseg] = run;
    }
    __syncthreads();
    for (int e = tid; e < nseg; e += nt) mfill[e] = 0;
    __syncthreads();
    for (int e = tid; e < nseg; e += nt) {
        const int p = par[e];
        if (p >= 0) mlist[moff[p] + atomicAdd(&mfill[p], 1)] = (uint16_t)e;
    }
    __syncthreads();
    // each target: its joins by position, then running sums of their F
    for (int p = tid; p < nseg; p += nt) {
        const int b = moff[p], n = moff[p + 1] - b;
        for (int i = 1; i < n; ++i) {  // insertion sort (join lists are short)
            const uint16_t x = mlist[b + i];
            int j = i - 1;
            while (j >= 0 && mpos[mlist[b + j]] > mpos[x]) {
                mlist[b + j + 1] = mlist[b + j];
                --j;
            }
            mlist[b + j + 1] = x;
        }
        OV run = 0;
        for (int i = 0; i < n; ++i) {
            run += F[mlist[b + i]];
            pre[b + i] = run;
        }
    }
    __syncthreads();

    // ---- every forest cell: read-modify-write its output
    int ovf = 0;
    const double inv = ldexp(1.0, -qo);
    for (int j = tid; j < nef; j += nt) {
        const uint32_t cp = a.ef_cp[eb + j];
        const int e = a.ef_seg[eb + j];
        const int ci = (int)(cp >> 16), pos = (int)(cp & 0xFFFFu);
        OV o = inT[e];
        int lo = moff[e], hi = moff[e + 1];  // joins into e at positions <= pos
        const int b = lo;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)mpos[mlist[mid]] <= pos) lo = mid + 1;
            else hi = mid;
        }
        if (lo > b) o += pre[lo - 1];
        if (!o) continue;
        const int r = ci / WS, c = ci - r * WS;
        const size_t oi = (size_t)(R0 + r) * ras.po + (size_t)(C0 + c);
        if constexpr (VALM == 0) {
            uint32_t *p = reinterpret_cast<uint32_t *>(ras.out) + oi;
            const unsigned long long s64 = (unsigned long long)*p + o;
            if (s64 >> 32) ovf = 1;
            *p = (uint32_t)s64;
        } else {
            float *p = reinterpret_cast<float *>(ras.out) + oi;
            *p = (float)((double)*p + (double)o * inv);
        }
    }
    ovf = __syncthreads_or(ovf);
    if (tid == 0 && ovf) status_report(a.st, FA_FLAG_OVERFLOW, 0, NO_INDEX);
}

// ---------------------------------------------------------------------------
// perimeter-graph (exit forest) resolve
// ---------------------------------------------------------------------------
struct ForestArgs {
    int64_t tiles;
    int pmax;
    int64_t cells;
    int valm;
    const uint32_t *nexit;
    const uint16_t *link;
    const uint32_t *node_dst;
    const double *node_val;
    void *x, *dl0, *dl1;  // u64 (counts) or u128 (fixed-point sums) per node
    uint32_t *J0, *J1;
    uint32_t *misc;  // [0] max|w| bits, [1 + k] active nodes in round k
    StatusBlock *st;
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
    V *x = reinterpret_cast<V *>(f.x), *dl0 = reinterpret_cast<V *>(f.dl0),
      *dl1 = reinterpret_cast<V *>(f.dl1);
    const uint32_t n = f.nexit[tile];
    const int q = f.valm ? fix_scale(f.cells, f.misc[0]) : 0;
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const double v = f.node_val[node];
        if constexpr (sizeof(V) == 8) x[node] = (V)v;  // an exact integer count
        else x[node] = f.valm ? d2fix(v, q) : (u128)(unsigned long long)v;
        dl0[node] = 0;
        dl1[node] = 0;
        const uint32_t dst = f.node_dst[node];
        const uint16_t l = f.link[dst];
        f.J0[node] = l == LINK_TERM ? NODE_NONE : (dst / f.pmax) * f.pmax + l;
    }
}

// One doubling round: x_{k+1}(v) = x_k(v) + sum over u with J_k(u) = v of
// x_k(u), J_{k+1} = J_k o J_k.  After rounds 0..m-1 every node holds the sum
// of A_loc over all nodes at most 2^m - 1 links upstream, i.e. the product
// (I + P)(I + P^2)...(I + P^(2^(m-1))) applied to A_loc, which equals
// (I - P)^-1 A_loc once 2^m exceeds the longest path.
template <class V>
__global__ void k_forest_round(ForestArgs f, int k) {
    if (k > 0 && f.misc[k] == 0) return;  // round k-1 moved nothing: done
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    V *x = reinterpret_cast<V *>(f.x);
    V *dprev = reinterpret_cast<V *>((k & 1) ? f.dl0 : f.dl1);
    V *dcur = reinterpret_cast<V *>((k & 1) ? f.dl1 : f.dl0);
    const uint32_t *Jc = (k & 1) ? f.J1 : f.J0;
    uint32_t *Jn = (k & 1) ? f.J0 : f.J1;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int nact = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        V xv = x[node];
        if (k > 0) {
            const V d = dprev[node];
            if (d) {
                xv += d;
                x[node] = xv;
                dprev[node] = 0;
            }
        }
        const uint32_t jj = Jc[node];
        if (jj != NODE_NONE) {
            atomic_add_v(&dcur[jj], xv);
            Jn[node] = Jc[jj];
            ++nact;
        } else {
            Jn[node] = NODE_NONE;
        }
    }
    nact = warp_sum(nact);
    if (lane == 0 && nact) atomicAdd(&f.misc[1 + k], (uint32_t)nact);
}

// Absorb whatever is still pending and flag nodes whose paths never ended
// (a cross-tile cycle).
template <class V>
__global__ void k_forest_final(ForestArgs f, int kmax) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    V *x = reinterpret_cast<V *>(f.x), *dl0 = reinterpret_cast<V *>(f.dl0),
      *dl1 = reinterpret_cast<V *>(f.dl1);
    const bool live = f.misc[kmax] != 0;
    const uint32_t *Jl = (kmax & 1) ? f.J1 : f.J0;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int ncyc = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const V d = dl0[node] + dl1[node];
        if (d) x[node] += d;
        if (live && Jl[node] != NODE_NONE) ++ncyc;
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
    const size_t T = (size_t)g.tiles(), S = T * g.pmax;
    w.kmax = jump_rounds((int64_t)S);
    w.status = c.take<uint8_t>(64);
    w.misc = c.take<uint32_t>(2 + w.kmax);
    w.nexit = c.take<uint32_t>(T);
    w.link = c.take<uint16_t>(S);
    w.node_dst = c.take<uint32_t>(S);
    w.node_val = c.take<double>(S);
    w.x = c.take<u128>(S);
    w.dl0 = c.take<u128>(S);
    w.dl1 = c.take<u128>(S);
    w.J0 = c.take<uint32_t>(S);
    w.J1 = c.take<uint32_t>(S);
    const size_t cells = T * (size_t)g.th * g.tw, inf = T * (size_t)(g.pmax + 8);
    w.ef_hdr = c.take<uint32_t>(T * 4);
    w.ef_cp = c.take<uint32_t>(cells);
    w.ef_seg = c.take<uint16_t>(cells);
    w.seg_merge = c.take<uint32_t>(S);
    w.inf_src = c.take<uint32_t>(inf);
    w.inf_seg = c.take<uint16_t>(inf);
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

// Shared-memory limit and blocks per SM of k_solve<VALM, TMA> for a tile shape
// (set and queried once per shape).
template <int VALM, int TMA>
static cudaError_t solve_config(const Geom &g, int &blocks_per_sm) {
    static int configured = 0;
    static int per_sm = 0, per_sm_smem = -1, per_sm_nt = -1;
    const size_t smem = solve_smem_bytes(g.th, g.tw, VALM, TMA);
    cudaError_t e = set_smem(k_solve<VALM, TMA>, smem, configured);
    if (e != cudaSuccess) return e;
    const int nt = solve_threads(g.th, g.tw);
    if (per_sm_smem != (int)smem || per_sm_nt != nt) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<VALM, TMA>, nt, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        per_sm_smem = (int)smem;
        per_sm_nt = nt;
    }
    blocks_per_sm = per_sm;
    return cudaSuccess;
}

template <int VALM>
static cudaError_t offsets_config(const Geom &g) {
    static int configured = 0;
    return set_smem(k_offsets<VALM>, offsets_smem_bytes(g.th, g.tw), configured);
}

template <int VALM, int TMA>
static cudaError_t launch_solve_k(const Geom &g, const TileArgs &ta, const CUtensorMap &m,
                                  cudaStream_t s) {
    int per_sm = 1;
    cudaError_t e = solve_config<VALM, TMA>(g, per_sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ta.T, (int64_t)per_sm * sm_count());
    k_solve<VALM, TMA><<<grid, solve_threads(g.th, g.tw), solve_smem_bytes(g.th, g.tw, VALM, TMA), s>>>(ta, m);
    return cudaGetLastError();
}

template <int VALM>
static cudaError_t launch_solve(const Geom &g, const TileArgs &ta, const uint8_t *codes,
                                int64_t pc, const uint8_t *mask, bool allow_tma, cudaStream_t s) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const bool packed = g.code_format == FA_CODES_NIBBLE;
    const int mode = packed ? LOAD_TMA_PACKED : LOAD_TMA;
    if (allow_tma && solve_smem_bytes(g.th, g.tw, VALM, mode) <= 227 * 1024 &&
        make_code_map(g, codes, pc, mask, packed, &m))
        return packed ? launch_solve_k<VALM, LOAD_TMA_PACKED>(g, ta, m, s)
                      : launch_solve_k<VALM, LOAD_TMA>(g, ta, m, s);
    return launch_solve_k<VALM, LOAD_PLAIN>(g, ta, m, s);
}

template <int VALM>
static cudaError_t launch_offsets(const Geom &g, const TileArgs &ta, cudaStream_t s) {
    cudaError_t e = offsets_config<VALM>(g);
    if (e != cudaSuccess) return e;
    k_offsets<VALM><<<(unsigned)ta.T, 128, offsets_smem_bytes(g.th, g.tw), s>>>(ta);
    return cudaGetLastError();
}

// Sets the kernels' shared-memory limits and caches their occupancy and the SM
// count ahead of a stream capture (done on first use otherwise).  Batches
// never stage codes by TMA.
cudaError_t prepare_forward(const Geom &g, int val_mode) {
    int per_sm = 1;
    cudaError_t e = val_mode ? solve_config<1, LOAD_PLAIN>(g, per_sm) : solve_config<0, LOAD_PLAIN>(g, per_sm);
    if (e == cudaSuccess) e = val_mode ? offsets_config<1>(g) : offsets_config<0>(g);
    sm_count();
    return e;
}

// Status reset, pass 1, the perimeter-graph resolve and pass 2 for the tiles
// described by `ta` (one raster, or a batch through ta.rtab).
static cudaError_t run_pipeline(const Geom &g, TileArgs ta, int val_mode, const FwdWork &ws,
                                void *status, const uint8_t *tma_codes, int64_t tma_pc,
                                const uint8_t *tma_mask, cudaStream_t s) {
    StatusBlock *st = reinterpret_cast<StatusBlock *>(status ? status : ws.status);
    k_init_status<<<1, 64, 0, s>>>(st, ws.misc, 2 + ws.kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ta.T == 0) return cudaSuccess;

    ta.th = g.th;
    ta.tw = g.tw;
    ta.pmax = g.pmax;
    ta.nib = g.code_format == FA_CODES_NIBBLE;
    ta.nexit = ws.nexit;
    ta.link = ws.link;
    ta.node_dst = ws.node_dst;
    ta.node_val = ws.node_val;
    ta.G = ws.x;
    ta.st = st;
    ta.maxw = ws.misc;
    ta.ef_hdr = ws.ef_hdr;
    ta.ef_cp = ws.ef_cp;
    ta.ef_seg = ws.ef_seg;
    ta.seg_merge = ws.seg_merge;
    ta.inf_src = ws.inf_src;
    ta.inf_seg = ws.inf_seg;

    timing_mark(0, s);
    const bool tma = !(g.flags & FA_OPT_NO_TMA) && ta.rtab == nullptr;
    e = val_mode ? launch_solve<1>(g, ta, tma_codes, tma_pc, tma_mask, tma, s)
                 : launch_solve<0>(g, ta, tma_codes, tma_pc, tma_mask, tma, s);
    if (e != cudaSuccess) return e;
    timing_mark(1, s);

    ForestArgs f;
    f.tiles = ta.T;
    f.pmax = g.pmax;
    f.cells = ta.fcells;
    f.valm = val_mode;
    f.nexit = ws.nexit;
    f.link = ws.link;
    f.node_dst = ws.node_dst;
    f.node_val = ws.node_val;
    f.x = ws.x;
    f.dl0 = ws.dl0;
    f.dl1 = ws.dl1;
    f.J0 = ws.J0;
    f.J1 = ws.J1;
    f.misc = ws.misc;
    f.st = st;
    const unsigned fb = (unsigned)((f.tiles * 32 + 255) / 256);
    if (val_mode) {
        k_forest_init<u128><<<fb, 256, 0, s>>>(f);
        for (int k = 0; k < ws.kmax; ++k) k_forest_round<u128><<<fb, 256, 0, s>>>(f, k);
        k_forest_final<u128><<<fb, 256, 0, s>>>(f, ws.kmax);
    } else {
        k_forest_init<unsigned long long><<<fb, 256, 0, s>>>(f);
        for (int k = 0; k < ws.kmax; ++k) k_forest_round<unsigned long long><<<fb, 256, 0, s>>>(f, k);
        k_forest_final<unsigned long long><<<fb, 256, 0, s>>>(f, ws.kmax);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_mark(2, s);
    e = val_mode ? launch_offsets<1>(g, ta, s) : launch_offsets<0>(g, ta, s);
    timing_mark(3, s);
    timing_set_count(3);
    return e;
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
    r.w = w;
    r.pw = pw;
    r.out = out;
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
    return run_pipeline(g, ta, val_mode, ws, status, codes, pc, mask, s);
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
