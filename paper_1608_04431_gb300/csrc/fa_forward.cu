// Forward D8 flow accumulation: tile passes and perimeter-graph resolve.
//
// Pipeline for one raster (Section 3 of the paper, EVICT strategy):
//   pass 1  k_tile<.., 1>   per tile: Algorithm 1 (dependency counts, then the
//                           queue-free equivalent of its Kahn loop) and
//                           Algorithm 2 (each perimeter cell's exit link);
//                           emits the tile-local accumulation at every exit
//                           cell and the target of its flow (Section 3.2).
//   resolve k_forest_*      the global flow graph over exit cells
//                           (Section 3.2): G(e) = A_loc(e) + sum of G over the
//                           exits whose flow enters the tile at a cell linked
//                           to e, by pointer-jumping rounds.
//   pass 2  k_tile<.., 2>   per tile: recompute the tile (EVICT, Section 3.3)
//                           with w'(p) = w(p) + in(p), where in(p) is the flow
//                           entering at perimeter cell p from neighbouring
//                           tiles, and write A.  Adding in(p) to the weight of
//                           p carries it along p's whole downstream path, which
//                           is what Algorithm 3 does when it adds the offset
//                           to every cell downstream of the entry.
#include <climits>
#include <type_traits>

#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

constexpr uint16_t LINK_TERM = 0xFFFF;   // flow path ends inside the tile
constexpr uint32_t NODE_NONE = 0xFFFFFFFFu;
constexpr long long NO_INDEX = LLONG_MAX;

struct TileArgs {
    int64_t rows, cols;
    int th, tw, tiles_x, pmax;
    const uint8_t *codes;
    int64_t pc;
    const uint8_t *mask;
    int64_t pm;
    const float *w;
    int64_t pw;
    void *out;
    int64_t po;
    uint32_t *nexit;
    uint16_t *link;
    uint32_t *node_dst;
    double *node_val;
    const u128 *G;
    StatusBlock *st;
    uint32_t *maxw;
};

// fixed-point scale: |sum| <= cells * max|w| < 2^124 * 2^-q
__device__ __forceinline__ int fix_scale(int64_t cells, uint32_t maxw_bits) {
    float mw = __uint_as_float(maxw_bits);
    if (!(mw > 0.0f) || maxw_bits >= 0x7f800000u) return 0;
    int e;
    frexp((double)cells * (double)mw, &e);  // bound < 2^e
    return 124 - e;
}

template <class V>
struct ValOps;

template <>
struct ValOps<uint32_t> {
    __device__ static uint32_t zero() { return 0u; }
};
template <>
struct ValOps<FF> {
    __device__ static FF zero() { return FF{0.0f, 0.0f}; }
};

__device__ __forceinline__ int off_of(int k, int W2) { return dir_dr(k) * W2 + dir_dc(k); }

// block-wide sum / min helpers (blockDim.x <= 1024, multiple of 32)
__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ long long warp_min_ll(long long v) {
    for (int o = 16; o; o >>= 1) {
        long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}
__device__ __forceinline__ uint32_t warp_max_u(uint32_t v) {
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Exclusive scan of one int per thread over the block; returns the prefix and
// writes the total to *total.  Uses s_warp (>= 32 ints of shared memory).
__device__ int block_exclusive_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_warp[lane] = t;  // inclusive warp-total prefix
    }
    __syncthreads();
    int before = wid ? s_warp[wid - 1] : 0;
    *total = s_warp[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <int VALM>
struct ValType {
    typedef uint32_t type;
};
template <>
struct ValType<1> {
    typedef FF type;
};

// shared-memory bytes for a tile pass
__host__ __device__ inline size_t tile_smem_bytes(int th, int tw, int valm) {
    size_t nh = (size_t)(th + 2) * (tw + 2);
    size_t vb = valm ? 8 : 4;
    size_t b = nh * vb;                  // val
    b += ((nh + 3) / 4) * 4;             // packed counters
    b += nh;                             // effective codes
    b += nh;                             // predecessor masks
    b = (b + 1) & ~size_t(1);
    b += (size_t)(2 * th + 2 * tw) * 2;  // exit ranks per perimeter slot
    return b;
}

// ---------------------------------------------------------------------------
// per-tile pass (PASS 1 or 2)
// ---------------------------------------------------------------------------
template <int VALM, int PASS>
__global__ void __launch_bounds__(256) k_tile(TileArgs a) {
    typedef typename ValType<VALM>::type V;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_warp[33];
    __shared__ int s_cnt_bad, s_cnt_cyc, s_flags;
    __shared__ long long s_first;
    __shared__ uint32_t s_maxw;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int t = blockIdx.x;
    const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
    const int64_t R0 = (int64_t)ty * a.th, C0 = (int64_t)tx * a.tw;
    const int h = (int)min((int64_t)a.th, a.rows - R0);
    const int w = (int)min((int64_t)a.tw, a.cols - C0);
    const int W2 = w + 2, NH = (h + 2) * W2;
    const int NHmax = (a.th + 2) * (a.tw + 2);
    const int n_in = h * w;

    V *val = reinterpret_cast<V *>(smem);
    uint32_t *cnt4 = reinterpret_cast<uint32_t *>(smem + sizeof(V) * NHmax);
    uint8_t *cnt8 = reinterpret_cast<uint8_t *>(cnt4);
    uint8_t *ec = reinterpret_cast<uint8_t *>(cnt4 + (NHmax + 3) / 4);
    uint8_t *pmk = ec + NHmax;
    uint16_t *rank = reinterpret_cast<uint16_t *>(
        (reinterpret_cast<uintptr_t>(pmk + NHmax) + 1) & ~uintptr_t(1));

    if (tid == 0) {
        s_cnt_bad = 0;
        s_cnt_cyc = 0;
        s_flags = 0;
        s_first = NO_INDEX;
        s_maxw = 0;
    }

    // ---- load the tile's codes with a one-cell halo (Algorithm 1's F) -------
    int nbad = 0;
    long long fbad = NO_INDEX;
    for (int i = tid; i < NH; i += nt) {
        const int hr = i / W2, hc = i - hr * W2;
        const int64_t gr = R0 - 1 + hr, gc = C0 - 1 + hc;
        uint8_t e = 0;
        if (gr >= 0 && gr < a.rows && gc >= 0 && gc < a.cols) {
            const uint8_t k = a.codes[gr * a.pc + gc];
            const bool inside = hr >= 1 && hr <= h && hc >= 1 && hc <= w;
            if (k > 9) {
                if (PASS == 1 && inside) {
                    ++nbad;
                    fbad = min(fbad, (long long)(gr * a.cols + gc));
                }
            } else if (k != 0 && !(a.mask && a.mask[gr * a.pm + gc])) {
                e = k | (inside ? 0 : HALO);
            }
        }
        ec[i] = e;
    }
    __syncthreads();

    // ---- dependency counts D from in-tile upstream neighbours (gather) ------
    uint32_t maxw = 0;
    int nonfinite = 0;
    for (int j = tid; j < n_in; j += nt) {
        const int r = j / w, c = j - r * w;
        const int i = (r + 1) * W2 + (c + 1);
        const uint8_t e = ec[i];
        uint8_t m = 0;
        V v0 = ValOps<V>::zero();
        if (e) {
#pragma unroll
            for (int k = 1; k <= 8; ++k) {
                const uint8_t en = ec[i + off_of(k, W2)];
                if (en && !(en & HALO) && (en & 15) == dir_rev(k)) m |= uint8_t(1u << (k - 1));
            }
            if constexpr (VALM == 0) {
                v0 = 1u;
            } else {
                const float wv = a.w ? a.w[(R0 + r) * a.pw + (C0 + c)] : 1.0f;
                const uint32_t b = __float_as_uint(wv) & 0x7fffffffu;
                if (b >= 0x7f800000u) nonfinite = 1;
                maxw = max(maxw, b);
                v0 = FF{wv, 0.0f};
            }
        }
        pmk[i] = m;
        cnt8[i] = (uint8_t)__popc(m);
        val[i] = v0;
    }
    __syncthreads();

    int ovf = 0;
    // ---- pass 2: add the inflow from neighbouring tiles to entry cells -----
    if constexpr (PASS == 2) {
        const int P = perim_count(h, w);
        const int q = VALM ? fix_scale(a.rows * a.cols, *a.maxw) : 0;
        for (int s = tid; s < P; s += nt) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            if (!ec[i]) continue;
            u128 inflow = 0;
            bool any = false;
#pragma unroll
            for (int k = 1; k <= 8; ++k) {
                const uint8_t en = ec[i + off_of(k, W2)];
                if ((en & HALO) && (en & 15) == dir_rev(k)) {
                    const int64_t gr = R0 + r + dir_dr(k), gc = C0 + c + dir_dc(k);
                    const int tyh = (int)(gr / a.th), txh = (int)(gc / a.tw);
                    const int hh = (int)min((int64_t)a.th, a.rows - (int64_t)tyh * a.th);
                    const int wh = (int)min((int64_t)a.tw, a.cols - (int64_t)txh * a.tw);
                    const int sh = slot_of((int)(gr - (int64_t)tyh * a.th),
                                           (int)(gc - (int64_t)txh * a.tw), hh, wh);
                    const size_t tbase = ((size_t)tyh * a.tiles_x + txh) * a.pmax;
                    const uint16_t l = a.link[tbase + sh];
                    if (l != LINK_TERM) {  // always an exit rank: h drains out of its tile
                        inflow += a.G[tbase + l];
                        any = true;
                    }
                }
            }
            if (!any) continue;
            if constexpr (VALM == 0) {
                const uint64_t s64 = (uint64_t)val[i] + (uint64_t)inflow;
                if ((inflow >> 32) != 0 || (s64 >> 32) != 0) ovf = 1;
                val[i] = (uint32_t)s64;
            } else {
                val[i] = ff_add(val[i], fix2ff(inflow, q));
            }
        }
        __syncthreads();
    }

    // ---- Kahn loop without a queue: walk from every source; a cell is final
    // once its last in-tile upstream neighbour is, and the thread that
    // delivers that last dependency carries on downstream (pull-gather in
    // fixed E..SE order keeps floating-point sums deterministic). -------------
    for (int j = tid; j < n_in; j += nt) {
        const int r = j / w, c = j - r * w;
        const int i0 = (r + 1) * W2 + (c + 1);
        if (!ec[i0] || pmk[i0]) continue;
        int cur = i0;
        for (int step = 0; step < n_in; ++step) {
            uint8_t m = pmk[cur];
            if constexpr (VALM == 0) {
                uint64_t s64 = val[cur];
                while (m) {
                    const int k = __ffs(m);
                    m &= m - 1;
                    s64 += val[cur + off_of(k, W2)];
                }
                if (s64 >> 32) ovf = 1;
                val[cur] = (uint32_t)s64;
            } else {
                FF v = val[cur];
                while (m) {
                    const int k = __ffs(m);
                    m &= m - 1;
                    v = ff_add(v, val[cur + off_of(k, W2)]);
                }
                val[cur] = v;
            }
            const int k = ec[cur] & 15;
            if (k == 9) break;
            const int nxt = cur + off_of(k, W2);
            const uint8_t et = ec[nxt];
            if (!et || (et & HALO)) break;
            __threadfence_block();
            const int sh = (nxt & 3) * 8;
            const uint32_t old = atomicSub(&cnt4[nxt >> 2], 1u << sh);
            if (((old >> sh) & 0xffu) != 1u) break;
            __threadfence_block();
            cur = nxt;
        }
    }
    __syncthreads();

    if constexpr (PASS == 1) {
        // ---- cells never finalised lie on in-tile cycles ------------------
        int ncyc = 0;
        long long fcyc = NO_INDEX;
        for (int j = tid; j < n_in; j += nt) {
            const int r = j / w, c = j - r * w;
            const int i = (r + 1) * W2 + (c + 1);
            if (ec[i] && cnt8[i]) {
                ++ncyc;
                fcyc = min(fcyc, (long long)((R0 + r) * a.cols + (C0 + c)));
            }
        }
        // ---- exit cells (flow leaves the tile into a valid cell) get ranks -
        const int P = perim_count(h, w);
        const int chunk = (P + nt - 1) / nt;
        const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
        int mine = 0;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            bool ex = false;
            if (k >= 1 && k <= 8) ex = (ec[i + off_of(k, W2)] & HALO) != 0;
            mine += ex;
        }
        int total;
        int rk = block_exclusive_scan(mine, s_warp, &total);
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            bool ex = false;
            if (k >= 1 && k <= 8) ex = (ec[i + off_of(k, W2)] & HALO) != 0;
            rank[s] = ex ? (uint16_t)rk++ : LINK_TERM;
        }
        __syncthreads();
        // ---- Algorithm 2 for every perimeter cell; exit records -----------
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = tid; s < P; s += nt) {
            int r, c;
            cell_of(s, h, w, r, c);
            int cur = (r + 1) * W2 + (c + 1);
            uint16_t lk = LINK_TERM;
            if (ec[cur]) {
                for (int step = 0; step <= n_in; ++step) {
                    const int k = ec[cur] & 15;
                    if (k == 9) break;
                    const int nxt = cur + off_of(k, W2);
                    const uint8_t et = ec[nxt];
                    if (!et) break;
                    if (et & HALO) {
                        const int cr = cur / W2 - 1, cc = cur - (cur / W2) * W2 - 1;
                        lk = rank[slot_of(cr, cc, h, w)];
                        break;
                    }
                    cur = nxt;
                }
            }
            a.link[tbase + s] = lk;
            const uint16_t myrank = rank[s];
            if (myrank != LINK_TERM) {
                const int i = (r + 1) * W2 + (c + 1);
                const int k = ec[i] & 15;
                const int64_t gr = R0 + r + dir_dr(k), gc = C0 + c + dir_dc(k);
                const int tyd = (int)(gr / a.th), txd = (int)(gc / a.tw);
                const int hd = (int)min((int64_t)a.th, a.rows - (int64_t)tyd * a.th);
                const int wd = (int)min((int64_t)a.tw, a.cols - (int64_t)txd * a.tw);
                const int sd = slot_of((int)(gr - (int64_t)tyd * a.th),
                                       (int)(gc - (int64_t)txd * a.tw), hd, wd);
                a.node_dst[tbase + myrank] =
                    (uint32_t)(((size_t)tyd * a.tiles_x + txd) * a.pmax + sd);
                double v;
                if constexpr (VALM == 0) v = (double)val[i];
                else v = (double)val[i].hi + (double)val[i].lo;
                a.node_val[tbase + myrank] = v;
            }
        }
        if (tid == 0) a.nexit[t] = (uint32_t)total;
        // ---- status -------------------------------------------------------
        nbad = warp_sum(nbad);
        ncyc = warp_sum(ncyc);
        fbad = warp_min_ll(min(fbad, fcyc));
        maxw = warp_max_u(maxw);
        nonfinite = warp_sum(nonfinite);
        if ((tid & 31) == 0) {
            if (nbad) atomicAdd(&s_cnt_bad, nbad);
            if (ncyc) atomicAdd(&s_cnt_cyc, ncyc);
            if (fbad != NO_INDEX) atomicMin(&s_first, fbad);
            if (maxw) atomicMax(&s_maxw, maxw);
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
    } else {
        // ---- pass 2: write A (0 for NoData and for cells on cycles) --------
        for (int j = tid; j < n_in; j += nt) {
            const int r = j / w, c = j - r * w;
            const int i = (r + 1) * W2 + (c + 1);
            const bool fin = ec[i] && !cnt8[i];
            const size_t o = (size_t)(R0 + r) * a.po + (C0 + c);
            if constexpr (VALM == 0) {
                reinterpret_cast<uint32_t *>(a.out)[o] = fin ? val[i] : 0u;
            } else {
                reinterpret_cast<float *>(a.out)[o] = fin ? ff_round(val[i]) : 0.0f;
            }
        }
        ovf = __syncthreads_or(ovf);
        if (tid == 0 && ovf) status_report(a.st, FA_FLAG_OVERFLOW, 0, NO_INDEX);
    }
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
    u128 *x, *dl0, *dl1;
    uint32_t *J0, *J1;
    uint32_t *misc;  // [0] max|w| bits, [1 + k] active nodes in round k
    StatusBlock *st;
};

__global__ void k_forest_init(ForestArgs f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t n = f.nexit[tile];
    const int q = f.valm ? fix_scale(f.cells, f.misc[0]) : 0;
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const double v = f.node_val[node];
        f.x[node] = f.valm ? d2fix(v, q) : (u128)(unsigned long long)v;
        f.dl0[node] = 0;
        f.dl1[node] = 0;
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
__global__ void k_forest_round(ForestArgs f, int k) {
    if (k > 0 && f.misc[k] == 0) return;  // round k-1 moved nothing: done
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    u128 *dprev = (k & 1) ? f.dl0 : f.dl1;
    u128 *dcur = (k & 1) ? f.dl1 : f.dl0;
    const uint32_t *Jc = (k & 1) ? f.J1 : f.J0;
    uint32_t *Jn = (k & 1) ? f.J0 : f.J1;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int nact = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        u128 xv = f.x[node];
        if (k > 0) {
            const u128 d = dprev[node];
            if (d) {
                xv += d;
                f.x[node] = xv;
                dprev[node] = 0;
            }
        }
        const uint32_t jj = Jc[node];
        if (jj != NODE_NONE) {
            atomic_add_u128(&dcur[jj], xv);
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
__global__ void k_forest_final(ForestArgs f, int kmax) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const bool live = f.misc[kmax] != 0;
    const uint32_t *Jl = (kmax & 1) ? f.J1 : f.J0;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int ncyc = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const u128 d = f.dl0[node] + f.dl1[node];
        if (d) f.x[node] += d;
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
    // node ids are tile * pmax + rank in 32 bits
    if ((double)g.tiles() * g.pmax >= 4.0e9) return false;
    return true;
}

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
    (void)dry;
    return c.used() + 256;
}

template <int VALM, int PASS>
static cudaError_t launch_tile(const Geom &g, const TileArgs &ta, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(g.th, g.tw, VALM);
    static int configured = 0;
    if (smem > 48 * 1024 && configured < (int)smem) {
        cudaError_t e = cudaFuncSetAttribute(k_tile<VALM, PASS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = (int)smem;
    }
    const int cells = g.th * g.tw;
    int nt = cells >= 256 ? 256 : ((cells + 31) / 32) * 32;
    k_tile<VALM, PASS><<<(unsigned)g.tiles(), nt, smem, s>>>(ta);
    return cudaGetLastError();
}

cudaError_t launch_forward(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                           int64_t pm, const float *w, int64_t pw, void *out, int64_t po,
                           int val_mode, const FwdWork &ws, void *status, cudaStream_t s) {
    StatusBlock *st = reinterpret_cast<StatusBlock *>(status ? status : ws.status);
    k_init_status<<<1, 64, 0, s>>>(st, ws.misc, 2 + ws.kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (g.rows == 0 || g.cols == 0) return cudaSuccess;

    TileArgs ta;
    ta.rows = g.rows;
    ta.cols = g.cols;
    ta.th = g.th;
    ta.tw = g.tw;
    ta.tiles_x = g.tiles_x;
    ta.pmax = g.pmax;
    ta.codes = codes;
    ta.pc = pc;
    ta.mask = mask;
    ta.pm = pm;
    ta.w = w;
    ta.pw = pw;
    ta.out = out;
    ta.po = po;
    ta.nexit = ws.nexit;
    ta.link = ws.link;
    ta.node_dst = ws.node_dst;
    ta.node_val = ws.node_val;
    ta.G = reinterpret_cast<const u128 *>(ws.x);
    ta.st = st;
    ta.maxw = ws.misc;

    timing_mark(0, s);
    e = val_mode ? launch_tile<1, 1>(g, ta, s) : launch_tile<0, 1>(g, ta, s);
    if (e != cudaSuccess) return e;
    timing_mark(1, s);

    ForestArgs f;
    f.tiles = g.tiles();
    f.pmax = g.pmax;
    f.cells = g.rows * g.cols;
    f.valm = val_mode;
    f.nexit = ws.nexit;
    f.link = ws.link;
    f.node_dst = ws.node_dst;
    f.node_val = ws.node_val;
    f.x = reinterpret_cast<u128 *>(ws.x);
    f.dl0 = reinterpret_cast<u128 *>(ws.dl0);
    f.dl1 = reinterpret_cast<u128 *>(ws.dl1);
    f.J0 = ws.J0;
    f.J1 = ws.J1;
    f.misc = ws.misc;
    f.st = st;
    const unsigned fb = (unsigned)((f.tiles * 32 + 255) / 256);
    k_forest_init<<<fb, 256, 0, s>>>(f);
    for (int k = 0; k < ws.kmax; ++k) k_forest_round<<<fb, 256, 0, s>>>(f, k);
    k_forest_final<<<fb, 256, 0, s>>>(f, ws.kmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_mark(2, s);
    e = val_mode ? launch_tile<1, 2>(g, ta, s) : launch_tile<0, 2>(g, ta, s);
    timing_mark(3, s);
    timing_set_count(3);
    return e;
}

}  // namespace fa
