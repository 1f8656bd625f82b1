// Flow accumulation with absorption: Eq. 1 with alpha(n, p) = a(n) for the one
// downstream cell p = d(n) of n, a(n) in [0, 1] (Section 2: flow may be
// absorbed on its way downhill but never increased):
//     A(p) = w(p) + sum over n with d(n) = p of a(n) A(n).
// Same tile decomposition as the plain forms (Section 3):
//
//   pass 1  k_abs_tile<1>  per tile: every cell's in-tile path end and the
//                          product of a along the way, by gather pointer
//                          jumping; A_loc of each exit as the sum of w times
//                          that product over the cells whose paths end there;
//                          the exits ranked, each with A_loc(e), a(e) and the
//                          slot d(e) leads to; every perimeter slot with the
//                          exit its path reaches (Algorithm 2) and its product.
//   forest  k_abs_forest_* G(e) = A_loc(e) + sum over exits e' leading to e of
//                          a(e') P(d(e')) G(e'), P the product of a from the
//                          entry d(e') to e: pointer jumping with multipliers
//                          over the exit forest (Section 3.2).
//   pass 2  k_abs_tile<2>  the tile solved again (EVICT, Section 3.3) with
//                          a(h) G(h) added at every entry cell for each
//                          outside cell h draining into it; writes A.
//
// Everything is integer arithmetic, so results are bitwise reproducible and no
// FP64 is used (it is slow on this GPU): values are 64-bit fixed point with a
// per-tile scale 2^q chosen from the tile's terms so that every partial sum
// stays below 2^62 (factors <= 1 never raise a sum), 128-bit fixed point in
// the forest; factors are Q1.63 (a * 2^63), and a value times a factor is the
// top of a 64 x 64 -> 128-bit product.  Truncations are below 2^-62 of the
// tile's total per operation.
#include <algorithm>
#include <cstring>

#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

constexpr uint16_t ABS_NONE = 0xFFFF;
constexpr uint64_t Q63_ONE = 1ull << 63;
constexpr int ABS_CPT = 4;  // cells per thread of a tile block

// ---------------------------------------------------------------------------
// integer fixed-point helpers
// ---------------------------------------------------------------------------
// float -> Q1.63, for 0 <= a <= 1 (a * 2^63, truncated)
__device__ __forceinline__ uint64_t factor_q63(float a) {
    const uint32_t b = __float_as_uint(a);
    int e = (int)((b >> 23) & 0xFFu);
    uint64_t m = b & 0x7FFFFFu;
    if (e == 0) {
        if (!m) return 0;
        e = 1;
    } else {
        m |= 0x800000u;
    }
    const int sh = e - 87;  // a = m 2^(e - 150); a 2^63 = m 2^(e - 87)
    return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0);
}

// (x y) >> 63 for Q1.63 factors x, y <= 2^63.  For y < 2^63 that is the high
// word of x (2y); y = 2^63 is the factor 1.
__device__ __forceinline__ uint64_t mul_q63(uint64_t x, uint64_t y) {
    return y == Q63_ONE ? x : __umul64hi(x, y << 1);
}

// a signed 64-bit fixed-point value times a Q1.63 factor (truncated to zero)
__device__ __forceinline__ long long scale_q63(long long x, uint64_t m) {
    const uint64_t ax = x < 0 ? (uint64_t)(-x) : (uint64_t)x;
    const uint64_t r = m == Q63_ONE ? ax : __umul64hi(ax, m << 1);
    return x < 0 ? -(long long)r : (long long)r;
}

// a signed 128-bit fixed-point value (|v| < 2^126) times a Q1.63 factor
__device__ __forceinline__ u128 scale128_q63(u128 v, uint64_t m) {
    const bool neg = (i128)v < 0;
    const u128 a = neg ? (u128)(-(i128)v) : v;
    const u128 plo = (u128)(uint64_t)a * m, phi = (u128)(uint64_t)(a >> 64) * m;
    const u128 r = (phi << 1) + (plo >> 63);
    return neg ? (u128)(-(i128)r) : r;
}

// a signed 128-bit fixed-point value times 2^sh (arithmetic shift)
__device__ __forceinline__ u128 shift_signed(u128 v, int sh) {
    if (sh >= 0) return sh >= 128 ? (u128)0 : (u128)((i128)v << sh);
    if (sh <= -128) return (i128)v < 0 ? ~(u128)0 : (u128)0;
    return (u128)((i128)v >> (-sh));
}

// float -> signed 64-bit fixed point x 2^q (truncated toward zero); the caller
// guarantees |x| 2^q < 2^62
__device__ __forceinline__ long long float_to_fix(float x, int q) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu);
    uint64_t m = b & 0x7FFFFFu;
    if (e == 0) {
        if (!m) return 0;
        e = 1;
    } else {
        m |= 0x800000u;
    }
    const int sh = e - 150 + q;
    const uint64_t v = sh >= 0 ? (sh < 40 ? (m << sh) : 0) : (sh > -64 ? (m >> (-sh)) : 0);
    return (b >> 31) ? -(long long)v : (long long)v;
}

// Adds a 64-bit two's-complement value to a shared-memory word with two 32-bit
// atomics: the carry of each addition into the high word is known from the
// low word's old value, so the high word receives exactly the carries of all
// additions.
__device__ __forceinline__ void smem_add64(long long *p, long long v) {
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const uint32_t lo = (uint32_t)(unsigned long long)v, hi = (uint32_t)((unsigned long long)v >> 32);
    const uint32_t old = atomicAdd(&w[0], lo);
    const uint32_t h = hi + (old + lo < old ? 1u : 0u);
    if (h) atomicAdd(&w[1], h);
}

// 2^e as a float, -126 <= e <= 127
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// signed 64-bit fixed point x 2^-q -> float, rounded once
__device__ __forceinline__ float fix_to_float(long long x, int q) {
    float f = __ll2float_rn(x);
    // scale by 2^-q in exact power-of-two steps
    int s = -q;
    while (s > 126) { f = __fmul_rn(f, pow2f(126)); s -= 126; }
    while (s < -126) { f = __fmul_rn(f, pow2f(-126)); s += 126; }
    return __fmul_rn(f, pow2f(s));
}

// floor(log2 |x|) of a finite nonzero float (subnormals included)
__device__ __forceinline__ int float_exp(float x) {
    const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu;
    const int e = (int)(b >> 23);
    return e ? e - 127 : (31 - __clz(b)) - 149;
}

// floor(log2 |v|) of a nonzero signed 128-bit fixed point value at scale 2^qf
__device__ __forceinline__ int fix128_exp(u128 v, int qf) {
    const u128 a = (i128)v < 0 ? (u128)(-(i128)v) : v;
    return 127 - clz128(a) - qf;
}

// floor(n / d) for n, d < 2^16 as one multiply: with m = ceil(2^32 / d),
// n m / 2^32 exceeds n / d by less than n / 2^32 < 1 / d, which cannot reach
// the next integer
struct FastDiv {
    uint64_t m;
    __device__ explicit FastDiv(int d) : m(((1ull << 32) + (uint64_t)d - 1) / (uint64_t)d) {}
    __device__ int operator()(int n) const { return (int)(((uint64_t)(uint32_t)n * m) >> 32); }
};

// cell m of the halo ring of an (h + 2) x W2 box: top row, bottom row, then
// the left and right columns between them
__device__ __forceinline__ void ring_cell(int m, int h, int W2, int &hr, int &hc) {
    if (m < W2) { hr = 0; hc = m; return; }
    m -= W2;
    if (m < W2) { hr = h + 1; hc = m; return; }
    m -= W2;
    if (m < h) { hr = 1 + m; hc = 0; return; }
    hr = 1 + (m - h);
    hc = W2 - 1;
}

__host__ __device__ inline int ceil_log2(int64_t n) {
    int k = 0;
    while (((int64_t)1 << k) < n) ++k;
    return k;
}

// Scale of a tile whose terms all satisfy |v| < 2^(emax + 1), n of them: every
// partial sum stays below 2^62 (factors are at most 1).  Clamped so that the
// output conversion stays in range.
__device__ __forceinline__ int abs_tile_scale(int emax, int64_t n) {
    const int q = 62 - (emax + 1 + ceil_log2(n > 0 ? n : 1));
    return max(-200, min(q, 300));
}

// Scale of the exit forest: node values are bounded by the raster's total,
// below cells * 2^(emax + 1); 126 bits of headroom.
__device__ __forceinline__ int abs_forest_scale(int emax, int64_t cells) {
    return 126 - (emax + 1 + ceil_log2(cells > 0 ? cells : 1));
}

// emax is kept in a uint32 for atomicMax: biased by this much
constexpr int EMAX_BIAS = 4096;
constexpr uint32_t EMAX_NONE = 0;  // no nonzero weight anywhere

// ---------------------------------------------------------------------------
struct AbsArgs {
    int64_t rows, cols;
    int th, tw, tiles_x, pmax, nib;
    const uint8_t *codes;
    int64_t pc;
    const uint8_t *mask;
    int64_t pm;
    const float *w;  // NULL = unit weights
    int64_t pw;
    const float *a;
    int64_t pa;
    float *out;
    int64_t po;
    uint32_t *nexit;
    int32_t *tile_q;
    uint16_t *link;       // [T*pmax] slot -> rank of the exit its path reaches, or LINK_TERM
    uint32_t *node_dst;   // [T*pmax] exit rank -> global slot of d(e)
    long long *node_x;    // [T*pmax] exit rank -> A_loc(e), tile fixed point
    uint64_t *node_fac;   // [T*pmax] exit rank -> a(e), Q1.63
    uint64_t *slot_prod;  // [T*pmax] slot -> product of a along its in-tile path, Q1.63
    const u128 *G;        // [T*pmax] exit rank -> resolved flow, forest fixed point
    uint32_t *misc;       // [0] biased max exponent of |w|
    StatusBlock *st;
};

__host__ __device__ inline size_t abs_smem_bytes(int th, int tw) {
    const size_t nh = (size_t)(th + 2) * (tw + 2), nc = (size_t)th * tw;
    size_t b = nc * (8 + 8 + 8);                     // value, round inflow, multiplier
    b += nc * 2;                                     // jump pointer
    b += (size_t)(2 * th + 2 * tw) * 2;              // exit rank per slot
    b += nh;                                         // codes with halo
    return (b + 15) & ~size_t(15);
}

__host__ __device__ inline int abs_threads(int th, int tw) {
    const int need = (th * tw + ABS_CPT - 1) / ABS_CPT;
    return min(1024, max(32, ((need + 31) / 32) * 32));
}

bool absorb_tile_ok(const Geom &g) {
    return (int64_t)g.th * g.tw <= 1024 * ABS_CPT && abs_smem_bytes(g.th, g.tw) <= 227 * 1024;
}

// code of raster cell (gr, gc) (bytes or packed)
__device__ __forceinline__ uint32_t abs_code(const AbsArgs &a, int64_t gr, int64_t gc) {
    return a.nib ? ((uint32_t)a.codes[gr * a.pc + (gc >> 1)] >> ((gc & 1) << 2)) & 15u
                 : (uint32_t)a.codes[gr * a.pc + gc];
}

// global perimeter slot of raster cell (gr, gc): its tile's base plus its slot
__device__ __forceinline__ size_t abs_global_slot(const AbsArgs &a, int64_t gr, int64_t gc) {
    const int ty = (int)(gr / a.th), tx = (int)(gc / a.tw);
    const int hh = (int)min((int64_t)a.th, a.rows - (int64_t)ty * a.th);
    const int ww = (int)min((int64_t)a.tw, a.cols - (int64_t)tx * a.tw);
    const int s = slot_of((int)(gr - (int64_t)ty * a.th), (int)(gc - (int64_t)tx * a.tw), hh, ww);
    return ((size_t)ty * a.tiles_x + tx) * a.pmax + s;
}

template <int PASS>
__global__ void __launch_bounds__(1024) k_abs_tile(AbsArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_warp[33];
    __shared__ int s_emax, s_flags, s_bad, s_cyc;
    __shared__ long long s_first;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t t = blockIdx.x;
    const int ty = (int)(t / a.tiles_x), tx = (int)(t - (int64_t)ty * a.tiles_x);
    const int64_t R0 = (int64_t)ty * a.th, C0 = (int64_t)tx * a.tw;
    const int h = (int)min((int64_t)a.th, a.rows - R0);
    const int w = (int)min((int64_t)a.tw, a.cols - C0);
    const int W2 = w + 2, NH = (h + 2) * W2;
    const int NC = a.th * a.tw;  // compact cell j = r * w + c, j < h * w
    const int n_in = h * w;
    const int P = perim_count(h, w);
    const int NR = 2 * W2 + 2 * h;  // halo ring cells
    const FastDiv div_w(w), div_W2(W2);

    long long *X = reinterpret_cast<long long *>(smem);
    long long *D = X + NC;
    uint64_t *M = reinterpret_cast<uint64_t *>(D + NC);
    uint16_t *J = reinterpret_cast<uint16_t *>(M + NC);
    uint16_t *rank = J + NC;
    uint8_t *ec = reinterpret_cast<uint8_t *>(rank + 2 * a.th + 2 * a.tw);

    if (tid == 0) {
        s_emax = INT_MIN;
        s_flags = 0;
        s_bad = 0;
        s_cyc = 0;
        s_first = NO_INDEX;
    }
    // ---- codes of the tile and its halo ring (0 = NoData, HALO outside)
    int nbad = 0;
    long long fbad = NO_INDEX;
    for (int i = tid; i < NH; i += nt) {
        const int hr = div_W2(i), hc = i - hr * W2;
        const int64_t gr = R0 - 1 + hr, gc = C0 - 1 + hc;
        uint8_t e = 0;
        if (gr >= 0 && gr < a.rows && gc >= 0 && gc < a.cols) {
            const uint32_t k = abs_code(a, gr, gc);
            const bool inside = hr >= 1 && hr <= h && hc >= 1 && hc <= w;
            if (PASS == 1 && inside && k > 9) {
                ++nbad;
                fbad = min(fbad, (long long)(gr * a.cols + gc));
            }
            if (k >= 1 && k <= 9 && !(a.mask && a.mask[gr * a.pm + gc])) e = (uint8_t)(k | (inside ? 0 : HALO));
        }
        ec[i] = e;
    }
    __syncthreads();

    // ---- own cells: successor, factor, weight exponent
    int emax = INT_MIN, bad_factor = 0;
    long long fbf = NO_INDEX;
    for (int j = tid; j < n_in; j += nt) {
        const int r = div_w(j), c = j - r * w;
        const int i = (r + 1) * W2 + (c + 1);
        const uint8_t e = ec[i];
        uint16_t nx = ABS_NONE;
        uint64_t m = 0;
        if (e) {
            const int64_t gr = R0 + r, gc = C0 + c;
            const float wv = a.w ? a.w[gr * a.pw + gc] : 1.0f;
            const float av = a.a[gr * a.pa + gc];
            const bool wok = (__float_as_uint(wv) & 0x7FFFFFFFu) < 0x7F800000u;
            const bool aok = av >= 0.0f && av <= 1.0f;  // false for NaN
            if (!wok || !aok) {
                bad_factor = 1;
                fbf = min(fbf, (long long)(gr * a.cols + gc));
            }
            if (wok && wv != 0.0f) emax = max(emax, float_exp(wv));
            const int k = e & 15;
            if (k <= 8) {
                const int n = i + off_of(k, W2);
                const uint8_t en = ec[n];
                if (en && !(en & HALO)) {
                    nx = (uint16_t)((r + dir_dr(k)) * w + (c + dir_dc(k)));
                    m = aok ? factor_q63(av) : 0;
                }
            }
        }
        J[j] = nx;
        M[j] = m;
    }
    if (emax != INT_MIN) atomicMax(&s_emax, emax);

    // ---- pass 2: the flow entering from outside, a(h) G(h) for every halo
    // cell h draining into the tile (h is an exit of its own tile)
    int qf = 0;
    if constexpr (PASS == 2) {
        const uint32_t gm = a.misc[0];
        qf = abs_forest_scale(gm == EMAX_NONE ? 0 : (int)gm - EMAX_BIAS, a.rows * a.cols);
        int emi = INT_MIN;
        for (int m = tid; m < NR; m += nt) {
            int hr, hc;
            ring_cell(m, h, W2, hr, hc);
            const int i = hr * W2 + hc;
            const uint8_t e = ec[i];
            if (!(e & HALO) || (e & 15) > 8) continue;
            const int k = e & 15;
            const int nr = hr + dir_dr(k), nc = hc + dir_dc(k);
            if (nr < 1 || nr > h || nc < 1 || nc > w) continue;
            const int n = nr * W2 + nc;
            if (!ec[n] || (ec[n] & HALO)) continue;
            const size_t gs = abs_global_slot(a, R0 - 1 + hr, C0 - 1 + hc);
            const uint16_t lk = a.link[gs];
            if (lk == LINK_TERM) continue;  // never: h's successor is valid and outside its tile
            const size_t node = gs - gs % (size_t)a.pmax + lk;
            const u128 v = scale128_q63(a.G[node], a.node_fac[node]);
            if (v) emi = max(emi, fix128_exp(v, qf));
        }
        if (emi != INT_MIN) atomicMax(&s_emax, emi);
    }
    __syncthreads();
    const int q = abs_tile_scale(s_emax == INT_MIN ? 0 : s_emax, (int64_t)n_in + P + 8);

    auto is_exit = [&](int i) {
        const int k = ec[i] & 15;
        return k >= 1 && k <= 8 && (ec[i + off_of(k, W2)] & HALO);
    };
    // a path ends at a cell without an in-tile successor (pointer doubling on
    // an in-tile cycle whose length is a power of two also comes back to the
    // cell itself, so the pointer alone does not tell)
    auto is_end = [&](int i) {
        const int k = ec[i] & 15;
        if (k < 1 || k > 8) return true;
        const uint8_t en = ec[i + off_of(k, W2)];
        return !en || (en & HALO);
    };
    const int maxr = ceil_log2(n_in > 1 ? n_in : 2) + 2;
    int ncyc = 0;
    long long fcyc = NO_INDEX;

    if constexpr (PASS == 2) {
        // ---- values at the tile's scale, the inflow added at entry cells
        for (int j = tid; j < n_in; j += nt) {
            const int r = div_w(j), c = j - r * w;
            long long x = 0;
            if (ec[(r + 1) * W2 + (c + 1)]) x = float_to_fix(a.w ? a.w[(R0 + r) * a.pw + (C0 + c)] : 1.0f, q);
            X[j] = x;
            D[j] = 0;
        }
        __syncthreads();
        for (int m = tid; m < NR; m += nt) {
            int hr, hc;
            ring_cell(m, h, W2, hr, hc);
            const int i = hr * W2 + hc;
            const uint8_t e = ec[i];
            if (!(e & HALO) || (e & 15) > 8) continue;
            const int k = e & 15;
            const int nr = hr + dir_dr(k), nc = hc + dir_dc(k);
            if (nr < 1 || nr > h || nc < 1 || nc > w) continue;
            const int n = nr * W2 + nc;
            if (!ec[n] || (ec[n] & HALO)) continue;
            const size_t gs = abs_global_slot(a, R0 - 1 + hr, C0 - 1 + hc);
            const uint16_t lk = a.link[gs];
            if (lk == LINK_TERM) continue;
            const size_t node = gs - gs % (size_t)a.pmax + lk;
            const u128 v = scale128_q63(a.G[node], a.node_fac[node]);
            const u128 vq = shift_signed(v, q - qf);  // forest scale -> tile scale
            const int p = (nr - 1) * w + (nc - 1);
            smem_add64(&X[p], (long long)(uint64_t)vq);
        }
        __syncthreads();

        // ---- pointer jumping with multipliers: x_{k+1}(v) = x_k(v) + sum over
        // u with J_k(u) = v of M_k(u) x_k(u); J_{k+1} = J_k o J_k, M_{k+1}(u) =
        // M_k(u) M_k(J_k(u)) (the product of a over the 2^(k+1) cells u leaves)
        int active = 0;
        for (int j = tid; j < n_in; j += nt) active |= J[j] != ABS_NONE;
        active = __syncthreads_or(active);
        for (int round = 0; round < maxr && active; ++round) {
            for (int j = tid; j < n_in; j += nt) {
                const uint16_t nx = J[j];
                if (nx != ABS_NONE) {
                    const long long v = scale_q63(X[j], M[j]);
                    if (v) smem_add64(&D[nx], v);
                }
            }
            __syncthreads();
            uint16_t nj[ABS_CPT];
            uint64_t nm[ABS_CPT];
            int act = 0;
#pragma unroll
            for (int u = 0; u < ABS_CPT; ++u) {
                const int j = tid + u * nt;
                nj[u] = ABS_NONE;
                nm[u] = 0;
                if (j >= n_in) continue;
                X[j] += D[j];
                D[j] = 0;
                const uint16_t nx = J[j];
                if (nx != ABS_NONE) {
                    nj[u] = J[nx];
                    if (nj[u] != ABS_NONE) {
                        nm[u] = mul_q63(M[j], M[nx]);
                        act = 1;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < ABS_CPT; ++u) {
                const int j = tid + u * nt;
                if (j >= n_in) continue;
                J[j] = nj[u];
                M[j] = nm[u];
            }
            active = __syncthreads_or(act);
        }
        for (int j = tid; j < n_in; j += nt) {
            const int r = div_w(j), c = j - r * w;
            a.out[(size_t)(R0 + r) * a.po + (C0 + c)] =
                ec[(r + 1) * W2 + (c + 1)] ? fix_to_float(X[j], q) : 0.0f;
        }
    } else {
        // ---- every cell's path end R and the product of a along the way Pp
        // (excluding the end), by gather jumping: R(j) -> R(R(j)),
        // Pp(j) -> Pp(j) Pp(R(j)); a path's last cell points at itself with
        // product 1.  J and M hold R and Pp.
        for (int j = tid; j < n_in; j += nt) {
            if (J[j] == ABS_NONE) {
                J[j] = (uint16_t)j;
                M[j] = Q63_ONE;
            }
            X[j] = 0;
        }
        __syncthreads();
        int active = 1;
        for (int round = 0; round < maxr && active; ++round) {
            // a cell whose pointer already names its path's end is settled:
            // nothing to read, multiply or write
            uint16_t nj[ABS_CPT];
            uint64_t nm[ABS_CPT];
            int act = 0, moved = 0;
#pragma unroll
            for (int u = 0; u < ABS_CPT; ++u) {
                const int j = tid + u * nt;
                nj[u] = ABS_NONE;
                if (j >= n_in) continue;
                const uint16_t nx = J[j];
                const uint16_t n2 = J[nx];
                if (n2 == nx) continue;
                nj[u] = n2;
                nm[u] = mul_q63(M[j], M[nx]);
                moved |= 1 << u;
                act |= J[n2] != n2;  // not settled after this round
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < ABS_CPT; ++u) {
                if (!((moved >> u) & 1)) continue;
                const int j = tid + u * nt;
                J[j] = nj[u];
                M[j] = nm[u];
            }
            active = __syncthreads_or(act);
        }
        // ---- A_loc at the exits: every cell y adds w(y) Pp(y) to the exit its
        // path ends at (cells whose jumps never settled lie on or drain into
        // an in-tile cycle)
        for (int j = tid; j < n_in; j += nt) {
            const int r = div_w(j), c = j - r * w;
            if (!ec[(r + 1) * W2 + (c + 1)]) continue;
            const int last = J[j];
            const int lr = div_w(last), lc = last - lr * w;
            const int li = (lr + 1) * W2 + (lc + 1);
            if (J[last] != last || !is_end(li)) {
                ++ncyc;
                fcyc = min(fcyc, (long long)((R0 + r) * a.cols + (C0 + c)));
                continue;
            }
            if (!is_exit(li)) continue;
            const long long x = scale_q63(float_to_fix(a.w ? a.w[(R0 + r) * a.pw + (C0 + c)] : 1.0f, q), M[j]);
            if (x) smem_add64(&X[last], x);
        }
        // ---- exits in slot order
        const int chunk = (P + nt - 1) / nt;
        const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
        int mine = 0;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            mine += is_exit((r + 1) * W2 + (c + 1));
        }
        int total;
        int rk = block_exclusive_scan(mine, s_warp, &total);  // its barriers publish X
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            if (is_exit(i)) {
                const int k = ec[i] & 15;
                const int64_t gr = R0 + r, gc = C0 + c;
                a.node_dst[tbase + rk] = (uint32_t)abs_global_slot(a, gr + dir_dr(k), gc + dir_dc(k));
                a.node_x[tbase + rk] = X[r * w + c];
                const float av = a.a[gr * a.pa + gc];
                a.node_fac[tbase + rk] = (av >= 0.0f && av <= 1.0f) ? factor_q63(av) : 0;
                rank[s] = (uint16_t)rk++;
            } else {
                rank[s] = LINK_TERM;
            }
        }
        __syncthreads();
        for (int s = tid; s < P; s += nt) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int j = r * w + c;
            uint16_t lk = LINK_TERM;
            uint64_t prod = 0;
            if (ec[(r + 1) * W2 + (c + 1)]) {
                const int last = J[j];
                const int lr = div_w(last), lc = last - lr * w;
                if (J[last] == last && is_exit((lr + 1) * W2 + (lc + 1)))  // an exit is a path end
                    lk = rank[slot_of(lr, lc, h, w)];
                prod = M[j];
            }
            a.link[tbase + s] = lk;
            a.slot_prod[tbase + s] = prod;
        }
        if (tid == 0) {
            a.nexit[t] = (uint32_t)total;
            a.tile_q[t] = q;
        }
        // ---- status and the raster's largest weight exponent
        if (tid == 0 && s_emax != INT_MIN) atomicMax(&a.misc[0], (uint32_t)(s_emax + EMAX_BIAS));
        nbad = warp_sum(nbad);
        ncyc = warp_sum(ncyc);
        bad_factor = warp_sum(bad_factor);
        fbad = warp_min_ll(min(fbad, min(fcyc, fbf)));
        if ((tid & 31) == 0) {
            if (nbad) atomicAdd(&s_bad, nbad);
            if (ncyc) atomicAdd(&s_cyc, ncyc);
            if (bad_factor) atomicOr(&s_flags, FA_FLAG_NONFINITE);
            if (fbad != NO_INDEX) atomicMin(&s_first, fbad);
        }
        __syncthreads();
        if (tid == 0) {
            int fl = s_flags | (s_bad ? FA_FLAG_BAD_CODE : 0) | (s_cyc ? FA_FLAG_CYCLE : 0);
            if (fl) status_report(a.st, fl, s_bad + s_cyc, s_first);
        }
    }
}

// ---------------------------------------------------------------------------
// exit forest with multipliers
// ---------------------------------------------------------------------------
struct AbsForest {
    int64_t tiles, cells;
    int pmax;
    const uint32_t *nexit;
    const int32_t *tile_q;
    const uint16_t *link;
    const uint32_t *node_dst;
    const long long *node_x;
    const uint64_t *node_fac;
    const uint64_t *slot_prod;
    u128 *x, *dl0, *dl1;
    uint32_t *J0, *J1;
    uint64_t *M0, *M1;
    uint32_t *misc;  // [0] biased max exponent, [1 + k] nodes that scattered in round k
    StatusBlock *st;
};

__global__ void k_abs_forest_init(AbsForest f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t gm = f.misc[0];
    const int qf = abs_forest_scale(gm == EMAX_NONE ? 0 : (int)gm - EMAX_BIAS, f.cells);
    const uint32_t n = f.nexit[tile];
    const int qt = f.tile_q[tile];
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        f.x[node] = shift_signed((u128)(i128)f.node_x[node], qf - qt);
        f.dl0[node] = 0;
        f.dl1[node] = 0;
        const uint32_t dst = f.node_dst[node];
        const uint16_t l = f.link[dst];
        f.J0[node] = l == LINK_TERM ? NODE_NONE : (dst / f.pmax) * f.pmax + l;
        // the share of e's flow that reaches the next exit
        f.M0[node] = mul_q63(f.node_fac[node], f.slot_prod[dst]);
    }
}

// x_{k+1}(v) = x_k(v) + sum over u with J_k(u) = v of M_k(u) x_k(u); the
// inflow of round k - 1 is folded in first
__global__ void k_abs_forest_round(AbsForest f, int k) {
    if (k > 0 && f.misc[k] == 0) return;  // round k - 1 moved nothing: done
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    u128 *dprev = (k & 1) ? f.dl0 : f.dl1;
    u128 *dcur = (k & 1) ? f.dl1 : f.dl0;
    const uint32_t *Jc = (k & 1) ? f.J1 : f.J0;
    uint32_t *Jn = (k & 1) ? f.J0 : f.J1;
    const uint64_t *Mc = (k & 1) ? f.M1 : f.M0;
    uint64_t *Mn = (k & 1) ? f.M0 : f.M1;
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
            const uint64_t m = Mc[node];
            const u128 v = scale128_q63(xv, m);
            if (v) atomic_add_u128(&dcur[jj], v);
            const uint32_t j2 = Jc[jj];
            Jn[node] = j2;
            Mn[node] = j2 == NODE_NONE ? 0 : mul_q63(m, Mc[jj]);
            ++nact;
        } else {
            Jn[node] = NODE_NONE;
        }
    }
    nact = warp_sum(nact);
    if (lane == 0 && nact) atomicAdd(&f.misc[1 + k], (uint32_t)nact);
}

__global__ void k_abs_forest_final(AbsForest f, int kmax) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const bool live = f.misc[kmax] != 0;  // the last round still moved flow
    const uint32_t *Jl = (kmax & 1) ? f.J1 : f.J0;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int ncyc = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        f.x[node] += f.dl0[node] + f.dl1[node];
        if (live && Jl[node] != NODE_NONE) ++ncyc;
    }
    ncyc = warp_sum(ncyc);
    if (lane == 0 && ncyc) status_report(f.st, FA_FLAG_CYCLE, ncyc, NO_INDEX);
}

__global__ void k_abs_init_status(StatusBlock *st, uint32_t *misc, int nmisc) {
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
struct AbsWork {
    int kmax;
    uint8_t *status;
    uint32_t *misc, *nexit, *node_dst, *J0, *J1;
    int32_t *tile_q;
    uint16_t *link;
    long long *node_x;
    uint64_t *node_fac, *slot_prod, *M0, *M1;
    u128 *x, *dl0, *dl1;
};

size_t carve_absorb(void *ws, size_t bytes, const Geom &g, AbsWork &w) {
    Carver c(ws, bytes);
    const size_t T = (size_t)g.tiles(), S = T * g.pmax;
    FwdWork fw;
    carve_forward(nullptr, 0, g, fw, true);
    w.kmax = fw.kmax;
    w.status = c.take<uint8_t>(64);
    w.misc = c.take<uint32_t>(2 + w.kmax);
    w.nexit = c.take<uint32_t>(T);
    w.tile_q = c.take<int32_t>(T);
    w.link = c.take<uint16_t>(S);
    w.node_dst = c.take<uint32_t>(S);
    w.node_x = c.take<long long>(S);
    w.node_fac = c.take<uint64_t>(S);
    w.slot_prod = c.take<uint64_t>(S);
    w.x = c.take<u128>(S);
    w.dl0 = c.take<u128>(S);
    w.dl1 = c.take<u128>(S);
    w.J0 = c.take<uint32_t>(S);
    w.J1 = c.take<uint32_t>(S);
    w.M0 = c.take<uint64_t>(S);
    w.M1 = c.take<uint64_t>(S);
    return c.used() + 256;
}

template <int PASS>
static cudaError_t launch_abs_tile(const Geom &g, const AbsArgs &aa, cudaStream_t s) {
    const size_t smem = abs_smem_bytes(g.th, g.tw);
    static int configured = 0;
    if (smem > 48 * 1024 && configured < (int)smem) {
        cudaError_t e = cudaFuncSetAttribute(k_abs_tile<PASS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = (int)smem;
    }
    k_abs_tile<PASS><<<(unsigned)g.tiles(), abs_threads(g.th, g.tw), smem, s>>>(aa);
    return cudaGetLastError();
}

cudaError_t launch_absorb(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                          int64_t pm, const float *wts, int64_t pw, const float *fac, int64_t pf,
                          float *out, int64_t po, const AbsWork &ws, void *status, cudaStream_t s) {
    StatusBlock *st = reinterpret_cast<StatusBlock *>(status ? status : ws.status);
    k_abs_init_status<<<1, 64, 0, s>>>(st, ws.misc, 2 + ws.kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (g.rows == 0 || g.cols == 0) return cudaSuccess;

    AbsArgs aa;
    std::memset(&aa, 0, sizeof(aa));
    aa.rows = g.rows;
    aa.cols = g.cols;
    aa.th = g.th;
    aa.tw = g.tw;
    aa.tiles_x = g.tiles_x;
    aa.pmax = g.pmax;
    aa.nib = g.code_format == FA_CODES_NIBBLE;
    aa.codes = codes;
    aa.pc = pc;
    aa.mask = mask;
    aa.pm = pm;
    aa.w = wts;
    aa.pw = pw;
    aa.a = fac;
    aa.pa = pf;
    aa.out = out;
    aa.po = po;
    aa.nexit = ws.nexit;
    aa.tile_q = ws.tile_q;
    aa.link = ws.link;
    aa.node_dst = ws.node_dst;
    aa.node_x = ws.node_x;
    aa.node_fac = ws.node_fac;
    aa.slot_prod = ws.slot_prod;
    aa.G = ws.x;
    aa.misc = ws.misc;
    aa.st = st;
    timing_mark(0, s);
    e = launch_abs_tile<1>(g, aa, s);
    if (e != cudaSuccess) return e;
    timing_mark(1, s);

    AbsForest f;
    f.tiles = g.tiles();
    f.cells = g.rows * g.cols;
    f.pmax = g.pmax;
    f.nexit = ws.nexit;
    f.tile_q = ws.tile_q;
    f.link = ws.link;
    f.node_dst = ws.node_dst;
    f.node_x = ws.node_x;
    f.node_fac = ws.node_fac;
    f.slot_prod = ws.slot_prod;
    f.x = ws.x;
    f.dl0 = ws.dl0;
    f.dl1 = ws.dl1;
    f.J0 = ws.J0;
    f.J1 = ws.J1;
    f.M0 = ws.M0;
    f.M1 = ws.M1;
    f.misc = ws.misc;
    f.st = st;
    const unsigned fb = (unsigned)((f.tiles * 32 + 255) / 256);
    k_abs_forest_init<<<fb, 256, 0, s>>>(f);
    for (int k = 0; k < ws.kmax; ++k) k_abs_forest_round<<<fb, 256, 0, s>>>(f, k);
    k_abs_forest_final<<<fb, 256, 0, s>>>(f, ws.kmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_mark(2, s);
    e = launch_abs_tile<2>(g, aa, s);
    timing_mark(3, s);
    timing_set_count(3);
    return e;
}

}  // namespace fa

using namespace fa;

static bool aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

// Options with the absorption default tile (32 x 64: two tile blocks per SM,
// the fastest of the measured shapes) where the caller left the shape at 0.
static fa_options absorb_options(const fa_options *opts) {
    fa_options o = opts ? *opts : fa_options{0, 0, 0, 0};
    if (!o.tile_h) o.tile_h = 32;
    if (!o.tile_w) o.tile_w = 64;
    return o;
}

extern "C" size_t fa_absorb_workspace_size(int64_t rows, int64_t cols, const fa_options *opts) {
    Geom g;
    const fa_options o = absorb_options(opts);
    if (!make_geom(rows, cols, &o, g) || !absorb_tile_ok(g)) return 0;
    AbsWork w;
    return carve_absorb(nullptr, ~size_t(0) >> 1, g, w);
}

extern "C" fa_status fa_accumulate_absorb(const uint8_t *codes, int64_t rows, int64_t cols,
                                          int64_t pitch_codes, const float *weights,
                                          int64_t pitch_w, const float *factors, int64_t pitch_f,
                                          const uint8_t *mask, int64_t pitch_mask, float *out,
                                          int64_t pitch_out, void *workspace, size_t ws_bytes,
                                          const fa_options *opts, int32_t *d_status, void *stream) {
    Geom g;
    const fa_options o = absorb_options(opts);
    if (!make_geom(rows, cols, &o, g) || !absorb_tile_ok(g)) return FA_ERR_INVALID_ARG;
    const bool empty = rows == 0 || cols == 0;
    if (!empty) {
        if (!codes || !factors || !out) return FA_ERR_INVALID_ARG;
        if (pitch_codes < code_row_bytes(cols, g.code_format) || pitch_f < cols || pitch_out < cols)
            return FA_ERR_INVALID_ARG;
        if (weights && pitch_w < cols) return FA_ERR_INVALID_ARG;
        if (mask && pitch_mask < cols) return FA_ERR_INVALID_ARG;
        if (!aligned4(out) || !aligned4(factors) || (weights && !aligned4(weights)))
            return FA_ERR_INVALID_ARG;
    }
    if (d_status && (reinterpret_cast<uintptr_t>(d_status) & 7)) return FA_ERR_INVALID_ARG;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return FA_ERR_WORKSPACE;
    AbsWork w;
    const size_t need = carve_absorb(workspace, ws_bytes, g, w);
    if (ws_bytes < need) return FA_ERR_WORKSPACE;
    const cudaError_t e = launch_absorb(g, codes, pitch_codes, mask, pitch_mask, weights, pitch_w,
                                        factors, pitch_f, out, pitch_out, w, d_status,
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
