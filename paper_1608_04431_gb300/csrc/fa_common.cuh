// Device-side building blocks shared by the flow-accumulation kernels.
//
// Code encoding (one byte per cell): 0 NoData, 1..8 = E, NE, N, NW, W, SW, S,
// SE, 9 NoFlow, 10..255 invalid.  Row 0 is north.
#pragma once

#include <climits>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fa {

typedef unsigned __int128 u128;
typedef __int128 i128;

// ---------------------------------------------------------------------------
// direction decoding without memory lookups: (dr+1) and (dc+1) for codes 0..9
// packed two bits per code into one 32-bit constant each.
// ---------------------------------------------------------------------------
constexpr uint32_t pack2(const int (&v)[10]) {
    uint32_t p = 0;
    for (int k = 0; k < 10; ++k) p |= uint32_t(v[k] + 1) << (2 * k);
    return p;
}
constexpr int kDRtab[10] = {0, 0, -1, -1, -1, 0, 1, 1, 1, 0};
constexpr int kDCtab[10] = {0, 1, 1, 0, -1, -1, -1, 0, 1, 0};
constexpr uint32_t kDRP = pack2(kDRtab);
constexpr uint32_t kDCP = pack2(kDCtab);

__host__ __device__ __forceinline__ int dir_dr(int k) { return int((kDRP >> (2 * k)) & 3u) - 1; }
__host__ __device__ __forceinline__ int dir_dc(int k) { return int((kDCP >> (2 * k)) & 3u) - 1; }
// the direction that points back: E<->W, NE<->SW, N<->S, NW<->SE
__host__ __device__ __forceinline__ int dir_rev(int k) { return ((k + 3) & 7) + 1; }

// Effective code byte kept in shared memory for the tile and its one-cell halo:
// 0 = NoData / off-grid / masked / invalid; otherwise the code 1..9, with
// HALO set for a valid cell that lies outside the tile.
constexpr uint8_t HALO = 0x10;

// ---------------------------------------------------------------------------
// perimeter slots of an h x w tile: top row west->east, right column north->
// south, bottom row east->west, left column south->north; each perimeter cell
// exactly once.  P = w (h == 1), h (w == 1), else 2w + 2h - 4.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int perim_count(int h, int w) {
    if (h == 1) return w;
    if (w == 1) return h;
    return 2 * w + 2 * h - 4;
}

__host__ __device__ __forceinline__ int slot_of(int r, int c, int h, int w) {
    if (h == 1) return c;
    if (w == 1) return r;
    if (r == 0) return c;
    if (c == w - 1) return w - 1 + r;
    if (r == h - 1) return (w + h - 2) + (w - 1 - c);
    return (2 * w + h - 3) + (h - 1 - r);  // c == 0, 1 <= r <= h-2
}

__host__ __device__ __forceinline__ void cell_of(int s, int h, int w, int &r, int &c) {
    if (h == 1) { r = 0; c = s; return; }
    if (w == 1) { r = s; c = 0; return; }
    if (s < w) { r = 0; c = s; return; }
    s -= w;
    if (s < h - 1) { r = 1 + s; c = w - 1; return; }
    s -= h - 1;
    if (s < w - 1) { r = h - 1; c = w - 2 - s; return; }
    s -= w - 1;
    r = h - 2 - s;
    c = 0;
}

// ---------------------------------------------------------------------------
// compensated float pair (hi + lo, |lo| <= ulp(hi)/2): ~48-bit sums from FP32
// arithmetic (Knuth TwoSum, then a Fast2Sum renormalisation).  The _rn
// intrinsics keep the compiler from contracting or reordering the steps.
// ---------------------------------------------------------------------------
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return FF{hi, lo};
}

__device__ __forceinline__ float ff_round(FF a) { return __fadd_rn(a.hi, a.lo); }

// ---------------------------------------------------------------------------
// 128-bit two's-complement fixed point with 2^-q resolution, used for the
// cross-tile (perimeter graph) sums: integer addition is associative, so the
// order in which atomics land cannot change a single bit of the result.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int clz128(u128 a) {
    uint64_t hi = uint64_t(a >> 64), lo = uint64_t(a);
    return hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
}

__device__ __forceinline__ u128 shl_s(u128 v, int sh) {
    if (sh >= 128 || sh <= -128) return 0;
    return sh >= 0 ? (v << sh) : (v >> (-sh));
}

// exact for any double whose bits at and above 2^-q fit; lower bits truncated
// toward zero.
__device__ __forceinline__ u128 d2fix(double x, int q) {
    if (x == 0.0) return 0;
    int e;
    double m = frexp(x, &e);  // x = m * 2^e, 0.5 <= |m| < 1
    long long mi = (long long)ldexp(m, 53);
    bool neg = mi < 0;
    u128 v = (u128)(unsigned long long)(neg ? -mi : mi);
    v = shl_s(v, e - 53 + q);
    return neg ? (u128)(-(i128)v) : v;
}

// nearest-ish double of a fixed-point value (top 64 bits rounded to 53)
__device__ __forceinline__ double fix2d(u128 v, int q) {
    bool neg = (int64_t)(uint64_t)(v >> 64) < 0;
    u128 a = neg ? (u128)(-(i128)v) : v;
    if (a == 0) return 0.0;
    int top = 127 - clz128(a);
    int sh = top - 63;
    uint64_t t = sh >= 0 ? uint64_t(a >> sh) : uint64_t(a << (-sh));
    double d = ldexp((double)t, sh - q);
    return neg ? -d : d;
}

__device__ __forceinline__ FF fix2ff(u128 v, int q) {
    double d = fix2d(v, q);
    float hi = (float)d;
    u128 r = v - d2fix((double)hi, q);  // exact residual in fixed point
    float lo = (float)fix2d(r, q);
    return FF{hi, lo};
}

__device__ __forceinline__ void atomic_add_u128(u128 *addr, u128 v) {
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    unsigned long long *p = reinterpret_cast<unsigned long long *>(addr);
    unsigned long long old = atomicAdd(p, lo);
    if (old + lo < old) hi += 1ull;  // carry out of the low word
    if (hi) atomicAdd(p + 1, hi);
}

// ---------------------------------------------------------------------------
// device status block (see fa.h): flags, count, smallest offending index
// ---------------------------------------------------------------------------
struct StatusBlock {
    int32_t flags;
    int32_t count;
    long long first;  // smallest offending cell index, LLONG_MAX when none
};

__device__ __forceinline__ void status_report(StatusBlock *st, int flag, int n, long long first) {
    atomicOr(&st->flags, flag);
    if (n) atomicAdd(&st->count, n);
    if (first != 0x7fffffffffffffffll) atomicMin(&st->first, first);
}

// ---------------------------------------------------------------------------
// shared constants and block/warp helpers
// ---------------------------------------------------------------------------
constexpr uint16_t LINK_TERM = 0xFFFF;   // flow path ends inside the tile
constexpr uint32_t NODE_NONE = 0xFFFFFFFFu;
constexpr long long NO_INDEX = LLONG_MAX;

__device__ __forceinline__ int off_of(int k, int W2) { return dir_dr(k) * W2 + dir_dc(k); }

// block-wide sum / min helpers (blockDim.x <= 1024, multiple of 32)
// Named barrier `id` (1..15) over the first n threads of the block (n a
// multiple of 32); the block-wide barrier is id 0.
__device__ __forceinline__ void bar_sync_n(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Named barrier that also returns whether any participating thread passed
// a nonzero `pred`.
__device__ __forceinline__ int bar_or_n(int id, int n, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %3, 0;\n\t"
        "bar.red.or.pred q, %1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(id), "r"(n), "r"(pred)
        : "memory");
    return r;
}

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
static __device__ int block_exclusive_scan(int v, int *s_warp, int *total) {
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

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) and mbarrier helpers, inline PTX for sm_103a
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// 2-D tiled load of the box at (x, y) of `map` into dst; completes `bar`'s
// transaction count.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// The SM's global nanosecond timer.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Default bound of a device-side wait: a staged copy of a few kilobytes
// completes within microseconds, so a wait still pending after one second
// will not complete.
constexpr uint64_t kWaitLimitNs = 1000000000ull;
// Bounded wait for phase `parity` of `bar`: polls until the phase completes
// or `limit_ns` of global time have passed since the first poll; false if the
// bound ran out.  A failed try_wait suspends the thread for a few
// microseconds, so the timer is read a few hundred thousand times a second.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

}  // namespace fa
