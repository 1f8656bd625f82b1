// D8 flow codes from an elevation raster: the step before accumulation.
//
// The paper treats the direction step as a separate algorithm (Fig. 1) and
// the accumulation as valid for any non-divergent metric, which sends a cell's
// flow to a single neighbour (Section 2); D8 takes the steepest descent, and
// flats are routed towards lower terrain only.  The rules, one per cell:
//   - NoData (mask byte != 0): code 0;
//   - a cell on the raster's border drains off the grid, perpendicular to its
//     edge (N, S, W, E) and diagonally at the corners (NW, NE, SW, SE);
//   - otherwise the valid neighbour with the largest positive slope, slope =
//     drop for E, N, W, S and drop * (1/sqrt 2) for the diagonals, drop =
//     z(cell) - z(neighbour); neighbours in the order E, NE, N, NW, W, SW, S,
//     SE, a later one winning only when strictly steeper;
//   - no positive slope: the first NoData neighbour in that order, else
//     NoFlow (9).
// The slope is decided in float32 with one rounded subtraction and one
// rounded multiplication by the float nearest 1/sqrt 2 (no fused operation),
// so every platform takes the same decision.
//
// One thread computes four consecutive cells of eight consecutive rows,
// sliding a 3 x 6 window of elevations (and NoData bits) down the rows: each
// row of the window is loaded once (one 16-byte load and two scalars), and
// each output row is one 4-byte store.
#include <algorithm>

#include "fa_common.cuh"
#include "fa_internal.h"

namespace {

constexpr float kInvSqrt2 = 0.70710678118654752440f;

struct D8Args {
    const float *z;
    int64_t pz;
    const uint8_t *nd;
    int64_t pnd;
    uint8_t *out;
    int64_t po;
    int64_t rows, cols;
};

__device__ __forceinline__ uint32_t border_code(bool top, bool bottom, bool left, bool right) {
    if (top && left) return 4;
    if (top && right) return 2;
    if (bottom && left) return 6;
    if (bottom && right) return 8;
    if (top) return 3;
    if (bottom) return 7;
    if (left) return 5;
    return 1;
}

constexpr int kRows = 8;  // consecutive rows per thread (rolling window)

// Row rr of the window around the thread's four cells c0..c0+3: elevations of
// columns c0-1..c0+4 and a NoData bit per column (0 outside the raster).
__device__ __forceinline__ void load_row(const D8Args &a, int64_t rr, int64_t c0, bool vz, bool vn,
                                         float v[6], uint32_t &nd) {
    nd = 0u;
    if (rr < 0 || rr >= a.rows) {
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = 0.0f;
        return;
    }
    const float *zr = a.z + rr * a.pz;
    if (vz) {
        const float4 m = __ldg(reinterpret_cast<const float4 *>(zr + c0));
        v[1] = m.x;
        v[2] = m.y;
        v[3] = m.z;
        v[4] = m.w;
    } else {
#pragma unroll
        for (int j = 1; j <= 4; ++j) v[j] = c0 + j - 1 < a.cols ? __ldg(zr + c0 + j - 1) : 0.0f;
    }
    v[0] = c0 >= 1 ? __ldg(zr + c0 - 1) : 0.0f;
    v[5] = c0 + 4 < a.cols ? __ldg(zr + c0 + 4) : 0.0f;
    if (a.nd) {
        const uint8_t *nr = a.nd + rr * a.pnd;
        if (vn) {
            const uint32_t m = __vcmpne4(__ldg(reinterpret_cast<const unsigned int *>(nr + c0)), 0u);
            // byte b (all ones when NoData) -> window bit b + 1
            nd = ((m & 1u) << 1) | ((m >> 6) & 4u) | ((m >> 13) & 8u) | ((m >> 20) & 16u);
        } else {
#pragma unroll
            for (int j = 1; j <= 4; ++j)
                if (c0 + j - 1 < a.cols && __ldg(nr + c0 + j - 1)) nd |= 1u << j;
        }
        if (c0 >= 1 && __ldg(nr + c0 - 1)) nd |= 1u;
        if (c0 + 4 < a.cols && __ldg(nr + c0 + 4)) nd |= 32u;
    }
}

// One thread: four consecutive cells of kRows consecutive rows, keeping the
// window's previous two rows in registers so each row is loaded once.
__global__ void __launch_bounds__(256, 4) k_d8(D8Args a) {
    const int64_t G = (a.cols + 3) >> 2;  // four-cell groups per row
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int64_t c0 = 4 * g;
    const bool full = c0 + 4 <= a.cols;
    const bool vz = full && ((reinterpret_cast<uintptr_t>(a.z) | ((uintptr_t)a.pz << 2)) & 15) == 0;
    const bool vn = full && ((reinterpret_cast<uintptr_t>(a.nd) | (uintptr_t)a.pnd) & 3) == 0;
    const bool vo = full && ((reinterpret_cast<uintptr_t>(a.out) | (uintptr_t)a.po) & 3) == 0;
    const int64_t r0 = ((int64_t)blockIdx.y * blockDim.y + threadIdx.y) * kRows;
    if (r0 >= a.rows) return;
    float v[3][6];  // rows r-1, r, r+1
    uint32_t ndm[3];
    load_row(a, r0 - 1, c0, vz, vn, v[0], ndm[0]);
    load_row(a, r0, c0, vz, vn, v[1], ndm[1]);
#pragma unroll 1
    for (int i = 0; i < kRows; ++i) {
        const int64_t r = r0 + i;
        if (r >= a.rows) break;
        load_row(a, r + 1, c0, vz, vn, v[2], ndm[2]);
        uint32_t codes = 0;
        if (!(ndm[0] | ndm[1] | ndm[2]) && r > 0 && r < a.rows - 1 && c0 > 0 && c0 + 4 < a.cols) {
            // the common case: four interior cells and no NoData in the window
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float zc = v[1][q + 1];
                float best = 0.0f;
                uint32_t pick = 9u;
#pragma unroll
                for (int k = 1; k <= 8; ++k) {
                    const float drop = __fsub_rn(zc, v[fa::dir_dr(k) + 1][q + 1 + fa::dir_dc(k)]);
                    const float slope = (k & 1) ? drop : __fmul_rn(drop, kInvSqrt2);
                    if (slope > best) {
                        best = slope;
                        pick = (uint32_t)k;
                    }
                }
                codes |= pick << (8 * q);
            }
        } else
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t c = c0 + q;
            if (c >= a.cols) break;
            uint32_t code;
            if ((ndm[1] >> (q + 1)) & 1u) {
                code = 0;
            } else if (r == 0 || r == a.rows - 1 || c == 0 || c == a.cols - 1) {
                code = border_code(r == 0, r == a.rows - 1, c == 0, c == a.cols - 1);
            } else {
                const float zc = v[1][q + 1];
                float best = 0.0f;
                uint32_t pick = 0, into_nd = 0;
#pragma unroll
                for (int k = 1; k <= 8; ++k) {
                    const int d = fa::dir_dr(k) + 1, j = q + 1 + fa::dir_dc(k);
                    if ((ndm[d] >> j) & 1u) {
                        if (!into_nd) into_nd = (uint32_t)k;
                        continue;
                    }
                    const float drop = __fsub_rn(zc, v[d][j]);
                    const float slope = (k & 1) ? drop : __fmul_rn(drop, kInvSqrt2);
                    if (slope > best) {
                        best = slope;
                        pick = (uint32_t)k;
                    }
                }
                code = pick ? pick : (into_nd ? into_nd : 9u);
            }
            codes |= code << (8 * q);
        }
        uint8_t *orow = a.out + r * a.po + c0;
        if (vo) {
            *reinterpret_cast<uint32_t *>(orow) = codes;
        } else {
            for (int q = 0; q < 4 && c0 + q < a.cols; ++q) orow[q] = (uint8_t)(codes >> (8 * q));
        }
        // slide the window down one row
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            v[0][j] = v[1][j];
            v[1][j] = v[2][j];
        }
        ndm[0] = ndm[1];
        ndm[1] = ndm[2];
    }
}

}  // namespace

extern "C" fa_status fa_d8_codes(const float *dem, int64_t rows, int64_t cols, int64_t pitch_dem,
                                 const uint8_t *nodata, int64_t pitch_nodata, uint8_t *codes,
                                 int64_t pitch_codes, void *stream) {
    if (rows < 0 || cols < 0) return FA_ERR_INVALID_ARG;
    if (rows == 0 || cols == 0) return FA_OK;
    if (!dem || !codes || pitch_dem < cols || pitch_codes < cols) return FA_ERR_INVALID_ARG;
    if (nodata && pitch_nodata < cols) return FA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(dem) & 3) return FA_ERR_INVALID_ARG;
    D8Args a{dem, pitch_dem, nodata, pitch_nodata, codes, pitch_codes, rows, cols};
    const int64_t G = (cols + 3) >> 2;
    const int64_t chunks = (rows + kRows - 1) / kRows;  // row chunks of kRows
    if ((chunks + 3) / 4 > 65535) return FA_ERR_INVALID_ARG;  // more than 2,097,120 rows
    const dim3 block(64, 4);
    const dim3 grid((unsigned)((G + 63) / 64), (unsigned)((chunks + 3) / 4));
    k_d8<<<grid, block, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
