// Code translation and packing: foreign direction codes to this library's
// codes through a 256-entry table, written one per byte or packed two per
// byte (Section 4 notes that the ten code values fit in half a byte).
//
// One thread handles eight consecutive cells of a row: one 8-byte load of
// source codes when the row allows it, eight table lookups in shared memory,
// and one 8-byte (bytes) or 4-byte (nibbles) store.  The kernel moves 1 B in
// and 1 B (or 0.5 B) out per cell and is bound by HBM bandwidth.
#include <algorithm>

#include "fa_internal.h"

namespace {

struct RecodeArgs {
    const uint8_t *src;
    int64_t ps;
    uint8_t *dst;
    int64_t pd;
    int64_t rows, cols;
    int nib;
    int has_table;
    uint8_t table[256];
};

__global__ void __launch_bounds__(256) k_recode(const RecodeArgs a) {
    __shared__ uint8_t lut[256];
    const int tid = threadIdx.x;
    lut[tid] = a.has_table ? a.table[tid] : (uint8_t)tid;  // blockDim.x == 256
    __syncthreads();
    const int64_t G = (a.cols + 7) >> 3;  // eight-cell groups per row
    const bool vs = ((reinterpret_cast<uintptr_t>(a.src) | (uintptr_t)a.ps) & 7) == 0;
    const bool vd = ((reinterpret_cast<uintptr_t>(a.dst) | (uintptr_t)a.pd) & (a.nib ? 3 : 7)) == 0;
    for (int64_t r = blockIdx.y; r < a.rows; r += gridDim.y) {
        const uint8_t *sr = a.src + r * a.ps;
        uint8_t *dr = a.dst + r * a.pd;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + tid; g < G; g += (int64_t)gridDim.x * blockDim.x) {
            const int64_t c0 = g << 3;
            const int n = (int)min((int64_t)8, a.cols - c0);
            uint32_t t[8];
            if (vs && n == 8) {
                const uint2 v = *reinterpret_cast<const uint2 *>(sr + c0);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    t[k] = lut[(v.x >> (8 * k)) & 0xFFu];
                    t[k + 4] = lut[(v.y >> (8 * k)) & 0xFFu];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) t[k] = k < n ? lut[sr[c0 + k]] : 0u;
            }
            if (!a.nib) {
                if (vd && n == 8) {
                    *reinterpret_cast<uint2 *>(dr + c0) =
                        make_uint2(t[0] | (t[1] << 8) | (t[2] << 16) | (t[3] << 24),
                                   t[4] | (t[5] << 8) | (t[6] << 16) | (t[7] << 24));
                } else {
                    for (int k = 0; k < n; ++k) dr[c0 + k] = (uint8_t)t[k];
                }
            } else {
                uint32_t packed = 0;  // byte k: cell 2k low nibble, cell 2k + 1 high nibble
#pragma unroll
                for (int k = 0; k < 8; ++k) packed |= min(t[k], 15u) << (4 * k);
                uint8_t *dp = dr + (c0 >> 1);
                if (vd && n == 8) {
                    *reinterpret_cast<uint32_t *>(dp) = packed;
                } else {
                    for (int k = 0; k < (n + 1) >> 1; ++k) dp[k] = (uint8_t)(packed >> (8 * k));
                }
            }
        }
    }
}

}  // namespace

extern "C" fa_status fa_recode(const uint8_t *src, int64_t rows, int64_t cols, int64_t pitch_src,
                               const uint8_t *table, uint8_t *dst, int64_t pitch_dst,
                               int32_t dst_format, void *stream) {
    if (rows < 0 || cols < 0) return FA_ERR_INVALID_ARG;
    if (dst_format != FA_CODES_BYTE && dst_format != FA_CODES_NIBBLE) return FA_ERR_INVALID_ARG;
    if (rows == 0 || cols == 0) return FA_OK;
    if (!src || !dst || pitch_src < cols || pitch_dst < fa::code_row_bytes(cols, dst_format))
        return FA_ERR_INVALID_ARG;
    RecodeArgs a;
    a.src = src;
    a.ps = pitch_src;
    a.dst = dst;
    a.pd = pitch_dst;
    a.rows = rows;
    a.cols = cols;
    a.nib = dst_format == FA_CODES_NIBBLE;
    a.has_table = table != nullptr;
    for (int i = 0; i < 256; ++i) a.table[i] = table ? table[i] : (uint8_t)i;
    const int64_t G = (cols + 7) >> 3;
    const dim3 grid((unsigned)std::min<int64_t>((G + 255) / 256, 1024),
                    (unsigned)std::min<int64_t>(rows, 65535));
    k_recode<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
