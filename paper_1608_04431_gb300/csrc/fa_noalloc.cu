// fa_accumulate_noalloc: fa_accumulate for callers that cannot allocate.
//
// Some callers can hand this library their input and output rasters but have
// no way to give it scratch memory: a plugin host whose interface passes only
// the caller's buffers, a pipeline that reserves every byte of device memory
// up front and forbids allocation once it runs, or a program whose device
// memory belongs to another framework's allocator that it cannot ask for more.
// For them this entry point takes its scratch from one fixed buffer compiled
// into the library (FA_NOALLOC_SCRATCH_BYTES), so a call allocates nothing.
//
// The buffer is a file-scope __device__ array.  On the host its name only
// stands in for the symbol; the device address comes from
// cudaGetSymbolAddress, asked on every call with the caller's device current
// (cheap once the module is loaded, and never stale: a device reset or a new
// primary context may load the module at another address).  The first call on
// a device may load the library's module there, so make it outside any stream
// capture.  Every call on a device shares the one buffer: calls that may
// overlap on the GPU (different streams, or host threads without ordering
// between them) race and corrupt each other's results, so serialise them.
// The buffer keeps whatever the previous call left in it; the pipeline resets
// the parts it reads before writing them (the status block and the round
// counters are cleared by its first kernel; every per-tile and per-node record
// is written before it is read), so no stale value reaches a result.
#include "fa_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FA_NOALLOC_SCRATCH_BYTES];

bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

}  // namespace

extern "C" fa_status fa_accumulate_noalloc(const uint8_t *codes, int64_t rows, int64_t cols,
                                           int64_t pitch_codes, const float *weights,
                                           int64_t pitch_w, const uint8_t *mask,
                                           int64_t pitch_mask, void *out, fa_out_dtype out_dtype,
                                           int64_t pitch_out, const fa_options *opts,
                                           int32_t *d_status, void *stream) {
    using namespace fa;
    Geom g;
    if (!make_geom(rows, cols, opts, g)) return FA_ERR_INVALID_ARG;
    if (out_dtype != FA_OUT_U32 && out_dtype != FA_OUT_F32) return FA_ERR_INVALID_ARG;
    if (out_dtype == FA_OUT_U32 && weights) return FA_ERR_INVALID_ARG;
    if (!forward_tile_ok(g, out_dtype == FA_OUT_F32 ? 1 : 0)) return FA_ERR_INVALID_ARG;
    // the limit callers can query: fa_workspace_size (the forward pass needs
    // no more than that)
    if (fa_workspace_size(rows, cols, opts) > (size_t)FA_NOALLOC_SCRATCH_BYTES) return FA_ERR_TOO_LARGE;
    const bool empty = rows == 0 || cols == 0;
    if (!empty) {
        if (!codes || !out) return FA_ERR_INVALID_ARG;
        if (pitch_codes < code_row_bytes(cols, g.code_format) || pitch_out < cols) return FA_ERR_INVALID_ARG;
        if (weights && pitch_w < cols) return FA_ERR_INVALID_ARG;
        if (mask && pitch_mask < cols) return FA_ERR_INVALID_ARG;
        if (!aligned_to(out, 4) || (weights && !aligned_to(weights, 4))) return FA_ERR_INVALID_ARG;
    }
    if (d_status && !aligned_to(d_status, 8)) return FA_ERR_INVALID_ARG;
    void *scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch)
        return FA_ERR_CUDA;
    FwdWork w;
    carve_forward(scratch, (size_t)FA_NOALLOC_SCRATCH_BYTES, g, w, false);
    // phase timing would create CUDA events on first use: none on this thread
    const bool timing = timing_swap(false);
    const cudaError_t err =
        launch_forward(g, codes, pitch_codes, mask, pitch_mask, weights, pitch_w, out, pitch_out,
                       out_dtype == FA_OUT_F32 ? 1 : 0, w, d_status, (cudaStream_t)stream);
    timing_swap(timing);
    return err == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
