// extern "C" entry points of libfa.so (declared in include/fa.h): argument
// validation, workspace carving and stream launches.  No device allocation.
#include <climits>
#include <cstring>

#include "fa_internal.h"

using namespace fa;

namespace {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

}  // namespace

extern "C" int32_t fa_version(void) { return 100; }

// ---- phase timing ---------------------------------------------------------
namespace {
bool g_timing = false;
// per host thread: phase events are not recorded while set (tuning loops,
// graph capture, the no-allocation entry point), whatever g_timing says, so
// one thread suppressing them never changes another thread's setting
thread_local bool t_quiet = false;
cudaEvent_t g_ev[kMaxPhase + 1];
bool g_ev_made = false;
int g_phases = 0;
}  // namespace

namespace fa {
void timing_mark(int i, cudaStream_t s) {
    if (!g_timing || t_quiet || i > kMaxPhase) return;
    if (!g_ev_made) {
        for (int j = 0; j <= kMaxPhase; ++j) cudaEventCreate(&g_ev[j]);
        g_ev_made = true;
    }
    cudaEventRecord(g_ev[i], s);
}
void timing_set_count(int n) {
    if (g_timing && !t_quiet) g_phases = n;
}
bool timing_swap(bool on) {
    const bool was = !t_quiet;
    t_quiet = !on;
    return was;
}
}  // namespace fa

extern "C" void fa_timing_enable(int32_t on) {
    g_timing = on != 0;
    if (!g_timing) g_phases = 0;
}

extern "C" int32_t fa_timing_read(float *ms, int32_t n) {
    if (!g_ev_made || g_phases == 0) return 0;
    if (cudaEventSynchronize(g_ev[g_phases]) != cudaSuccess) return -1;
    int m = g_phases < n ? g_phases : n;
    for (int i = 0; i < m; ++i)
        if (cudaEventElapsedTime(&ms[i], g_ev[i], g_ev[i + 1]) != cudaSuccess) return -1;
    return m;
}

extern "C" int32_t fa_kernel_launches(int64_t rows, int64_t cols, const fa_options *opts) {
    Geom g;
    if (!make_geom(rows, cols, opts, g)) return -1;
    if (rows == 0 || cols == 0) return 1;  // the status reset only
    return 8;  // status reset, pass 1, forest init, in-degree, starts, walk, final, pass 2
}

extern "C" size_t fa_workspace_size(int64_t rows, int64_t cols, const fa_options *opts) {
    Geom g;
    if (!make_geom(rows, cols, opts, g)) return 0;
    FwdWork w;
    AdjWork a;
    const size_t f = carve_forward(nullptr, 0, g, w, true);
    const size_t b = carve_adjoint(nullptr, 0, g, a);
    return f > b ? f : b;
}

extern "C" fa_status fa_accumulate(const uint8_t *codes, int64_t rows, int64_t cols,
                                   int64_t pitch_codes, const float *weights, int64_t pitch_w,
                                   const uint8_t *mask, int64_t pitch_mask, void *out,
                                   fa_out_dtype out_dtype, int64_t pitch_out, void *workspace,
                                   size_t ws_bytes, const fa_options *opts, int32_t *d_status,
                                   void *stream) {
    Geom g;
    if (!make_geom(rows, cols, opts, g)) return FA_ERR_INVALID_ARG;
    if (out_dtype != FA_OUT_U32 && out_dtype != FA_OUT_F32) return FA_ERR_INVALID_ARG;
    if (out_dtype == FA_OUT_U32 && weights) return FA_ERR_INVALID_ARG;
    if (!forward_tile_ok(g, out_dtype == FA_OUT_F32 ? 1 : 0)) return FA_ERR_INVALID_ARG;
    const bool empty = rows == 0 || cols == 0;
    if (!empty) {
        if (!codes || !out) return FA_ERR_INVALID_ARG;
        if (pitch_codes < code_row_bytes(cols, g.code_format) || pitch_out < cols) return FA_ERR_INVALID_ARG;
        if (weights && pitch_w < cols) return FA_ERR_INVALID_ARG;
        if (mask && pitch_mask < cols) return FA_ERR_INVALID_ARG;
        if (!aligned(out, 4) || (weights && !aligned(weights, 4))) return FA_ERR_INVALID_ARG;
    }
    if (d_status && !aligned(d_status, 8)) return FA_ERR_INVALID_ARG;
    if (!workspace || !aligned(workspace, 256)) return FA_ERR_WORKSPACE;
    FwdWork w;
    const size_t need = carve_forward(workspace, ws_bytes, g, w, false);
    if (ws_bytes < need) return FA_ERR_WORKSPACE;
    cudaError_t e = launch_forward(g, codes, pitch_codes, mask, pitch_mask, weights, pitch_w, out,
                                   pitch_out, out_dtype == FA_OUT_F32 ? 1 : 0, w, d_status,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}

extern "C" fa_status fa_status_read(const int32_t *d_status, const void *workspace, void *stream,
                                    int64_t *count, int64_t *first_index) {
    const void *src = d_status ? (const void *)d_status : workspace;
    if (!src) return FA_ERR_INVALID_ARG;
    int32_t host[FA_STATUS_WORDS];
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(host, src, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FA_ERR_CUDA;
    long long first;
    std::memcpy(&first, host + 2, sizeof(first));
    if (count) *count = host[1];
    if (first_index) *first_index = first == LLONG_MAX ? -1 : first;
    const int32_t f = host[0];
    if (f & FA_FLAG_BAD_CODE) return FA_ERR_BAD_CODE;
    if (f & FA_FLAG_CYCLE) return FA_ERR_CYCLE;
    if (f & FA_FLAG_NONFINITE) return FA_ERR_NONFINITE;
    if (f & FA_FLAG_TIMEOUT) return FA_ERR_TIMEOUT;
    if (f & FA_FLAG_OVERFLOW) return FA_WARN_OVERFLOW;
    return FA_OK;
}

extern "C" fa_status fa_accumulate_adjoint(const uint8_t *codes, int64_t rows, int64_t cols,
                                           int64_t pitch_codes, const uint8_t *mask,
                                           int64_t pitch_mask, const float *grad_out,
                                           int64_t pitch_g, float *grad_w, int64_t pitch_gw,
                                           void *workspace, size_t ws_bytes,
                                           const fa_options *opts, int32_t *d_status,
                                           void *stream) {
    Geom g;
    if (!make_geom(rows, cols, opts, g) || !adjoint_fits(g)) return FA_ERR_INVALID_ARG;
    const bool empty = rows == 0 || cols == 0;
    if (!empty) {
        if (!codes || !grad_out || !grad_w) return FA_ERR_INVALID_ARG;
        if (pitch_codes < code_row_bytes(cols, g.code_format) || pitch_g < cols || pitch_gw < cols)
            return FA_ERR_INVALID_ARG;
        if (mask && pitch_mask < cols) return FA_ERR_INVALID_ARG;
        if (!aligned(grad_out, 4) || !aligned(grad_w, 4)) return FA_ERR_INVALID_ARG;
    }
    if (d_status && !aligned(d_status, 8)) return FA_ERR_INVALID_ARG;
    if (!workspace || !aligned(workspace, 256)) return FA_ERR_WORKSPACE;
    AdjWork w;
    const size_t need = carve_adjoint(workspace, ws_bytes, g, w);
    if (ws_bytes < need) return FA_ERR_WORKSPACE;
    cudaError_t e = launch_adjoint(g, codes, pitch_codes, mask, pitch_mask, grad_out, pitch_g,
                                   grad_w, pitch_gw, w, d_status, (cudaStream_t)stream);
    return e == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}
