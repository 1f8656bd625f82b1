// Tile-shape autotuner: times the forward pipeline on the caller's own data
// for a fixed list of candidate tile shapes and returns the fastest.
//
// The tile shape trades the work inside a tile (jump rounds grow with the
// tile's longest path, shared memory limits the tiles resident per SM)
// against the perimeter graph (its node count falls as tiles grow).  Which
// shape wins depends on the raster (drainage lengths, size) and the
// weighting, so it is measured rather than modelled.  Every candidate gives
// the same integer results (tile-shape invariance), so tuning never changes
// an answer beyond the rounding of float sums.
#include <algorithm>

#include "fa_internal.h"

namespace {

struct Shape {
    int th, tw;
};
// 64 x 64 first: the default, and the winner on ties
const Shape kCandidates[] = {{64, 64},  {64, 128}, {128, 64}, {96, 64},  {64, 96}, {32, 128},
                             {128, 32}, {48, 64},  {32, 64},  {64, 32},  {32, 256}, {48, 128}};
constexpr int kReps = 3;  // timed runs per candidate after one untimed run

fa_options with_shape(const fa_options *base, Shape s) {
    fa_options o = base ? *base : fa_options{0, 0, 0, 0};
    o.tile_h = s.th;
    o.tile_w = s.tw;
    return o;
}

bool shape_usable(int64_t rows, int64_t cols, const fa_options &o, int valm) {
    fa::Geom g;
    return fa::make_geom(rows, cols, &o, g) && fa::forward_tile_ok(g, valm);
}

// Times fn() on `s`: one untimed call, then the fastest of kReps timed calls
// (each between its own pair of events); negative on error.
template <class F>
float time_on(cudaStream_t s, F fn) {
    if (fn() != FA_OK) return -1.0f;
    cudaEvent_t ev[kReps + 1];
    int made = 0;
    for (; made <= kReps; ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
    float best = -1.0f;
    bool ok = made == kReps + 1 && cudaEventRecord(ev[0], s) == cudaSuccess;
    for (int r = 0; ok && r < kReps; ++r)
        ok = fn() == FA_OK && cudaEventRecord(ev[r + 1], s) == cudaSuccess;
    ok = ok && cudaEventSynchronize(ev[kReps]) == cudaSuccess;
    for (int r = 0; ok && r < kReps; ++r) {
        float ms = 0.0f;
        ok = cudaEventElapsedTime(&ms, ev[r], ev[r + 1]) == cudaSuccess;
        if (ok && (best < 0.0f || ms < best)) best = ms;
    }
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    return ok ? best : -1.0f;
}

}  // namespace

extern "C" size_t fa_autotune_workspace_size(int64_t rows, int64_t cols, const fa_options *opts) {
    size_t need = 0;
    for (const Shape &s : kCandidates) {
        const fa_options o = with_shape(opts, s);
        if (shape_usable(rows, cols, o, 0)) need = std::max(need, fa_workspace_size(rows, cols, &o));
    }
    return need;
}

extern "C" fa_status fa_autotune(const uint8_t *codes, int64_t rows, int64_t cols,
                                 int64_t pitch_codes, const float *weights, int64_t pitch_w,
                                 const uint8_t *mask, int64_t pitch_mask, void *out,
                                 fa_out_dtype out_dtype, int64_t pitch_out, void *workspace,
                                 size_t ws_bytes, const fa_options *opts, void *stream,
                                 fa_options *best) {
    if (!best) return FA_ERR_INVALID_ARG;
    const int valm = out_dtype == FA_OUT_F32 ? 1 : 0;
    cudaStream_t s = (cudaStream_t)stream;
    float best_ms = -1.0f;
    fa_options chosen{};
    fa_status first_err = FA_ERR_INVALID_ARG;
    const bool timing = fa::timing_swap(false);  // no phase events while tuning
    for (const Shape &sh : kCandidates) {
        const fa_options o = with_shape(opts, sh);
        if (!shape_usable(rows, cols, o, valm)) continue;
        if (fa_workspace_size(rows, cols, &o) > ws_bytes) {
            first_err = FA_ERR_WORKSPACE;
            continue;
        }
        fa_status st = FA_OK;
        const float ms = time_on(s, [&]() {
            st = fa_accumulate(codes, rows, cols, pitch_codes, weights, pitch_w, mask, pitch_mask,
                               out, out_dtype, pitch_out, workspace, ws_bytes, &o, nullptr, stream);
            return st;
        });
        if (ms < 0.0f) {
            fa::timing_swap(timing);
            return st != FA_OK ? st : FA_ERR_CUDA;  // the arguments are wrong for every shape
        }
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            chosen = o;
        }
    }
    fa::timing_swap(timing);
    if (best_ms < 0.0f) return first_err;
    // leave the chosen shape's result in `out`
    const fa_status st = fa_accumulate(codes, rows, cols, pitch_codes, weights, pitch_w, mask,
                                       pitch_mask, out, out_dtype, pitch_out, workspace, ws_bytes,
                                       &chosen, nullptr, stream);
    if (st != FA_OK) return st;
    *best = chosen;
    return FA_OK;
}

extern "C" size_t fa_autotune_batched_workspace_size(const fa_raster *rasters, int32_t n_rasters,
                                                     int32_t n_fields, const fa_options *opts) {
    size_t need = 0;
    for (const Shape &s : kCandidates) {
        const fa_options o = with_shape(opts, s);
        need = std::max(need, fa_batched_workspace_size(rasters, n_rasters, n_fields, &o));
    }
    return need;
}

extern "C" fa_status fa_autotune_batched(const fa_raster *rasters, int32_t n_rasters,
                                         int32_t n_fields, void *workspace, size_t ws_bytes,
                                         const fa_options *opts, void *stream, fa_options *best) {
    if (!best) return FA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float best_ms = -1.0f;
    fa_options chosen{};
    fa_status first_err = FA_ERR_INVALID_ARG;
    const bool timing = fa::timing_swap(false);
    for (const Shape &sh : kCandidates) {
        const fa_options o = with_shape(opts, sh);
        const size_t need = fa_batched_workspace_size(rasters, n_rasters, n_fields, &o);
        if (need == 0) continue;  // shape not usable for this batch
        if (need > ws_bytes) {
            first_err = FA_ERR_WORKSPACE;
            continue;
        }
        fa_status st = FA_OK;
        const float ms = time_on(s, [&]() {
            st = fa_accumulate_batched(rasters, n_rasters, n_fields, workspace, ws_bytes, &o,
                                       nullptr, stream);
            return st;
        });
        if (ms < 0.0f) {
            fa::timing_swap(timing);
            return st != FA_OK ? st : FA_ERR_CUDA;
        }
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            chosen = o;
        }
    }
    fa::timing_swap(timing);
    if (best_ms < 0.0f) return first_err;
    const fa_status st = fa_accumulate_batched(rasters, n_rasters, n_fields, workspace, ws_bytes,
                                               &chosen, nullptr, stream);
    if (st != FA_OK) return st;
    *best = chosen;
    return FA_OK;
}
