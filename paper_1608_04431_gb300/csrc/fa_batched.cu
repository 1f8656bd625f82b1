// Batched flow accumulation: many rasters, and several weight fields sharing
// one raster's codes, in one pass of the tile pipeline.
//
// Every raster becomes one entry of a device table of raster descriptors
// holding all its fields; the tiles of all rasters are numbered globally,
// raster after raster, and the persistent tile passes and the perimeter-graph
// resolve each run once over that single tile sequence.  A tile's flow
// topology (successors, dependency counts, inflow masks, the cells that start
// the walks, exits and entry links) is worked out once from its codes and
// then used for each of its fields in turn; the resolve carries every
// field's value per node over one shared pointer structure.  Perimeter-graph
// nodes are (global tile, exit rank), so flow never crosses from one raster
// to another.  A plan captures the launches of one batch in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fa_internal.h"

using namespace fa;

namespace {

bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

struct BatchLayout {
    Geom g;                         // tile shape; tiles_x = T, tiles_y = 1 for the carve
    std::vector<RasterDesc> table;  // one entry per raster, with all its fields
    int64_t T = 0;
    int64_t cells_bound = 0;
    int val_mode = 0;
    size_t fwd_bytes = 0, table_off = 0, total = 0;
};

// Validates a batch and lays out its descriptor table and workspace.
fa_status plan_batch(const fa_raster *rasters, int32_t n, int32_t k, const fa_options *opts,
                     BatchLayout &L) {
    if (n < 0 || k < 0 || k > FA_MAX_FIELDS || (n > 0 && !rasters)) return FA_ERR_INVALID_ARG;
    if (!make_geom(1, 1, opts, L.g)) return FA_ERR_INVALID_ARG;
    L.val_mode = k > 0 ? 1 : 0;
    if (!forward_tile_ok(L.g, L.val_mode)) return FA_ERR_INVALID_ARG;
    const int nf = k > 0 ? k : 1;
    L.table.clear();
    L.T = 0;
    L.cells_bound = 0;
    for (int i = 0; i < n; ++i) {
        const fa_raster &r = rasters[i];
        if (r.rows < 0 || r.cols < 0) return FA_ERR_INVALID_ARG;
        const bool empty = r.rows == 0 || r.cols == 0;
        if (!empty) {
            if (!r.codes || r.pitch_codes < code_row_bytes(r.cols, L.g.code_format) || r.pitch_out < r.cols)
                return FA_ERR_INVALID_ARG;
            if (r.mask && r.pitch_mask < r.cols) return FA_ERR_INVALID_ARG;
            if (k > 0 && r.pitch_w < r.cols) return FA_ERR_INVALID_ARG;
        }
        Geom gi;
        if (!make_geom(r.rows, r.cols, opts, gi)) return FA_ERR_INVALID_ARG;
        for (int f = 0; f < nf && !empty; ++f) {
            if (!r.out[f] || !aligned_to(r.out[f], 4)) return FA_ERR_INVALID_ARG;
            if (k > 0 && (!r.weights[f] || !aligned_to(r.weights[f], 4))) return FA_ERR_INVALID_ARG;
        }
        if (empty) continue;
        RasterDesc d;
        std::memset(&d, 0, sizeof(d));
        d.codes = r.codes;
        d.pc = r.pitch_codes;
        d.mask = r.mask;
        d.pm = r.pitch_mask;
        for (int f = 0; f < nf; ++f) {
            d.w[f] = k > 0 ? r.weights[f] : nullptr;
            d.out[f] = r.out[f];
        }
        d.pw = r.pitch_w;
        d.po = r.pitch_out;
        d.rows = r.rows;
        d.cols = r.cols;
        d.tiles_x = gi.tiles_x;
        d.tiles_y = gi.tiles_y;
        d.tile_base = L.T;
        L.table.push_back(d);
        L.T += gi.tiles();
        L.cells_bound = std::max<int64_t>(L.cells_bound, r.rows * r.cols);
    }
    if ((double)L.T * L.g.pmax >= 4.0e9) return FA_ERR_INVALID_ARG;
    L.g.tiles_x = (int)std::max<int64_t>(L.T, 1);
    L.g.tiles_y = 1;
    L.g.nf = nf;
    FwdWork w;
    L.fwd_bytes = carve_forward(nullptr, 0, L.g, w, true);
    L.table_off = (L.fwd_bytes + 255) & ~size_t(255);
    L.total = L.table_off + L.table.size() * sizeof(RasterDesc) + 256;
    return FA_OK;
}

fa_status enqueue_batch(const BatchLayout &L, void *workspace, size_t ws_bytes,
                        int32_t *d_status, cudaStream_t s, bool upload) {
    if (!workspace || !aligned_to(workspace, 256)) return FA_ERR_WORKSPACE;
    if (ws_bytes < L.total) return FA_ERR_WORKSPACE;
    if (d_status && !aligned_to(d_status, 8)) return FA_ERR_INVALID_ARG;
    FwdWork w;
    carve_forward(workspace, ws_bytes, L.g, w, false);
    RasterDesc *d_tab = reinterpret_cast<RasterDesc *>((uint8_t *)workspace + L.table_off);
    if (upload && !L.table.empty()) {
        if (cudaMemcpyAsync(d_tab, L.table.data(), L.table.size() * sizeof(RasterDesc),
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return FA_ERR_CUDA;
    }
    const cudaError_t e = launch_forward_batched(L.g, d_tab, (int)L.table.size(), L.T,
                                                 L.cells_bound, L.val_mode, w, d_status, s);
    return e == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}

}  // namespace

struct fa_plan_s {
    BatchLayout layout;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" size_t fa_batched_workspace_size(const fa_raster *rasters, int32_t n_rasters,
                                            int32_t n_fields, const fa_options *opts) {
    BatchLayout L;
    if (plan_batch(rasters, n_rasters, n_fields, opts, L) != FA_OK) return 0;
    return L.total;
}

extern "C" fa_status fa_accumulate_batched(const fa_raster *rasters, int32_t n_rasters,
                                           int32_t n_fields, void *workspace, size_t ws_bytes,
                                           const fa_options *opts, int32_t *d_status,
                                           void *stream) {
    BatchLayout L;
    const fa_status st = plan_batch(rasters, n_rasters, n_fields, opts, L);
    if (st != FA_OK) return st;
    return enqueue_batch(L, workspace, ws_bytes, d_status, (cudaStream_t)stream, true);
}

extern "C" fa_status fa_batched_plan_create(const fa_raster *rasters, int32_t n_rasters,
                                            int32_t n_fields, void *workspace, size_t ws_bytes,
                                            const fa_options *opts, int32_t *d_status,
                                            void *stream, fa_plan *plan) {
    if (!plan) return FA_ERR_INVALID_ARG;
    *plan = nullptr;
    fa_plan p = new fa_plan_s;
    fa_status st = plan_batch(rasters, n_rasters, n_fields, opts, p->layout);
    if (st != FA_OK) {
        delete p;
        return st;
    }
    if (!workspace || !aligned_to(workspace, 256) || ws_bytes < p->layout.total) {
        delete p;
        return FA_ERR_WORKSPACE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the descriptor table is uploaded once; the graph reads it in place
    RasterDesc *d_tab = reinterpret_cast<RasterDesc *>((uint8_t *)workspace + p->layout.table_off);
    if (!p->layout.table.empty() &&
        (cudaMemcpyAsync(d_tab, p->layout.table.data(),
                         p->layout.table.size() * sizeof(RasterDesc), cudaMemcpyHostToDevice,
                         s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
        delete p;
        return FA_ERR_CUDA;
    }
    if (prepare_forward(p->layout.g, p->layout.val_mode) != cudaSuccess) {
        delete p;
        return FA_ERR_CUDA;
    }
    // capture on a private stream so the caller's stream is never in capture mode
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return FA_ERR_CUDA;
    }
    const bool timing = timing_swap(false);  // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_batch(p->layout, workspace, ws_bytes, d_status, cs, false);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        p->graph = g;
        if (st == FA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
    }
    timing_swap(timing);
    cudaStreamDestroy(cs);
    if (st != FA_OK || e != cudaSuccess) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return st != FA_OK ? st : FA_ERR_CUDA;
    }
    *plan = p;
    return FA_OK;
}

extern "C" fa_status fa_plan_launch(fa_plan plan, void *stream) {
    if (!plan || !plan->exec) return FA_ERR_INVALID_ARG;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? FA_OK : FA_ERR_CUDA;
}

extern "C" void fa_plan_destroy(fa_plan plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
}
