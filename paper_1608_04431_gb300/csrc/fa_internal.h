// Host-side declarations shared by the translation units of libfa.so.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/fa.h"

namespace fa {

// Geometry of the tile decomposition of one raster (Section 3: the raster is
// subdivided into equal rectangular tiles; the last row/column may be ragged).
struct Geom {
    int64_t rows, cols;
    int th, tw;          // nominal tile shape
    int tiles_x, tiles_y;
    int pmax;            // per-tile slot capacity: 2*th + 2*tw >= perimeter cells
    int flags;           // FA_OPT_* from fa_options
    int code_format;     // FA_CODES_BYTE or FA_CODES_NIBBLE
    int nf = 1;          // weight fields carried per raster (1 for counts)
    int64_t tiles() const { return (int64_t)tiles_x * tiles_y; }
};

// Bytes a row of codes needs in a code format (the smallest valid pitch).
inline int64_t code_row_bytes(int64_t cols, int code_format) {
    return code_format == FA_CODES_NIBBLE ? (cols + 1) / 2 : cols;
}

bool make_geom(int64_t rows, int64_t cols, const fa_options *opts, Geom &g);

// One raster as the kernels see it (for batches, a device-resident table).
// All rasters of a batch share the tile shape and the number of weight fields
// (w[0 .. nf-1], out[0 .. nf-1]; counts use w[0] = NULL and out[0]); their
// tiles are numbered globally, raster after raster, starting at tile_base.
struct RasterDesc {
    const uint8_t *codes;
    int64_t pc;
    const uint8_t *mask;
    int64_t pm;
    const float *w[FA_MAX_FIELDS];
    int64_t pw;
    void *out[FA_MAX_FIELDS];
    int64_t po;
    int64_t rows, cols;
    int32_t tiles_x, tiles_y;
    int64_t tile_base;
};
// whether the forward tile kernel supports this tile shape (shared memory and
// 16-bit cell indices); valm 0 = uint32 counts, 1 = float32
bool forward_tile_ok(const Geom &g, int valm);

// Workspace carving: every region 256-byte aligned.
struct Carver {
    uintptr_t base, cur, end;
    explicit Carver(void *p, size_t n) : base((uintptr_t)p), cur((uintptr_t)p), end((uintptr_t)p + n) {}
    template <class T>
    T *take(size_t count) {
        cur = (cur + 255) & ~uintptr_t(255);
        T *p = (T *)cur;
        cur += count * sizeof(T);
        return p;
    }
    size_t used() const { return cur - base; }
    bool fits() const { return cur <= end; }
};

// Forward workspace regions (device pointers).  Perimeter-graph nodes are
// (tile, exit rank) = tile * pmax + rank; per node and weight field f the
// values sit at node * nf + f.
struct FwdWork {
    void *status;          // StatusBlock (16 bytes)
    uint32_t *misc;        // [0] max |w| bits, [1] nodes finished by the resolve walks
    uint32_t *nexit;       // [T] exits per tile
    uint16_t *link;        // [T*pmax] perimeter slot -> exit rank its path reaches, 0xFFFF = none
    uint32_t *node_dst;    // [T*pmax] exit rank -> global slot id of its target cell
    double *node_val;      // [T*pmax*nf] exit rank -> tile-local accumulation A_loc
    void *x;               // [T*pmax*nf] u128 forest values (G after resolve)
    uint32_t *J0, *J1;     // [T*pmax] successor node, predecessors still to come
    unsigned long long *infl;  // [T*pmax] counts: flow arriving at each perimeter slot from outside
    int kmax;              // rounds of a pointer-jumping solve over T*pmax nodes (absorption)
};

size_t carve_forward(void *ws, size_t bytes, const Geom &g, FwdWork &w, bool dry);

// Solves a forest of exit nodes with integer (uint64) values by the
// last-arriver walks of the tile resolve: `groups` groups of up to `pmax`
// nodes (node id = group * pmax + rank, nexit[group] ranks in use); node
// `id` flows to the node linked from slot node_dst[id] (link[slot] = rank in
// that slot's group, 0xFFFF = the path ends), with value node_val[id] (an
// exact integer in a double).  x receives the solved values G; infl, if not
// NULL, receives per slot the sum of G over the nodes whose node_dst is that
// slot (the flow entering it, Section 3.2's in(p)); J0 and J1 are scratch of
// groups * pmax words each, misc[0..1] two counters, and a node on a cycle is
// reported in `status`.
cudaError_t resolve_exit_forest_u64(int64_t groups, int pmax, const uint32_t *nexit,
                                    const uint16_t *link, const uint32_t *node_dst,
                                    const double *node_val, unsigned long long *x,
                                    unsigned long long *infl, uint32_t *J0, uint32_t *J1,
                                    uint32_t *misc, void *status, cudaStream_t s);

// Phase timing: records an event on `s` at phase boundary `i` (0..kMaxPhase)
// when enabled; no-op otherwise.
constexpr int kMaxPhase = 8;
void timing_mark(int i, cudaStream_t s);
void timing_set_count(int n);
// on this host thread only: allows (true) or suppresses (false) phase
// events; returns the previous setting of this thread
bool timing_swap(bool on);

// Configures the forward kernels (shared-memory limits, device queries) so
// that a later stream capture makes no first-use attribute calls.
cudaError_t prepare_forward(const Geom &g, int val_mode);

// Launch the forward pipeline over a batch described by a device table of
// `nr` rasters (tiles numbered globally, `T` in all; every raster's weights
// NULL and uint32 outputs when val_mode is 0; g.nf fields per raster); the
// workspace is carved for T tiles.  cells_bound bounds the cell count of any
// raster (fixed-point scale).
cudaError_t launch_forward_batched(const Geom &g, const RasterDesc *d_tab, int nr, int64_t T,
                                   int64_t cells_bound, int val_mode, const FwdWork &ws,
                                   void *status, cudaStream_t s);

// Additions to a counts pipeline for rasters that are blocks of a larger one
// (the out-of-core form), all indexed tile * pmax + slot: inj is flow entering
// the block at that perimeter slot from outside it (added along the slot's
// path in the tile), injx the same flow at the slot of the exit cell that
// path reaches (added to that exit's value before the resolve), or NULL;
// off64, if set, receives the flow that enters each tile (from other tiles or
// from outside the block) as uint64 offsets per cell (pitch of the output),
// instead of adding it to the uint32 output, which then holds only A_loc.
struct PipeHooks {
    const unsigned long long *inj, *injx;
    unsigned long long *off64;
};
cudaError_t launch_forward_hooked(const Geom &g, const uint8_t *codes, int64_t pc, void *out,
                                  int64_t po, const FwdWork &ws, void *status, const PipeHooks &hooks,
                                  cudaStream_t s);

// Launch the whole forward pipeline on `stream`.  val_mode 0: uint32 counts
// (weights must be NULL); 1: float32 output (weights or unit).
cudaError_t launch_forward(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                           int64_t pm, const float *w, int64_t pw, void *out, int64_t po,
                           int val_mode, const FwdWork &ws, void *status, cudaStream_t s);

// Adjoint workspace regions (device pointers); FF values stored as 8 bytes.
struct AdjWork {
    void *status;
    uint32_t *misc;       // [1 + k] exit nodes still jumping after round k
    uint32_t *nexit;      // [T]
    uint16_t *link;       // [T*pmax] perimeter slot -> exit rank, 0xFFFF = terminates
    uint32_t *node_dst;   // [T*pmax] exit rank -> global slot id of its target
    uint64_t *lam_slot;   // [T*pmax] in-tile path sums on perimeter slots
    uint64_t *v0, *v1;    // [T*pmax] forest jump values
    uint64_t *outv;       // [T*pmax] out(e) per exit
    uint32_t *J0, *J1;    // [T*pmax] forest jump pointers
    int kmax;
};

size_t carve_adjoint(void *ws, size_t bytes, const Geom &g, AdjWork &w);
bool adjoint_fits(const Geom &g);
cudaError_t launch_adjoint(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                           int64_t pm, const float *gin, int64_t pg, float *out, int64_t po,
                           const AdjWork &ws, void *status, cudaStream_t s);

}  // namespace fa
