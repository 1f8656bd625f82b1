/*
 * fa.h -- C ABI of the GB300 (sm_103a) D8 flow-accumulation library (libfa.so).
 *
 * Operation (Eq. 1 with alpha restricted to {0,1}, Section 2): for every valid
 * cell p of a raster of single-direction (D8) flow codes,
 *     A(p) = w(p) + sum of A(n) over the neighbours n whose one downstream cell is p,
 * i.e. the count (w = 1) or weighted sum of all cells upslope of p, p included.
 * The library computes it with the paper's tile decomposition (Section 3):
 * a per-tile solve (Algorithm 1) that also links each perimeter cell to the
 * tile exit its flow path reaches (Algorithm 2), a global solve over those
 * perimeter links (Section 3.2), and a finalising per-tile pass (Algorithm 3,
 * Section 3.3) that adds the flow entering each tile from other tiles.  For
 * counts the first pass leaves each tile's own accumulation in the output and
 * the finalising pass adds the entering flow along the in-tile path of each
 * entry cell (the codes are read twice, the output written once and updated
 * on those paths); for float sums the finalising pass solves each tile again
 * with the entering flow added at its entry cells (the EVICT strategy of
 * Section 3: codes and weights read twice, the output written once).
 *
 * Raster conventions (all entry points):
 *  - Row-major, row 0 = north; every raster argument has its own row pitch in
 *    ELEMENTS (>= cols).  All raster pointers are DEVICE pointers owned by the
 *    caller (except for the out-of-core and shard entry points, whose rasters
 *    and records are HOST memory); the library never allocates device memory
 *    on these paths: all scratch comes from the caller's workspace (size from
 *    *_workspace_size), which must be 256-byte aligned.
 *  - Codes, one byte per cell: 0 = NoData, 1..8 = E, NE, N, NW, W, SW, S, SE
 *    (offsets (0,+1) (-1,+1) (-1,0) (-1,-1) (0,-1) (+1,-1) (+1,0) (+1,+1)),
 *    9 = NoFlow.  Codes 10..255 are invalid: reported as FA_ERR_BAD_CODE in the
 *    device status and treated as NoData.  The paper fixes one byte and ten
 *    values per code (Section 4, Data Types) but no numbering; this is ours.
 *  - Packed codes (fa_options.code_format = FA_CODES_NIBBLE): the same values
 *    in four bits, two cells per byte.  Cell c of row r is in byte
 *    r * pitch_codes + c / 2, low nibble for even c, high nibble for odd c;
 *    pitch_codes counts BYTES and must be >= (cols + 1) / 2.  Nibbles 10..15
 *    are invalid as above.  Section 4 notes that ten values fit in half a
 *    byte; this halves the code traffic (4.5 B/cell for counts instead of 5).
 *  - Optional NoData mask (uint8, nonzero = NoData); a cell is NoData if its
 *    code is 0 or invalid or its mask byte is nonzero.
 *  - A cell has no downstream cell (its flow leaves the system) when it is
 *    NoFlow, or its target is off the grid or NoData (Algorithm 1 skips such
 *    targets; Algorithm 2 treats outside-of-data cells as NoData).  NoFlow
 *    cells keep what they receive.  NoData cells get output 0.
 *
 * Asynchrony and errors:
 *  - Every compute entry point enqueues work on `stream` (a cudaStream_t; NULL
 *    = legacy default stream) and returns without synchronising.
 *  - Host-detectable errors (NULL pointers, bad sizes or pitches, dtype
 *    mismatch, workspace too small or misaligned) return synchronously with
 *    nothing enqueued.
 *  - Conditions found on the device (invalid codes, cycles, uint32 overflow,
 *    non-finite weights, a bounded wait that ran out) are recorded in a device
 *    status block of FA_STATUS_WORDS int32 words (8-byte aligned): d_status if
 *    non-NULL, else a block inside the workspace.  fa_status_read() copies it
 *    back.  The library never traps or asserts on the device.
 *  - Results are bitwise reproducible run to run for a fixed tile shape and
 *    input (no atomics-dependent floating-point ordering).
 */
#ifndef FA_H
#define FA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FA_OK = 0,
    FA_WARN_OVERFLOW = 1,     /* a uint32 count wrapped: outputs are mod 2^32 */
    FA_ERR_INVALID_ARG = -1,  /* host-side argument check failed */
    FA_ERR_BAD_CODE = -2,     /* a code in 10..255 was found (treated as NoData) */
    FA_ERR_CYCLE = -3,        /* the flow graph has a cycle; cells on it are unspecified */
    FA_ERR_WORKSPACE = -4,    /* workspace NULL, too small or misaligned */
    FA_ERR_CUDA = -5,         /* a CUDA runtime call failed */
    FA_ERR_TIMEOUT = -6,      /* a bounded device wait ran out */
    FA_ERR_NONFINITE = -7,    /* a weight or gradient was NaN or infinite */
    FA_ERR_TOO_LARGE = -8     /* fa_accumulate_noalloc: raster needs more than its fixed scratch */
} fa_status;

typedef enum { FA_OUT_U32 = 0, FA_OUT_F32 = 1 } fa_out_dtype;

/* Device status block: word 0 = bitmask of FA_FLAG_*, word 1 = number of
 * offending cells or perimeter-graph nodes, words 2-3 = smallest offending cell
 * index r*cols + c as a little-endian int64 (INT64_MAX while none was found;
 * fa_status_read reports that as -1).  Reset at the start of every call. */
#define FA_STATUS_WORDS 4
#define FA_FLAG_BAD_CODE 1
#define FA_FLAG_CYCLE 2
#define FA_FLAG_OVERFLOW 4
#define FA_FLAG_TIMEOUT 8
#define FA_FLAG_NONFINITE 16

/* Tile shape: 0 = library default (64 x 64).  For fa_accumulate, batches,
 * fa_accumulate_noalloc and the out-of-core blocks: 1 <= tile_h, tile_w,
 * tile_h * tile_w <= 8192 and (tile_h + 2) * (tile_w + 2) <= 16383 (the words
 * of a tile and its one-cell ring are numbered in 14 bits); the tile's shared
 * memory must also fit, which rules out only very narrow, tall tiles (the
 * staged codes take (tile_h + 2) * (tile_w + 32 rounded up to a multiple of
 * 16) bytes).  The adjoint and absorption forms state their own limits.
 * Other shapes return FA_ERR_INVALID_ARG.  Results do not depend on the tile
 * shape, except for the rounding of floating-point sums.
 * flags: FA_OPT_NO_TMA disables staging code tiles into shared memory with the
 * Tensor Memory Accelerator (used for single rasters when they allow it:
 * 16-byte aligned codes and pitch, tile width a multiple of 16 (32 for packed
 * codes), no mask raster); results are identical either way.
 * code_format: FA_CODES_BYTE (0, one byte per cell) or FA_CODES_NIBBLE (1, two
 * cells per byte; see the raster conventions above).  It applies to every
 * codes argument of the call (fa_accumulate, fa_accumulate_noalloc,
 * fa_accumulate_adjoint, fa_autotune and every raster of a batch); other
 * values are FA_ERR_INVALID_ARG. */
#define FA_OPT_NO_TMA 1
#define FA_CODES_BYTE 0
#define FA_CODES_NIBBLE 1
typedef struct {
    int32_t tile_h, tile_w;
    int32_t flags, code_format;
} fa_options;

/* Library version as major*10000 + minor*100 + patch. */
int32_t fa_version(void);

/* Number of kernel launches one fa_accumulate call enqueues for this shape
 * (useful for graph capture and launch accounting); -1 if arguments are
 * invalid. */
int32_t fa_kernel_launches(int64_t rows, int64_t cols, const fa_options *opts);

/* Workspace bytes that fa_accumulate and fa_accumulate_adjoint need for a
 * rows x cols raster (any output dtype and weighting).  Returns 0 if the
 * arguments are invalid. */
size_t fa_workspace_size(int64_t rows, int64_t cols, const fa_options *opts);

/*
 * Flow accumulation of one raster (Eq. 1; Sections 3.1-3.3, Algorithms 1-3).
 *   codes    [rows x pitch_codes] uint8 D8 codes (device).
 *   weights  [rows x pitch_w] float32 per-cell weights w(p) (device), or NULL
 *            for unit weights (upslope cell counts).
 *   mask     [rows x pitch_mask] uint8 NoData mask (device) or NULL.
 *   out      [rows x pitch_out] uint32 (FA_OUT_U32, counts mod 2^32; requires
 *            weights == NULL) or float32 (FA_OUT_F32; sums kept as
 *            compensated float pairs, about 48 bits, added in a fixed order
 *            inside tiles, and in 128-bit fixed point across tiles, then
 *            rounded once to float32).
 *   workspace, ws_bytes: caller-owned device scratch, >= fa_workspace_size().
 *   d_status: device int32[FA_STATUS_WORDS] or NULL (see above).
 * rows or cols == 0 is valid and enqueues nothing but the status reset.
 */
fa_status fa_accumulate(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch_codes,
                        const float *weights, int64_t pitch_w, const uint8_t *mask,
                        int64_t pitch_mask, void *out, fa_out_dtype out_dtype,
                        int64_t pitch_out, void *workspace, size_t ws_bytes,
                        const fa_options *opts, int32_t *d_status, void *stream);

/*
 * Batches.  Many rasters, each with its own shape, and up to FA_MAX_FIELDS
 * weight fields sharing one raster's codes, accumulated in one pass of the
 * tile pipeline (Sections 3.1-3.3): the tiles of all rasters form one tile
 * sequence for the persistent tile passes, each tile's flow topology is
 * worked out once from its codes and used for every field in turn, and one
 * perimeter-graph resolve carries all fields (its nodes are (tile, exit), so
 * no flow crosses from one raster to another).  Each result equals
 * fa_accumulate on that raster and field with the same tile shape: bit for
 * bit for uint32 counts; float32 sums may differ in the last place, since the
 * perimeter graph's fixed-point scale is set by the largest raster and
 * weight of the batch.  Every raster uses opts' tile shape; batches
 * never stage codes by TMA.
 *
 * Errors (returned before anything is enqueued): FA_ERR_INVALID_ARG for
 * n_rasters < 0, n_fields outside 0..FA_MAX_FIELDS, a bad tile shape, and, for
 * a non-empty raster, NULL codes, NULL or 4-byte-misaligned out[k] or
 * weights[k] (k < max(n_fields, 1)), or a pitch below cols (below (cols + 1)
 * / 2 for packed codes); FA_ERR_WORKSPACE
 * for a NULL, not 256-byte-aligned or too small workspace; FA_ERR_CUDA if a
 * launch or copy fails.  Rasters with rows == 0 or cols == 0 are skipped.
 * Device-side findings (bad codes, cycles, non-finite weights) go to the
 * status block as for fa_accumulate; first_index is then a cell index within
 * the raster where it was found, not a batch position.
 */
#define FA_MAX_FIELDS 16
typedef struct {
    const uint8_t *codes;               /* device, row-major [rows x pitch_codes] bytes */
    int64_t rows, cols, pitch_codes;
    const uint8_t *mask;                /* device NoData mask [rows x pitch_mask], or NULL */
    int64_t pitch_mask;
    const float *weights[FA_MAX_FIELDS];/* device float32 [rows x pitch_w] (first n_fields) */
    int64_t pitch_w;
    void *out[FA_MAX_FIELDS];           /* device outputs [rows x pitch_out] (first max(n_fields,1)) */
    int64_t pitch_out;
} fa_raster;

/* Workspace bytes for a batch (0 if it is invalid).  n_fields == 0 means unit
 * weights: uint32 counts into out[0]; 1..FA_MAX_FIELDS means float32 sums,
 * weights[k] -> out[k] (float32). */
size_t fa_batched_workspace_size(const fa_raster *rasters, int32_t n_rasters, int32_t n_fields,
                                 const fa_options *opts);

/* Accumulate a batch, asynchronously on `stream`.  `rasters` is a host array
 * of n_rasters descriptors; the descriptor table is copied into the workspace
 * on `stream`, so the host array may be reused once the call returns.  The
 * caller owns every buffer; the library keeps nothing after the call. */
fa_status fa_accumulate_batched(const fa_raster *rasters, int32_t n_rasters, int32_t n_fields,
                                void *workspace, size_t ws_bytes, const fa_options *opts,
                                int32_t *d_status, void *stream);

/* A batch captured once in a CUDA graph and replayed by fa_plan_launch: the
 * same launches as fa_accumulate_batched, without their host-side cost.  The
 * plan reads the batch's buffers at replay time (new weights written in place
 * give new results) and keeps using `workspace`, which holds its descriptor
 * table: keep all of them allocated at the same addresses until
 * fa_plan_destroy, and do not overlap two replays of one plan.  Creation
 * uploads the table and synchronises `stream` once; capture runs on a private
 * stream, so `stream` is never left in capture mode.  Errors as for
 * fa_accumulate_batched; *plan is NULL on failure (FA_ERR_INVALID_ARG if plan
 * itself is NULL).  fa_plan_launch returns FA_ERR_INVALID_ARG for a NULL plan
 * and FA_ERR_CUDA if the graph launch fails; fa_plan_destroy(NULL) is a no-op. */
typedef struct fa_plan_s *fa_plan;
fa_status fa_batched_plan_create(const fa_raster *rasters, int32_t n_rasters, int32_t n_fields,
                                 void *workspace, size_t ws_bytes, const fa_options *opts,
                                 int32_t *d_status, void *stream, fa_plan *plan);
fa_status fa_plan_launch(fa_plan plan, void *stream);
void fa_plan_destroy(fa_plan plan);

/*
 * D8 flow codes from elevations: the direction step that runs before the
 * accumulation (Section 2: a non-divergent metric sends a cell's flow to a
 * single neighbour; D8 follows the steepest descent; flats are routed towards
 * lower terrain only; Fig. 1 treats this step as a separate algorithm).
 *   dem      [rows x pitch_dem] float32 elevations (device, 4-byte aligned).
 *   nodata   [rows x pitch_nodata] uint8 (device) or NULL: nonzero = NoData.
 *   codes    [rows x pitch_codes] uint8 output (device), in this file's code
 *            encoding.
 * Per cell: NoData gets 0; a border cell drains off the grid (N, S, W or E,
 * diagonal at the corners); otherwise the valid neighbour with the largest
 * positive slope (drop, times 1/sqrt 2 for diagonals; ties to the first of
 * E, NE, N, NW, W, SW, S, SE); with no positive slope, the first NoData
 * neighbour in that order, else NoFlow.  Slopes are decided in float32 with
 * correctly rounded operations (no fused multiply-add), so results are exact
 * and platform-independent.  NaN elevations are not NoData: use the mask.
 * Asynchronous on `stream`; rows or cols == 0 enqueue nothing.  Returns
 * FA_ERR_INVALID_ARG for negative sizes, NULL buffers, pitches below cols,
 * a misaligned dem or more than 2,097,120 rows, FA_ERR_CUDA if the launch
 * fails.
 */
fa_status fa_d8_codes(const float *dem, int64_t rows, int64_t cols, int64_t pitch_dem,
                      const uint8_t *nodata, int64_t pitch_nodata, uint8_t *codes,
                      int64_t pitch_codes, void *stream);

/*
 * Code translation and packing.  Rasters coded in another scheme (for example
 * one bit per direction, 1 = E, 2 = SE, 4 = S, ..., 128 = NE) are brought to
 * this file's codes through a table, and codes can be packed two per byte for
 * FA_CODES_NIBBLE (Section 4: ten values fit in half a byte).
 *   src        [rows x pitch_src] uint8 (device), one byte per cell.
 *   table      HOST array of 256 bytes: cell value v becomes table[v]; NULL
 *              keeps v.  The table is copied into the launch, so it may be
 *              reused as soon as the call returns.
 *   dst        device output in dst_format: FA_CODES_BYTE writes
 *              [rows x pitch_dst] bytes (pitch_dst >= cols); FA_CODES_NIBBLE
 *              writes [rows x pitch_dst] bytes of packed codes (pitch_dst >=
 *              (cols + 1) / 2), where a translated value above 15 is written
 *              as 15 (invalid either way) and the unused high nibble of an
 *              odd-width row's last byte is 0.
 * src and dst must not overlap.  Asynchronous on `stream`; rows or cols == 0
 * enqueue nothing.  Returns FA_ERR_INVALID_ARG for negative sizes, NULL
 * buffers, short pitches or an unknown dst_format, FA_ERR_CUDA if the launch
 * fails.
 */
fa_status fa_recode(const uint8_t *src, int64_t rows, int64_t cols, int64_t pitch_src,
                    const uint8_t *table, uint8_t *dst, int64_t pitch_dst, int32_t dst_format,
                    void *stream);

/*
 * Tile-shape autotuner.  The tile shape trades work inside a tile against the
 * size of the perimeter graph (Section 3.2 grows with the number of tiles),
 * and the best trade depends on the raster, so it is measured: fa_autotune
 * runs fa_accumulate on the caller's own inputs with each candidate shape
 * (64x64, 64x128, 128x64, 96x64, 64x96, 32x128, 128x32, 48x64, 32x64, 64x32,
 * 32x256, 48x128, skipping those the weighting or the workspace does not
 * allow), times each on `stream` with CUDA events (one untimed call, then the
 * fastest of three timed calls; the call synchronises `stream`), writes the fastest shape to *best
 * (other fields copied from opts, which may be NULL) and leaves that shape's
 * result in `out`.  Every shape gives the same counts, and float sums that
 * differ only by rounding.  Arguments as for fa_accumulate; the workspace
 * must hold fa_autotune_workspace_size() bytes (shapes that do not fit are
 * skipped).  Returns the first error fa_accumulate reports for an argument
 * problem, FA_ERR_WORKSPACE if no candidate fits, FA_ERR_INVALID_ARG if no
 * candidate is allowed or best is NULL.  Nothing is cached: pass *best as
 * `opts` to later calls.
 * fa_autotune_batched does the same for a batch (fa_accumulate_batched; one
 * shape for the whole batch), with fa_autotune_batched_workspace_size().
 */
size_t fa_autotune_workspace_size(int64_t rows, int64_t cols, const fa_options *opts);
fa_status fa_autotune(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch_codes,
                      const float *weights, int64_t pitch_w, const uint8_t *mask,
                      int64_t pitch_mask, void *out, fa_out_dtype out_dtype, int64_t pitch_out,
                      void *workspace, size_t ws_bytes, const fa_options *opts, void *stream,
                      fa_options *best);
size_t fa_autotune_batched_workspace_size(const fa_raster *rasters, int32_t n_rasters,
                                          int32_t n_fields, const fa_options *opts);
fa_status fa_autotune_batched(const fa_raster *rasters, int32_t n_rasters, int32_t n_fields,
                              void *workspace, size_t ws_bytes, const fa_options *opts,
                              void *stream, fa_options *best);

/*
 * fa_accumulate for callers that cannot allocate device memory.  The paper has
 * no counterpart: this exists for programs that can pass their own input and
 * output rasters but cannot supply scratch -- plugin hosts that expose only the
 * caller's buffers, pipelines that reserve all device memory at start-up and
 * forbid allocation afterwards, or programs whose memory is owned by another
 * framework's allocator.  Arguments and results are those of fa_accumulate
 * without the workspace: the scratch is one buffer of FA_NOALLOC_SCRATCH_BYTES
 * compiled into the library (every GPU that loads its module keeps it until
 * the process exits), and the call allocates nothing.
 *  - Size limit: rasters whose fa_workspace_size() exceeds
 *    FA_NOALLOC_SCRATCH_BYTES return FA_ERR_TOO_LARGE with nothing enqueued
 *    (with the default 64 x 64 tiles that is about 23 million cells: square
 *    rasters up to 4800 x 4800 fit, 4801 x 4801 does not).
 *  - Every call looks up the buffer's device address on the current device
 *    (cudaGetSymbolAddress); the first call on a device may load the
 *    library's module there, so make that first call outside any stream
 *    capture.
 *  - All calls on a device share the buffer: calls that can overlap on the GPU
 *    race and give wrong results; order them on one stream or synchronise.
 *  - d_status may be NULL, in which case device-detected conditions are
 *    recorded only inside the shared buffer and cannot be read back.
 *  - Phase timing is not recorded for these calls.
 */
#define FA_NOALLOC_SCRATCH_BYTES (64u << 20)
fa_status fa_accumulate_noalloc(const uint8_t *codes, int64_t rows, int64_t cols,
                                int64_t pitch_codes, const float *weights, int64_t pitch_w,
                                const uint8_t *mask, int64_t pitch_mask, void *out,
                                fa_out_dtype out_dtype, int64_t pitch_out, const fa_options *opts,
                                int32_t *d_status, void *stream);

/*
 * Adjoint (transpose) of fa_accumulate with respect to the weights.  Eq. 1 with
 * alpha in {0,1} is linear in w: A = (I - P)^-1 w, P the one-successor flow
 * matrix (Section 2).  Given grad_out = dL/dA this writes
 *     grad_w = dL/dw = (I - P)^-T grad_out,  i.e.  grad_w(c) = sum of grad_out
 * over c's downstream path, c included (the cells whose accumulation w(c)
 * feeds).  Same tile decomposition as fa_accumulate (Sections 3.1-3.3), with
 * pointer jumping over each tile's flow forest and over the exit forest.
 *   codes, mask      as in fa_accumulate.
 *   grad_out         [rows x pitch_g] float32 (device).
 *   grad_w           [rows x pitch_gw] float32 (device); 0 at NoData cells.
 *   workspace        >= fa_workspace_size() bytes.
 * Cells on a cycle, or whose downstream path enters one, are unspecified and
 * FA_ERR_CYCLE is recorded.  The jump tables live in shared memory, so the
 * tile must satisfy 25*(tile_h+2)*(tile_w+2) + 4*(tile_h+tile_w) <= 232448
 * bytes (64x64 and 64x128 fit; 128x128 does not); other shapes return
 * FA_ERR_INVALID_ARG.  Sums are compensated float pairs, rounded once.
 */
fa_status fa_accumulate_adjoint(const uint8_t *codes, int64_t rows, int64_t cols,
                                int64_t pitch_codes, const uint8_t *mask, int64_t pitch_mask,
                                const float *grad_out, int64_t pitch_g, float *grad_w,
                                int64_t pitch_gw, void *workspace, size_t ws_bytes,
                                const fa_options *opts, int32_t *d_status, void *stream);

/*
 * Accumulation with absorption.  Eq. 1 in full: A(p) = w(p) + sum of
 * alpha(n, p) A(n), where alpha(n, p) is the fraction of n's accumulated flow
 * that reaches p and flow may be absorbed but never increased on its way
 * (Section 2).  For a one-successor (D8) metric alpha(n, p) is nonzero only
 * for p = d(n), so it is one factor a(n) per cell:
 *     A(p) = w(p) + sum over n with d(n) = p of a(n) A(n),   0 <= a(n) <= 1.
 * a = 1 everywhere gives fa_accumulate's float sums.  Same tile decomposition
 * (Sections 3.1-3.3): a tile solve that also records, for every perimeter
 * cell, the exit its path reaches and the product of a along the way; a
 * perimeter-graph solve with those products as multipliers; and a second tile
 * solve with the flow entering each tile added at its entry cells (EVICT).
 * All arithmetic is integer (64-bit fixed point per tile, 128-bit across
 * tiles, factors in 1.63 fixed point), so results are bitwise reproducible.
 *   codes, mask        as in fa_accumulate (opts->code_format applies).
 *   weights            [rows x pitch_w] float32 (device) or NULL (unit weights).
 *   factors            [rows x pitch_f] float32 a(n) in [0, 1] (device); the
 *                      factor of a cell without a downstream cell is unused.
 *   out                [rows x pitch_out] float32 (device); 0 at NoData.
 *   workspace          >= fa_absorb_workspace_size() bytes, 256-byte aligned.
 * Tiles must hold at most 4096 cells (a shape left at 0 here means 32 x 64,
 * the fastest measured); other shapes return
 * FA_ERR_INVALID_ARG, as do NULL codes, factors or out, short pitches and
 * misaligned float buffers.  Device-side findings: FA_ERR_NONFINITE for a
 * non-finite weight or a factor outside [0, 1] (results unspecified),
 * FA_ERR_BAD_CODE and FA_ERR_CYCLE as for fa_accumulate.
 */
size_t fa_absorb_workspace_size(int64_t rows, int64_t cols, const fa_options *opts);
fa_status fa_accumulate_absorb(const uint8_t *codes, int64_t rows, int64_t cols,
                               int64_t pitch_codes, const float *weights, int64_t pitch_w,
                               const float *factors, int64_t pitch_f, const uint8_t *mask,
                               int64_t pitch_mask, float *out, int64_t pitch_out, void *workspace,
                               size_t ws_bytes, const fa_options *opts, int32_t *d_status,
                               void *stream);

/*
 * Out-of-core accumulation: unit-weight counts of a raster whose codes and
 * output stay in HOST memory, for rasters larger than the device (Section 2
 * sets rasters beyond one machine's memory as the aim; Section 3 with EVICT:
 * only one block and the perimeter data are held at once).  The raster is cut
 * into outer blocks of block_rows x block_cols cells; each block's codes,
 * with a one-cell ring, are copied to the device twice: pass A solves the
 * block by the tile pipeline of fa_accumulate and records its perimeter graph
 * (Algorithm 2 at block level), the perimeter graphs of all blocks are solved
 * on the device (Section 3.2), and pass C solves the block again with the
 * flow entering from other blocks given to the tile pipeline as extra inflow
 * at the block's entry cells, which carries it along the paths (Algorithm 3),
 * and copies the block's counts out.  Copies run on two streams of the
 * library's own, overlapping the solves when the host buffers are pinned; the
 * call is SYNCHRONOUS (it returns after the last copy out).
 *   codes       [rows x pitch_codes] one byte per cell, HOST memory (pinned
 *               or pageable); FA_CODES_NIBBLE is not accepted.
 *   out         [rows x pitch_out] uint64 counts, HOST memory; exact for any
 *               raster size; 0 at NoData.
 *   block_rows, block_cols  outer block shape (0 = 16384; a side longer
 *               than the raster's is cut to it); perim(block) =
 *               2 (block_rows + block_cols) - 4 must be <= 65534, and
 *               blocks x perim < 2^32 - 1.
 *   workspace   device, >= fa_ooc_workspace_size(), 256-byte aligned: two
 *               code buffers, one uint32 and two uint64 block buffers, the
 *               tile pipeline's workspace for one block plus 16 bytes per
 *               perimeter slot of its tiles, and 38 bytes per perimeter slot
 *               of every block.
 *   opts        tile shape and flags for the block solves (as fa_accumulate).
 * Returns the decoded device status (as fa_status_read: BAD_CODE, CYCLE, ...)
 * after completion, FA_ERR_INVALID_ARG / FA_ERR_WORKSPACE for bad arguments
 * (nothing enqueued) or FA_ERR_CUDA.  d_status as in fa_accumulate.  Results
 * equal fa_accumulate's counts on the same raster, cell for cell.
 */
size_t fa_ooc_workspace_size(int64_t rows, int64_t cols, int64_t block_rows, int64_t block_cols,
                             const fa_options *opts);
fa_status fa_accumulate_ooc(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch_codes,
                            uint64_t *out, int64_t pitch_out, int64_t block_rows,
                            int64_t block_cols, void *workspace, size_t ws_bytes,
                            const fa_options *opts, int32_t *d_status, void *stream);

/*
 * Shard form: fa_accumulate_ooc's three stages run by separate processes
 * (one per GPU), exchanging only the perimeter records: the paper's two
 * MapReduces (Section 3, Algorithm 3; Section 4 counts the data sent).  The
 * raster is cut into outer blocks as in fa_accumulate_ooc (same block_rows,
 * block_cols, opts in every call of one solve); a shard owns a band of whole
 * block rows [band0, band1) (blocks band0 * nbx .. band1 * nbx - 1, row-major
 * block numbering):
 *   1. every shard:  fa_shard_export   pass A on its blocks -> their records;
 *   2. gather the records of all blocks in one process;
 *   3. that process: fa_shard_resolve  the blocks' perimeter graph solved
 *                    (Section 3.2) -> in(p) for every block perimeter slot;
 *   4. scatter each shard's part of in(p);
 *   5. every shard:  fa_shard_finish   pass C on its blocks -> uint64 counts.
 * The result equals fa_accumulate_ooc's (and fa_accumulate's counts), cell
 * for cell.  All three calls are SYNCHRONOUS on `stream`; records, in(p),
 * codes and counts are HOST memory; workspace is device memory of at least
 * fa_ooc_workspace_size(rows, cols, block_rows, block_cols, opts) bytes,
 * 256-byte aligned (fa_shard_resolve uses only its perimeter-graph part).
 * d_status and the returned status as in fa_accumulate_ooc: export reports
 * invalid codes and in-block cycles of its blocks, resolve cycles through
 * several blocks, finish its blocks' conditions again.
 *
 * fa_shard_geometry: block_grid[0] = nby (block rows), block_grid[1] = nbx
 * (blocks per block row), *pmax = record slots per block; FA_ERR_INVALID_ARG
 * where fa_ooc_workspace_size would return 0.
 *
 * Records of blocks [b0, b1) (b = band0 * nbx ..), host arrays:
 *   nexit     [b1 - b0]          uint32 outer exits of each block;
 *   link      [(b1 - b0) * pmax] uint16 per block perimeter slot (slots
 *             clockwise from the block's top-left cell: top row west to
 *             east, right column north to south, bottom row east to west,
 *             left column south to north; a one-row or one-column block in
 *             cell order): the exit rank its path reaches in the block,
 *             0xFFFF for none (an exit links to its own rank);
 *   node_dst  [(b1 - b0) * pmax] uint32 per exit rank: global slot id
 *             (block * pmax + slot) of the cell its flow enters;
 *   node_val  [(b1 - b0) * pmax] double per exit rank: its block-local
 *             accumulation A_loc (an exact integer).
 * Entries past nexit[b] are 0.  The ranks' order depends on scheduling; the
 * in(p) and counts computed from them do not.
 *
 * Codes: codes points at raster row codes_row0 and holds codes_rows rows of
 * pitch_codes bytes, which must include every row the band's blocks read:
 * rows max(band0 * bh - 1, 0) .. min(band1 * bh + 1, rows) - 1 (the band and
 * its ring rows), bh being the block height in use (block_rows, 0 = 16384,
 * cut to the raster's rows).
 *
 * fa_shard_resolve takes the records of ALL nby * nbx blocks (concatenated in
 * block order) and writes inflow [nby * nbx * pmax]: per block perimeter slot
 * the flow entering that cell from other blocks (uint64).  Records are
 * checked on the host first (nexit <= pmax, targets inside the raster, links
 * none or an exit of their block): FA_ERR_INVALID_ARG otherwise, nothing run.
 *
 * fa_shard_finish takes inflow [(b1 - b0) * pmax] (the band's part, from
 * slot b0 * pmax) and writes out: raster rows band0 * bh ..
 * min(band1 * bh, rows) - 1, row 0 first, pitch_out elements apart.
 *
 * An empty band (band0 == band1) is valid: nothing is read or written.
 */
fa_status fa_shard_geometry(int64_t rows, int64_t cols, int64_t block_rows, int64_t block_cols,
                            int64_t *block_grid, int32_t *pmax);
fa_status fa_shard_export(const uint8_t *codes, int64_t codes_row0, int64_t codes_rows,
                          int64_t pitch_codes, int64_t rows, int64_t cols, int64_t block_rows,
                          int64_t block_cols, int64_t band0, int64_t band1, uint32_t *nexit,
                          uint16_t *link, uint32_t *node_dst, double *node_val, void *workspace,
                          size_t ws_bytes, const fa_options *opts, int32_t *d_status, void *stream);
fa_status fa_shard_resolve(int64_t rows, int64_t cols, int64_t block_rows, int64_t block_cols,
                           const uint32_t *nexit, const uint16_t *link, const uint32_t *node_dst,
                           const double *node_val, uint64_t *inflow, void *workspace,
                           size_t ws_bytes, int32_t *d_status, void *stream);
fa_status fa_shard_finish(const uint8_t *codes, int64_t codes_row0, int64_t codes_rows,
                          int64_t pitch_codes, int64_t rows, int64_t cols, int64_t block_rows,
                          int64_t block_cols, int64_t band0, int64_t band1, const uint64_t *inflow,
                          uint64_t *out, int64_t pitch_out, void *workspace, size_t ws_bytes,
                          const fa_options *opts, int32_t *d_status, void *stream);

/*
 * Copies the device status block back (synchronises `stream`) and maps it to
 * the most severe fa_status: BAD_CODE, then CYCLE, NONFINITE, TIMEOUT, then
 * FA_WARN_OVERFLOW, else FA_OK.  count / first_index may be NULL.
 * d_status NULL means the block inside `workspace`.
 */
fa_status fa_status_read(const int32_t *d_status, const void *workspace, void *stream,
                         int64_t *count, int64_t *first_index);

/*
 * Self-test of the bounded device wait.  The staged tile loads of pass 1 wait
 * on an mbarrier for each copy; that wait gives up after a time limit, sets
 * FA_FLAG_TIMEOUT in the status block and lets the kernel return, so a copy
 * that never completes becomes an error status instead of a hang.  This call
 * runs that same wait, with a limit of limit_ns nanoseconds (0 .. 1e10),
 * against a barrier phase that no arrival or copy will ever complete, with no
 * copy in flight: the status block d_status (device int32[FA_STATUS_WORDS],
 * 8-byte aligned, required) is reset and then records FA_FLAG_TIMEOUT with a
 * count of 1, which fa_status_read reports as FA_ERR_TIMEOUT.  The GPU context
 * stays usable.  The paper has no counterpart (it has no device waits).
 * Asynchronous on `stream`; FA_ERR_INVALID_ARG for a NULL or misaligned
 * d_status or a limit out of range, FA_ERR_CUDA if the launch fails.
 */
fa_status fa_selftest_wait_timeout(int64_t limit_ns, int32_t *d_status, void *stream);

/*
 * Phase timing (a tracing aid, not part of the computation).  While enabled,
 * each fa_accumulate call records CUDA events on its own stream at the
 * boundaries of its phases: pass 1 (per-tile solve and perimeter links,
 * Section 3.1), the perimeter-graph resolve (Section 3.2) and pass 2 (the
 * finalising per-tile pass, Section 3.3).  fa_timing_read synchronises on the
 * last event of the most recent call and writes up to n phase durations in
 * milliseconds; it returns how many phases it wrote (0 if none was recorded,
 * -1 on a CUDA error).  Events are created on first use; one thread and one
 * device at a time.
 */
void fa_timing_enable(int32_t on);
int32_t fa_timing_read(float *ms, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* FA_H */
