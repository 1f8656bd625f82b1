/*
 * CPU oracle for D8 flow accumulation -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  The product path never calls it; it shares no code, header,
 * table or constant with the CUDA library.
 *
 * What it computes (Eq. 1 with alpha restricted to {0,1}, Section 2):
 *     A(p) = w(p) + sum over neighbours n whose single downstream cell is p of A(n)
 * for every valid cell p; NoData cells get 0.  It solves Eq. 1 the way the
 * paper's single-tile algorithm does (Algorithm 1), applied to the whole raster
 * as one tile, which is the "simple implementation ... verified by inspection"
 * the paper uses as its correctness authority (Section 6, Correctness):
 *   1. dependency counts D(t) = number of valid cells whose downstream cell is t;
 *   2. a FIFO queue seeded with every valid cell with D = 0;
 *   3. pop c: A(c) += w(c); if c has a downstream cell t: A(t) += A(c),
 *      D(t) -= 1, push t when D(t) reaches 0.
 * Counts are uint64 and weighted sums FP64.  Valid cells left with D > 0 lie on
 * cycles (in a graph where every cell has one successor nothing but the cycle
 * itself lies downstream of a cycle); they are reported and their values are
 * left partial.
 *
 * Codes: 0 NoData, 1..8 = E, NE, N, NW, W, SW, S, SE, 9 NoFlow, 10..255 invalid
 * (counted, treated as NoData).  A cell is NoData if its code is 0 or invalid,
 * or if mask != NULL and mask[cell] != 0.  Row 0 is north.  The downstream
 * cell d(c) does not exist when c is NoFlow, when the target is off the grid or
 * when the target is NoData (Algorithm 1 skips such targets; Algorithm 2
 * treats the outside of the data as NoData).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -march flags).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* code k -> (dr, dc); index 0 unused.  E NE N NW W SW S SE */
static const int ODR[10] = {0, 0, -1, -1, -1, 0, 1, 1, 1, 0};
static const int ODC[10] = {0, 1, 1, 0, -1, -1, -1, 0, 1, 0};

typedef struct {
    const uint8_t *codes;
    const uint8_t *mask;
    int64_t rows, cols, pitch, mpitch;
} raster;

static int valid_cell(const raster *R, int64_t r, int64_t c) {
    if (r < 0 || c < 0 || r >= R->rows || c >= R->cols) return 0;
    uint8_t k = R->codes[r * R->pitch + c];
    if (k == 0 || k > 9) return 0;
    if (R->mask && R->mask[r * R->mpitch + c]) return 0;
    return 1;
}

/* d(c) as a dense index r*cols+c, or -1 when c has no downstream cell. */
static int64_t downstream(const raster *R, int64_t r, int64_t c) {
    uint8_t k = R->codes[r * R->pitch + c];
    if (k == 0 || k >= 9) return -1;
    int64_t rr = r + ODR[k], cc = c + ODC[k];
    if (!valid_cell(R, rr, cc)) return -1;
    return rr * R->cols + cc;
}

/*
 * Kahn pass over the whole raster (Algorithm 1 steps 1-5).  Fills next[] with
 * d(c) (-1 if none, -2 for NoData) and order[] with the FIFO pop order, and
 * returns the number of popped cells.  deg is scratch of rows*cols bytes (a
 * cell has at most 8 upstream neighbours).
 */
static int64_t kahn_order(const raster *R, int64_t *next, int64_t *order, uint8_t *deg,
                          int64_t *n_bad, int64_t *n_valid) {
    int64_t n = R->rows * R->cols, bad = 0, nv = 0;
    memset(deg, 0, (size_t)n);
    for (int64_t r = 0; r < R->rows; ++r)
        for (int64_t c = 0; c < R->cols; ++c) {
            int64_t i = r * R->cols + c;
            uint8_t k = R->codes[r * R->pitch + c];
            if (k > 9) ++bad;
            if (!valid_cell(R, r, c)) { next[i] = -2; continue; }
            ++nv;
            next[i] = downstream(R, r, c);
            if (next[i] >= 0) deg[next[i]]++;
        }
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < n; ++i)
        if (next[i] != -2 && deg[i] == 0) order[tail++] = i;
    while (head < tail) {
        int64_t c = order[head++];
        int64_t t = next[c];
        if (t >= 0 && --deg[t] == 0) order[tail++] = t;
    }
    if (n_bad) *n_bad = bad;
    if (n_valid) *n_valid = nv;
    return tail;
}

/* state[i]: 0 NoData, 1 finalized, 2 on a cycle (value unspecified). */
static void fill_state(int64_t n, const int64_t *next, const int64_t *order, int64_t popped,
                       uint8_t *state, int64_t *n_cycle) {
    if (!state) return;
    for (int64_t i = 0; i < n; ++i) state[i] = next[i] == -2 ? 0 : 2;
    for (int64_t j = 0; j < popped; ++j) state[order[j]] = 1;
    if (n_cycle) {
        int64_t cyc = 0;
        for (int64_t i = 0; i < n; ++i) cyc += state[i] == 2;
        *n_cycle = cyc;
    }
}

/*
 * Unit-weight accumulation (upslope cell counts), uint64, dense rows*cols out.
 * Returns 0, or -1 on allocation failure.  Algorithm 1 with w = 1.
 */
int fa_oracle_counts(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                     const uint8_t *mask, int64_t mpitch, uint64_t *out, uint8_t *state,
                     int64_t *n_cycle, int64_t *n_bad) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t n = rows * cols;
    int64_t *next = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *deg = (uint8_t *)malloc((size_t)(n ? n : 1));
    if (!next || !order || !deg) { free(next); free(order); free(deg); return -1; }
    /* steps 1-2: dependency counts; step 3: seed; steps 4-5: pop and push */
    int64_t nv;
    int64_t popped = kahn_order(&R, next, order, deg, n_bad, &nv);
    memset(out, 0, (size_t)n * sizeof(uint64_t));
    /* replay the FIFO order: a cell's predecessors were all popped earlier */
    for (int64_t j = 0; j < popped; ++j) {
        int64_t c = order[j];
        out[c] += 1;
        if (next[c] >= 0) out[next[c]] += out[c];
    }
    /* cells on cycles never popped: their own unit is not added (partial) */
    fill_state(n, next, order, popped, state, n_cycle);
    free(next); free(order); free(deg);
    return 0;
}

/* Weighted accumulation in FP64 from float weights (pitch in elements). */
int fa_oracle_weighted(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                       const uint8_t *mask, int64_t mpitch, const float *w, int64_t wpitch,
                       double *out, uint8_t *state, int64_t *n_cycle, int64_t *n_bad) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t n = rows * cols;
    int64_t *next = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *deg = (uint8_t *)malloc((size_t)(n ? n : 1));
    if (!next || !order || !deg) { free(next); free(order); free(deg); return -1; }
    int64_t nv;
    int64_t popped = kahn_order(&R, next, order, deg, n_bad, &nv);
    memset(out, 0, (size_t)n * sizeof(double));
    for (int64_t j = 0; j < popped; ++j) {
        int64_t c = order[j];
        int64_t r = c / cols, cc = c % cols;
        out[c] += (double)w[r * wpitch + cc];
        if (next[c] >= 0) out[next[c]] += out[c];
    }
    fill_state(n, next, order, popped, state, n_cycle);
    free(next); free(order); free(deg);
    return 0;
}

/*
 * Accumulation with absorption: Eq. 1 with alpha(n, p) = a(n) for the one
 * downstream cell p of n (and 0 elsewhere), a(n) in [0, 1] -- Section 2 lets
 * flow be absorbed on its way downhill but never increased, so the share a
 * cell passes on is at most what it holds:
 *     A(p) = w(p) + sum over n with d(n) = p of a(n) A(n).
 * Same Kahn order as fa_oracle_weighted (FP64); w NULL means unit weights.
 * a(n) of a cell without a downstream cell is never used.
 */
int fa_oracle_absorb(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                     const uint8_t *mask, int64_t mpitch, const float *w, int64_t wpitch,
                     const float *a, int64_t apitch, double *out, uint8_t *state,
                     int64_t *n_cycle, int64_t *n_bad) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t n = rows * cols;
    int64_t *next = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *deg = (uint8_t *)malloc((size_t)(n ? n : 1));
    if (!next || !order || !deg) { free(next); free(order); free(deg); return -1; }
    int64_t nv;
    int64_t popped = kahn_order(&R, next, order, deg, n_bad, &nv);
    memset(out, 0, (size_t)n * sizeof(double));
    for (int64_t j = 0; j < popped; ++j) {
        int64_t c = order[j];
        int64_t r = c / cols, cc = c % cols;
        out[c] += w ? (double)w[r * wpitch + cc] : 1.0;
        if (next[c] >= 0) out[next[c]] += (double)a[r * apitch + cc] * out[c];
    }
    fill_state(n, next, order, popped, state, n_cycle);
    free(next); free(order); free(deg);
    return 0;
}

/*
 * Transpose product (the adjoint of Eq. 1 with alpha in {0,1}): with
 * A = (I - P)^-1 w, the gradient of <g, A> with respect to w is
 * lam = (I - P)^-T g, i.e. lam(c) = g(c) + lam(d(c)), the sum of g along c's
 * downstream path.  Computed by walking the Kahn pop order backwards, so d(c)
 * is final before c.  FP64.  state: 0 NoData, 1 exact, 2 unspecified (the cell
 * is on a cycle or its downstream path enters one).
 */
int fa_oracle_adjoint(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                      const uint8_t *mask, int64_t mpitch, const float *g, int64_t gpitch,
                      double *lam, uint8_t *state, int64_t *n_cycle, int64_t *n_bad) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t n = rows * cols;
    int64_t *next = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *deg = (uint8_t *)malloc((size_t)(n ? n : 1));
    uint8_t *ok = (uint8_t *)malloc((size_t)(n ? n : 1));
    if (!next || !order || !deg || !ok) {
        free(next); free(order); free(deg); free(ok);
        return -1;
    }
    int64_t nv;
    int64_t popped = kahn_order(&R, next, order, deg, n_bad, &nv);
    memset(lam, 0, (size_t)n * sizeof(double));
    memset(ok, 0, (size_t)n);
    for (int64_t j = popped - 1; j >= 0; --j) {
        int64_t c = order[j];
        int64_t r = c / cols, cc = c % cols;
        double v = (double)g[r * gpitch + cc];
        int good = 1;
        if (next[c] >= 0) {
            if (ok[next[c]]) v += lam[next[c]];
            else good = 0; /* downstream cell never popped: path enters a cycle */
        }
        lam[c] = v;
        ok[c] = (uint8_t)good;
    }
    if (state) {
        int64_t cyc = 0;
        for (int64_t i = 0; i < n; ++i) {
            state[i] = next[i] == -2 ? 0 : (ok[i] ? 1 : 2);
            cyc += state[i] == 2;
        }
        if (n_cycle) *n_cycle = cyc;
    }
    free(next); free(order); free(deg); free(ok);
    return 0;
}

/*
 * Brute force from the definition: every valid cell y adds w(y) (1 if w is
 * NULL) to each cell on its downstream path, itself included.  A walk longer
 * than the number of cells has entered a cycle and is abandoned; the cells it
 * reached are flagged in state as 2.  O(n * path length): small rasters only.
 */
int fa_oracle_bruteforce(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                         const uint8_t *mask, int64_t mpitch, const float *w, int64_t wpitch,
                         double *out, uint8_t *state) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t n = rows * cols;
    memset(out, 0, (size_t)n * sizeof(double));
    if (state)
        for (int64_t i = 0; i < n; ++i)
            state[i] = valid_cell(&R, i / cols, i % cols) ? 1 : 0;
    for (int64_t y = 0; y < n; ++y) {
        int64_t r = y / cols, c = y % cols;
        if (!valid_cell(&R, r, c)) continue;
        double wy = w ? (double)w[r * wpitch + c] : 1.0;
        int64_t cur = y, steps = 0;
        while (cur >= 0 && steps <= n) {
            out[cur] += wy;
            cur = downstream(&R, cur / cols, cur % cols);
            ++steps;
        }
        if (cur >= 0 && state) {
            /* cycle: flag the cycle cells reached */
            int64_t s = cur;
            for (int64_t t = 0; t <= n; ++t) {
                state[s] = 2;
                s = downstream(&R, s / cols, s % cols);
                if (s < 0 || s == cur) break;
            }
        }
    }
    return 0;
}

/*
 * Streaming Eq. 1 residual check for uint32 results (mod 2^32): for every valid
 * cell p, A(p) == 1 + sum of A(n) over neighbours n with d(n) = p (unit weights),
 * and A(p) == 0 at NoData.  One row sweep, O(1) extra memory.  For an acyclic
 * input the integer solution of Eq. 1 is unique, so zero mismatches proves the
 * whole raster exact.  Returns the number of mismatching cells; *first gets the
 * first mismatching index (r*cols+c) or -1.
 */
int64_t fa_oracle_residual_u32_rows(const uint8_t *codes, int64_t rows, int64_t cols,
                                    int64_t pitch, const uint8_t *mask, int64_t mpitch,
                                    const uint32_t *A, int64_t apitch, int64_t r_begin,
                                    int64_t r_end, int64_t *first);

int64_t fa_oracle_residual_u32(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                               const uint8_t *mask, int64_t mpitch, const uint32_t *A,
                               int64_t apitch, int64_t *first) {
    return fa_oracle_residual_u32_rows(codes, rows, cols, pitch, mask, mpitch, A, apitch, 0, rows,
                                       first);
}

/* The same check restricted to the rows r_begin .. r_end - 1 of the raster
 * (the neighbours are still read from the whole raster), so that disjoint row
 * bands of one raster can be checked independently. */
int64_t fa_oracle_residual_u32_rows(const uint8_t *codes, int64_t rows, int64_t cols,
                                    int64_t pitch, const uint8_t *mask, int64_t mpitch,
                                    const uint32_t *A, int64_t apitch, int64_t r_begin,
                                    int64_t r_end, int64_t *first) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t bad = 0, f = -1;
    if (r_begin < 0) r_begin = 0;
    if (r_end > rows) r_end = rows;
    for (int64_t r = r_begin; r < r_end; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            uint32_t expect;
            if (!valid_cell(&R, r, c)) {
                expect = 0;
            } else {
                expect = 1u;
                for (int k = 1; k <= 8; ++k) {
                    int64_t rr = r + ODR[k], cc = c + ODC[k];
                    if (!valid_cell(&R, rr, cc)) continue;
                    if (downstream(&R, rr, cc) == r * cols + c) expect += A[rr * apitch + cc];
                }
            }
            if (A[r * apitch + c] != expect) {
                if (f < 0) f = r * cols + c;
                ++bad;
            }
        }
    if (first) *first = f;
    return bad;
}

/*
 * Conservation (Eq. 1 summed over the raster): every valid cell's weight
 * ends in exactly one terminal cell, a valid cell without a downstream cell
 * (NoFlow, or flow off the grid or into NoData).  Over the rows r_begin ..
 * r_end - 1 this adds A over the terminal cells (as uint64, from uint32
 * results) into *outlet_sum and counts the valid cells into *n_valid.  Over a
 * whole acyclic raster with unit weights the two totals are equal, and equal
 * modulo 2^32 when some terminal count wrapped in uint32.
 */
void fa_oracle_outlet_sum_u32(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                              const uint8_t *mask, int64_t mpitch, const uint32_t *A,
                              int64_t apitch, int64_t r_begin, int64_t r_end,
                              uint64_t *outlet_sum, int64_t *n_valid) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    uint64_t s = 0;
    int64_t nv = 0;
    if (r_begin < 0) r_begin = 0;
    if (r_end > rows) r_end = rows;
    for (int64_t r = r_begin; r < r_end; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            if (!valid_cell(&R, r, c)) continue;
            ++nv;
            if (downstream(&R, r, c) < 0) s += A[r * apitch + c];
        }
    *outlet_sum = s;
    *n_valid = nv;
}

/*
 * The residual check and the conservation sum for uint64 counts (results too
 * large for uint32, as from rasters of 2^32 cells or more): the same Eq. 1
 * test, A(p) == 1 + sum of A(n) over the neighbours n with d(n) = p, in exact
 * uint64 arithmetic with no wrap-around, on rows r_begin .. r_end - 1.
 */
int64_t fa_oracle_residual_u64_rows(const uint8_t *codes, int64_t rows, int64_t cols,
                                    int64_t pitch, const uint8_t *mask, int64_t mpitch,
                                    const uint64_t *A64, int64_t apitch, int64_t r_begin,
                                    int64_t r_end, int64_t *first) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t bad = 0, f = -1;
    if (r_begin < 0) r_begin = 0;
    if (r_end > rows) r_end = rows;
    for (int64_t r = r_begin; r < r_end; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            uint64_t expect;
            if (!valid_cell(&R, r, c)) {
                expect = 0;
            } else {
                expect = 1;
                for (int k = 1; k <= 8; ++k) {
                    int64_t rr = r + ODR[k], cc = c + ODC[k];
                    if (!valid_cell(&R, rr, cc)) continue;
                    if (downstream(&R, rr, cc) == r * cols + c) expect += A64[rr * apitch + cc];
                }
            }
            if (A64[r * apitch + c] != expect) {
                if (f < 0) f = r * cols + c;
                ++bad;
            }
        }
    if (first) *first = f;
    return bad;
}

void fa_oracle_outlet_sum_u64(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                              const uint8_t *mask, int64_t mpitch, const uint64_t *A64,
                              int64_t apitch, int64_t r_begin, int64_t r_end,
                              uint64_t *outlet_sum, int64_t *n_valid) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    uint64_t s = 0;
    int64_t nv = 0;
    if (r_begin < 0) r_begin = 0;
    if (r_end > rows) r_end = rows;
    for (int64_t r = r_begin; r < r_end; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            if (!valid_cell(&R, r, c)) continue;
            ++nv;
            if (downstream(&R, r, c) < 0) s += A64[r * apitch + c];
        }
    *outlet_sum = s;
    *n_valid = nv;
}

/*
 * Eq. 1's solution at chosen cells, one query at a time, from its plain
 * meaning: A(p) is the sum of w over p's upstream area, the valid cells whose
 * flow path passes through p, p included.  The area is gathered by a
 * depth-first search against the flow: from a cell u, every valid neighbour n
 * with d(n) = u belongs to it.  Each cell has a single downstream cell, so
 * the area is a tree and no cell is reached twice; only a query on a cycle
 * would never end, so the search stops after as many cells as the raster has
 * and reports size -1 (value NaN) for it.  Sums in FP64, w == NULL meaning
 * unit weights; a NoData query gets 0 and size 0.  Returns the number of
 * cells visited over all queries, or -1 if the stack could not be allocated.
 */
int64_t fa_oracle_upstream_sums(const uint8_t *codes, int64_t rows, int64_t cols, int64_t pitch,
                                const uint8_t *mask, int64_t mpitch, const float *w,
                                int64_t wpitch, const int64_t *query, int64_t nq, double *out,
                                int64_t *size) {
    raster R = {codes, mask, rows, cols, pitch, mpitch};
    int64_t cap = 1024, visited = 0;
    int64_t *stack = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    if (!stack) return -1;
    for (int64_t q = 0; q < nq; ++q) {
        const int64_t p = query[q];
        out[q] = 0.0;
        size[q] = 0;
        if (!valid_cell(&R, p / cols, p % cols)) continue;
        double sum = 0.0;
        int64_t n = 0, top = 0;
        stack[top++] = p;
        while (top > 0 && n <= rows * cols) {
            const int64_t u = stack[--top];
            const int64_t r = u / cols, c = u % cols;
            sum += w ? (double)w[r * wpitch + c] : 1.0;
            ++n;
            for (int k = 1; k <= 8; ++k) {
                const int64_t rr = r + ODR[k], cc = c + ODC[k];
                if (!valid_cell(&R, rr, cc) || downstream(&R, rr, cc) != u) continue;
                if (top == cap) {
                    int64_t *grown = (int64_t *)realloc(stack, (size_t)(2 * cap) * sizeof(int64_t));
                    if (!grown) {
                        free(stack);
                        return -1;
                    }
                    stack = grown;
                    cap *= 2;
                }
                stack[top++] = rr * cols + cc;
            }
        }
        visited += n;
        if (top > 0) {  /* the bound ran out: p lies on a cycle */
            out[q] = 0.0 / 0.0;
            size[q] = -1;
        } else {
            out[q] = sum;
            size[q] = n;
        }
    }
    free(stack);
    return visited;
}

/*
 * D8 flow codes from elevations, the step before accumulation (Section 2: a
 * non-divergent metric sends a cell's flow to a single neighbour; D8 takes the
 * steepest descent; flats are routed towards lower terrain only; Fig. 1 treats
 * the direction step as a separate algorithm).  The rules, one per cell:
 *   - NoData (nodata != NULL and nodata[cell] != 0): code 0;
 *   - a cell on the raster's border drains off the grid, perpendicular to its
 *     edge (N, S, W, E) and diagonally at the corners (NW, NE, SW, SE);
 *   - otherwise the valid neighbour with the largest positive slope, slope =
 *     drop for E, N, W, S and drop * (1/sqrt 2) for the diagonals, drop =
 *     z(cell) - z(neighbour); neighbours are tried in the order E, NE, N, NW,
 *     W, SW, S, SE and a later one must be strictly steeper to win;
 *   - no positive slope: the first NoData neighbour in that order (flow leaves
 *     the data there), else NoFlow (9).
 * The decision is taken in float32: the drop is one float subtraction, the
 * diagonal factor the float nearest 1/sqrt 2, one float multiplication each
 * (built with -ffp-contract=off, so nothing is fused).
 */
int fa_oracle_d8(const float *z, int64_t rows, int64_t cols, int64_t pitch_z,
                 const uint8_t *nodata, int64_t pitch_nd, uint8_t *codes) {
    const float inv_sqrt2 = 0.70710678118654752440f;
    for (int64_t r = 0; r < rows; ++r) {
        for (int64_t c = 0; c < cols; ++c) {
            uint8_t *out = &codes[r * cols + c];
            if (nodata && nodata[r * pitch_nd + c]) {
                *out = 0;
                continue;
            }
            const int top = r == 0, bottom = r == rows - 1, left = c == 0, right = c == cols - 1;
            if (top || bottom || left || right) {
                if (top && left) *out = 4;
                else if (top && right) *out = 2;
                else if (bottom && left) *out = 6;
                else if (bottom && right) *out = 8;
                else if (top) *out = 3;
                else if (bottom) *out = 7;
                else if (left) *out = 5;
                else *out = 1;
                continue;
            }
            const float zc = z[r * pitch_z + c];
            float best = 0.0f;
            uint8_t code = 0, into_nodata = 0;
            for (int k = 1; k <= 8; ++k) {
                const int64_t rn = r + ODR[k], cn = c + ODC[k];
                if (nodata && nodata[rn * pitch_nd + cn]) {
                    if (!into_nodata) into_nodata = (uint8_t)k;
                    continue;
                }
                const float drop = zc - z[rn * pitch_z + cn];
                const float slope = (k == 1 || k == 3 || k == 5 || k == 7) ? drop : drop * inv_sqrt2;
                if (slope > best) {
                    best = slope;
                    code = (uint8_t)k;
                }
            }
            *out = code ? code : (into_nodata ? into_nodata : 9);
        }
    }
    return 0;
}
