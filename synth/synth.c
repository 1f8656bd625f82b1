/*
 * Seeded terrain helpers for synthetic D8 flow-direction rasters.
 *
 * Test and benchmark input infrastructure shared by the oracle side and the
 * CUDA side.  Nothing here computes flow accumulation: these routines turn an
 * elevation raster into a drained surface (priority-flood depression filling
 * with an epsilon gradient) and then into one-byte D8 codes.  The paper treats
 * both steps as a black box in front of the method (Section 2 on depression
 * filling and flats; Fig. 3 caption).
 *
 * Code encoding (one byte per cell):
 *   0 = NoData, 1..8 = E, NE, N, NW, W, SW, S, SE, 9 = NoFlow.
 * Row 0 is north; r grows south.  Offsets (dr, dc) per code:
 *   E (0,+1) NE (-1,+1) N (-1,0) NW (-1,-1) W (0,-1) SW (+1,-1) S (+1,0) SE (+1,+1)
 *
 * Built with -ffp-contract=off so that x86-64 and aarch64 produce the same
 * bits from the same float input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int SDR[9] = {0, 0, -1, -1, -1, 0, 1, 1, 1};
static const int SDC[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};

/* ---- radix heap on the bit pattern of non-negative float elevations -------
 * Priority-flood only ever pushes keys >= the last popped key, so a monotone
 * radix heap (Ahuja, Mehlhorn, Orlin & Tarjan 1990) orders it exactly.  Keys
 * equal to the last popped key are served in LIFO order, which is a fixed,
 * machine-independent order. */
typedef struct {
    uint32_t *key;
    int64_t *idx;
    int64_t n, cap;
} rbucket;

typedef struct {
    rbucket b[33];
    uint32_t last;
    int64_t size;
} rheap;

static int rb_push(rbucket *b, uint32_t k, int64_t i) {
    if (b->n == b->cap) {
        int64_t nc = b->cap ? b->cap * 2 : 1024;
        uint32_t *nk = (uint32_t *)realloc(b->key, (size_t)nc * sizeof(uint32_t));
        if (!nk) return -1;
        b->key = nk;
        int64_t *ni = (int64_t *)realloc(b->idx, (size_t)nc * sizeof(int64_t));
        if (!ni) return -1;
        b->idx = ni;
        b->cap = nc;
    }
    b->key[b->n] = k;
    b->idx[b->n] = i;
    b->n++;
    return 0;
}

static int rbucket_of(uint32_t k, uint32_t last) {
    uint32_t x = k ^ last;
    return x ? 32 - __builtin_clz(x) : 0;
}

static int rheap_push(rheap *h, float z, int64_t i) {
    uint32_t k;
    memcpy(&k, &z, 4);
    h->size++;
    return rb_push(&h->b[rbucket_of(k, h->last)], k, i);
}

static int rheap_pop(rheap *h, float *z, int64_t *i) {
    if (h->b[0].n == 0) {
        int j = 1;
        while (h->b[j].n == 0) ++j;
        rbucket *src = &h->b[j];
        uint32_t m = src->key[0];
        for (int64_t t = 1; t < src->n; ++t)
            if (src->key[t] < m) m = src->key[t];
        h->last = m;
        for (int64_t t = 0; t < src->n; ++t)
            if (rb_push(&h->b[rbucket_of(src->key[t], m)], src->key[t], src->idx[t])) return -1;
        src->n = 0;
    }
    rbucket *b0 = &h->b[0];
    b0->n--;
    memcpy(z, &b0->key[b0->n], 4);
    *i = b0->idx[b0->n];
    h->size--;
    return 0;
}

static void rheap_free(rheap *h) {
    for (int j = 0; j < 33; ++j) { free(h->b[j].key); free(h->b[j].idx); }
}

/*
 * Priority-flood with an epsilon gradient (Barnes et al. 2014, cited in the
 * paper's Section 2).  Seeds are valid cells on the raster edge or next to a
 * NoData cell.  Every other valid cell ends strictly higher than the cell that
 * reached it, so each one has a strictly lower neighbour and drains to a seed.
 * z (non-negative) is modified in place; nodata != 0 marks NoData cells (left
 * untouched).  Returns 0, or -1 on allocation failure.
 */
static int priority_flood(float *z, const uint8_t *nodata, int64_t rows, int64_t cols, float eps,
                          int kstep);

int synth_priority_flood_eps(float *z, const uint8_t *nodata, int64_t rows, int64_t cols,
                             float eps) {
    return priority_flood(z, nodata, rows, cols, eps, 1);
}

/* The same with the flood spreading to the four edge neighbours only (E, N,
 * W, S): every cell that is not a seed ends strictly above one of its edge
 * neighbours.  A bilinear upsampling of such a surface keeps a strictly lower
 * neighbour at every fine cell (used for the 1e10-cell scale raster). */
int synth_priority_flood_eps4(float *z, const uint8_t *nodata, int64_t rows, int64_t cols,
                              float eps) {
    return priority_flood(z, nodata, rows, cols, eps, 2);
}

static int priority_flood(float *z, const uint8_t *nodata, int64_t rows, int64_t cols, float eps,
                          int kstep) {
    int64_t n = rows * cols;
    uint8_t *closed = (uint8_t *)calloc((size_t)n, 1);
    if (!closed) return -1;
    rheap h;
    memset(&h, 0, sizeof(h));
    int rc = 0;
    for (int64_t r = 0; r < rows && !rc; ++r) {
        for (int64_t c = 0; c < cols; ++c) {
            int64_t i = r * cols + c;
            if (nodata[i]) continue;
            int seed = (r == 0 || c == 0 || r == rows - 1 || c == cols - 1);
            for (int k = 1; k <= 8 && !seed; ++k) {
                int64_t rr = r + SDR[k], cc = c + SDC[k];
                if (nodata[rr * cols + cc]) seed = 1;
            }
            if (seed) {
                closed[i] = 1;
                if (rheap_push(&h, z[i], i)) { rc = -1; break; }
            }
        }
    }
    while (!rc && h.size > 0) {
        float tz;
        int64_t ti;
        if (rheap_pop(&h, &tz, &ti)) { rc = -1; break; }
        int64_t r = ti / cols, c = ti % cols;
        for (int k = 1; k <= 8; k += kstep) {
            int64_t rr = r + SDR[k], cc = c + SDC[k];
            if (rr < 0 || cc < 0 || rr >= rows || cc >= cols) continue;
            int64_t j = rr * cols + cc;
            if (closed[j] || nodata[j]) continue;
            closed[j] = 1;
            if (z[j] <= tz) {
                float lim = tz + eps;
                if (!(lim > tz)) lim = nextafterf(tz, INFINITY);
                z[j] = lim;
            }
            if (rheap_push(&h, z[j], j)) { rc = -1; break; }
        }
    }
    free(closed);
    rheap_free(&h);
    return rc;
}

/*
 * D8 steepest descent (O'Callaghan & Mark 1984, cited in the paper's Section 2):
 * slope = drop / distance with distance 1 or sqrt(2); strict '>' so the first
 * neighbour in E..SE order wins ties.  Edge cells drain off-grid: edge rows and
 * columns point outward perpendicular to the edge, corners diagonally.  A valid
 * cell with no strictly lower valid neighbour points into its first NoData
 * neighbour (E..SE order) if it has one, else gets NoFlow.
 */
void synth_d8(const float *z, const uint8_t *nodata, int64_t rows, int64_t cols,
              uint8_t *codes) {
    const double inv_sqrt2 = 0.70710678118654752440;
    for (int64_t r = 0; r < rows; ++r) {
        for (int64_t c = 0; c < cols; ++c) {
            int64_t i = r * cols + c;
            if (nodata[i]) { codes[i] = 0; continue; }
            int top = r == 0, bot = r == rows - 1, lef = c == 0, rig = c == cols - 1;
            if (top || bot || lef || rig) {
                uint8_t k;
                if (top && lef) k = 4;        /* NW */
                else if (top && rig) k = 2;   /* NE */
                else if (bot && lef) k = 6;   /* SW */
                else if (bot && rig) k = 8;   /* SE */
                else if (top) k = 3;          /* N */
                else if (bot) k = 7;          /* S */
                else if (lef) k = 5;          /* W */
                else k = 1;                   /* E */
                codes[i] = k;
                continue;
            }
            double best = 0.0;
            uint8_t code = 0, first_nodata = 0;
            for (int k = 1; k <= 8; ++k) {
                int64_t j = (r + SDR[k]) * cols + (c + SDC[k]);
                if (nodata[j]) {
                    if (!first_nodata) first_nodata = (uint8_t)k;
                    continue;
                }
                double drop = (double)z[i] - (double)z[j];
                double s = (k & 1) ? drop : drop * inv_sqrt2; /* odd codes are E,N,W,S */
                if (s > best) { best = s; code = (uint8_t)k; }
            }
            if (!code) code = first_nodata ? first_nodata : 9;
            codes[i] = code;
        }
    }
}

/* Bilinear upsampling by an integer factor f (cell centres aligned), used for
 * the coarse-to-fine scale raster. out has (rows*f) x (cols*f) cells. */
void synth_bilinear_up(const float *in, int64_t rows, int64_t cols, int64_t f, float *out) {
    int64_t R = rows * f, C = cols * f;
    for (int64_t r = 0; r < R; ++r) {
        double y = ((double)r + 0.5) / (double)f - 0.5;
        if (y < 0) y = 0;
        if (y > rows - 1) y = (double)(rows - 1);
        int64_t y0 = (int64_t)y;
        int64_t y1 = y0 + 1 < rows ? y0 + 1 : y0;
        double fy = y - (double)y0;
        for (int64_t c = 0; c < C; ++c) {
            double x = ((double)c + 0.5) / (double)f - 0.5;
            if (x < 0) x = 0;
            if (x > cols - 1) x = (double)(cols - 1);
            int64_t x0 = (int64_t)x;
            int64_t x1 = x0 + 1 < cols ? x0 + 1 : x0;
            double fx = x - (double)x0;
            double a = in[y0 * cols + x0], b = in[y0 * cols + x1];
            double cc = in[y1 * cols + x0], d = in[y1 * cols + x1];
            double v = (a * (1.0 - fx) + b * fx) * (1.0 - fy) + (cc * (1.0 - fx) + d * fx) * fy;
            out[r * C + c] = (float)v;
        }
    }
}
