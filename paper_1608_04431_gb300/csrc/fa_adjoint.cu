// Adjoint (transpose) of D8 flow accumulation.
//
// Accumulation is linear in the weights: with P the one-successor flow matrix
// (Eq. 1 with alpha in {0,1}), A = (I - P)^-1 w.  The gradient of a loss L with
// respect to w is therefore lam = (I - P)^-T g with g = dL/dA, i.e.
//     lam(c) = g(c) + lam(d(c)),
// the sum of g along c's downstream path.  Path sums suit pointer jumping
// (each cell has one successor), so every level here is a gather that reads
// only the previous round: no atomics, fixed summation structure, bitwise
// reproducible.
//
//   pass 1  k_adj_tile<1>  per tile: in-tile path sums lam_loc and the last
//                          in-tile cell of every path by pointer jumping in
//                          shared memory; emits lam_loc on perimeter slots and
//                          the exit link of every perimeter slot (the same
//                          links Algorithm 2 defines).
//   forest  k_adj_*        out(e) = lam(d(e)) = lam_loc(d(e)) + out(succ(e))
//                          over the exit forest, pointer jumping on global
//                          arrays, one gather round per launch.
//   pass 2  k_adj_tile<2>  recompute the tile (EVICT) with g'(e) = g(e) + out(e)
//                          at exit cells, which carries each exit's downstream
//                          remainder to every cell upstream of it; write lam.
#include "fa_common.cuh"
#include "fa_internal.h"

namespace fa {

constexpr uint16_t IDX_NONE = 0xFFFF;

struct AdjArgs {
    int64_t rows, cols;
    int th, tw, tiles_x, pmax;
    const uint8_t *codes;
    int64_t pc;
    int nib;  // codes packed two per byte: column c in byte c / 2, odd c high nibble
    const uint8_t *mask;
    int64_t pm;
    const float *g;
    int64_t pg;
    float *out;
    int64_t po;
    uint32_t *nexit;
    uint16_t *link;
    uint32_t *node_dst;
    FF *lam_slot;  // [T*pmax] lam_loc on perimeter slots (pass 1)
    const FF *outv;  // [T*pmax] out(e) per exit rank (pass 2)
    StatusBlock *st;
};

__host__ __device__ inline size_t adj_smem_bytes(int th, int tw) {
    size_t nh = (size_t)(th + 2) * (tw + 2);
    size_t b = 2 * nh * sizeof(FF);          // S double buffer
    b += 2 * nh * sizeof(uint16_t);          // J double buffer
    b += 2 * nh * sizeof(uint16_t);          // R double buffer
    b += nh;                                 // effective codes
    b = (b + 1) & ~size_t(1);
    b += (size_t)(2 * th + 2 * tw) * 2;      // exit ranks
    return b;
}

template <int PASS>
__global__ void __launch_bounds__(256) k_adj_tile(AdjArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_warp[33];
    __shared__ int s_cyc, s_nonfinite;
    __shared__ long long s_first;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int t = blockIdx.x;
    const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
    const int64_t R0 = (int64_t)ty * a.th, C0 = (int64_t)tx * a.tw;
    const int h = (int)min((int64_t)a.th, a.rows - R0);
    const int w = (int)min((int64_t)a.tw, a.cols - C0);
    const int W2 = w + 2, NH = (h + 2) * W2;
    const int NHmax = (a.th + 2) * (a.tw + 2);
    const int n_in = h * w;

    FF *S0 = reinterpret_cast<FF *>(smem);
    FF *S1 = S0 + NHmax;
    uint16_t *J0 = reinterpret_cast<uint16_t *>(S1 + NHmax);
    uint16_t *J1 = J0 + NHmax;
    uint16_t *Rr0 = J1 + NHmax;
    uint16_t *Rr1 = Rr0 + NHmax;
    uint8_t *ec = reinterpret_cast<uint8_t *>(Rr1 + NHmax);
    uint16_t *rank = reinterpret_cast<uint16_t *>(
        (reinterpret_cast<uintptr_t>(ec + NHmax) + 1) & ~uintptr_t(1));

    if (tid == 0) {
        s_cyc = 0;
        s_nonfinite = 0;
        s_first = NO_INDEX;
    }
    for (int i = tid; i < NH; i += nt) {
        const int hr = i / W2, hc = i - hr * W2;
        const int64_t gr = R0 - 1 + hr, gc = C0 - 1 + hc;
        uint8_t e = 0;
        if (gr >= 0 && gr < a.rows && gc >= 0 && gc < a.cols) {
            const uint32_t k = a.nib ? ((uint32_t)a.codes[gr * a.pc + (gc >> 1)] >> ((gc & 1) << 2)) & 15u
                                     : (uint32_t)a.codes[gr * a.pc + gc];
            const bool inside = hr >= 1 && hr <= h && hc >= 1 && hc <= w;
            if (k >= 1 && k <= 9 && !(a.mask && a.mask[gr * a.pm + gc]))
                e = k | (inside ? 0 : HALO);
        }
        ec[i] = e;
    }
    __syncthreads();

    // ---- round 0 state: S = g, J = in-tile successor, R = self ---------------
    int active = 0, nonfinite = 0;
    for (int j = tid; j < n_in; j += nt) {
        const int r = j / w, c = j - r * w;
        const int i = (r + 1) * W2 + (c + 1);
        const uint8_t e = ec[i];
        FF s{0.0f, 0.0f};
        uint16_t nx = IDX_NONE;
        if (e) {
            const float gv = a.g[(R0 + r) * a.pg + (C0 + c)];
            if ((__float_as_uint(gv) & 0x7fffffffu) >= 0x7f800000u) nonfinite = 1;
            s = FF{gv, 0.0f};
            const int k = e & 15;
            if (k <= 8) {
                const int n = i + off_of(k, W2);
                const uint8_t en = ec[n];
                if (en && !(en & HALO)) nx = (uint16_t)n;
            }
        }
        S0[i] = s;
        J0[i] = nx;
        Rr0[i] = (uint16_t)i;
        active |= nx != IDX_NONE;
    }
    __syncthreads();

    if constexpr (PASS == 2) {
        // fold each exit's downstream remainder out(e) into g(e)
        const int P = perim_count(h, w);
        const int chunk = (P + nt - 1) / nt;
        const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
        int mine = 0;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            if (k >= 1 && k <= 8 && (ec[i + off_of(k, W2)] & HALO)) ++mine;
        }
        int total;
        int rk = block_exclusive_scan(mine, s_warp, &total);
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            if (k >= 1 && k <= 8 && (ec[i + off_of(k, W2)] & HALO)) {
                S0[i] = ff_add(S0[i], a.outv[tbase + rk]);
                ++rk;
            }
        }
        __syncthreads();
    }

    // ---- pointer jumping: S_{k+1}(i) = S_k(i) + S_k(J_k(i)),
    //      J_{k+1} = J_k o J_k, R_{k+1}(i) = R_k(J_k(i)) (last cell reached) ----
    FF *Sc = S0, *Sn = S1;
    uint16_t *Jc = J0, *Jn = J1, *Rc = Rr0, *Rn = Rr1;
    int maxr = 1;
    while ((1 << maxr) <= n_in) ++maxr;
    ++maxr;
    active = __syncthreads_or(active);
    int round = 0;
    for (; round < maxr && active; ++round) {
        int act = 0;
        for (int j = tid; j < n_in; j += nt) {
            const int r = j / w, c = j - r * w;
            const int i = (r + 1) * W2 + (c + 1);
            const uint16_t nx = Jc[i];
            if (nx != IDX_NONE) {
                Sn[i] = ff_add(Sc[i], Sc[nx]);
                const uint16_t nn = Jc[nx];
                Jn[i] = nn;
                Rn[i] = Rc[nx];
                act |= nn != IDX_NONE;
            } else {
                Sn[i] = Sc[i];
                Jn[i] = IDX_NONE;
                Rn[i] = Rc[i];
            }
        }
        active = __syncthreads_or(act);
        FF *ts = Sc; Sc = Sn; Sn = ts;
        uint16_t *tj = Jc; Jc = Jn; Jn = tj;
        uint16_t *tr = Rc; Rc = Rn; Rn = tr;
    }
    // cells whose jumps never ended sit on (or upstream of) an in-tile cycle
    int ncyc = 0;
    long long fcyc = NO_INDEX;
    if (active) {
        for (int j = tid; j < n_in; j += nt) {
            const int r = j / w, c = j - r * w;
            const int i = (r + 1) * W2 + (c + 1);
            if (Jc[i] != IDX_NONE) {
                ++ncyc;
                fcyc = min(fcyc, (long long)((R0 + r) * a.cols + (C0 + c)));
            }
        }
    }

    if constexpr (PASS == 1) {
        const int P = perim_count(h, w);
        const int chunk = (P + nt - 1) / nt;
        const int s0 = min(P, tid * chunk), s1 = min(P, s0 + chunk);
        int mine = 0;
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            if (k >= 1 && k <= 8 && (ec[i + off_of(k, W2)] & HALO)) ++mine;
        }
        int total;
        int rk = block_exclusive_scan(mine, s_warp, &total);
        for (int s = s0; s < s1; ++s) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            const int k = ec[i] & 15;
            const bool ex = k >= 1 && k <= 8 && (ec[i + off_of(k, W2)] & HALO);
            rank[s] = ex ? (uint16_t)rk++ : LINK_TERM;
        }
        __syncthreads();
        const size_t tbase = (size_t)t * a.pmax;
        for (int s = tid; s < P; s += nt) {
            int r, c;
            cell_of(s, h, w, r, c);
            const int i = (r + 1) * W2 + (c + 1);
            uint16_t lk = LINK_TERM;
            if (ec[i] && Jc[i] == IDX_NONE) {
                const int last = Rc[i];
                const int k = ec[last] & 15;
                if (k >= 1 && k <= 8 && (ec[last + off_of(k, W2)] & HALO)) {
                    const int lr = last / W2 - 1, lc = last - (last / W2) * W2 - 1;
                    lk = rank[slot_of(lr, lc, h, w)];
                }
            }
            a.link[tbase + s] = lk;
            a.lam_slot[tbase + s] = Sc[i];
            const uint16_t myrank = rank[s];
            if (myrank != LINK_TERM) {
                const int k = ec[i] & 15;
                const int64_t gr = R0 + r + dir_dr(k), gc = C0 + c + dir_dc(k);
                const int tyd = (int)(gr / a.th), txd = (int)(gc / a.tw);
                const int hd = (int)min((int64_t)a.th, a.rows - (int64_t)tyd * a.th);
                const int wd = (int)min((int64_t)a.tw, a.cols - (int64_t)txd * a.tw);
                const int sd = slot_of((int)(gr - (int64_t)tyd * a.th),
                                       (int)(gc - (int64_t)txd * a.tw), hd, wd);
                a.node_dst[tbase + myrank] =
                    (uint32_t)(((size_t)tyd * a.tiles_x + txd) * a.pmax + sd);
            }
        }
        if (tid == 0) a.nexit[t] = (uint32_t)total;
        ncyc = warp_sum(ncyc);
        fcyc = warp_min_ll(fcyc);
        nonfinite = warp_sum(nonfinite);
        if ((tid & 31) == 0) {
            if (ncyc) atomicAdd(&s_cyc, ncyc);
            if (fcyc != NO_INDEX) atomicMin(&s_first, fcyc);
            if (nonfinite) atomicOr(&s_nonfinite, 1);
        }
        __syncthreads();
        if (tid == 0) {
            int fl = (s_cyc ? FA_FLAG_CYCLE : 0) | (s_nonfinite ? FA_FLAG_NONFINITE : 0);
            if (fl) status_report(a.st, fl, s_cyc, s_first);
        }
    } else {
        for (int j = tid; j < n_in; j += nt) {
            const int r = j / w, c = j - r * w;
            const int i = (r + 1) * W2 + (c + 1);
            a.out[(size_t)(R0 + r) * a.po + (C0 + c)] = ec[i] ? ff_round(Sc[i]) : 0.0f;
        }
    }
}

// ---------------------------------------------------------------------------
// exit forest: out(e) = c(e) + out(succ(e)), c(e) = lam_loc(d(e))
// ---------------------------------------------------------------------------
struct AdjForest {
    int64_t tiles;
    int pmax;
    const uint32_t *nexit;
    const uint16_t *link;
    const uint32_t *node_dst;
    const FF *lam_slot;
    FF *v0, *v1, *outv;
    uint32_t *J0, *J1;
    uint32_t *misc;  // [1 + k] nodes still jumping after round k
    StatusBlock *st;
};

__global__ void k_adj_forest_init(AdjForest f) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const uint32_t dst = f.node_dst[node];
        f.v0[node] = f.lam_slot[dst];
        const uint16_t l = f.link[dst];
        f.J0[node] = l == LINK_TERM ? NODE_NONE : (dst / f.pmax) * f.pmax + l;
    }
}

__global__ void k_adj_forest_round(AdjForest f, int k) {
    if (k > 0 && f.misc[k] == 0) return;  // every path already ended
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    const FF *vc = (k & 1) ? f.v1 : f.v0;
    FF *vn = (k & 1) ? f.v0 : f.v1;
    const uint32_t *Jc = (k & 1) ? f.J1 : f.J0;
    uint32_t *Jn = (k & 1) ? f.J0 : f.J1;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int nact = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        const uint32_t jj = Jc[node];
        if (jj != NODE_NONE) {
            vn[node] = ff_add(vc[node], vc[jj]);
            const uint32_t nn = Jc[jj];
            Jn[node] = nn;
            nact += nn != NODE_NONE;
        } else {
            vn[node] = vc[node];
            Jn[node] = NODE_NONE;
        }
    }
    nact = warp_sum(nact);
    if (lane == 0 && nact) atomicAdd(&f.misc[1 + k], (uint32_t)nact);
}

// the last executed round m is the first with no node still jumping; its
// output sits in buffer (m + 1) & 1
__global__ void k_adj_forest_final(AdjForest f, int kmax) {
    const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= f.tiles) return;
    int m = 0;
    while (m < kmax - 1 && f.misc[1 + m] != 0) ++m;
    const bool cyc = f.misc[1 + m] != 0;
    const FF *vf = ((m + 1) & 1) ? f.v1 : f.v0;
    const uint32_t *Jf = ((m + 1) & 1) ? f.J1 : f.J0;
    const uint32_t n = f.nexit[tile];
    const size_t base = (size_t)tile * f.pmax;
    int ncyc = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const size_t node = base + j;
        f.outv[node] = vf[node];
        if (cyc && Jf[node] != NODE_NONE) ++ncyc;
    }
    ncyc = warp_sum(ncyc);
    if (lane == 0 && ncyc) status_report(f.st, FA_FLAG_CYCLE, ncyc, NO_INDEX);
}

__global__ void k_adj_init_status(StatusBlock *st, uint32_t *misc, int nmisc) {
    const int i = threadIdx.x;
    if (i == 0) {
        st->flags = 0;
        st->count = 0;
        st->first = NO_INDEX;
    }
    for (int j = i; j < nmisc; j += blockDim.x) misc[j] = 0;
}

// ---------------------------------------------------------------------------
size_t carve_adjoint(void *ws, size_t bytes, const Geom &g, AdjWork &w) {
    Carver c(ws, bytes);
    const size_t T = (size_t)g.tiles(), S = T * g.pmax;
    FwdWork fw;
    carve_forward(nullptr, 0, g, fw, true);
    w.kmax = fw.kmax;
    w.status = c.take<uint8_t>(64);
    w.misc = c.take<uint32_t>(2 + w.kmax);
    w.nexit = c.take<uint32_t>(T);
    w.link = c.take<uint16_t>(S);
    w.node_dst = c.take<uint32_t>(S);
    w.lam_slot = c.take<uint64_t>(S);
    w.v0 = c.take<uint64_t>(S);
    w.v1 = c.take<uint64_t>(S);
    w.outv = c.take<uint64_t>(S);
    w.J0 = c.take<uint32_t>(S);
    w.J1 = c.take<uint32_t>(S);
    return c.used() + 256;
}

template <int PASS>
static cudaError_t launch_adj_tile(const Geom &g, const AdjArgs &aa, cudaStream_t s) {
    const size_t smem = adj_smem_bytes(g.th, g.tw);
    static int configured = 0;
    if (smem > 48 * 1024 && configured < (int)smem) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_tile<PASS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = (int)smem;
    }
    const int cells = g.th * g.tw;
    const int nt = cells >= 256 ? 256 : ((cells + 31) / 32) * 32;
    k_adj_tile<PASS><<<(unsigned)g.tiles(), nt, smem, s>>>(aa);
    return cudaGetLastError();
}

bool adjoint_fits(const Geom &g) { return adj_smem_bytes(g.th, g.tw) <= 227 * 1024; }

cudaError_t launch_adjoint(const Geom &g, const uint8_t *codes, int64_t pc, const uint8_t *mask,
                           int64_t pm, const float *gin, int64_t pg, float *out, int64_t po,
                           const AdjWork &ws, void *status, cudaStream_t s) {
    StatusBlock *st = reinterpret_cast<StatusBlock *>(status ? status : ws.status);
    k_adj_init_status<<<1, 64, 0, s>>>(st, ws.misc, 2 + ws.kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (g.rows == 0 || g.cols == 0) return cudaSuccess;

    AdjArgs aa;
    aa.rows = g.rows;
    aa.cols = g.cols;
    aa.th = g.th;
    aa.tw = g.tw;
    aa.tiles_x = g.tiles_x;
    aa.pmax = g.pmax;
    aa.codes = codes;
    aa.pc = pc;
    aa.nib = g.code_format == FA_CODES_NIBBLE;
    aa.mask = mask;
    aa.pm = pm;
    aa.g = gin;
    aa.pg = pg;
    aa.out = out;
    aa.po = po;
    aa.nexit = ws.nexit;
    aa.link = ws.link;
    aa.node_dst = ws.node_dst;
    aa.lam_slot = reinterpret_cast<FF *>(ws.lam_slot);
    aa.outv = reinterpret_cast<const FF *>(ws.outv);
    aa.st = st;
    timing_mark(0, s);
    e = launch_adj_tile<1>(g, aa, s);
    if (e != cudaSuccess) return e;
    timing_mark(1, s);

    AdjForest f;
    f.tiles = g.tiles();
    f.pmax = g.pmax;
    f.nexit = ws.nexit;
    f.link = ws.link;
    f.node_dst = ws.node_dst;
    f.lam_slot = reinterpret_cast<const FF *>(ws.lam_slot);
    f.v0 = reinterpret_cast<FF *>(ws.v0);
    f.v1 = reinterpret_cast<FF *>(ws.v1);
    f.outv = reinterpret_cast<FF *>(ws.outv);
    f.J0 = ws.J0;
    f.J1 = ws.J1;
    f.misc = ws.misc;
    f.st = st;
    const unsigned fb = (unsigned)((f.tiles * 32 + 255) / 256);
    k_adj_forest_init<<<fb, 256, 0, s>>>(f);
    for (int k = 0; k < ws.kmax; ++k) k_adj_forest_round<<<fb, 256, 0, s>>>(f, k);
    k_adj_forest_final<<<fb, 256, 0, s>>>(f, ws.kmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    timing_mark(2, s);
    e = launch_adj_tile<2>(g, aa, s);
    timing_mark(3, s);
    timing_set_count(3);
    return e;
}

}  // namespace fa
