// Series actions and the downward pass (Sections 3 and 6, Figs. 7-8).
//
//   DH  (EVALM, Lemma 4): every query of Q adds
//        sum_{|a|<p} A_a h_a((x_q - x_R)/s),  A_a = M_a(R) s^-|a|,
//   DL  (DIRECTL, Lemma 5): Q's local coefficients gain
//        B_b += (1/b!) sum_{r in R} w_r h_b((x_r - x_Q)/s),
//   H2L (Lemma 1 / Lemma 6): B_b += ((-1)^|b| / b!) sum_{|a|<p} A_a h_{a+b}((x_Q - x_R)/s),
//   downward pass (Fig. 8): the FD estimates of every ancestor and the local
//        expansion shifted by L2L (Lemma 3) to each leaf, evaluated there
//        (EVALL) and added to the base-case and DH sums.
// Multivariate Hermite functions are evaluated as e^{-|t|^2} prod_d H_{a_d}(t_d)
// with the physicists' polynomials from the three-term recurrence.  All of
// this is FP64 (it touches few pairs; its rounding is far below eps).
#include <math.h>

#include "gs_frontier.cuh"
#include "gs_internal.h"
#include "gs_tree.cuh"

namespace gs {

constexpr int kSerTB = 128;
constexpr int kMaxT = 1024;      // series terms supported by the DL / H2L kernels
constexpr int kMaxDP = 64;       // D * (orders) table entries per point
constexpr int kLaneT = 20;       // H2L lane-per-action path: at most kLaneT terms
constexpr int kDlLane = 32;      // DL lane-per-reference path: at most kDlLane coefficients
constexpr int kDlStride = 33;    //   accumulator row stride (doubles)
constexpr int kLaneH = 32;       //   and kLaneH Hermite values (D (2p - 1))

struct SeriesParams {
    int D, nh, P, T;
    SeriesTables tb;
    const void *qxs, *rxs;
    int dtype;
    const int32_t *rperm;
    const float *w;
    int64_t qn, rn;
    const double *qcenter, *rcenter;
    const double *rmom;
    const double *inv_s;     // 1 / sqrt(2 h_j^2)
    double *Gq;              // sorted queries x nh
    double *B;               // query nodes x nh x T
    int32_t *pL;             // query nodes x nh
    const double *est;       // query nodes x nh FD estimates
    const int32_t *qperm;
    double *out;             // caller order, M x nh
    int q_depth;
};

__device__ __forceinline__ int node_depth(int64_t node) { return 63 - __clzll(node + 1); }

__device__ __forceinline__ double coord(const void *xs, int dtype, int64_t p, int D, int d) {
    return dtype == GS_F64 ? ((const double *)xs)[p * D + d] : (double)((const float *)xs)[p * D + d];
}

// H_0..H_{n-1}(t) into h[0..n)
__device__ __forceinline__ void hermite_polys(double t, int n, double *h) {
    h[0] = 1.0;
    if (n > 1) h[1] = 2.0 * t;
    for (int k = 1; k + 1 < n; ++k) h[k + 1] = 2.0 * t * h[k] - 2.0 * k * h[k - 1];
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory layout of the series kernels: the multi-index exponent
// table (T x D bytes) and degrees (T bytes) of the whole order-P set, then
// one region per warp.
__device__ __forceinline__ void load_tables(const SeriesTables &tb, int D, uint8_t *al_s, uint8_t *dg_s) {
    for (int i = threadIdx.x; i < tb.T * D; i += blockDim.x) al_s[i] = tb.alpha[i];
    for (int i = threadIdx.x; i < tb.T; i += blockDim.x) dg_s[i] = tb.deg[i];
    __syncthreads();
}

__host__ __device__ inline int table_bytes(int T, int D) { return ((T * D + 7) / 8 + (T + 7) / 8) * 8; }

// Work chunks: a DH action over a large query node or a DL action over a
// large reference node is split into pieces of kChunk (DH) or kChunkDL (DL)
// points -- DL pieces are larger because each piece ends with one atomic add
// per coefficient into the query node's expansion, which all pieces of an
// action share; piece counts
// are prefix-summed and warps take pieces from the flattened list.
constexpr int kChunk = 64;
constexpr int kChunkDL = 512;

__global__ void k_chunk_count(const SeriesEntry *__restrict__ ent, int64_t ne, int use_q, int64_t nq, int64_t nr,
                              long long *cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = use_q ? ent[e].q : ent[e].r;
        const int dd = node_depth(node);
        const int64_t ii = node - ((1ll << dd) - 1);
        const int64_t n = use_q ? nq : nr;
        const int64_t c = level_begin(n, dd, ii + 1) - level_begin(n, dd, ii);
        const int chunk = use_q ? kChunk : kChunkDL;
        cnt[e] = (c + chunk - 1) / chunk;
    }
}

// entry owning flattened piece c (off = exclusive prefix of piece counts)
__device__ __forceinline__ int64_t owner(const long long *off, int64_t ne, long long c) {
    int64_t lo = 0, hi = ne - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// DH: one warp per piece of kChunk queries; lanes over queries; per-lane
// Hermite polynomial tables in shared memory (lane-minor, conflict-free)
// ---------------------------------------------------------------------------
__global__ void k_series_dh(SeriesParams sp, const SeriesEntry *__restrict__ ent, int64_t ne,
                            const long long *__restrict__ off, const long long *__restrict__ npieces) {
    extern __shared__ double smem_d[];
    const int D = sp.D, T = sp.T, P = sp.P;
    uint8_t *al_s = (uint8_t *)smem_d;
    uint8_t *dg_s = al_s + ((T * D + 7) / 8) * 8;
    load_tables(sp.tb, D, al_s, dg_s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *A = smem_d + table_bytes(T, D) / 8 + (size_t)w * (T + D * P * 32);
    double *Hs = A + T;
    const long long C = *npieces;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (long long c = blockIdx.x * (int64_t)(blockDim.x >> 5) + w; c < C; c += warps) {
        const int64_t e = owner(off, ne, c);
        const SeriesEntry E = ent[e];
        const int p = E.p, Tp = sp.tb.Tp[p];
        const double is = sp.inv_s[E.j];
        const double *mom = sp.rmom + (int64_t)E.r * T;
        __syncwarp();
        for (int a = lane; a < Tp; a += 32) {
            double v = mom[a];
            for (int k = 0; k < dg_s[a]; ++k) v *= is;
            A[a] = v;
        }
        __syncwarp();
        const double *cR = sp.rcenter + (int64_t)E.r * D;
        const int qd = node_depth(E.q);
        const int64_t qi = E.q - ((1ll << qd) - 1);
        const int64_t b = level_begin(sp.qn, qd, qi) + (c - off[e]) * kChunk;
        const int64_t en = min(b + kChunk, level_begin(sp.qn, qd, qi + 1));
        for (int64_t pos = b + lane; pos < en; pos += 32) {
            double t2 = 0.0;
            for (int d = 0; d < D; ++d) {
                const double t = (coord(sp.qxs, sp.dtype, pos, D, d) - cR[d]) * is;
                double h0 = 1.0, h1 = 2.0 * t;
                Hs[(d * p) * 32 + lane] = h0;
                if (p > 1) Hs[(d * p + 1) * 32 + lane] = h1;
                for (int k = 1; k + 1 < p; ++k) {
                    const double h2 = 2.0 * t * h1 - 2.0 * k * h0;
                    Hs[(d * p + k + 1) * 32 + lane] = h2;
                    h0 = h1;
                    h1 = h2;
                }
                t2 += t * t;
            }
            double s = 0.0;
            for (int a = 0; a < Tp; ++a) {
                const uint8_t *al = al_s + a * D;
                double pr = A[a];
                for (int d = 0; d < D; ++d) pr *= Hs[(d * p + al[d]) * 32 + lane];
                s += pr;
            }
            atomicAdd(&sp.Gq[pos * sp.nh + E.j], s * exp(-t2));
        }
    }
}

// ---------------------------------------------------------------------------
// DL: one warp per piece of kChunkDL references.  Up to kDlLane coefficients:
// lanes over references, each adding its references' contributions to every
// coefficient in its own row of a shared accumulator (row stride 33 doubles,
// so both the row-wise adds and the column sums are conflict-free), then
// lanes over coefficients sum the 32 rows.  More coefficients: lanes over the
// coefficients b, the piece's references in groups of 32 with their Hermite
// tables built cooperatively.  Partial coefficients are added atomically.
// ---------------------------------------------------------------------------
__global__ void k_series_dl(SeriesParams sp, const SeriesEntry *__restrict__ ent, int64_t ne,
                            const long long *__restrict__ off, const long long *__restrict__ npieces) {
    extern __shared__ double smem_d[];
    const int D = sp.D, T = sp.T, P = sp.P;
    uint8_t *al_s = (uint8_t *)smem_d;
    uint8_t *dg_s = al_s + ((T * D + 7) / 8) * 8;
    load_tables(sp.tb, D, al_s, dg_s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int DPp = D * P;
    double *Hr = smem_d + table_bytes(T, D) / 8 + (size_t)w * (32 * DPp + 32 + 32 * kDlStride);
    double *we = Hr + 32 * DPp;
    double *acc_s = we + 32;   // [32 lanes][kDlStride]
    const long long C = *npieces;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (long long c = blockIdx.x * (int64_t)(blockDim.x >> 5) + w; c < C; c += warps) {
        const int64_t e = owner(off, ne, c);
        const SeriesEntry E = ent[e];
        const int p = E.p, Tp = sp.tb.Tp[p];
        const double is = sp.inv_s[E.j];
        const double *cQ = sp.qcenter + (int64_t)E.q * D;
        const int rd = node_depth(E.r);
        const int64_t ri = E.r - ((1ll << rd) - 1);
        const int64_t rb = level_begin(sp.rn, rd, ri) + (c - off[e]) * kChunkDL;
        const int64_t re = min(rb + kChunkDL, level_begin(sp.rn, rd, ri + 1));
        double *Bq = sp.B + ((int64_t)E.q * sp.nh + E.j) * T;
        if (Tp <= kDlLane) {
            double *row = acc_s + lane * kDlStride;
            double *H = Hr + lane * DPp;
            for (int bt = 0; bt < Tp; ++bt) row[bt] = 0.0;
            for (int64_t pos = rb + lane; pos < re; pos += 32) {
                double v2 = 0.0;
                for (int d = 0; d < D; ++d) {
                    const double v = (coord(sp.rxs, sp.dtype, pos, D, d) - cQ[d]) * is;
                    hermite_polys(v, p, &H[d * p]);
                    v2 += v * v;
                }
                const double wr = (double)sp.w[sp.rperm[pos]] * exp(-v2);
                for (int bt = 0; bt < Tp; ++bt) {
                    const uint8_t *be = al_s + bt * D;
                    double pr = wr;
                    for (int d = 0; d < D; ++d) pr *= H[d * p + be[d]];
                    row[bt] += pr;
                }
            }
            __syncwarp();
            for (int bt = lane; bt < Tp; bt += 32) {
                double sum = 0.0;
                for (int l = 0; l < 32; ++l) sum += acc_s[l * kDlStride + bt];
                atomicAdd(&Bq[bt], sum * sp.tb.inv_fact[bt]);
            }
            __syncwarp();
            if (lane == 0) atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], p);
            continue;
        }
        for (int b0 = 0; b0 < Tp; b0 += 32) {
            const int bt = b0 + lane;
            const uint8_t *be = al_s + (bt < Tp ? bt : 0) * D;
            double acc = 0.0;
            for (int64_t c0 = rb; c0 < re; c0 += 32) {
                const int nc = (int)min((int64_t)32, re - c0);
                __syncwarp();
                if (lane < nc) {
                    const int64_t pos = c0 + lane;
                    double v2 = 0.0;
                    double *H = Hr + lane * DPp;
                    for (int d = 0; d < D; ++d) {
                        const double v = (coord(sp.rxs, sp.dtype, pos, D, d) - cQ[d]) * is;
                        hermite_polys(v, p, &H[d * p]);
                        v2 += v * v;
                    }
                    we[lane] = (double)sp.w[sp.rperm[pos]] * exp(-v2);
                }
                __syncwarp();
                if (bt < Tp) {
                    for (int r = 0; r < nc; ++r) {
                        const double *H = Hr + r * DPp;
                        double pr = we[r];
                        for (int d = 0; d < D; ++d) pr *= H[d * p + be[d]];
                        acc += pr;
                    }
                }
            }
            if (bt < Tp) atomicAdd(&Bq[bt], acc * sp.tb.inv_fact[bt]);
        }
        if (lane == 0) atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], p);
    }
}

// ---------------------------------------------------------------------------
// H2L.  Warps take tiles of 32 consecutive actions.  Orders 1 and 2 (the
// bulk of the actions: one and 1 + D coefficients) take one lane each, with
// the Lemma 1 sums written out (H_1(t) = 2t, H_2(t) = 4t^2 - 2):
//   b = 0:    s_0   = A_0 + sum_i A_{e_i} H_1(t_i),
//   b = e_k:  s_e_k = H_1(t_k) (s_0 - A_{e_k} H_1(t_k)) + A_{e_k} H_2(t_k)
//                   = 2 (t_k s_0 - A_{e_k}),
// B_b += (-1)^|b| e^{-|t|^2} s_b.  When all 32 actions of a tile add into
// the same (Q, h) they are summed across the warp first.  Middle orders
// (at most kLaneT terms) also take one lane each, with A_a and the 1-D
// Hermite polynomials of t = (x_Q - x_R)/s (orders 0 .. 2p-2) in a
// lane-interleaved shared buffer.  Higher orders are done one at a time by
// the whole warp: lanes over b, loop over a.
// ---------------------------------------------------------------------------
__global__ void k_series_h2l(SeriesParams sp, FrontierState *__restrict__ fs, const SeriesEntry *__restrict__ ent,
                             const unsigned long long *__restrict__ ne_end) {
    extern __shared__ double smem_d[];
    const int D = sp.D, T = sp.T, P = sp.P;
    uint8_t *al_s = (uint8_t *)smem_d;
    uint8_t *dg_s = al_s + ((T * D + 7) / 8) * 8;
    load_tables(sp.tb, D, al_s, dg_s);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nHmax = 2 * P - 1;
    double *A = smem_d + table_bytes(T, D) / 8 + (size_t)w * (T + D * nHmax);
    double *Hs = A + T;
    double *lanebuf = smem_d + table_bytes(T, D) / 8 + (size_t)(blockDim.x >> 5) * (T + D * nHmax) +
                      (size_t)w * 32 * (kLaneT + kLaneH);
    // the whole list, or the general bucket of a bucketed list
    const int64_t ne = ne_end ? (int64_t)*ne_end : fs->series_count[2];
    const unsigned full = 0xffffffffu;
    // tiles are taken in list order from a counter: the high-order actions
    // of the upper levels come first and the cheap leaf-level ones fill in
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(&fs->work, 1ull);
        const int64_t t0 = (int64_t)__shfl_sync(full, tile, 0) * 32;
        if (t0 >= ne) break;
        const int64_t e = t0 + lane;
        SeriesEntry E;
        E.q = 0; E.r = 0; E.j = 0; E.p = 0; E.method = 0;
        if (e < ne) E = ent[e];
        // ---- orders 1 and 2: one lane per action
        const bool small = E.p >= 1 && E.p <= 2;
        double s0 = 0.0, et = 0.0;
        double is = 0.0;
        const double *mom = sp.rmom + (int64_t)E.r * T;
        const double *cq = sp.qcenter + (int64_t)E.q * D, *cr = sp.rcenter + (int64_t)E.r * D;
        if (small) {
            is = sp.inv_s[E.j];
            double t2 = 0.0;
            s0 = mom[0];
            for (int d = 0; d < D; ++d) {
                const double t = (cq[d] - cr[d]) * is;
                t2 += t * t;
                if (E.p == 2) s0 += (mom[1 + d] * is) * (2.0 * t);
            }
            et = exp(-t2);
        }
        const long long key = small ? (long long)E.q * sp.nh + E.j : -1 - lane;
        const bool uniform = __all_sync(full, key == __shfl_sync(full, key, 0));
        double *Bq = sp.B + (small ? key : 0) * T;
        if (uniform) {
            const double v = warp_sum_d(et * s0);
            const int pmax = __reduce_max_sync(full, E.p);
            if (lane == 0) {
                atomicAdd(&Bq[0], v);
                atomicMax(&sp.pL[key], pmax);
            }
            if (pmax == 2) {
                const double m2et = -2.0 * et;
                for (int k = 0; k < D; ++k) {
                    double u = 0.0;
                    if (E.p == 2) u = m2et * ((cq[k] - cr[k]) * is * s0 - mom[1 + k] * is);
                    u = warp_sum_d(u);
                    if (lane == 0) atomicAdd(&Bq[1 + k], u);
                }
            }
        } else if (small) {
            atomicAdd(&Bq[0], et * s0);
            atomicMax(&sp.pL[key], (int)E.p);
            if (E.p == 2) {
                const double m2et = -2.0 * et;
                for (int k = 0; k < D; ++k) atomicAdd(&Bq[1 + k], m2et * ((cq[k] - cr[k]) * is * s0 - mom[1 + k] * is));
            }
        }
        // ---- middle orders (T_p <= kLaneT, D (2p-1) <= kLaneH): one lane per
        // action, its A_a and Hermite values in a lane-interleaved buffer
        const bool mid = E.p > 2 && sp.tb.Tp[E.p] <= kLaneT && D * (2 * E.p - 1) <= kLaneH;
        if (mid) {
            const int p = E.p, Tp = sp.tb.Tp[p], nH = 2 * p - 1;
            const double ism = sp.inv_s[E.j];
            double *Al = lanebuf + lane, *Hl = lanebuf + kLaneT * 32 + lane;
            for (int a = 0; a < Tp; ++a) {
                double v = mom[a];
                for (int k = 0; k < dg_s[a]; ++k) v *= ism;
                Al[a * 32] = v;
            }
            double t2 = 0.0;
            for (int d = 0; d < D; ++d) {
                const double tau = (cq[d] - cr[d]) * ism;
                t2 += tau * tau;
                double hm = 1.0, hc = 2.0 * tau;
                Hl[(d * nH) * 32] = 1.0;
                Hl[(d * nH + 1) * 32] = hc;
                for (int k = 1; k + 1 < nH; ++k) {
                    const double hn = 2.0 * tau * hc - 2.0 * k * hm;
                    Hl[(d * nH + k + 1) * 32] = hn;
                    hm = hc;
                    hc = hn;
                }
            }
            const double etm = exp(-t2);
            double *Bm = sp.B + ((int64_t)E.q * sp.nh + E.j) * T;
            for (int bt = 0; bt < Tp; ++bt) {
                const uint8_t *be = al_s + bt * D;
                double sacc = 0.0;
                for (int a = 0; a < Tp; ++a) {
                    const uint8_t *al = al_s + a * D;
                    double pr = Al[a * 32];
                    for (int d = 0; d < D; ++d) pr *= Hl[(d * nH + al[d] + be[d]) * 32];
                    sacc += pr;
                }
                const double sign = (dg_s[bt] & 1) ? -1.0 : 1.0;
                atomicAdd(&Bm[bt], sign * sp.tb.inv_fact[bt] * etm * sacc);
            }
            atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], p);
        }
        // ---- higher orders: the whole warp per action
        unsigned big = __ballot_sync(full, E.p > 2 && !mid);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const SeriesEntry Eb = ent[t0 + src];
            const int p = Eb.p, Tp = sp.tb.Tp[p];
            const int nH = 2 * p - 1;
            const double isb = sp.inv_s[Eb.j];
            const double *momb = sp.rmom + (int64_t)Eb.r * T;
            __syncwarp();
            for (int a = lane; a < Tp; a += 32) {
                double v = momb[a];
                for (int k = 0; k < dg_s[a]; ++k) v *= isb;
                A[a] = v;
            }
            double t2 = 0.0;
            if (lane < D) {
                const double tau = (sp.qcenter[(int64_t)Eb.q * D + lane] - sp.rcenter[(int64_t)Eb.r * D + lane]) * isb;
                hermite_polys(tau, nH, &Hs[lane * nH]);
                t2 = tau * tau;
            }
            t2 = warp_sum_d(t2);
            __syncwarp();
            const double etb = exp(-t2);
            double *Bb = sp.B + ((int64_t)Eb.q * sp.nh + Eb.j) * T;
            for (int bt = lane; bt < Tp; bt += 32) {
                const uint8_t *be = al_s + bt * D;
                double sacc = 0.0;
                for (int a = 0; a < Tp; ++a) {
                    const uint8_t *al = al_s + a * D;
                    double pr = A[a];
                    for (int d = 0; d < D; ++d) pr *= Hs[d * nH + al[d] + be[d]];
                    sacc += pr;
                }
                const double sign = (dg_s[bt] & 1) ? -1.0 : 1.0;
                atomicAdd(&Bb[bt], sign * sp.tb.inv_fact[bt] * etb * sacc);
            }
            if (lane == 0) atomicMax(&sp.pL[(int64_t)Eb.q * sp.nh + Eb.j], p);
        }
    }
}

// ---------------------------------------------------------------------------
// H2L in three dimensions, one lane per action.  The translation
//   C_beta = sum_{|alpha| < p} A_alpha prod_d h_{alpha_d + beta_d}(tau_d)
// separates over the dimensions, so it is summed one dimension at a time:
// for each a1,
//   X1[a2,b3] = sum_a3 A[a1,a2,a3] H3[a3+b3]
//   X2[b2,b3] = sum_a2 X1[a2,b3] H2[a2+b2]
//   C[c1,c2,c3] += X2[c2,c3] H1[a1+c1],
// every range cut to total degree < p: 2 p T_p + (p(p+1)/2)^2 multiply-adds
// instead of T_p^2 (D + 1) for the double sum (order 4: 260 against 1600,
// order 6: 1113 against 12544).
// Only one a1 slice of X1 and X2 is live at a time.  e^{-|tau|^2} is folded
// into the scaled moments and (-1)^{|beta|} / beta! comes from a table, so
// each coefficient costs one multiply on the way out.  The same terms as
// k_series_h2l, added in another order.
// ---------------------------------------------------------------------------
constexpr int kH2lBuckets = 5;   // 0: k_series_h2l; 1..4: k_series_h2l_d3 at orders 3..6

__device__ __forceinline__ int h2l_bucket(int D, int p) { return (D == 3 && p >= 3 && p <= 6) ? p - 2 : 0; }

// Hermite values of k_series_h2l_d3 in registers up to this order
template <int P>
constexpr bool kHermReg = P <= 5;

// dense register slot of (c1, c2, c3), c1 + c2 + c3 < P (c1 outermost)
template <int P>
__host__ __device__ constexpr int slot_of(int c1, int c2, int c3) {
    int s = 0;
    for (int i = 0; i < c1; ++i) s += (P - i) * (P - i + 1) / 2;
    for (int j = 0; j < c2; ++j) s += P - c1 - j;
    return s + c3;
}

template <int P>
__global__ void __launch_bounds__(128) k_series_h2l_d3(SeriesParams sp, const SeriesEntry *__restrict__ ent,
                                                       const unsigned long long *__restrict__ bounds) {
    constexpr int TP = P * (P + 1) * (P + 2) / 6;   // C(P + 2, 3) terms of total degree < P
    constexpr int NH = 2 * P - 1;                   // Hermite orders 0 .. 2P - 2
    __shared__ uint8_t idx3[P * P * P];             // (a1, a2, a3) -> graded-lex position
    __shared__ double sif[TP];                      // (-1)^{|beta|} / beta!
    __shared__ double h2l_hs[kHermReg<P> ? 1 : 3 * NH * 128];
    for (int a = threadIdx.x; a < TP; a += blockDim.x) {
        const uint8_t *al = sp.tb.alpha + 3 * a;
        idx3[(al[0] * P + al[1]) * P + al[2]] = (uint8_t)a;
        sif[a] = ((al[0] + al[1] + al[2]) & 1) ? -sp.tb.inv_fact[a] : sp.tb.inv_fact[a];
    }
    __syncthreads();
    const int64_t b0 = (int64_t)bounds[0], b1 = (int64_t)bounds[1];
    for (int64_t e = b0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b1;
         e += (int64_t)gridDim.x * blockDim.x) {
        const SeriesEntry E = ent[e];
        const double is = sp.inv_s[E.j];
        const double *mom = sp.rmom + (int64_t)E.r * sp.T;
        const double *cq = sp.qcenter + (int64_t)E.q * 3, *cr = sp.rcenter + (int64_t)E.r * 3;
        // Hermite values: registers up to order 5; at order 6 a per-thread
        // column of shared memory, so the coefficients fit in registers
        double Hr[kHermReg<P> ? 3 : 1][kHermReg<P> ? NH : 1];
        auto H = [&](int d, int k) -> double & {
            if constexpr (kHermReg<P>) return Hr[d][k];
            else return h2l_hs[(d * NH + k) * 128 + threadIdx.x];
        };
        double t2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double tau = (cq[d] - cr[d]) * is;
            t2 += tau * tau;
            double hm = 1.0, hc = 2.0 * tau;
            H(d, 0) = hm;
            H(d, 1) = hc;
#pragma unroll
            for (int k = 1; k + 1 < NH; ++k) {
                const double hn = 2.0 * tau * hc - 2.0 * k * hm;
                H(d, k + 1) = hn;
                hm = hc;
                hc = hn;
            }
        }
        double ip[P];   // e^{-|tau|^2} s^-k
        ip[0] = exp(-t2);
#pragma unroll
        for (int k = 1; k < P; ++k) ip[k] = ip[k - 1] * is;
        double C[TP];
#pragma unroll
        for (int k = 0; k < TP; ++k) C[k] = 0.0;
#pragma unroll
        for (int a1 = 0; a1 < P; ++a1) {
            double X1[P][P];   // [a2][b3], a1 + a2 < P
#pragma unroll
            for (int a2 = 0; a1 + a2 < P; ++a2) {
                double A[P];
#pragma unroll
                for (int a3 = 0; a1 + a2 + a3 < P; ++a3)
                    A[a3] = mom[idx3[(a1 * P + a2) * P + a3]] * ip[a1 + a2 + a3];
#pragma unroll
                for (int b3 = 0; b3 < P; ++b3) {
                    double acc = 0.0;
#pragma unroll
                    for (int a3 = 0; a1 + a2 + a3 < P; ++a3) acc = fma(A[a3], H(2, a3 + b3), acc);
                    X1[a2][b3] = acc;
                }
            }
#pragma unroll
            for (int c2 = 0; c2 < P; ++c2)
#pragma unroll
                for (int c3 = 0; c2 + c3 < P; ++c3) {
                    double x2 = 0.0;   // X2[c2, c3] of this slice
#pragma unroll
                    for (int a2 = 0; a1 + a2 < P; ++a2) x2 = fma(X1[a2][c3], H(1, a2 + c2), x2);
#pragma unroll
                    for (int c1 = 0; c1 + c2 + c3 < P; ++c1) {
                        C[slot_of<P>(c1, c2, c3)] = fma(x2, H(0, a1 + c1), C[slot_of<P>(c1, c2, c3)]);
                    }
                }
        }
        double *Bm = sp.B + ((int64_t)E.q * sp.nh + E.j) * sp.T;
#pragma unroll
        for (int c1 = 0; c1 < P; ++c1)
#pragma unroll
            for (int c2 = 0; c1 + c2 < P; ++c2)
#pragma unroll
                for (int c3 = 0; c1 + c2 + c3 < P; ++c3) {
                    const int k = idx3[(c1 * P + c2) * P + c3];
                    atomicAdd(&Bm[k], sif[k] * C[slot_of<P>(c1, c2, c3)]);
                }
        atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], P);
    }
}

// Bucket the H2L list by kernel: counts (per warp, then per block, then one
// global atomic per block and bucket), the start of each bucket, then a
// scatter that reserves each block chunk's range per bucket with one global
// atomic.  The order inside a bucket is free: every action adds into B with
// atomics.
__global__ void __launch_bounds__(256) k_h2l_count(const SeriesEntry *__restrict__ ent,
                                                   const FrontierState *__restrict__ fs, int D, int64_t cap,
                                                   unsigned long long *cnt) {
    __shared__ unsigned int c[kH2lBuckets];
    if (threadIdx.x < kH2lBuckets) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t ne = fs->series_count[2] < cap ? fs->series_count[2] : cap;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps step together, so every shuffle has all 32 lanes
    for (int64_t w0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); w0 < ne; w0 += stride) {
        const int64_t e = w0 + lane;
        const int b = e < ne ? h2l_bucket(D, ent[e].p) : -1;
        const unsigned m = __match_any_sync(0xffffffffu, b);
        if (b >= 0 && lane == __ffs(m) - 1) atomicAdd(&c[b], (unsigned)__popc(m));
    }
    __syncthreads();
    if (threadIdx.x < kH2lBuckets && c[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

__global__ void k_h2l_starts(const unsigned long long *cnt, unsigned long long *cur, unsigned long long *bounds) {
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int b = 0; b < kH2lBuckets; ++b) {
            cur[b] = s;
            bounds[b] = s;
            s += cnt[b];
        }
        bounds[kH2lBuckets] = s;
    }
}

__global__ void __launch_bounds__(256) k_h2l_scatter(const SeriesEntry *__restrict__ ent,
                                                     const FrontierState *__restrict__ fs, int D, int64_t cap,
                                                     unsigned long long *cur, SeriesEntry *out) {
    __shared__ unsigned int sc[kH2lBuckets];          // this chunk's count per bucket
    __shared__ unsigned long long sb[kH2lBuckets];    // its reserved start per bucket
    const int64_t ne = fs->series_count[2] < cap ? fs->series_count[2] : cap;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the whole block steps through chunks of blockDim entries together
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < ne; base += stride) {
        if (threadIdx.x < kH2lBuckets) sc[threadIdx.x] = 0;
        __syncthreads();
        const int64_t e = base + threadIdx.x;
        SeriesEntry E;
        int b = -1;
        if (e < ne) {
            E = ent[e];
            b = h2l_bucket(D, E.p);
        }
        const unsigned m = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(m) - 1;
        unsigned woff = 0;
        if (b >= 0 && lane == leader) woff = atomicAdd(&sc[b], (unsigned)__popc(m));
        woff = __shfl_sync(0xffffffffu, woff, leader);
        __syncthreads();
        if (threadIdx.x < kH2lBuckets)
            sb[threadIdx.x] = sc[threadIdx.x] ? atomicAdd(&cur[threadIdx.x], (unsigned long long)sc[threadIdx.x]) : 0ull;
        __syncthreads();
        if (b >= 0) out[sb[b] + woff + __popc(m & lt)] = E;
        __syncthreads();   // sc and sb are rewritten by the next chunk
    }
}

// ---------------------------------------------------------------------------
// downward pass, one query level at a time: L2L of every (node, j) with a
// local expansion into both children (Lemma 3)
// ---------------------------------------------------------------------------
// Moving the centre of sum_b B_b u^b by delta (u -> u + delta) factors over
// the dimensions, (u + delta)^b = prod_d (u_d + delta_d)^{b_d}, and the
// truncation |b| < p is closed under lowering an exponent, so Lemma 3's
// shift equals D one-dimensional shifts applied in turn.  Along dimension d
// the coefficients of a line alpha0 + k e_d (k < n) are the coefficients of
// a polynomial in u_d, shifted in place by repeated synthetic division:
//   for i = 0 .. n-2, for k = n-2 down to i:  c_k += delta_d c_{k+1},
// n (n - 1) / 2 multiply-adds per line.  One warp per (node, j); each lane
// takes a (child, line) and copies the line into its own scratch row.
constexpr int kL2lWarps = 4;
constexpr int kL2lLine = 17;     // longest line (P <= 16) plus one
__host__ __device__ inline size_t l2l_smem_per_warp(int T) { return (size_t)(2 * T + 32 * kL2lLine) * sizeof(double); }

__global__ void __launch_bounds__(kL2lWarps * 32) k_l2l_level(SeriesParams sp, int k) {
    extern __shared__ double l2l_s[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int T = sp.T, D = sp.D;
    double *buf = l2l_s + (size_t)w * (2 * T + 32 * kL2lLine);
    double *line = buf + 2 * T + lane;          // this lane's scratch, stride 32
    const int64_t nn = 1ll << k;
    const int64_t items = nn * sp.nh;
    const int64_t warps = (int64_t)gridDim.x * kL2lWarps;
    for (int64_t it = (int64_t)blockIdx.x * kL2lWarps + w; it < items; it += warps) {
        const int64_t node = nn - 1 + it / sp.nh;
        const int j = (int)(it % sp.nh);
        const int pl = sp.pL[node * sp.nh + j];
        if (pl == 0) continue;
        const int Tp = sp.tb.Tp[pl];
        const double is = sp.inv_s[j];
        const double *Bp = sp.B + (node * sp.nh + j) * T;
        for (int a = lane; a < Tp; a += 32) {
            const double b = Bp[a];
            buf[a] = b;
            buf[T + a] = b;
        }
        __syncwarp();
        for (int d = 0; d < D; ++d) {
            const double cp = sp.qcenter[node * D + d];
            const double dl0 = (sp.qcenter[(2 * node + 1) * D + d] - cp) * is;
            const double dl1 = (sp.qcenter[(2 * node + 2) * D + d] - cp) * is;
            const int nl = sp.tb.l2s_nlines[d * 17 + pl];
            const int32_t *starts = sp.tb.l2s_line + (size_t)d * T;
            const int32_t *nxt = sp.tb.l2s_next + (size_t)d * T;
            for (int v = lane; v < 2 * nl; v += 32) {
                const int c = v >= nl;
                const int a0 = starts[v - c * nl];
                const int n = pl - sp.tb.deg[a0];
                if (n < 2) continue;
                double *bc = buf + c * T;
                const double dl = c ? dl1 : dl0;
                int a = a0;
                for (int i = 0; i < n; ++i) {
                    line[32 * i] = bc[a];
                    a = nxt[a];
                }
                for (int i = 0; i + 1 < n; ++i)
                    for (int q = n - 2; q >= i; --q) line[32 * q] = fma(dl, line[32 * (q + 1)], line[32 * q]);
                a = a0;
                for (int i = 0; i < n; ++i) {
                    bc[a] = line[32 * i];
                    a = nxt[a];
                }
            }
            __syncwarp();
        }
        for (int c = 0; c < 2; ++c) {
            const int64_t ch = 2 * node + 1 + c;
            double *Bc = sp.B + (ch * sp.nh + j) * T;
            for (int a = lane; a < Tp; a += 32) Bc[a] += buf[c * T + a];
            if (lane == 0) {
                int32_t *pc = &sp.pL[ch * sp.nh + j];
                if (*pc < pl) *pc = pl;
            }
        }
        __syncwarp();
    }
}

// leaves: out = base + DH + sum of ancestors' FD estimates + EVALL(B)
// Final values, one warp per (query leaf, bandwidth).  Local expansions of
// at most kFinLane terms are evaluated one query per lane, u = (x_q - x_Q)/s,
// by Horner's rule on the tree that links each multi-index a to dpred(a) (a
// with its last non-zero exponent lowered by one, always earlier in the
// graded order): S(a) = B_a + sum over the children c of u_{dim(c)} S(c), so
// that S(0) = sum_a B_a u^a.  Walking the terms from the last to the first,
// each one is final when reached and adds u_{dim(a)} S(a) into its parent:
// one multiply-add per term, in a lane-interleaved shared buffer.  Longer
// expansions: lanes over the terms, one query at a time.
constexpr int kFinLane = 64;
// doubles of shared memory per warp: the partial sums of the longest local
// expansion evaluated per lane (at most kFinLane terms), then u for D dims
__host__ __device__ inline int fin_terms(int T) { return T < kFinLane ? T : kFinLane; }
__host__ __device__ inline size_t fin_doubles_per_warp(int T, int D) { return (size_t)(fin_terms(T) + D) * 32; }
__global__ void __launch_bounds__(kSerTB) k_final(SeriesParams sp) {
    extern __shared__ double fin_s[];   // per warp: partial sums S [terms][32 lanes], u [D][32 lanes]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int depth = sp.q_depth, D = sp.D;
    const int64_t nl = 1ll << depth;
    const int64_t items = nl * sp.nh;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + w; it < items; it += warps) {
        const int64_t i = it / sp.nh;
        const int j = (int)(it % sp.nh);
        const int64_t leaf = nl - 1 + i;
        double es = 0.0;
        for (int64_t a = leaf;; a = (a - 1) / 2) {
            es += sp.est[a * sp.nh + j];
            if (a == 0) break;
        }
        const int pl = sp.pL ? sp.pL[leaf * sp.nh + j] : 0;
        const int Tp = pl > 0 ? sp.tb.Tp[pl] : 0;
        const double is = sp.inv_s[j];
        const double *Bl = sp.B ? sp.B + (leaf * sp.nh + j) * sp.T : nullptr;
        const int64_t b = level_begin(sp.qn, depth, i), e = level_begin(sp.qn, depth, i + 1);
        double *acc = fin_s + (size_t)w * fin_doubles_per_warp(sp.T, D) + lane;
        double *uw = acc - lane + fin_terms(sp.T) * 32;   // this warp's u region
        if (Tp <= kFinLane) {
            const double *cQ = sp.qcenter + leaf * D;
            for (int64_t pos = b + lane; pos < e; pos += 32) {
                double v = sp.Gq[pos * sp.nh + j] + es;
                if (Tp > 0) {
                    for (int d = 0; d < D; ++d) uw[d * 32 + lane] = (coord(sp.qxs, sp.dtype, pos, D, d) - cQ[d]) * is;
                    for (int a = 0; a < Tp; ++a) acc[a * 32] = Bl[a];
                    for (int a = Tp - 1; a >= 1; --a) {
                        double *pa = acc + sp.tb.dpred[a] * 32;
                        *pa = fma(uw[sp.tb.pred_dim[a] * 32 + lane], acc[a * 32], *pa);
                    }
                    v += acc[0];
                }
                sp.out[(int64_t)sp.qperm[pos] * sp.nh + j] = v;
            }
            continue;
        }
        for (int64_t pos = b; pos < e; ++pos) {
            double v = sp.Gq[pos * sp.nh + j] + es;
            if (Tp > 0) {
                for (int d = lane; d < D; d += 32)
                    uw[d] = (coord(sp.qxs, sp.dtype, pos, D, d) - sp.qcenter[leaf * D + d]) * is;
                __syncwarp();
                double s = 0.0;
                for (int a = lane; a < Tp; a += 32) {
                    const uint8_t *al = sp.tb.alpha + a * D;
                    double m = Bl[a];
                    for (int d = 0; d < D; ++d)
                        for (int q = 0; q < al[d]; ++q) m *= uw[d];
                    s += m;
                }
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                v += s;
                __syncwarp();
            }
            if (lane == 0) sp.out[(int64_t)sp.qperm[pos] * sp.nh + j] = v;
        }
    }
}

int run_series_and_final(const TraversalIn &in, FrontierBufs &fb, const SeriesTables *tb, double *Gq,
                         double *B, int32_t *pL, double *out, CallCtx &cx) {
    cudaStream_t st = cx.st;
    SeriesParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.D = in.D;
    sp.nh = in.nh;
    sp.P = in.P;
    sp.T = tb ? tb->T : 0;
    if (tb) sp.tb = *tb;
    sp.qxs = in.qt->xs;
    sp.rxs = in.rt->xs;
    sp.dtype = in.qt->dtype;
    sp.rperm = in.rt->perm;
    sp.w = in.weights;
    sp.qn = in.qt->n;
    sp.rn = in.rt->n;
    sp.qcenter = in.qt->center;
    sp.rcenter = in.rt->center;
    sp.rmom = in.rt->moments;
    sp.inv_s = fb.inv_s;
    sp.Gq = Gq;
    sp.B = B;
    sp.pL = pL;
    sp.est = fb.est;
    sp.qperm = in.qt->perm;
    sp.out = out;
    sp.q_depth = in.qt->depth;
    if (tb && B) {
        if (sp.D * (2 * in.P - 1) > 2 * kMaxDP || tb->T > kMaxT) {
            set_error("series order too high for the series kernels (D=%d, P=%d)", in.D, in.P);
            return GS_ERR_ARG;
        }
        cx.phase(GS_PH_SERIES);
        int rc;
        const int tbytes = table_bytes(sp.T, sp.D);
        // pieces of the DH (queries) and DL (references) actions
        long long *pieces[2] = {nullptr, nullptr};
        SeriesEntry *h2l_sorted = nullptr;          // the H2L list bucketed by kernel (D = 3)
        unsigned long long *h2l_ctl = nullptr;
        auto free_pieces = [&]() {
            for (int m = 0; m < 2; ++m)
                if (pieces[m]) cudaFreeAsync(pieces[m], st);
        };
        for (int m = 0; m < 2; ++m) {
            const int64_t ne = fb.n_series[m];
            if (ne == 0) continue;
            const cudaError_t e = dev_malloc_async((void **)&pieces[m], (size_t)(ne + 1) * sizeof(long long), st);
            if (e != cudaSuccess) {
                free_pieces();
                return cuda_fail(e, "series pieces");
            }
            k_chunk_count<<<(unsigned)((ne + 255) / 256 < 4096 ? (ne + 255) / 256 : 4096), 256, 0, st>>>(
                fb.series[m], ne, m == 0, sp.qn, sp.rn, pieces[m]);
            cx.launches += 1;
            if ((rc = scan_i64(pieces[m], ne, pieces[m] + ne, cx))) {
                free_pieces();
                return rc;
            }
        }
        auto launch = [&](int which, int64_t n, size_t per_warp) -> int {
            if (n <= 0) return GS_OK;
            int wpb = 8;
            while (wpb > 1 && tbytes + wpb * per_warp > 200 * 1024) wpb >>= 1;
            const size_t sm = tbytes + wpb * per_warp;
            if (sm > 220 * 1024) {
                set_error("series order too high for shared memory (D=%d, P=%d)", sp.D, sp.P);
                return GS_ERR_ARG;
            }
            const unsigned grid = (unsigned)(fb.grid_warps / wpb);
            const void *fn = which == 0 ? (const void *)k_series_dh
                           : which == 1 ? (const void *)k_series_dl : (const void *)k_series_h2l;
            allow_max_smem(fn);
            if (which == 0)
                k_series_dh<<<grid, wpb * 32, sm, st>>>(sp, fb.series[0], n, pieces[0], pieces[0] + n);
            else if (which == 1)
                k_series_dl<<<grid, wpb * 32, sm, st>>>(sp, fb.series[1], n, pieces[1], pieces[1] + n);
            else {
                GS_CUDA_TRY(cudaMemsetAsync(&fb.fs->work, 0, sizeof(unsigned long long), st));
                int64_t g = ((n + 31) / 32 + wpb - 1) / wpb;
                const int64_t mx = fb.grid_warps / wpb;
                const unsigned grid_h = (unsigned)(g < 1 ? 1 : (g > mx ? mx : g));
                if (!h2l_sorted) {
                    k_series_h2l<<<grid_h, wpb * 32, sm, st>>>(sp, fb.fs, fb.series[2], nullptr);
                } else {
                    // three-dimensional orders 3 and 4 in their own kernels,
                    // everything else in the general one
                    const unsigned long long *bnd = h2l_ctl + 2 * kH2lBuckets;
                    const unsigned gd = (unsigned)(fb.grid_warps / 4);
                    k_series_h2l<<<grid_h, wpb * 32, sm, st>>>(sp, fb.fs, h2l_sorted, bnd + 1);
                    k_series_h2l_d3<3><<<gd, 128, 0, st>>>(sp, h2l_sorted, bnd + 1);
                    if (sp.P >= 4) k_series_h2l_d3<4><<<gd, 128, 0, st>>>(sp, h2l_sorted, bnd + 2);
                    if (sp.P >= 5) k_series_h2l_d3<5><<<gd, 128, 0, st>>>(sp, h2l_sorted, bnd + 3);
                    if (sp.P >= 6) k_series_h2l_d3<6><<<gd, 128, 0, st>>>(sp, h2l_sorted, bnd + 4);
                    cx.launches += 1 + (sp.P >= 4) + (sp.P >= 5) + (sp.P >= 6);
                }
            }
            cx.launches += 1;
            return cx.check(which == 0 ? "k_series_dh" : which == 1 ? "k_series_dl" : "k_series_h2l");
        };
        cx.mark(0);
        rc = launch(0, fb.n_series[0], 8 * (size_t)(sp.T + sp.D * sp.P * 32));
        cx.mark(1);
        if (!rc) rc = launch(1, fb.n_series[1], 8 * (size_t)(32 * sp.D * sp.P + 32 + 32 * kDlStride));
        cx.mark(2);
        if (!rc && sp.D == 3 && sp.P >= 3 && fb.n_series[2] > 0) {
            // bucket the H2L list: ctl = counts, cursors, bounds (kH2lBuckets + 1)
            constexpr int kCtl = 3 * kH2lBuckets + 1;
            cudaError_t e = dev_malloc_async((void **)&h2l_ctl, kCtl * sizeof(unsigned long long), st);
            if (e == cudaSuccess)
                e = dev_malloc_async((void **)&h2l_sorted, (size_t)fb.n_series[2] * sizeof(SeriesEntry), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(h2l_ctl, 0, kCtl * sizeof(unsigned long long), st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "H2L buckets");
            } else {
                const int64_t blocks = (fb.n_series[2] + 255) / 256;
                const unsigned gb = (unsigned)(blocks < 4096 ? blocks : 4096);
                k_h2l_count<<<gb, 256, 0, st>>>(fb.series[2], fb.fs, sp.D, fb.n_series[2], h2l_ctl);
                k_h2l_starts<<<1, 32, 0, st>>>(h2l_ctl, h2l_ctl + kH2lBuckets, h2l_ctl + 2 * kH2lBuckets);
                k_h2l_scatter<<<gb, 256, 0, st>>>(fb.series[2], fb.fs, sp.D, fb.n_series[2], h2l_ctl + kH2lBuckets,
                                                  h2l_sorted);
                cx.launches += 3;
                rc = cx.check("H2L buckets");
            }
        }
        if (!rc) rc = launch(2, fb.n_series[2], 8 * (size_t)(sp.T + sp.D * (2 * sp.P - 1) + 32 * (kLaneT + kLaneH)));
        if (h2l_sorted) cudaFreeAsync(h2l_sorted, st);
        if (h2l_ctl) cudaFreeAsync(h2l_ctl, st);
        cx.mark(-1);
        free_pieces();
        if (rc) return rc;
        cx.phase(GS_PH_DOWN);
        const size_t l2l_sm = kL2lWarps * l2l_smem_per_warp(sp.T);
        if (in.qt->depth > 0 && l2l_sm > 220 * 1024) {
            set_error("series order too high for the L2L kernel (D=%d, P=%d)", sp.D, sp.P);
            return GS_ERR_ARG;
        }
        allow_max_smem((const void *)k_l2l_level);
        for (int k = 0; k < in.qt->depth; ++k) {
            const int64_t warps = (1ll << k) * in.nh;
            const int64_t blocks = (warps + kL2lWarps - 1) / kL2lWarps;
            const int64_t mx = fb.grid_warps / kL2lWarps;
            k_l2l_level<<<(unsigned)(blocks < mx ? blocks : mx), kL2lWarps * 32, l2l_sm, st>>>(sp, k);
            cx.launches += 1;
            if ((rc = cx.check("k_l2l_level"))) return rc;
        }
    }
    cx.phase(GS_PH_DOWN);
    allow_max_smem((const void *)k_final);
    k_final<<<fb.grid_warps / 4, kSerTB, (kSerTB / 32) * fin_doubles_per_warp(sp.T, sp.D) * sizeof(double), st>>>(sp);
    cx.launches += 1;
    if (int rc2 = cx.check("k_final")) return rc2;
    cx.phase(GS_PH_OTHER);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "series / downward launch");
    return GS_OK;
}

}  // namespace gs
