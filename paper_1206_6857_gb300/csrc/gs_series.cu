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

// ---------------------------------------------------------------------------
// DH: one warp per action, lanes over the queries of Q
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_series_dh(SeriesParams sp, const FrontierState *__restrict__ fs, const SeriesEntry *__restrict__ ent) {
    const int64_t ne = fs->series_count[0];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int D = sp.D;
    for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); e < ne; e += warps) {
        const SeriesEntry E = ent[e];
        const int p = E.p, Tp = sp.tb.Tp[p];
        const double is = sp.inv_s[E.j];
        double ispow[16];
        ispow[0] = 1.0;
        for (int k = 1; k < p; ++k) ispow[k] = ispow[k - 1] * is;
        const double *mom = sp.rmom + (int64_t)E.r * sp.T;
        const double *cR = sp.rcenter + (int64_t)E.r * D;
        const int qd = node_depth(E.q);
        const int64_t qi = E.q - ((1ll << qd) - 1);
        const int64_t b = level_begin(sp.qn, qd, qi), en = level_begin(sp.qn, qd, qi + 1);
        for (int64_t pos = b + lane; pos < en; pos += 32) {
            double H[kMaxDP];
            double t2 = 0.0;
            for (int d = 0; d < D; ++d) {
                const double t = (coord(sp.qxs, sp.dtype, pos, D, d) - cR[d]) * is;
                hermite_polys(t, p, &H[d * p]);
                t2 += t * t;
            }
            double s = 0.0;
            for (int a = 0; a < Tp; ++a) {
                const uint8_t *al = sp.tb.alpha + a * D;
                double pr = mom[a] * ispow[sp.tb.deg[a]];
                for (int d = 0; d < D; ++d) pr *= H[d * p + al[d]];
                s += pr;
            }
            atomicAdd(&sp.Gq[pos * sp.nh + E.j], s * exp(-t2));
        }
    }
}

// ---------------------------------------------------------------------------
// DL: one warp per action, lanes over the references of R; each coefficient
// is reduced across the warp and banked by lane (b mod 32)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_series_dl(SeriesParams sp, const FrontierState *__restrict__ fs, const SeriesEntry *__restrict__ ent) {
    const int64_t ne = fs->series_count[1];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int D = sp.D;
    for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); e < ne; e += warps) {
        const SeriesEntry E = ent[e];
        const int p = E.p, Tp = sp.tb.Tp[p];
        const double is = sp.inv_s[E.j];
        const double *cQ = sp.qcenter + (int64_t)E.q * D;
        const int rd = node_depth(E.r);
        const int64_t ri = E.r - ((1ll << rd) - 1);
        const int64_t rb = level_begin(sp.rn, rd, ri), re = level_begin(sp.rn, rd, ri + 1);
        double acc[kMaxT / 32];
        for (int i = 0; i < (Tp + 31) / 32; ++i) acc[i] = 0.0;
        for (int64_t c0 = rb; c0 < re; c0 += 32) {
            const int64_t pos = c0 + lane;
            const bool valid = pos < re;
            double H[kMaxDP];
            double we = 0.0;
            if (valid) {
                double v2 = 0.0;
                for (int d = 0; d < D; ++d) {
                    const double v = (coord(sp.rxs, sp.dtype, pos, D, d) - cQ[d]) * is;
                    hermite_polys(v, p, &H[d * p]);
                    v2 += v * v;
                }
                we = (double)sp.w[sp.rperm[pos]] * exp(-v2);
            } else {
                for (int i = 0; i < D * p; ++i) H[i] = 0.0;
            }
            for (int a = 0; a < Tp; ++a) {
                const uint8_t *be = sp.tb.alpha + a * D;
                double pr = we;
                for (int d = 0; d < D; ++d) pr *= H[d * p + be[d]];
                pr = warp_sum_d(pr);
                if ((a & 31) == lane) acc[a >> 5] += pr;
            }
        }
        double *Bq = sp.B + ((int64_t)E.q * sp.nh + E.j) * sp.T;
        for (int a = lane; a < Tp; a += 32) atomicAdd(&Bq[a], acc[a >> 5] * sp.tb.inv_fact[a]);
        if (lane == 0) atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], p);
    }
}

// ---------------------------------------------------------------------------
// H2L: one warp per action, lanes over b, loop over a; the 1-D Hermite
// polynomials of tau = (x_Q - x_R)/s up to order 2p-2 sit in shared memory
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_series_h2l(SeriesParams sp, const FrontierState *__restrict__ fs, const SeriesEntry *__restrict__ ent) {
    __shared__ double Hs[8][2 * kMaxDP];
    const int64_t ne = fs->series_count[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int D = sp.D;
    for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + w; e < ne; e += warps) {
        const SeriesEntry E = ent[e];
        const int p = E.p, Tp = sp.tb.Tp[p];
        const int nH = 2 * p - 1;   // orders 0 .. 2p-2
        const double is = sp.inv_s[E.j];
        double ispow[16];
        ispow[0] = 1.0;
        for (int k = 1; k < p; ++k) ispow[k] = ispow[k - 1] * is;
        const double *mom = sp.rmom + (int64_t)E.r * sp.T;
        __syncwarp();
        double t2 = 0.0;
        if (lane < D) {
            const double tau = (sp.qcenter[(int64_t)E.q * D + lane] - sp.rcenter[(int64_t)E.r * D + lane]) * is;
            hermite_polys(tau, nH, &Hs[w][lane * nH]);
            t2 = tau * tau;
        }
        t2 = warp_sum_d(t2);
        __syncwarp();
        const double et = exp(-t2);
        double *Bq = sp.B + ((int64_t)E.q * sp.nh + E.j) * sp.T;
        for (int bt = lane; bt < Tp; bt += 32) {
            const uint8_t *be = sp.tb.alpha + bt * D;
            double s = 0.0;
            for (int a = 0; a < Tp; ++a) {
                const uint8_t *al = sp.tb.alpha + a * D;
                double pr = mom[a] * ispow[sp.tb.deg[a]];
                for (int d = 0; d < D; ++d) pr *= Hs[w][d * nH + al[d] + be[d]];
                s += pr;
            }
            const double sign = (sp.tb.deg[bt] & 1) ? -1.0 : 1.0;
            atomicAdd(&Bq[bt], sign * sp.tb.inv_fact[bt] * et * s);
        }
        if (lane == 0) atomicMax(&sp.pL[(int64_t)E.q * sp.nh + E.j], p);
    }
}

// ---------------------------------------------------------------------------
// downward pass, one query level at a time: L2L of every (node, j) with a
// local expansion into both children (Lemma 3)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSerTB) k_l2l_level(SeriesParams sp, int k) {
    __shared__ double pw[2][kMaxDP];
    const int64_t nn = 1ll << k;
    const int64_t items = nn * sp.nh;
    const int D = sp.D;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t node = nn - 1 + it / sp.nh;
        const int j = (int)(it % sp.nh);
        const int pl = sp.pL[node * sp.nh + j];
        if (pl == 0) continue;
        const int Tp = sp.tb.Tp[pl];
        const double is = sp.inv_s[j];
        const double *Bp = sp.B + (node * sp.nh + j) * sp.T;
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * D; t += blockDim.x) {
            const int c = t / D, d = t % D;
            const int64_t ch = 2 * node + 1 + c;
            const double dl = (sp.qcenter[ch * D + d] - sp.qcenter[node * D + d]) * is;
            double v = 1.0;
            for (int q = 0; q < pl; ++q) {
                pw[c][d * pl + q] = v;
                v *= dl;
            }
        }
        __syncthreads();
        for (int c = 0; c < 2; ++c) {
            const int64_t ch = 2 * node + 1 + c;
            double *Bc = sp.B + (ch * sp.nh + j) * sp.T;
            for (int a = threadIdx.x; a < Tp; a += blockDim.x) {
                double s = 0.0;
                for (int e2 = sp.tb.l2l_off[a]; e2 < sp.tb.l2l_off[a + 1]; ++e2) {
                    const int bt = sp.tb.l2l_pairs[2 * e2], dt = sp.tb.l2l_pairs[2 * e2 + 1];
                    if (bt >= Tp) continue;
                    const uint8_t *de = sp.tb.alpha + dt * D;
                    double m = sp.tb.l2l_coef[e2] * Bp[bt];
                    for (int d = 0; d < D; ++d) m *= pw[c][d * pl + de[d]];
                    s += m;
                }
                Bc[a] += s;
            }
            if (threadIdx.x == 0) {
                int32_t *pc = &sp.pL[ch * sp.nh + j];
                if (*pc < pl) *pc = pl;
            }
        }
    }
}

// leaves: out = base + DH + sum of ancestors' FD estimates + EVALL(B)
__global__ void __launch_bounds__(kSerTB) k_final(SeriesParams sp) {
    __shared__ double us[kSerTB / 32][32];
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
        for (int64_t pos = b; pos < e; ++pos) {
            double v = sp.Gq[pos * sp.nh + j] + es;
            if (Tp > 0) {
                for (int d = lane; d < D; d += 32)
                    us[w][d] = (coord(sp.qxs, sp.dtype, pos, D, d) - sp.qcenter[leaf * D + d]) * is;
                __syncwarp();
                double s = 0.0;
                for (int a = lane; a < Tp; a += 32) {
                    const uint8_t *al = sp.tb.alpha + a * D;
                    double m = Bl[a];
                    for (int d = 0; d < D; ++d)
                        for (int q = 0; q < al[d]; ++q) m *= us[w][d];
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
        auto grid_for = [&](int64_t n) {
            int64_t g = (n + 7) / 8;
            const int64_t mx = fb.grid_warps / 8;
            return (unsigned)(g < 1 ? 1 : (g > mx ? mx : g));
        };
        if (fb.n_series[0] > 0) {
            k_series_dh<<<grid_for(fb.n_series[0]), 256, 0, st>>>(sp, fb.fs, fb.series[0]);
            cx.launches += 1;
            if ((rc = cx.check("k_series_dh"))) return rc;
        }
        if (fb.n_series[1] > 0) {
            k_series_dl<<<grid_for(fb.n_series[1]), 256, 0, st>>>(sp, fb.fs, fb.series[1]);
            cx.launches += 1;
            if ((rc = cx.check("k_series_dl"))) return rc;
        }
        if (fb.n_series[2] > 0) {
            k_series_h2l<<<grid_for(fb.n_series[2]), 256, 0, st>>>(sp, fb.fs, fb.series[2]);
            cx.launches += 1;
            if ((rc = cx.check("k_series_h2l"))) return rc;
        }
        cx.phase(GS_PH_DOWN);
        for (int k = 0; k < in.qt->depth; ++k) {
            const int64_t items = (1ll << k) * in.nh;
            k_l2l_level<<<(unsigned)(items < 65535 ? items : 65535), kSerTB, 0, st>>>(sp, k);
            cx.launches += 1;
            if ((rc = cx.check("k_l2l_level"))) return rc;
        }
    }
    cx.phase(GS_PH_DOWN);
    k_final<<<fb.grid_warps / 4, kSerTB, 0, st>>>(sp);
    cx.launches += 1;
    if (int rc2 = cx.check("k_final")) return rc2;
    cx.phase(GS_PH_OTHER);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "series / downward launch");
    return GS_OK;
}

}  // namespace gs
