// Breadth-first node-pair frontier: the dual-tree recursion of Fig. 1 / Fig. 7
// (DITO) restated level-synchronously so that every pair of an iteration is
// processed in parallel.
//
// Iteration t holds pairs (Q, R, j) with Q at depth min(t, dQ) and R at
// depth min(t, dR), grouped by (j, Q) with R ascending.  One warp handles one
// group:
//   pass 1  delta_min / delta_max from the bounding boxes (Section 5), the
//           group's lower bound G^min = (finished lower bounds of Q and its
//           ancestors) + sum of W_R K(delta_max) over the group's pairs,
//           raised to w_min(Q) (monochromatic) and to the floor 2^f W;
//   pass 2  per pair: its token share W_T * W_R / sum W_R, the FD test with
//           tokens (Fig. 7), then bestMethod (Fig. 6) over DH / DL / H2L with
//           the Lemma 4-6 bounds against the Theorem 2 budget, else a
//           leaf-leaf base case (banks W_R, DITOBase) or a split.
// The group's token, finished lower bound and FD estimate are then reduced
// in a fixed order (32 lane-strided partial sums and an xor butterfly) and
// inherited by the child groups.  A column scan over groups gives every
// group its output offsets, and a second warp-per-group pass writes the
// child frontier (still grouped and sorted), the base-case pairs and the
// series actions.
//
// Every decision is taken with IEEE operations in a fixed order and no FMA
// contraction (this file is compiled with -fmad=false): kernel bounds in FP32
// with rigorous margins and an exp2 written for this purpose, budgets and
// comparisons in FP64, and FP32 screens that only skip FP64 tests they prove
// to fail.  The pair lists are therefore reproducible bit for bit by a plain
// CPU evaluation of the same formulas.
#include <math.h>

#include <mutex>

#include "gs_frontier.cuh"
#include "gs_internal.h"
#include "gs_mlp.cuh"
#include "gs_tree.cuh"

namespace gs {

__constant__ float c_e2[8];   // ln2^n / n!, rounded to FP32

static const double kSqrt2 = 1.4142135623730951;
#define F32_LO18 0x1.ffff8p-1f    // 1 - 2^-18
#define F32_HI18 0x1.00004p+0f    // 1 + 2^-18
#define F32_LO20 0x1.ffffep-1f    // 1 - 2^-20
#define F32_HI20 0x1.00001p+0f    // 1 + 2^-20
#define F32_TINY 0x1p-125f
#define F32_AMAX 125.0f

// 2^x in FP32 for -125 <= x <= 0: k = rint(x), f = x - k, 2^f by Horner on
// its degree-7 Taylor polynomial, times 2^k built exactly.  Relative error
// below 2^-20 (covered by the bound margins).  rint comes from one FP32 add
// of 1.5 * 2^23 (in [2^23, 2^24) the spacing is 1, and round-to-nearest-even
// of the sum is 1.5 * 2^23 + rint(x) because 1.5 * 2^23 is even); the
// integer k is then the difference of the bit patterns.  The same values as
// rintf and a float-to-int conversion, without conversion instructions
// (they share the slow FP64 pipe on this GPU).
__device__ __forceinline__ float exp2_f32(float x) {
    const float magic = 0x1.8p+23f;
    const float t = __fadd_rn(x, magic);
    const float k = __fsub_rn(t, magic);
    const int ki = __float_as_int(t) - __float_as_int(magic);
    const float f = x - k;
    float p = c_e2[7];
#pragma unroll
    for (int n = 6; n >= 0; --n) p = p * f + c_e2[n];
    return p * __int_as_float((ki + 127) << 23);
}

__device__ __forceinline__ double rpow(double r, int p) {
    double o = 1.0;
    for (int i = 0; i < p; ++i) o = o * r;
    return o;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// warp_sum of a value that is often zero on every lane: skipped then (a sum
// of zeros is +0 either way)
__device__ __forceinline__ double warp_sum_sparse(double v) {
    return __any_sync(0xffffffffu, v != 0.0) ? warp_sum(v) : 0.0;
}

// The same butterfly with its value needed on lane 0 only: at each step only
// the lanes whose partial sum lane 0 still reads add (own + higher partner,
// the pairs and the order of warp_sum), so the FP64 pipe does 31 additions
// instead of 160.  Lane 0's result equals warp_sum's.
__device__ __forceinline__ double warp_sum_lane0(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, v, m);
        if (lane < m) v = v + o;
    }
    return v;
}
__device__ __forceinline__ double warp_sum_sparse_lane0(double v) {
    return __any_sync(0xffffffffu, v != 0.0) ? warp_sum_lane0(v) : 0.0;
}

// xor-butterfly sums in FP32 with every addition rounded down / up
__device__ __forceinline__ float warp_sum_rd(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, m));
    return v;
}
__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, m));
    return v;
}

struct FrontierParams {
    int D, nh, P, selector, tokens, mono;
    int best_first;       // look-ahead of each group's largest bound gaps (GS_FLAG_BEST_FIRST)
    int t, q_depth, r_depth, q_leaf, r_leaf;
    int floor_log2;
    int64_t qn, rn;
    const float *qlo32, *qhi32, *rlo32, *rhi32;
    const double *qrad;
    const float *qwmin;
    const double *rrad, *rW;
    const float *rrad32;  // reference radii rounded down to FP32
    const float *rW32d, *rW32u;   // reference weight sums rounded down / up to FP32
    const double *inv_h;
    double *fin, *tok, *est;
    float *geo;           // per pair cache: K(delta_max) lower, K(delta_min) upper, e^{-dmin^2/4h^2} upper,
                          // the pair's lower bound of its kernel sum (W_R K(delta_max) or the look-ahead's)
    double F[17], BT[17], Dpow[34];
    double cw[4];         // cost weights of c_DH, c_DL, c_H2L, c_Direct
    // weighted bestMethod costs of this iteration, for node sizes floor(n / 2^depth) + {0, 1}
    double cDH[2][17], cDL[2][17], cH2L[17], cex[2][2];
    const float *mlp;     // selector network parameters (learned ordering)
    // pair log (training data of the selector), indexed by global pair id
    float *lfeat;
    int8_t *lpc;
    int32_t *lnq, *lnr;
    int64_t *lpar;
    const int64_t *pid;   // parent id of each pair of this iteration (null at the root)
    int64_t log_base;     // id of this iteration's first pair
    float c32[64];        // log2(e) / 2h_j^2 rounded to FP32
};

__device__ __forceinline__ int64_t node_size(int64_t n, int depth, int64_t node) {
    const int64_t i = node - ((1ll << depth) - 1);
    return level_begin(n, depth, i + 1) - level_begin(n, depth, i);
}

// floats per warp of the per-group screen tables (4 x 17)
constexpr int kTab = 68;
// Best-first look-ahead: a pair whose bound gap W_R (K(delta_min) - K(delta_max))
// is at least 1 / kBestFirst of its group's total gap (so at most kBestFirst
// pairs per group, the largest gaps) contributes the lower bound of its
// reference node's two children to G^min when that is larger.
constexpr float kBestFirst = 8.f;
static_assert(sizeof(FrontierParams) <= 4096, "kernel parameters above 4 KB");

struct KBounds {
    float kmax, kmin, e4;
};

// Rigorous FP32 bounds of the kernel over a node pair (Section 5's
// delta_min / delta_max from the bounding boxes, which are stored rounded
// outward): squared distances, exponent arguments and exponentials carry
// relative margins of 2^-18, 2^-20 and 2^-18, each larger than the rounding
// they cover.
__device__ __forceinline__ KBounds kernel_bounds(const FrontierParams &fp, int64_t q, int64_t r, float c32) {
    float gsum = 0.f, fsum = 0.f;
    for (int d = 0; d < fp.D; ++d) {
        const float ql = fp.qlo32[q * fp.D + d], qh = fp.qhi32[q * fp.D + d];
        const float rl = fp.rlo32[r * fp.D + d], rh = fp.rhi32[r * fp.D + d];
        const float g = fmaxf(0.f, fmaxf(rl - qh, ql - rh));
        const float f = fmaxf(qh - rl, rh - ql);
        gsum = gsum + g * g;
        fsum = fsum + f * f;
    }
    const float dmin2 = gsum * F32_LO18, dmax2 = fsum * F32_HI18;
    const float amax = (dmax2 * c32) * F32_HI20;
    const float amin = (dmin2 * c32) * F32_LO20;
    const float a4 = amin * 0.5f;
    KBounds b;
    b.kmax = amax > F32_AMAX ? 0.f : exp2_f32(-amax) * F32_LO18;
    b.kmin = amin > F32_AMAX ? F32_TINY : exp2_f32(-amin) * F32_HI18;
    b.e4 = a4 > F32_AMAX ? F32_TINY : exp2_f32(-a4) * F32_HI18;
    return b;
}

// ---------------------------------------------------------------------------
// K1: decisions
// ---------------------------------------------------------------------------
// MODE 0: rule (Fig. 6) or FD only; MODE 1: learned ordering of the
// certified actions; MODE 2: FD-only decisions with every pair logged.
// The rule's decisions are latency-bound (dependent global loads, FP64 tests
// on a few lanes): four blocks of 256 threads per SM (64 registers, a few
// hundred bytes spilled to L1) run the C2 LSCV sweep's frontier in 83 ms
// against 106 ms with two blocks and no spills (three: 90 ms).
template <int MODE>
__global__ void __launch_bounds__(256, MODE == 0 ? 4 : 1)
k_front_decide(FrontierParams fp, FrontierState *fs, const Group *__restrict__ groups,
               const int32_t *__restrict__ pr, uint8_t *__restrict__ dec, int32_t *__restrict__ cnt,
               int4 *__restrict__ trace, int64_t trace_cap) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = fs->ngroups[fp.t];
    const double Wtot = fs->Wtot, floorW = fs->floorW, eps_t = fs->eps_t;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t trace_base = fs->trace_count;
    __shared__ float s_tab[8][kTab];
    __shared__ __align__(16) float s_w[MODE == 1 ? kMlpParams + 3 : 2];
    if constexpr (MODE == 1) {
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) s_w[i] = fp.mlp[i];
        __syncthreads();
    }
    const double diam = fs->diam;
    for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < ng; g += warps) {
        const Group G = groups[g];
        const int64_t q = G.q;
        const int j = G.j;
        const double invh = fp.inv_h[j];
        const float c32 = fp.c32[j];
        // pass 1: kernel bounds of every pair, lower bound over the group.
        // The lane sums and the butterfly run in FP32 rounded towards -inf
        // (the lower bound, from W_R rounded down) and +inf (the weight sum
        // the token is shared by, from W_R rounded up): a smaller lower bound
        // and a larger weight sum keep every budget valid.
        float s_dl = 0.f, s_W = 0.f;
        if (fp.best_first && !fp.r_leaf) {
            // Best-first ordering within the group: the pairs with the largest
            // bound gaps (those a priority queue on the gap would expand first)
            // are expanded one level on the reference side before any decision,
            // and the lower bound of the two children,
            //   W_R1 K(delta_max(Q, R1)) + W_R2 K(delta_max(Q, R2)) >= W_R K(delta_max(Q, R)),
            // replaces the pair's own in G^min.  Gaps in FP32 rounded to nearest,
            // their group sum rounded up; the selection only has to be
            // reproducible, every lower bound stays rigorous.
            float s_gap = 0.f;
            for (int k = lane; k < G.cnt; k += 32) {
                const int64_t r = pr[G.off + k];
                const KBounds kb = kernel_bounds(fp, q, r, c32);
                float *gc = fp.geo + 4 * (G.off + k);
                gc[0] = kb.kmax;
                gc[1] = kb.kmin;
                gc[2] = kb.e4;
                s_gap = __fadd_ru(s_gap, __fmul_rn(fp.rW32u[r], __fsub_rn(kb.kmin, kb.kmax)));
                s_W = __fadd_ru(s_W, fp.rW32u[r]);
            }
            const float gap_tot = warp_sum_ru(s_gap);
            for (int k = lane; k < G.cnt; k += 32) {
                const int64_t r = pr[G.off + k];
                float *gc = fp.geo + 4 * (G.off + k);
                const float kmax = gc[0];
                float dl = __fmul_rd(fp.rW32d[r], kmax);
                const float gap = __fmul_rn(fp.rW32u[r], __fsub_rn(gc[1], kmax));
                if (gap > 0.f && __fmul_rn(gap, kBestFirst) >= gap_tot) {
                    const int64_t r1 = 2 * r + 1, r2 = 2 * r + 2;
                    const float k1 = kernel_bounds(fp, q, r1, c32).kmax;
                    const float k2 = kernel_bounds(fp, q, r2, c32).kmax;
                    dl = fmaxf(dl, __fadd_rd(__fmul_rd(fp.rW32d[r1], k1), __fmul_rd(fp.rW32d[r2], k2)));
                }
                gc[3] = dl;
                s_dl = __fadd_rd(s_dl, dl);
            }
        } else {
            for (int k = lane; k < G.cnt; k += 32) {
                const int64_t r = pr[G.off + k];
                const KBounds kb = kernel_bounds(fp, q, r, c32);
                float *gc = fp.geo + 4 * (G.off + k);
                const float dl = __fmul_rd(fp.rW32d[r], kb.kmax);
                *reinterpret_cast<float4 *>(gc) = make_float4(kb.kmax, kb.kmin, kb.e4, dl);
                s_dl = __fadd_rd(s_dl, dl);
                s_W = __fadd_ru(s_W, fp.rW32u[r]);
            }
        }
        const float front32 = warp_sum_rd(s_dl), Wg32 = warp_sum_ru(s_W);
        const int64_t qj = q * fp.nh + j;
        const int64_t cq = node_size(fp.qn, fp.q_depth, q);
        // per group: token per unit weight and the Theorem 2 scale W / (eps G),
        // and the FP32 thresholds derived from them.  Lane 0 computes them and
        // the warp reads them by shuffle (FP64 runs at a low rate; a value
        // every lane computes costs 32 lanes of it).
        // FP32 screen of the FD test (n_fd <= allot  <=>  (K(dmin)-K(dmax)) kappa/2 <= 1 + share):
        // pairs it rejects fail the exact FP64 test by a margin of 1e-4, so the
        // FP64 test only runs where it can succeed; decisions are unchanged.
        // Screen of the series bounds: see thrL below.
        double front = 0.0, fin0 = 0.0, tok0 = 0.0, rQ = 0.0, share = 0.0, kappa = 0.0;
        float hk32 = 0.f, thr32 = 0.f, thrL = 0.f, invhd = 0.f;
        int screen_i = 0;
        if (lane == 0) {
            front = (double)front32;
            const double Wg = (double)Wg32;
            fin0 = fp.fin[qj];
            tok0 = fp.tok[qj];
            double Gb = fin0 + front;
            if (fp.mono) Gb = fmax(Gb, (double)fp.qwmin[q]);
            Gb = fmax(Gb, floorW);
            rQ = fp.qrad[q] * invh;
            share = tok0 / Wg;
            kappa = Wtot / (eps_t * Gb);
            const double st = fp.tokens ? share : 0.0;
            screen_i = 0.5 * kappa < 1e37;   // kappa/2 representable in FP32
            hk32 = screen_i ? (float)(0.5 * kappa) : 0.f;
            thr32 = (float)(1.0 + st) * 1.0001f;
            thrL = __fmul_ru(__double2float_ru(1.0 + st), 0x1.00001p+0f);
            invhd = __double2float_rd(invh);
        }
        const unsigned full = 0xffffffffu;
        rQ = __shfl_sync(full, rQ, 0);
        share = __shfl_sync(full, share, 0);
        kappa = __shfl_sync(full, kappa, 0);
        hk32 = __shfl_sync(full, hk32, 0);
        thr32 = __shfl_sync(full, thr32, 0);
        thrL = __shfl_sync(full, thrL, 0);
        invhd = __shfl_sync(full, invhd, 0);
        const bool screen = __shfl_sync(full, screen_i, 0) != 0;
        // pass 2: decisions
        float s_bank = 0.f, s_fin = 0.f;   // FP32 rounded down, like the lower bound
        double s_paid = 0.0, s_est = 0.0;
        int n_fd = 0, n_dh = 0, n_dl = 0, n_h2l = 0, n_base = 0, n_split = 0;
        const double share_t = fp.tokens ? share : 0.0;
        // Screen of the series bounds: a lower bound of E_p kappa / W_R computed
        // with every FP32 operation rounded down from inputs rounded down
        // (overflow gives FLT_MAX, underflow rounds towards zero, so it is a
        // lower bound whatever the magnitudes).  The exact FP64 test passes
        // only if E_p kappa / W_R <= (1 + share)(1 + 2^-40), so a lower bound
        // above (1 + share)(1 + 2^-20) rejects only bounds the FP64 test
        // rejects.  Per group and order: hk = F_p kappa, gdl = hk r_Q^p (DL),
        // A = r_Q^p and B = C(D+p-1, D) tail_p (H2L).
        const bool series = (MODE == 2 ? fp.selector != GS_SEL_EXHAUSTIVE
                                        : (fp.selector == GS_SEL_RULE || fp.selector == GS_SEL_MLP)) &&
                            fp.P >= 1;
        // (thrL = (1 + share)(1 + 2^-20) rounded up, from lane 0)
        float *tab = s_tab[threadIdx.x >> 5];
        // per-group feature constants of the selector
        const float hkf = (float)(0.5 * kappa < 1e37 ? 0.5 * kappa : 1e37);
        const float thrf = (float)(1.0 + share_t);
        const float lhd = plog2_f((float)(diam * invh));
        __syncwarp();
        if (series && lane >= 1 && lane <= fp.P) {
            const int p = lane;
            const float hk = __double2float_rd(fp.F[p] * kappa);
            const float rq = __double2float_rd(rQ);
            float a = 1.f;
            for (int i = 0; i < p; ++i) a = __fmul_rd(a, rq);
            float tl = 1.f;
            const double x2 = kSqrt2 * rQ;
            if (!(x2 <= 1.0)) {
                const float x2d = __double2float_rd(x2);
                for (int i = 0; i < p - 1; ++i) tl = __fmul_rd(tl, x2d);
            }
            tab[0 * 17 + p] = hk;
            tab[1 * 17 + p] = __fmul_rd(hk, a);
            tab[2 * 17 + p] = a;
            tab[3 * 17 + p] = __fmul_rd(__double2float_rd(fp.BT[p]), tl);
        }
        __syncwarp();
        const int iq = (int)(cq - (fp.qn >> fp.q_depth));
        for (int k = lane; k < G.cnt; k += 32) {
            const int64_t r = pr[G.off + k];
            const float4 gc = *reinterpret_cast<const float4 *>(fp.geo + 4 * (G.off + k));
            const float kmax32 = gc.x, kmin32 = gc.y;
            const float e4f = gc.z;
            const double WR = fp.rW[r];
            int method = (fp.q_leaf && fp.r_leaf) ? M_BASE : M_SPLIT;
            int pord = 0;
            double spent = 0.0;
            bool decided = false;
            if (fp.selector != GS_SEL_EXHAUSTIVE && !(screen && (kmin32 - kmax32) * hk32 > thr32)) {
                const double kmax = (double)kmax32, kmin = (double)kmin32;
                const double allot = fp.tokens ? WR * share : 0.0;
                const double e_fd = (WR * (kmin - kmax)) * 0.5;
                const double n_fd = e_fd * kappa - WR;
                if (n_fd <= allot) {
                    method = M_FD;
                    spent = n_fd;
                    decided = true;
                    s_est = s_est + (WR * (kmin + kmax)) * 0.5;
                }
            }
            const int64_t crn = node_size(fp.rn, fp.r_depth, r);
            // learned ordering: the network is consulted where the pair's
            // exhaustive work is large enough to repay its inference; other
            // pairs take the rule
            const bool big = MODE == 1 && cq * crn >= (int64_t)GS_MLP_MIN_WORK;
            if ((MODE == 0 || (MODE == 1 && !big)) && !decided && series) {
                // bestMethod (Fig. 6).  Costs grow with p, so a method whose
                // cost already reaches the best so far (or exceeds c_Direct)
                // cannot be chosen and its remaining bounds are skipped; the
                // choice is the same as evaluating every bound.  Costs are
                // positive, so their order is that of their bit patterns.
                const int ir = (int)(crn - (fp.rn >> fp.r_depth));
                const long long c_ex = __double_as_longlong(fp.cex[iq][ir]);
                long long best_c = 0x7ff0000000000000ll;   // +inf
                double best_need = 0.0;
                int best_m = -1, best_p = 0;
                const float rRd = __fmul_rd(fp.rrad32[r], invhd);
                const float srd = __fmul_rd(rRd, 0x1.6a09e6p+0f);   // sqrt(2) rounded down
                bool have64 = false;
                double base = 0.0, rR = 0.0, sr = 0.0, allot = 0.0;
                for (int m = M_DH; m <= M_H2L; ++m) {
                    float pw = 1.f;
                    for (int p = 1; p <= fp.P; ++p) {
                        const double cd = m == M_DH ? fp.cDH[iq][p] : (m == M_DL ? fp.cDL[ir][p] : fp.cH2L[p]);
                        const long long c = __double_as_longlong(cd);
                        if (c >= best_c || c > c_ex) break;
                        float lb;
                        if (m == M_DH) {
                            pw = __fmul_rd(pw, rRd);
                            lb = __fmul_rd(__fmul_rd(e4f, tab[p]), pw);
                        } else if (m == M_DL) {
                            lb = __fmul_rd(e4f, tab[17 + p]);
                        } else {
                            pw = __fmul_rd(pw, srd);
                            lb = __fmul_rd(__fmul_rd(e4f, tab[p]), __fadd_rd(tab[34 + p], __fmul_rd(pw, tab[51 + p])));
                        }
                        if (lb > thrL) continue;
                        if (!have64) {
                            have64 = true;
                            base = WR * (double)e4f;
                            rR = fp.rrad[r] * invh;
                            sr = kSqrt2 * rR;
                            allot = fp.tokens ? WR * share : 0.0;
                        }
                        double Ep;
                        if (m == M_DH) {
                            Ep = (base * fp.F[p]) * rpow(rR, p);
                        } else if (m == M_DL) {
                            Ep = (base * fp.F[p]) * rpow(rQ, p);
                        } else {
                            const double x2 = kSqrt2 * rQ;
                            const double tail = (x2 <= 1.0) ? 1.0 : rpow(x2, p - 1);
                            Ep = (base * fp.F[p]) * (rpow(rQ, p) + (rpow(sr, p) * fp.BT[p]) * tail);
                        }
                        const double np_ = Ep * kappa - WR;
                        if (np_ <= allot) {
                            best_c = c;
                            best_m = m;
                            best_p = p;
                            best_need = np_;
                            break;
                        }
                    }
                }
                if (best_m >= 0) {
                    method = best_m;
                    pord = best_p;
                    spent = best_need;
                    decided = true;
                }
            }
            if (MODE == 2 || big) {
                // smallest certified order of each series method (no cost cut-offs)
                const bool fd_pruned = decided;
                int pc3[3] = {0, 0, 0};
                double need3[3] = {0.0, 0.0, 0.0};
                if (!decided && series) {
                    const float rRd = __fmul_rd(fp.rrad32[r], invhd);
                    const float srd = __fmul_rd(rRd, 0x1.6a09e6p+0f);
                    const double base = WR * (double)e4f;
                    const double rR = fp.rrad[r] * invh;
                    const double sr = kSqrt2 * rR;
                    const double allot = fp.tokens ? WR * share : 0.0;
                    for (int m = M_DH; m <= M_H2L; ++m) {
                        float pw = 1.f;
                        for (int p = 1; p <= fp.P; ++p) {
                            float lb;
                            if (m == M_DH) {
                                pw = __fmul_rd(pw, rRd);
                                lb = __fmul_rd(__fmul_rd(e4f, tab[p]), pw);
                            } else if (m == M_DL) {
                                lb = __fmul_rd(e4f, tab[17 + p]);
                            } else {
                                pw = __fmul_rd(pw, srd);
                                lb = __fmul_rd(__fmul_rd(e4f, tab[p]), __fadd_rd(tab[34 + p], __fmul_rd(pw, tab[51 + p])));
                            }
                            if (lb > thrL) continue;
                            double Ep;
                            if (m == M_DH) {
                                Ep = (base * fp.F[p]) * rpow(rR, p);
                            } else if (m == M_DL) {
                                Ep = (base * fp.F[p]) * rpow(rQ, p);
                            } else {
                                const double x2 = kSqrt2 * rQ;
                                const double tail = (x2 <= 1.0) ? 1.0 : rpow(x2, p - 1);
                                Ep = (base * fp.F[p]) * (rpow(rQ, p) + (rpow(sr, p) * fp.BT[p]) * tail);
                            }
                            const double np_ = Ep * kappa - WR;
                            if (np_ <= allot) {
                                pc3[m - 1] = p;
                                need3[m - 1] = np_;
                                break;
                            }
                        }
                    }
                }
                const bool contested = (pc3[0] | pc3[1] | pc3[2]) != 0;
                const int64_t cr = crn;
                const bool consult = contested;
                float xf[kMlpIn];
                if (!fd_pruned && (MODE == 2 || consult)) {
                    // pair features: kernel bounds, node sizes, D, FD budget ratio,
                    // radii / h, W_R / W, level, diameter / h, PLIMIT
                    xf[0] = plog2_f(kmin32);
                    xf[1] = plog2_f(kmax32);
                    xf[2] = plog2_f((float)cq);
                    xf[3] = plog2_f((float)cr);
                    xf[4] = (float)fp.D;
                    xf[5] = plog2_f(__fdiv_rn(thrf, __fmul_rn(__fsub_rn(kmin32, kmax32), hkf)));
                    xf[6] = plog2_f((float)rQ);
                    xf[7] = plog2_f((float)(fp.rrad[r] * invh));
                    xf[8] = plog2_f((float)(WR / Wtot));
                    xf[9] = (float)fp.t;
                    xf[10] = lhd;
                    xf[11] = (float)fp.P;
                }
                if constexpr (MODE == 1) {
                    int best = 4;
                    if (consult) {
                        // highest-scoring certified action; split / base case is always certified
                        float o[kMlpOut];
                        mlp_infer(s_w, xf, o);
                        best = -1;
                        for (int a = 1; a <= 4; ++a) {
                            const bool cert = a == 4 || pc3[a - 1] > 0;
                            if (cert && (best < 0 || o[a] > o[best])) best = a;
                        }
                    }
                    if (best <= 3) {
                        method = best;
                        pord = pc3[best - 1];
                        spent = need3[best - 1];
                        decided = true;
                    }
                } else {
                    const int64_t gid = fp.log_base + G.off + k;
                    fp.lnq[gid] = (int32_t)cq;
                    fp.lnr[gid] = (int32_t)cr;
                    fp.lpar[gid] = fp.pid ? fp.pid[G.off + k] : -1;
                    int8_t *pc = fp.lpc + 4 * gid;
                    pc[0] = (int8_t)pc3[0];
                    pc[1] = (int8_t)pc3[1];
                    pc[2] = (int8_t)pc3[2];
                    pc[3] = (int8_t)(fd_pruned ? LOG_FD : (method == M_BASE ? LOG_BASE : LOG_SPLIT));
                    if (!fd_pruned)
                        for (int i = 0; i < kMlpIn; ++i) fp.lfeat[kMlpIn * gid + i] = xf[i];
                }
            }
            if (method == M_FD || (method >= M_DH && method <= M_H2L)) s_paid = s_paid + spent;
            if (method == M_BASE) s_bank = __fadd_rd(s_bank, fp.rW32d[r]);
            // at a leaf-leaf iteration no pair splits, so this sum equals pass 1's s_dl
            if (method != M_SPLIT && !(fp.q_leaf && fp.r_leaf)) s_fin = __fadd_rd(s_fin, gc.w);
            n_fd += method == M_FD;
            n_dh += method == M_DH;
            n_dl += method == M_DL;
            n_h2l += method == M_H2L;
            n_base += method == M_BASE;
            n_split += method == M_SPLIT;
            dec[G.off + k] = (uint8_t)(method | (pord << 3));
            if (trace) {
                const int64_t ti = trace_base + G.off + k;
                if (ti < trace_cap)
                    trace[ti] = make_int4((int)q, (int)r, j, method | (pord << 8) | (fp.t << 16));
            }
        }
        const float bank32 = warp_sum_rd(s_bank);
        const float fin32 = (fp.q_leaf && fp.r_leaf) ? 0.f : warp_sum_rd(s_fin);
        const double paid = warp_sum_sparse_lane0(s_paid);   // lane 0's values below
        const double est_add = warp_sum_sparse_lane0(s_est);
        int n_m[6] = {n_fd, n_dh, n_dl, n_h2l, n_base, n_split};
#pragma unroll
        for (int m = 0; m < 6; ++m) n_m[m] = __reduce_add_sync(0xffffffffu, n_m[m]);
        if (lane == 0) {
            const double banked = (double)bank32;
            const double fin_add = (fp.q_leaf && fp.r_leaf) ? front : (double)fin32;
            // Fig. 7's token update over the whole group: pruned pairs pay their
            // need, base cases bank W_R, splits leave the token alone
            const double tok_new = fp.tokens ? fmax(0.0, (tok0 + banked) - paid) : 0.0;
            const double fin_new = fin0 + fin_add;
            fp.fin[qj] = fin_new;
            fp.tok[qj] = tok_new;
            fp.est[qj] = fp.est[qj] + est_add;
            if (!fp.q_leaf) {
                for (int c = 1; c <= 2; ++c) {
                    fp.fin[(2 * q + c) * fp.nh + j] = fin_new;
                    fp.tok[(2 * q + c) * fp.nh + j] = tok_new;
                }
            }
            const int n_sp = n_m[M_SPLIT];
            int child_pairs, child_groups;
            if (fp.q_leaf) {
                child_pairs = 2 * n_sp;
                child_groups = n_sp > 0;
            } else if (fp.r_leaf) {
                child_pairs = 2 * n_sp;
                child_groups = n_sp > 0 ? 2 : 0;
            } else {
                child_pairs = 4 * n_sp;
                child_groups = n_sp > 0 ? 2 : 0;
            }
            int32_t *c = cnt + g * kCols;
            c[C_PAIRS] = child_pairs;
            c[C_GROUPS] = child_groups;
            c[C_BASE] = n_m[M_BASE];
            c[C_DH] = n_m[M_DH];
            c[C_DL] = n_m[M_DL];
            c[C_H2L] = n_m[M_H2L];
            c[C_BGROUPS] = n_m[M_BASE] > 0;
            for (int m = 0; m < 6; ++m)
                if (n_m[m]) atomicAdd(&fs->method_count[m], (unsigned long long)n_m[m]);
        }
    }
}

// ---------------------------------------------------------------------------
// column scan over groups (3 phases, fixed grid)
// ---------------------------------------------------------------------------
constexpr int kColGrid = 256;
constexpr int kColTB = 256;

__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *tot) {
    __shared__ long long wsum[kColTB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long s = lane < kColTB / 32 ? wsum[lane] : 0;
        long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += u;
        }
        if (lane < kColTB / 32) wsum[lane] = si - s;
        if (lane == kColTB / 32 - 1) *tot = si;
    }
    __syncthreads();
    const long long r = wsum[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kColTB)
k_cols_partial(const FrontierState *fs, int t, const int32_t *__restrict__ cnt, long long *partial) {
    __shared__ long long tot;
    const int64_t ng = fs->ngroups[t];
    const int64_t chunk = (ng + gridDim.x - 1) / gridDim.x;
    const int64_t g0 = blockIdx.x * chunk, g1 = min(g0 + chunk, ng);
    for (int c = 0; c < kCols; ++c) {
        long long s = 0;
        for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) s += cnt[g * kCols + c];
        block_excl_scan_ll(s, &tot);
        if (threadIdx.x == 0) partial[c * kColGrid + blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(kColTB) k_cols_scan_partials(FrontierState *fs, long long *partial) {
    __shared__ long long tot;
    for (int c = 0; c < kCols; ++c) {
        const long long v = partial[c * kColGrid + threadIdx.x];
        const long long e = block_excl_scan_ll(v, &tot);
        partial[c * kColGrid + threadIdx.x] = e;
        if (threadIdx.x == 0) fs->totals[c] = tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kColTB)
k_cols_offsets(const FrontierState *fs, int t, const int32_t *__restrict__ cnt, const long long *__restrict__ partial,
               long long *off) {
    __shared__ long long tot;
    const int64_t ng = fs->ngroups[t];
    const int64_t chunk = (ng + gridDim.x - 1) / gridDim.x;
    const int64_t g0 = blockIdx.x * chunk, g1 = min(g0 + chunk, ng);
    for (int c = 0; c < kCols; ++c) {
        long long carry = partial[c * kColGrid + blockIdx.x];
        for (int64_t t0 = g0; t0 < g1; t0 += blockDim.x) {
            const int64_t g = t0 + threadIdx.x;
            const long long v = g < g1 ? cnt[g * kCols + c] : 0;
            const long long e = block_excl_scan_ll(v, &tot);
            if (g < g1) off[g * kCols + c] = carry + e;
            carry += tot;
        }
    }
}

// the same column scan by one CTA, for frontiers of at most kColSmall groups
// (one launch instead of three)
constexpr int64_t kColSmall = 4096;

__global__ void __launch_bounds__(kColTB)
k_cols_small(FrontierState *fs, int t, const int32_t *__restrict__ cnt, long long *off) {
    __shared__ long long tot;
    const int64_t ng = fs->ngroups[t];
    for (int c = 0; c < kCols; ++c) {
        long long carry = 0;
        for (int64_t t0 = 0; t0 < ng; t0 += blockDim.x) {
            const int64_t g = t0 + threadIdx.x;
            const long long v = g < ng ? cnt[g * kCols + c] : 0;
            const long long e = block_excl_scan_ll(v, &tot);
            if (g < ng) off[g * kCols + c] = carry + e;
            carry += tot;
        }
        if (threadIdx.x == 0) fs->totals[c] = carry;
    }
}

// ---------------------------------------------------------------------------
// K2: write the child frontier, base pairs and series actions
// ---------------------------------------------------------------------------
struct EmitOut {
    Group *groups_next;
    int32_t *pr_next;
    Group *base_groups;
    int32_t *base_r;
    SeriesEntry *series[3];
    int64_t *pid_next;    // pair log: parent id of every child pair (null when not logging)
    int64_t log_base;
};

__global__ void __launch_bounds__(256)
k_front_emit(FrontierState *fs, int t, int q_leaf, int r_leaf, const Group *__restrict__ groups,
             const int32_t *__restrict__ pr, const uint8_t *__restrict__ dec, const int32_t *__restrict__ cnt,
             const long long *__restrict__ off, EmitOut eo) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = fs->ngroups[t];
    const int64_t base0 = fs->base_count, bg0 = fs->base_groups;
    const int64_t ser0[3] = {fs->series_count[0], fs->series_count[1], fs->series_count[2]};
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < ng; g += warps) {
        const Group G = groups[g];
        const int32_t *c = cnt + g * kCols;
        const long long *o = off + g * kCols;
        const int64_t o_pairs = o[C_PAIRS], o_groups = o[C_GROUPS], o_base = base0 + o[C_BASE];
        const int64_t o_bg = bg0 + o[C_BGROUPS];
        int64_t o_ser[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) o_ser[m] = ser0[m] + o[C_DH + m];
        const int n_split = q_leaf ? c[C_PAIRS] / 2 : (r_leaf ? c[C_PAIRS] / 2 : c[C_PAIRS] / 4);
        const int per_child = r_leaf ? n_split : 2 * n_split;
        int run_s = 0, run_b = 0, run_x[3] = {0, 0, 0};
        for (int k0 = 0; k0 < G.cnt; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < G.cnt;
            const int d = valid ? dec[G.off + k] : 0xff;
            const int m = d & 7;
            const bool isS = valid && m == M_SPLIT, isB = valid && m == M_BASE;
            const unsigned bS = __ballot_sync(0xffffffffu, isS), bB = __ballot_sync(0xffffffffu, isB);
            unsigned bX[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) bX[x] = __ballot_sync(0xffffffffu, valid && m == M_DH + x);
            const int32_t r = valid ? pr[G.off + k] : 0;
            if (isS) {
                const int rank = run_s + __popc(bS & lt_mask);
                const int64_t gid = eo.log_base + G.off + k;
                if (!q_leaf && !r_leaf) {
                    for (int cc = 0; cc < 2; ++cc) {
                        const int64_t p = o_pairs + (int64_t)cc * per_child + 2 * rank;
                        eo.pr_next[p] = 2 * r + 1;
                        eo.pr_next[p + 1] = 2 * r + 2;
                        if (eo.pid_next) eo.pid_next[p] = eo.pid_next[p + 1] = gid;
                    }
                } else if (q_leaf) {
                    const int64_t p = o_pairs + 2 * rank;
                    eo.pr_next[p] = 2 * r + 1;
                    eo.pr_next[p + 1] = 2 * r + 2;
                    if (eo.pid_next) eo.pid_next[p] = eo.pid_next[p + 1] = gid;
                } else {
                    for (int cc = 0; cc < 2; ++cc) {
                        const int64_t p = o_pairs + (int64_t)cc * per_child + rank;
                        eo.pr_next[p] = r;
                        if (eo.pid_next) eo.pid_next[p] = gid;
                    }
                }
            }
            if (isB) eo.base_r[o_base + run_b + __popc(bB & lt_mask)] = r;
            // the three series lists, indexed by compile-time constants so that
            // the per-list counters stay in registers
#pragma unroll
            for (int x = 0; x < 3; ++x)
                if (valid && m == M_DH + x) {
                    SeriesEntry e;
                    e.q = G.q;
                    e.r = r;
                    e.j = (int16_t)G.j;
                    e.p = (int8_t)(d >> 3);
                    e.method = (int8_t)m;
                    e.pad = 0;
                    eo.series[x][o_ser[x] + run_x[x] + __popc(bX[x] & lt_mask)] = e;
                }
            run_s += __popc(bS);
            run_b += __popc(bB);
#pragma unroll
            for (int x = 0; x < 3; ++x) run_x[x] += __popc(bX[x]);
        }
        if (lane == 0) {
            if (n_split > 0) {
                if (q_leaf) {
                    Group ng_;
                    ng_.q = G.q; ng_.j = G.j; ng_.off = o_pairs; ng_.cnt = 2 * n_split; ng_.pad = 0;
                    eo.groups_next[o_groups] = ng_;
                } else {
                    for (int cc = 0; cc < 2; ++cc) {
                        Group ng_;
                        ng_.q = 2 * G.q + 1 + cc; ng_.j = G.j; ng_.off = o_pairs + (int64_t)cc * per_child;
                        ng_.cnt = per_child; ng_.pad = 0;
                        eo.groups_next[o_groups + cc] = ng_;
                    }
                }
            }
            if (c[C_BASE] > 0) {
                Group bg;
                bg.q = G.q; bg.j = G.j; bg.off = o_base; bg.cnt = c[C_BASE]; bg.pad = 0;
                eo.base_groups[o_bg] = bg;
            }
        }
    }
}

__global__ void k_front_advance(FrontierState *fs, int t) {
    fs->trace_count += fs->npairs[t];
    fs->ngroups[t + 1] = fs->totals[C_GROUPS];
    fs->npairs[t + 1] = fs->totals[C_PAIRS];
    fs->base_count += fs->totals[C_BASE];
    for (int m = 0; m < 3; ++m) fs->series_count[m] += fs->totals[C_DH + m];
    fs->base_groups += fs->totals[C_BGROUPS];
}

// initial frontier: one group (root, j) with the single pair (root, root) per
// bandwidth; eps for the traversal after the FP32 base-case charge.
__global__ void k_front_init(FrontierState *fs, Group *groups, int32_t *pr, int nh, const double *rW,
                             const double *rlo, const double *rhi, Ingest *ing, int64_t N, int D, int floor_log2,
                             double eps, int64_t run, double extra_rho) {
    const int j = threadIdx.x;
    if (j < nh) {
        Group g;
        g.q = 0; g.j = j; g.off = j; g.cnt = 1; g.pad = 0;
        groups[j] = g;
        pr[j] = 0;
    }
    if (j == 0) {
        const double W = rW[0];
        const double wmax = (double)__uint_as_float(ing->wmax_bits);
        const double u = 5.9604644775390625e-08;   // 2^-24
        double rho = 0.6931471805599453 * 64.0 * (double)(D + 5) * u;   // d^2 (D+3), the FMA, l
        rho = rho + 4.76837158203125e-07;          // 2^-21
        rho = rho + (double)(run + 1) * u;      // FP32 sums over one reference leaf, then compensated
        rho = rho + ldexp(1.0, -63 - floor_log2) * (((double)N * wmax) / W);
        rho = rho + extra_rho;                   // the tensor-core base case's charge, when enabled
        fs->rho = rho;
        fs->eps_t = eps - rho;
        fs->Wtot = W;
        fs->floorW = W * ldexp(1.0, floor_log2);
        fs->ngroups[0] = nh;
        fs->npairs[0] = nh;
        double d2 = 0.0;
        for (int d = 0; d < D; ++d) d2 = d2 + (rhi[d] - rlo[d]) * (rhi[d] - rlo[d]);
        fs->diam = sqrt(d2);
        if (!(fs->eps_t > 0.5 * eps)) atomicOr(&ing->status, ST_EPS);
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static bool g_consts_ready[64] = {false};
static std::mutex g_consts_mu;

// exp2 coefficients ln2^n / n! built in FP64 by repeated multiplication,
// then rounded to FP32; uploaded once per device
static int ensure_consts() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_consts_mu);
    if (dev >= 0 && dev < 64 && g_consts_ready[dev]) return GS_OK;
    float c[8];
    double t = 1.0;
    for (int n = 0; n < 8; ++n) {
        c[n] = (float)t;
        t = (t * 0.6931471805599453) / (double)(n + 1);
    }
    GS_CUDA_TRY(cudaMemcpyToSymbol(c_e2, c, sizeof(c)));
    if (dev >= 0 && dev < 64) g_consts_ready[dev] = true;
    return GS_OK;
}

static unsigned long long binom_u64(int a, int b) {
    unsigned long long r = 1;
    for (int i = 1; i <= b; ++i) r = r * (unsigned long long)(a - b + i) / (unsigned long long)i;
    return r;
}

static double factd(int m) {
    double f = 1.0;
    for (int q = 2; q <= m; ++q) f = f * (double)q;
    return f;
}

// worst-case list memory below which a traversal runs without per-iteration
// host reads of its totals
constexpr double kPresizedBytes = 64.0 * 1024 * 1024;

// Grow a device array to hold at least `need` elements, keeping the first
// `keep` elements.
template <typename E>
static int grow(E **ptr, int64_t *cap, int64_t need, int64_t keep, cudaStream_t st) {
    if (need <= *cap) return GS_OK;
    int64_t nc = *cap * 2;
    if (nc < need + need / 2) nc = need + need / 2;
    E *np = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&np, (size_t)nc * sizeof(E), st));
    if (keep > 0 && *ptr) GS_CUDA_TRY(cudaMemcpyAsync(np, *ptr, (size_t)keep * sizeof(E), cudaMemcpyDeviceToDevice, st));
    if (*ptr) cudaFreeAsync(*ptr, st);
    *ptr = np;
    *cap = nc;
    return GS_OK;
}

int run_frontier(const TraversalIn &in, FrontierBufs &fb, CallCtx &cx) {
    cudaStream_t st = cx.st;
    int rc = cx.check("before frontier");
    if (rc) return rc;
    rc = ensure_consts();
    if (rc) return rc;
    FrontierParams fp;
    memset(&fp, 0, sizeof(fp));
    fp.D = in.D;
    fp.nh = in.nh;
    fp.P = in.P;
    fp.selector = in.selector;
    fp.tokens = in.tokens;
    fp.mono = in.mono;
    fp.best_first = (in.flags & GS_FLAG_BEST_FIRST) != 0;
    fp.floor_log2 = in.floor_log2;
    fp.qn = in.qt->n;
    fp.rn = in.rt->n;
    fp.qlo32 = in.qt->lo32; fp.qhi32 = in.qt->hi32; fp.qrad = in.qt->rad; fp.qwmin = in.qt->wmin;
    fp.rlo32 = in.rt->lo32; fp.rhi32 = in.rt->hi32; fp.rrad = in.rt->rad; fp.rW = in.rt->W;
    fp.rrad32 = in.rt->rad32;
    fp.rW32d = in.rt->W32d;
    fp.rW32u = in.rt->W32u;
    fp.inv_h = fb.inv_h;
    for (int j = 0; j < in.nh; ++j) fp.c32[j] = (float)(1.4426950408889634 / ((2.0 * in.h[j]) * in.h[j]));
    fp.fin = fb.fin; fp.tok = fb.tok; fp.est = fb.est;
    for (int k = 0; k < 4; ++k) fp.cw[k] = in.cost_w[k];
    const int D = in.D;
    // Lemma 4-6 factor C(D+p-1, D-1) / sqrt((floor(p/D)!)^(D-p') (ceil(p/D)!)^p'),
    // C(D+p-1, D), and D^k, all from exact integers
    for (int p = 1; p <= 16 && p <= in.P; ++p) {
        const int pp = p % D;
        double prod = 1.0;
        for (int i = 0; i < D - pp; ++i) prod = prod * factd(p / D);
        for (int i = 0; i < pp; ++i) prod = prod * factd((p + D - 1) / D);
        fp.F[p] = (double)binom_u64(D + p - 1, D - 1) / sqrt(prod);
        fp.BT[p] = (double)binom_u64(D + p - 1, D);
    }
    fp.Dpow[0] = 1.0;
    for (int k = 1; k < 34; ++k) fp.Dpow[k] = fp.Dpow[k - 1] * (double)D;

    // Small problems: every list at its worst-case size up front, so that the
    // iterations run without reading their totals on the host (one read after
    // the last).  The pairs of iteration t are distinct (query node, reference
    // node, bandwidth) triples of levels min(t, depth), so there are at most
    // nh 2^min(t, dQ) 2^min(t, dR) of them, and every action list holds at most
    // the sum of that over the iterations.
    const int T = in.qt->depth > in.rt->depth ? in.qt->depth : in.rt->depth;
    const int qd = in.qt->depth, rd = in.rt->depth;
    bool presized = !in.log && !fb.trace && qd + rd <= 40;
    int64_t pmax = 0, psum = 0;
    if (presized) {
        for (int t = 0; t <= T; ++t) {
            const int64_t p = (int64_t)in.nh << ((t < qd ? t : qd) + (t < rd ? t : rd));
            pmax = p > pmax ? p : pmax;
            psum += p;
        }
        const double bytes = (double)pmax * (2 * sizeof(int32_t) + 1 + 4 * sizeof(float)) +
                             (double)psum * (sizeof(int32_t) + 3 * sizeof(SeriesEntry));
        presized = bytes <= kPresizedBytes;
    }
    if (presized) {
        for (int b = 0; b < 2; ++b)
            if ((rc = grow(&fb.pr[b], &fb.cap_pr[b], pmax, 0, st))) return rc;
        if ((rc = grow(&fb.dec, &fb.cap_pairs, pmax, 0, st))) return rc;
        if ((rc = grow(&fb.geo, &fb.cap_geo, 4 * pmax, 0, st))) return rc;
        if ((rc = grow(&fb.base_r, &fb.cap_base, psum, 0, st))) return rc;
        for (int m = 0; m < 3; ++m)
            if ((rc = grow(&fb.series[m], &fb.cap_series[m], psum, 0, st))) return rc;
    }
    k_front_init<<<1, 64, 0, st>>>(fb.fs, fb.groups[0], fb.pr[0], in.nh, in.rt->W, in.rt->lo, in.rt->hi,
                                   (Ingest *)in.ing, in.rt->n, in.D, in.floor_log2, in.eps,
                                   (in.rt->n + (1ll << in.rt->depth) - 1) >> in.rt->depth,
                                   tc_base_enabled(in.D, in.qt->dtype, in.flags, in.qt->n, in.qt->depth, in.rt->n,
                                                   in.rt->depth, in.nh)
                                       ? tc_charge()
                                       : 0.0);
    cx.launches += 1;
    if ((rc = cx.check("k_front_init"))) return rc;
    int cur = 0;
    int64_t ng = in.nh, npairs = in.nh;
    int64_t base_count = 0, bgroups = 0, ser_count[3] = {0, 0, 0};
    int64_t log_base = 0;
    const int max_grid = fb.grid_warps / 8;
    fp.mlp = in.mlp;
    for (int t = 0; t <= T && (presized || ng > 0); ++t) {
        fp.t = t;
        fp.q_depth = t < in.qt->depth ? t : in.qt->depth;
        fp.r_depth = t < in.rt->depth ? t : in.rt->depth;
        fp.q_leaf = t >= in.qt->depth;
        fp.r_leaf = t >= in.rt->depth;
        // bestMethod costs (Fig. 6) times their weights; node sizes at a level
        // are floor(n / 2^depth) or one more, so each cost takes two values
        for (int a = 0; a < 2; ++a) {
            const double cq = (double)((fp.qn >> fp.q_depth) + a);
            const double cr = (double)((fp.rn >> fp.r_depth) + a);
            for (int p = 1; p <= 16 && p <= in.P; ++p) {
                fp.cDH[a][p] = (cq * fp.Dpow[p + 1]) * fp.cw[0];
                fp.cDL[a][p] = (cr * fp.Dpow[p + 1]) * fp.cw[1];
            }
            for (int b = 0; b < 2; ++b)
                fp.cex[a][b] = (((double)D * cq) * (double)((fp.rn >> fp.r_depth) + b)) * fp.cw[3];
        }
        for (int p = 1; p <= 16 && p <= in.P; ++p) fp.cH2L[p] = fp.Dpow[2 * p + 1] * fp.cw[2];
        // this iteration's per-pair arrays
        if (!presized) {
            if ((rc = grow(&fb.dec, &fb.cap_pairs, npairs, 0, st))) return rc;
            if ((rc = grow(&fb.geo, &fb.cap_geo, 4 * npairs, 0, st))) return rc;
        }
        fp.geo = fb.geo;
        PairLog *lg = in.log;
        if (lg) {
            // the pair log grows by this iteration's pairs
            if (t + 1 >= 80) {
                set_error("pair log: too many iterations");
                return GS_ERR_ARG;
            }
            const int64_t need = log_base + npairs, keep = log_base;
            if (need > lg->cap) {
                const int64_t nc = need + need / 2 > 2 * lg->cap ? need + need / 2 : 2 * lg->cap;
                int64_t c1 = lg->cap * kMlpIn, c2 = lg->cap * 4, c3 = lg->cap, c4 = lg->cap, c5 = lg->cap;
                if ((rc = grow(&lg->feat, &c1, nc * kMlpIn, keep * kMlpIn, st))) return rc;
                if ((rc = grow(&lg->pc, &c2, nc * 4, keep * 4, st))) return rc;
                if ((rc = grow(&lg->nq, &c3, nc, keep, st))) return rc;
                if ((rc = grow(&lg->nr, &c4, nc, keep, st))) return rc;
                if ((rc = grow(&lg->par, &c5, nc, keep, st))) return rc;
                lg->cap = c5;
            }
            lg->iter_off[t] = log_base;
            fp.lfeat = lg->feat; fp.lpc = lg->pc; fp.lnq = lg->nq; fp.lnr = lg->nr; fp.lpar = lg->par;
            fp.pid = t == 0 ? nullptr : lg->pid[cur];
            fp.log_base = log_base;
        }
        // presized: the grid for this level's largest possible group count
        // (the kernels read the actual count on the device)
        const int64_t ngb = presized ? (int64_t)in.nh << (t < qd ? t : qd) : ng;
        const int grid = (int)((ngb + 7) / 8 < max_grid ? (ngb + 7) / 8 : max_grid);
        if (lg)
            k_front_decide<2><<<grid, 256, 0, st>>>(fp, fb.fs, fb.groups[cur], fb.pr[cur], fb.dec, fb.cnt, fb.trace,
                                                    fb.trace_cap);
        else if (in.selector == GS_SEL_MLP)
            k_front_decide<1><<<grid, 256, 0, st>>>(fp, fb.fs, fb.groups[cur], fb.pr[cur], fb.dec, fb.cnt, fb.trace,
                                                    fb.trace_cap);
        else
            k_front_decide<0><<<grid, 256, 0, st>>>(fp, fb.fs, fb.groups[cur], fb.pr[cur], fb.dec, fb.cnt, fb.trace,
                                                    fb.trace_cap);
        if ((rc = cx.check("k_front_decide"))) return rc;
        if (ngb <= kColSmall) {
            k_cols_small<<<1, kColTB, 0, st>>>(fb.fs, t, fb.cnt, fb.off);
            cx.launches += 2;
        } else {
            k_cols_partial<<<kColGrid, kColTB, 0, st>>>(fb.fs, t, fb.cnt, fb.partial);
            k_cols_scan_partials<<<1, kColTB, 0, st>>>(fb.fs, fb.partial);
            k_cols_offsets<<<kColGrid, kColTB, 0, st>>>(fb.fs, t, fb.cnt, fb.partial, fb.off);
            cx.launches += 4;
        }
        if ((rc = cx.check("k_cols_*"))) return rc;
        if (presized) {
            EmitOut eo;
            eo.groups_next = fb.groups[cur ^ 1];
            eo.pr_next = fb.pr[cur ^ 1];
            eo.base_groups = fb.base_groups;
            eo.base_r = fb.base_r;
            for (int m = 0; m < 3; ++m) eo.series[m] = fb.series[m];
            eo.pid_next = nullptr;
            eo.log_base = 0;
            k_front_emit<<<grid, 256, 0, st>>>(fb.fs, t, fp.q_leaf, fp.r_leaf, fb.groups[cur], fb.pr[cur], fb.dec,
                                               fb.cnt, fb.off, eo);
            k_front_advance<<<1, 1, 0, st>>>(fb.fs, t);
            cx.launches += 2;
            if ((rc = cx.check("k_front_emit"))) return rc;
            cur ^= 1;
            continue;
        }
        // read this iteration's totals and make room for what it will write
        GS_CUDA_TRY(cudaMemcpyAsync(fb.host_totals, &fb.fs->totals[0], kCols * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        int64_t tot[kCols];
        for (int c = 0; c < kCols; ++c) tot[c] = fb.host_totals[c];
        if (tot[C_GROUPS] > fb.cap_groups || bgroups + tot[C_BGROUPS] > fb.cap_base_groups) {
            set_error("internal: group count above its bound");
            return GS_ERR_CUDA;
        }
        if ((rc = grow(&fb.pr[cur ^ 1], &fb.cap_pr[cur ^ 1], tot[C_PAIRS], 0, st))) return rc;
        if ((rc = grow(&fb.base_r, &fb.cap_base, base_count + tot[C_BASE], base_count, st))) return rc;
        for (int m = 0; m < 3; ++m)
            if ((rc = grow(&fb.series[m], &fb.cap_series[m], ser_count[m] + tot[C_DH + m], ser_count[m], st)))
                return rc;
        EmitOut eo;
        eo.groups_next = fb.groups[cur ^ 1];
        eo.pr_next = fb.pr[cur ^ 1];
        eo.base_groups = fb.base_groups;
        eo.base_r = fb.base_r;
        for (int m = 0; m < 3; ++m) eo.series[m] = fb.series[m];
        eo.pid_next = nullptr;
        eo.log_base = log_base;
        if (lg) {
            if ((rc = grow(&lg->pid[cur ^ 1], &lg->cap_pid[cur ^ 1], tot[C_PAIRS], 0, st))) return rc;
            eo.pid_next = lg->pid[cur ^ 1];
        }
        k_front_emit<<<grid, 256, 0, st>>>(fb.fs, t, fp.q_leaf, fp.r_leaf, fb.groups[cur], fb.pr[cur], fb.dec,
                                           fb.cnt, fb.off, eo);
        k_front_advance<<<1, 1, 0, st>>>(fb.fs, t);
        cx.launches += 3;
        if ((rc = cx.check("k_front_emit"))) return rc;
        ng = tot[C_GROUPS];
        log_base += npairs;
        if (lg) {
            lg->niter = t + 1;
            lg->iter_off[t + 1] = log_base;
        }
        npairs = tot[C_PAIRS];
        base_count += tot[C_BASE];
        bgroups += tot[C_BGROUPS];
        for (int m = 0; m < 3; ++m) ser_count[m] += tot[C_DH + m];
        cur ^= 1;
    }
    if (presized) {
        // the action-list lengths, read once
        GS_CUDA_TRY(cudaMemcpyAsync(fb.host_totals, &fb.fs->base_count, 6 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                    st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        base_count = fb.host_totals[0];
        bgroups = fb.host_totals[1];
        for (int m = 0; m < 3; ++m) ser_count[m] = fb.host_totals[3 + m];
    }
    for (int m = 0; m < 3; ++m) fb.n_series[m] = ser_count[m];
    fb.n_base_groups = bgroups;
    fb.n_base = base_count;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "frontier launch");
    return GS_OK;
}

}  // namespace gs
