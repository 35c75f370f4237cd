// Training data of the pair selector (not in the paper).
//
// A traversal with FD-only decisions explores every pair that any policy
// with the same FD test can reach, and logs, per pair: its 12 features, the
// smallest order at which each series method (DH, DL, H2L) is certified,
// its node sizes and its parent.  A bottom-up pass over that log (last
// iteration first) gives every pair the modelled cost of its cheapest
// certified handling:
//   FD-pruned:  0
//   leaf pair:  min(base case n_Q n_R u_base, certified series)
//   internal:   min(sum over children (best(child) + u_pair), certified series)
// and, where a series method is certified and N_Q N_R >= GS_MLP_MIN_WORK
// (the pairs the selector is consulted on), the action reaching that
// minimum (DH = 1, DL = 2, H2L = 3, split / base case = 4) as the training
// label, weighted by its regret (second cheapest minus cheapest cost) over
// the problem's mean regret.
// Series costs follow the kernels' operation counts (FP64 lane slots):
//   DH  u_act + n_Q (T_p (D+1) + 3 D p + 30) u_dh
//   DL  u_act + n_R (T_p' (D+1) + 3 D p + 30) u_dl, T_p' = T_p (one lane per
//       reference, T_p <= 32) or 32 ceil(T_p / 32) (lanes over coefficients)
//   H2L u_act + U_p u_h2l,   T_p = C(D+p-1, D), with U_p the H2L kernel's path:
//       p = 1: 4D + 30; p = 2: 16D + 30 (one lane, Lemma 1 written out);
//       D = 3, p = 3..6: 2 p T_p + (p(p+1)/2)^2 + 80 (one lane, summed one
//       dimension at a time);
//       T_p <= 20 and D(2p-1) <= 32: T_p^2 (D+1) + T_p D + 3D(2p-1) + 30 (one lane);
//       otherwise 32 (ceil(T_p/32) T_p (D+1) + 40) (one warp).
#include <math.h>
#include <string.h>

#include "gs_internal.h"
#include "gs_mlp.cuh"

namespace gs {

struct DpArgs {
    const int8_t *pc;
    const int32_t *nq, *nr;
    const int64_t *par;
    double *childsum, *fdsum, *best, *regret;
    int8_t *label;
    double u_pair, u_base, u_dh, u_dl, u_h2l, u_act;
    int D;
    double Tp[17];
};

__device__ __forceinline__ double series_cost(const DpArgs &a, int m, int p, double nq, double nr) {
    const double T = a.Tp[p], D = (double)a.D;
    if (m == 0) return a.u_act + nq * (T * (D + 1.0) + 3.0 * D * p + 30.0) * a.u_dh;
    if (m == 1) {
        const double Tl = T <= 32.0 ? T : 32.0 * ceil(T / 32.0);
        return a.u_act + nr * (Tl * (D + 1.0) + 3.0 * D * p + 30.0) * a.u_dl;
    }
    double U;
    if (p == 1)
        U = 4.0 * D + 30.0;
    else if (p == 2)
        U = 16.0 * D + 30.0;
    else if (a.D == 3 && p <= 6)   // the separable three-dimensional kernel
        U = 2.0 * p * T + (0.5 * p * (p + 1)) * (0.5 * p * (p + 1)) + 80.0;
    else if (T <= 20.0 && a.D * (2 * p - 1) <= 32)
        U = T * T * (D + 1.0) + T * D + 3.0 * D * (2 * p - 1) + 30.0;
    else
        U = 32.0 * (ceil(T / 32.0) * T * (D + 1.0) + 40.0);
    return a.u_act + U * a.u_h2l;
}

__global__ void k_dp_iter(DpArgs a, int64_t g0, int64_t g1) {
    for (int64_t g = g0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < g1;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int8_t *pc = a.pc + 4 * g;
        const int kind = pc[3];
        double b = 0.0, fd = 0.0, b2 = 0.0;
        int lab = -1;
        if (kind != LOG_FD) {
            const double nq = (double)a.nq[g], nr = (double)a.nr[g];
            b = kind == LOG_BASE ? nq * nr * a.u_base : a.childsum[g];
            fd = kind == LOG_BASE ? nq * nr * a.u_base : a.fdsum[g];
            b2 = INFINITY;   // second cheapest certified action
            int l = 4;
            bool any = false;
            for (int m = 0; m < 3; ++m) {
                const int p = pc[m];
                if (p <= 0) continue;
                any = true;
                const double c = series_cost(a, m, p, nq, nr);
                if (c < b) {
                    b2 = b;
                    b = c;
                    l = m + 1;
                } else if (c < b2) {
                    b2 = c;
                }
            }
            // samples only where the selector is consulted
            if (any && (int64_t)a.nq[g] * a.nr[g] >= (int64_t)GS_MLP_MIN_WORK) lab = l;
        }
        a.best[g] = b;
        a.label[g] = (int8_t)lab;
        a.regret[g] = lab >= 0 ? b2 - b : 0.0;
        const int64_t par = a.par[g];
        if (par >= 0) {
            atomicAdd(&a.childsum[par], b + a.u_pair);
            atomicAdd(&a.fdsum[par], fd + a.u_pair);
        }
    }
}

__global__ void k_root_totals(const DpArgs a, int64_t n0, double *tot) {
    double b = 0.0, f = 0.0;
    for (int64_t g = threadIdx.x; g < n0; g += blockDim.x) {
        b += a.best[g] + a.u_pair;
        const int kind = a.pc[4 * g + 3];
        const double nq = (double)a.nq[g], nr = (double)a.nr[g];
        f += (kind == LOG_BASE ? nq * nr * a.u_base : (kind == LOG_SPLIT ? a.fdsum[g] : 0.0)) + a.u_pair;
    }
    atomicAdd(&tot[0], b);
    atomicAdd(&tot[1], f);
}

__global__ void k_sample_flags(const int8_t *label, const double *regret, int64_t n, long long *flag,
                               double *regret_sum) {
    double acc = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        flag[g] = label[g] >= 0;
        if (label[g] >= 0) acc += regret[g];
    }
    if (acc != 0.0) atomicAdd(regret_sum, acc);
}

// weight of a sample: its regret (second cheapest minus cheapest certified
// action) over the problem's mean regret, so that decisions that cost more
// when taken wrongly count more
__global__ void k_sample_scatter(const int8_t *label, const float *feat, const double *regret, const long long *off,
                                 int64_t n, const double *regret_sum, float *x, int32_t *y, float *s) {
    const long long ns = off[n];
    const double mean = ns > 0 ? *regret_sum / (double)ns : 1.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        if (label[g] < 0) continue;
        const int64_t o = off[g];
        for (int k = 0; k < kMlpIn; ++k) x[o * kMlpIn + k] = feat[g * kMlpIn + k];
        y[o] = label[g];
        if (s) s[o] = mean > 0.0 ? (float)(regret[g] / mean) : 1.f;
    }
}

static void free_log(PairLog &lg, cudaStream_t st) {
    void *ptrs[] = {lg.feat, lg.pc, lg.nq, lg.nr, lg.par, lg.pid[0], lg.pid[1]};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, st);
    lg = PairLog();
}

}  // namespace gs

using namespace gs;

extern "C" int gs_selector_samples(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                                   int D, int dtype, const double *h, int nh, double eps, const gs_opts *opts,
                                   const double *unit_cost, float *x, int32_t *y, float *s, int64_t cap,
                                   int64_t *n_samples, double *model_cost, void *stream) {
    if (!unit_cost || !n_samples || !(eps > 0.0) || cap < 0 || (cap > 0 && (!x || !y))) {
        set_error("gs_selector_samples: bad arguments (unit_cost, n_samples, eps > 0, x / y)");
        return GS_ERR_ARG;
    }
    for (int k = 0; k < 6; ++k)
        if (!(unit_cost[k] >= 0.0) || !isfinite(unit_cost[k])) {
            set_error("gs_selector_samples: unit_cost[%d] must be finite and >= 0", k);
            return GS_ERR_ARG;
        }
    *n_samples = 0;
    cudaStream_t st = (cudaStream_t)stream;
    gs_opts o;
    gs_opts_default(&o);
    if (opts) o = *opts;
    o.selector = GS_SEL_FD_ONLY;
    double *out = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&out, (size_t)(M > 0 ? M : 1) * nh * sizeof(double), st));
    PairLog lg;
    int rc = sum_impl(queries, M, refs, weights, N, D, dtype, h, nh, eps, out, &o, stream, nullptr, nullptr, &lg);
    cudaFreeAsync(out, st);
    if (rc) {
        free_log(lg, st);
        return rc;
    }
    const int64_t total = lg.iter_off[lg.niter];
    DpArgs a;
    memset(&a, 0, sizeof(a));
    a.pc = lg.pc; a.nq = lg.nq; a.nr = lg.nr; a.par = lg.par;
    a.u_pair = unit_cost[0]; a.u_base = unit_cost[1]; a.u_dh = unit_cost[2]; a.u_dl = unit_cost[3];
    a.u_h2l = unit_cost[4]; a.u_act = unit_cost[5];
    a.D = D;
    for (int p = 1; p <= 16; ++p) {
        double c = 1.0;   // C(D+p-1, D)
        for (int i = 1; i <= D; ++i) c = c * (double)(p - 1 + i) / (double)i;
        a.Tp[p] = c;
    }
    double *dbuf = nullptr, *tot = nullptr;
    int8_t *label = nullptr;
    long long *flag = nullptr;
    CallCtx cx;
    cx.st = st;
    cudaError_t e = dev_malloc_async((void **)&dbuf, (size_t)(4 * total + 3) * sizeof(double), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&label, (size_t)(total + 1), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&flag, (size_t)(total + 1) * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbuf, 0, (size_t)(4 * total + 3) * sizeof(double), st);
    if (e != cudaSuccess) rc = cuda_fail(e, "gs_selector_samples scratch");
    if (!rc) {
        a.childsum = dbuf;
        a.fdsum = dbuf + total;
        a.best = dbuf + 2 * total;
        a.regret = dbuf + 3 * total;
        a.label = label;
        tot = dbuf + 4 * total;   // [0] cheapest policy, [1] FD-only policy, [2] regret sum
        for (int t = lg.niter - 1; t >= 0; --t) {
            const int64_t g0 = lg.iter_off[t], g1 = lg.iter_off[t + 1];
            if (g1 <= g0) continue;
            const int64_t blocks = (g1 - g0 + 255) / 256;
            k_dp_iter<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(a, g0, g1);
        }
        k_root_totals<<<1, 256, 0, st>>>(a, lg.iter_off[1], tot);
        const int64_t blocks = (total + 255) / 256;
        const unsigned grid = (unsigned)(blocks < 8192 ? (blocks > 0 ? blocks : 1) : 8192);
        k_sample_flags<<<grid, 256, 0, st>>>(label, a.regret, total, flag, tot + 2);
        rc = scan_i64(flag, total, flag + total, cx);
    }
    long long nsamp = 0;
    double htot[2] = {0.0, 0.0};
    if (!rc) {
        e = cudaMemcpyAsync(&nsamp, flag + total, sizeof(nsamp), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(htot, tot, sizeof(htot), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "gs_selector_samples");
    }
    if (!rc) {
        *n_samples = nsamp;
        if (model_cost) {
            model_cost[0] = htot[0];
            model_cost[1] = htot[1];
        }
        if (nsamp > cap) {
            set_error("gs_selector_samples: %lld samples exceed the capacity %lld", nsamp, (long long)cap);
            rc = GS_ERR_CAPACITY;
        } else if (nsamp > 0) {
            const int64_t blocks = (total + 255) / 256;
            k_sample_scatter<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, st>>>(
                label, lg.feat, a.regret, flag, total, tot + 2, x, y, s);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "sample scatter");
        }
    }
    if (dbuf) cudaFreeAsync(dbuf, st);
    if (label) cudaFreeAsync(label, st);
    if (flag) cudaFreeAsync(flag, st);
    free_log(lg, st);
    cudaStreamSynchronize(st);
    return rc;
}
