// C-ABI entry points: argument checks, scratch management, dispatch to the
// exhaustive or dual-tree path, and the single end-of-call status read.
#include <math.h>

#include <atomic>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gs_internal.h"

namespace gs {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static std::atomic<long long> g_fail_countdown{-1};

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    long long c = g_fail_countdown.load();
    while (c >= 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = scratch_pool(&pool);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// The library's own stream-ordered pool, one per device.  The device's
// default pool returns freed memory to the CUDA driver at every synchronisation,
// so a traversal that synchronises once per frontier iteration would map
// its lists afresh each time; this pool keeps freed memory until
// gs_trim_memory releases it.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

cudaError_t scratch_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

bool CallCtx::debug_sync_enabled() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("GS_DEBUG_SYNC");
        v = (e && e[0] && e[0] != '0') ? 1 : 0;
    }
    return v == 1;
}

int CallCtx::check(const char *what) {
    if (!debug) return GS_OK;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return GS_OK;
}

int check_common(const void *queries, int64_t M, const void *refs, const float *weights,
                        int64_t N, int D, int dtype, const double *h, int nh, double eps,
                        double *out) {
    if (!queries || !refs || !weights || !out || !h) {
        set_error("NULL array argument");
        return GS_ERR_ARG;
    }
    if (M < 1 || N < 1) {
        set_error("M=%lld and N=%lld must be >= 1", (long long)M, (long long)N);
        return GS_ERR_ARG;
    }
    if (D < 1 || D > 32) {
        set_error("D=%d outside [1, 32]", D);
        return GS_ERR_ARG;
    }
    if (dtype != GS_F32 && dtype != GS_F64) {
        set_error("dtype %d is neither GS_F32 nor GS_F64", dtype);
        return GS_ERR_ARG;
    }
    if (nh < 1 || nh > 64) {
        set_error("nh=%d outside [1, 64]", nh);
        return GS_ERR_ARG;
    }
    for (int j = 0; j < nh; ++j)
        if (!(h[j] > 0.0) || !isfinite(h[j])) {
            set_error("bandwidth h[%d]=%g is not finite and positive", j, h[j]);
            return GS_ERR_ARG;
        }
    if (!(eps >= 0.0 && eps < 1.0)) {
        set_error("eps=%g outside [0, 1)", eps);
        return GS_ERR_ARG;
    }
    return GS_OK;
}

int status_to_code(unsigned st) {
    if (st & ST_NONFINITE) {
        set_error("non-finite coordinate or weight");
        return GS_ERR_NONFINITE;
    }
    if (st & ST_WEIGHT) {
        set_error("a weight is <= 0 (weights must be positive)");
        return GS_ERR_WEIGHT;
    }
    if (st & ST_CAPACITY) {
        set_error("a device work list exceeded its capacity");
        return GS_ERR_CAPACITY;
    }
    if (st & ST_TIMEOUT) {
        set_error("a bounded device wait gave up");
        return GS_ERR_TIMEOUT;
    }
    if (st & ST_EPS) {
        set_error("eps is too small: the FP32 base-case error bound takes more than half of it");
        return GS_ERR_ARG;
    }
    if (st & ST_INTERNAL) {
        set_error("internal consistency check failed on the device");
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

// LSCV partial sums per bandwidth j (one pass over the points per j, sums
// in registers, then the warp and the block, one atomic per block):
//   acc[3j]   += wbar_i G_{sqrt2 h}(x_i)
//   acc[3j+1] += wbar_i (G_h(x_i) - w_i) / (W - w_i)
//   acc[3j+2] += wbar_i G_h(x_i) / (W - w_i)
__global__ void __launch_bounds__(256) k_lscv_sums(const double *__restrict__ G, const float *__restrict__ w,
                                                   int64_t N, int nh, const Ingest *__restrict__ ing, double *acc) {
    __shared__ double sh[3][8];
    const double W = ing->wsum;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int j = 0; j < nh; ++j) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double wi = (double)w[i], wb = wi / W, den = W - wi;
            const double gh = G[i * 2 * nh + j], g2 = G[i * 2 * nh + nh + j];
            a0 += wb * g2;
            a1 += wb * (gh - wi) / den;
            a2 += wb * gh / den;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            sh[0][wp] = a0;
            sh[1][wp] = a1;
            sh[2][wp] = a2;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[threadIdx.x][k];
            atomicAdd(&acc[3 * j + threadIdx.x], s);
        }
        __syncthreads();
    }
}

// LSCV scores from the sums G (caller order, N x 2nh: h then sqrt(2) h) and
// the weight total in *ing (device), on the host at the end:
//   score = (4 pi h^2)^{-D/2} sum_i wbar_i G_{sqrt2 h}(x_i) / W
//         - 2 (2 pi h^2)^{-D/2} sum_i wbar_i (G_h(x_i) - w_i) / (W - w_i)
// and the bound eps implies on it: every G is within a relative eps of its
// exact value, so the first term moves by at most eps times itself and the
// leave-one-out term by at most 2 eps (2 pi h^2)^{-D/2} sum_i wbar_i G_h(x_i)
// / (W - w_i).
int lscv_scores(const double *G, const float *weights, int64_t N, int D, const double *h, int nh, double eps,
                const Ingest *ing, double *score, double *score_err, cudaStream_t st) {
    double *acc = nullptr;
    cudaError_t e = dev_malloc_async((void **)&acc, 3 * 32 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 3 * 32 * sizeof(double), st);
    if (e == cudaSuccess) {
        int64_t blocks = (N + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        k_lscv_sums<<<(unsigned)blocks, 256, 0, st>>>(G, weights, N, nh, ing, acc);
        e = cudaGetLastError();
    }
    double hacc[3 * 32];
    Ingest hing;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hing, ing, sizeof(hing), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (acc) cudaFreeAsync(acc, st);
    if (e != cudaSuccess) return cuda_fail(e, "lscv scores");
    const double W = hing.wsum;
    const double pi = 3.141592653589793;
    for (int j = 0; j < nh; ++j) {
        const double c2 = pow(4.0 * pi * h[j] * h[j], -0.5 * D);
        const double c1 = pow(2.0 * pi * h[j] * h[j], -0.5 * D);
        score[j] = c2 * hacc[3 * j] / W - 2.0 * c1 * hacc[3 * j + 1];
        if (score_err) score_err[j] = eps * (c2 * hacc[3 * j] / W + 2.0 * c1 * hacc[3 * j + 2]);
    }
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" {

const char *gs_version(void) { return "gbsum 0.1 (sm_103a)"; }

const char *gs_last_error(void) { return g_err; }

int gs_opts_default(gs_opts *o) {
    if (!o) {
        set_error("gs_opts_default: NULL");
        return GS_ERR_ARG;
    }
    memset(o, 0, sizeof(*o));
    o->leaf_size = 32;
    o->floor_log2 = -40;
    o->selector = GS_SEL_RULE;
    o->cost_weight[0] = GS_COST_DH;
    o->cost_weight[1] = GS_COST_DL;
    o->cost_weight[2] = GS_COST_H2L;
    o->cost_weight[3] = GS_COST_DIRECT;
    return GS_OK;
}

}  // extern "C"

int gs::sum_impl(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N, int D,
                 int dtype, const double *h, int nh, double eps, double *out, const gs_opts *opts, void *stream,
                 gs_stats *stats, TraceOut *trace, PairLog *log) {
    g_err[0] = 0;
    int rc = check_common(queries, M, refs, weights, N, D, dtype, h, nh, eps, out);
    if (rc) return rc;
    gs_opts o;
    gs_opts_default(&o);
    if (opts) {
        o = *opts;
        if (o.leaf_size == 0) o.leaf_size = 32;
        if (o.floor_log2 == 0) o.floor_log2 = -40;
        if (o.cost_weight[0] == 0 && o.cost_weight[1] == 0 && o.cost_weight[2] == 0 && o.cost_weight[3] == 0) {
            o.cost_weight[0] = GS_COST_DH;
            o.cost_weight[1] = GS_COST_DL;
            o.cost_weight[2] = GS_COST_H2L;
            o.cost_weight[3] = GS_COST_DIRECT;
        }
    }
    for (int k = 0; k < 4; ++k)
        if (!(o.cost_weight[k] > 0.0) || !isfinite(o.cost_weight[k])) {
            set_error("cost_weight[%d]=%g must be finite and positive", k, o.cost_weight[k]);
            return GS_ERR_ARG;
        }
    if (o.selector < GS_SEL_RULE || o.selector > GS_SEL_EXHAUSTIVE) {
        set_error("unknown selector %d", o.selector);
        return GS_ERR_ARG;
    }
    if (o.selector == GS_SEL_MLP && !o.selector_params) {
        set_error("GS_SEL_MLP needs gs_opts.selector_params (the trained network)");
        return GS_ERR_ARG;
    }
    if (o.floor_log2 < -1000 || o.floor_log2 > -1) {
        set_error("floor_log2=%d outside [-1000, -1]", o.floor_log2);
        return GS_ERR_ARG;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t st = (cudaStream_t)stream;
    const double small_work = o.small_work > 0.0 ? o.small_work : (D <= 2 ? GS_SMALL_WORK_D2 : GS_SMALL_WORK);
    const bool exhaustive = eps == 0.0 || ((o.flags & GS_FLAG_SMALL_EXHAUSTIVE) && !trace && !log &&
                                           (double)M * (double)N * (double)nh <= small_work);

    CallCtx cx;
    cx.st = st;
    cx.stats = stats;
    cx.phase(GS_PH_INGEST);
    Ingest *ing = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&ing, sizeof(Ingest), st));
    cudaError_t e = launch_ingest(ing, queries, M, refs, weights, N, D, dtype, cx);
    if (e != cudaSuccess) {
        cudaFreeAsync(ing, st);
        return cuda_fail(e, "ingest launch");
    }
    unsigned status = 0;
    if (exhaustive) {
        rc = exhaustive_sum(queries, M, refs, weights, N, D, dtype, h, nh, ing, out, cx);
        Ingest hing;
        if (rc == GS_OK) {
            e = cudaMemcpyAsync(&hing, ing, sizeof(Ingest), cudaMemcpyDeviceToHost, st);
            cx.end();
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "gs_sum");
            status = hing.status;
        }
        if (rc == GS_OK && stats) stats->point_pairs_base = M * N * nh;
    } else {
        rc = dualtree_sum(queries, M, refs, weights, N, D, dtype, h, nh, eps, out, o, cx, ing, trace, &status, log);
    }
    cudaFreeAsync(ing, st);
    if (rc == GS_OK) rc = status_to_code(status);
    if (rc == GS_OK && stats) cx.finish();
    return rc;
}

extern "C" {

int gs_sum(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
           int D, int dtype, const double *h, int nh, double eps, double *out,
           const gs_opts *opts, void *stream, gs_stats *stats) {
    return sum_impl(queries, M, refs, weights, N, D, dtype, h, nh, eps, out, opts, stream, stats, nullptr);
}

int gs_sum_trace(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                 int D, int dtype, const double *h, int nh, double eps, double *out,
                 const gs_opts *opts, void *stream, gs_stats *stats, int32_t *trace, int64_t trace_cap,
                 int64_t *trace_len, int32_t *qperm, int32_t *rperm) {
    if (eps == 0.0) {
        set_error("gs_sum_trace needs eps > 0 (the exhaustive path has no traversal)");
        return GS_ERR_ARG;
    }
    TraceOut t;
    t.trace = trace;
    t.cap = trace ? trace_cap : 0;
    t.len = trace_len;
    t.qperm = qperm;
    t.rperm = rperm;
    if (trace_len) *trace_len = 0;
    return sum_impl(queries, M, refs, weights, N, D, dtype, h, nh, eps, out, opts, stream, stats, &t);
}

int gs_lscv(const void *pts, int64_t N, int D, int dtype, const float *weights, const double *h, int nh,
            double eps, double *score, double *score_err, const gs_opts *opts, void *stream, gs_stats *stats) {
    g_err[0] = 0;
    if (!score) {
        set_error("gs_lscv: NULL score");
        return GS_ERR_ARG;
    }
    if (N < 2) {
        set_error("gs_lscv needs N >= 2");
        return GS_ERR_ARG;
    }
    if (nh < 1 || nh > 32 || !h) {
        set_error("gs_lscv: nh=%d outside [1, 32]", nh);
        return GS_ERR_ARG;
    }
    double hh[64];
    for (int j = 0; j < nh; ++j) {
        hh[j] = h[j];
        hh[nh + j] = h[j] * 1.4142135623730951;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *G = nullptr;
    Ingest *ing = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&G, (size_t)N * 2 * nh * sizeof(double), st));
    int rc = sum_impl(pts, N, pts, weights, N, D, dtype, hh, 2 * nh, eps, G, opts, stream, stats, nullptr);
    if (rc == GS_OK) {
        // total weight (the library's own ingest reduction), then the scores
        cudaError_t e = dev_malloc_async((void **)&ing, sizeof(Ingest), st);
        CallCtx cx;
        cx.st = st;
        if (e == cudaSuccess) e = launch_ingest(ing, pts, N, pts, weights, N, D, dtype, cx);
        rc = e == cudaSuccess ? lscv_scores(G, weights, N, D, h, nh, eps, ing, score, score_err, st)
                              : cuda_fail(e, "gs_lscv");
    }
    cudaFreeAsync(G, st);
    if (ing) cudaFreeAsync(ing, st);
    return rc;
}

int gs_sum_host(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                int D, int dtype, const double *h, int nh, double eps, double *out,
                const gs_opts *opts, void *stream, gs_stats *stats) {
    g_err[0] = 0;
    int rc = check_common(queries, M, refs, weights, N, D, dtype, h, nh, eps, out);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dtype == GS_F64 ? sizeof(double) : sizeof(float);
    const bool mono = queries == refs;
    void *dq = nullptr, *dr = nullptr;
    float *dw = nullptr;
    double *dout = nullptr;
    cudaError_t e = dev_malloc_async(&dr, (size_t)N * D * es, st);
    if (e == cudaSuccess && !mono) e = dev_malloc_async(&dq, (size_t)M * D * es, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dw, (size_t)N * sizeof(float), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dout, (size_t)M * nh * sizeof(double), st);
    if (e == cudaSuccess) {
        if (mono) dq = dr;
        e = cudaMemcpyAsync(dr, refs, (size_t)N * D * es, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !mono)
            e = cudaMemcpyAsync(dq, queries, (size_t)M * D * es, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dw, weights, (size_t)N * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "gs_sum_host upload");
        } else {
            rc = gs_sum(dq, M, dr, dw, N, D, dtype, h, nh, eps, dout, opts, stream, stats);
            if (rc == GS_OK) {
                e = cudaMemcpyAsync(out, dout, (size_t)M * nh * sizeof(double), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) rc = cuda_fail(e, "gs_sum_host download");
            }
        }
    } else {
        rc = cuda_fail(e, "gs_sum_host scratch");
    }
    if (dr) cudaFreeAsync(dr, st);
    if (!mono && dq) cudaFreeAsync(dq, st);
    if (dw) cudaFreeAsync(dw, st);
    if (dout) cudaFreeAsync(dout, st);
    return rc;
}

int gs_lscv_host(const void *pts, int64_t N, int D, int dtype, const float *weights, const double *h, int nh,
                 double eps, double *score, double *score_err, const gs_opts *opts, void *stream,
                 gs_stats *stats) {
    g_err[0] = 0;
    if (!pts || !weights) {
        set_error("gs_lscv_host: NULL array argument");
        return GS_ERR_ARG;
    }
    if (N < 2 || D < 1 || D > 32 || (dtype != GS_F32 && dtype != GS_F64)) {
        set_error("gs_lscv_host: bad N, D or dtype");
        return GS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = dtype == GS_F64 ? sizeof(double) : sizeof(float);
    void *dp = nullptr;
    float *dw = nullptr;
    int rc = GS_OK;
    cudaError_t e = dev_malloc_async(&dp, (size_t)N * D * es, st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dw, (size_t)N * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, pts, (size_t)N * D * es, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, weights, (size_t)N * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        rc = cuda_fail(e, "gs_lscv_host upload");
    else
        rc = gs_lscv(dp, N, D, dtype, dw, h, nh, eps, score, score_err, opts, stream, stats);
    if (dp) cudaFreeAsync(dp, st);
    if (dw) cudaFreeAsync(dw, st);
    return rc;
}

void gs_debug_fail_alloc(long long n) { g_fail_countdown.store(n < 0 ? -1 : n); }

int gs_trim_memory(size_t keep_bytes) {
    g_err[0] = 0;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(&pool);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, keep_bytes);
    return e == cudaSuccess ? GS_OK : cuda_fail(e, "gs_trim_memory");
}

int gs_pool_bytes(uint64_t *reserved, uint64_t *used) {
    g_err[0] = 0;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(&pool);
    uint64_t r = 0, u = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e != cudaSuccess) return cuda_fail(e, "gs_pool_bytes");
    if (reserved) *reserved = r;
    if (used) *used = u;
    return GS_OK;
}

int gs_probe_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, void *stream) {
    g_err[0] = 0;
    if (!ex2_per_sm_clk || !ffma_per_sm_clk) {
        set_error("gs_probe_rates: NULL output");
        return GS_ERR_ARG;
    }
    return probe_rates(ex2_per_sm_clk, ffma_per_sm_clk, (cudaStream_t)stream);
}

}  // extern "C"
