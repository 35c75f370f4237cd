// Dual-tree Gaussian summation driver (Sections 5-6): trees, moments,
// frontier iterations, base case, series actions and the downward pass, all
// enqueued on one stream with no host synchronisation until the single status
// read at the end.  If a device work list outgrew its capacity the traversal
// is re-run with four times the capacity (the trees are kept).
#include <math.h>
#include <string.h>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

int dp_for(int D) {
    static const int dps[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 24, 32};
    for (int v : dps)
        if (D <= v) return v;
    return 32;
}

int plimit_for(int D) {
    // Section 6: PLIMIT = 8 (D=2), 6 (D=3), 4 (D=5), 2 (D=6), 1 (D>6);
    // D=4 is not stated (5 is used), D=1 uses 8.
    switch (D) {
        case 1: return 8;
        case 2: return 8;
        case 3: return 6;
        case 4: return 5;
        case 5: return 4;
        case 6: return 2;
        default: return 1;
    }
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static void free_bufs(FrontierBufs &fb, cudaStream_t st) {
    // inv_4h2, inv_h and inv_s live inside the inv_2h2 allocation
    void *ptrs[] = {fb.fs, fb.groups[0], fb.groups[1], fb.pr[0], fb.pr[1], fb.dec, fb.geo, fb.cnt, fb.off,
                    fb.partial, fb.base_groups, fb.base_r, fb.series[0], fb.series[1], fb.series[2], fb.fin,
                    fb.tok, fb.est, fb.inv_2h2, fb.evals};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, st);
    FrontierBufs keep;
    keep.trace = fb.trace;
    keep.trace_cap = fb.trace_cap;
    keep.grid_warps = fb.grid_warps;
    keep.host_totals = fb.host_totals;
    fb = keep;
}

#define GS_ALLOC(ptr, bytes) GS_CUDA_TRY(dev_malloc_async((void **)&(ptr), (size_t)(bytes), st))

// pinned host scratch for the per-iteration totals (one per host thread)
static int64_t *host_scratch() {
    static thread_local int64_t *p = nullptr;
    if (!p && cudaMallocHost((void **)&p, 64 * sizeof(int64_t)) != cudaSuccess) p = nullptr;
    return p;
}

static int alloc_bufs(FrontierBufs &fb, int64_t nodesQ, int nh, const double *h, int64_t initial, cudaStream_t st) {
    fb.host_totals = host_scratch();
    if (!fb.host_totals) {
        set_error("pinned host allocation failed");
        return GS_ERR_OOM;
    }
    GS_ALLOC(fb.fs, sizeof(FrontierState));
    GS_CUDA_TRY(cudaMemsetAsync(fb.fs, 0, sizeof(FrontierState), st));
    for (int b = 0; b < 2; ++b) {
        GS_ALLOC(fb.groups[b], fb.cap_groups * sizeof(Group));
        fb.cap_pr[b] = initial;
        GS_ALLOC(fb.pr[b], initial * sizeof(int32_t));
    }
    fb.cap_pairs = initial;
    GS_ALLOC(fb.dec, initial);
    fb.cap_geo = 4 * initial;
    GS_ALLOC(fb.geo, 4 * initial * sizeof(float));
    GS_ALLOC(fb.cnt, fb.cap_groups * kCols * sizeof(int32_t));
    GS_ALLOC(fb.off, fb.cap_groups * kCols * sizeof(long long));
    GS_ALLOC(fb.partial, kCols * 256 * sizeof(long long));
    GS_ALLOC(fb.base_groups, fb.cap_base_groups * sizeof(Group));
    fb.cap_base = initial;
    GS_ALLOC(fb.base_r, initial * sizeof(int32_t));
    for (int m = 0; m < 3; ++m) {
        fb.cap_series[m] = initial / 4 > 1024 ? initial / 4 : 1024;
        GS_ALLOC(fb.series[m], fb.cap_series[m] * sizeof(SeriesEntry));
    }
    const size_t ns = (size_t)nodesQ * nh * sizeof(double);
    GS_ALLOC(fb.fin, ns);
    GS_ALLOC(fb.tok, ns);
    GS_ALLOC(fb.est, ns);
    GS_CUDA_TRY(cudaMemsetAsync(fb.fin, 0, ns, st));
    GS_CUDA_TRY(cudaMemsetAsync(fb.tok, 0, ns, st));
    GS_CUDA_TRY(cudaMemsetAsync(fb.est, 0, ns, st));
    GS_ALLOC(fb.inv_2h2, 4 * 64 * sizeof(double));
    fb.inv_4h2 = fb.inv_2h2 + 64;
    fb.inv_h = fb.inv_2h2 + 128;
    fb.inv_s = fb.inv_2h2 + 192;
    double hc[4 * 64];
    memset(hc, 0, sizeof(hc));
    for (int j = 0; j < nh; ++j) {
        hc[j] = 1.0 / ((2.0 * h[j]) * h[j]);
        hc[64 + j] = 1.0 / ((4.0 * h[j]) * h[j]);
        hc[128 + j] = 1.0 / h[j];
        hc[192 + j] = 1.0 / sqrt(2.0 * h[j] * h[j]);
    }
    // pageable source: the runtime stages hc before returning, so it may go out of scope
    GS_CUDA_TRY(cudaMemcpyAsync(fb.inv_2h2, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    // evals[0]: every base-case term; evals[1]: those of the tensor-core kernel
    GS_ALLOC(fb.evals, 2 * sizeof(unsigned long long));
    GS_CUDA_TRY(cudaMemsetAsync(fb.evals, 0, 2 * sizeof(unsigned long long), st));
    return GS_OK;
}

int dualtree_sum(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N, int D,
                 int dtype, const double *h, int nh, double eps, double *out, const gs_opts &o, CallCtx &cx,
                 Ingest *ing, TraceOut *trace, unsigned *status_out, PairLog *log) {
    cudaStream_t st = cx.st;
    const int L = o.leaf_size;
    if (L < 2 || L > 128) {
        set_error("leaf_size=%d outside [2, 128]", L);
        return GS_ERR_ARG;
    }
    const bool mono = queries == refs && M == N;
    const int DP = dp_for(D);
    const int stride = record_stride(D);
    int rc;
    TreeDev rt, qt;
    cx.phase(GS_PH_TREE);
    rc = build_tree(refs, weights, N, D, dtype, L, ing, DP, stride, true, cx, &rt);
    if (rc) return rc;
    if (mono) {
        qt = rt;
    } else {
        rc = build_tree(queries, nullptr, M, D, dtype, L, ing, DP, stride, false, cx, &qt);
        if (rc) {
            free_tree(rt, st);
            return rc;
        }
    }
    rc = dualtree_run(qt, rt, mono, weights, D, h, nh, eps, out, o, cx, ing, trace, status_out, log);
    free_tree(rt, st);
    if (!mono) free_tree(qt, st);
    return rc;
}

int dualtree_run(const TreeDev &qt_in, const TreeDev &rt_in, bool mono, const float *weights, int D,
                 const double *h, int nh, double eps, double *out, const gs_opts &o, CallCtx &cx, Ingest *ing,
                 TraceOut *trace, unsigned *status_out, PairLog *log) {
    cudaStream_t st = cx.st;
    const int DP = dp_for(D);
    int rc = GS_OK;
    // shallow copies: this call's moments live in rt and are freed here
    TreeDev rt = rt_in;
    TreeDev qt = mono ? rt_in : qt_in;
    rt.moments = nullptr;
    rt.mom_terms = 0;
    int P = o.plimit > 0 ? o.plimit : plimit_for(D);
    if (P > 16) P = 16;
    const bool series = (o.selector == GS_SEL_RULE || o.selector == GS_SEL_MLP) && P >= 1;
    SeriesTables tb;
    if (series) {
        if (D * (2 * P - 1) > 128 || D * P > 64) {
            set_error("series order P=%d too high for D=%d (needs D*(2P-1) <= 128 and D*P <= 64)", P, D);
            rc = GS_ERR_ARG;
        }
        if (!rc) rc = build_series_tables(D, P, &tb, st);
        if (!rc && tb.T > 1024) {
            set_error("series order P=%d in D=%d needs %d terms (limit 1024)", P, D, tb.T);
            rc = GS_ERR_ARG;
        }
        if (!rc) rc = build_moments(rt, weights, tb, cx);
        if (rc) {
            free_series_tables(&tb, st);
            if (rt.moments) cudaFreeAsync(rt.moments, st);
            return rc;
        }
    }
    TraversalIn in;
    in.qt = &qt;
    in.rt = &rt;
    in.ing = ing;
    in.weights = weights;
    in.h = h;
    in.D = D;
    in.nh = nh;
    in.P = P;
    in.selector = o.selector;
    in.tokens = o.no_tokens ? 0 : 1;
    in.mono = mono;
    in.floor_log2 = o.floor_log2;
    in.eps = eps;

    for (int k = 0; k < 4; ++k) in.cost_w[k] = o.cost_weight[k];
    in.flags = o.flags;
    in.mlp = o.selector_params;
    in.log = log;
    const int64_t lq = 1ll << qt.depth;
    FrontierBufs fb;
    fb.grid_warps = sm_count() * 64;
    if (trace && trace->trace) {
        fb.trace = (int4 *)trace->trace;
        fb.trace_cap = trace->cap;
    }
    double *Gq = nullptr, *B = nullptr;
    int32_t *pL = nullptr;
    FrontierState hfs;
    Ingest hing;
    fb.cap_groups = (int64_t)nh * lq;
    fb.cap_base_groups = (int64_t)nh * lq;
    const int64_t initial = o.pair_capacity > 0 ? o.pair_capacity : ((int64_t)16 * nh * lq > (1 << 16) ? (int64_t)16 * nh * lq : (1 << 16));
    rc = alloc_bufs(fb, qt.nodes, nh, h, initial, st);
    if (!rc) {
        cx.phase(GS_PH_FRONTIER);
        rc = run_frontier(in, fb, cx);
    }
    if (!rc) {
        // outputs of the base case and the series (freed below whatever happens)
        rc = [&]() -> int {
            GS_ALLOC(Gq, (size_t)qt.n * nh * sizeof(double));
            GS_CUDA_TRY(cudaMemsetAsync(Gq, 0, (size_t)qt.n * nh * sizeof(double), st));
            if (series) {
                GS_ALLOC(B, (size_t)qt.nodes * nh * tb.T * sizeof(double));
                GS_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)qt.nodes * nh * tb.T * sizeof(double), st));
                GS_ALLOC(pL, (size_t)qt.nodes * nh * sizeof(int32_t));
                GS_CUDA_TRY(cudaMemsetAsync(pL, 0, (size_t)qt.nodes * nh * sizeof(int32_t), st));
            }
            return GS_OK;
        }();
        if (!rc)
            rc = (merged_base_possible(in) && !(o.flags & GS_FLAG_NO_MERGE)) ? run_basecase_merged(in, fb, Gq, DP, cx)
                                                                             : run_basecase(in, fb, Gq, DP, cx);
    }
    if (!rc) rc = run_series_and_final(in, fb, series ? &tb : nullptr, Gq, B, pL, out, cx);
    if (!rc && trace && trace->qperm) {
        cudaError_t e = cudaMemcpyAsync(trace->qperm, qt.perm, qt.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "trace query permutation");
    }
    if (!rc && trace && trace->rperm) {
        cudaError_t e = cudaMemcpyAsync(trace->rperm, rt.perm, rt.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "trace reference permutation");
    }
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&hfs, fb.fs, sizeof(hfs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hing, ing, sizeof(hing), cudaMemcpyDeviceToHost, st);
        unsigned long long hev2[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(hev2, fb.evals, sizeof(hev2), cudaMemcpyDeviceToHost, st);
        const unsigned long long hev = hev2[0];
        cx.end();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "dual-tree");
        if (!rc && cx.stats) {
            gs_stats *s = cx.stats;
            s->pairs_fd = (int64_t)hfs.method_count[M_FD];
            s->pairs_dh = (int64_t)hfs.method_count[M_DH];
            s->pairs_dl = (int64_t)hfs.method_count[M_DL];
            s->pairs_h2l = (int64_t)hfs.method_count[M_H2L];
            s->pairs_base = (int64_t)hfs.method_count[M_BASE];
            s->pairs_split = (int64_t)hfs.method_count[M_SPLIT];
            s->point_pairs_base = (int64_t)hev;
            s->point_pairs_tc = (int64_t)hev2[1];
            s->levels = (qt.depth > rt.depth ? qt.depth : rt.depth) + 1;
            s->retries = 0;
            s->fp32_rel_bound = hfs.rho;
            s->eps_traversal = hfs.eps_t;
        }
        if (!rc && trace && trace->len) *trace->len = hfs.trace_count;
    }
    if (Gq) cudaFreeAsync(Gq, st);
    if (B) cudaFreeAsync(B, st);
    if (pL) cudaFreeAsync(pL, st);
    free_bufs(fb, st);
    if (series) free_series_tables(&tb, st);
    if (rt.moments) cudaFreeAsync(rt.moments, st);
    if (rc) return rc;
    *status_out = hing.status;
    return GS_OK;
}

}  // namespace gs
