// Built trees that outlive a call: gs_build_tree, gs_sum_trees, gs_tree_free.
//
// A handle keeps the kd-tree of one point set (Section 5's node boxes,
// weights and packed records, built once) so that several sums over the
// same data -- other bandwidths, other eps, other query sets -- skip the
// build.  A reference tree also keeps a copy of the weights and the summary
// of its inputs (largest weight, checks), which every later sum needs.
#include <string.h>

#include "gs_internal.h"

using namespace gs;

struct gs_tree {
    int device = 0;
    TreeDev t;
    Ingest *ing = nullptr;    // device: input checks and weight range of this point set
    float *w = nullptr;       // device copy of the weights in caller order (reference trees)
    int leaf = 32;
};

static void destroy(gs_tree *h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_tree(h->t, nullptr);
    if (h->ing) cudaFree(h->ing);
    if (h->w) cudaFree(h->w);
    cudaDeviceSynchronize();
    cudaSetDevice(cur);
    delete h;
}

extern "C" int gs_build_tree(const void *pts, int dtype, int64_t n, int D, const float *weights,
                             const gs_opts *opts, void *stream, gs_tree **out) {
    if (!out) {
        set_error("gs_build_tree: NULL out");
        return GS_ERR_ARG;
    }
    *out = nullptr;
    if (!pts || n < 1 || D < 1 || D > 32 || (dtype != GS_F32 && dtype != GS_F64)) {
        set_error("gs_build_tree: bad points (n=%lld, D=%d, dtype=%d)", (long long)n, D, dtype);
        return GS_ERR_ARG;
    }
    const int L = opts && opts->leaf_size ? opts->leaf_size : 32;
    if (L < 2 || L > 128) {
        set_error("leaf_size=%d outside [2, 128]", L);
        return GS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gs_tree *h = new gs_tree();
    cudaGetDevice(&h->device);
    h->leaf = L;
    CallCtx cx;
    cx.st = st;
    int rc = GS_OK;
    cudaError_t e = dev_malloc_async((void **)&h->ing, sizeof(Ingest), st);
    if (e == cudaSuccess && weights) {
        e = dev_malloc_async((void **)&h->w, (size_t)n * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->w, weights, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = launch_ingest(h->ing, pts, n, pts, weights, n, D, dtype, cx);
    if (e != cudaSuccess) rc = cuda_fail(e, "gs_build_tree");
    if (!rc) rc = build_tree(pts, weights, n, D, dtype, L, h->ing, dp_for(D), record_stride(D), weights != nullptr,
                             cx, &h->t);
    Ingest hing;
    if (!rc) {
        e = cudaMemcpyAsync(&hing, h->ing, sizeof(Ingest), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "gs_build_tree");
    }
    if (!rc && (hing.status & ST_NONFINITE)) {
        set_error("non-finite coordinate or weight");
        rc = GS_ERR_NONFINITE;
    }
    if (!rc && (hing.status & ST_WEIGHT)) {
        set_error("a weight is <= 0 (weights must be positive)");
        rc = GS_ERR_WEIGHT;
    }
    if (rc) {
        cudaStreamSynchronize(st);
        destroy(h);
        return rc;
    }
    *out = h;
    return GS_OK;
}

extern "C" void gs_tree_free(gs_tree *t) { destroy(t); }

extern "C" int gs_sum_trees(const gs_tree *qt, const gs_tree *rt, const double *h, int nh, double eps, double *out,
                            const gs_opts *opts, void *stream, gs_stats *stats) {
    if (!qt || !rt || !h || !out || nh < 1 || nh > 64) {
        set_error("gs_sum_trees: NULL tree, h or out, or nh outside [1, 64]");
        return GS_ERR_ARG;
    }
    if (!rt->w) {
        set_error("gs_sum_trees: the reference tree was built without weights");
        return GS_ERR_ARG;
    }
    if (qt->t.D != rt->t.D || qt->t.dtype != rt->t.dtype || qt->leaf != rt->leaf) {
        set_error("gs_sum_trees: trees differ in D, dtype or leaf size");
        return GS_ERR_ARG;
    }
    if (!(eps > 0.0 && eps < 1.0)) {
        set_error("gs_sum_trees: eps=%g must lie in (0, 1) (gs_sum computes exhaustive sums)", eps);
        return GS_ERR_ARG;
    }
    for (int j = 0; j < nh; ++j)
        if (!(h[j] > 0.0) || !isfinite(h[j])) {
            set_error("bandwidth h[%d]=%g must be finite and positive", j, h[j]);
            return GS_ERR_ARG;
        }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != qt->device || dev != rt->device) {
        set_error("gs_sum_trees: the trees live on another device");
        return GS_ERR_ARG;
    }
    gs_opts o;
    gs_opts_default(&o);
    if (opts) {
        o = *opts;
        if (o.floor_log2 == 0) o.floor_log2 = -40;
        if (o.cost_weight[0] == 0 && o.cost_weight[1] == 0 && o.cost_weight[2] == 0 && o.cost_weight[3] == 0) {
            o.cost_weight[0] = GS_COST_DH;
            o.cost_weight[1] = GS_COST_DL;
            o.cost_weight[2] = GS_COST_H2L;
            o.cost_weight[3] = GS_COST_DIRECT;
        }
    }
    o.leaf_size = rt->leaf;
    for (int k = 0; k < 4; ++k)
        if (!(o.cost_weight[k] > 0.0) || !isfinite(o.cost_weight[k])) {
            set_error("cost_weight[%d]=%g must be finite and positive", k, o.cost_weight[k]);
            return GS_ERR_ARG;
        }
    if (o.selector < GS_SEL_RULE || o.selector > GS_SEL_EXHAUSTIVE ||
        (o.selector == GS_SEL_MLP && !o.selector_params)) {
        set_error("gs_sum_trees: bad selector %d (GS_SEL_MLP needs selector_params)", o.selector);
        return GS_ERR_ARG;
    }
    if (o.floor_log2 < -1000 || o.floor_log2 > -1) {
        set_error("floor_log2=%d outside [-1000, -1]", o.floor_log2);
        return GS_ERR_ARG;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t st = (cudaStream_t)stream;
    CallCtx cx;
    cx.st = st;
    cx.stats = stats;
    cx.phase(GS_PH_INGEST);
    // this call's status word, starting from the reference set's summary
    Ingest *ing = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&ing, sizeof(Ingest), st));
    cudaError_t e = cudaMemcpyAsync(ing, rt->ing, sizeof(Ingest), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(ing, st);
        return cuda_fail(e, "gs_sum_trees");
    }
    unsigned status = 0;
    const bool mono = qt == rt;
    int rc = dualtree_run(qt->t, rt->t, mono, rt->w, rt->t.D, h, nh, eps, out, o, cx, ing, nullptr, &status);
    cudaFreeAsync(ing, st);
    if (rc == GS_OK) rc = status_to_code(status);
    if (rc == GS_OK && stats) cx.finish();
    return rc;
}

extern "C" int gs_lscv_trees(const gs_tree *t, const double *h, int nh, double eps, double *score, double *score_err,
                             const gs_opts *opts, void *stream, gs_stats *stats) {
    if (!t || !h || !score || nh < 1 || nh > 32) {
        set_error("gs_lscv_trees: NULL tree, h or score, or nh outside [1, 32]");
        return GS_ERR_ARG;
    }
    if (!t->w) {
        set_error("gs_lscv_trees: the tree was built without weights");
        return GS_ERR_ARG;
    }
    if (t->t.n < 2) {
        set_error("gs_lscv_trees needs N >= 2");
        return GS_ERR_ARG;
    }
    double hh[64];
    for (int j = 0; j < nh; ++j) {
        hh[j] = h[j];
        hh[nh + j] = h[j] * 1.4142135623730951;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = t->t.n;
    double *G = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&G, (size_t)N * 2 * nh * sizeof(double), st));
    int rc = gs_sum_trees(t, t, hh, 2 * nh, eps, G, opts, stream, stats);
    if (rc == GS_OK) rc = lscv_scores(G, t->w, N, t->t.D, h, nh, eps, t->ing, score, score_err, st);
    cudaFreeAsync(G, st);
    return rc;
}
