// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"
#include "gs_frontier.cuh"
#include "gs_tree.cuh"

namespace gs {

// Device-side status word bits (set with atomicOr by any kernel; read once
// by the host at the end of a call).
enum : unsigned {
    ST_NONFINITE = 1u << 0,
    ST_WEIGHT = 1u << 1,
    ST_CAPACITY = 1u << 2,
    ST_TIMEOUT = 1u << 3,
    ST_INTERNAL = 1u << 4,
    ST_EPS = 1u << 5,        // eps too small for the FP32 base-case error charge
};

// Summary of the inputs, produced on the device by the ingest kernels.
struct Ingest {
    unsigned status;      // ST_* bits
    unsigned wmax_bits;   // largest weight (positive floats order like their bit patterns)
    unsigned wmin_bits;   // smallest weight
    unsigned pad;
    double wsum;          // sum of weights (order unspecified)
};

// Per-call host context: the stream, launch counters and (when the caller
// asked for statistics) CUDA events bracketing each phase.
struct CallCtx {
    cudaStream_t st = nullptr;
    gs_stats *stats = nullptr;
    int64_t launches = 0, launches_base = 0;
    static constexpr int kMaxMarks = 256;
    cudaEvent_t ev[kMaxMarks];
    int ev_phase[kMaxMarks];
    int nev = 0;
    int open_phase = -1;
    // GS_DEBUG_SYNC=1 in the environment: synchronise and check after every
    // launch site that calls check(), naming the kernel in the error.
    bool debug = debug_sync_enabled();
    static bool debug_sync_enabled();
    int check(const char *what);

    // Start timing `phase` (closing any open one).  No-op without stats.
    void phase(int ph) {
        if (!stats) return;
        if (nev + 1 >= kMaxMarks) return;
        if (cudaEventCreate(&ev[nev]) != cudaSuccess) return;
        cudaEventRecord(ev[nev], st);
        ev_phase[nev] = ph;
        ++nev;
        open_phase = ph;
    }
    void end() { phase(-1); }
    // Time one launch into stats->ms_series[slot] (slot 0-2) or
    // stats->ms_base_kernels[slot - kTimerBase] (kTimerBase: the tensor-core
    // kernel, kTimerBase + 1: the direct one): mark(slot) before it, mark(-1)
    // after.  No-op without stats.
    static constexpr int kMaxTimers = 24;
    static constexpr int kTimerBase = 3;
    cudaEvent_t tev[kMaxTimers];
    int tslot[kMaxTimers];
    int ntev = 0;
    void mark(int slot) {
        if (!stats || ntev >= kMaxTimers) return;
        if (cudaEventCreate(&tev[ntev]) != cudaSuccess) return;
        cudaEventRecord(tev[ntev], st);
        tslot[ntev] = slot;
        ++ntev;
    }
    // After the stream has been synchronised: fold event pairs into stats.
    void finish() {
        if (!stats) return;
        for (int i = 0; i + 1 < nev; ++i) {
            if (ev_phase[i] < 0 || ev_phase[i] >= GS_NPHASE) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) stats->ms_phase[ev_phase[i]] += ms;
        }
        if (nev >= 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[0], ev[nev - 1]) == cudaSuccess) stats->ms_total = ms;
        }
        for (int i = 0; i + 1 < ntev; ++i) {
            if (tslot[i] < 0 || tslot[i] > kTimerBase + 1) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, tev[i], tev[i + 1]) != cudaSuccess) continue;
            if (tslot[i] >= kTimerBase)
                stats->ms_base_kernels[tslot[i] - kTimerBase] += ms;
            else
                stats->ms_series[tslot[i]] += ms;
        }
        stats->launches = launches;
        stats->launches_base = launches_base;
    }
    ~CallCtx() {
        for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
        for (int i = 0; i < ntev; ++i) cudaEventDestroy(tev[i]);
    }
};

// Let `fn` launch with up to the device's opt-in maximum of dynamic shared
// memory.  The attribute is per function and shared by every host thread, so
// it is always set to that same maximum (never to one launch's size, which a
// concurrent caller could lower between another's set and launch).
inline cudaError_t allow_max_smem(const void *fn) {
    int dev = 0, mx = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
    return e;
}

// Every device scratch allocation of the library goes through here
// (stream-ordered, from the library's pool of the current device).
// gs_debug_fail_alloc arms a one-shot failure of a later allocation, so
// tests can check that a failed allocation surfaces as GS_ERR_OOM and leaves
// the library usable.
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);

// The library's memory pool of the current device (created on first use;
// freed memory stays in it until gs_trim_memory).
cudaError_t scratch_pool(cudaMemPool_t *out);

// Device status bits -> GS_ERR_* code (and message); GS_OK when clear.
int status_to_code(unsigned st);

// LSCV scores (and their eps-implied bounds) of nh bandwidths from the sums
// G (caller order, N x 2nh: h then sqrt(2) h) and the weight total in *ing;
// synchronises the stream.
int lscv_scores(const double *G, const float *weights, int64_t N, int D, const double *h, int nh, double eps,
                const Ingest *ing, double *score, double *score_err, cudaStream_t st);

// Host-side error reporting (thread-local message).
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define GS_CUDA_TRY(call)                                         \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) return gs::cuda_fail(e__, #call); \
    } while (0)

// Reset *ing (status 0, wmax 0, wmin +inf, wsum 0) and run the input checks
// over refs/weights (and queries when distinct).  Asynchronous on stream.
cudaError_t launch_ingest(Ingest *ing, const void *queries, int64_t M, const void *refs,
                          const float *weights, int64_t N, int D, int dtype, CallCtx &cx);

// Exhaustive sums (Section 1 definition, FP32 terms, FP64 per query):
// out[q*nh + j] for all q < M, j < nh.  neg_c[j] = -log2(e) / (2 h_j^2).
// Allocates and frees its own packed-reference scratch on the stream.
int exhaustive_sum(const void *queries, int64_t M, const void *refs, const float *weights,
                   int64_t N, int D, int dtype, const double *h, int nh, const Ingest *ing,
                   double *out, CallCtx &cx);

// Argument checks shared by gs_sum and the batched entry point.
int check_common(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N, int D,
                 int dtype, const double *h, int nh, double eps, double *out);

// Exhaustive sums of many problems with few launches (FP32 points, D <= 8:
// exhaustive_groupable): every listed problem (probs[idx[k]]) is summed as
// gs_sum with eps = 0 would, its code written to status[idx[k]]; synchronises
// the stream once.  Returns GS_OK or the first failing code.
bool exhaustive_groupable(const gs_problem &p);
int exhaustive_batch(const gs_problem *probs, const int *idx, int n, cudaStream_t st, int32_t *status,
                     gs_stats *stats);

// ---- dual-tree path -------------------------------------------------------
// Per-pair record of a logged traversal (training data of the pair
// selector), indexed by global pair id (iterations in order, pairs of an
// iteration in frontier order).  Arrays grow between iterations.
struct PairLog {
    float *feat = nullptr;        // 12 features (pairs whose FD test failed)
    int8_t *pc = nullptr;         // smallest certified order of DH, DL, H2L (0: none); kind
    int32_t *nq = nullptr, *nr = nullptr;
    int64_t *par = nullptr;       // parent pair id (-1 at the root iteration)
    int64_t cap = 0;
    int64_t *pid[2] = {nullptr, nullptr};   // parent id of each pair slot, per frontier buffer
    int64_t cap_pid[2] = {0, 0};
    int64_t iter_off[80] = {0};   // first pair id of each iteration; iter_off[niter] = total
    int niter = 0;
};
enum : int { LOG_FD = 0, LOG_BASE = 1, LOG_SPLIT = 2 };

// One merged base-case entry: a reference leaf (heap number) and the mask of
// the bandwidths (bits ranked by ascending h) its query leaf needs.
struct MergedEntry {
    int32_t r;
    uint32_t mask;
};

struct TraversalIn {
    const TreeDev *qt = nullptr, *rt = nullptr;
    const Ingest *ing = nullptr;
    const float *weights = nullptr;
    const double *h = nullptr;   // host
    int D = 0, nh = 0, P = 0, selector = 0, tokens = 1, mono = 0, floor_log2 = -40;
    double eps = 0.0;
    double cost_w[4] = {GS_COST_DH, GS_COST_DL, GS_COST_H2L, GS_COST_DIRECT};
    int flags = 0;                // gs_opts.flags
    const float *mlp = nullptr;   // selector network (GS_SEL_MLP)
    PairLog *log = nullptr;       // log every pair (FD-only decisions)
};

struct FrontierBufs {
    FrontierState *fs = nullptr;
    Group *groups[2] = {nullptr, nullptr};
    int32_t *pr[2] = {nullptr, nullptr};
    uint8_t *dec = nullptr;
    int32_t *cnt = nullptr;
    long long *off = nullptr, *partial = nullptr;
    Group *base_groups = nullptr;
    int32_t *base_r = nullptr;
    SeriesEntry *series[3] = {nullptr, nullptr, nullptr};   // DH, DL, H2L action lists
    float *geo = nullptr;           // per pair (4 floats): K(delta_max), K(delta_min), e^{-dmin^2/4h^2}, lower bound
    double *fin = nullptr, *tok = nullptr, *est = nullptr;
    double *inv_2h2 = nullptr, *inv_4h2 = nullptr, *inv_h = nullptr, *inv_s = nullptr;
    unsigned long long *evals = nullptr;
    int4 *trace = nullptr;
    int64_t trace_cap = 0;
    int64_t cap_pairs = 0, cap_groups = 0, cap_base = 0, cap_base_groups = 0, cap_series[3] = {0, 0, 0};
    int64_t cap_pr[2] = {0, 0};     // capacity of each pair buffer
    int64_t cap_geo = 0;
    int64_t n_series[3] = {0, 0, 0};// actions per list after the traversal (host copy)
    int64_t n_base_groups = 0;
    int64_t n_base = 0;             // base-case list entries (query leaf, bandwidth, reference leaf)
    int grid_warps = 0;
    int64_t *host_totals = nullptr; // pinned host scratch (kCols + 8 int64)
};

int build_tree(const void *x, const float *w, int64_t n, int D, int dtype, int L, const Ingest *ing, int DP,
               int rec_stride, bool with_weights, CallCtx &cx, TreeDev *out);
int build_moments(TreeDev &t, const float *w, const SeriesTables &tb, CallCtx &cx);
void free_tree(TreeDev &t, cudaStream_t st);
int build_series_tables(int D, int P, SeriesTables *tb, cudaStream_t st);
void free_series_tables(SeriesTables *tb, cudaStream_t st);
int run_frontier(const TraversalIn &in, FrontierBufs &fb, CallCtx &cx);
int run_basecase(const TraversalIn &in, FrontierBufs &fb, double *Gq, int DP, CallCtx &cx);
bool merged_base_possible(const TraversalIn &in);
// In-place exclusive prefix sum of n int64 values; *total (device) receives the sum.
int scan_i64(long long *v, int64_t n, long long *total, CallCtx &cx);
int run_basecase_merged(const TraversalIn &in, FrontierBufs &fb, double *Gq, int DP, CallCtx &cx);
// Tensor-core base case (9 <= D <= 16, FP32 points, leaves of at most 128
// points): whether a call takes it, and the extra FP32 charge it needs.
bool tc_base_enabled(int D, int dtype, int flags, int64_t qn, int q_depth, int64_t rn, int r_depth, int nh);
double tc_charge();
// Splits the merged entries (ent, off over lq query-leaf rows) between the
// tensor-core kernel (entries whose pair passes the error guard) and the
// direct kernel: runs the former and leaves the latter in (ent_dir, off_dir),
// allocated on the stream (the caller frees them).
int run_basecase_tc(const TraversalIn &in, const MergedEntry *ent, const long long *off, int64_t lq,
                    long long total, const float *negc, const int *jcol, const double *h_by_bit, double *Gq,
                    MergedEntry **ent_dir, long long **off_dir, unsigned long long *evals, CallCtx &cx);
int run_series_and_final(const TraversalIn &in, FrontierBufs &fb, const SeriesTables *tb, double *Gq,
                         double *B, int32_t *pL, double *out, CallCtx &cx);

// Padded dimension used by the FP32 record layouts (1..8, 12, 16, 24, 32).
int dp_for(int D);
int plimit_for(int D);

// Optional outputs of a dual-tree call used by tests and tools.
struct TraceOut {
    int32_t *trace = nullptr;     // device, 4 x cap int32
    int64_t cap = 0;
    int64_t *len = nullptr;       // host
    int32_t *qperm = nullptr;     // device, M (may be NULL)
    int32_t *rperm = nullptr;     // device, N (may be NULL)
};

int dualtree_sum(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N, int D,
                 int dtype, const double *h, int nh, double eps, double *out, const gs_opts &o, CallCtx &cx,
                 Ingest *ing, TraceOut *trace, unsigned *status_out, PairLog *log = nullptr);
// The traversal, series, base case and downward pass on trees already built
// (qt ignored when mono); `weights` are the references' weights in caller
// order (for the moments).  The trees are not modified.
int dualtree_run(const TreeDev &qt, const TreeDev &rt, bool mono, const float *weights, int D,
                 const double *h, int nh, double eps, double *out, const gs_opts &o, CallCtx &cx, Ingest *ing,
                 TraceOut *trace, unsigned *status_out, PairLog *log = nullptr);
// floats per packed FP32 record (dimension bucket + log2 weight, 16-byte units)
inline int record_stride(int D) { return (((dp_for(D) + 1) * 4 + 15) / 16) * 4; }

// gs_sum with its options checked; trace and log are optional.
int sum_impl(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N, int D,
             int dtype, const double *h, int nh, double eps, double *out, const gs_opts *opts, void *stream,
             gs_stats *stats, TraceOut *trace, PairLog *log = nullptr);

// Instruction-rate probe (see gs_probe_rates).
int probe_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, cudaStream_t st);

}  // namespace gs
