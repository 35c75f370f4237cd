// Many independent Gaussian-sum problems in one call (a batch of KDE
// problems of uneven N and D).  Problems summed exhaustively (eps = 0, or
// small ones under GS_FLAG_SMALL_EXHAUSTIVE) with FP32 points and D <= 8 go
// through the grouped exhaustive path: a handful of launches for all of them
// together.  Every other problem is a full gs_sum: its own trees, frontier
// and base case.  A problem's traversal is a chain of small launches with one
// host read per frontier iteration, so the batch keeps the GPU busy by
// running several problems at once: worker host threads, each with its own
// stream, take problems largest-first from a shared counter, while the
// calling thread runs the grouped path on a stream of its own.  The caller's
// stream is joined at both ends with events.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <string.h>

#include "gs_internal.h"

using namespace gs;

static int cu_ok(cudaError_t e, const char *what) { return e == cudaSuccess ? GS_OK : cuda_fail(e, what); }

extern "C" int gs_sum_batched(int nprob, const gs_problem *probs, const gs_opts *opts, int nworkers, void *stream,
                              gs_stats *stats, int32_t *status) {
    if (nprob < 0 || (nprob > 0 && !probs) || nworkers < 0) {
        set_error("gs_sum_batched: bad arguments (nprob, probs, nworkers)");
        return GS_ERR_ARG;
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    if (nprob == 0) return GS_OK;
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    if (nworkers == 0) nworkers = 8;
    if (nworkers > nprob) nworkers = nprob;
    cudaStream_t caller = (cudaStream_t)stream;
    // exhaustive problems the grouped path takes; the rest, largest first (M N nh)
    const bool small_ex = opts && (opts->flags & GS_FLAG_SMALL_EXHAUSTIVE);
    const double small_work = opts && opts->small_work > 0.0 ? opts->small_work : 0.0;   // 0: by D
    std::vector<int> grouped, order;
    for (int i = 0; i < nprob; ++i) {
        const gs_problem &p = probs[i];
        const double sw = small_work > 0.0 ? small_work : (p.D <= 2 ? GS_SMALL_WORK_D2 : GS_SMALL_WORK);
        const bool exh = p.eps == 0.0 || (small_ex && (double)p.M * (double)p.N * (double)p.nh <= sw);
        if (exh && exhaustive_groupable(p) &&
            check_common(p.queries, p.M, p.refs, p.weights, p.N, p.D, p.dtype, p.h, p.nh, p.eps, p.out) == GS_OK)
            grouped.push_back(i);
        else
            order.push_back(i);
    }
    const int nrest = (int)order.size();
    if (nworkers > nrest) nworkers = nrest > 0 ? nrest : 1;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)probs[a].M * (double)probs[a].N * probs[a].nh;
        const double wb = (double)probs[b].M * (double)probs[b].N * probs[b].nh;
        return wa > wb;
    });
    cudaEvent_t start = nullptr, stop = nullptr;
    GS_CUDA_TRY(cudaEventCreate(&start));
    GS_CUDA_TRY(cudaEventCreate(&stop));
    GS_CUDA_TRY(cudaEventRecord(start, caller));
    std::atomic<int> next{0};
    std::mutex mu;
    int first_rc = GS_OK;
    std::string first_msg;
    std::vector<gs_stats> wstats(nworkers);
    std::vector<cudaEvent_t> done(nworkers, nullptr);
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        int rc = cu_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "worker stream");
        if (rc == GS_OK) rc = cu_ok(cudaStreamWaitEvent(st, start, 0), "worker start");
        if (rc == GS_OK) rc = cu_ok(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming), "worker event");
        memset(&wstats[w], 0, sizeof(gs_stats));
        for (int k; rc == GS_OK && (k = next.fetch_add(1)) < nrest;) {
            const int i = order[k];
            const gs_problem &p = probs[i];
            gs_stats ps;
            const int r = sum_impl(p.queries, p.M, p.refs, p.weights, p.N, p.D, p.dtype, p.h, p.nh, p.eps, p.out,
                                   opts, st, stats ? &ps : nullptr, nullptr);
            if (status) status[i] = r;
            if (r != GS_OK) {
                std::lock_guard<std::mutex> lk(mu);
                if (first_rc == GS_OK) {
                    first_rc = r;
                    first_msg = "problem " + std::to_string(i) + ": " + gs_last_error();
                }
                continue;
            }
            if (stats) {
                gs_stats &a = wstats[w];
                a.pairs_fd += ps.pairs_fd; a.pairs_dh += ps.pairs_dh; a.pairs_dl += ps.pairs_dl;
                a.pairs_h2l += ps.pairs_h2l; a.pairs_base += ps.pairs_base; a.pairs_split += ps.pairs_split;
                a.point_pairs_base += ps.point_pairs_base; a.point_pairs_tc += ps.point_pairs_tc; a.launches += ps.launches;
                a.launches_base += ps.launches_base;
                if (ps.levels > a.levels) a.levels = ps.levels;
                a.retries += ps.retries;
                if (ps.fp32_rel_bound > a.fp32_rel_bound) a.fp32_rel_bound = ps.fp32_rel_bound;
                for (int k2 = 0; k2 < GS_NPHASE; ++k2) a.ms_phase[k2] += ps.ms_phase[k2];
                for (int k2 = 0; k2 < 3; ++k2) a.ms_series[k2] += ps.ms_series[k2];
            }
        }
        if (done[w]) cudaEventRecord(done[w], st);
        if (st) cudaStreamDestroy(st);   // destruction waits for the stream's work in the background
        if (rc != GS_OK) {
            std::lock_guard<std::mutex> lk(mu);
            if (first_rc == GS_OK) {
                first_rc = rc;
                first_msg = gs_last_error();
            }
        }
    };
    std::vector<std::thread> th;
    for (int w = 0; w < nworkers && nrest > 0; ++w) th.emplace_back(worker, w);
    // the grouped exhaustive problems, on a stream of their own
    gs_stats gstats;
    memset(&gstats, 0, sizeof(gstats));
    cudaStream_t gst = nullptr;
    cudaEvent_t gdone = nullptr;
    if (!grouped.empty()) {
        int grc = cu_ok(cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking), "grouped stream");
        if (grc == GS_OK) grc = cu_ok(cudaStreamWaitEvent(gst, start, 0), "grouped start");
        if (grc == GS_OK) grc = cu_ok(cudaEventCreateWithFlags(&gdone, cudaEventDisableTiming), "grouped event");
        if (grc == GS_OK)
            grc = exhaustive_batch(probs, grouped.data(), (int)grouped.size(), gst, status, stats ? &gstats : nullptr);
        if (grc != GS_OK) {
            if (status && !gdone)
                for (int i : grouped) status[i] = grc;
            std::lock_guard<std::mutex> lk(mu);
            if (first_rc == GS_OK) {
                first_rc = grc;
                first_msg = std::string("grouped exhaustive problems: ") + gs_last_error();
            }
        }
        if (gdone) cudaEventRecord(gdone, gst);
    }
    for (auto &t : th) t.join();
    if (gdone) {
        cudaStreamWaitEvent(caller, gdone, 0);
        cudaEventDestroy(gdone);
    }
    if (gst) cudaStreamDestroy(gst);
    for (int w = 0; w < nworkers; ++w)
        if (done[w]) {
            cudaStreamWaitEvent(caller, done[w], 0);
            cudaEventDestroy(done[w]);
        }
    cudaEventRecord(stop, caller);
    cudaError_t e = cudaEventSynchronize(stop);
    if (stats && e == cudaSuccess) {
        stats->point_pairs_base += gstats.point_pairs_base;
        stats->launches += gstats.launches;
        stats->launches_base += gstats.launches_base;
        for (int w = 0; w < nworkers; ++w) {
            const gs_stats &a = wstats[w];
            stats->pairs_fd += a.pairs_fd; stats->pairs_dh += a.pairs_dh; stats->pairs_dl += a.pairs_dl;
            stats->pairs_h2l += a.pairs_h2l; stats->pairs_base += a.pairs_base; stats->pairs_split += a.pairs_split;
            stats->point_pairs_base += a.point_pairs_base; stats->point_pairs_tc += a.point_pairs_tc; stats->launches += a.launches;
            stats->launches_base += a.launches_base;
            if (a.levels > stats->levels) stats->levels = a.levels;
            stats->retries += a.retries;
            if (a.fp32_rel_bound > stats->fp32_rel_bound) stats->fp32_rel_bound = a.fp32_rel_bound;
            for (int k = 0; k < GS_NPHASE; ++k) stats->ms_phase[k] += a.ms_phase[k];
            for (int k = 0; k < 3; ++k) stats->ms_series[k] += a.ms_series[k];
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, start, stop) == cudaSuccess) stats->ms_total = ms;
    }
    cudaEventDestroy(start);
    cudaEventDestroy(stop);
    if (first_rc != GS_OK) {
        set_error("%s", first_msg.c_str());
        return first_rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "gs_sum_batched");
    return GS_OK;
}
