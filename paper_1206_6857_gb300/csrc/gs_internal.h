// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// Device-side status word bits (set with atomicOr by any kernel; read once
// by the host at the end of a call).
enum : unsigned {
    ST_NONFINITE = 1u << 0,
    ST_WEIGHT = 1u << 1,
    ST_CAPACITY = 1u << 2,
    ST_TIMEOUT = 1u << 3,
    ST_INTERNAL = 1u << 4,
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
        stats->launches = launches;
        stats->launches_base = launches_base;
    }
    ~CallCtx() {
        for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    }
};

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

// Instruction-rate probe (see gs_probe_rates).
int probe_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, cudaStream_t st);

}  // namespace gs
