// Device-side kd-tree and multi-index tables shared by the dual-tree kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// Complete kd-tree over n points: depth d = min{k : ceil(n / 2^k) <= L};
// heap-numbered nodes, node (level k, index i) = 2^k - 1 + i, holding the
// sorted positions [floor(i n / 2^k), floor((i+1) n / 2^k)).
struct TreeDev {
    int64_t n = 0;
    int D = 0;
    int depth = 0;
    int64_t nodes = 0;
    int dtype = 0;            // GS_F32 / GS_F64 of the source points
    int32_t *perm = nullptr;  // sorted position -> original index
    void *xs = nullptr;       // n x D permuted coordinates (source dtype)
    double *lo = nullptr, *hi = nullptr, *center = nullptr;   // nodes x D
    float *lo32 = nullptr, *hi32 = nullptr;  // boxes rounded outward to FP32
    double *rad = nullptr;    // half the widest extent
    float *rad32 = nullptr;   // rad rounded down to FP32
    double *W = nullptr;      // weight sums
    float *W32d = nullptr, *W32u = nullptr;   // W rounded down / up to FP32
    float *wmin = nullptr;    // smallest weight (monochromatic lower bound)
    int32_t *split_dim = nullptr;
    float *rec = nullptr;     // packed FP32 records in sorted order (base case)
    int rec_stride = 0;       // floats per record
    double *moments = nullptr;// nodes x T raw moments (reference tree only)
    int mom_terms = 0;
};

__host__ __device__ inline int64_t level_begin(int64_t n, int k, int64_t i) { return (i * n) >> k; }

// Multi-index tables in graded lexicographic order (|alpha| ascending;
// inside a degree, lexicographically descending), for orders up to P.
struct SeriesTables {
    int D = 0, P = 0, T = 0;           // T = C(D+P-1, D)
    int Tp[17] = {0};                  // Tp[p] = terms with |alpha| < p
    uint8_t *alpha = nullptr;          // T x D exponents
    uint8_t *deg = nullptr;            // T
    int32_t *pred = nullptr;           // alpha with its last non-zero entry zeroed
    uint8_t *pred_dim = nullptr;       // that entry's dimension
    int32_t *dpred = nullptr;          // alpha with its last non-zero entry decreased by one
    double *inv_fact = nullptr;        // 1 / alpha!
    // H2H: for each gamma, the (alpha, beta) index pairs with alpha + beta = gamma
    int32_t *h2h_off = nullptr;        // T + 1
    int32_t *h2h_pairs = nullptr;      // 2 per entry
    // L2L one dimension at a time: the multi-indices along dimension d form
    // lines alpha0, alpha0 + e_d, alpha0 + 2 e_d, ... (alpha0_d = 0)
    int32_t *l2s_next = nullptr;       // D x T: index of alpha + e_d (-1 past order P)
    int32_t *l2s_line = nullptr;       // D x T: the line starts alpha0 of dimension d, in table order
    int32_t *l2s_nlines = nullptr;     // D x 17: lines of dimension d whose start has degree < p
    void *mem = nullptr;               // single device allocation holding all of the above
};

}  // namespace gs
