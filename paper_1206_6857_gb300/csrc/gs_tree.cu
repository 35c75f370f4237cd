// kd-tree build, node statistics, packed base-case records and reference
// node moments (Section 6: "construct two trees ... Hermite moments of order
// PLIMIT pre-computed for the reference tree"; Fig. 5 buildLeaf /
// buildInternal with H2H).
//
// Tree: complete binary kd-tree of depth d = min{k : ceil(n/2^k) <= L}.
// Node (k, i) owns sorted positions [floor(i n/2^k), floor((i+1) n/2^k)).
// A node splits on the widest dimension of its bounding box (lowest index on
// ties); its left child receives the floor((2i+1) n / 2^(k+1)) - begin
// smallest points by the key (coordinate, original index).  Partitions are
// stable, so inside every leaf the points stay in ascending original order.
//
// The build runs level by level over all nodes of a level at once:
//   bbox   -- segmented min/max with order-preserving integer keys (atomics)
//   select -- radix select of the split rank per node, 8 bits per pass
//   split  -- packed (less, equal) counts, device-wide exclusive scan, then a
//             stable scatter of the permutation and the coordinates.
// This translation unit is compiled without FMA contraction so the node
// statistics (centres, radii) match a plain IEEE evaluation.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_tree.cuh"

namespace gs {

// --------------------------------------------------------------------------
// order-preserving integer keys
// --------------------------------------------------------------------------
template <typename T>
struct Key;
template <>
struct Key<float> {
    using K = uint32_t;
    static constexpr int BITS = 32;
    __device__ static K enc(float f) {
        f = f + 0.0f;   // -0 -> +0
        uint32_t u = __float_as_uint(f);
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    __device__ static float dec(K k) {
        uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
        return __uint_as_float(u);
    }
};
template <>
struct Key<double> {
    using K = unsigned long long;
    static constexpr int BITS = 64;
    __device__ static K enc(double f) {
        f = f + 0.0;
        unsigned long long u = (unsigned long long)__double_as_longlong(f);
        return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    }
    __device__ static double dec(K k) {
        unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
        return __longlong_as_double((long long)u);
    }
};

__device__ __forceinline__ int64_t node_of(int64_t p, int k, int64_t n) {
    return (((p + 1) << k) - 1) / n;
}

template <typename K>
struct SelState {
    K prefix;
    uint32_t rem;        // rank still to place inside the current prefix
    uint32_t cnt_less;   // elements strictly below the prefix so far
    int32_t dim;
    int32_t pad;
};

constexpr int kTB = 256;

// --------------------------------------------------------------------------
// per-level kernels
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_level_bbox(const T *__restrict__ xs, int64_t n, int D, int k,
                             typename Key<T>::K *bmin, typename Key<T>::K *bmax) {
    using K = typename Key<T>::K;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t p = base + lane;
        const bool valid = p < n;
        const int64_t i = valid ? node_of(p, k, n) : -1;
        const int64_t i0 = __shfl_sync(0xffffffffu, i, 0);
        const bool uniform = __all_sync(0xffffffffu, !valid || i == i0);
        for (int d = 0; d < D; ++d) {
            K v = valid ? Key<T>::enc(xs[p * D + d]) : 0;
            if (uniform) {
                K mn = valid ? v : ~(K)0, mx = valid ? v : (K)0;
                for (int o = 16; o > 0; o >>= 1) {
                    K a = __shfl_xor_sync(0xffffffffu, mn, o), b = __shfl_xor_sync(0xffffffffu, mx, o);
                    mn = a < mn ? a : mn;
                    mx = b > mx ? b : mx;
                }
                if (lane == 0) {
                    atomicMin(&bmin[i0 * D + d], mn);
                    atomicMax(&bmax[i0 * D + d], mx);
                }
            } else if (valid) {
                atomicMin(&bmin[i * D + d], v);
                atomicMax(&bmax[i * D + d], v);
            }
        }
    }
}

template <typename T>
__global__ void k_level_select_dim(int64_t n, int D, int k, const typename Key<T>::K *bmin,
                                   const typename Key<T>::K *bmax, int32_t *split_dim,
                                   SelState<typename Key<T>::K> *sel) {
    const int64_t nn = 1ll << k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        double best = -1.0;
        for (int d = 0; d < D; ++d) {
            const double lo = (double)Key<T>::dec(bmin[i * D + d]);
            const double hi = (double)Key<T>::dec(bmax[i * D + d]);
            const double ext = hi - lo;
            if (ext > best) {
                best = ext;
                s = d;
            }
        }
        const int64_t b = level_begin(n, k, i);
        const int64_t mid = ((2 * i + 1) * n) >> (k + 1);
        split_dim[nn - 1 + i] = s;
        SelState<typename Key<T>::K> st;
        st.prefix = 0;
        st.rem = (uint32_t)(mid - b);
        st.cnt_less = 0;
        st.dim = s;
        st.pad = 0;
        sel[i] = st;
    }
}

constexpr int kHistChunk = 2048;

template <typename T>
__global__ void __launch_bounds__(kTB)
k_level_hist(const T *__restrict__ xs, int64_t n, int D, int k, int shift,
             const SelState<typename Key<T>::K> *__restrict__ sel, uint32_t *hist) {
    using K = typename Key<T>::K;
    __shared__ uint32_t sh[256];
    const int64_t p0 = (int64_t)blockIdx.x * kHistChunk;
    if (p0 >= n) return;
    const int64_t p1 = min(p0 + kHistChunk, n);
    const int64_t i_first = node_of(p0, k, n), i_last = node_of(p1 - 1, k, n);
    const bool single = i_first == i_last;
    const bool all_match = shift + 8 >= Key<T>::BITS;
    if (single) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) sh[t] = 0;
        __syncthreads();
        const SelState<K> st = sel[i_first];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const K key = Key<T>::enc(xs[p * D + st.dim]);
            if (all_match || ((key ^ st.prefix) >> (shift + 8)) == 0)
                atomicAdd(&sh[(unsigned)(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 256; t += blockDim.x)
            if (sh[t]) atomicAdd(&hist[i_first * 256 + t], sh[t]);
    } else {
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t i = node_of(p, k, n);
            const SelState<K> st = sel[i];
            const K key = Key<T>::enc(xs[p * D + st.dim]);
            if (all_match || ((key ^ st.prefix) >> (shift + 8)) == 0)
                atomicAdd(&hist[i * 256 + ((unsigned)(key >> shift) & 255u)], 1u);
        }
    }
}

template <typename K>
__global__ void k_level_pick(int k, int shift, const uint32_t *__restrict__ hist, SelState<K> *sel) {
    const int lane = threadIdx.x & 31;
    const int64_t nn = 1ll << k;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < nn; i += warps) {
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            c[t] = hist[i * 256 + lane * 8 + t];
            tot += c[t];
        }
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t excl = incl - tot;
        SelState<K> st = sel[i];
        if (excl <= st.rem && st.rem < incl) {
            uint32_t cum = excl;
            int digit = lane * 8;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (st.rem < cum + c[t]) {
                    digit = lane * 8 + t;
                    break;
                }
                cum += c[t];
            }
            st.prefix |= ((K)digit) << shift;
            st.cnt_less += cum;
            st.rem -= cum;
            sel[i] = st;
        }
    }
}

// packed (less-than-pivot << 32 | equal-to-pivot) for position p
template <typename T>
__device__ __forceinline__ unsigned long long part_flags(const T *xs, int64_t p, int D, int k, int64_t n,
                                                         const SelState<typename Key<T>::K> *sel) {
    const int64_t i = node_of(p, k, n);
    const SelState<typename Key<T>::K> st = sel[i];
    const typename Key<T>::K key = Key<T>::enc(xs[p * D + st.dim]);
    return ((unsigned long long)(key < st.prefix) << 32) | (unsigned long long)(key == st.prefix);
}

constexpr int kScanGrid = 1024;

__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v, unsigned long long *tot) {
    __shared__ unsigned long long wsum[kTB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < kTB / 32 ? wsum[lane] : 0ull;
        unsigned long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += u;
        }
        if (lane < kTB / 32) wsum[lane] = si - s;
        if (lane == kTB / 32 - 1) *tot = si;
    }
    __syncthreads();
    const unsigned long long r = wsum[w] + incl - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kTB)
k_part_sum(const T *__restrict__ xs, int64_t n, int D, int k, const SelState<typename Key<T>::K> *sel,
           unsigned long long *partial) {
    __shared__ unsigned long long tot;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = blockIdx.x * chunk, p1 = min(p0 + chunk, n);
    unsigned long long s = 0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) s += part_flags<T>(xs, p, D, k, n, sel);
    block_excl_scan_u64(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kTB) k_scan_partials_u64(unsigned long long *partial, int m) {
    __shared__ unsigned long long tot;
    unsigned long long carry = 0;
    for (int b0 = 0; b0 < m; b0 += kTB) {
        const int b = b0 + threadIdx.x;
        const unsigned long long v = b < m ? partial[b] : 0ull;
        const unsigned long long e = block_excl_scan_u64(v, &tot);
        if (b < m) partial[b] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kTB)
k_part_prefix(const T *__restrict__ xs, int64_t n, int D, int k, const SelState<typename Key<T>::K> *sel,
              const unsigned long long *__restrict__ partial, unsigned long long *S) {
    __shared__ unsigned long long tot;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = blockIdx.x * chunk, p1 = min(p0 + chunk, n);
    unsigned long long carry = partial[blockIdx.x];
    for (int64_t t0 = p0; t0 < p1; t0 += blockDim.x) {
        const int64_t p = t0 + threadIdx.x;
        const unsigned long long v = p < p1 ? part_flags<T>(xs, p, D, k, n, sel) : 0ull;
        const unsigned long long e = block_excl_scan_u64(v, &tot);
        if (p < p1) S[p] = carry + e;
        carry += tot;
    }
}

template <typename T>
__global__ void k_part_scatter(const T *__restrict__ xs, const int32_t *__restrict__ perm, int64_t n, int D,
                               int k, const SelState<typename Key<T>::K> *__restrict__ sel,
                               const unsigned long long *__restrict__ S, T *xs_out, int32_t *perm_out,
                               unsigned *status) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = node_of(p, k, n);
        const int64_t b = level_begin(n, k, i);
        const int64_t mid = ((2 * i + 1) * n) >> (k + 1);
        const SelState<typename Key<T>::K> st = sel[i];
        const unsigned long long base = S[b], sp = S[p];
        const int64_t lt_before = (int64_t)((sp >> 32) - (base >> 32));
        const int64_t eq_before = (int64_t)((sp & 0xffffffffull) - (base & 0xffffffffull));
        const int64_t r_eq = st.rem;
        const int64_t left_before = lt_before + (eq_before < r_eq ? eq_before : r_eq);
        const typename Key<T>::K key = Key<T>::enc(xs[p * D + st.dim]);
        const bool left = key < st.prefix || (key == st.prefix && eq_before < r_eq);
        const int64_t np = left ? b + left_before : mid + (p - b - left_before);
        const int64_t e = level_begin(n, k, i + 1);
        if (np < b || np >= e || (left && np >= mid) || (!left && np < mid)) {
            atomicOr(status, ST_INTERNAL);   // inconsistent split: never write outside the node
            continue;
        }
        perm_out[np] = perm[p];
        for (int d = 0; d < D; ++d) xs_out[np * D + d] = xs[p * D + d];
    }
}

// --------------------------------------------------------------------------
// one level of small nodes in one launch: a CTA per node takes the node's
// bounding box, its split dimension, the radix select of the split rank and
// the stable scatter, with the same arithmetic and order as the per-level
// kernels above (so the tree is identical); used for the levels whose nodes
// hold at most kNodeFused points, where the per-level kernels are launch-bound.
// The node's keys in the split dimension are staged in shared memory once, so
// the select passes and the scatter read no global memory.
// --------------------------------------------------------------------------
constexpr int64_t kNodeFused = 16384;

// exclusive block-wide scan for NT threads (NT a multiple of 32, at most 1024)
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan_n(unsigned long long v, unsigned long long *tot) {
    __shared__ unsigned long long wsum[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const unsigned long long s = lane < NT / 32 ? wsum[lane] : 0ull;
        unsigned long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += u;
        }
        if (lane < NT / 32) wsum[lane] = si - s;
        if (lane == NT / 32 - 1) *tot = si;
    }
    __syncthreads();
    const unsigned long long r = wsum[w] + incl - v;
    __syncthreads();
    return r;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_level_node(const T *__restrict__ xs, const int32_t *__restrict__ perm, int64_t n, int D, int k,
             int32_t *split_dim, T *xs_out, int32_t *perm_out, unsigned *status) {
    using K = typename Key<T>::K;
    extern __shared__ unsigned long long s_dyn[];
    K *s_key = reinterpret_cast<K *>(s_dyn);   // the node's keys in the split dimension
    __shared__ K s_min[32], s_max[32];
    __shared__ uint32_t s_hist[256];
    __shared__ K s_prefix;
    __shared__ uint32_t s_rem;
    __shared__ int s_dim;
    __shared__ unsigned long long s_tot;
    const int64_t nn = 1ll << k;
    const int64_t i = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t b = level_begin(n, k, i), e = level_begin(n, k, i + 1);
    const int cnt = (int)(e - b);
    const int64_t mid = ((2 * i + 1) * n) >> (k + 1);
    // bounding box (order-preserving keys)
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        s_min[d] = ~(K)0;
        s_max[d] = (K)0;
    }
    __syncthreads();
    for (int d = 0; d < D; ++d) {
        K mn = ~(K)0, mx = (K)0;
        for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
            const K v = Key<T>::enc(xs[p * D + d]);
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const K a = __shfl_xor_sync(0xffffffffu, mn, o), c = __shfl_xor_sync(0xffffffffu, mx, o);
            mn = a < mn ? a : mn;
            mx = c > mx ? c : mx;
        }
        if (lane == 0) {
            atomicMin(&s_min[d], mn);
            atomicMax(&s_max[d], mx);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int sd = 0;
        double best = -1.0;
        for (int d = 0; d < D; ++d) {
            const double ext = (double)Key<T>::dec(s_max[d]) - (double)Key<T>::dec(s_min[d]);
            if (ext > best) {
                best = ext;
                sd = d;
            }
        }
        split_dim[nn - 1 + i] = sd;
        s_dim = sd;
        s_prefix = 0;
        s_rem = (uint32_t)(mid - b);
    }
    __syncthreads();
    const int dim = s_dim;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) s_key[q] = Key<T>::enc(xs[(b + q) * D + dim]);
    // radix select of rank (mid - b), 8 bits per pass from the top
    for (int shift = Key<T>::BITS - 8; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) s_hist[t] = 0u;
        __syncthreads();
        const K prefix = s_prefix;
        const bool all_match = shift + 8 >= Key<T>::BITS;
        // warp-aggregated: lanes with the same digit add once (the top digits
        // of nearby coordinates are mostly equal)
        for (int q0 = threadIdx.x & ~31; q0 < cnt; q0 += blockDim.x) {
            const int q = q0 + lane;
            unsigned digit = 256u;   // no count
            if (q < cnt) {
                const K key = s_key[q];
                if (all_match || ((key ^ prefix) >> (shift + 8)) == 0) digit = (unsigned)(key >> shift) & 255u;
            }
            const unsigned same = __match_any_sync(0xffffffffu, digit);
            if (digit < 256u && lane == __ffs(same) - 1) atomicAdd(&s_hist[digit], (unsigned)__popc(same));
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t c[8], tot = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                c[t] = s_hist[lane * 8 + t];
                tot += c[t];
            }
            uint32_t incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t excl = incl - tot;
            const uint32_t rem = s_rem;
            if (excl <= rem && rem < incl) {
                uint32_t cum = excl;
                int digit = lane * 8;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (rem < cum + c[t]) {
                        digit = lane * 8 + t;
                        break;
                    }
                    cum += c[t];
                }
                s_prefix = prefix | (((K)digit) << shift);
                s_rem = rem - cum;
            }
        }
        __syncthreads();
    }
    const K prefix = s_prefix;
    const int64_t r_eq = s_rem;
    // stable scatter: (less, equal) counts before each point by a block scan
    unsigned long long carry = 0;
    for (int q0 = 0; q0 < cnt; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool valid = q < cnt;
        const K key = valid ? s_key[q] : (K)0;
        const unsigned long long f =
            valid ? (((unsigned long long)(key < prefix) << 32) | (unsigned long long)(key == prefix)) : 0ull;
        const unsigned long long ex = carry + block_excl_scan_n<NT>(f, &s_tot);
        carry += s_tot;
        if (!valid) continue;
        const int64_t p = b + q;
        const int64_t lt_before = (int64_t)(ex >> 32);
        const int64_t eq_before = (int64_t)(ex & 0xffffffffull);
        const int64_t left_before = lt_before + (eq_before < r_eq ? eq_before : r_eq);
        const bool left = key < prefix || (key == prefix && eq_before < r_eq);
        const int64_t np = left ? b + left_before : mid + (p - b - left_before);
        if (np < b || np >= e || (left && np >= mid) || (!left && np < mid)) {
            atomicOr(status, ST_INTERNAL);   // inconsistent split: never write outside the node
            continue;
        }
        perm_out[np] = perm[p];
        for (int d = 0; d < D; ++d) xs_out[np * D + d] = xs[p * D + d];
    }
}

// --------------------------------------------------------------------------
// node statistics
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_leaf_stats(const T *__restrict__ xs, const int32_t *__restrict__ perm,
                             const float *__restrict__ w, int64_t n, int D, int depth, double *lo, double *hi,
                             double *W, float *wmin) {
    const int64_t nl = 1ll << depth;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = nl - 1 + i;
        const int64_t b = level_begin(n, depth, i), e = level_begin(n, depth, i + 1);
        for (int d = 0; d < D; ++d) {
            T mn = xs[b * D + d], mx = mn;
            for (int64_t p = b + 1; p < e; ++p) {
                const T v = xs[p * D + d];
                mn = v < mn ? v : mn;
                mx = v > mx ? v : mx;
            }
            lo[node * D + d] = (double)mn;
            hi[node * D + d] = (double)mx;
        }
        double s = 0.0;
        float m = INFINITY;
        for (int64_t p = b; p < e; ++p) {
            const float wv = w ? w[perm[p]] : 1.0f;
            s = s + (double)wv;
            m = fminf(m, wv);
        }
        W[node] = s;
        wmin[node] = m;
    }
}

__global__ void k_internal_stats(int D, int k, double *lo, double *hi, double *W, float *wmin) {
    const int64_t nn = 1ll << k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = nn - 1 + i, l = 2 * node + 1, r = 2 * node + 2;
        for (int d = 0; d < D; ++d) {
            lo[node * D + d] = fmin(lo[l * D + d], lo[r * D + d]);
            hi[node * D + d] = fmax(hi[l * D + d], hi[r * D + d]);
        }
        W[node] = W[l] + W[r];
        wmin[node] = fminf(wmin[l], wmin[r]);
    }
}

// every internal level, bottom up, in one CTA (small trees: one launch
// instead of one per level); same operations as k_internal_stats
__global__ void k_internal_stats_all(int D, int depth, double *lo, double *hi, double *W, float *wmin) {
    for (int k = depth - 1; k >= 0; --k) {
        const int64_t nn = 1ll << k;
        for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) {
            const int64_t node = nn - 1 + i, l = 2 * node + 1, r = 2 * node + 2;
            for (int d = 0; d < D; ++d) {
                lo[node * D + d] = fmin(lo[l * D + d], lo[r * D + d]);
                hi[node * D + d] = fmax(hi[l * D + d], hi[r * D + d]);
            }
            W[node] = W[l] + W[r];
            wmin[node] = fminf(wmin[l], wmin[r]);
        }
        __syncthreads();
    }
}

__global__ void k_center_rad(int64_t nodes, int D, const double *lo, const double *hi, double *center,
                             double *rad, float *rad32, float *lo32, float *hi32, const double *W, float *W32d,
                             float *W32u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nodes; i += (int64_t)gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int d = 0; d < D; ++d) {
            const double a = lo[i * D + d], b = hi[i * D + d];
            lo32[i * D + d] = __double2float_rd(a);
            hi32[i * D + d] = __double2float_ru(b);
            center[i * D + d] = (a + b) * 0.5;
            const double hx = (b - a) * 0.5;
            r = d == 0 ? hx : (hx > r ? hx : r);
        }
        rad[i] = r;
        rad32[i] = __double2float_rd(r);
        W32d[i] = __double2float_rd(W[i]);
        W32u[i] = __double2float_ru(W[i]);
    }
}

// packed FP32 records in sorted order: DP coordinates (relative to the leaf
// centre for FP64 input, raw for FP32 input), then log2(w / w_max) for
// reference trees (0 for query-only trees), zero padding to `stride`.
template <typename T>
__global__ void k_pack_sorted(const T *__restrict__ xs, const int32_t *__restrict__ perm,
                              const float *__restrict__ w, int64_t n, int D, int DP, int stride, int depth,
                              const double *__restrict__ center, const Ingest *__restrict__ ing, float *rec) {
    const double wmax = ing ? (double)__uint_as_float(ing->wmax_bits) : 1.0;
    const int64_t nl = 1ll << depth;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        float *o = rec + p * stride;
        const int64_t leaf = nl - 1 + node_of(p, depth, n);
        for (int d = 0; d < DP; ++d) {
            float v = 0.f;
            if (d < D) {
                if (sizeof(T) == 8)
                    v = (float)((double)xs[p * D + d] - center[leaf * D + d]);
                else
                    v = (float)xs[p * D + d];
            }
            o[d] = v;
        }
        o[DP] = w ? (float)log2((double)w[perm[p]] / wmax) : 0.f;
        for (int d = DP + 1; d < stride; ++d) o[d] = 0.f;
    }
}

// --------------------------------------------------------------------------
// moments: M_alpha = sum_r w_r (x_r - c)^alpha / alpha!  (bandwidth-free
// Hermite moments; A_alpha = M_alpha s^-|alpha|).  Leaves directly, internal
// nodes by H2H (Lemma 2), exact at finite order.
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_leaf_moments(const T *__restrict__ xs, const int32_t *__restrict__ perm,
                               const float *__restrict__ w, int64_t n, int D, int depth,
                               const double *__restrict__ center, SeriesTables tb, double *mom) {
    extern __shared__ double smem[];
    const int64_t nl = 1ll << depth;
    const int64_t i = blockIdx.x;
    if (i >= nl) return;
    const int64_t node = nl - 1 + i;
    const int64_t b = level_begin(n, depth, i), e = level_begin(n, depth, i + 1);
    const int cnt = (int)(e - b);
    double *df = smem;               // cnt x D
    double *ws = smem + cnt * D;     // cnt
    for (int t = threadIdx.x; t < cnt * D; t += blockDim.x) {
        const int r = t / D, d = t % D;
        df[t] = (double)xs[(b + r) * D + d] - center[node * D + d];
    }
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) ws[t] = (double)w[perm[b + t]];
    __syncthreads();
    for (int a = threadIdx.x; a < tb.T; a += blockDim.x) {
        const uint8_t *al = tb.alpha + a * D;
        double acc = 0.0;
        for (int r = 0; r < cnt; ++r) {
            double m = ws[r];
            for (int d = 0; d < D; ++d)
                for (int q = 0; q < al[d]; ++q) m *= df[r * D + d];
            acc += m;
        }
        mom[node * tb.T + a] = acc * tb.inv_fact[a];
    }
}

__global__ void k_h2h_moments(int D, int k, const double *__restrict__ center, SeriesTables tb, double *mom) {
    extern __shared__ double smem[];
    const int64_t nn = 1ll << k;
    const int64_t i = blockIdx.x;
    if (i >= nn) return;
    const int64_t node = nn - 1 + i;
    double *P = smem;   // 2 x T: Delta_c^beta / beta! for both children
    for (int c = 0; c < 2; ++c) {
        const int64_t ch = 2 * node + 1 + c;
        for (int bt = threadIdx.x; bt < tb.T; bt += blockDim.x) {
            const uint8_t *be = tb.alpha + bt * D;
            double m = tb.inv_fact[bt];
            for (int d = 0; d < D; ++d) {
                const double dl = center[ch * D + d] - center[node * D + d];
                for (int q = 0; q < be[d]; ++q) m *= dl;
            }
            P[c * tb.T + bt] = m;
        }
    }
    __syncthreads();
    const int64_t l = 2 * node + 1, r = 2 * node + 2;
    for (int g = threadIdx.x; g < tb.T; g += blockDim.x) {
        double acc = 0.0;
        for (int e = tb.h2h_off[g]; e < tb.h2h_off[g + 1]; ++e) {
            const int a = tb.h2h_pairs[2 * e], bt = tb.h2h_pairs[2 * e + 1];
            acc += mom[l * tb.T + a] * P[bt] + mom[r * tb.T + a] * P[tb.T + bt];
        }
        mom[node * tb.T + g] = acc;
    }
}

// --------------------------------------------------------------------------
// host: multi-index tables
// --------------------------------------------------------------------------
static void enum_layer(int deg, int D, std::vector<int> &cur, std::vector<std::vector<int>> &out) {
    if ((int)cur.size() == D - 1) {
        cur.push_back(deg);
        out.push_back(cur);
        cur.pop_back();
        return;
    }
    for (int a = deg; a >= 0; --a) {
        cur.push_back(a);
        enum_layer(deg - a, D, cur, out);
        cur.pop_back();
    }
}

static int make_series_tables(int D, int P, SeriesTables *tb) {
    std::vector<std::vector<int>> al;
    for (int deg = 0; deg < P; ++deg) {
        std::vector<int> cur;
        enum_layer(deg, D, cur, al);
    }
    const int T = (int)al.size();
    if (T > 8192) {
        set_error("series order P=%d in D=%d needs %d terms (limit 8192)", P, D, T);
        return GS_ERR_ARG;
    }
    std::map<std::vector<int>, int> index;
    for (int i = 0; i < T; ++i) index[al[i]] = i;
    SeriesTables h;
    h.D = D;
    h.P = P;
    h.T = T;
    for (int p = 0; p <= 16; ++p) h.Tp[p] = 0;
    for (int i = 0; i < T; ++i) {
        int dg = 0;
        for (int v : al[i]) dg += v;
        for (int p = dg + 1; p <= 16; ++p) h.Tp[p]++;
    }
    std::vector<uint8_t> alpha(T * D), deg(T), pdim(T);
    std::vector<int32_t> pred(T), dpred(T);
    std::vector<double> invf(T);
    std::vector<int32_t> hoff(T + 1), hp;
    std::vector<int32_t> snext((size_t)D * T, -1), sline((size_t)D * T, 0), snl((size_t)D * 17, 0);
    auto fact = [](int m) { double f = 1.0; for (int q = 2; q <= m; ++q) f *= q; return f; };
    for (int i = 0; i < T; ++i) {
        int dg = 0, last = -1;
        double f = 1.0;
        for (int d = 0; d < D; ++d) {
            alpha[i * D + d] = (uint8_t)al[i][d];
            dg += al[i][d];
            f *= fact(al[i][d]);
            if (al[i][d] > 0) last = d;
        }
        deg[i] = (uint8_t)dg;
        invf[i] = 1.0 / f;
        if (last < 0) {
            pred[i] = -1;
            dpred[i] = -1;
            pdim[i] = 0;
        } else {
            std::vector<int> b = al[i];
            b[last] = 0;
            pred[i] = index[b];
            std::vector<int> c = al[i];
            c[last] -= 1;
            dpred[i] = index[c];
            pdim[i] = (uint8_t)last;
        }
    }
    for (int g = 0; g < T; ++g) {
        hoff[g] = (int32_t)(hp.size() / 2);
        for (int a = 0; a < T; ++a) {
            bool le = true;
            std::vector<int> b(D);
            for (int d = 0; d < D; ++d) {
                if (al[a][d] > al[g][d]) le = false;
                b[d] = al[g][d] - al[a][d];
            }
            if (!le) continue;
            hp.push_back(a);
            hp.push_back(index[b]);
        }
    }
    hoff[T] = (int32_t)(hp.size() / 2);
    // separable L2L: successor along each dimension and the line starts
    for (int d = 0; d < D; ++d) {
        int n = 0;
        for (int a = 0; a < T; ++a) {
            if ((int)deg[a] + 1 < P) {
                std::vector<int> b = al[a];
                b[d] += 1;
                snext[(size_t)d * T + a] = index[b];
            }
            if (al[a][d] == 0) {
                sline[(size_t)d * T + n++] = a;
                for (int p = deg[a] + 1; p <= 16; ++p) snl[d * 17 + p]++;
            }
        }
    }
    // one device allocation, 8-byte aligned sections
    auto al8 = [](size_t b) { return (b + 7) & ~(size_t)7; };
    size_t o_alpha = 0, o_deg = al8(o_alpha + alpha.size()), o_pdim = al8(o_deg + T), o_pred = al8(o_pdim + T);
    size_t o_invf = al8(o_pred + 4 * T), o_hoff = al8(o_invf + 8 * T), o_hp = al8(o_hoff + 4 * (T + 1));
    size_t o_snext = al8(o_hp + 4 * hp.size()), o_sline = al8(o_snext + 4 * snext.size());
    size_t o_snl = al8(o_sline + 4 * sline.size());
    size_t o_dpred = al8(o_snl + 4 * snl.size());
    size_t total = al8(o_dpred + 4 * T);
    std::vector<uint8_t> host(total, 0);
    memcpy(&host[o_alpha], alpha.data(), alpha.size());
    memcpy(&host[o_deg], deg.data(), T);
    memcpy(&host[o_pdim], pdim.data(), T);
    memcpy(&host[o_pred], pred.data(), 4 * T);
    memcpy(&host[o_invf], invf.data(), 8 * T);
    memcpy(&host[o_hoff], hoff.data(), 4 * (T + 1));
    if (!hp.empty()) memcpy(&host[o_hp], hp.data(), 4 * hp.size());
    memcpy(&host[o_snext], snext.data(), 4 * snext.size());
    memcpy(&host[o_sline], sline.data(), 4 * sline.size());
    memcpy(&host[o_snl], snl.data(), 4 * snl.size());
    memcpy(&host[o_dpred], dpred.data(), 4 * T);
    uint8_t *dm = nullptr;
    GS_CUDA_TRY(cudaMalloc((void **)&dm, total));   // cached for the life of the process
    cudaError_t e = cudaMemcpy(dm, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dm);
        return cuda_fail(e, "series tables upload");
    }
    h.mem = dm;
    h.alpha = dm + o_alpha;
    h.deg = dm + o_deg;
    h.pred_dim = dm + o_pdim;
    h.pred = (int32_t *)(dm + o_pred);
    h.inv_fact = (double *)(dm + o_invf);
    h.h2h_off = (int32_t *)(dm + o_hoff);
    h.h2h_pairs = (int32_t *)(dm + o_hp);
    h.l2s_next = (int32_t *)(dm + o_snext);
    h.l2s_line = (int32_t *)(dm + o_sline);
    h.l2s_nlines = (int32_t *)(dm + o_snl);
    h.dpred = (int32_t *)(dm + o_dpred);
    *tb = h;
    return GS_OK;
}

// Tables depend only on (device, D, P): built once and kept for the process.
static std::map<std::tuple<int, int, int>, SeriesTables> g_tables;
static std::mutex g_tables_mu;

int build_series_tables(int D, int P, SeriesTables *tb, cudaStream_t st) {
    (void)st;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tables_mu);
    auto key = std::make_tuple(dev, D, P);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
        *tb = it->second;
        return GS_OK;
    }
    SeriesTables t;
    int rc = make_series_tables(D, P, &t);
    if (rc) return rc;
    g_tables[key] = t;
    *tb = t;
    return GS_OK;
}

void free_series_tables(SeriesTables *tb, cudaStream_t st) {
    (void)st;
    *tb = SeriesTables();   // the cached device copy stays alive
}

// --------------------------------------------------------------------------
// host: build
// --------------------------------------------------------------------------
static int tree_depth_for(int64_t n, int L) {
    int d = 0;
    while ((n + (1ll << d) - 1) >> d > L) ++d;
    return d;
}

static int gridn(int64_t n, int t = kTB, int cap = 8192) {
    int64_t b = (n + t - 1) / t;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__global__ void k_iota(int32_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}
static void launch_iota(int32_t *p, int64_t n, cudaStream_t st) { k_iota<<<gridn(n), kTB, 0, st>>>(p, n); }

template <typename T>
static int build_impl(const T *x, const float *w, int64_t n, int D, int L, const Ingest *ing, int DP,
                      int rec_stride, bool with_weights, CallCtx &cx, TreeDev *out) {
    using K = typename Key<T>::K;
    cudaStream_t st = cx.st;
    TreeDev t;
    t.n = n;
    t.D = D;
    t.depth = tree_depth_for(n, L);
    t.nodes = (2ll << t.depth) - 1;
    t.dtype = sizeof(T) == 8 ? GS_F64 : GS_F32;
    const int64_t nodes = t.nodes;
    const int64_t maxlev = t.depth > 0 ? (1ll << (t.depth - 1)) : 1;
    T *xa = nullptr, *xb = nullptr;
    int32_t *pa = nullptr, *pb = nullptr;
    K *bmin = nullptr, *bmax = nullptr;
    SelState<K> *sel = nullptr;
    uint32_t *hist = nullptr;
    unsigned long long *partial = nullptr, *S = nullptr;
    // on any early return: free the scratch and whatever of the tree exists
    struct Guard {
        cudaStream_t st;
        TreeDev *t;
        void **ptrs[10];
        bool ok = false;
        ~Guard() {
            if (ok) return;
            for (void **pp : ptrs)
                if (*pp) cudaFreeAsync(*pp, st);
            free_tree(*t, st);
        }
    } guard{st, &t, {(void **)&xa, (void **)&xb, (void **)&pa, (void **)&pb, (void **)&bmin, (void **)&bmax,
                     (void **)&sel, (void **)&hist, (void **)&partial, (void **)&S}};
    GS_CUDA_TRY(dev_malloc_async((void **)&xa, n * D * sizeof(T), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&xb, n * D * sizeof(T), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&pa, n * sizeof(int32_t), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&pb, n * sizeof(int32_t), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&bmin, maxlev * D * sizeof(K), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&bmax, maxlev * D * sizeof(K), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&sel, maxlev * sizeof(SelState<K>), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&hist, maxlev * 256 * sizeof(uint32_t), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&partial, kScanGrid * sizeof(unsigned long long), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&S, n * sizeof(unsigned long long), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.lo, nodes * D * sizeof(double), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.hi, nodes * D * sizeof(double), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.center, nodes * D * sizeof(double), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.lo32, nodes * D * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.hi32, nodes * D * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.rad, nodes * sizeof(double), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.rad32, nodes * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.W32d, nodes * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.W32u, nodes * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.W, nodes * sizeof(double), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.wmin, nodes * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.split_dim, nodes * sizeof(int32_t), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&t.rec, n * rec_stride * sizeof(float), st));
    GS_CUDA_TRY(cudaMemcpyAsync(xa, x, n * D * sizeof(T), cudaMemcpyDeviceToDevice, st));
    GS_CUDA_TRY(cudaMemsetAsync(t.split_dim, 0xff, nodes * sizeof(int32_t), st));
    launch_iota(pa, n, st);
    cx.launches += 1;

    for (int k = 0; k < t.depth; ++k) {
        const int64_t nn = 1ll << k;
        if (((n + nn - 1) >> k) <= kNodeFused) {
            // every node of this level has at most kNodeFused points: one launch
            const int64_t seg = (n + nn - 1) >> k;   // the largest node of the level
            const size_t sm = (size_t)seg * sizeof(K);
            if (seg > 2048) {
                GS_CUDA_TRY(allow_max_smem((const void *)k_level_node<T, 1024>));
                k_level_node<T, 1024><<<(unsigned)nn, 1024, sm, st>>>(xa, pa, n, D, k, t.split_dim, xb, pb,
                                                                      (unsigned *)&ing->status);
            } else {
                k_level_node<T, 256><<<(unsigned)nn, 256, sm, st>>>(xa, pa, n, D, k, t.split_dim, xb, pb,
                                                                    (unsigned *)&ing->status);
            }
            cx.launches += 1;
            if (int rc = cx.check("tree level (per node)")) return rc;
            T *tx = xa; xa = xb; xb = tx;
            int32_t *tp = pa; pa = pb; pb = tp;
            continue;
        }
        GS_CUDA_TRY(cudaMemsetAsync(bmin, 0xff, nn * D * sizeof(K), st));
        GS_CUDA_TRY(cudaMemsetAsync(bmax, 0x00, nn * D * sizeof(K), st));
        k_level_bbox<T><<<gridn(n), kTB, 0, st>>>(xa, n, D, k, bmin, bmax);
        k_level_select_dim<T><<<gridn(nn), kTB, 0, st>>>(n, D, k, bmin, bmax, t.split_dim, sel);
        cx.launches += 2;
        for (int shift = Key<T>::BITS - 8; shift >= 0; shift -= 8) {
            GS_CUDA_TRY(cudaMemsetAsync(hist, 0, nn * 256 * sizeof(uint32_t), st));
            k_level_hist<T><<<(unsigned)((n + kHistChunk - 1) / kHistChunk), kTB, 0, st>>>(xa, n, D, k, shift, sel, hist);
            k_level_pick<K><<<gridn(nn * 32), kTB, 0, st>>>(k, shift, hist, sel);
            cx.launches += 2;
        }
        k_part_sum<T><<<kScanGrid, kTB, 0, st>>>(xa, n, D, k, sel, partial);
        k_scan_partials_u64<<<1, kTB, 0, st>>>(partial, kScanGrid);
        k_part_prefix<T><<<kScanGrid, kTB, 0, st>>>(xa, n, D, k, sel, partial, S);
        k_part_scatter<T><<<gridn(n), kTB, 0, st>>>(xa, pa, n, D, k, sel, S, xb, pb, (unsigned *)&ing->status);
        cx.launches += 4;
        if (int rc = cx.check("tree level")) return rc;
        T *tx = xa; xa = xb; xb = tx;
        int32_t *tp = pa; pa = pb; pb = tp;
    }
    k_leaf_stats<T><<<gridn(1ll << t.depth), kTB, 0, st>>>(xa, pa, w, n, D, t.depth, t.lo, t.hi, t.W, t.wmin);
    cx.launches += 1;
    if (t.depth <= 12) {
        k_internal_stats_all<<<1, 1024, 0, st>>>(D, t.depth, t.lo, t.hi, t.W, t.wmin);
        cx.launches += 1;
    } else {
        for (int k = t.depth - 1; k >= 0; --k) {
            k_internal_stats<<<gridn(1ll << k), kTB, 0, st>>>(D, k, t.lo, t.hi, t.W, t.wmin);
            cx.launches += 1;
        }
    }
    k_center_rad<<<gridn(nodes), kTB, 0, st>>>(nodes, D, t.lo, t.hi, t.center, t.rad, t.rad32, t.lo32, t.hi32, t.W, t.W32d, t.W32u);
    k_pack_sorted<T><<<gridn(n), kTB, 0, st>>>(xa, pa, with_weights ? w : nullptr, n, D, DP, rec_stride, t.depth,
                                               t.center, ing, t.rec);
    cx.launches += 2;
    t.rec_stride = rec_stride;
    t.perm = pa;   // now owned by the tree
    t.xs = xa;
    xa = nullptr;
    pa = nullptr;
    for (void **pp : guard.ptrs)
        if (*pp) {
            cudaFreeAsync(*pp, st);
            *pp = nullptr;
        }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tree build launch");
    guard.ok = true;
    *out = t;
    return GS_OK;
}

int build_tree(const void *x, const float *w, int64_t n, int D, int dtype, int L, const Ingest *ing, int DP,
               int rec_stride, bool with_weights, CallCtx &cx, TreeDev *out) {
    if (n >= (1ll << 31)) {
        set_error("n=%lld exceeds 2^31 - 1 points", (long long)n);
        return GS_ERR_ARG;
    }
    if (dtype == GS_F64)
        return build_impl<double>((const double *)x, w, n, D, L, ing, DP, rec_stride, with_weights, cx, out);
    return build_impl<float>((const float *)x, w, n, D, L, ing, DP, rec_stride, with_weights, cx, out);
}

int build_moments(TreeDev &t, const float *w, const SeriesTables &tb, CallCtx &cx) {
    cudaStream_t st = cx.st;
    GS_CUDA_TRY(dev_malloc_async((void **)&t.moments, t.nodes * tb.T * sizeof(double), st));
    t.mom_terms = tb.T;
    const int64_t nl = 1ll << t.depth;
    const int64_t maxcnt = (t.n + nl - 1) / nl;
    const size_t sm = (size_t)maxcnt * (t.D + 1) * sizeof(double);
    if (sm > 200 * 1024) {
        set_error("leaf too large for the moment kernel");
        return GS_ERR_ARG;
    }
    if (sm > 48 * 1024) {
        if (t.dtype == GS_F64)
            allow_max_smem((const void *)k_leaf_moments<double>);
        else
            allow_max_smem((const void *)k_leaf_moments<float>);
    }
    if (t.dtype == GS_F64)
        k_leaf_moments<double><<<(unsigned)nl, 128, sm, st>>>((const double *)t.xs, t.perm, w, t.n, t.D, t.depth,
                                                              t.center, tb, t.moments);
    else
        k_leaf_moments<float><<<(unsigned)nl, 128, sm, st>>>((const float *)t.xs, t.perm, w, t.n, t.D, t.depth,
                                                             t.center, tb, t.moments);
    cx.launches += 1;
    const size_t sm2 = 2 * (size_t)tb.T * sizeof(double);
    if (sm2 > 48 * 1024) allow_max_smem((const void *)k_h2h_moments);
    for (int k = t.depth - 1; k >= 0; --k) {
        k_h2h_moments<<<(unsigned)(1ll << k), 128, sm2, st>>>(t.D, k, t.center, tb, t.moments);
        cx.launches += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
    if (int rc = cx.check("moments")) return rc;
    return GS_OK;
}

void free_tree(TreeDev &t, cudaStream_t st) {
    void *ptrs[] = {t.perm, t.xs, t.lo, t.hi, t.center, t.rad, t.W, t.wmin, t.split_dim, t.rec, t.moments,
                    t.lo32, t.hi32, t.rad32, t.W32d, t.W32u};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, st);
    t = TreeDev();
}

}  // namespace gs
