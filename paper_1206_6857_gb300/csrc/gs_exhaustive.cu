// Input checks, reference packing and the exhaustive Gaussian sum.
//
// The exhaustive sum is the plain definition of Section 1,
//     G(x_q; h_j) = sum_r w_r exp(-||x_q - x_r||^2 / (2 h_j^2)),
// evaluated for every (query, reference, bandwidth).  It is the dual-tree
// method's comparison point ("Naive" in the Section 7 tables) and its
// exhaustive (eps = 0) mode.
//
// Arithmetic: the squared distance is formed in FP32 from coordinate
// differences (FP64 differences rounded to FP32 when the input is FP64), the
// weight is folded into the exponent as l_r = log2(w_r / w_max), and each
// term is 2^(d^2 * (-log2(e) / 2h^2) + l_r) on the MUFU ex2 unit.  Terms are
// summed in FP32 over runs of 64 references and the runs in FP64 per query;
// w_max is multiplied back at the end.
//
// Layout: references are repacked once into 16-byte-aligned records
// (coordinates, l_r) padded to a whole number of shared-memory tiles with
// l = -inf records; CTAs stage one tile at a time in shared memory and every
// thread reads each record as a broadcast, holding QPT queries and NJ
// bandwidths in registers.  A 3-D grid spans query blocks x reference splits
// x bandwidth chunks; splits are chosen so the grid covers every SM several
// times even when M is small, and then accumulate with FP64 atomics.
#include <algorithm>
#include <utility>
#include <vector>

#include <math.h>
#include <stdarg.h>
#include <string.h>
#include <stdio.h>

#include "gs_device.cuh"
#include "gs_internal.h"

namespace gs {

// --------------------------------------------------------------------------
// Ingest: finiteness, positivity, weight range
// --------------------------------------------------------------------------
__global__ void k_ingest_reset(Ingest *ing) {
    ing->status = 0;
    ing->wmax_bits = 0;
    ing->wmin_bits = 0x7f800000u;
    ing->pad = 0;
    ing->wsum = 0.0;
}

template <typename T>
__global__ void k_ingest_points(const T *__restrict__ x, int64_t n, Ingest *ing) {
    unsigned bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite((double)x[i])) bad = ST_NONFINITE;
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(&ing->status, bad);
}

__global__ void k_ingest_weights(const float *__restrict__ w, int64_t n, Ingest *ing) {
    unsigned bad = 0;
    float wmax = 0.f, wmin = INFINITY;
    double wsum = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float wi = w[i];
        if (!isfinite(wi)) {
            bad |= ST_NONFINITE;
        } else if (!(wi > 0.f)) {
            bad |= ST_WEIGHT;
        } else {
            wmax = fmaxf(wmax, wi);
            wmin = fminf(wmin, wi);
            wsum += wi;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    for (int o = 16; o > 0; o >>= 1) {
        wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
        wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&ing->status, bad);
        atomicMax(&ing->wmax_bits, __float_as_uint(wmax));
        atomicMin(&ing->wmin_bits, __float_as_uint(wmin));
        atomicAdd(&ing->wsum, wsum);
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_ingest(Ingest *ing, const void *queries, int64_t M, const void *refs,
                          const float *weights, int64_t N, int D, int dtype, CallCtx &cx) {
    cudaStream_t st = cx.st;
    cx.launches += 3 + (queries != refs);
    k_ingest_reset<<<1, 1, 0, st>>>(ing);
    const int64_t nq = M * D, nr = N * D;
    if (dtype == GS_F64) {
        k_ingest_points<double><<<grid_for(nr, 256), 256, 0, st>>>((const double *)refs, nr, ing);
        if (queries != refs)
            k_ingest_points<double><<<grid_for(nq, 256), 256, 0, st>>>((const double *)queries, nq, ing);
    } else {
        k_ingest_points<float><<<grid_for(nr, 256), 256, 0, st>>>((const float *)refs, nr, ing);
        if (queries != refs)
            k_ingest_points<float><<<grid_for(nq, 256), 256, 0, st>>>((const float *)queries, nq, ing);
    }
    if (weights) k_ingest_weights<<<grid_for(N, 256), 256, 0, st>>>(weights, N, ing);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Reference packing
// --------------------------------------------------------------------------
template <typename T, int DP>
__global__ void k_pack_refs(const T *__restrict__ x, const float *__restrict__ w, int64_t N,
                            int64_t Npad, int D, const Ingest *__restrict__ ing, T *__restrict__ rec) {
    constexpr int NT = RefRec<T, DP>::NT;
    const double wmax = (double)__uint_as_float(ing->wmax_bits);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Npad;
         i += (int64_t)gridDim.x * blockDim.x) {
        T *o = rec + i * NT;
        if (i < N) {
            for (int d = 0; d < DP; ++d) o[d] = d < D ? x[i * D + d] : (T)0;
            o[DP] = (T)log2((double)w[i] / wmax);
        } else {
            for (int d = 0; d < DP; ++d) o[d] = (T)0;
            o[DP] = (T)(-INFINITY);
        }
        for (int k = DP + 1; k < NT; ++k) o[k] = (T)0;
    }
}

// --------------------------------------------------------------------------
// Exhaustive kernel
// --------------------------------------------------------------------------
struct NegC {
    float v[64];   // -log2(e) / (2 h_j^2), j < nh
};

constexpr int kThreads = 256;   // three blocks per SM (at most 80 registers a thread)
constexpr int kRun = 64;   // references per FP32 partial sum

template <typename T, int DP>
struct TileCfg {
    static constexpr int NT = RefRec<T, DP>::NT;
    static constexpr int TILE = (NT * sizeof(T) <= 64) ? 128 : 64;
    // FP32 records of at most 8 dimensions are staged with every float
    // twice, for the packed path (two queries per f32x2 operation)
    static constexpr bool X2 = sizeof(T) == 4 && DP <= 8;
    static constexpr int SMEM = TILE * NT * (X2 ? 2 : 1);   // staged T slots
};

template <typename T, int NT>
__device__ __forceinline__ void load_rec(const T *p, T (&v)[NT]) {
    if constexpr (sizeof(T) == 4) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int k = 0; k < NT / 4; ++k) {
            float4 f = p4[k];
            v[4 * k] = f.x; v[4 * k + 1] = f.y; v[4 * k + 2] = f.z; v[4 * k + 3] = f.w;
        }
    } else {
        const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int k = 0; k < NT / 2; ++k) {
            double2 f = p2[k];
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
}

// One tile of the exhaustive sum: query block bx (kThreads * QPT queries),
// reference range [by * chunk, (by + 1) * chunk) of the packed records, the NJ
// bandwidths starting at bz * NJ (nc: their -log2(e) / 2h^2, 0 beyond nh).
template <typename T, int DP, int NJ, int QPT>
__device__ __forceinline__ void exhaustive_tile(const T *__restrict__ qx, int64_t M, int D, const T *__restrict__ rec,
                                                int64_t chunk, int64_t Npad, const float (&nc)[NJ], int nh,
                                                const Ingest *__restrict__ ing, double *__restrict__ out, int atomic,
                                                int64_t bx, int64_t by, int bz, T *tile) {
    using Cfg = TileCfg<T, DP>;
    constexpr int NT = Cfg::NT, TILE = Cfg::TILE;
    const int j0 = bz * NJ;

    T xq[QPT][DP];
    int64_t qi[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        qi[k] = bx * (kThreads * QPT) + k * kThreads + threadIdx.x;
        const int64_t qs = qi[k] < M ? qi[k] : M - 1;
#pragma unroll
        for (int d = 0; d < DP; ++d) xq[k][d] = d < D ? qx[qs * D + d] : (T)0;
    }

    double acc[QPT][NJ];
#pragma unroll
    for (int k = 0; k < QPT; ++k)
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) acc[k][jj] = 0.0;

    const int64_t r0 = by * chunk;
    const int64_t r1 = min(r0 + chunk, Npad);
    if constexpr (Cfg::X2) {
        static_assert(QPT == 2, "the packed path takes two queries per thread");
        // Two queries per register pair: the same FP32 operations as the
        // scalar loop below, element by element (so the same sums), with
        // one f32x2 instruction for both queries' differences, squared
        // distances, exponent arguments and partial sums.
        f2_t xq2[DP], nc2[NJ];
#pragma unroll
        for (int d = 0; d < DP; ++d) xq2[d] = f2_pack(xq[0][d], xq[1][d]);
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) nc2[jj] = f2_pack(nc[jj], nc[jj]);
        for (int64_t t0 = r0; t0 < r1; t0 += TILE) {
            __syncthreads();
            {
                // records staged as (x_0, x_0, x_1, x_1, ..., l, l, ...)
                const float4 *src = reinterpret_cast<const float4 *>(rec + t0 * NT);
                float4 *dst = reinterpret_cast<float4 *>(tile);
                constexpr int NV = TILE * NT / 4;
                for (int v = threadIdx.x; v < NV; v += kThreads) {
                    const float4 f = src[v];
                    dst[2 * v] = make_float4(f.x, f.x, f.y, f.y);
                    dst[2 * v + 1] = make_float4(f.z, f.z, f.w, f.w);
                }
            }
            __syncthreads();
            const ulonglong2 *tp = reinterpret_cast<const ulonglong2 *>(tile);
#pragma unroll 1
            for (int rr0 = 0; rr0 < TILE; rr0 += kRun) {
                f2_t part[NJ];
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) part[jj] = 0ull;
#pragma unroll 4
                for (int rr = rr0; rr < rr0 + kRun; ++rr) {
                    f2_t rv[NT];
#pragma unroll
                    for (int v = 0; v < NT / 2; ++v) {
                        const ulonglong2 u = tp[rr * (NT / 2) + v];
                        rv[2 * v] = u.x;
                        rv[2 * v + 1] = u.y;
                    }
                    f2_t d2 = 0ull;
#pragma unroll
                    for (int d = 0; d < DP; ++d) {
                        const f2_t df = f2_sub(xq2[d], rv[d]);
                        d2 = f2_fma(df, df, d2);
                    }
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        float a0, a1;
                        f2_unpack(f2_fma(d2, nc2[jj], rv[DP]), a0, a1);
                        part[jj] = f2_add(part[jj], f2_pack(ex2_approx(a0), ex2_approx(a1)));
                    }
                }
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    float p0, p1;
                    f2_unpack(part[jj], p0, p1);
                    acc[0][jj] += (double)p0;
                    acc[1][jj] += (double)p1;
                }
            }
        }
    } else {
        for (int64_t t0 = r0; t0 < r1; t0 += TILE) {
            __syncthreads();
            {
                // TILE*NT elements of T = TILE*NT*sizeof(T)/16 vectors of 16 bytes
                const float4 *src = reinterpret_cast<const float4 *>(rec + t0 * NT);
                float4 *dst = reinterpret_cast<float4 *>(tile);
                constexpr int NV = TILE * NT * (int)sizeof(T) / 16;
                for (int v = threadIdx.x; v < NV; v += kThreads) dst[v] = src[v];
            }
            __syncthreads();
    #pragma unroll 1
            for (int rr0 = 0; rr0 < TILE; rr0 += kRun) {
                float part[QPT][NJ];
    #pragma unroll
                for (int k = 0; k < QPT; ++k)
    #pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) part[k][jj] = 0.f;
    #pragma unroll 4
                for (int rr = rr0; rr < rr0 + kRun; ++rr) {
                    T rv[NT];
                    load_rec<T, NT>(tile + rr * NT, rv);
                    const float l = (float)rv[DP];
    #pragma unroll
                    for (int k = 0; k < QPT; ++k) {
                        float d2 = 0.f;
    #pragma unroll
                        for (int d = 0; d < DP; ++d) {
                            const float df = (float)(xq[k][d] - rv[d]);
                            d2 = fmaf(df, df, d2);
                        }
    #pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) part[k][jj] += ex2_approx(fmaf(d2, nc[jj], l));
                    }
                }
    #pragma unroll
                for (int k = 0; k < QPT; ++k)
    #pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) acc[k][jj] += (double)part[k][jj];
            }
        }
    }

    const double wmax = (double)__uint_as_float(ing->wmax_bits);
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
        if (qi[k] >= M) continue;
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            const int j = j0 + jj;
            if (j >= nh) continue;
            const double v = acc[k][jj] * wmax;
            if (atomic)
                atomicAdd(out + qi[k] * nh + j, v);
            else
                out[qi[k] * nh + j] = v;
        }
    }
}

template <typename T, int DP, int NJ, int QPT>
__global__ void __launch_bounds__(kThreads, 3)
k_exhaustive(const T *__restrict__ qx, int64_t M, int D, const T *__restrict__ rec,
             int64_t chunk, int64_t Npad, NegC negc, int nh, const Ingest *__restrict__ ing,
             double *__restrict__ out, int atomic) {
    using Cfg = TileCfg<T, DP>;
    __shared__ __align__(16) T tile[Cfg::SMEM];
    const int j0 = blockIdx.z * NJ;
    float nc[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) nc[jj] = (j0 + jj < nh) ? negc.v[j0 + jj] : 0.f;
    exhaustive_tile<T, DP, NJ, QPT>(qx, M, D, rec, chunk, Npad, nc, nh, ing, out, atomic, blockIdx.x, blockIdx.y,
                                    blockIdx.z, tile);
}

static int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <typename T, int DP, int NJ>
static int run_exhaustive(const void *queries, int64_t M, const void *refs, const float *weights,
                          int64_t N, int D, const double *h, int nh, const Ingest *ing,
                          double *out, CallCtx &cx) {
    cudaStream_t st = cx.st;
    using Cfg = TileCfg<T, DP>;
    constexpr int NT = Cfg::NT, TILE = Cfg::TILE;
    constexpr int QPT = (DP <= 8) ? 2 : 1;
    const int64_t Npad = (N + TILE - 1) / TILE * TILE;
    T *rec = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&rec, (size_t)Npad * NT * sizeof(T), st));
    k_pack_refs<T, DP><<<grid_for(Npad, 256), 256, 0, st>>>((const T *)refs, weights, N, Npad, D,
                                                              ing, rec);
    cx.launches += 1;
    NegC nc;
    for (int j = 0; j < 64; ++j) nc.v[j] = 0.f;
    for (int j = 0; j < nh; ++j) nc.v[j] = (float)(-1.4426950408889634 / (2.0 * h[j] * h[j]));

    const int64_t bx = (M + kThreads * QPT - 1) / (kThreads * QPT);
    const int nz = (nh + NJ - 1) / NJ;
    const int64_t tiles = Npad / TILE;
    const int64_t target = (int64_t)num_sms() * 8;
    int64_t splits = (target + bx * nz - 1) / (bx * nz);
    if (splits < 1) splits = 1;
    if (splits > tiles) splits = tiles;
    if (splits > 65535) splits = 65535;
    const int64_t chunk = (tiles + splits - 1) / splits * TILE;
    splits = (Npad + chunk - 1) / chunk;
    if (bx > 2147483647LL) {
        cudaFreeAsync(rec, st);
        set_error("too many queries for one launch");
        return GS_ERR_ARG;
    }
    if (splits > 1) GS_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)M * nh * sizeof(double), st));
    dim3 grid((unsigned)bx, (unsigned)splits, (unsigned)nz);
    cx.phase(GS_PH_BASE);
    k_exhaustive<T, DP, NJ, QPT><<<grid, kThreads, 0, st>>>((const T *)queries, M, D, rec, chunk,
                                                           Npad, nc, nh, ing, out, splits > 1);
    cx.launches += 1;
    cx.launches_base += 1;
    cx.phase(GS_PH_OTHER);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(rec, st);
    if (e != cudaSuccess) return cuda_fail(e, "k_exhaustive launch");
    return GS_OK;
}

template <typename T, int DP>
static int dispatch_nj(const void *q, int64_t M, const void *r, const float *w, int64_t N, int D,
                       const double *h, int nh, const Ingest *ing, double *out, CallCtx &st) {
    if (nh <= 1) return run_exhaustive<T, DP, 1>(q, M, r, w, N, D, h, nh, ing, out, st);
    if (nh <= 2) return run_exhaustive<T, DP, 2>(q, M, r, w, N, D, h, nh, ing, out, st);
    if (nh <= 4) return run_exhaustive<T, DP, 4>(q, M, r, w, N, D, h, nh, ing, out, st);
    return run_exhaustive<T, DP, 8>(q, M, r, w, N, D, h, nh, ing, out, st);
}

template <typename T>
static int dispatch_d(const void *q, int64_t M, const void *r, const float *w, int64_t N, int D,
                      const double *h, int nh, const Ingest *ing, double *out, CallCtx &st) {
#define GS_CASE(DPV) \
    if (D <= DPV) return dispatch_nj<T, DPV>(q, M, r, w, N, D, h, nh, ing, out, st);
    GS_CASE(1) GS_CASE(2) GS_CASE(3) GS_CASE(4) GS_CASE(5) GS_CASE(6) GS_CASE(7) GS_CASE(8)
    GS_CASE(12) GS_CASE(16) GS_CASE(24) GS_CASE(32)
#undef GS_CASE
    set_error("D=%d exceeds 32", D);
    return GS_ERR_ARG;
}

int exhaustive_sum(const void *queries, int64_t M, const void *refs, const float *weights,
                   int64_t N, int D, int dtype, const double *h, int nh, const Ingest *ing,
                   double *out, CallCtx &st) {
    if (dtype == GS_F64)
        return dispatch_d<double>(queries, M, refs, weights, N, D, h, nh, ing, out, st);
    return dispatch_d<float>(queries, M, refs, weights, N, D, h, nh, ing, out, st);
}

// --------------------------------------------------------------------------
// Many small problems in one launch.  The problems of a batch that are summed
// exhaustively are grouped by dimension bucket and bandwidth-chunk size; a
// group runs as four launches whatever its size: reset and ingest of every
// problem's inputs, packing of every problem's references, then one
// exhaustive launch over the flattened (problem, query block, bandwidth
// chunk) tiles, largest problems first.  Each problem's references are
// covered by a single tile row (no reference splits), so outputs are written
// once, without atomics.
// --------------------------------------------------------------------------
struct GroupProb {
    const void *q, *r;
    const float *w;
    double *out;
    void *rec;          // packed references, Npad records
    Ingest *ing;
    int64_t M, N, Npad, bx;
    int D, nh, nz, pad;
    long long tile0;    // first flattened tile of this problem
    float negc[64];
};

__global__ void k_group_reset(GroupProb *gp, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        Ingest *g = gp[i].ing;
        g->status = 0;
        g->wmax_bits = 0;
        g->wmin_bits = 0x7f800000u;
        g->pad = 0;
        g->wsum = 0.0;
    }
}

// the checks of launch_ingest for problem blockIdx.y
__global__ void k_group_ingest(const GroupProb *__restrict__ gp) {
    const GroupProb &P = gp[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned bad = 0;
    const int64_t nr = P.N * P.D, nq = P.q != P.r ? P.M * P.D : 0;
    for (int64_t i = i0; i < nr; i += stride)
        if (!isfinite(((const float *)P.r)[i])) bad |= ST_NONFINITE;
    for (int64_t i = i0; i < nq; i += stride)
        if (!isfinite(((const float *)P.q)[i])) bad |= ST_NONFINITE;
    float wmax = 0.f, wmin = INFINITY;
    double wsum = 0.0;
    for (int64_t i = i0; i < P.N; i += stride) {
        const float wi = P.w[i];
        if (!isfinite(wi)) {
            bad |= ST_NONFINITE;
        } else if (!(wi > 0.f)) {
            bad |= ST_WEIGHT;
        } else {
            wmax = fmaxf(wmax, wi);
            wmin = fminf(wmin, wi);
            wsum += wi;
        }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    for (int o = 16; o > 0; o >>= 1) {
        wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
        wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&P.ing->status, bad);
        atomicMax(&P.ing->wmax_bits, __float_as_uint(wmax));
        atomicMin(&P.ing->wmin_bits, __float_as_uint(wmin));
        atomicAdd(&P.ing->wsum, wsum);
    }
}

template <int DP>
__global__ void k_group_pack(const GroupProb *__restrict__ gp) {
    const GroupProb &P = gp[blockIdx.y];
    constexpr int NT = RefRec<float, DP>::NT;
    const double wmax = (double)__uint_as_float(P.ing->wmax_bits);
    const float *x = (const float *)P.r;
    float *rec = (float *)P.rec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P.Npad;
         i += (int64_t)gridDim.x * blockDim.x) {
        float *o = rec + i * NT;
        if (i < P.N) {
            for (int d = 0; d < DP; ++d) o[d] = d < P.D ? x[i * P.D + d] : 0.f;
            o[DP] = (float)log2((double)P.w[i] / wmax);
        } else {
            for (int d = 0; d < DP; ++d) o[d] = 0.f;
            o[DP] = -INFINITY;
        }
        for (int k = DP + 1; k < NT; ++k) o[k] = 0.f;
    }
}

template <int DP, int NJ>
__global__ void __launch_bounds__(kThreads, 3) k_group_exhaustive(const GroupProb *__restrict__ gp, int nprob) {
    using Cfg = TileCfg<float, DP>;
    constexpr int QPT = (DP <= 8) ? 2 : 1;
    __shared__ __align__(16) float tile[Cfg::SMEM];
    const long long t = blockIdx.x;
    int lo = 0, hi = nprob - 1;   // the problem owning tile t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gp[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const GroupProb &P = gp[lo];
    const long long local = t - P.tile0;
    const int bz = (int)(local % P.nz);
    const int64_t bx = local / P.nz;
    float nc[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) nc[jj] = (bz * NJ + jj < P.nh) ? P.negc[bz * NJ + jj] : 0.f;
    exhaustive_tile<float, DP, NJ, QPT>((const float *)P.q, P.M, P.D, (const float *)P.rec, P.Npad, P.Npad, nc,
                                        P.nh, P.ing, P.out, 0, bx, 0, bz, tile);
}

template <int DP, int NJ>
static int launch_group(const gs_problem *probs, const std::vector<int> &ids, cudaStream_t st, void **block,
                        GroupProb **dgp_out, std::vector<GroupProb> &hgp, int64_t &launches) {
    using Cfg = TileCfg<float, DP>;
    constexpr int NT = Cfg::NT, TILE = Cfg::TILE, QPT = (DP <= 8) ? 2 : 1;
    const int n = (int)ids.size();
    hgp.assign(n, GroupProb());
    size_t rec_bytes = 0;
    long long tiles = 0;
    for (int k = 0; k < n; ++k) {
        const gs_problem &p = probs[ids[k]];
        GroupProb &g = hgp[k];
        memset(&g, 0, sizeof(g));
        g.q = p.queries;
        g.r = p.refs;
        g.w = p.weights;
        g.out = p.out;
        g.M = p.M;
        g.N = p.N;
        g.D = p.D;
        g.nh = p.nh;
        g.Npad = (p.N + TILE - 1) / TILE * TILE;
        g.bx = (p.M + kThreads * QPT - 1) / (kThreads * QPT);
        g.nz = (p.nh + NJ - 1) / NJ;
        g.tile0 = tiles;
        tiles += g.bx * g.nz;
        for (int j = 0; j < p.nh; ++j) g.negc[j] = (float)(-1.4426950408889634 / (2.0 * p.h[j] * p.h[j]));
        rec_bytes += (size_t)g.Npad * NT * sizeof(float);
    }
    if (tiles > 2147483647LL || n > 65535) {
        set_error("gs_sum_batched: exhaustive group too large for one launch");
        return GS_ERR_ARG;
    }
    const size_t head = ((n * sizeof(GroupProb) + 255) / 256) * 256;
    const size_t ings = ((n * sizeof(Ingest) + 255) / 256) * 256;
    GS_CUDA_TRY(dev_malloc_async(block, head + ings + rec_bytes, st));
    unsigned char *base = (unsigned char *)*block;
    size_t off = head + ings;
    for (int k = 0; k < n; ++k) {
        hgp[k].ing = (Ingest *)(base + head) + k;
        hgp[k].rec = base + off;
        off += (size_t)hgp[k].Npad * NT * sizeof(float);
    }
    GroupProb *dgp = (GroupProb *)base;
    GS_CUDA_TRY(cudaMemcpyAsync(dgp, hgp.data(), n * sizeof(GroupProb), cudaMemcpyHostToDevice, st));
    k_group_reset<<<(n + 127) / 128, 128, 0, st>>>(dgp, n);
    k_group_ingest<<<dim3(32, n), 256, 0, st>>>(dgp);
    k_group_pack<DP><<<dim3(32, n), 256, 0, st>>>(dgp);
    k_group_exhaustive<DP, NJ><<<(unsigned)tiles, kThreads, 0, st>>>(dgp, n);
    launches += 4;
    *dgp_out = dgp;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GS_OK : cuda_fail(e, "grouped exhaustive launch");
}

template <int DP>
static int launch_group_nj(int nj, const gs_problem *probs, const std::vector<int> &ids, cudaStream_t st,
                           void **block, GroupProb **dgp, std::vector<GroupProb> &hgp, int64_t &launches) {
    if (nj == 1) return launch_group<DP, 1>(probs, ids, st, block, dgp, hgp, launches);
    if (nj == 2) return launch_group<DP, 2>(probs, ids, st, block, dgp, hgp, launches);
    if (nj == 4) return launch_group<DP, 4>(probs, ids, st, block, dgp, hgp, launches);
    return launch_group<DP, 8>(probs, ids, st, block, dgp, hgp, launches);
}

bool exhaustive_groupable(const gs_problem &p) { return p.dtype == GS_F32 && p.D >= 1 && p.D <= 8; }

int exhaustive_batch(const gs_problem *probs, const int *idx, int n, cudaStream_t st, int32_t *status,
                     gs_stats *stats) {
    // groups: (dimension bucket, bandwidths per chunk), problems largest first
    std::vector<std::vector<int>> groups(9 * 4);
    for (int k = 0; k < n; ++k) {
        const gs_problem &p = probs[idx[k]];
        const int nj = p.nh <= 1 ? 0 : (p.nh <= 2 ? 1 : (p.nh <= 4 ? 2 : 3));
        groups[dp_for(p.D) * 4 + nj].push_back(idx[k]);
    }
    std::vector<void *> blocks;
    std::vector<std::pair<std::vector<int>, std::vector<GroupProb>>> launched;
    int64_t launches = 0;
    int rc = GS_OK;
    for (int key = 0; key < (int)groups.size() && rc == GS_OK; ++key) {
        std::vector<int> &ids = groups[key];
        if (ids.empty()) continue;
        std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) {
            return (double)probs[a].M * probs[a].N * probs[a].nh > (double)probs[b].M * probs[b].N * probs[b].nh;
        });
        const int DP = key / 4, nj = 1 << (key % 4);
        void *block = nullptr;
        GroupProb *dgp = nullptr;
        std::vector<GroupProb> hgp;
        switch (DP) {
            case 1: rc = launch_group_nj<1>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 2: rc = launch_group_nj<2>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 3: rc = launch_group_nj<3>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 4: rc = launch_group_nj<4>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 5: rc = launch_group_nj<5>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 6: rc = launch_group_nj<6>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            case 7: rc = launch_group_nj<7>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
            default: rc = launch_group_nj<8>(nj, probs, ids, st, &block, &dgp, hgp, launches); break;
        }
        if (block) blocks.push_back(block);
        if (rc == GS_OK) launched.emplace_back(ids, hgp);
    }
    // one status read for every grouped problem
    std::vector<std::vector<Ingest>> hing(launched.size());
    for (size_t g = 0; g < launched.size() && rc == GS_OK; ++g) {
        hing[g].resize(launched[g].first.size());
        cudaError_t e = cudaMemcpyAsync(hing[g].data(), launched[g].second[0].ing,
                                        hing[g].size() * sizeof(Ingest), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "grouped exhaustive status");
    }
    if (rc == GS_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "grouped exhaustive");
    }
    int first = GS_OK;
    if (rc == GS_OK)
        for (size_t g = 0; g < launched.size(); ++g)
            for (size_t k = 0; k < launched[g].first.size(); ++k) {
                const int i = launched[g].first[k];
                const int r = status_to_code(hing[g][k].status);
                if (status) status[i] = r;
                if (r != GS_OK && first == GS_OK) {
                    first = r;
                    char msg[256];
                    snprintf(msg, sizeof(msg), "%s", gs_last_error());
                    set_error("problem %d: %s", i, msg);
                }
                if (stats) stats->point_pairs_base += launched[g].second[k].M * launched[g].second[k].N *
                                                      (int64_t)launched[g].second[k].nh;
            }
    if (rc != GS_OK && status)   // the batch itself failed: every problem of it reports that
        for (int k = 0; k < n; ++k) status[idx[k]] = rc;
    if (stats) {
        stats->launches += launches;
        stats->launches_base += (int64_t)launched.size();
    }
    for (void *b : blocks) cudaFreeAsync(b, st);
    return rc != GS_OK ? rc : first;
}

// --------------------------------------------------------------------------
// Allocation-free exhaustive sum.
//
// Some callers cannot let a library call cudaMalloc: runtimes that own all
// device memory through their own allocator and forbid direct allocations,
// processes that allocate everything up front and must not fail or stall in
// the middle of a run, and code that cannot afford the implicit
// synchronisation an allocation may cause.  For them this variant of the
// exhaustive sum keeps its scratch -- the status word and the packed
// reference records -- in one fixed array in the library's device memory
// instead of allocating it.  The caller still provides inputs and outputs.
//
// The array exists once per device that uses it and stays resident until the
// process exits (or the device is reset).  The CUDA runtime loads a library's
// device code lazily, so the first call on a device is the one that maps the
// array, and that step may allocate inside the driver; a caller that must
// not allocate mid-run makes one warm-up call at start-up, before any stream
// capture.  Every call uses the same array, so calls whose GPU
// work overlaps (concurrent streams, several host threads) race on it and
// must be serialised by the caller.  Each call resets the status word and
// overwrites the records it reads, so nothing depends on what a previous call
// left there.
// --------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = (size_t)16 << 20;   // 16 MiB
constexpr size_t kNoAllocHeader = 256;               // status word (Ingest) at the start

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, with the device current, and checked before it
// goes to a kernel.  It is looked up on every call rather than cached: the
// lookup is a host-side table read once the library's device code is loaded
// on the device, and an address cached across cudaDeviceReset (which destroys
// the array with the context) or written by several host threads at once
// would be a hazard for nothing.
static int noalloc_scratch(void **out) {
    void *p = nullptr;
    GS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (!p) {
        set_error("cudaGetSymbolAddress returned no address for the fixed scratch array");
        return GS_ERR_CUDA;
    }
    *out = p;
    return GS_OK;
}

template <typename T, int DP, int NJ>
static int run_exhaustive_noalloc(const void *queries, int64_t M, const void *refs, const float *weights,
                                  int64_t N, int D, const double *h, int nh, unsigned char *scratch,
                                  double *out, cudaStream_t st) {
    using Cfg = TileCfg<T, DP>;
    constexpr int NT = Cfg::NT, TILE = Cfg::TILE;
    constexpr int QPT = (DP <= 8) ? 2 : 1;
    const int64_t Npad = (N + TILE - 1) / TILE * TILE;
    const int64_t max_pad = (int64_t)((kNoAllocBytes - kNoAllocHeader) / (NT * sizeof(T))) / TILE * TILE;
    if (Npad > max_pad) {
        set_error("gs_sum_exhaustive_noalloc: N=%lld references exceed the %lld the library's fixed "
                  "16 MiB scratch holds for D=%d", (long long)N, (long long)max_pad, D);
        return GS_ERR_ARG;
    }
    Ingest *ing = reinterpret_cast<Ingest *>(scratch);
    T *rec = reinterpret_cast<T *>(scratch + kNoAllocHeader);
    CallCtx cx;
    cx.st = st;
    cudaError_t e = launch_ingest(ing, queries, M, refs, weights, N, D, sizeof(T) == 8 ? GS_F64 : GS_F32, cx);
    if (e != cudaSuccess) return cuda_fail(e, "ingest launch");
    k_pack_refs<T, DP><<<grid_for(Npad, 256), 256, 0, st>>>((const T *)refs, weights, N, Npad, D, ing, rec);
    NegC nc;
    for (int j = 0; j < 64; ++j) nc.v[j] = 0.f;
    for (int j = 0; j < nh; ++j) nc.v[j] = (float)(-1.4426950408889634 / (2.0 * h[j] * h[j]));
    const int64_t bx = (M + kThreads * QPT - 1) / (kThreads * QPT);
    const int nz = (nh + NJ - 1) / NJ;
    const int64_t tiles = Npad / TILE;
    const int64_t target = (int64_t)num_sms() * 8;
    int64_t splits = (target + bx * nz - 1) / (bx * nz);
    if (splits < 1) splits = 1;
    if (splits > tiles) splits = tiles;
    if (splits > 65535) splits = 65535;
    const int64_t chunk = (tiles + splits - 1) / splits * TILE;
    splits = (Npad + chunk - 1) / chunk;
    if (bx > 2147483647LL) {
        set_error("too many queries for one launch");
        return GS_ERR_ARG;
    }
    if (splits > 1) GS_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)M * nh * sizeof(double), st));
    dim3 grid((unsigned)bx, (unsigned)splits, (unsigned)nz);
    k_exhaustive<T, DP, NJ, QPT><<<grid, kThreads, 0, st>>>((const T *)queries, M, D, rec, chunk, Npad, nc, nh, ing,
                                                           out, splits > 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_exhaustive launch");
    Ingest hing;
    e = cudaMemcpyAsync(&hing, ing, sizeof(Ingest), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "gs_sum_exhaustive_noalloc");
    if (hing.status & ST_NONFINITE) {
        set_error("non-finite coordinate or weight");
        return GS_ERR_NONFINITE;
    }
    if (hing.status & ST_WEIGHT) {
        set_error("a weight is <= 0 (weights must be positive)");
        return GS_ERR_WEIGHT;
    }
    return GS_OK;
}

template <typename T, int DP>
static int noalloc_nj(const void *q, int64_t M, const void *r, const float *w, int64_t N, int D, const double *h,
                      int nh, unsigned char *scr, double *out, cudaStream_t st) {
    if (nh <= 1) return run_exhaustive_noalloc<T, DP, 1>(q, M, r, w, N, D, h, nh, scr, out, st);
    if (nh <= 2) return run_exhaustive_noalloc<T, DP, 2>(q, M, r, w, N, D, h, nh, scr, out, st);
    if (nh <= 4) return run_exhaustive_noalloc<T, DP, 4>(q, M, r, w, N, D, h, nh, scr, out, st);
    return run_exhaustive_noalloc<T, DP, 8>(q, M, r, w, N, D, h, nh, scr, out, st);
}

template <typename T>
static int noalloc_d(const void *q, int64_t M, const void *r, const float *w, int64_t N, int D, const double *h,
                     int nh, unsigned char *scr, double *out, cudaStream_t st) {
#define GS_CASE(DPV) \
    if (D <= DPV) return noalloc_nj<T, DPV>(q, M, r, w, N, D, h, nh, scr, out, st);
    GS_CASE(1) GS_CASE(2) GS_CASE(3) GS_CASE(4) GS_CASE(5) GS_CASE(6) GS_CASE(7) GS_CASE(8)
    GS_CASE(12) GS_CASE(16) GS_CASE(24) GS_CASE(32)
#undef GS_CASE
    set_error("D=%d exceeds 32", D);
    return GS_ERR_ARG;
}

// --------------------------------------------------------------------------
// Instruction-rate probe: independent ex2 / FFMA chains on every SM, timed
// with the per-SM cycle counter.  Each block records its SM and its start and
// end cycle; an SM's rate is the work of all blocks it ran over the span from
// the first start to the last end (one counter per SM, so spans are exact).
// --------------------------------------------------------------------------
constexpr int kProbeIters = 4096;
constexpr int kProbeChains = 8;

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(256) k_probe(float *sink, long long *rec) {
    float v[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = 0.1f + 0.01f * c + 1e-6f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 4
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            if (KIND == 0)
                v[c] = ex2_approx(-v[c]);
            else
                v[c] = fmaf(v[c], 0.9999f, 1e-4f);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += v[c];
    if (s == 12345.f) sink[threadIdx.x] = s;   // keeps the chains live
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = t0;
        rec[3 * blockIdx.x + 1] = t1;
        rec[3 * blockIdx.x + 2] = (long long)smid();
    }
}

int probe_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, cudaStream_t st) {
    const int sms = num_sms();
    const int threads = 256;
    const int nb = sms * 4;
    float *sink = nullptr;
    long long *rec = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&sink, 256 * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&rec, 3 * nb * sizeof(long long), st));
    long long *hr = (long long *)malloc(3 * nb * sizeof(long long));
    const int maxsm = 1024;
    long long *lo = (long long *)malloc(maxsm * sizeof(long long));
    long long *hi = (long long *)malloc(maxsm * sizeof(long long));
    int *cnt = (int *)malloc(maxsm * sizeof(int));
    double rates[2] = {0, 0};
    int rc = GS_OK;
    for (int kind = 0; kind < 2 && rc == GS_OK; ++kind) {
        for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up
            if (kind == 0)
                k_probe<0><<<nb, threads, 0, st>>>(sink, rec);
            else
                k_probe<1><<<nb, threads, 0, st>>>(sink, rec);
        }
        cudaError_t e = cudaMemcpyAsync(hr, rec, 3 * nb * sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "probe");
            break;
        }
        for (int i = 0; i < maxsm; ++i) { lo[i] = (long long)9e18; hi[i] = 0; cnt[i] = 0; }
        for (int b = 0; b < nb; ++b) {
            int sm = (int)hr[3 * b + 2];
            if (sm < 0 || sm >= maxsm) continue;
            if (hr[3 * b] < lo[sm]) lo[sm] = hr[3 * b];
            if (hr[3 * b + 1] > hi[sm]) hi[sm] = hr[3 * b + 1];
            cnt[sm]++;
        }
        double sum = 0;
        int used = 0;
        const double per_block = (double)threads * kProbeIters * kProbeChains;
        for (int i = 0; i < maxsm; ++i)
            if (cnt[i] > 0 && hi[i] > lo[i]) {
                sum += per_block * cnt[i] / (double)(hi[i] - lo[i]);
                used++;
            }
        rates[kind] = used ? sum / used : 0.0;
    }
    free(hr); free(lo); free(hi); free(cnt);
    cudaFreeAsync(sink, st);
    cudaFreeAsync(rec, st);
    if (rc != GS_OK) return rc;
    *ex2_per_sm_clk = rates[0];
    *ffma_per_sm_clk = rates[1];
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_sum_exhaustive_noalloc(const void *queries, int64_t M, const void *refs, const float *weights,
                                         int64_t N, int D, int dtype, const double *h, int nh, double *out,
                                         void *stream) {
    using namespace gs;
    if (!queries || !refs || !weights || !out || !h) {
        set_error("NULL array argument");
        return GS_ERR_ARG;
    }
    if (M < 1 || N < 1 || D < 1 || D > 32 || nh < 1 || nh > 64 || (dtype != GS_F32 && dtype != GS_F64)) {
        set_error("gs_sum_exhaustive_noalloc: bad size, dimension, bandwidth count or dtype");
        return GS_ERR_ARG;
    }
    for (int j = 0; j < nh; ++j)
        if (!(h[j] > 0.0) || !isfinite(h[j])) {
            set_error("bandwidth h[%d]=%g is not finite and positive", j, h[j]);
            return GS_ERR_ARG;
        }
    void *scr = nullptr;
    int rc = noalloc_scratch(&scr);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == GS_F64)
        return noalloc_d<double>(queries, M, refs, weights, N, D, h, nh, (unsigned char *)scr, out, st);
    return noalloc_d<float>(queries, M, refs, weights, N, D, h, nh, (unsigned char *)scr, out, st);
}
