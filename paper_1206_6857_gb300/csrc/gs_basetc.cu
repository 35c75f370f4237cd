// Leaf-leaf base case for 9 <= D <= 16 with the cross term on the tensor
// cores (the D N_Q N_R part of Section 6's c_Direct).
//
// For a leaf pair (Q, R) with FP32 centres c_Q, c_R, a query q = c_Q + u and a
// reference r = c_R + v,
//     ||q - r||^2 = alpha_q + beta_r - 2 gamma,
//     alpha_q = ||q - c_R||^2,   beta_r = ||v||^2 - 2 (c_Q - c_R).v,   gamma = u.v.
// alpha (per query) and beta (per reference) cost D operations per point per
// leaf pair on the FP32 pipe; gamma, the D operations per (query, reference),
// is a 128 x N matrix product on the tensor cores.
//
// Exactness of the product.  Every leaf's centred coordinates are scaled by a
// power of two 2^s (s per leaf, so the largest magnitude lies in
// [2^28, 2^29)) and rounded to integers U (30-bit two's complement range),
// which are split into three balanced base-2^10 digits
//     U = U2 2^20 + U1 2^10 + U0,   U0, U1 in [-512, 511], |U2| <= 512,
// each held exactly by FP16.  The tensor core forms
//     P4 = sum_d U2 V2,  P3 = sum_d (U2 V1 + U1 V2),  P2 = sum_d (U2 V0 + U1 V1 + U0 V2)
// in three FP32 accumulators.  Every product is an integer of magnitude at
// most 2^18 and every partial sum an integer below 48 * 2^18 < 2^24, so each
// accumulator is exact whatever the order and rounding of the tensor core's
// FP32 additions.  gamma = 2^(20 - s_Q - s_R) (P4 2^20 + P3 2^10 + P2) up to the
// dropped groups (U1 V0 + U0 V1) 2^10 + U0 V0.
//
// Error charge (first order in u = 2^-24, D <= 16, rho_Q / rho_R the
// Euclidean radii of the leaves about their centres):
//   |d2~ - d2| <= (D+4) u d2 + u [(4D+10) d rho_R + (4D+11) rho_R^2 + (2D+21) rho_Q rho_R],
// from alpha (D+2) u alpha, beta (D+3) u (rho_R^2 + 2 |c_Q - c_R| rho_R), gamma
// 6.3 u rho_Q rho_R (FP32 rounding of the centred coordinates 2u, the
// quantisation 2^-26 rho_Q rho_R, the dropped groups 2^-23 rho_Q rho_R, the two
// FP32 steps recombining P4, P3, P2 2.05u) and the last two FP32 operations,
// with alpha <= (d + rho_R)^2 and |c_Q - c_R| <= d + rho_Q + rho_R.  The
// relative part is charged like the direct base case's argument rounding
// (over exponents down to 2^-64, plus two roundings of the exponent argument);
// the absolute part, at d <= 9.42 h (the largest distance whose term is above
// 2^-64) and the pair's smallest bandwidth, must stay within
// tau = 2^kTcGuardLog2 in log2 units: pairs that fail that guard are summed by
// the direct FP32 kernel instead.  The traversal's FP32 charge rho (Theorem 2's
// eps budget) carries ln2 (64 (D+6) u + tau) for the argument whenever this
// path is enabled.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include "gs_device.cuh"
#include "gs_internal.h"
#include "gs_tc.cuh"
#include "gs_tree.cuh"

namespace gs {

constexpr int kTcRows = 128;               // M of the MMA: query rows (leaf size <= 128)
constexpr int kTcChunk = 32;               // N of the MMA: reference columns per chunk
constexpr int kTcWG = 4;                   // warpgroups per CTA
constexpr int kTcDigitBytes = kTcRows * 32;    // one digit tile: 128 rows x 16 FP16
constexpr int kTcLeafBytes = 3 * kTcDigitBytes;  // three digits of one leaf
constexpr int kTcRecFloats = 20;           // largest record (RefRec<float, 16>::NT): shared-memory sizing
constexpr int kTcBlk = 8;                  // bandwidths accumulated per pass
constexpr uint32_t kTcWaitPolls = 1u << 22;    // bounded wait on the MMA completion barrier

static_assert(RefRec<float, 16>::NT == kTcRecFloats, "record layout");

// byte offset of element (row, k) in a K-major, unswizzled tile of 16-bit
// elements: 8-row x 16-byte core matrices; the two K halves 128 bytes apart
// (LBO), 8-row groups 256 bytes apart (SBO)
__host__ __device__ constexpr uint32_t tc_off(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------------------
// leaf tiles: FP32 centre, scale exponent, Euclidean radius and the three
// digit tiles of every leaf of a tree
// ---------------------------------------------------------------------------
struct TcLeaves {
    unsigned char *tiles = nullptr;   // nleaves x kTcLeafBytes
    float *c32 = nullptr;             // nleaves x 16 (FP32 centre, zero beyond D)
    int32_t *scale = nullptr;         // nleaves: s (coordinates scaled by 2^s)
    double *rad = nullptr;            // nleaves: max_x ||x - c||_2 (rounded up)
    int64_t nleaves = 0;
};

__device__ __forceinline__ void split_digits(int32_t U, int32_t &d2, int32_t &d1, int32_t &d0) {
    d0 = ((U + 512) & 1023) - 512;
    int32_t t = (U - d0) >> 10;
    d1 = ((t + 512) & 1023) - 512;
    d2 = (t - d1) >> 10;
}

// One CTA (128 threads) per leaf: thread t takes the leaf's t-th point.
__global__ void __launch_bounds__(128) k_tc_leaf_tiles(const float *__restrict__ rec, int rec_stride, int64_t n,
                                                       int depth, const double *__restrict__ center, int D,
                                                       TcLeaves L) {
    __shared__ float s_max[4];
    __shared__ double s_rad[4];
    const int64_t i = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t node = ((int64_t)1 << depth) - 1 + i;
    const int64_t b = level_begin(n, depth, i), e = level_begin(n, depth, i + 1);
    const int cnt = (int)(e - b);
    float c[16], uh[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) c[d] = d < D ? (float)center[node * D + d] : 0.f;
    float mx = 0.f;
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < 16; ++d) {
        const float x = (t < cnt && d < D) ? rec[(b + t) * rec_stride + d] : c[d];
        uh[d] = x - c[d];
        mx = fmaxf(mx, fabsf(uh[d]));
        const double dx = (double)x - (double)c[d];
        r2 += dx * dx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    }
    if ((t & 31) == 0) {
        s_max[t >> 5] = mx;
        s_rad[t >> 5] = r2;
    }
    __syncthreads();
    mx = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
    r2 = fmax(fmax(s_rad[0], s_rad[1]), fmax(s_rad[2], s_rad[3]));
    int s = 0;
    if (mx > 0.f) {
        int ex;
        frexpf(mx, &ex);   // mx = m 2^ex, m in [0.5, 1): |u| 2^(29 - ex) < 2^29
        s = 29 - ex;
    }
    if (t == 0) {
        L.scale[i] = s;
        L.rad[i] = sqrt(r2) * (1.0 + 1e-12);
#pragma unroll
        for (int d = 0; d < 16; ++d) L.c32[i * 16 + d] = c[d];
    }
    __half dg[3][16];
#pragma unroll
    for (int d = 0; d < 16; ++d) {
        const int32_t U = (int32_t)rintf(ldexpf(uh[d], s));
        int32_t a2, a1, a0;
        split_digits(U, a2, a1, a0);
        dg[0][d] = __int2half_rn(a2);
        dg[1][d] = __int2half_rn(a1);
        dg[2][d] = __int2half_rn(a0);
    }
    unsigned char *tile = L.tiles + i * (int64_t)kTcLeafBytes;
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
            uint4 v;
            __half *hv = reinterpret_cast<__half *>(&v);
#pragma unroll
            for (int k = 0; k < 8; ++k) hv[k] = t < cnt ? dg[g][kh * 8 + k] : __int2half_rn(0);
            *reinterpret_cast<uint4 *>(tile + g * kTcDigitBytes + tc_off(t, kh * 8)) = v;
        }
}

// blocks of 256 threads (8 warps, one query-leaf row per warp) for lq rows
static unsigned grid_for_rows(int64_t lq) {
    const int64_t b = (lq + 7) / 8;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

static int build_tc_leaves(const TreeDev &t, TcLeaves &L, CallCtx &cx) {
    cudaStream_t st = cx.st;
    L.nleaves = (int64_t)1 << t.depth;
    GS_CUDA_TRY(dev_malloc_async((void **)&L.tiles, (size_t)L.nleaves * kTcLeafBytes, st));
    GS_CUDA_TRY(dev_malloc_async((void **)&L.c32, (size_t)L.nleaves * 16 * sizeof(float), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&L.scale, (size_t)L.nleaves * sizeof(int32_t), st));
    GS_CUDA_TRY(dev_malloc_async((void **)&L.rad, (size_t)L.nleaves * sizeof(double), st));
    k_tc_leaf_tiles<<<(unsigned)L.nleaves, 128, 0, st>>>(t.rec, t.rec_stride, t.n, t.depth, t.center, t.D, L);
    cx.launches += 1;
    return cx.check("k_tc_leaf_tiles");
}

static void free_tc_leaves(TcLeaves &L, cudaStream_t st) {
    if (L.tiles) cudaFreeAsync(L.tiles, st);
    if (L.c32) cudaFreeAsync(L.c32, st);
    if (L.scale) cudaFreeAsync(L.scale, st);
    if (L.rad) cudaFreeAsync(L.rad, st);
    L = TcLeaves();
}

// ---------------------------------------------------------------------------
// routing: the guard of every merged entry, evaluated at its smallest bandwidth
// ---------------------------------------------------------------------------
constexpr int kTcGuardLog2 = -11;           // tau: absolute exponent error allowed (log2 units)

struct TcGuard {
    double k_lin;       // u log2(e) (4D+10) 9.42 / 2            (times rho_R / h)
    double k_sq;        // u log2(e) / 2                          (times [(4D+11) rho_R^2 + (2D+21) rho_Q rho_R] / h^2)
    double a_rr, a_qr;  // 4D+11, 2D+21
    double tau;
    double inv_h[32];   // by mask bit: 1 / h
};

__host__ __device__ inline double tc_guard_value(const TcGuard &g, int bit, double rq, double rr) {
    const double ih = g.inv_h[bit];
    return g.k_lin * rr * ih + g.k_sq * (g.a_rr * rr * rr + g.a_qr * rq * rr) * (ih * ih);
}

__device__ __forceinline__ bool tc_guard_ok(const TcGuard &g, uint32_t mask, double rq, double rr) {
    return tc_guard_value(g, __ffs(mask) - 1, rq, rr) <= g.tau;   // lowest bit: smallest bandwidth
}

// Per query-leaf row: entries passing the guard go to the tensor-core list,
// the others to the direct list (both in ascending R, row offsets from a scan).
__global__ void k_tc_count(const MergedEntry *__restrict__ ent, const long long *__restrict__ off, int64_t lq,
                           const double *__restrict__ qrad, const double *__restrict__ rrad, int64_t rleaf0,
                           TcGuard g, long long *cnt_tc, long long *cnt_dir) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < lq; i += warps) {
        int c = 0;
        const double rq = qrad[i];
        for (long long e = off[i] + lane; e < off[i + 1]; e += 32) {
            const MergedEntry E = ent[e];
            c += tc_guard_ok(g, E.mask, rq, rrad[E.r - rleaf0]) ? 1 : 0;
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) {
            cnt_tc[i] = c;
            cnt_dir[i] = (off[i + 1] - off[i]) - c;
        }
    }
}

__global__ void k_tc_split(const MergedEntry *__restrict__ ent, const long long *__restrict__ off, int64_t lq,
                           const double *__restrict__ qrad, const double *__restrict__ rrad, int64_t rleaf0,
                           TcGuard g, const long long *__restrict__ off_tc, const long long *__restrict__ off_dir,
                           MergedEntry *ent_tc, MergedEntry *ent_dir) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < lq; i += warps) {
        const double rq = qrad[i];
        long long ot = off_tc[i], od = off_dir[i];
        for (long long e0 = off[i]; e0 < off[i + 1]; e0 += 32) {
            const long long e = e0 + lane;
            const bool valid = e < off[i + 1];
            MergedEntry E;
            E.r = 0;
            E.mask = 0;
            bool ok = false;
            if (valid) {
                E = ent[e];
                ok = tc_guard_ok(g, E.mask, rq, rrad[E.r - rleaf0]);
            }
            const unsigned bt = __ballot_sync(0xffffffffu, valid && ok);
            const unsigned bd = __ballot_sync(0xffffffffu, valid && !ok);
            if (valid && ok) ent_tc[ot + __popc(bt & lt)] = E;
            if (valid && !ok) ent_dir[od + __popc(bd & lt)] = E;
            ot += __popc(bt);
            od += __popc(bd);
        }
    }
}

// ---------------------------------------------------------------------------
// the tensor-core base-case kernel
// ---------------------------------------------------------------------------
struct TcParams {
    const float *qrec, *rrec;     // packed FP32 records (coordinates, log2(w / w_max)), 20 floats each
    int64_t qn, rn;
    int q_depth, r_depth;
    const unsigned char *qtiles, *rtiles;
    const float *qc32, *rc32;
    const int32_t *qscale, *rscale;
    int D, nh;
    int stride;         // floats per record (16 for D <= 12, 20 for D <= 16); log2(w / w_max) at lwi
    int lwi;
    float negc[32];     // by mask bit: -log2(e) / (2 h^2)
    int jcol[32];       // by mask bit: output column
    double *Gq;
    Ingest *ing;
    unsigned long long *evals;
    int *next_leaf;     // work counter (zeroed before the launch)
};

// dynamic shared memory layout of one CTA (byte offsets)
struct TcSmem {
    static constexpr int kRecBytes = kTcRows * kTcRecFloats * 4;          // 10 KB of records per leaf
    static constexpr int A = 0;                                          // query digit tiles
    static constexpr int QREC = A + kTcLeafBytes;                        // query records
    static constexpr int CQ = QREC + kRecBytes;                          // query leaf centre (16 floats)
    static constexpr int STAGE = CQ + 64;                                // per warpgroup: 2 x (tiles, records, centre)
    static constexpr int STAGE_ONE = kTcLeafBytes + kRecBytes + 64;
    static constexpr int BL = STAGE + kTcWG * 2 * STAGE_ONE;             // per warpgroup: (beta, lw) x 128
    static constexpr int MISC = BL + kTcWG * kTcRows * 8;                 // mbarriers, TMEM address, flags
    static constexpr int TOTAL = MISC + 192;
    // the cross-warpgroup reduction at the end of a query leaf reuses STAGE
    static constexpr int RED = STAGE;
};
static_assert(TcSmem::TOTAL <= 227 * 1024, "shared memory");
static_assert(kTcWG * kTcRows * kTcBlk * 8 <= kTcWG * 2 * TcSmem::STAGE_ONE, "reduction fits the stage area");

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tc::smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 16 reference columns for NJ bandwidths: gamma from the three accumulators,
// the squared distance and each exponent argument two columns per packed
// f32x2 operation; the exponentials are summed per column parity in scalar
// FP32 (part[k][0] even columns, part[k][1] odd).  bl holds, per column pair,
// (beta_i, beta_i+1, lw_i, lw_i+1), so one 16-byte load gives both pairs.
template <int NJ>
__device__ __forceinline__ void tc_cols16(const float (&a4)[16], const float (&a3)[16], const float (&a2)[16],
                                          const float *bl, f2_t alpha2, f2_t m2s2, const f2_t (&c2)[NJ],
                                          float (&part)[NJ][2]) {
    const f2_t k1024 = f2_pack(1024.f, 1024.f);
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
        const float4 b = *reinterpret_cast<const float4 *>(bl + 2 * i);
        f2_t g = f2_fma(f2_pack(a4[i], a4[i + 1]), k1024, f2_pack(a3[i], a3[i + 1]));
        g = f2_fma(g, k1024, f2_pack(a2[i], a2[i + 1]));
        const f2_t ab = f2_add(alpha2, f2_pack(b.x, b.y));
        const f2_t d2 = f2_fma(g, m2s2, ab);
        const f2_t lw = f2_pack(b.z, b.w);
#pragma unroll
        for (int k = 0; k < NJ; ++k) {
            float x0, x1;
            f2_unpack(f2_fma(d2, c2[k], lw), x0, x1);
            part[k][0] += ex2_approx(x0);
            part[k][1] += ex2_approx(x1);
        }
    }
}

// Everything a warpgroup needs to run the chunks of one entry.
struct TcEntryCtx {
    uint32_t tmem_lane;     // this thread's lane, the warpgroup's first column
    uint32_t tmem_mma;      // lane 0, the warpgroup's first column
    uint32_t a0, b0;        // shared addresses of the query and reference digit tiles
    uint32_t idesc;
    uint64_t *full;         // the MMAs of the current chunk completed (1 arrival)
    volatile int *abort;    // the warpgroup's give-up flag
    int bar_id;
    bool leader;            // the thread that issues the MMAs
    uint32_t fparity;       // parity of the next completion phase
};

// The warpgroup's accumulators: columns g * 32, g = 0, 1, 2 for P4, P3, P2 of
// one 32-column chunk.  Issued once every lane has read the previous chunk.
__device__ __forceinline__ void tc_issue_chunk(const TcEntryCtx &x, int c) {
    tc::fence_after_sync();
    const uint32_t bb = x.b0 + (uint32_t)(c * kTcChunk * 32);
    const uint32_t d = x.tmem_mma;
    auto A = [&](int g) { return tc::smem_desc(x.a0 + g * kTcDigitBytes, 128, 256); };
    auto B = [&](int g) { return tc::smem_desc(bb + g * kTcDigitBytes, 128, 256); };
    // digit g of a tile at + g * kTcDigitBytes: 0 = U2, 1 = U1, 2 = U0
    tc::mma_f16(d + 0 * kTcChunk, A(0), B(0), x.idesc, 0);   // P4 = U2 V2
    tc::mma_f16(d + 1 * kTcChunk, A(0), B(1), x.idesc, 0);   // P3 = U2 V1
    tc::mma_f16(d + 1 * kTcChunk, A(1), B(0), x.idesc, 1);   //    + U1 V2
    tc::mma_f16(d + 2 * kTcChunk, A(0), B(2), x.idesc, 0);   // P2 = U2 V0
    tc::mma_f16(d + 2 * kTcChunk, A(1), B(1), x.idesc, 1);   //    + U1 V1
    tc::mma_f16(d + 2 * kTcChunk, A(2), B(0), x.idesc, 1);   //    + U0 V2
    tc::mma_commit(x.full);
}

// The chunks of one entry.  Chunk 0 was issued by the caller (its MMAs ran
// while beta and alpha were formed); chunk c + 1 is issued as soon as every
// lane has read chunk c.  The NJ bandwidths are the lowest set bits of m;
// their per-entry sums go into the compensated per-slot sums.
template <int NJ>
__device__ __forceinline__ void tc_entry(TcEntryCtx &x, int nchunks, const float *bl, f2_t alpha2, f2_t m2s2,
                                         uint32_t m, const float *negc, float (&ksum)[kTcBlk],
                                         float (&kcmp)[kTcBlk]) {
    f2_t c2[NJ];
    float part[NJ][2];
    {
        uint32_t mm = m;
#pragma unroll
        for (int k = 0; k < NJ; ++k) {
            const float c = negc[__ffs(mm) - 1];
            c2[k] = f2_pack(c, c);
            part[k][0] = part[k][1] = 0.f;
            mm &= mm - 1;
        }
    }
    for (int c = 0; c < nchunks; ++c) {
        if (c > 0 && x.leader && !*x.abort) tc_issue_chunk(x, c);
        if (!*x.abort && !tc::mbar_wait_bounded(x.full, x.fparity, kTcWaitPolls)) *x.abort = 1;
        x.fparity ^= 1u;
        tc::fence_after_sync();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float a4[16], a3[16], a2[16];
            const uint32_t ta = x.tmem_lane + (uint32_t)(16 * half);
            tc::tmem_ld16(ta + 0 * kTcChunk, a4);
            tc::tmem_ld16(ta + 1 * kTcChunk, a3);
            tc::tmem_ld16(ta + 2 * kTcChunk, a2);
            tc::tmem_wait_ld();
            tc_cols16<NJ>(a4, a3, a2, bl + 2 * (kTcChunk * c + 16 * half), alpha2, m2s2, c2, part);
        }
        tc::fence_before_sync();
        tc::bar_sync(x.bar_id, 128);   // every lane has read the accumulators
    }
    // FP32 sum over the reference leaf, then compensated across leaves
    uint32_t mm = m;
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
        const int slot = __ffs(mm) - 1;
        mm &= mm - 1;
        const float v = part[k][0] + part[k][1];
#pragma unroll
        for (int kk = 0; kk < kTcBlk; ++kk)
            if (kk == slot) {
                const float y = v - kcmp[kk];
                const float s2 = ksum[kk] + y;
                kcmp[kk] = (s2 - ksum[kk]) - y;
                ksum[kk] = s2;
            }
    }
}

__global__ void __launch_bounds__(kTcWG * 128, 1)
k_basecase_tc(TcParams p, const MergedEntry *__restrict__ ent, const long long *__restrict__ off, int64_t lq) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x;
    const int wg = tid >> 7;          // warpgroup
    const int t = tid & 127;          // query row (tensor-memory lane) of this thread
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + TcSmem::MISC);     // one per warpgroup
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + TcSmem::MISC + 128);
    int *s_leaf = reinterpret_cast<int *>(sm + TcSmem::MISC + 136);
    // a warpgroup whose completion wait gave up sets its own flag (read by its
    // threads after its own barrier); the CTA reads all four after __syncthreads
    volatile int *s_abort = reinterpret_cast<volatile int *>(sm + TcSmem::MISC + 144);
    auto any_abort = [&]() { return (s_abort[0] | s_abort[1] | s_abort[2] | s_abort[3]) != 0; };
    unsigned char *sA = sm + TcSmem::A;
    const float *sQrec = reinterpret_cast<const float *>(sm + TcSmem::QREC);
    float *sCq = reinterpret_cast<float *>(sm + TcSmem::CQ);
    float *bl = reinterpret_cast<float *>(sm + TcSmem::BL) + wg * kTcRows * 2;

    if (tid < 32) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int w = 0; w < kTcWG; ++w) tc::mbar_init(&mbar[w], 1);
        for (int w = 0; w < 4; ++w) s_abort[w] = 0;
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    TcEntryCtx x;
    x.tmem_mma = *tmem_slot + (uint32_t)(wg * 128);
    x.tmem_lane = x.tmem_mma + ((uint32_t)((t >> 5) * 32) << 16);
    x.a0 = tc::smem_u32(sA);
    x.idesc = tc::idesc_f16_f32(kTcRows, kTcChunk);
    x.full = mbar + wg;
    x.fparity = 0;
    x.abort = s_abort + wg;
    x.bar_id = 1 + wg;
    x.leader = t == 0;
    const int64_t rleaf0 = ((int64_t)1 << p.r_depth) - 1;
    const double wmax = (double)__uint_as_float(p.ing->wmax_bits);
    unsigned long long evals = 0;
    const int nblk = (p.nh + kTcBlk - 1) / kTcBlk;

    for (;;) {
        __syncthreads();   // every thread has read the previous leaf number
        if (tid == 0) *s_leaf = atomicAdd(p.next_leaf, 1);
        __syncthreads();
        const int64_t i = *s_leaf;
        if (i >= lq || any_abort()) break;
        const long long e0 = off[i], e1 = off[i + 1];
        if (e0 == e1) continue;
        const int64_t qb = level_begin(p.qn, p.q_depth, i), qe = level_begin(p.qn, p.q_depth, i + 1);
        const int nq = (int)(qe - qb);
        // the query leaf: digit tiles, records and centre
        {
            const unsigned char *src = p.qtiles + i * (int64_t)kTcLeafBytes;
            for (int v = tid; v < kTcLeafBytes / 16; v += blockDim.x) cp16(sA + 16 * v, src + 16 * v);
            const float *rs = p.qrec + qb * p.stride;
            for (int v = tid; v < nq * (p.stride / 4); v += blockDim.x)
                cp16((unsigned char *)sQrec + 16 * v, rs + 4 * v);
            if (tid < 4) cp16(sCq + 4 * tid, p.qc32 + i * 16 + 4 * tid);
            cp_commit();
            cp_wait<0>();
            tc::fence_proxy_async_smem();
        }
        __syncthreads();
        const int sQ = p.qscale[i];
        for (int jb = 0; jb < nblk; ++jb) {
            const uint32_t bmask = 0xFFu << (kTcBlk * jb);
            float ksum[kTcBlk], kcmp[kTcBlk];
#pragma unroll
            for (int k = 0; k < kTcBlk; ++k) ksum[k] = kcmp[k] = 0.f;
            auto next_used = [&](long long e) {
                while (e < e1 && !(ent[e].mask & bmask)) e += kTcWG;
                return e;
            };
            // stage entry e's reference leaf into buffer b: tiles, records, centre
            auto stage = [&](long long e, int b) {
                const int64_t ri = ent[e].r - rleaf0;
                const int64_t rb = level_begin(p.rn, p.r_depth, ri), re = level_begin(p.rn, p.r_depth, ri + 1);
                unsigned char *dst = sm + TcSmem::STAGE + (wg * 2 + b) * TcSmem::STAGE_ONE;
                const unsigned char *src = p.rtiles + ri * (int64_t)kTcLeafBytes;
                for (int v = t; v < kTcLeafBytes / 16; v += 128) cp16(dst + 16 * v, src + 16 * v);
                const float *rs = p.rrec + rb * p.stride;
                const int nv = (int)(re - rb) * (p.stride / 4);
                for (int v = t; v < nv; v += 128) cp16(dst + kTcLeafBytes + 16 * v, rs + 4 * v);
                if (t < 4) cp16(dst + kTcLeafBytes + TcSmem::kRecBytes + 16 * t, p.rc32 + ri * 16 + 4 * t);
                cp_commit();
            };
            long long e = next_used(e0 + wg);
            int buf = 0;
            if (e < e1) stage(e, 0);
            while (e < e1) {
                const long long en = next_used(e + kTcWG);
                if (en < e1) {
                    stage(en, buf ^ 1);
                    cp_wait<1>();
                } else {
                    cp_wait<0>();
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                tc::bar_sync(x.bar_id, 128);
                const MergedEntry E = ent[e];
                const int64_t ri = E.r - rleaf0;
                const int nr = (int)(level_begin(p.rn, p.r_depth, ri + 1) - level_begin(p.rn, p.r_depth, ri));
                const unsigned char *st_tiles = sm + TcSmem::STAGE + (wg * 2 + buf) * TcSmem::STAGE_ONE;
                const float *st_rec = reinterpret_cast<const float *>(st_tiles + kTcLeafBytes);
                const float *cR = st_rec + TcSmem::kRecBytes / 4;
                const int nchunks = (nr + kTcChunk - 1) / kTcChunk;
                x.b0 = tc::smem_u32(st_tiles);
                // chunk 0's MMAs run while beta and alpha are formed
                if (x.leader && !*x.abort) tc_issue_chunk(x, 0);
                float beta = 0.f, lw = -INFINITY, alpha = 0.f;
                {
                    // 16-byte shared loads (centres and records are 16-byte aligned);
                    // record slots at or past D are masked to zero (slot D holds the
                    // log-weight when D <= 12)
                    float cRv[16], dl[16];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float4 a = reinterpret_cast<const float4 *>(cR)[v];
                        const float4 b = reinterpret_cast<const float4 *>(sCq)[v];
                        cRv[4 * v] = a.x; cRv[4 * v + 1] = a.y; cRv[4 * v + 2] = a.z; cRv[4 * v + 3] = a.w;
                        dl[4 * v] = b.x - a.x; dl[4 * v + 1] = b.y - a.y;
                        dl[4 * v + 2] = b.z - a.z; dl[4 * v + 3] = b.w - a.w;
                    }
                    if (t < nr) {
                        const float *rv = st_rec + t * p.stride;
                        float x[16];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float4 a = reinterpret_cast<const float4 *>(rv)[v];
                            x[4 * v] = a.x; x[4 * v + 1] = a.y; x[4 * v + 2] = a.z; x[4 * v + 3] = a.w;
                        }
                        float s = 0.f;
#pragma unroll
                        for (int d = 0; d < 16; ++d) {
                            const float v = (d < p.D ? x[d] : 0.f) - cRv[d];
                            s = fmaf(v, v - 2.f * dl[d], s);
                        }
                        beta = s;
                        lw = rv[p.lwi];
                    }
                    if (t < nq) {
                        const float *qv = sQrec + t * p.stride;
                        float x[16];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float4 a = reinterpret_cast<const float4 *>(qv)[v];
                            x[4 * v] = a.x; x[4 * v + 1] = a.y; x[4 * v + 2] = a.z; x[4 * v + 3] = a.w;
                        }
                        float s = 0.f;
#pragma unroll
                        for (int d = 0; d < 16; ++d) {
                            const float a = (d < p.D ? x[d] : 0.f) - cRv[d];
                            s = fmaf(a, a, s);
                        }
                        alpha = s;
                    }
                }
                bl[4 * (t >> 1) + (t & 1)] = beta;         // (beta_i, beta_i+1, lw_i, lw_i+1) per pair
                bl[4 * (t >> 1) + 2 + (t & 1)] = lw;
                const uint32_t m = (E.mask & bmask) >> (kTcBlk * jb);
                const int nj = __popc(m);
                evals += (unsigned long long)nj * (unsigned long long)nr;
                const float m2s = ldexpf(-2.f, 20 - sQ - __ldg(p.rscale + ri));
                const f2_t m2s2 = f2_pack(m2s, m2s), alpha2 = f2_pack(alpha, alpha);
                tc::bar_sync(x.bar_id, 128);   // (beta, lw) visible
                const float *negc = p.negc + kTcBlk * jb;
                switch (nj) {
                    case 1: tc_entry<1>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 2: tc_entry<2>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 3: tc_entry<3>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 4: tc_entry<4>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 5: tc_entry<5>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 6: tc_entry<6>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    case 7: tc_entry<7>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                    default: tc_entry<8>(x, nchunks, bl, alpha2, m2s2, m, negc, ksum, kcmp); break;
                }
                if (*x.abort) break;
                buf ^= 1;
                e = en;
            }
            cp_wait<0>();
            __syncthreads();
            if (any_abort()) break;
            // cross-warpgroup reduction in FP64 (fixed order), then the output
            double *red = reinterpret_cast<double *>(sm + TcSmem::RED);
#pragma unroll
            for (int k = 0; k < kTcBlk; ++k) red[(wg * kTcBlk + k) * kTcRows + t] = (double)ksum[k] - (double)kcmp[k];
            __syncthreads();
            for (int xx = tid; xx < kTcBlk * kTcRows; xx += blockDim.x) {
                const int k = xx / kTcRows, row = xx % kTcRows;
                const int bit = kTcBlk * jb + k;
                if (row >= nq || bit >= p.nh) continue;
                double v = 0.0;
                for (int w = 0; w < kTcWG; ++w) v += red[(w * kTcBlk + k) * kTcRows + row];
                if (v != 0.0) atomicAdd(&p.Gq[(qb + row) * p.nh + p.jcol[bit]], v * wmax);
            }
        }
        if (p.evals && t == 0 && evals) {
            atomicAdd(p.evals, evals * (unsigned long long)nq);
            atomicAdd(p.evals + 1, evals * (unsigned long long)nq);
        }
        evals = 0;
    }
    __syncthreads();
    if (any_abort() && tid == 0) atomicOr(&p.ing->status, ST_TIMEOUT);
    cp_wait<0>();
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(*tmem_slot, 512);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool tc_base_enabled(int D, int dtype, int flags, int64_t qn, int q_depth, int64_t rn, int r_depth, int nh) {
    if (D < 9 || D > 16 || dtype != GS_F32 || (flags & (GS_FLAG_NO_TC | GS_FLAG_NO_MERGE)) || nh > 32) return false;
    const int64_t maxq = (qn + (1ll << q_depth) - 1) >> q_depth;
    const int64_t maxr = (rn + (1ll << r_depth) - 1) >> r_depth;
    return maxq <= kTcRows && maxr <= kTcRows;
}

// extra charge on top of the direct base case's: two more roundings of the
// exponent argument over exponents down to 2^-64, and the guard's tau
double tc_charge() {
    const double u = 5.9604644775390625e-08;
    return 0.6931471805599453 * (64.0 * 2.0 * u + ldexp(1.0, kTcGuardLog2));
}

int run_basecase_tc(const TraversalIn &in, const MergedEntry *ent, const long long *off, int64_t lq,
                    long long total, const float *negc, const int *jcol, const double *h_by_bit, double *Gq,
                    MergedEntry **ent_dir_out, long long **off_dir_out, unsigned long long *evals, CallCtx &cx) {
    cudaStream_t st = cx.st;
    TcLeaves LQ, LR;
    const bool mono = in.qt == in.rt;
    long long *cnt = nullptr;      // 2 x (lq + 1): tensor-core and direct counts -> offsets
    MergedEntry *ent_tc = nullptr, *ent_dir = nullptr;
    int *counter = nullptr;
    int rc = GS_OK;
    auto release = [&]() {
        free_tc_leaves(LR, st);
        if (!mono) free_tc_leaves(LQ, st);
        if (cnt) cudaFreeAsync(cnt, st);
        if (ent_tc) cudaFreeAsync(ent_tc, st);
        if (counter) cudaFreeAsync(counter, st);
    };
    rc = build_tc_leaves(*in.rt, LR, cx);
    if (!rc) {
        if (mono)
            LQ = LR;
        else
            rc = build_tc_leaves(*in.qt, LQ, cx);
    }
    cudaError_t e = cudaSuccess;
    if (!rc) e = dev_malloc_async((void **)&cnt, (size_t)2 * (lq + 2) * sizeof(long long), st);
    if (!rc && e == cudaSuccess) e = dev_malloc_async((void **)&ent_tc, (size_t)(total > 0 ? total : 1) * sizeof(MergedEntry), st);
    if (!rc && e == cudaSuccess) e = dev_malloc_async((void **)&ent_dir, (size_t)(total > 0 ? total : 1) * sizeof(MergedEntry), st);
    if (!rc && e == cudaSuccess) e = dev_malloc_async((void **)&counter, sizeof(int), st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "tensor-core base case scratch");
    if (rc) {
        if (ent_dir) cudaFreeAsync(ent_dir, st);
        release();
        return rc;
    }
    TcGuard g;
    const double u = 5.9604644775390625e-08, l2e = 1.4426950408889634;
    const int D = in.D;
    g.k_lin = u * l2e * (4.0 * D + 10.0) * 9.42 / 2.0;
    g.k_sq = u * l2e / 2.0;
    g.a_rr = 4.0 * D + 11.0;
    g.a_qr = 2.0 * D + 21.0;
    g.tau = ldexp(1.0, kTcGuardLog2);
    for (int b = 0; b < 32; ++b) g.inv_h[b] = b < in.nh ? 1.0 / h_by_bit[b] : 0.0;
    const int64_t rleaf0 = (1ll << in.rt->depth) - 1;
    long long *cnt_tc = cnt, *cnt_dir = cnt + (lq + 2);
    k_tc_count<<<grid_for_rows(lq), 256, 0, st>>>(ent, off, lq, LQ.rad, LR.rad, rleaf0, g, cnt_tc, cnt_dir);
    cx.launches += 1;
    rc = scan_i64(cnt_tc, lq, cnt_tc + lq, cx);
    if (!rc) rc = scan_i64(cnt_dir, lq, cnt_dir + lq, cx);
    if (!rc) {
        k_tc_split<<<grid_for_rows(lq), 256, 0, st>>>(ent, off, lq, LQ.rad, LR.rad, rleaf0, g, cnt_tc, cnt_dir,
                                                      ent_tc, ent_dir);
        cx.launches += 1;
        rc = cx.check("k_tc_split");
    }
    if (!rc) {
        TcParams tp;
        memset(&tp, 0, sizeof(tp));
        tp.qrec = in.qt->rec;
        tp.rrec = in.rt->rec;
        tp.qn = in.qt->n;
        tp.rn = in.rt->n;
        tp.q_depth = in.qt->depth;
        tp.r_depth = in.rt->depth;
        tp.qtiles = LQ.tiles;
        tp.rtiles = LR.tiles;
        tp.qc32 = LQ.c32;
        tp.rc32 = LR.c32;
        tp.qscale = LQ.scale;
        tp.rscale = LR.scale;
        tp.D = D;
        tp.nh = in.nh;
        tp.stride = in.rt->rec_stride;
        tp.lwi = dp_for(D);
        for (int b = 0; b < 32; ++b) {
            tp.negc[b] = negc[b];
            tp.jcol[b] = jcol[b];
        }
        tp.Gq = Gq;
        tp.ing = const_cast<Ingest *>(in.ing);
        tp.evals = evals;
        tp.next_leaf = counter;
        e = cudaMemsetAsync(counter, 0, sizeof(int), st);
        if (e == cudaSuccess) e = allow_max_smem((const void *)k_basecase_tc);
        if (e == cudaSuccess) {
            int sms = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t grid = lq < sms ? lq : sms;
            cx.phase(GS_PH_BASE_TC);
            cx.mark(CallCtx::kTimerBase);
            k_basecase_tc<<<(unsigned)(grid > 0 ? grid : 1), kTcWG * 128, TcSmem::TOTAL, st>>>(tp, ent_tc, cnt_tc,
                                                                                                lq);
            cx.mark(-1);
            cx.phase(GS_PH_BASE);
            cx.launches += 1;
            cx.launches_base += 1;
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "k_basecase_tc");
        if (!rc) rc = cx.check("k_basecase_tc");
    }
    if (rc) {
        cudaFreeAsync(ent_dir, st);
        release();
        return rc;
    }
    // the direct list and its offsets go back to the caller (offsets live in cnt)
    *ent_dir_out = ent_dir;
    long long *off_dir = nullptr;
    e = dev_malloc_async((void **)&off_dir, (size_t)(lq + 2) * sizeof(long long), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(off_dir, cnt_dir, (size_t)(lq + 1) * sizeof(long long), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        if (off_dir) cudaFreeAsync(off_dir, st);
        cudaFreeAsync(ent_dir, st);
        *ent_dir_out = nullptr;
        release();
        return cuda_fail(e, "tensor-core base case offsets");
    }
    *off_dir_out = off_dir;
    release();
    return GS_OK;
}

// ---------------------------------------------------------------------------
// self-check of the fixed-point product: one warpgroup, raw accumulators out
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
k_tc_dot_check(const int32_t *__restrict__ U, const int32_t *__restrict__ V, int N, float *P, unsigned *status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm, *sB = sm + kTcLeafBytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * kTcLeafBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + 2 * kTcLeafBytes + 8);
    const int t = threadIdx.x;
    if (t < 32) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_fence_init();
    }
    for (int side = 0; side < 2; ++side) {
        const int32_t *X = side ? V : U;
        const bool valid = side ? t < N : true;
        unsigned char *tile = side ? sB : sA;
        __half dg[3][16];
#pragma unroll
        for (int d = 0; d < 16; ++d) {
            int32_t a2 = 0, a1 = 0, a0 = 0;
            if (valid) split_digits(X[t * 16 + d], a2, a1, a0);
            dg[0][d] = __int2half_rn(a2);
            dg[1][d] = __int2half_rn(a1);
            dg[2][d] = __int2half_rn(a0);
        }
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                uint4 v;
                __half *hv = reinterpret_cast<__half *>(&v);
#pragma unroll
                for (int k = 0; k < 8; ++k) hv[k] = dg[g][kh * 8 + k];
                *reinterpret_cast<uint4 *>(tile + g * kTcDigitBytes + tc_off(t, kh * 8)) = v;
            }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tmem_slot;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_f16_f32(kTcRows, N);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
        auto A = [&](int g) { return tc::smem_desc(a0 + g * kTcDigitBytes, 128, 256); };
        auto B = [&](int g) { return tc::smem_desc(b0 + g * kTcDigitBytes, 128, 256); };
        tc::mma_f16(tm + 0 * 128, A(0), B(0), idesc, 0);
        tc::mma_f16(tm + 1 * 128, A(0), B(1), idesc, 0);
        tc::mma_f16(tm + 1 * 128, A(1), B(0), idesc, 1);
        tc::mma_f16(tm + 2 * 128, A(0), B(2), idesc, 0);
        tc::mma_f16(tm + 2 * 128, A(1), B(1), idesc, 1);
        tc::mma_f16(tm + 2 * 128, A(2), B(0), idesc, 1);
        tc::mma_commit(mbar);
    }
    // the warp-collective tensor-memory loads below need one decision for all
    const bool ok = __syncthreads_and(tc::mbar_wait_bounded(mbar, 0, kTcWaitPolls) ? 1 : 0) != 0;
    if (!ok && t == 0) atomicOr(status, ST_TIMEOUT);
    tc::fence_after_sync();
    if (ok) {
        const uint32_t lane_base = (uint32_t)((t >> 5) * 32) << 16;
        for (int g = 0; g < 3; ++g)
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tm + lane_base + g * 128 + c0, v);
                tc::tmem_wait_ld();
                for (int k = 0; k < 16; ++k) P[((size_t)g * kTcRows + t) * N + c0 + k] = v[k];
            }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 32) tc::tmem_dealloc(tm, 512);
}

int tc_dot_check(const int32_t *U, const int32_t *V, int N, float *P, cudaStream_t st) {
    int32_t *dU = nullptr, *dV = nullptr;
    float *dP = nullptr;
    unsigned *dS = nullptr;
    int rc = GS_OK;
    cudaError_t e = dev_malloc_async((void **)&dU, kTcRows * 16 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dV, (size_t)kTcRows * 16 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dP, (size_t)3 * kTcRows * N * sizeof(float), st);
    if (e == cudaSuccess) e = dev_malloc_async((void **)&dS, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dS, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dV, 0, (size_t)kTcRows * 16 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dU, U, kTcRows * 16 * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dV, V, (size_t)N * 16 * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    const int smem = 2 * kTcLeafBytes + 64;
    if (e == cudaSuccess) e = allow_max_smem((const void *)k_tc_dot_check);
    if (e == cudaSuccess) {
        k_tc_dot_check<<<1, 128, smem, st>>>(dU, dV, N, dP, dS);
        e = cudaGetLastError();
    }
    unsigned hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(P, dP, (size_t)3 * kTcRows * N * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, dS, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "gs_tc_dot_check");
    else if (hs & ST_TIMEOUT) {
        set_error("gs_tc_dot_check: the tensor-core completion barrier did not arrive");
        rc = GS_ERR_TIMEOUT;
    }
    if (dU) cudaFreeAsync(dU, st);
    if (dV) cudaFreeAsync(dV, st);
    if (dP) cudaFreeAsync(dP, st);
    if (dS) cudaFreeAsync(dS, st);
    return rc;
}

}  // namespace gs

extern "C" int gs_tc_dot_check(const int32_t *U, const int32_t *V, int N, float *P, void *stream) {
    using namespace gs;
    if (!U || !V || !P || N < 16 || N > 128 || N % 16) {
        set_error("gs_tc_dot_check: NULL pointer or N=%d not a multiple of 16 in [16, 128]", N);
        return GS_ERR_ARG;
    }
    for (int i = 0; i < kTcRows * 16; ++i)
        if (U[i] < -(1 << 29) || U[i] > (1 << 29)) {
            set_error("gs_tc_dot_check: U[%d] outside [-2^29, 2^29]", i);
            return GS_ERR_ARG;
        }
    for (int i = 0; i < N * 16; ++i)
        if (V[i] < -(1 << 29) || V[i] > (1 << 29)) {
            set_error("gs_tc_dot_check: V[%d] outside [-2^29, 2^29]", i);
            return GS_ERR_ARG;
        }
    return tc_dot_check(U, V, N, P, (cudaStream_t)stream);
}
