// Leaf-leaf base case with the bandwidths of one leaf pair merged.
//
// The traversal emits its base cases per bandwidth: (query leaf Q, h_j, list
// of reference leaves).  A bandwidth sweep leaves the same leaf pair
// unpruned for several neighbouring bandwidths, and every one of them needs
// the same squared distances.  This pass folds the per-bandwidth lists into
// one list of (Q, R, bandwidth mask) entries per query leaf.  In complete
// kd-trees every leaf-leaf pair meets in the same frontier iteration, so each
// (Q, h_j) has at most one list:
//   index   -- the list of each (Q, mask bit) in a lq x 32 table;
//   count   -- per query leaf, the bandwidth masks built in shared memory one
//              slice of reference leaves at a time, nonzero masks counted;
//   scan    -- row offsets;
//   write   -- the masks rebuilt and the (R, mask) entries written in ascending R.
// Global scratch grows with the number of base pairs (the lists and the
// entries), not with lq x lr; the lq x lr mask words exist only in shared
// memory, one slice per CTA at a time.
// The base-case kernel then forms each squared distance once per (query,
// reference) and evaluates one exponential per bandwidth in the mask
// (Section 1's sum term, DITOBase of Fig. 7).  Sums: FP32 over the terms of
// one reference leaf, then compensated (Kahan) FP32 per (bandwidth, query)
// across leaves, then FP64 across warps.
#include <limits.h>
#include <math.h>

#include "gs_device.cuh"
#include "gs_frontier.cuh"
#include "gs_internal.h"
#include "gs_tree.cuh"

namespace gs {

struct BitMap {
    int8_t rank[64];    // bandwidth j -> mask bit (bandwidths ranked by ascending h)
};

// A second base group for the same (query leaf, bandwidth) would mean leaf
// pairs met in two frontier iterations, which complete trees rule out; it is
// reported (ST_INTERNAL) rather than merged.
__global__ void k_row_groups(const Group *__restrict__ bgroups, int64_t nbg, int64_t qleaf0, BitMap bm,
                             int32_t *gidx, Ingest *ing) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nbg; g += (int64_t)gridDim.x * blockDim.x) {
        const Group G = bgroups[g];
        if (atomicCAS(&gidx[(G.q - qleaf0) * 32 + bm.rank[G.j]], -1, (int32_t)g) != -1)
            atomicOr(&ing->status, ST_INTERNAL);
    }
}

// One CTA per query-leaf row (grid-stride): the row's bandwidth masks are
// built in shared memory, one slice of kSlice reference leaves at a time
// (atomicOr of bit b for every reference leaf on the list of mask bit b), then
// the nonzero masks of the slice are counted (WRITE = false: cnt_off[row] =
// count) or written in ascending R at cnt_off[row] (WRITE = true: each thread
// takes a contiguous run of words; a block-wide exclusive scan of the run
// counts orders the writes).
constexpr int kSlice = 16384;
constexpr int kMergeThreads = 256;

template <bool WRITE>
__global__ void __launch_bounds__(kMergeThreads)
k_row_masks(const Group *__restrict__ bgroups, const int32_t *__restrict__ base_r, const int32_t *__restrict__ gidx,
            int64_t lq, int64_t lr, int64_t rleaf0, long long *__restrict__ cnt_off, MergedEntry *__restrict__ ent) {
    extern __shared__ uint32_t smask[];          // kSlice words
    __shared__ int s_warp[kMergeThreads / 32];
    constexpr int kRun = kSlice / kMergeThreads;  // words per thread
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int64_t i = blockIdx.x; i < lq; i += gridDim.x) {
        long long o = WRITE ? cnt_off[i] : 0;
        long long total = 0;
        for (int64_t s0 = 0; s0 < lr; s0 += kSlice) {
            for (int k = t; k < kSlice; k += kMergeThreads) smask[k] = 0u;
            __syncthreads();
            for (int b = 0; b < 32; ++b) {
                const int32_t g = gidx[i * 32 + b];
                if (g < 0) continue;
                const Group G = bgroups[g];
                for (int k = t; k < G.cnt; k += kMergeThreads) {
                    const int64_t rl = (int64_t)base_r[G.off + k] - rleaf0 - s0;
                    if (rl >= 0 && rl < kSlice) atomicOr(&smask[rl], 1u << b);
                }
            }
            __syncthreads();
            int c = 0;
#pragma unroll 8
            for (int k = 0; k < kRun; ++k) c += smask[t * kRun + k] != 0u;
            // block-wide exclusive scan of the per-thread counts
            int incl = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (lane == 31) s_warp[w] = incl;
            __syncthreads();
            int before = 0, slice_total = 0;
            for (int k = 0; k < kMergeThreads / 32; ++k) {
                if (k < w) before += s_warp[k];
                slice_total += s_warp[k];
            }
            if (WRITE) {
                long long pos = o + total + before + (incl - c);
                for (int k = 0; k < kRun; ++k) {
                    const uint32_t m = smask[t * kRun + k];
                    if (m) {
                        MergedEntry e;
                        e.r = (int32_t)(rleaf0 + s0 + t * kRun + k);
                        e.mask = m;
                        ent[pos++] = e;
                    }
                }
            }
            total += slice_total;
            __syncthreads();   // the slice and s_warp are reused
        }
        if (!WRITE && t == 0) cnt_off[i] = total;
    }
}

constexpr int kMW = 4;   // warps per CTA

// The packed f32x2 path takes two query slots per register pair.
__host__ __device__ constexpr bool merged_x2(int DP, int QPL) { return QPL >= 2 && DP <= 16; }

struct MergedParams {
    const float *qrec, *rrec;
    const float *rrec2;      // reference records with every float duplicated (packed path)
    int64_t qn, rn;
    int q_depth, r_depth;
    const double *qcenter, *rcenter;
    int D, nh;
    float negc[32];     // by mask bit: -log2(e) / (2 h^2)
    int jcol[32];       // by mask bit: output column (bandwidth index)
    double *Gq;
    const Ingest *ing;
    unsigned long long *evals;
};

// Sum over one reference leaf (staged in shared memory) for NJ bandwidths
// at once: one squared distance per (query, reference), NJ exponentials.
template <int DP, int QPL, bool ANCH, int NJ>
__device__ __forceinline__ void leaf_terms(const float (&xq)[QPL][DP], const float (&dc)[DP], const float4 *rp,
                                           int nr, const float (&c)[8], float (&part)[QPL][8]) {
    constexpr int NT = RefRec<float, DP>::NT;
#pragma unroll
    for (int s = 0; s < QPL; ++s)
#pragma unroll
        for (int k = 0; k < NJ; ++k) part[s][k] = 0.f;
#pragma unroll 2
    for (int i = 0; i < nr; ++i) {
        float rv[NT];
#pragma unroll
        for (int v = 0; v < NT / 4; ++v) {
            const float4 f = rp[i * (NT / 4) + v];
            rv[4 * v] = f.x; rv[4 * v + 1] = f.y; rv[4 * v + 2] = f.z; rv[4 * v + 3] = f.w;
        }
        const float l = rv[DP];
#pragma unroll
        for (int s = 0; s < QPL; ++s) {
            float d2 = 0.f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                const float df = ANCH ? (xq[s][d] - rv[d]) + dc[d] : xq[s][d] - rv[d];
                d2 = fmaf(df, df, d2);
            }
#pragma unroll
            for (int k = 0; k < NJ; ++k) part[s][k] += ex2_approx(fmaf(d2, c[k], l));
        }
    }
}

// leaf_terms for two query slots per register pair: the staged reference
// records hold every float twice, (x_0, x_0, x_1, x_1, ..., l, l, ...), so a
// 16-byte shared load gives two broadcast pairs.  Same operations, in the
// same order, as the scalar version; up to 8 bandwidths share one squared
// distance (the scalar version takes 4 at a time).
template <int DP, int QPL, bool ANCH, int NJ>
__device__ __forceinline__ void leaf_terms_x2(const f2_t (&xq)[QPL / 2][DP], const f2_t (&dc)[DP],
                                              const ulonglong2 *rp, int nr, const f2_t (&c)[8],
                                              f2_t (&part)[QPL / 2][8]) {
    constexpr int NT = RefRec<float, DP>::NT;   // pairs per staged record
#pragma unroll
    for (int s = 0; s < QPL / 2; ++s)
#pragma unroll
        for (int k = 0; k < 8; ++k) part[s][k] = 0ull;
#pragma unroll 4
    for (int i = 0; i < nr; ++i) {
        f2_t rv[NT];
#pragma unroll
        for (int v = 0; v < NT / 2; ++v) {
            const ulonglong2 u = rp[i * (NT / 2) + v];
            rv[2 * v] = u.x;
            rv[2 * v + 1] = u.y;
        }
#pragma unroll
        for (int s = 0; s < QPL / 2; ++s) {
            f2_t d2 = 0ull;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
                f2_t df = f2_sub(xq[s][d], rv[d]);
                if (ANCH) df = f2_add(df, dc[d]);
                d2 = f2_fma(df, df, d2);
            }
#pragma unroll
            for (int k = 0; k < NJ; ++k) {
                float a0, a1;
                f2_unpack(f2_fma(d2, c[k], rv[DP]), a0, a1);
                part[s][k] = f2_add(part[s][k], f2_pack(ex2_approx(a0), ex2_approx(a1)));
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int kBlk = 8;   // bandwidths accumulated per pass

// shared memory a CTA can use on one SM (228 KB, less 1 KB reserved per CTA
// at three CTAs)
constexpr size_t kSmemPerSm = 225 * 1024;

// staging buffers per warp: two unless two would leave fewer than three CTAs
// per SM at leaves of 32 QPL points (the shape the launch takes for
// monochromatic data)
__host__ __device__ constexpr int merged_nbuf(int DP, int QPL) {
    return 3 * (size_t)kMW *
                       (2 * kBlk * QPL * 32 +
                        2 * 32 * QPL * (merged_x2(DP, QPL) ? 2 : 1) * (((DP + 1) * 4 + 15) / 16 * 4)) *
                       sizeof(float) >
                   kSmemPerSm
               ? 1
               : 2;
}

// Shared memory per warp: Kahan sums and compensations for one block of
// kBlk bandwidths (2 x kBlk x QPL x 32 floats), then nbuf staging buffers of
// lmax reference records each (two: the next leaf is copied while this one is
// summed; one, where two would leave fewer than three CTAs per SM: the next
// leaf is copied after this one).  Mask bits are bandwidths in ascending h, so
// the bandwidths a leaf pair needs are consecutive; the CTA makes one pass
// over its entries per block of kBlk bandwidths, blocks starting at the
// lowest bandwidth any of its entries needs.
template <int DP, int QPL, bool ANCH>
__global__ void __launch_bounds__(32 * kMW)
k_basecase_merged(MergedParams bp, const MergedEntry *__restrict__ ent, const long long *__restrict__ off,
                  int64_t lq, int lmax) {
    constexpr int NT = RefRec<float, DP>::NT;
    constexpr bool X2 = merged_x2(DP, QPL);
    constexpr int nbuf = merged_nbuf(DP, QPL);
    constexpr int NS = X2 ? 2 * NT : NT;   // floats per staged reference record
    constexpr int KS = kBlk * QPL * 32;
    extern __shared__ float sm_f[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x;
    const int64_t e0 = off[i], e1 = off[i + 1];
    if (e0 == e1) return;
    const int nh = bp.nh;
    const size_t per_warp = (size_t)2 * KS + (size_t)nbuf * lmax * NS;
    float *ksum = sm_f + (size_t)w * per_warp;
    float *kcmp = ksum + KS;
    float *stage = ksum + 2 * KS;   // nbuf x lmax x NS floats, 16-byte aligned
    const int64_t qleaf0 = (1ll << bp.q_depth) - 1, rleaf0 = (1ll << bp.r_depth) - 1;
    const int64_t qnode = qleaf0 + i;
    const int64_t qb = level_begin(bp.qn, bp.q_depth, i), qe = level_begin(bp.qn, bp.q_depth, i + 1);
    const int nq = (int)(qe - qb);
    float xq[QPL][DP];
#pragma unroll
    for (int s = 0; s < QPL; ++s) {
        const int qq = lane + 32 * s;
        const int64_t pos = qb + (qq < nq ? qq : 0);
#pragma unroll
        for (int d = 0; d < DP; ++d) xq[s][d] = bp.qrec[pos * NT + d];
    }
    // stage the reference leaf of entry e into buffer b (cooperative 16-byte async copies)
    auto stage_leaf = [&](int64_t e, int b) {
        const int64_t ri = ent[e].r - rleaf0;
        const int64_t rb = level_begin(bp.rn, bp.r_depth, ri), re = level_begin(bp.rn, bp.r_depth, ri + 1);
        const int nv = (int)(re - rb) * (NS / 4);
        const float4 *src = reinterpret_cast<const float4 *>((X2 ? bp.rrec2 : bp.rrec) + rb * NS);
        float4 *dst = reinterpret_cast<float4 *>(stage + (size_t)b * lmax * NS);
        for (int v = lane; v < nv; v += 32) cp_async16(dst + v, src + v);
        cp_async_commit();
    };
    const double wmax = (double)__uint_as_float(bp.ing->wmax_bits);
    unsigned long long evals = 0;
    // the blocks start at the lowest bandwidth this query leaf's entries use,
    // so a leaf pair's (consecutive) bandwidths are split across passes only
    // when the leaf's whole range is wider than a block
    __shared__ uint32_t s_union[kMW];
    uint32_t un = 0u;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) un |= ent[e].mask;
    un = __reduce_or_sync(0xffffffffu, un);
    if (lane == 0) s_union[w] = un;
    __syncthreads();
    un = 0u;
#pragma unroll
    for (int ww = 0; ww < kMW; ++ww) un |= s_union[ww];
    const int b0 = __ffs(un) - 1, b1 = 31 - __clz(un);
    const int nblk = (b1 - b0) / kBlk + 1;
    for (int jb = 0; jb < nblk; ++jb) {
        const int sh = b0 + kBlk * jb;     // first mask bit of this block (<= b1 <= 31)
        const uint32_t bmask = 0xFFu << sh;
        for (int t = lane; t < 2 * KS; t += 32) ksum[t] = 0.f;
        auto next_used = [&](int64_t e) {
            while (e < e1 && !(ent[e].mask & bmask)) e += kMW;
            return e;
        };
        int64_t e = next_used(e0 + w);
        int buf = 0;
        if (e < e1) stage_leaf(e, 0);
        while (e < e1) {
            const int64_t en = next_used(e + kMW);
            if (nbuf == 2 && en < e1) {   // a compile-time test
                stage_leaf(en, buf ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            const MergedEntry E = ent[e];
            const int64_t ri = E.r - rleaf0;
            const int nr = (int)(level_begin(bp.rn, bp.r_depth, ri + 1) - level_begin(bp.rn, bp.r_depth, ri));
            float dc[DP];
#pragma unroll
            for (int d = 0; d < DP; ++d)
                dc[d] = (ANCH && d < bp.D)
                            ? (float)(bp.qcenter[qnode * bp.D + d] - bp.rcenter[(int64_t)E.r * bp.D + d])
                            : 0.f;
            const float *rp = stage + (size_t)buf * lmax * NS;
            uint32_t m = (E.mask & bmask) >> sh;
            evals += (unsigned long long)__popc(m) * (unsigned long long)nr;
            while (m) {
                int ks[8];
                float c[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                int nj = 0;
                while (m && nj < (X2 ? 8 : 4)) {
                    const int k = __ffs(m) - 1;
                    m &= m - 1;
                    ks[nj] = k;
                    c[nj] = bp.negc[sh + k];
                    ++nj;
                }
                float part[QPL][8];
                if constexpr (X2) {
                    constexpr int QH = QPL / 2 > 0 ? QPL / 2 : 1;
                    f2_t xq2[QH][DP], dc2[DP], c2[8], part2[QH][8];
#pragma unroll
                    for (int h2 = 0; h2 < QH; ++h2)
#pragma unroll
                        for (int d = 0; d < DP; ++d) xq2[h2][d] = f2_pack(xq[2 * h2][d], xq[2 * h2 + 1][d]);
#pragma unroll
                    for (int d = 0; d < DP; ++d) dc2[d] = f2_pack(dc[d], dc[d]);
#pragma unroll
                    for (int k = 0; k < 8; ++k) c2[k] = f2_pack(c[k], c[k]);
                    const ulonglong2 *rp2 = reinterpret_cast<const ulonglong2 *>(rp);
                    switch (nj) {
                        case 1: leaf_terms_x2<DP, QPL, ANCH, 1>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 2: leaf_terms_x2<DP, QPL, ANCH, 2>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 3: leaf_terms_x2<DP, QPL, ANCH, 3>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 4: leaf_terms_x2<DP, QPL, ANCH, 4>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 5: leaf_terms_x2<DP, QPL, ANCH, 5>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 6: leaf_terms_x2<DP, QPL, ANCH, 6>(xq2, dc2, rp2, nr, c2, part2); break;
                        case 7: leaf_terms_x2<DP, QPL, ANCH, 7>(xq2, dc2, rp2, nr, c2, part2); break;
                        default: leaf_terms_x2<DP, QPL, ANCH, 8>(xq2, dc2, rp2, nr, c2, part2); break;
                    }
#pragma unroll
                    for (int h2 = 0; h2 < QH; ++h2)
#pragma unroll
                        for (int k = 0; k < 8; ++k) f2_unpack(part2[h2][k], part[2 * h2][k], part[2 * h2 + 1][k]);
                } else {
                    const float4 *rp4 = reinterpret_cast<const float4 *>(rp);
                    switch (nj) {
                        case 1: leaf_terms<DP, QPL, ANCH, 1>(xq, dc, rp4, nr, c, part); break;
                        case 2: leaf_terms<DP, QPL, ANCH, 2>(xq, dc, rp4, nr, c, part); break;
                        case 3: leaf_terms<DP, QPL, ANCH, 3>(xq, dc, rp4, nr, c, part); break;
                        default: leaf_terms<DP, QPL, ANCH, 4>(xq, dc, rp4, nr, c, part); break;
                    }
                }
                for (int k = 0; k < nj; ++k) {
#pragma unroll
                    for (int s = 0; s < QPL; ++s) {
                        const int slot = (ks[k] * QPL + s) * 32 + lane;
                        const float y = part[s][k] - kcmp[slot];
                        const float t = ksum[slot] + y;
                        kcmp[slot] = (t - ksum[slot]) - y;
                        ksum[slot] = t;
                    }
                }
            }
            __syncwarp();   // everyone is done with this buffer before it is refilled
            if constexpr (nbuf == 2)
                buf ^= 1;
            else if (en < e1)
                stage_leaf(en, 0);
            e = en;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < KS; t += blockDim.x) {
            const int k = t / (QPL * 32), s = (t / 32) % QPL, ln = t % 32;
            const int qq = ln + 32 * s;
            const int bit = sh + k;
            if (qq >= nq || bit >= nh) continue;
            double v = 0.0;
            for (int ww = 0; ww < kMW; ++ww) {
                const float *ks2 = sm_f + (size_t)ww * per_warp;
                v += (double)ks2[t] - (double)ks2[KS + t];
            }
            if (v != 0.0) atomicAdd(&bp.Gq[(qb + qq) * nh + bp.jcol[bit]], v * wmax);
        }
        __syncthreads();
    }
    if (bp.evals && lane == 0 && evals) atomicAdd(bp.evals, evals * (unsigned long long)nq);
}

template <int DP>
static int launch_merged_dp(int qpl, bool anch, const MergedParams &bp, const MergedEntry *ent, const long long *off,
                            int64_t lq, int lmax, cudaStream_t st) {
    constexpr int NT = RefRec<float, DP>::NT;
    // shared memory sized from the instantiated QPL (the kernel indexes with it)
#define GS_M(Q, A)                                                                                  \
    do {                                                                                            \
        const size_t ns = merged_x2(DP, Q) ? 2 * NT : NT;                                            \
        const size_t sm =                                                                           \
            (size_t)kMW * (2 * kBlk * (Q) * 32 + merged_nbuf(DP, Q) * lmax * ns) * sizeof(float);    \
        if (sm > 220 * 1024) return GS_ERR_UNSUPPORTED;                                             \
        allow_max_smem((const void *)k_basecase_merged<DP, Q, A>);                                   \
        k_basecase_merged<DP, Q, A><<<(unsigned)lq, 32 * kMW, sm, st>>>(bp, ent, off, lq, lmax);    \
    } while (0)
    if (anch) {
        if (qpl <= 1) GS_M(1, true); else if (qpl <= 2) GS_M(2, true); else GS_M(4, true);
    } else {
        if (qpl <= 1) GS_M(1, false); else if (qpl <= 2) GS_M(2, false); else GS_M(4, false);
    }
#undef GS_M
    return GS_OK;
}

// shared memory of the merged kernel for records of NT floats, query slots
// per lane qpl (instantiated as 1, 2 or 4) and leaves of at most lmax points
static size_t merged_smem(int DP, int NT, int qpl, int lmax) {
    const int Q = qpl <= 1 ? 1 : (qpl <= 2 ? 2 : 4);
    const size_t ns = merged_x2(DP, Q) ? 2 * NT : NT;
    return (size_t)kMW * (2 * kBlk * Q * 32 + merged_nbuf(DP, Q) * lmax * ns) * sizeof(float);
}

static void merged_shape(const TraversalIn &in, int &qpl, int &lmax) {
    const int64_t lq = 1ll << in.qt->depth, lr = 1ll << in.rt->depth;
    const int64_t maxq = (in.qt->n + lq - 1) / lq;
    qpl = (int)((maxq + 31) / 32);
    lmax = (int)((in.rt->n + lr - 1) / lr);
}

bool merged_base_possible(const TraversalIn &in) {
    const int64_t lq = 1ll << in.qt->depth, lr = 1ll << in.rt->depth;
    int qpl, lmax;
    merged_shape(in, qpl, lmax);
    const int DP = dp_for(in.D);
    const int NT = (int)(((DP + 1) * sizeof(float) + 15) / 16) * 4;
    (void)lq;
    (void)lr;
    return in.nh <= 32 && qpl <= 4 && merged_smem(DP, NT, qpl, lmax) <= 220 * 1024;
}

// records with every float duplicated, for the packed path
__global__ void k_dup_records(const float *__restrict__ rec, int64_t nf, float2 *rec2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = rec[i];
        rec2[i] = make_float2(v, v);
    }
}

int run_basecase_merged(const TraversalIn &in, FrontierBufs &fb, double *Gq, int DP, CallCtx &cx) {
    cudaStream_t st = cx.st;
    const int64_t lq = 1ll << in.qt->depth, lr = 1ll << in.rt->depth;
    const int64_t qleaf0 = lq - 1, rleaf0 = lr - 1;
    cx.phase(GS_PH_BASE);
    if (fb.n_base_groups == 0) {
        cx.phase(GS_PH_OTHER);
        return GS_OK;
    }
    int32_t *gidx = nullptr;   // lq x 32: base group of (query leaf, mask bit), -1 if none
    long long *off = nullptr;
    MergedEntry *ent = nullptr, *ent_dir = nullptr;
    long long *off_dir = nullptr;
    float *rec2 = nullptr;
    // a failed call frees what this phase holds, so the pool gets it back
    auto release = [&]() {
        if (gidx) cudaFreeAsync(gidx, st);
        if (off) cudaFreeAsync(off, st);
        if (ent) cudaFreeAsync(ent, st);
        if (ent_dir) cudaFreeAsync(ent_dir, st);
        if (off_dir) cudaFreeAsync(off_dir, st);
        if (rec2) cudaFreeAsync(rec2, st);
    };
#define GS_TRY_M(call)                        \
    do {                                      \
        cudaError_t e__ = (call);             \
        if (e__ != cudaSuccess) {             \
            release();                        \
            return cuda_fail(e__, #call);     \
        }                                     \
    } while (0)
    GS_TRY_M(dev_malloc_async((void **)&gidx, (size_t)lq * 32 * sizeof(int32_t), st));
    GS_TRY_M(cudaMemsetAsync(gidx, 0xFF, (size_t)lq * 32 * sizeof(int32_t), st));
    GS_TRY_M(dev_malloc_async((void **)&off, (size_t)(lq + 2) * sizeof(long long), st));
    const int grid = fb.grid_warps / 8;
    // mask bit of each bandwidth: its rank in ascending h
    int order[64];
    for (int j = 0; j < in.nh; ++j) order[j] = j;
    for (int a = 1; a < in.nh; ++a)
        for (int b = a; b > 0 && in.h[order[b]] < in.h[order[b - 1]]; --b) {
            const int t = order[b];
            order[b] = order[b - 1];
            order[b - 1] = t;
        }
    BitMap bmap;
    for (int b = 0; b < in.nh; ++b) bmap.rank[order[b]] = (int8_t)b;
    k_row_groups<<<grid, 256, 0, st>>>(fb.base_groups, fb.n_base_groups, qleaf0, bmap, gidx, (Ingest *)in.ing);
    const unsigned mgrid = (unsigned)(lq < 4096 ? lq : 4096);
    GS_TRY_M(allow_max_smem((const void *)k_row_masks<false>));
    GS_TRY_M(allow_max_smem((const void *)k_row_masks<true>));
    k_row_masks<false><<<mgrid, kMergeThreads, kSlice * sizeof(uint32_t), st>>>(fb.base_groups, fb.base_r, gidx, lq, lr,
                                                                             rleaf0, off, nullptr);
    cx.launches += 2;
    if (int rc0 = scan_i64(off, lq, off + lq, cx)) {
        release();
        return rc0;
    }
    // the entries: at most one per base-list entry (each has a bandwidth bit),
    // so small calls size them by that and skip reading the exact count; the
    // tensor-core split needs the count on the host
    const bool tc = tc_base_enabled(in.D, in.qt->dtype, in.flags, in.qt->n, in.qt->depth, in.rt->n, in.rt->depth,
                                    in.nh);
    long long total = 0;
    if (!tc && (double)fb.n_base * sizeof(MergedEntry) <= 64.0 * 1024 * 1024) {
        total = fb.n_base;
    } else {
        GS_TRY_M(cudaMemcpyAsync(&total, off + lq, sizeof(total), cudaMemcpyDeviceToHost, st));
        GS_TRY_M(cudaStreamSynchronize(st));
    }
    GS_TRY_M(dev_malloc_async((void **)&ent, (size_t)(total > 0 ? total : 1) * sizeof(MergedEntry), st));
    k_row_masks<true><<<mgrid, kMergeThreads, kSlice * sizeof(uint32_t), st>>>(fb.base_groups, fb.base_r, gidx, lq, lr,
                                                                            rleaf0, off, ent);
    cx.launches += 1;
    cudaFreeAsync(gidx, st);
    gidx = nullptr;
    int rc = cx.check("merge base pairs");
    if (!rc) {
        MergedParams bp;
        memset(&bp, 0, sizeof(bp));
        bp.qrec = in.qt->rec;
        bp.rrec = in.rt->rec;
        bp.qn = in.qt->n;
        bp.rn = in.rt->n;
        bp.q_depth = in.qt->depth;
        bp.r_depth = in.rt->depth;
        bp.qcenter = in.qt->center;
        bp.rcenter = in.rt->center;
        bp.D = in.D;
        bp.nh = in.nh;
        for (int b = 0; b < in.nh; ++b) {
            const double hb = in.h[order[b]];
            bp.negc[b] = (float)(-1.4426950408889634 / (2.0 * hb * hb));
            bp.jcol[b] = order[b];
        }
        bp.Gq = Gq;
        bp.ing = in.ing;
        bp.evals = fb.evals;
        // 9 <= D <= 16: the leaf pairs that pass the tensor-core error guard are
        // summed there; the direct kernel below takes the rest
        const MergedEntry *ent_run = ent;
        const long long *off_run = off;
        if (tc) {
            double h_by_bit[32];
            for (int b = 0; b < 32; ++b) h_by_bit[b] = b < in.nh ? in.h[order[b]] : 1.0;
            rc = run_basecase_tc(in, ent, off, lq, total, bp.negc, bp.jcol, h_by_bit, Gq, &ent_dir, &off_dir,
                                 fb.evals, cx);
            if (rc) {
                release();
                cx.phase(GS_PH_OTHER);
                return rc;
            }
            ent_run = ent_dir;
            off_run = off_dir;
        }
        int qpl, lmax;
        merged_shape(in, qpl, lmax);
        const bool anch = in.qt->dtype == GS_F64;
        const int Q = qpl <= 1 ? 1 : (qpl <= 2 ? 2 : 4);
        if (merged_x2(DP, Q)) {
            const int64_t nf = in.rt->n * (int64_t)in.rt->rec_stride;
            GS_TRY_M(dev_malloc_async((void **)&rec2, (size_t)nf * 2 * sizeof(float), st));
            k_dup_records<<<grid, 256, 0, st>>>(in.rt->rec, nf, (float2 *)rec2);
            cx.launches += 1;
            bp.rrec2 = rec2;
        }
        cx.mark(CallCtx::kTimerBase + 1);
        switch (DP) {
            case 1: rc = launch_merged_dp<1>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 2: rc = launch_merged_dp<2>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 3: rc = launch_merged_dp<3>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 4: rc = launch_merged_dp<4>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 5: rc = launch_merged_dp<5>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 6: rc = launch_merged_dp<6>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 7: rc = launch_merged_dp<7>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 8: rc = launch_merged_dp<8>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 12: rc = launch_merged_dp<12>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 16: rc = launch_merged_dp<16>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            case 24: rc = launch_merged_dp<24>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
            default: rc = launch_merged_dp<32>(qpl, anch, bp, ent_run, off_run, lq, lmax, st); break;
        }
        cx.mark(-1);
        cx.launches += 1;
        cx.launches_base += 1;
        if (!rc) rc = cx.check("k_basecase_merged");
    }
    release();
#undef GS_TRY_M
    cx.phase(GS_PH_OTHER);
    if (rc) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "merged base case launch");
    return GS_OK;
}

}  // namespace gs
