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
//
// Expanded squared distance (FP32 points, D <= 8, not in the paper): with u =
// q - c_R and v = r - c_R about the reference leaf's FP32 centre,
// ||q - r||^2 = (|v|^2 - 2 u.v) + |u|^2.  Per reference the records hold
// -2v, |v|^2 and l = log2(w / w_max); per (query, leaf pair) |u|^2 is formed
// once; per (query, reference) D fused multiply-adds and one addition replace
// the D subtractions and D multiply-adds of the direct form.  Error (first
// order in u = 2^-24, rho_R the Euclidean radius of R about c_R, d =
// ||q - r||, arg = c d^2 + l):
//   |arg~ - arg| <= |c| u [(D+4) d^2 + (4D+4) d rho_R + 5D rho_R^2] + u |arg~|
// (u and v rounded once each: 2 d (|u| + |v|); |u|^2 and |v|^2 as FMA chains:
// D |u|^2 and D |v|^2; the chain -2 u.v + |v|^2: D (|v|^2 + 2 |u| |v|); the
// addition of |u|^2 and c's rounding: d^2 each; the last FMA: |arg|), with
// |u| <= d + rho_R and |v| <= rho_R.  The relative part is charged like the
// direct kernel's argument rounding (D+5 there with l's rounding, D+6 here),
// over exponents down to 2^-64; the absolute part, at d <= 9.42 h and the bandwidth h of
// each mask bit, must stay within tau = 2^kXpGuardLog2 in log2 units, else
// that bit of the leaf pair stays with the direct kernel.  The traversal's
// FP32 charge carries ln2 (128 u + tau) whenever this path is enabled (two
// roundings of the argument, one of them slack).
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
    // expanded-distance path
    const float *rxp;        // per reference: (-2 v_d, -2 v_d) for d < DP, (|v|^2, |v|^2), (l, l), padding
    const float *rc32;       // per reference leaf: FP32 centre c_R (8 floats)
    unsigned long long *evals_x;   // terms of this kernel (besides evals)
};

// floats per expanded-distance reference record: DP + 2 duplicated pairs,
// rounded up to 16-byte units
__host__ __device__ constexpr int xp_rec_floats(int DP) { return ((2 * (DP + 2)) + 3) / 4 * 4; }

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

// leaf_terms_x2 on the expanded squared distance: two query slots per
// register pair; the staged record of a reference is (m_d, m_d) for
// m_d = -2 v_d, then (|v|^2, |v|^2) and (l, l), l = log2(w / w_max); per slot
// pair u2 holds the queries' u = q - c_R and b2 their |u|^2.  Per (query,
// reference) D FFMAs (|v|^2 - 2 u.v) and one FADD (+ |u|^2); per bandwidth
// one FFMA (argument c_k d^2 + l), one ex2 and one FADD, as the direct form.
template <int DP, int QPL, int NJ>
__device__ __forceinline__ void leaf_terms_xp(const f2_t (&u2)[QPL / 2][DP], const f2_t (&b2)[QPL / 2],
                                              const ulonglong2 *rp, int nr, const f2_t (&c)[8],
                                              f2_t (&part)[QPL / 2][8]) {
    constexpr int NP = xp_rec_floats(DP) / 2;   // pairs per staged record
#pragma unroll
    for (int s = 0; s < QPL / 2; ++s)
#pragma unroll
        for (int k = 0; k < 8; ++k) part[s][k] = 0ull;
#pragma unroll 4
    for (int i = 0; i < nr; ++i) {
        f2_t rv[NP];
#pragma unroll
        for (int v = 0; v < NP / 2; ++v) {
            const ulonglong2 u = rp[i * (NP / 2) + v];
            rv[2 * v] = u.x;
            rv[2 * v + 1] = u.y;
        }
#pragma unroll
        for (int s = 0; s < QPL / 2; ++s) {
            f2_t t = rv[DP];
#pragma unroll
            for (int d = 0; d < DP; ++d) t = f2_fma(u2[s][d], rv[d], t);
            t = f2_add(t, b2[s]);
#pragma unroll
            for (int k = 0; k < NJ; ++k) {
                float a0, a1;
                f2_unpack(f2_fma(t, c[k], rv[DP + 1]), a0, a1);
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

// Shared memory per warp: Kahan sums and compensations for one block of
// kBlk bandwidths (2 x kBlk x QPL x 32 floats), then two staging buffers of
// lmax reference records each.  Mask bits are bandwidths in ascending h, so
// the bandwidths a leaf pair needs are consecutive; the CTA makes one pass
// over its entries per block of kBlk bandwidths, blocks starting at the
// lowest bandwidth any of its entries needs.
//
// XP: the expanded squared distance (packed path, FP32 points only): the
// staged records are the expanded-distance ones and each leaf pair's query
// values are taken about the reference leaf's centre.
template <int DP, int QPL, bool ANCH, bool XP>
__global__ void __launch_bounds__(32 * kMW, XP ? (QPL == 2 ? 5 : 4) : 1)
k_basecase_merged(MergedParams bp, const MergedEntry *__restrict__ ent, const long long *__restrict__ off,
                  int64_t lq, int lmax) {
    constexpr int NT = RefRec<float, DP>::NT;
    constexpr bool X2 = merged_x2(DP, QPL);
    static_assert(!XP || (X2 && !ANCH), "the expanded form runs on the packed FP32 path");
    constexpr int NS = XP ? xp_rec_floats(DP) : (X2 ? 2 * NT : NT);   // floats per staged reference record
    constexpr int KS = kBlk * QPL * 32;
    extern __shared__ float sm_f[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x;
    const int64_t e0 = off[i], e1 = off[i + 1];
    if (e0 == e1) return;
    const int nh = bp.nh;
    const size_t per_warp = (size_t)2 * KS + (size_t)2 * lmax * NS;
    float *ksum = sm_f + (size_t)w * per_warp;
    float *kcmp = ksum + KS;
    float *stage = ksum + 2 * KS;   // 2 x lmax x NT floats, 16-byte aligned
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
        const float4 *src = reinterpret_cast<const float4 *>((XP ? bp.rxp : (X2 ? bp.rrec2 : bp.rrec)) + rb * NS);
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
    if (un == 0u) return;   // every entry of this row belongs to the other kernel
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
            if (en < e1) {
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
            // expanded form: u = q - c_R and |u|^2 per query slot (one leaf pair)
            constexpr int QX = XP ? QPL / 2 : 1;
            f2_t xu2[QX][DP], xb2[QX];
            if constexpr (XP) {
                float cr[DP];
#pragma unroll
                for (int d = 0; d < DP; ++d) cr[d] = bp.rc32[ri * 8 + d];
#pragma unroll
                for (int h2 = 0; h2 < QX; ++h2) {
                    float ua[DP], ub[DP];
#pragma unroll
                    for (int d = 0; d < DP; ++d) {
                        ua[d] = xq[2 * h2][d] - cr[d];
                        ub[d] = xq[2 * h2 + 1][d] - cr[d];
                    }
                    float ba = ua[0] * ua[0], bb = ub[0] * ub[0];
#pragma unroll
                    for (int d = 1; d < DP; ++d) {
                        ba = fmaf(ua[d], ua[d], ba);
                        bb = fmaf(ub[d], ub[d], bb);
                    }
#pragma unroll
                    for (int d = 0; d < DP; ++d) xu2[h2][d] = f2_pack(ua[d], ub[d]);
                    xb2[h2] = f2_pack(ba, bb);
                }
            }
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
                if constexpr (XP) {
                    constexpr int QH = QPL / 2;
                    f2_t c2[8], part2[QH][8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) c2[k] = f2_pack(c[k], c[k]);
                    const ulonglong2 *rp2 = reinterpret_cast<const ulonglong2 *>(rp);
                    switch (nj) {
                        case 1: leaf_terms_xp<DP, QPL, 1>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 2: leaf_terms_xp<DP, QPL, 2>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 3: leaf_terms_xp<DP, QPL, 3>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 4: leaf_terms_xp<DP, QPL, 4>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 5: leaf_terms_xp<DP, QPL, 5>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 6: leaf_terms_xp<DP, QPL, 6>(xu2, xb2, rp2, nr, c2, part2); break;
                        case 7: leaf_terms_xp<DP, QPL, 7>(xu2, xb2, rp2, nr, c2, part2); break;
                        default: leaf_terms_xp<DP, QPL, 8>(xu2, xb2, rp2, nr, c2, part2); break;
                    }
#pragma unroll
                    for (int h2 = 0; h2 < QH; ++h2)
#pragma unroll
                        for (int k = 0; k < 8; ++k) f2_unpack(part2[h2][k], part[2 * h2][k], part[2 * h2 + 1][k]);
                } else if constexpr (X2) {
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
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (k >= nj) break;
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
            buf ^= 1;
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
    if (XP && bp.evals_x && lane == 0 && evals) atomicAdd(bp.evals_x, evals * (unsigned long long)nq);
}

template <int DP>
static int launch_merged_dp(int qpl, bool anch, bool xp, const MergedParams &bp, const MergedEntry *ent,
                            const long long *off, int64_t lq, int lmax, cudaStream_t st) {
    constexpr int NT = RefRec<float, DP>::NT;
    // shared memory sized from the instantiated QPL (the kernel indexes with it)
#define GS_M(Q, A, X)                                                                               \
    do {                                                                                            \
        const size_t ns = (X) ? xp_rec_floats(DP) : (merged_x2(DP, Q) ? 2 * NT : NT);                \
        const size_t sm = (size_t)kMW * (2 * kBlk * (Q) * 32 + 2 * lmax * ns) * sizeof(float);     \
        if (sm > 220 * 1024) return GS_ERR_UNSUPPORTED;                                             \
        allow_max_smem((const void *)k_basecase_merged<DP, Q, A, X>);                                \
        k_basecase_merged<DP, Q, A, X><<<(unsigned)lq, 32 * kMW, sm, st>>>(bp, ent, off, lq, lmax); \
    } while (0)
    if (xp) {
        if constexpr (DP <= 8) {
            if (qpl <= 1 || anch) return GS_ERR_UNSUPPORTED;
            if (qpl <= 2) GS_M(2, false, true); else GS_M(4, false, true);
            return GS_OK;
        } else {
            return GS_ERR_UNSUPPORTED;
        }
    }
    if (anch) {
        if (qpl <= 1) GS_M(1, true, false); else if (qpl <= 2) GS_M(2, true, false); else GS_M(4, true, false);
    } else {
        if (qpl <= 1) GS_M(1, false, false); else if (qpl <= 2) GS_M(2, false, false); else GS_M(4, false, false);
    }
#undef GS_M
    return GS_OK;
}

// shared memory of the merged kernel for records of NT floats, query slots
// per lane qpl (instantiated as 1, 2 or 4) and leaves of at most lmax points
static size_t merged_smem(int DP, int NT, int qpl, int lmax, bool xp = false) {
    const int Q = qpl <= 1 ? 1 : (qpl <= 2 ? 2 : 4);
    const size_t ns = xp ? xp_rec_floats(DP) : (merged_x2(DP, Q) ? 2 * NT : NT);
    return (size_t)kMW * (2 * kBlk * Q * 32 + 2 * lmax * ns) * sizeof(float);
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
    return in.nh <= 32 && qpl <= 4 && merged_smem(DP, NT, qpl, lmax) <= 220 * 1024 &&
           (DP > 8 || merged_smem(DP, NT, qpl, lmax, true) <= 220 * 1024);
}

// ---------------------------------------------------------------------------
// expanded-distance path: per reference leaf its FP32 centre, the records
// about it and the mask bits whose bandwidth passes the error guard
// ---------------------------------------------------------------------------
constexpr int kXpGuardLog2 = -13;   // tau: absolute exponent error allowed (log2 units)

struct XpGuard {
    double k_lin;       // u log2(e) / 2 (4D+7) 9.42        (times rho_R / h)
    double k_sq;        // u log2(e) / 2 (5D+2)             (times rho_R^2 / h^2)
    double tau;
    double inv_h[32];   // by mask bit: 1 / h
    int nh;
};

// One CTA (128 threads) per reference leaf.  Records: m_d = -2 fl(r_d - c_d),
// |v|^2 (the FMA chain the error bound assumes) and the direct records' l,
// each duplicated; the Euclidean radius about c_R in FP64 (x and c are FP32,
// so x - c is exact), rounded up; pass[i] = the mask bits b whose guard
// u log2(e)/2 [(4D+7) 9.42 rho_R / h_b + (5D+2) rho_R^2 / h_b^2] <= tau
// (coefficients above the bound's first-order ones: second-order slack).
// The guard decreases with h and bits rank bandwidths by ascending h, so the
// passing bits are the top ones.
template <int DP>
__global__ void __launch_bounds__(128) k_xp_leaves(const float *__restrict__ rec, int rec_stride, int64_t n,
                                                   int depth, const double *__restrict__ center, int D,
                                                   XpGuard g, float *rxp, float *c32, uint32_t *pass) {
    constexpr int NS = xp_rec_floats(DP);
    __shared__ double s_rad[4];
    const int64_t i = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t node = ((int64_t)1 << depth) - 1 + i;
    const int64_t b = level_begin(n, depth, i), e = level_begin(n, depth, i + 1);
    float c[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) c[d] = d < D ? (float)center[node * D + d] : 0.f;
    double r2 = 0.0;
    for (int64_t p = b + t; p < e; p += blockDim.x) {
        float v[DP];
        double q2 = 0.0;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float x = d < D ? rec[p * rec_stride + d] : 0.f;
            v[d] = x - c[d];
            const double dx = (double)x - (double)c[d];
            q2 += dx * dx;
        }
        r2 = fmax(r2, q2);
        float s = v[0] * v[0];
#pragma unroll
        for (int d = 1; d < DP; ++d) s = fmaf(v[d], v[d], s);
        const float l = rec[p * rec_stride + DP];   // log2(w / w_max), as the direct kernel's records
        float *o = rxp + p * NS;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            o[2 * d] = -2.f * v[d];
            o[2 * d + 1] = -2.f * v[d];
        }
        o[2 * DP] = s;
        o[2 * DP + 1] = s;
        o[2 * DP + 2] = l;
        o[2 * DP + 3] = l;
#pragma unroll
        for (int k = 2 * DP + 4; k < NS; ++k) o[k] = 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if ((t & 31) == 0) s_rad[t >> 5] = r2;
    __syncthreads();
    if (t == 0) {
        r2 = fmax(fmax(s_rad[0], s_rad[1]), fmax(s_rad[2], s_rad[3]));
        const double rad = sqrt(r2) * (1.0 + 1e-12);
        for (int d = 0; d < 8; ++d) c32[i * 8 + d] = d < DP ? c[d] : 0.f;
        int bmin = 32;
        for (int bit = 0; bit < g.nh; ++bit) {
            const double x = rad * g.inv_h[bit];
            if (g.k_lin * x + g.k_sq * x * x <= g.tau) {
                bmin = bit;
                break;
            }
        }
        pass[i] = bmin >= 32 ? 0u : (0xFFFFFFFFu << bmin);
    }
}

// Every merged entry split by its reference leaf's passing bits: those go to
// ent_x (same offsets), the rest stay in ent.
__global__ void k_xp_split(MergedEntry *ent, int64_t total, const uint32_t *__restrict__ pass, int64_t rleaf0,
                           MergedEntry *ent_x) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        MergedEntry E = ent[e];
        const uint32_t pm = pass[E.r - rleaf0];
        MergedEntry X;
        X.r = E.r;
        X.mask = E.mask & pm;
        ent_x[e] = X;
        E.mask &= ~pm;
        ent[e] = E;
    }
}

bool xp_base_enabled(int D, int dtype, int flags, int64_t qn, int q_depth, int64_t rn, int r_depth, int nh) {
    if (D > 8 || dtype != GS_F32 || (flags & GS_FLAG_NO_XP) || nh > 32) return false;
    const int64_t maxq = (qn + (1ll << q_depth) - 1) >> q_depth;
    const int64_t maxr = (rn + (1ll << r_depth) - 1) >> r_depth;
    return maxq > 32 && maxq <= 128 && maxr <= 128;
}

// extra charge on top of the direct base case's: two more roundings of the
// exponent argument over exponents down to 2^-64 (one needed, one slack) and
// the guard's tau
double xp_charge() {
    const double u = 5.9604644775390625e-08;
    return 0.6931471805599453 * (64.0 * 2.0 * u + ldexp(1.0, kXpGuardLog2));
}

template <int DP>
static void launch_xp_leaves(const TraversalIn &in, const XpGuard &g, float *rxp, float *c32, uint32_t *pass,
                             cudaStream_t st) {
    const TreeDev &t = *in.rt;
    k_xp_leaves<DP><<<(unsigned)(1ll << t.depth), 128, 0, st>>>(t.rec, t.rec_stride, t.n, t.depth, t.center, t.D,
                                                               g, rxp, c32, pass);
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
    MergedEntry *ent = nullptr, *ent_dir = nullptr, *ent_x = nullptr;
    long long *off_dir = nullptr;
    float *rec2 = nullptr, *rxp = nullptr, *xc32 = nullptr;
    uint32_t *xpass = nullptr;
    // a failed call frees what this phase holds, so the pool gets it back
    auto release = [&]() {
        if (gidx) cudaFreeAsync(gidx, st);
        if (off) cudaFreeAsync(off, st);
        if (ent) cudaFreeAsync(ent, st);
        if (ent_dir) cudaFreeAsync(ent_dir, st);
        if (off_dir) cudaFreeAsync(off_dir, st);
        if (rec2) cudaFreeAsync(rec2, st);
        if (ent_x) cudaFreeAsync(ent_x, st);
        if (rxp) cudaFreeAsync(rxp, st);
        if (xc32) cudaFreeAsync(xc32, st);
        if (xpass) cudaFreeAsync(xpass, st);
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
    long long total = 0;
    GS_TRY_M(cudaMemcpyAsync(&total, off + lq, sizeof(total), cudaMemcpyDeviceToHost, st));
    GS_TRY_M(cudaStreamSynchronize(st));
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
        if (tc_base_enabled(in.D, in.qt->dtype, in.flags, in.qt->n, in.qt->depth, in.rt->n, in.rt->depth, in.nh)) {
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
        // FP32, D <= 8: the bits whose reference leaf passes the guard go to
        // the expanded-distance kernel (launched first), the rest stay here
        const bool xp = xp_base_enabled(in.D, in.qt->dtype, in.flags, in.qt->n, in.qt->depth, in.rt->n,
                                        in.rt->depth, in.nh) &&
                        DP <= 8 && merged_x2(DP, Q) && !anch && ent_run == ent;
        if (xp) {
            constexpr double u = 5.9604644775390625e-08, hl2e = 0.5 * 1.4426950408889634;
            XpGuard g;
            memset(&g, 0, sizeof(g));
            g.k_lin = u * hl2e * (4.0 * in.D + 7.0) * 9.42;
            g.k_sq = u * hl2e * (5.0 * in.D + 2.0);
            g.tau = ldexp(1.0, kXpGuardLog2);
            g.nh = in.nh;
            for (int b = 0; b < in.nh; ++b) g.inv_h[b] = 1.0 / in.h[order[b]];
            const int NSX = xp_rec_floats(DP);
            GS_TRY_M(dev_malloc_async((void **)&rxp, (size_t)in.rt->n * NSX * sizeof(float), st));
            GS_TRY_M(dev_malloc_async((void **)&xc32, (size_t)lr * 8 * sizeof(float), st));
            GS_TRY_M(dev_malloc_async((void **)&xpass, (size_t)lr * sizeof(uint32_t), st));
            GS_TRY_M(dev_malloc_async((void **)&ent_x, (size_t)(total > 0 ? total : 1) * sizeof(MergedEntry), st));
            switch (DP) {
                case 1: launch_xp_leaves<1>(in, g, rxp, xc32, xpass, st); break;
                case 2: launch_xp_leaves<2>(in, g, rxp, xc32, xpass, st); break;
                case 3: launch_xp_leaves<3>(in, g, rxp, xc32, xpass, st); break;
                case 4: launch_xp_leaves<4>(in, g, rxp, xc32, xpass, st); break;
                case 5: launch_xp_leaves<5>(in, g, rxp, xc32, xpass, st); break;
                case 6: launch_xp_leaves<6>(in, g, rxp, xc32, xpass, st); break;
                case 7: launch_xp_leaves<7>(in, g, rxp, xc32, xpass, st); break;
                default: launch_xp_leaves<8>(in, g, rxp, xc32, xpass, st); break;
            }
            if (total > 0)
                k_xp_split<<<grid, 256, 0, st>>>(ent, total, xpass, rleaf0, ent_x);
            cx.launches += 2;
            rc = cx.check("expanded-distance records");
            if (!rc) {
                MergedParams bx = bp;
                bx.rxp = rxp;
                bx.rc32 = xc32;
                bx.evals_x = fb.evals ? fb.evals + 2 : nullptr;
                cx.mark(CallCtx::kTimerBase);
                switch (DP) {
                    case 1: rc = launch_merged_dp<1>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 2: rc = launch_merged_dp<2>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 3: rc = launch_merged_dp<3>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 4: rc = launch_merged_dp<4>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 5: rc = launch_merged_dp<5>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 6: rc = launch_merged_dp<6>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    case 7: rc = launch_merged_dp<7>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                    default: rc = launch_merged_dp<8>(qpl, false, true, bx, ent_x, off, lq, lmax, st); break;
                }
                cx.mark(-1);
                cx.launches += 1;
                cx.launches_base += 1;
                if (!rc) rc = cx.check("k_basecase_merged (expanded)");
            }
        }
        if (!rc && merged_x2(DP, Q)) {
            const int64_t nf = in.rt->n * (int64_t)in.rt->rec_stride;
            GS_TRY_M(dev_malloc_async((void **)&rec2, (size_t)nf * 2 * sizeof(float), st));
            k_dup_records<<<grid, 256, 0, st>>>(in.rt->rec, nf, (float2 *)rec2);
            cx.launches += 1;
            bp.rrec2 = rec2;
        }
        if (!rc) {
            cx.mark(CallCtx::kTimerBase + 1);
            switch (DP) {
                case 1: rc = launch_merged_dp<1>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 2: rc = launch_merged_dp<2>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 3: rc = launch_merged_dp<3>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 4: rc = launch_merged_dp<4>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 5: rc = launch_merged_dp<5>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 6: rc = launch_merged_dp<6>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 7: rc = launch_merged_dp<7>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 8: rc = launch_merged_dp<8>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 12: rc = launch_merged_dp<12>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 16: rc = launch_merged_dp<16>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                case 24: rc = launch_merged_dp<24>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
                default: rc = launch_merged_dp<32>(qpl, anch, false, bp, ent_run, off_run, lq, lmax, st); break;
            }
            cx.mark(-1);
            cx.launches += 1;
            cx.launches_base += 1;
            if (!rc) rc = cx.check("k_basecase_merged");
        }
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
