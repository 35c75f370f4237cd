// Leaf-leaf base case (DITOBase, Fig. 7): every query of a query leaf
// against every reference of the reference leaves the traversal left
// unpruned, for one bandwidth, summed exactly.
//
// Work unit: one base group = (query leaf Q, bandwidth j, list of reference
// leaves).  One warp owns a group; lane l holds query points l, l+32, ... of
// Q in registers (QPL per lane) and the warp streams the reference leaves:
// every reference record (FP32 coordinates + l_r = log2(w_r / w_max), 16-byte
// aligned) is read once per warp with a uniform-address load (one broadcast
// transaction from L1/L2), and each lane forms the squared distance in FP32
// from coordinate differences and adds 2^(d^2 * c_j + l_r) from the MUFU ex2
// unit.  Terms are summed in FP32 over one reference leaf, in compensated
// FP32 across leaves and in FP64 across warps; the group's per-query totals
// go to the sorted-order accumulator with FP64 atomics.  For FP64 input the records hold coordinates relative to
// their leaf centre and each leaf pair adds the FP64 centre difference
// (rounded once to FP32) to every coordinate difference.
#include <math.h>

#include "gs_device.cuh"
#include "gs_frontier.cuh"
#include "gs_internal.h"
#include "gs_tree.cuh"

namespace gs {

struct BaseParams {
    const float *qrec, *rrec;
    int64_t qn, rn;
    int q_depth, r_depth;
    const double *qcenter, *rcenter;   // for anchored (FP64-input) records
    int D, nh;
    float negc[64];                    // -log2(e) / (2 h_j^2)
    double *Gq;                        // sorted queries x nh
    const Ingest *ing;
    unsigned long long *evals;         // point-pair evaluations (statistics)
};

constexpr int kBaseWarps = 4;

// One CTA per base group; its warps take the group's reference leaves
// round-robin and their per-query sums are combined in shared memory before
// a single FP64 atomic per query.
template <int DP, int QPL, bool ANCH>
__global__ void __launch_bounds__(32 * kBaseWarps)
k_basecase(BaseParams bp, const Group *__restrict__ bgroups, const int32_t *__restrict__ base_r) {
    constexpr int NT = RefRec<float, DP>::NT;
    __shared__ double red[kBaseWarps][QPL * 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float wmax = __uint_as_float(bp.ing->wmax_bits);
    const int64_t qleaf0 = (1ll << bp.q_depth) - 1, rleaf0 = (1ll << bp.r_depth) - 1;
    const Group G = bgroups[blockIdx.x];
    const int64_t qi = G.q - qleaf0;
    const int64_t qb = level_begin(bp.qn, bp.q_depth, qi), qe = level_begin(bp.qn, bp.q_depth, qi + 1);
    const int nq = (int)(qe - qb);
    const float c = bp.negc[G.j];
    float xq[QPL][DP];
#pragma unroll
    for (int s = 0; s < QPL; ++s) {
        const int qq = lane + 32 * s;
        const int64_t pos = qb + (qq < nq ? qq : 0);
#pragma unroll
        for (int d = 0; d < DP; ++d) xq[s][d] = bp.qrec[pos * NT + d];
    }
    // summation: FP32 over one reference leaf, then a compensated (Kahan)
    // FP32 sum across leaves, FP64 across warps -- the scheme the FP32 error
    // charge covers ((L_R - 1) u for the leaf, 2 u for the compensated sum)
    // and the one of the merged base case; no FP64 work per leaf
    float ksum[QPL], kcmp[QPL];
#pragma unroll
    for (int s = 0; s < QPL; ++s) {
        ksum[s] = 0.f;
        kcmp[s] = 0.f;
    }
    unsigned long long grp_refs = 0;
    for (int k = w; k < G.cnt; k += kBaseWarps) {
        const int64_t rnode = base_r[G.off + k];
        const int64_t ri = rnode - rleaf0;
        const int64_t rb = level_begin(bp.rn, bp.r_depth, ri), re = level_begin(bp.rn, bp.r_depth, ri + 1);
        float dc[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) dc[d] = 0.f;
        if (ANCH) {
            for (int d = 0; d < bp.D; ++d)
                dc[d] = (float)(bp.qcenter[G.q * bp.D + d] - bp.rcenter[rnode * bp.D + d]);
        }
        float part[QPL];
#pragma unroll
        for (int s = 0; s < QPL; ++s) part[s] = 0.f;
        const float4 *rp = reinterpret_cast<const float4 *>(bp.rrec + rb * NT);
        const int nr = (int)(re - rb);
#pragma unroll 4
        for (int i = 0; i < nr; ++i) {
            float rv[NT];
#pragma unroll
            for (int v = 0; v < NT / 4; ++v) {
                const float4 f = __ldg(rp + i * (NT / 4) + v);
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
                part[s] += ex2_approx(fmaf(d2, c, l));
            }
        }
#pragma unroll
        for (int s = 0; s < QPL; ++s) {
            const float y = __fsub_rn(part[s], kcmp[s]);
            const float t = __fadd_rn(ksum[s], y);
            kcmp[s] = __fsub_rn(__fsub_rn(t, ksum[s]), y);
            ksum[s] = t;
        }
        grp_refs += (unsigned long long)nr;
    }
#pragma unroll
    for (int s = 0; s < QPL; ++s) red[w][s * 32 + lane] = (double)ksum[s] - (double)kcmp[s];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int s = 0; s < QPL; ++s) {
            const int qq = lane + 32 * s;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kBaseWarps; ++k) v += red[k][s * 32 + lane];
            if (qq < nq) atomicAdd(&bp.Gq[(qb + qq) * bp.nh + G.j], v * (double)wmax);
        }
    }
    if (bp.evals && lane == 0 && grp_refs) atomicAdd(bp.evals, grp_refs * (unsigned long long)nq);
}

template <int DP>
static void launch_dp(int qpl, bool anch, const BaseParams &bp, const FrontierState *fs, const Group *bg,
                      const int32_t *br, int64_t grid, cudaStream_t st) {
    (void)fs;
#define GS_L(Q, A) k_basecase<DP, Q, A><<<(unsigned)grid, 32 * kBaseWarps, 0, st>>>(bp, bg, br)
    if (anch) {
        if (qpl <= 1) GS_L(1, true); else if (qpl <= 2) GS_L(2, true); else GS_L(4, true);
    } else {
        if (qpl <= 1) GS_L(1, false); else if (qpl <= 2) GS_L(2, false); else GS_L(4, false);
    }
#undef GS_L
}

int run_basecase(const TraversalIn &in, FrontierBufs &fb, double *Gq, int DP, CallCtx &cx) {
    BaseParams bp;
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
    for (int j = 0; j < in.nh; ++j) bp.negc[j] = (float)(-1.4426950408889634 / (2.0 * in.h[j] * in.h[j]));
    bp.Gq = Gq;
    bp.ing = in.ing;
    bp.evals = fb.evals;
    const int64_t maxq = (in.qt->n + (1ll << in.qt->depth) - 1) >> in.qt->depth;
    const int qpl = (int)((maxq + 31) / 32);
    if (qpl > 4) {
        set_error("leaf size above 128 is not supported by the base case");
        return GS_ERR_ARG;
    }
    const bool anch = in.qt->dtype == GS_F64;
    const int64_t grid = fb.n_base_groups;
    cx.phase(GS_PH_BASE);
    if (grid == 0) {
        cx.phase(GS_PH_OTHER);
        return GS_OK;
    }
    cx.mark(CallCtx::kTimerBase + 1);
    switch (DP) {
        case 1: launch_dp<1>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 2: launch_dp<2>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 3: launch_dp<3>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 4: launch_dp<4>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 5: launch_dp<5>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 6: launch_dp<6>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 7: launch_dp<7>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 8: launch_dp<8>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 12: launch_dp<12>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 16: launch_dp<16>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        case 24: launch_dp<24>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
        default: launch_dp<32>(qpl, anch, bp, fb.fs, fb.base_groups, fb.base_r, grid, cx.st); break;
    }
    cx.mark(-1);
    cx.launches += 1;
    cx.launches_base += 1;
    if (int rc = cx.check("k_basecase")) return rc;
    cx.phase(GS_PH_OTHER);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "base case launch");
    return GS_OK;
}

}  // namespace gs
