// Device-wide exclusive prefix sum of int64 counts (three phases over a
// fixed grid: per-block totals, a scan of the block totals, per-block
// rescans).  Used to turn per-item work counts into offsets.
#include "gs_internal.h"

namespace gs {

constexpr int kScanBlocks = 512;
constexpr int kScanThreads = 256;

__device__ __forceinline__ long long blk_excl(long long v, long long *tot) {
    __shared__ long long ws[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const long long s = lane < kScanThreads / 32 ? ws[lane] : 0;
        long long si = s;
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += u;
        }
        if (lane < kScanThreads / 32) ws[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *tot = si;
    }
    __syncthreads();
    const long long r = ws[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sum(const long long *v, int64_t n, long long *part) {
    __shared__ long long tot;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t a = blockIdx.x * chunk, b = min(a + chunk, n);
    long long s = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) s += v[i];
    blk_excl(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_part(long long *part, long long *total) {
    __shared__ long long tot;
    long long carry = 0;
    for (int b0 = 0; b0 < kScanBlocks; b0 += kScanThreads) {
        const long long v = part[b0 + threadIdx.x];
        const long long e = blk_excl(v, &tot);
        part[b0 + threadIdx.x] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(long long *v, int64_t n, const long long *part) {
    __shared__ long long tot;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t a = blockIdx.x * chunk, b = min(a + chunk, n);
    long long carry = part[blockIdx.x];
    for (int64_t t0 = a; t0 < b; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        const long long x = i < b ? v[i] : 0;
        const long long e = blk_excl(x, &tot);
        if (i < b) v[i] = carry + e;
        carry += tot;
    }
}

int scan_i64(long long *v, int64_t n, long long *total, CallCtx &cx) {
    long long *part = nullptr;
    GS_CUDA_TRY(dev_malloc_async((void **)&part, kScanBlocks * sizeof(long long), cx.st));
    k_scan_sum<<<kScanBlocks, kScanThreads, 0, cx.st>>>(v, n, part);
    k_scan_part<<<1, kScanThreads, 0, cx.st>>>(part, total);
    k_scan_apply<<<kScanBlocks, kScanThreads, 0, cx.st>>>(v, n, part);
    cx.launches += 3;
    cudaFreeAsync(part, cx.st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "scan launch");
    return cx.check("scan");
}

}  // namespace gs
