// Pair-selector network (12 -> 64 -> 64 -> 5, ReLU): parameter layout and
// the FP32 inference used both by the selector inside the traversal and by
// gs_mlp_forward.  Every product and sum is rounded separately and inputs
// are taken in ascending order, so the scores are reproducible bit for bit
// by a plain CPU evaluation.
#pragma once

#include <stdint.h>

namespace gs {

constexpr int kMlpIn = 12, kMlpHid = 64, kMlpOut = 5;
// blob offsets (floats): mu[12], sc[12], W1[12][64], b1[64], W2[64][64], b2[64], W3[64][5], b3[5]
constexpr int kOffMu = 0, kOffSc = 12, kOffW1 = 24, kOffB1 = kOffW1 + kMlpIn * kMlpHid,
              kOffW2 = kOffB1 + kMlpHid, kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid,
              kOffB3 = kOffW3 + kMlpHid * kMlpOut, kMlpParams = kOffB3 + kMlpOut;
static_assert(kMlpParams == 5341, "parameter blob size");

__device__ __forceinline__ float relu_f(float a) { return a > 0.f ? a : 0.f; }

// a + b * c with the product rounded before the sum (the _rn intrinsics are
// never contracted into an FMA)
__device__ __forceinline__ float muladd_rn(float a, float b, float c) { return __fadd_rn(a, __fmul_rn(b, c)); }

// Scores o[5] of one input x[12]; w is the parameter blob (shared memory).
// Layer 1 units are produced one at a time and folded into the layer 2 sums
// at once, so only the 64 layer 2 sums stay live.
__device__ __forceinline__ void mlp_infer(const float *__restrict__ w, const float (&x)[kMlpIn], float (&o)[kMlpOut]) {
    float z[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) z[k] = __fmul_rn(__fsub_rn(x[k], w[kOffMu + k]), w[kOffSc + k]);
    float a2[kMlpHid];
#pragma unroll
    for (int j = 0; j < kMlpHid; ++j) a2[j] = w[kOffB2 + j];
#pragma unroll 1
    for (int i = 0; i < kMlpHid; ++i) {
        float a1 = w[kOffB1 + i];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) a1 = muladd_rn(a1, z[k], w[kOffW1 + k * kMlpHid + i]);
        const float h = relu_f(a1);
        const float *row = w + kOffW2 + i * kMlpHid;
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) a2[j] = muladd_rn(a2[j], h, row[j]);
    }
#pragma unroll
    for (int c = 0; c < kMlpOut; ++c) o[c] = w[kOffB3 + c];
#pragma unroll
    for (int j = 0; j < kMlpHid; ++j) {
        const float g = relu_f(a2[j]);
#pragma unroll
        for (int c = 0; c < kMlpOut; ++c) o[c] = muladd_rn(o[c], g, w[kOffW3 + j * kMlpOut + c]);
    }
}

// Piecewise-linear log2 in FP32: x = m 2^e with m in [1, 2) gives e + (m - 1);
// 0 and subnormals give -150, +inf gives 128.
__device__ __forceinline__ float plog2_f(float x) {
    if (!(x >= 0x1p-126f)) return -150.f;
    if (isinf(x)) return 128.f;
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 255u) - 127;
    const float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    return __fadd_rn((float)e, __fsub_rn(m, 1.f));
}

}  // namespace gs
