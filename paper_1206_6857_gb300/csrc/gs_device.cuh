// Device helpers shared by the summation kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// 2^x on the MUFU pipe, flush-to-zero.  The PTX ISA documents ex2.approx.f32
// with a maximum relative error of 2^-22 over its range (subnormal results
// flush to +0); an argument of -inf gives +0.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 values in one 64-bit register pair, for the packed f32x2
// instructions of sm_100-family GPUs: element-wise IEEE operations, so a
// packed result rounds exactly like the two scalar ones.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Packed reference record for the kernel inner loops: DP coordinates
// (zero-padded beyond D), then l = log2(w / w_max), rounded up to 16-byte
// units.  A padding record has l = -inf and contributes exactly 0.
template <typename T, int DP>
struct RefRec {
    static constexpr int NV16 = (int)(((DP + 1) * sizeof(T) + 15) / 16);   // 16-byte units
    static constexpr int NT = NV16 * 16 / (int)sizeof(T);                  // T slots
};

}  // namespace gs
