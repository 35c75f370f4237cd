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

// Packed reference record for the kernel inner loops: DP coordinates
// (zero-padded beyond D), then l = log2(w / w_max), rounded up to 16-byte
// units.  A padding record has l = -inf and contributes exactly 0.
template <typename T, int DP>
struct RefRec {
    static constexpr int NV16 = (int)(((DP + 1) * sizeof(T) + 15) / 16);   // 16-byte units
    static constexpr int NT = NV16 * 16 / (int)sizeof(T);                  // T slots
};

}  // namespace gs
