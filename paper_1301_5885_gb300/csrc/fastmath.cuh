// fastmath.cuh -- the hardware approximate functions used by the FP32-pair
// kernels (PTX rsqrt.approx and ex2.approx, both on the MUFU unit).
#pragma once

namespace pb {

// 1/sqrt(x); +inf for x = 0; subnormals flushed to zero.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 2^x; exactly 1 for x = +0 and -0.
__device__ __forceinline__ float exp2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

}  // namespace pb
