// td_dist.cuh -- the square root shared by every FP32 direct distance kernel, and the packed
// two-lane FP32 operations (sub.rn.f32x2 / fma.rn.f32x2, sm_100+) some of them use: each lane
// of a packed operation is rounded exactly as the scalar operation would be.
#pragma once

#include <cuda_runtime.h>

namespace td {

// The square root that turns a sum of squared differences into a distance (Sec. IV's f(i,j)):
// the hardware approximation sqrt.approx.f32 (subnormal inputs kept, sqrt(+0) = +0), not the
// correctly rounded sqrt.rn.f32.  Its error is a couple of units in the last place at most
// (checked through td_edm at d = 1, where the exact answer is |a - b|), far inside the 2e-6
// relative tolerance the distance maps are held to, and it saves the refinement steps that
// took about a quarter of the issue slots of the map at three features.  Every FP32 direct
// distance in the library goes through it, so all strategies and kernels agree bit for bit.
__device__ __forceinline__ float dist_sqrt(float s)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(s));
    return r;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long sub_f32x2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace td
