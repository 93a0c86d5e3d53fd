// td_device.cuh -- device-side mapping functions for triangular-domain (td) problems.
//
// The paper's block-level mapping g(lambda) (arXiv:1308.1419, Sec. II-A, Eq. (theorem)) and
// the four strategies it is compared with (Sec. III-B): BB, UTM, RB and REC.  Every function
// returns coordinates in the lower triangle with diagonal: 0 <= j <= i.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace td {

// T(m) = m(m+1)/2, the row start of row m in the packed lower triangle (Eq. (matrix_indexing)).
__host__ __device__ __forceinline__ uint64_t tri(uint64_t m) { return (m * (m + 1)) >> 1; }

// g(lambda) of Eq. (theorem): i = floor(sqrt(1/4 + 2 lambda) - 1/2), j = lambda - T(i).
// sqrt(1/4 + 2 lambda) - 1/2 = (sqrt(8 lambda + 1) - 1) / 2.  The square root is taken the
// LTM-R way (Sec. III-A: sqrt(y) = y * rsqrt(y)), in FP32.  Instead of the paper's
// epsilon = 1e-4 repair, which it reports exact only up to N ~ 30720 at rho = 16, the row is
// corrected with exact 64-bit integer tests (the "block-level conditionals" the paper's
// conclusion proposes for larger ranges).  The FP32 estimate is within one row of the truth
// for lambda < 2^40, so one step in either direction suffices there.
__device__ __forceinline__ void ltm_g(uint64_t lam, uint32_t &i, uint32_t &j)
{
    const float y = __ull2float_rn(8ull * lam + 1ull);
    const float s = y * rsqrtf(y);
    uint32_t r = __float2uint_rz(fmaf(s, 0.5f, -0.5f));
    uint64_t t = tri(r);
    if (t > lam) {            // estimate one row too far down
        t -= r;
        --r;
    } else if (t + r + 1 <= lam) {  // one row too far up
        ++r;
        t += r;
    }
    i = r;
    j = static_cast<uint32_t>(lam - t);
}

// UTM (Avril et al., Sec. III-B) for a lower triangle of side N with its diagonal.  The
// strict upper triangle of side n = N + 1 has T(N) pairs; thread index k gives
//   a = floor(((2n+1) - sqrt(4n^2 - 4n - 8k + 1)) / 2),  row start K(a) = (a-1)(2n-a)/2,
//   b = (a+1) + k - K(a),
// and (a, b) is sent to i = N - a, j = b - a - 1 = k - K(a).  The radicand is formed exactly
// in 64-bit integers, the square root in FP32, and two integer conditionals repair a
// one-off row (the paper's "two conditional statements").
__device__ __forceinline__ void utm_map(uint64_t k, uint32_t N, uint32_t &i, uint32_t &j)
{
    const uint64_t n = static_cast<uint64_t>(N) + 1;
    const uint64_t D = 4 * n * n - 4 * n - 8 * k + 1;
    const float af = (__ull2float_rn(2 * n + 1) - sqrtf(__ull2float_rn(D))) * 0.5f;
    uint64_t a = __float2ull_rz(af);
    a = a < 1 ? 1 : (a > n - 1 ? n - 1 : a);
    uint64_t K = ((a - 1) * (2 * n - a)) >> 1;
    if (K > k) {
        --a;
        K = ((a - 1) * (2 * n - a)) >> 1;
    } else {
        const uint64_t K1 = (a * (2 * n - a - 1)) >> 1;
        if (K1 <= k) {
            ++a;
            K = K1;
        }
    }
    i = static_cast<uint32_t>(n - 1 - a);
    j = static_cast<uint32_t>(k - K);
}

// RB (Jung et al., Sec. III-B): the part of the triangle right of the middle column is
// rotated onto the space above the diagonal, giving a thread rectangle of T(N) threads.
// Even N: W = N/2 columns, H = N+1 rows; (x, y) with x < y -> (y-1, x), else
// (N-1-y, N-1-x).  Odd N: W = N/2 + 1, H = N; y >= x -> (y, x), else (N-1-y, N-x).
__host__ __device__ __forceinline__ void rb_dims(uint32_t N, uint32_t &W, uint32_t &H)
{
    if ((N & 1u) == 0) { W = N / 2; H = N + 1; }
    else               { W = N / 2 + 1; H = N; }
}

__device__ __forceinline__ void rb_map(uint32_t N, uint32_t x, uint32_t y, uint32_t &i, uint32_t &j)
{
    if ((N & 1u) == 0) {
        if (x < y) { i = y - 1; j = x; }
        else       { i = N - 1 - y; j = N - 1 - x; }
    } else {
        if (y >= x) { i = y; j = x; }
        else        { i = N - 1 - y; j = N - x; }
    }
}

// Probe hash: golden-ratio increment followed by the MurmurHash3 32-bit finaliser.
__device__ __forceinline__ uint32_t splitmix32(uint32_t x)
{
    uint32_t z = x + 0x9E3779B9u;
    z = (z ^ (z >> 16)) * 0x85EBCA6Bu;
    z = (z ^ (z >> 13)) * 0xC2B2AE35u;
    return z ^ (z >> 16);
}

}  // namespace td
