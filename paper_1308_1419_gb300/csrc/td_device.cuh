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

// g(lambda) without the diagonal (Eq. (theorem_nodiag)): i = floor(sqrt(1/4 + 2 lambda) + 1/2),
// with the strict triangle's own row start, j = lambda - i(i-1)/2 (the printed i(i+1)/2 gives
// j = -1 at lambda = 0).  sqrt(1/4 + 2 lambda) + 1/2 = (sqrt(8 lambda + 1) + 1) / 2; the same
// FP32 reciprocal-square-root estimate and exact +-1 row fix-up as ltm_g (exact for
// lambda < 2^40).  Row i holds i elements, so 0 <= j < i.
__device__ __forceinline__ void ltm_g_strict(uint64_t lam, uint32_t &i, uint32_t &j)
{
    const float y = __ull2float_rn(8ull * lam + 1ull);
    const float s = y * rsqrtf(y);
    uint32_t r = __float2uint_rz(fmaf(s, 0.5f, 0.5f));
    uint64_t t = (uint64_t(r) * (r - 1)) >> 1;  // strict row start of row r (r >= 1)
    if (t > lam) {                      // one row too far down
        --r;
        t -= r;
    } else if (t + r <= lam) {          // one row too far up
        t += r;
        ++r;
    }
    i = r;
    j = static_cast<uint32_t>(lam - t);
}

// g(lambda) as a functor (the mapper the LTM kernels are written against).
struct LtmExact {
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &i, uint32_t &j) const { ltm_g(lam, i, j); }
};

// The single-precision evaluations of i = floor(sqrt(1/4 + 2 lambda) - 1/2) that Sec. III-A
// times in the dummy kernel, each written with explicitly rounded operations (fused multiply-adds
// only where written, in LtmNewtonFma) so that it is one well-defined FP32 function; none carries
// a fix-up, so each is exact only
// while FP32 resolves the row boundaries.  j = lambda - T(i) in 64-bit integers, truncated.
__device__ __forceinline__ float ltm_radicand(uint64_t lam)  // x = 1/4 + 2 lambda, rounded
{
    return __fadd_rn(0.25f, __fmul_rn(2.0f, __ull2float_rn(lam)));
}

// LTM-X: the square root itself.
struct LtmSqrt {
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &i, uint32_t &j) const
    {
        i = __float2uint_rz(__fsub_rn(__fsqrt_rn(ltm_radicand(lam)), 0.5f));
        j = static_cast<uint32_t>(lam - tri(i));
    }
};

// LTM-N: the bit-level inverse-square-root seed 0x5f3759df - (bits(x) >> 1) (Lomont's
// analysis of the method), three Newton steps y <- y (3/2 - (x/2) y^2), sqrt(x) = x y, and the
// paper's epsilon 1e-4 added inside the floor.
struct LtmNewton {
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &i, uint32_t &j) const
    {
        const float x = ltm_radicand(lam), h = __fmul_rn(0.5f, x);
        float y = __int_as_float(0x5f3759df - (__float_as_int(x) >> 1));
#pragma unroll
        for (int k = 0; k < 3; ++k) y = __fmul_rn(y, __fsub_rn(1.5f, __fmul_rn(__fmul_rn(h, y), y)));
        i = __float2uint_rz(__fadd_rn(__fsub_rn(__fmul_rn(x, y), 0.5f), 1e-4f));
        j = static_cast<uint32_t>(lam - tri(i));
    }
};

// LTM-N as a CUDA compiler contracts it by default: each Newton step rounds t = (x/2) y, then fuses
// t y into the subtraction from 3/2 (y <- y fma(-t, y, 3/2)), and x y - 1/2 is one fused
// multiply-add; epsilon 1e-4 is added after it.  The paper's statement that LTM-N is exact for
// N <= 30720 at rho = 16 (lambda < T(1920)) holds for this evaluation and not for LtmNewton's.
struct LtmNewtonFma {
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &i, uint32_t &j) const
    {
        const float x = ltm_radicand(lam), h = __fmul_rn(0.5f, x);
        float y = __int_as_float(0x5f3759df - (__float_as_int(x) >> 1));
#pragma unroll
        for (int k = 0; k < 3; ++k) y = __fmul_rn(y, __fmaf_rn(-__fmul_rn(h, y), y, 1.5f));
        i = __float2uint_rz(__fadd_rn(__fmaf_rn(x, y, -0.5f), 1e-4f));
        j = static_cast<uint32_t>(lam - tri(i));
    }
};

// LTM-R: x rsqrtf(x) with the paper's epsilon 1e-4 added inside the floor.
struct LtmRsqrtEps {
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &i, uint32_t &j) const
    {
        const float x = ltm_radicand(lam);
        i = __float2uint_rz(__fadd_rn(__fsub_rn(__fmul_rn(x, rsqrtf(x)), 0.5f), 1e-4f));
        j = static_cast<uint32_t>(lam - tri(i));
    }
};

// UTM (Avril et al., Sec. III-B) for a lower triangle of side N with its diagonal.  The
// strict upper triangle of side n = N + 1 has T(N) pairs; thread index k gives
//   a = floor(((2n+1) - sqrt(4n^2 - 4n - 8k + 1)) / 2),  row start K(a) = (a-1)(2n-a)/2,
//   b = (a+1) + k - K(a),
// and (a, b) is sent to i = N - a, j = b - a - 1 = k - K(a).  The radicand is formed exactly
// in 64-bit integers, the square root in FP32, and integer row tests repair the estimate (the
// paper's "two conditional statements" when it is off by one row).
// RSQRT: the square root taken as y rsqrtf(y) (the reciprocal-square-root trick of Sec. III-A),
// as the block-level UTM of the paper's conclusion uses it; the fix-up keeps both exact.
template <bool RSQRT = false>
__device__ __forceinline__ void utm_map(uint64_t k, uint32_t N, uint32_t &i, uint32_t &j)
{
    const uint64_t n = static_cast<uint64_t>(N) + 1;
    const uint64_t D = 4 * n * n - 4 * n - 8 * k + 1;  // >= 9 for k < T(N)
    const float y = __ull2float_rn(D);
    const float af = (__ull2float_rn(2 * n + 1) - (RSQRT ? y * rsqrtf(y) : sqrtf(y))) * 0.5f;
    uint64_t a = __float2ull_rz(af);
    a = a < 1 ? 1 : (a > n - 1 ? n - 1 : a);
    // walk to the row with K(a) <= k < K(a + 1); K(1) = 0 <= k and K(n) = T(N) > k bound it.
    // The estimate is within one row for N below about 2^22 (one step, as the paper's two
    // conditionals); the FP32 error grows as N 2^-24, and the walk keeps larger N exact.
    uint64_t K = ((a - 1) * (2 * n - a)) >> 1;
    while (K > k) {
        --a;
        K = ((a - 1) * (2 * n - a)) >> 1;
    }
    for (;;) {
        const uint64_t K1 = (a * (2 * n - a - 1)) >> 1;
        if (K1 > k) break;
        ++a;
        K = K1;
    }
    i = static_cast<uint32_t>(n - 1 - a);
    j = static_cast<uint32_t>(k - K);
}

// Block-level UTM (the conjecture that closes the paper): the UTM formula applied to block indices
// lambda < T(nb) over the block triangle of side nb instead of to thread indices, with the
// reciprocal-square-root trick; blocks come row by row from the last block row up.
struct UtmBlock {
    uint32_t nb;
    __device__ __forceinline__ void operator()(uint64_t lam, uint32_t &bi, uint32_t &bj) const
    {
        utm_map<true>(lam, nb, bi, bj);
    }
};

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
