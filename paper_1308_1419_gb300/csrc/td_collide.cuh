// td_collide.cuh -- the collision predicate shared by the collision kernels (td_collide.cu,
// td_collide_chunked.cu, td_strict.cu): spheres p and q collide iff
// |c_p - c_q|^2 <= (r_p + r_q)^2, decided exactly for any int32 coordinates and radii; and its
// FP32 fast form with the band that proves it.
#pragma once

#include "td_device.cuh"

namespace td {

// The exact collision predicate |c_p - c_q|^2 <= (r_p + r_q)^2 in 32-bit integers, for
// coordinates in [-2^30, 2^30) and radii in [0, 2^14] (in_domain32): with R = r_p + r_q <= 2^15,
// each |delta| is clamped to R + 1 before squaring -- if all |delta| <= R nothing changes and the
// sum is exact (< 3 (2^15)^2 < 2^32); if one exceeds R the clamped sum exceeds R^2, and so does
// the true one.
__device__ __forceinline__ bool collide_exact32(const int4 &p, const int4 &q)
{
    const uint32_t R = static_cast<uint32_t>(p.w + q.w), R1 = R + 1;
    const int32_t ex = p.x - q.x, ey = p.y - q.y, ez = p.z - q.z;
    const uint32_t dx = min(static_cast<uint32_t>(ex < 0 ? -ex : ex), R1);
    const uint32_t dy = min(static_cast<uint32_t>(ey < 0 ? -ey : ey), R1);
    const uint32_t dz = min(static_cast<uint32_t>(ez < 0 ? -ez : ez), R1);
    return dx * dx + dy * dy + dz * dz <= R * R;
}

__device__ __forceinline__ bool in_domain32(const int4 &p)
{
    const int32_t lim = 1 << 30;
    return p.x >= -lim && p.x < lim && p.y >= -lim && p.y < lim && p.z >= -lim && p.z < lim && p.w >= 0 &&
           p.w <= (1 << 14);
}

// The same predicate for any int32 coordinates and radii: |delta_k| < 2^32 and |R| <= 2^32 in
// 64-bit integers; a |delta_k| above |R| decides the pair at once (its square alone exceeds R^2),
// otherwise every square is at most 2^64 and the sum of the three is compared with R^2 in 128-bit
// integers.
static __device__ __noinline__ bool collide_wide(const int4 &p, const int4 &q)
{
    const long long R = static_cast<long long>(p.w) + q.w;
    const unsigned long long aR = static_cast<unsigned long long>(R < 0 ? -R : R);
    const long long e[3] = {static_cast<long long>(p.x) - q.x, static_cast<long long>(p.y) - q.y,
                            static_cast<long long>(p.z) - q.z};
    unsigned __int128 s = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned long long a = static_cast<unsigned long long>(e[k] < 0 ? -e[k] : e[k]);
        if (a > aR) return false;
        s += static_cast<unsigned __int128>(a) * a;
    }
    return s <= static_cast<unsigned __int128>(aR) * aR;
}

// Exact for every int32 input: the 32-bit form inside its domain, the wide form outside it.
__device__ __forceinline__ bool collide_exact(const int4 &p, const int4 &q)
{
    return (in_domain32(p) && in_domain32(q)) ? collide_exact32(p, q) : collide_wide(p, q);
}

// The same predicate on the FP32 pipe, for coordinates and radii in (-2^23, 2^23) (small_sphere)
// carried as floats: coordinate differences are then integers below 2^24 and exact in FP32, and
// so is the radii sum R.  s = fma(dx, dx, fma(dy, dy, dz dz)) is within 3u s_t of the exact sum
// of squares s_t (u = 2^-24, first order), and diff = fma(-R, R, s) rounds s - R^2 once, so
// with D = s_t - R^2 the error of diff is at most 3u R^2 + 4u |D|.  The sign of diff can differ
// from that of D only if |D| <= 3.1u R^2, and then |diff| <= 6.2u R^2.  So with a band
// band_c = 2^-20 Rmax^2 = 16u Rmax^2 for a group of pairs, Rmax >= R for every pair of the
// group, |diff| > band_c proves the sign; *band reports a pair with |diff| <= band_c, which the
// caller must decide again with collide_exact.
__device__ __forceinline__ bool small_coords(const int4 &p)
{
    const int32_t lim = 1 << 23;
    return p.x > -lim && p.x < lim && p.y > -lim && p.y < lim && p.z > -lim && p.z < lim;
}

// small_coords and a radius in (-2^23, 2^23), so that radius sums are exact in FP32 too.
__device__ __forceinline__ bool small_sphere(const int4 &p)
{
    const int32_t lim = 1 << 23;
    return small_coords(p) && p.w > -lim && p.w < lim;
}

// diff = fl(s - R^2) of the pair, whose sign decides it unless |diff| <= band_c.
__device__ __forceinline__ float collide_f32_diff(const float4 &p, const float4 &q)
{
    const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
    const float s = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float R = p.w + q.w;
    return fmaf(-R, R, s);
}

__device__ __forceinline__ bool collide_f32_banded(const float4 &p, const float4 &q, float band_c, bool &band)
{
    const float diff = collide_f32_diff(p, q);
    band = fabsf(diff) <= band_c;
    return diff <= 0.0f;
}

}  // namespace td
