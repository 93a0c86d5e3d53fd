// td_collide.cuh -- the collision predicate shared by the collision kernels (td_collide.cu,
// td_collide_chunked.cu, td_strict.cu): spheres p and q collide iff
// |c_p - c_q|^2 <= (r_p + r_q)^2, decided exactly; and its FP32 fast form with the band that
// proves it.
#pragma once

#include "td_device.cuh"

namespace td {

// The exact collision predicate |c_p - c_q|^2 <= (r_p + r_q)^2 in 32-bit integers, for
// coordinates in [-2^30, 2^30) and radii in [0, 2^14]: with R = r_p + r_q <= 2^15, each |delta|
// is clamped to R + 1 before squaring -- if all |delta| <= R nothing changes and the sum is exact
// (< 3 (2^15)^2 < 2^32); if one exceeds R the clamped sum exceeds R^2, and so does the true one.
__device__ __forceinline__ bool collide_exact(const int4 &p, const int4 &q)
{
    const uint32_t R = static_cast<uint32_t>(p.w + q.w), R1 = R + 1;
    const int32_t ex = p.x - q.x, ey = p.y - q.y, ez = p.z - q.z;
    const uint32_t dx = min(static_cast<uint32_t>(ex < 0 ? -ex : ex), R1);
    const uint32_t dy = min(static_cast<uint32_t>(ey < 0 ? -ey : ey), R1);
    const uint32_t dz = min(static_cast<uint32_t>(ez < 0 ? -ez : ez), R1);
    return dx * dx + dy * dy + dz * dz <= R * R;
}

// The same predicate on the FP32 pipe, for coordinates in (-2^23, 2^23) (small_coords) carried
// as floats: coordinate differences are then integers below 2^24 and exact in FP32, and the
// radii sum R is exact.  s = fma(dx, dx, fma(dy, dy, dz dz)) is within 3u s_t of the exact sum
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

__device__ __forceinline__ bool collide_f32_banded(const float4 &p, const float4 &q, float band_c, bool &band)
{
    const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
    const float s = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float R = p.w + q.w;
    const float diff = fmaf(-R, R, s);
    band = fabsf(diff) <= band_c;
    return diff <= 0.0f;
}

}  // namespace td
