// td_collide.cu -- pairwise collision table, one of the td-problems named in the abstract and
// Sec. I of arXiv:1308.1419 (the UTM of Sec. III-B came from collision detection).
//
// Spheres i > j collide iff |c_i - c_j|^2 <= (r_i + r_j)^2, decided exactly.  The strict lower
// triangle is cut into 32 x 32 bit-tiles; tile (bi, bj), bj <= bi, is tile number T(bi) + bj of
// the tile triangle and owns table words [32 (T(bi) + bj), 32 (T(bi) + bj) + 32): word r holds
// row i = 32 bi + r, bit c (LSB first) column j = 32 bj + c.  One warp computes one tile:
// lane c holds sphere j, the 32 row spheres sit in shared memory and are read by broadcast,
// each row's 32 predicates become one word through __ballot_sync, and lane r keeps word r, so
// the tile leaves in one coalesced 128-byte store.  Tiles are issued by g(lambda) over the
// T(ceil(n/32)) tiles, or by BB over the bounding box of tiles.
//
// Exactness in 32-bit integers: with coordinates in [-2^30, 2^30) and radii in [0, 2^14],
// R = r_i + r_j <= 2^15.  Each |delta| is clamped to R + 1 before squaring: if every |delta|
// <= R the clamp changes nothing and the sum of squares is exact (< 3 (2^15)^2 < 2^32); if some
// |delta| > R the clamped sum exceeds R^2, and so does the true one.  Either way the unsigned
// 32-bit comparison equals the exact definition.
//
// Fast path on the FP32 pipe (full rate, where the integer ALU runs at half rate): when every
// coordinate of the tile's 64 spheres lies in (-2^23, 2^23), coordinate differences are exact
// in FP32, and s - R^2 = fma(-R, R, s) decides the pair unless it falls within one band for
// the whole tile, 2^-20 Rmax^2 with Rmax the largest row radius plus the largest column radius
// (collide_f32_banded gives the error bound).  If any pair of a tile falls inside the band, the
// whole tile is redone with the exact integer test above; tiles with larger coordinates use the
// integer test throughout.  The 32 row words stay in registers (a ballot result is the same in
// every lane) and lane 0 writes the tile's 128 bytes; only diagonal and edge tiles apply the
// validity mask (columns and rows below n, j < i on the diagonal).
#include "td_collide.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
namespace {

constexpr int kWarps = 8;

template <class Tiles, bool P>
__global__ void __launch_bounds__(32 * kWarps)
    k_collide(Tiles tiles, const int32_t *__restrict__ c, const int32_t *__restrict__ rad, uint32_t n,
              uint32_t *__restrict__ table)
{
    __shared__ int4 rows[kWarps][32];
    __shared__ float4 rowsf[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t first = uint64_t(blockIdx.x) * kWarps + warp;
    const uint64_t stride = P ? uint64_t(gridDim.x) * kWarps : tiles.units;
    for (uint64_t u = first; u < tiles.units; u += stride) {
        uint32_t bi, bj;
        if (!tiles(u, bi, bj)) continue;  // warp-uniform
        const uint32_t j = 32 * bj + lane, ir = 32 * bi + lane;
        int4 pj = make_int4(0, 0, 0, 0), pi = make_int4(0, 0, 0, 0);
        if (j < n) pj = make_int4(__ldg(c + 3 * uint64_t(j)), __ldg(c + 3 * uint64_t(j) + 1), __ldg(c + 3 * uint64_t(j) + 2), __ldg(rad + j));
        if (ir < n) pi = make_int4(__ldg(c + 3 * uint64_t(ir)), __ldg(c + 3 * uint64_t(ir) + 1), __ldg(c + 3 * uint64_t(ir) + 2), __ldg(rad + ir));
        const float4 fj = make_float4(float(pj.x), float(pj.y), float(pj.z), float(pj.w));
        __syncwarp();
        rows[warp][lane] = pi;
        rowsf[warp][lane] = make_float4(float(pi.x), float(pi.y), float(pi.z), float(pi.w));
        __syncwarp();
        // the 32 row words, warp-uniform: word r = ballot of row 32 bi + r
        uint32_t w[32];
        bool exact = !__all_sync(0xffffffffu, small_coords(pj) && small_coords(pi));
        if (!exact) {
            // FP32 pass; a pair within the tile's band marks the tile for the exact pass
            const float rmax = float(__reduce_max_sync(0xffffffffu, uint32_t(pi.w)) +
                                     __reduce_max_sync(0xffffffffu, uint32_t(pj.w)));
            const float band_c = 0x1p-20f * rmax * rmax;
            bool band = false;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                bool near;
                const bool hit = collide_f32_banded(rowsf[warp][r], fj, band_c, near);
                band = band || near;
                w[r] = __ballot_sync(0xffffffffu, hit);
            }
            exact = __any_sync(0xffffffffu, band);
        }
        if (exact) {  // integer pass for the whole tile (large coordinates, or a pair in the band)
#pragma unroll
            for (int r = 0; r < 32; ++r) w[r] = __ballot_sync(0xffffffffu, collide_exact(rows[warp][r], pj));
        }
        // keep columns below n, rows below n, and j < i on the diagonal
        if (bi == bj || 32 * bi + 32 > n) {
            const uint32_t colmask = __ballot_sync(0xffffffffu, j < n);
            const uint32_t rows_valid = n - 32 * bi >= 32 ? 32u : n - 32 * bi;
#pragma unroll
            for (int r = 0; r < 32; ++r)
                w[r] &= uint32_t(r) < rows_valid ? (colmask & (bi == bj ? ((1u << r) - 1u) : ~0u)) : 0u;
        }
        if (lane == 0) {  // the tile's 32 words: 128 contiguous bytes, 16-byte aligned
            uint4 *dst = reinterpret_cast<uint4 *>(table + (tri(bi) + bj) * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
    }
}

template <class Tiles>
td_status launch(const Tiles &t, bool P, const int32_t *c, const int32_t *r, uint32_t n, uint32_t *table,
                 cudaStream_t st, uint64_t *ctas)
{
    const uint64_t need = (t.units + kWarps - 1) / kWarps;
    if (P) {
        auto k = k_collide<Tiles, true>;
        const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, need);
        k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, c, r, n, table);
        *ctas += g;
    } else {
        k_collide<Tiles, false><<<dim3(static_cast<uint32_t>(need)), 32 * kWarps, 0, st>>>(t, c, r, n, table);
        *ctas += need;
    }
    return launch_status("td_collide kernel");
}

}  // namespace

td_status launch_collide(td_mapping m, td_schedule s, const int32_t *c, const int32_t *r, uint32_t n,
                         uint32_t *table, const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    const bool P = s == TD_SCHED_PERSISTENT;
    const uint32_t nt = (n + 31) / 32;
    if (m == TD_MAP_LTM) return launch(tiles::ltm_source(p), P, c, r, n, table, st, ctas);
    if (m == TD_MAP_UTM_BLOCK) return launch(tiles::UtmBlk{tri(nt), nt}, P, c, r, n, table, st, ctas);
    if (m == TD_MAP_BB) return launch(tiles::bb_source(p), P, c, r, n, table, st, ctas);
    return fail(TD_ERR_UNSUPPORTED, "td_collide supports LTM, BB and UTM-BLOCK");
}

}  // namespace td
