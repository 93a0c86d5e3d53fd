// td_collide.cu -- pairwise collision table, one of the td-problems named in the abstract and
// Sec. I of arXiv:1308.1419 (the UTM of Sec. III-B came from collision detection).
//
// Spheres i > j collide iff |c_i - c_j|^2 <= (r_i + r_j)^2, decided exactly.  The strict lower
// triangle is cut into 32 x 32 bit-tiles; tile (ti, tj), tj <= ti, is tile number T(ti) + tj of
// the tile triangle and owns table words [32 (T(ti) + tj), 32 (T(ti) + tj) + 32): word r holds
// row i = 32 ti + r, bit c (LSB first) column j = 32 tj + c.  The launch space is the triangle of
// 64 x 64 blocks (rho = 64), issued by g(lambda) over its T(ceil(n/64)) blocks or by BB over their
// bounding box; block (bi, bj) holds the tiles (2 bi + h, 2 bj + g), h, g in {0, 1}, except, on the
// diagonal, the tile (2 bi, 2 bi + 1) above it.  One warp computes one block: lane c holds the
// column spheres 64 bj + c and 64 bj + 32 + c, the 64 row spheres sit in shared memory and are
// read by broadcast (one load per row for two pairs), and each row's 2 x 32 predicates become the
// row's words of the two tiles through two __ballot_sync; lane r keeps row r's words, and the 32
// lanes store a tile's words as 128 contiguous bytes.
//
// Fast path on the FP32 pipe, when every coordinate and radius of the block's 128 spheres lies in
// (-2^23, 2^23): coordinate differences and radius sums are then exact in FP32.
//  - A pair with max(|dx|, |dy|) > |r_i + r_j| cannot collide (dx^2 or dy^2 alone exceeds the
//    squared radius sum), and that test is exact; a row whose 64 pairs all fail it gets zero
//    words at once (with centres spread over a large cube almost every row does).
//  - Other rows take s - R^2 = fma(-R, R, s) for their pairs, which decides a pair unless it falls
//    within one band for the block, 2^-20 Rmax^2 with Rmax the largest row radius plus the
//    largest column radius (collide_f32_diff and its error bound in td_collide.cuh).  Each lane
//    keeps the smallest |s - R^2| of each of its two columns; a tile with a pair inside the band
//    is redone with the exact integer test.
// Blocks with larger values use the exact test throughout: the 32-bit form when all the block's
// spheres lie in its domain (coordinates in [-2^30, 2^30), radii in [0, 2^14]), the 64/128-bit
// form otherwise, so every int32 input is decided exactly.  Only diagonal and edge tiles apply the
// validity mask (columns and rows below n, j < i on the diagonal).
// The same kernel also writes the strict bit array of td_collide_strict (pair (i, j), j < i, at
// bit i (i - 1) / 2 + j): the caller clears the array, and each masked row word that has a bit set
// is ORed, atomically, into the one or two array words it straddles (row pieces of neighbouring
// blocks share words).  With sparse collisions almost nothing is written.
#include "td_collide.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ int4 load_sphere(const int32_t *__restrict__ c, const int32_t *__restrict__ rad, uint32_t j,
                                            uint32_t n)
{
    if (j >= n) return make_int4(0, 0, 0, 0);
    return make_int4(__ldg(c + 3 * uint64_t(j)), __ldg(c + 3 * uint64_t(j) + 1), __ldg(c + 3 * uint64_t(j) + 2),
                     __ldg(rad + j));
}

__device__ __forceinline__ float4 to_f4(const int4 &p) { return make_float4(float(p.x), float(p.y), float(p.z), float(p.w)); }

// Lane r's word of tile (tr, tc) (row 32 tr + r) after the validity mask: columns and rows below
// n, j < i on the diagonal.  Warp-collective.
__device__ __forceinline__ uint32_t mask_word(uint32_t word, uint32_t tr, uint32_t tc, uint32_t n, uint32_t lane)
{
    if (tr == tc || 32 * tr + 32 > n || 32 * tc + 32 > n) {
        const uint32_t colmask = __ballot_sync(0xffffffffu, 32 * tc + lane < n);
        word &= 32 * tr + lane < n ? (colmask & (tr == tc ? ((1u << lane) - 1u) : ~0u)) : 0u;
    }
    return word;
}

// The tile table: lane r's masked word stored with the other lanes' words as 128 contiguous bytes.
__device__ __forceinline__ void store_word(uint32_t word, uint32_t tr, uint32_t tc, uint32_t n, uint32_t lane,
                                           uint32_t *__restrict__ table)
{
    table[(tri(tr) + tc) * 32 + lane] = mask_word(word, tr, tc, n, lane);
}

// The strict bit array (pair (i, j), j < i, at bit i (i - 1) / 2 + j, LSB first; cleared before
// the launch): lane r's masked word -- row i = 32 tr + r, columns 32 tc .. 32 tc + 31, so bits
// k0 = i (i - 1) / 2 + 32 tc onwards -- is ORed into the one or two words it straddles, and only
// if it has a bit set.  Every bit it holds is a real pair (j < i < n), so every word it touches
// lies inside the array.
__device__ __forceinline__ void or_strict(uint32_t word, uint32_t tr, uint32_t tc, uint32_t n, uint32_t lane,
                                          uint32_t *__restrict__ bits)
{
    word = mask_word(word, tr, tc, n, lane);
    if (word == 0) return;
    const uint64_t i = 32 * uint64_t(tr) + lane;  // i >= 1: row 0 has no pair and an empty word
    const uint64_t k0 = i * (i - 1) / 2 + 32 * uint64_t(tc);
    const uint32_t sh = static_cast<uint32_t>(k0 & 31u);
    uint32_t *w = bits + (k0 >> 5);
    atomicOr(w, word << sh);
    if (sh != 0 && (word >> (32 - sh)) != 0) atomicOr(w + 1, word >> (32 - sh));
}

// Exact pass of one tile: row spheres rows[0 .. 31] against this lane's column sphere q; returns
// lane r's word (row r).  Rarely taken on the fast path, so kept out of line (a smaller loop body
// for the instruction cache).
__device__ __noinline__ uint32_t exact_word(const int4 *rows, const int4 &q, bool in32, uint32_t lane)
{
    uint32_t mine = 0;
    if (in32) {
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            const uint32_t b = __ballot_sync(0xffffffffu, collide_exact32(rows[r], q));
            if (lane == uint32_t(r)) mine = b;
        }
    } else {
        for (int r = 0; r < 32; ++r) {
            const uint32_t b = __ballot_sync(0xffffffffu, collide_wide(rows[r], q));
            if (lane == uint32_t(r)) mine = b;
        }
    }
    return mine;
}

// kStrict: the strict bit array instead of the tile table (or_strict instead of store_word); the
// predicate passes are the same code, so both outputs hold the same decisions.
template <class Tiles, bool P, bool kStrict>
__global__ void __launch_bounds__(32 * kWarps)
    k_collide(Tiles tiles, const int32_t *__restrict__ c, const int32_t *__restrict__ rad, uint32_t n,
              uint32_t *__restrict__ table)
{
    __shared__ int4 rows[kWarps][64];
    __shared__ float4 rowsf[kWarps][64];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nt = (n + 31) / 32;  // tiles per side
    const uint64_t first = uint64_t(blockIdx.x) * kWarps + warp;
    const uint64_t stride = P ? uint64_t(gridDim.x) * kWarps : tiles.units;
    for (uint64_t u = first; u < tiles.units; u += stride) {
        uint32_t bi, bj;
        if (!tiles(u, bi, bj)) continue;  // warp-uniform
        const bool diag = bi == bj;
        const int4 q0 = load_sphere(c, rad, 64 * bj + lane, n), q1 = load_sphere(c, rad, 64 * bj + 32 + lane, n);
        const int4 p0 = load_sphere(c, rad, 64 * bi + lane, n), p1 = load_sphere(c, rad, 64 * bi + 32 + lane, n);
        __syncwarp();
        rows[warp][lane] = p0;
        rows[warp][32 + lane] = p1;
        rowsf[warp][lane] = to_f4(p0);
        rowsf[warp][32 + lane] = to_f4(p1);
        __syncwarp();
        const bool small =
            __all_sync(0xffffffffu, small_sphere(q0) && small_sphere(q1) && small_sphere(p0) && small_sphere(p1));
        const bool in32 =
            __all_sync(0xffffffffu, in_domain32(q0) && in_domain32(q1) && in_domain32(p0) && in_domain32(p1));
        float band_c = 0.0f;
        if (small) {
            const float rmax = float(__reduce_max_sync(0xffffffffu, uint32_t(max(abs(p0.w), abs(p1.w)))) +
                                     __reduce_max_sync(0xffffffffu, uint32_t(max(abs(q0.w), abs(q1.w)))));
            band_c = 0x1p-20f * rmax * rmax;
        }
        const float4 f0 = to_f4(q0), f1 = to_f4(q1);
#pragma unroll 1
        for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t tr = 2 * bi + h;  // tile row
            if (tr >= nt) break;
            // the second tile of the row, (tr, 2 bj + 1): inside the triangle and below the diagonal
            const bool second = !(diag && h == 0) && 2 * bj + 1 < nt;
            uint32_t mine0 = 0, mine1 = 0;  // this lane's words: row 32 tr + lane of the two tiles
            bool ex0 = !small, ex1 = !small;
            if (small) {
                float m0 = __int_as_float(0x7f800000), m1 = m0;  // smallest |s - R^2| per column
#pragma unroll 8
                for (int r = 0; r < 32; ++r) {
                    const float4 pr = rowsf[warp][32 * h + r];
                    const float R0 = pr.w + f0.w, R1 = pr.w + f1.w;
                    const float e0 = fmaxf(fabsf(pr.x - f0.x), fabsf(pr.y - f0.y));
                    const float e1 = fmaxf(fabsf(pr.x - f1.x), fabsf(pr.y - f1.y));
                    if (__any_sync(0xffffffffu, e0 <= fabsf(R0) || e1 <= fabsf(R1))) {
                        const float d0 = collide_f32_diff(pr, f0), d1 = collide_f32_diff(pr, f1);
                        m0 = fminf(m0, fabsf(d0));
                        m1 = fminf(m1, fabsf(d1));
                        const uint32_t b0 = __ballot_sync(0xffffffffu, d0 <= 0.0f);
                        const uint32_t b1 = __ballot_sync(0xffffffffu, d1 <= 0.0f);
                        if (lane == uint32_t(r)) {
                            mine0 = b0;
                            mine1 = b1;
                        }
                    }
                }
                ex0 = __any_sync(0xffffffffu, m0 <= band_c);
                ex1 = __any_sync(0xffffffffu, m1 <= band_c);
            }
            // exact pass of a tile: large values, or a pair in the band
            if (ex0) mine0 = exact_word(rows[warp] + 32 * h, q0, in32, lane);
            if (ex1 && second) mine1 = exact_word(rows[warp] + 32 * h, q1, in32, lane);
            if (kStrict) {
                or_strict(mine0, tr, 2 * bj, n, lane, table);
                if (second) or_strict(mine1, tr, 2 * bj + 1, n, lane, table);
            } else {
                store_word(mine0, tr, 2 * bj, n, lane, table);
                if (second) store_word(mine1, tr, 2 * bj + 1, n, lane, table);
            }
        }
    }
}

template <class Tiles, bool kStrict = false>
td_status launch(const Tiles &t, bool P, const int32_t *c, const int32_t *r, uint32_t n, uint32_t *table,
                 cudaStream_t st, uint64_t *ctas)
{
    const uint64_t need = (t.units + kWarps - 1) / kWarps;
    if (P) {
        auto k = k_collide<Tiles, true, kStrict>;
        const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, need);
        k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, c, r, n, table);
        *ctas += g;
    } else {
        k_collide<Tiles, false, kStrict><<<dim3(static_cast<uint32_t>(need)), 32 * kWarps, 0, st>>>(t, c, r, n, table);
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

td_status launch_collide_strict64(td_mapping m, const int32_t *c, const int32_t *r, uint32_t n, uint32_t *bits,
                                  uint64_t words, const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    td_status s = cuda_status(cudaMemsetAsync(bits, 0, words * 4, st), "strict collision bits clear");
    if (s != TD_OK) return s;
    if (m == TD_MAP_LTM) return launch<tiles::Ltm, true>(tiles::ltm_source(p), true, c, r, n, bits, st, ctas);
    if (m == TD_MAP_BB) return launch<tiles::Bb, true>(tiles::bb_source(p), true, c, r, n, bits, st, ctas);
    return fail(TD_ERR_UNSUPPORTED, "the strict collision bits by 64 x 64 blocks serve LTM and BB");
}

}  // namespace td
