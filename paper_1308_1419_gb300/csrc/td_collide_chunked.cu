// td_collide_chunked.cu -- the strict-lower collision bits of td_collide_strict (bit k of a
// uint32 array, word k / 32, LSB first, is c(i, j) for k = i(i-1)/2 + j, j < i), produced under
// the chunked schedule of the block strategies instead of the element-level strict g.
//
// The strict lower triangle of n spheres (the pairs Eq. (theorem_nodiag) of Sec. II-A maps) is
// the with-diagonal packed triangle of side n1 = n - 1 whose row i1 holds the pairs (i1 + 1, j),
// j <= i1, at T(i1) + j, T(m) = m(m+1)/2.  Its rho x rho blocks are issued by g(lambda) (Sec.
// II-A) or by BB, and warps walk strips of consecutive blocks as the chunked probe does: a run of
// blocks (bi, bj) .. (bi, bj + run - 1) covers, in each element row i1, the contiguous bit range
// T(i1) + [jlo, jhi), jlo = bj rho, jhi = min((bj + run) rho, i1 + 1), and each 32-bit word of
// the array is decided by the run holding its first bit.
//
// Per run, lane l holds the column spheres jlo + 32 g + l, g < NG, in registers (the run's
// columns and the 32 after them).  Per element row the row sphere is a broadcast load, and
// group g's 32 predicates become one ballot b_g over columns jlo + 32 g ...; with
// a = (T(i1) + jlo) mod 32 the bit of column jlo + 32 g + l sits at bit (a + l) mod 32 of word
// (T(i1) + jlo) / 32 + g (+1 when a + l >= 32), so that word is the funnel shift of b_(g-1)
// and b_g by a.  Lane g keeps word g and the row's words leave in one store.  The one word per
// row that runs past the end of row i1 into the next row(s) is decided lane by lane from global
// memory.
//
// The predicate is collide_exact's.  When every coordinate of the run's spheres is below 2^23
// in magnitude it is taken on the FP32 pipe (collide_f32_banded, one band for the run), and a row
// with a pair inside the band is decided again with the integer test (spheres reloaded, off the
// fast path);
// otherwise the integer test decides every pair of the run.
#include "td_collide.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
namespace {

constexpr uint32_t kWarps = 8, kStrip = 256;
constexpr int NG = kStrip / 32 + 1;  // column groups a lane holds: the widest run and 32 more columns

__device__ __forceinline__ int4 sphere(const int32_t *__restrict__ c, const int32_t *__restrict__ r, uint32_t j)
{
    return make_int4(__ldg(c + 3 * uint64_t(j)), __ldg(c + 3 * uint64_t(j) + 1), __ldg(c + 3 * uint64_t(j) + 2),
                     __ldg(r + j));
}

__device__ __forceinline__ float4 as_float4(const int4 &p) { return make_float4(float(p.x), float(p.y), float(p.z), float(p.w)); }

// The crossing word at position P (a multiple of 32, P < total): lane l decides bit P + l.
__device__ __forceinline__ bool crossing_bit(const int32_t *__restrict__ c, const int32_t *__restrict__ r, uint64_t P,
                                             uint32_t i1, uint64_t ti, uint64_t total, uint32_t lane)
{
    const uint64_t Pl = P + lane;
    if (Pl >= total) return false;
    uint32_t ii = i1;
    uint64_t tii = ti;
    while (Pl > tii + ii) {
        tii += ii + 1;
        ++ii;
    }
    return collide_exact(sphere(c, r, ii + 1), sphere(c, r, static_cast<uint32_t>(Pl - tii)));
}

// One run's element rows.  SMALL: cols hold the column spheres as floats (every coordinate of
// the run below 2^23) and band_c is the run's FP32 band (collide_f32_banded), else cols hold the
// integers (reinterpreted).  Every row decides all NG groups (the
// groups past the row's last word are not stored): a loop without an exit lets the groups'
// independent predicate chains overlap.
template <int RHO, bool SMALL>
__device__ __forceinline__ void run_rows(const float4 (&cols)[NG], float band_c, uint32_t bi, uint32_t jlo, uint32_t span, uint32_t n1,
                                         uint64_t total, const int32_t *__restrict__ c, const int32_t *__restrict__ r,
                                         uint32_t *__restrict__ bits, uint32_t lane)
{
    const uint32_t rend = min(bi * RHO + RHO, n1);  // element rows bi rho .. rend - 1
    int4 pn = sphere(c, r, bi * RHO + 1);
    for (uint32_t i1 = bi * RHO; i1 < rend; ++i1) {  // element row: pairs (i1 + 1, j), j <= i1
        const int4 p = pn;
        if (i1 + 1 < rend) pn = sphere(c, r, i1 + 2);  // the next row's sphere, loaded under this row
        const float4 pf = as_float4(p);
        const uint64_t ti = tri(i1);
        const uint32_t L = min(jlo + span, i1 + 1) - jlo;  // columns of the row in this run
        const uint32_t a = static_cast<uint32_t>(ti + jlo) & 31u;
        const uint64_t w0 = (ti + jlo) >> 5;
        uint32_t prev = 0, mine = 0;
        bool redo = false;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            bool hit;
            if (SMALL) {
                bool near;
                hit = collide_f32_banded(pf, cols[g], band_c, near);
                redo = redo || near;
            } else {
                const float4 q = cols[g];
                hit = collide_exact(p, make_int4(__float_as_int(q.x), __float_as_int(q.y), __float_as_int(q.z),
                                                 __float_as_int(q.w)));
            }
            const uint32_t b = __ballot_sync(0xffffffffu, hit);
            if (lane == uint32_t(g)) mine = __funnelshift_l(prev, b, a);  // word g: columns jlo + 32 g - a ..
            prev = b;
        }
        // words g_first = (a ? 1 : 0) .. g_last = (L - 1 + a) / 32 start inside the run; the last
        // one may run past the end of row i1
        const uint32_t g_first = a ? 1u : 0u, g_last = (L - 1 + a) >> 5;
        if (SMALL && __any_sync(0xffffffffu, redo)) {  // a pair in the FP32 band: the row again, exactly
            prev = 0;
            for (uint32_t g = 0; g <= g_last; ++g) {
                const uint32_t j = jlo + 32 * g + lane;  // columns past i1 feed no whole word
                const uint32_t b = __ballot_sync(0xffffffffu, j <= i1 && collide_exact(p, sphere(c, r, j)));
                if (lane == g) mine = __funnelshift_l(prev, b, a);
                prev = b;
            }
        }
        const bool cross = g_last >= g_first && 32u * g_last + 31u - a > i1 - jlo;
        const uint32_t g_full = cross ? g_last : g_last + 1;  // the words before it are whole
        if (lane >= g_first && lane < g_full) bits[w0 + lane] = mine;
        if (cross) {
            const uint64_t P = (w0 + g_last) << 5;
            const uint32_t word = __ballot_sync(0xffffffffu, crossing_bit(c, r, P, i1, ti, total, lane));
            if (lane == 0) bits[w0 + g_last] = word;
        }
    }
}

template <class Tiles, int RHO>
__global__ void __launch_bounds__(32 * kWarps) k_collide_chunked(Tiles tiles, uint32_t n1, uint32_t S,
                                                                 const int32_t *__restrict__ c,
                                                                 const int32_t *__restrict__ r,
                                                                 uint32_t *__restrict__ bits)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t total = tri(n1);
    const uint64_t warps = uint64_t(gridDim.x) * kWarps;
    const uint64_t strips = (tiles.units + S - 1) / S;
    for (uint64_t z = uint64_t(blockIdx.x) * kWarps + warp; z < strips; z += warps) {
        const uint64_t uend = min(tiles.units, (z + 1) * S);
        for (uint64_t u = z * S; u < uend;) {
            uint32_t bi, bj;
            const bool ok = tiles(u, bi, bj);
            const uint32_t run = tiles.run(u, ok, bi, bj, static_cast<uint32_t>(uend - u));
            u += run;
            if (!ok) continue;
            const uint32_t jlo = bj * RHO, span = run * RHO;
            int4 q[NG];
            bool small = true;
            uint32_t rm_c = 0, rm_r = 0;  // largest column and row radius of the run
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t j = jlo + 32 * g + lane;
                q[g] = (32u * g < span + 32u && j < n1) ? sphere(c, r, j) : make_int4(0, 0, 0, 0);
                small = small && small_coords(q[g]);
                rm_c = max(rm_c, uint32_t(q[g].w));
            }
            const uint32_t rlast = min(bi * RHO + RHO, n1);  // the run's row spheres: bi rho + 1 .. rlast
            for (uint32_t i = bi * RHO + 1 + lane; i <= rlast; i += 32) {
                const int4 pr = sphere(c, r, i);
                small = small && small_coords(pr);
                rm_r = max(rm_r, uint32_t(pr.w));
            }
            float4 cols[NG];
            if (__all_sync(0xffffffffu, small)) {
                const float rmax = float(__reduce_max_sync(0xffffffffu, rm_r) + __reduce_max_sync(0xffffffffu, rm_c));
#pragma unroll
                for (int g = 0; g < NG; ++g) cols[g] = as_float4(q[g]);
                run_rows<RHO, true>(cols, 0x1p-20f * rmax * rmax, bi, jlo, span, n1, total, c, r, bits, lane);
            } else {
#pragma unroll
                for (int g = 0; g < NG; ++g)
                    cols[g] = make_float4(__int_as_float(q[g].x), __int_as_float(q[g].y), __int_as_float(q[g].z),
                                          __int_as_float(q[g].w));
                run_rows<RHO, false>(cols, 0.0f, bi, jlo, span, n1, total, c, r, bits, lane);
            }
        }
    }
}

template <class Tiles, int RHO>
td_status launch_tiles(const Tiles &t, const int32_t *c, const int32_t *r, uint32_t n1, uint32_t *bits,
                       cudaStream_t st, uint64_t *ctas)
{
    if (t.units == 0) return TD_OK;
    auto k = k_collide_chunked<Tiles, RHO>;
    const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, ~0ull) * kWarps;
    const uint32_t w = chunked_strip_width(t.units, RHO, resident, kStrip, kStrip);
    if (w > kStrip || w < uint32_t(RHO)) return fail(TD_ERR_INVALID_ARG, "strict collision strip width %u", w);
    const uint32_t S = w / RHO;
    const uint64_t strips = (t.units + S - 1) / S;
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, (strips + kWarps - 1) / kWarps);
    k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, n1, S, c, r, bits);
    *ctas += g;
    return launch_status("td_collide_strict_blocks kernel");
}

template <int RHO>
td_status launch_rho(td_mapping m, const int32_t *c, const int32_t *r, uint32_t n1, uint32_t *bits, const Plan &p,
                     cudaStream_t st, uint64_t *ctas)
{
    if (m == TD_MAP_LTM) return launch_tiles<tiles::Ltm, RHO>(tiles::Ltm{tri(p.nb)}, c, r, n1, bits, st, ctas);
    if (m == TD_MAP_BB)
        return launch_tiles<tiles::Bb, RHO>(tiles::Bb{uint64_t(p.nb) * p.nb, p.nb}, c, r, n1, bits, st, ctas);
    return fail(TD_ERR_UNSUPPORTED, "the block-mapped strict collision bits serve LTM and BB");
}

}  // namespace

td_status launch_collide_chunked(td_mapping m, const int32_t *c, const int32_t *r, uint32_t n, uint32_t rho,
                                 uint32_t *bits, const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    if (n < 2) return TD_OK;
    switch (rho) {
    case 8: return launch_rho<8>(m, c, r, n - 1, bits, p, st, ctas);
    case 16: return launch_rho<16>(m, c, r, n - 1, bits, p, st, ctas);
    case 32: return launch_rho<32>(m, c, r, n - 1, bits, p, st, ctas);
    default: return fail(TD_ERR_INVALID_ARG, "the block-mapped strict collision bits need rho 8, 16 or 32 (got %u)", rho);
    }
}

}  // namespace td
