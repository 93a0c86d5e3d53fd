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
// Per run, the warp stages the run's column spheres (and the 32 after them) as float4s in its
// slice of shared memory, and the run's row spheres.  For element row i1 the first owned word
// starts at column q0 of the run, (T(i1) + jlo + q0) a multiple of 32, so lane l reading column
// q0 + 32 g + l makes the ballot of group g word g of the row itself: no shifting, one 16-byte
// shared load per pair, conflict-free.  The row's up to 8 words are decided in a loop without an
// exit (unused groups are computed and dropped) and written by lane 0.  The one word per row that
// runs past the end of row i1 into the next row(s) is decided lane by lane from global memory.
//
// The predicate is collide_exact's (exact for any int32 input).  When every coordinate and radius
// of the run's spheres is below 2^23 in magnitude it is taken on the FP32 pipe
// (collide_f32_banded, one band for the run; a radius that large or larger would not be exact
// in FP32), after an exact pre-test that rules out a group of 32 pairs at once when each pair has
// max(|dx|, |dy|) > |r_i + r_j|; a row
// with a pair inside the band is decided again with the integer test (spheres reloaded, off the
// fast path); otherwise the integer test decides every pair of the run (the staged values are
// then the integers, bit for bit).
#include "td_collide.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
namespace {

constexpr uint32_t kWarps = 8, kStrip = 256;
constexpr uint32_t kCols = kStrip + 32;  // staged columns per run: the widest run and 32 more
constexpr int NW = kStrip / 32;          // words per row and run, at most

__device__ __forceinline__ int4 sphere(const int32_t *__restrict__ c, const int32_t *__restrict__ r, uint32_t j)
{
    return make_int4(__ldg(c + 3 * uint64_t(j)), __ldg(c + 3 * uint64_t(j) + 1), __ldg(c + 3 * uint64_t(j) + 2),
                     __ldg(r + j));
}

__device__ __forceinline__ float4 as_float4(const int4 &p) { return make_float4(float(p.x), float(p.y), float(p.z), float(p.w)); }
__device__ __forceinline__ float4 bits_float4(const int4 &p)
{
    return make_float4(__int_as_float(p.x), __int_as_float(p.y), __int_as_float(p.z), __int_as_float(p.w));
}
__device__ __forceinline__ int4 bits_int4(const float4 &p)
{
    return make_int4(__float_as_int(p.x), __float_as_int(p.y), __float_as_int(p.z), __float_as_int(p.w));
}

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

// One run's element rows from the staged spheres.  SMALL: staged as floats, decided on the FP32
// pipe with band band_c; else staged as the integers and decided exactly.
template <int RHO, bool SMALL>
__device__ __forceinline__ void run_rows(const float4 *cols, const float4 *rows, float band_c, uint32_t bi, uint32_t jlo,
                                         uint32_t span, uint32_t n1, uint64_t total, const int32_t *__restrict__ c,
                                         const int32_t *__restrict__ r, uint32_t *__restrict__ bits, uint32_t lane)
{
    for (uint32_t rr = 0; rr < uint32_t(RHO); ++rr) {
        const uint32_t i1 = bi * RHO + rr;  // element row: pairs (i1 + 1, j), j <= i1
        if (i1 >= n1) break;
        const uint64_t ti = tri(i1);
        const uint32_t L = min(jlo + span, i1 + 1) - jlo;  // columns of the row in this run
        const uint64_t P0 = (ti + jlo + 31) & ~uint64_t(31);   // the first owned word
        const uint32_t q0 = static_cast<uint32_t>(P0 - ti - jlo);
        if (q0 >= L) continue;                                 // no word starts in this row and run
        const uint32_t nw = (L - q0 + 31) / 32;                // words starting in the run
        const bool cross = q0 + 32 * (nw - 1) + 31 > i1 - jlo; // the last one runs past the row end
        const uint32_t nfull = cross ? nw - 1 : nw;
        const float4 p = rows[rr];
        uint32_t w[NW];
        bool redo = false;
#pragma unroll
        for (int g = 0; g < NW; ++g) {
            const float4 q4 = cols[q0 + 32 * g + lane];
            if (SMALL) {
                // exact pre-test: max(|dx|, |dy|) > |r_i + r_j| rules the pair out; only a group
                // with a pair passing it takes the banded test
                const float e = fmaxf(fabsf(p.x - q4.x), fabsf(p.y - q4.y));
                w[g] = 0;
                if (__any_sync(0xffffffffu, e <= fabsf(p.w + q4.w))) {
                    bool near;
                    const bool hit = collide_f32_banded(p, q4, band_c, near);
                    redo = redo || (near && uint32_t(g) < nfull);
                    w[g] = __ballot_sync(0xffffffffu, hit);
                }
            } else {
                w[g] = __ballot_sync(0xffffffffu, collide_exact(bits_int4(p), bits_int4(q4)));
            }
        }
        if (SMALL && __any_sync(0xffffffffu, redo)) {  // a pair in the FP32 band: the row's words again, exactly
            const int4 pe = sphere(c, r, i1 + 1);
#pragma unroll
            for (int g = 0; g < NW; ++g)
                if (uint32_t(g) < nfull)
                    w[g] = __ballot_sync(0xffffffffu, collide_exact(pe, sphere(c, r, jlo + q0 + 32 * g + lane)));
        }
        uint32_t *wrow = bits + (P0 >> 5);
        if (lane == 0) {
#pragma unroll
            for (int g = 0; g < NW; ++g)
                if (uint32_t(g) < nfull) wrow[g] = w[g];
        }
        if (cross) {
            const uint32_t word =
                __ballot_sync(0xffffffffu, crossing_bit(c, r, P0 + 32 * uint64_t(nw - 1), i1, ti, total, lane));
            if (lane == 0) wrow[nw - 1] = word;
        }
    }
}

template <class Tiles, int RHO>
__global__ void __launch_bounds__(32 * kWarps) k_collide_chunked(Tiles tiles, uint32_t n1, uint32_t S, uint32_t rcap,
                                                                 const int32_t *__restrict__ c,
                                                                 const int32_t *__restrict__ r,
                                                                 uint32_t *__restrict__ bits)
{
    __shared__ __align__(16) float4 scol[kWarps][kCols];
    __shared__ __align__(16) float4 srow[kWarps][32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *cols = scol[warp], *rows = srow[warp];
    const uint64_t total = tri(n1);
    const uint64_t warps = uint64_t(gridDim.x) * kWarps;
    const uint64_t strips = (tiles.units + S - 1) / S;
    for (uint64_t z = uint64_t(blockIdx.x) * kWarps + warp; z < strips; z += warps) {
        const uint64_t uend = min(tiles.units, (z + 1) * S);
        for (uint64_t u = z * S; u < uend;) {
            uint32_t bi, bj;
            const bool ok = tiles(u, bi, bj);
            const uint32_t run = tiles.run(u, ok, bi, bj, static_cast<uint32_t>(min(uend - u, uint64_t(rcap))));
            u += run;
            if (!ok) continue;
            const uint32_t jlo = bj * RHO, span = run * RHO;
            __syncwarp();  // the previous run's reads of the slice are done
            bool small = true;
            uint32_t rm = 0;  // largest radius staged
#pragma unroll
            for (uint32_t k = 0; k < kCols / 32; ++k) {
                const uint32_t q = lane + 32 * k, j = jlo + q;
                const int4 s4 = (q < span + 32 && j < n1) ? sphere(c, r, j) : make_int4(0, 0, 0, 0);
                small = small && small_sphere(s4);
                rm = max(rm, uint32_t(abs(s4.w)));
                cols[q] = as_float4(s4);
            }
            uint32_t rmr = 0;
            {
                const uint32_t i1 = bi * RHO + lane;  // lane q < rho stages row sphere bi rho + q + 1
                const int4 p4 = (lane < uint32_t(RHO) && i1 < n1) ? sphere(c, r, i1 + 1) : make_int4(0, 0, 0, 0);
                small = small && small_sphere(p4);
                rmr = uint32_t(abs(p4.w));
                rows[lane] = as_float4(p4);
            }
            const bool all_small = __all_sync(0xffffffffu, small);
            if (!all_small) {  // large coordinates: the integers themselves, bit for bit
#pragma unroll
                for (uint32_t k = 0; k < kCols / 32; ++k) {
                    const uint32_t q = lane + 32 * k, j = jlo + q;
                    cols[q] = bits_float4((q < span + 32 && j < n1) ? sphere(c, r, j) : make_int4(0, 0, 0, 0));
                }
                const uint32_t i1 = bi * RHO + lane;
                rows[lane] = bits_float4((lane < uint32_t(RHO) && i1 < n1) ? sphere(c, r, i1 + 1) : make_int4(0, 0, 0, 0));
            }
            const float rmax = float(__reduce_max_sync(0xffffffffu, rm) + __reduce_max_sync(0xffffffffu, rmr));
            __syncwarp();
            if (all_small) run_rows<RHO, true>(cols, rows, 0x1p-20f * rmax * rmax, bi, jlo, span, n1, total, c, r, bits, lane);
            else run_rows<RHO, false>(cols, rows, 0.0f, bi, jlo, span, n1, total, c, r, bits, lane);
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
    const ChunkPlan cp = chunked_plan(t.units, RHO, resident, kStrip, kStrip);
    if (cp.W > kStrip || cp.W < uint32_t(RHO)) return fail(TD_ERR_INVALID_ARG, "strict collision run width %u", cp.W);
    const uint32_t S = cp.S;
    const uint64_t strips = (t.units + S - 1) / S;
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, (strips + kWarps - 1) / kWarps);
    k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, n1, S, cp.rcap, c, r, bits);
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
