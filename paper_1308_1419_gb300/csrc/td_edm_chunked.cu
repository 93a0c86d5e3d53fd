// td_edm_chunked.cu -- the Euclidean distance map of Sec. IV of arXiv:1308.1419 for few features
// (d <= 8) under the chunked schedule of the block strategies (g(lambda), BB, REC).  With few
// features the map is store-bound, and one element per thread (td_edm_pair.cu) leaves the HBM
// write rate far behind; this body stores aligned 16-byte chunks instead.
//
// Warps walk strips of consecutive units as the chunked probe does (td_probe.cu): a run of at most
// W / rho consecutive blocks (bi, bj) .. (bi, bj + run - 1) of one block row covers, in each of
// its rho element rows i, the contiguous packed range T(i) + [bj rho, min((bj + run) rho, i + 1)),
// and an aligned 16-byte chunk of the packed output is written by the run holding its first
// element.  Per run, the warp stages the column points x_j, j = bj rho .. bj rho + run rho + 3,
// in its slice of shared memory: one float4 per point for d = 3 and 4 (one 16-byte load per
// pair), feature-major rows otherwise.  Per element row it keeps x_i in registers and
// computes 128 columns at a time, lane l taking columns c + l + 32 m (m < 4: conflict-free shared
// reads); the 128 results go through a per-warp buffer so that lane l then stores the aligned
// chunk c + 4l .. c + 4l + 3 with one 16-byte streaming store.  A chunk that runs past the end of
// row i into the next row(s) (at most one per row) is computed from global memory after the run's
// rows, lane r taking row r, so the rows' crossings share their memory latency.
//
// The same kernel serves the strict lower triangle (td-problems without the diagonal, Eq.
// (theorem_nodiag) of Sec. II-A): its pairs (i, j), j < i < n, packed at i(i-1)/2 + j, form the
// with-diagonal packed triangle of side n - 1 whose row i' holds the pairs of point i' + 1 -- so
// the blocks of that triangle are mapped exactly as above and only the row point moves down by
// one (SHIFT = 1).
//
// Summation order as in every EDM kernel of libtd: t = x_i[k] - x_j[k], s = fma(t, t, s) for
// k = 0 .. d-1 from s = 0, then sqrtf -- bit-identical to td_edm_pair and the tiled kernels.
#include "td_internal.h"
#include "td_tiles.cuh"
#include "td_dist.cuh"

namespace td {
namespace {

constexpr uint32_t kWarps = 8, kMaxD = 8;
constexpr uint32_t kPad = 132;  // staged floats per feature row beyond the strip width (multiple of 4)

// d = 3 and 4 stage each column point as one float4 (one 16-byte shared load per pair); other d
// stage d feature rows.  Floats staged per column:
constexpr bool edm_chunk_pm(uint32_t d) { return d == 3 || d == 4; }
constexpr uint32_t edm_chunk_fpc(uint32_t d) { return edm_chunk_pm(d) ? 4u : d; }
// Widest strip a warp's shared-memory slice holds: (fpc sl + 128) floats per warp, sl = W + kPad.
// With more than 2 floats per column the slices of 512-element strips cost more occupancy than
// the longer runs gain (n = 32768, d = 4: 0.83 ms at 512, 0.73 ms at 256).
constexpr uint32_t edm_chunk_wmax(uint32_t d) { return edm_chunk_fpc(d) <= 2 ? 512u : 256u; }
constexpr size_t edm_chunk_smem(uint32_t d, uint32_t w)
{
    return size_t(kWarps) * (edm_chunk_fpc(d) * (w + kPad) + 128) * 4;
}

template <int D>
__device__ __forceinline__ float direct(const float *__restrict__ x, uint32_t d, uint32_t i, uint32_t j)
{
    const uint32_t dd = D ? D : d;
    const float *a = x + uint64_t(i) * dd, *b = x + uint64_t(j) * dd;
    float s = 0.0f;
#pragma unroll
    for (uint32_t k = 0; k < (D ? D : kMaxD); ++k) {
        if (D == 0 && k >= dd) break;
        const float t = __ldg(a + k) - __ldg(b + k);
        s = fmaf(t, t, s);
    }
    return dist_sqrt(s);
}

// The aligned chunk of packed elements P .. P + 3 that starts in row i (flat start ti) and runs
// past its end into the next row(s): the four (row, column) pairs are found first, then their
// point loads go out together, so one lane pays about one memory latency for the chunk.
template <int D, int SHIFT>
__device__ void crossing_chunk(const float *__restrict__ x, uint32_t d, uint32_t n, uint32_t i, uint64_t ti,
                               uint64_t P, float *__restrict__ out)
{
    uint32_t ii[4], jj[4];
    bool ok[4];
    uint32_t r = i;
    uint64_t tr = ti;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
        while (P + q > tr + r) {  // past the end of row r: into row r + 1
            tr += r + 1;
            ++r;
        }
        ok[q] = r < n;
        ii[q] = ok[q] ? r + SHIFT : 0u;
        jj[q] = ok[q] ? static_cast<uint32_t>(P + q - tr) : 0u;
    }
    if (D > 0) {
        float a[4][D ? D : 1], b[4][D ? D : 1];
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
#pragma unroll
            for (uint32_t k = 0; k < uint32_t(D); ++k) {
                a[q][k] = __ldg(x + uint64_t(ii[q]) * D + k);
                b[q][k] = __ldg(x + uint64_t(jj[q]) * D + k);
            }
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            float s = 0.0f;
#pragma unroll
            for (uint32_t k = 0; k < uint32_t(D); ++k) {
                const float t = a[q][k] - b[q][k];
                s = fmaf(t, t, s);
            }
            if (ok[q]) out[P + q] = dist_sqrt(s);
        }
    } else {
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
            if (ok[q]) out[P + q] = direct<0>(x, d, ii[q], jj[q]);
    }
}

// n: side of the packed triangle (the number of points minus SHIFT); row i of it pairs point
// i + SHIFT with the points j <= i.
template <class Tiles, int RHO, int D, int SHIFT>
__global__ void __launch_bounds__(32 * kWarps, 2) k_edm_chunked(Tiles tiles, uint32_t n, uint32_t S, uint32_t rcap, uint32_t sl,
                                                             const float *__restrict__ x, uint32_t d,
                                                             float *__restrict__ out)
{
    extern __shared__ __align__(16) float esm[];
    constexpr bool PM = edm_chunk_pm(D);  // column c staged as the float4 sx4[c] (d = 3, 4)
    const uint32_t dd = D ? D : d, fpc = PM ? 4u : dd;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *sx = esm + warp * (fpc * sl + 128);  // dd feature rows of sl floats: column c of the run
    float4 *sx4 = reinterpret_cast<float4 *>(sx);
    float *sres = sx + fpc * sl;                // results of the current 128 columns
    const uint64_t warps = uint64_t(gridDim.x) * kWarps;
    const uint64_t strips = (tiles.units + S - 1) / S;
    for (uint64_t z = uint64_t(blockIdx.x) * kWarps + warp; z < strips; z += warps) {
        const uint64_t uend = min(tiles.units, (z + 1) * S);
        for (uint64_t u = z * S; u < uend;) {
            uint32_t bi, bj;
            const bool ok = tiles(u, bi, bj);
            const uint32_t run = tiles.run(u, ok, bi, bj, static_cast<uint32_t>(min(uend - u, uint64_t(rcap))));
            u += Tiles::kRuns ? 1u : run;
            if (!ok) continue;
            const uint32_t jlo = bj * RHO, ncol = run * RHO + 4;
            __syncwarp();  // the previous run's reads of the slice are done
            for (uint32_t c = lane; c < ncol; c += 32) {
                const uint32_t j = jlo + c;
                const float *xj = x + uint64_t(j) * dd;
                if (PM) {
                    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (j < n) {
                        v.x = __ldg(xj);
                        v.y = __ldg(xj + 1);
                        v.z = __ldg(xj + 2);
                        if (D == 4) v.w = __ldg(xj + 3);
                    }
                    sx4[c] = v;
                } else {
#pragma unroll
                    for (uint32_t k = 0; k < (D ? D : kMaxD); ++k) {
                        if (D == 0 && k >= dd) break;
                        sx[k * sl + c] = j < n ? __ldg(xj + k) : 0.0f;
                    }
                }
            }
            __syncwarp();
            for (uint32_t r = 0; r < uint32_t(RHO); ++r) {
                const uint32_t i = bi * RHO + r;
                if (i >= n) break;
                const uint32_t jhi = min((bj + run) * RHO, i + 1);  // row-local end (exclusive)
                const uint64_t ti = tri(i);
                // first column >= jlo whose flat index T(i) + j is a multiple of 4
                const uint32_t c0 = jlo + ((4u - ((static_cast<uint32_t>(ti) + jlo) & 3u)) & 3u);
                float xi[D ? D : kMaxD];
#pragma unroll
                for (uint32_t k = 0; k < (D ? D : kMaxD); ++k) xi[k] = (D || k < dd) ? __ldg(x + uint64_t(i + SHIFT) * dd + k) : 0.0f;
                for (uint32_t jb = c0; jb < jhi; jb += 128) {
                    {
                        const uint32_t c = jb - jlo + lane;
                        float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                        if (PM) {
                            float4 q[4];
#pragma unroll
                            for (uint32_t m = 0; m < 4; ++m) q[m] = sx4[c + 32 * m];
                            const float qv[4][4] = {{q[0].x, q[0].y, q[0].z, q[0].w}, {q[1].x, q[1].y, q[1].z, q[1].w},
                                                    {q[2].x, q[2].y, q[2].z, q[2].w}, {q[3].x, q[3].y, q[3].z, q[3].w}};
#pragma unroll
                            for (uint32_t k = 0; k < uint32_t(D); ++k) {
                                float t[4];
#pragma unroll
                                for (uint32_t m = 0; m < 4; ++m) t[m] = xi[k] - qv[m][k];
#pragma unroll
                                for (uint32_t m = 0; m < 4; ++m) s[m] = fmaf(t[m], t[m], s[m]);
                            }
                        } else {
#pragma unroll
                            for (uint32_t k = 0; k < (D ? D : kMaxD); ++k) {
                                if (D == 0 && k >= dd) break;
                                float t[4];
#pragma unroll
                                for (uint32_t m = 0; m < 4; ++m) t[m] = xi[k] - sx[k * sl + c + 32 * m];
#pragma unroll
                                for (uint32_t m = 0; m < 4; ++m) s[m] = fmaf(t[m], t[m], s[m]);
                            }
                        }
#pragma unroll
                        for (uint32_t m = 0; m < 4; ++m) sres[lane + 32 * m] = dist_sqrt(s[m]);
                    }
                    __syncwarp();
                    const uint32_t j = jb + 4 * lane;
                    // a chunk that runs past the end of row i is left to the crossing pass below
                    if (j < jhi && j + 3 <= i)
                        __stcs(reinterpret_cast<float4 *>(out + ti + j), *reinterpret_cast<const float4 *>(sres + 4 * lane));
                    __syncwarp();  // sres is rewritten by the next column group
                }
            }
            // crossing pass: lane r takes element row bi rho + r, whose last chunk runs past the row
            // end unless the row ends on a 16-byte boundary; this run writes it if the chunk's first
            // element lies in the run's columns of that row
            if (lane < uint32_t(RHO)) {
                const uint32_t i = bi * RHO + lane;
                if (i < n) {
                    const uint64_t ti = tri(i), E = ti + i + 1;  // flat end (exclusive) of row i
                    const uint64_t Pc = (E - 1) & ~uint64_t(3);
                    const uint32_t jc = static_cast<uint32_t>(Pc - ti), jhi = min((bj + run) * RHO, i + 1);
                    if ((E & 3u) != 0 && Pc >= ti && jc >= jlo && jc < jhi)
                        crossing_chunk<D, SHIFT>(x, d, n, i, ti, Pc, out);
                }
            }
        }
    }
}

// Column-aligned form for d <= 4.  Lane l of a warp computes the four columns b .. b + 3,
// b = jlo + 124 m + 4 l (jlo a multiple of 4), for four element rows at a time: the columns' 4 d
// coordinates are contiguous and 16-byte aligned in x (b d a multiple of 4), so they come as d
// 16-byte loads (through L1, where every row of the run finds them) and serve 16 pairs.  The
// packed offset T(i) + b is T(i) mod 4 past the 16-byte grid for every lane alike, so the run's
// first aligned chunk of row i starts at column jlo + o_i, o_i = -T(i) mod 4, and the chunk of lane
// l holds lane l's last 4 - o_i values and lane l + 1's first o_i values (o_i shuffles down);
// lanes 0 .. 30 store, lane 31 only lends its values, so a step covers 124 columns.  Chunks that
// run past the row end are left to the crossing pass, as in the staged form.
template <int D>
__device__ __forceinline__ void load_cols4(const float *__restrict__ x, uint32_t b, uint32_t np, float (&q)[4][D])
{
    if (b + 4 <= np) {
        const float4 *p = reinterpret_cast<const float4 *>(x + uint64_t(b) * D);
        float f[4 * D];
#pragma unroll
        for (int v = 0; v < D; ++v) {
            const float4 t = __ldg(p + v);
            f[4 * v] = t.x;
            f[4 * v + 1] = t.y;
            f[4 * v + 2] = t.z;
            f[4 * v + 3] = t.w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int k = 0; k < D; ++k) q[c][k] = f[c * D + k];
    } else {  // the last points of x: no read past its end
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int k = 0; k < D; ++k) q[c][k] = b + c < np ? __ldg(x + uint64_t(b + c) * D + k) : 0.0f;
    }
}

// The aligned chunk of one row from this lane's four values and the next lane's (o uniform).
__device__ __forceinline__ float4 chunk_of(const float (&v)[4], uint32_t o)
{
    if (o == 0) return make_float4(v[0], v[1], v[2], v[3]);
    if (o == 1) return make_float4(v[1], v[2], v[3], __shfl_down_sync(0xffffffffu, v[0], 1));
    if (o == 2)
        return make_float4(v[2], v[3], __shfl_down_sync(0xffffffffu, v[0], 1), __shfl_down_sync(0xffffffffu, v[1], 1));
    return make_float4(v[3], __shfl_down_sync(0xffffffffu, v[0], 1), __shfl_down_sync(0xffffffffu, v[1], 1),
                       __shfl_down_sync(0xffffffffu, v[2], 1));
}

constexpr int kRows = 4;  // element rows per step of the column-aligned form

template <class Tiles, int RHO, int D, int SHIFT>
__global__ void __launch_bounds__(32 * kWarps) k_edm_stream(Tiles tiles, uint32_t n, uint32_t S, uint32_t rcap,
                                                            const float *__restrict__ x, float *__restrict__ out)
{
    static_assert(D >= 1 && D <= 4 && RHO % kRows == 0, "column-aligned form: 1 <= d <= 4");
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t np = n + SHIFT;  // points in x
    const uint64_t warps = uint64_t(gridDim.x) * kWarps;
    const uint64_t strips = (tiles.units + S - 1) / S;
    for (uint64_t z = uint64_t(blockIdx.x) * kWarps + warp; z < strips; z += warps) {
        const uint64_t uend = min(tiles.units, (z + 1) * S);
        for (uint64_t u = z * S; u < uend;) {
            uint32_t bi, bj;
            const bool ok = tiles(u, bi, bj);
            const uint32_t run = tiles.run(u, ok, bi, bj, static_cast<uint32_t>(min(uend - u, uint64_t(rcap))));
            u += Tiles::kRuns ? 1u : run;
            if (!ok) continue;
            const uint32_t jlo = bj * RHO, jend = (bj + run) * RHO;
            for (uint32_t r0 = 0; r0 < uint32_t(RHO); r0 += kRows) {
                const uint32_t i0 = bi * RHO + r0;
                if (i0 >= n) break;
                float xi[kRows][D];
                uint64_t ti[kRows];
                uint32_t o[kRows], lim[kRows];  // lim: owned chunks start before column jlo + lim
                uint32_t reach = 0;
#pragma unroll
                for (int a = 0; a < kRows; ++a) {
                    const uint32_t i = i0 + a;
                    ti[a] = tri(i);
                    o[a] = (4u - (static_cast<uint32_t>(ti[a]) & 3u)) & 3u;
                    lim[a] = i < n ? min(jend, i + 1) - jlo : 0u;
                    reach = max(reach, lim[a] > o[a] ? lim[a] - o[a] : 0u);
#pragma unroll
                    for (int k = 0; k < D; ++k) xi[a][k] = i < n ? __ldg(x + uint64_t(i + SHIFT) * D + k) : 0.0f;
                }
                for (uint32_t c0 = 0; c0 < reach; c0 += 124) {
                    const uint32_t c = c0 + 4 * lane;  // local column of this lane's first value
                    float q[4][D];
                    load_cols4<D>(x, jlo + c, np, q);
#pragma unroll
                    for (int a = 0; a < kRows; ++a) {
                        float v[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            float s = 0.0f;
#pragma unroll
                            for (int k = 0; k < D; ++k) {
                                const float t = xi[a][k] - q[m][k];
                                s = fmaf(t, t, s);
                            }
                            v[m] = dist_sqrt(s);
                        }
                        const float4 w = chunk_of(v, o[a]);
                        const uint32_t cs = c + o[a];  // local column of the chunk's first element
                        if (lane < 31 && cs < lim[a] && jlo + cs + 3 <= i0 + a)
                            __stcs(reinterpret_cast<float4 *>(out + ti[a] + jlo + cs), w);
                    }
                }
            }
            // crossing pass: lane r takes element row bi rho + r, whose last chunk runs past the row end
            // unless the row ends on a 16-byte boundary; this run writes it if its first element lies
            // in the run's columns of that row
            if (lane < uint32_t(RHO)) {
                const uint32_t i = bi * RHO + lane;
                if (i < n) {
                    const uint64_t t = tri(i), E = t + i + 1;
                    const uint64_t Pc = (E - 1) & ~uint64_t(3);
                    const uint32_t jc = static_cast<uint32_t>(Pc - t), jhi = min(jend, i + 1);
                    if ((E & 3u) != 0 && Pc >= t && jc >= jlo && jc < jhi)
                        crossing_chunk<D, SHIFT>(x, D, n, i, t, Pc, out);
                }
            }
        }
    }
}

template <class Tiles, int RHO, int D, int SHIFT = 0>
td_status launch_stream(const Tiles &t, const float *x, uint32_t n, float *out, cudaStream_t st, uint64_t *ctas)
{
    if (t.units == 0) return TD_OK;
    auto k = k_edm_stream<Tiles, RHO, D, SHIFT>;
    const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, ~0ull) * kWarps;
    const ChunkPlan cp = chunked_plan(t.units, RHO, resident, 2048, 8192);
    const uint64_t strips = (t.units + cp.S - 1) / cp.S;
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, (strips + kWarps - 1) / kWarps);
    k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, n, cp.S, cp.rcap, x, out);
    *ctas += g;
    return launch_status("td_edm chunked kernel (column-aligned)");
}

template <class Tiles, int RHO, int D, int SHIFT = 0>
td_status launch_tiles(const Tiles &t, const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st,
                       uint64_t *ctas)
{
    if (t.units == 0) return TD_OK;
    // three and four features: the column-aligned form (measured faster there); one, two and more
    // than four: the staged form
    if (D == 3 || D == 4) return launch_stream<Tiles, RHO, (D == 4 ? 4 : 3), SHIFT>(t, x, n, out, st, ctas);
    auto k = k_edm_chunked<Tiles, RHO, D, SHIFT>;
    const uint32_t wmax = edm_chunk_wmax(d);
    const size_t smax = edm_chunk_smem(d, wmax);
    td_status s = set_dynamic_smem_once(reinterpret_cast<const void *>(k), smax);
    if (s != TD_OK) return s;
    const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, smax, ~0ull) * kWarps;
    const ChunkPlan cp = chunked_plan(t.units, RHO, resident, wmax, wmax);
    const uint32_t sl = cp.W + kPad;
    const size_t smem = edm_chunk_smem(d, cp.W);
    const uint64_t strips = (t.units + cp.S - 1) / cp.S;
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, smem, (strips + kWarps - 1) / kWarps);
    k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, smem, st>>>(t, n, cp.S, cp.rcap, sl, x, d, out);
    *ctas += g;
    return launch_status("td_edm chunked kernel");
}

// g(lambda) under the chunked schedule, by runs: the plan comes from the block count as for the
// other sources, then the warps take runs of R = min(run cap, strip) blocks numbered by
// tiles::LtmRuns, one run per strip, so that no run crosses the end of a block row (consecutive
// lambda would cut a strip in two at every row end of the triangle).
template <int RHO, int D, int SHIFT = 0>
td_status launch_ltm_runs(const Plan &p, const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st,
                          uint64_t *ctas)
{
    const uint64_t blocks = p.sliced ? p.slice_units : tri(p.nb);
    if (blocks == 0) return TD_OK;
    if (D == 3 || D == 4) {
        auto k = k_edm_stream<tiles::LtmRuns, RHO, (D == 4 ? 4 : 3), SHIFT>;
        const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, ~0ull) * kWarps;
        const ChunkPlan cp = chunked_plan(blocks, RHO, resident, 2048, 8192);
        uint32_t R = cp.S < cp.rcap ? cp.S : cp.rcap;
        // a row's steps cover 124 columns each and its chunks reach 3 columns past the run: trim the
        // run to the most blocks that still fit whole steps (16 -> 15 blocks at rho 16, 64 -> 61)
        const uint32_t steps = (R * RHO + 3) / 124;
        if (steps >= 1 && (steps * 124 - 3) / RHO >= 1) R = min(R, (steps * 124 - 3) / RHO);
        if (R == 1)  // runs of one block: the blocks themselves, by g(lambda) alone
            return launch_stream<tiles::Ltm, RHO, (D == 4 ? 4 : 3), SHIFT>(tiles::ltm_source(p), x, n, out, st, ctas);
        const tiles::LtmRuns t = tiles::ltm_runs_source(p, R);
        const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, 0, (t.units + kWarps - 1) / kWarps);
        k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, 0, st>>>(t, n, 1u, R, x, out);
        *ctas += g;
        return launch_status("td_edm chunked kernel (column-aligned, runs)");
    }
    auto k = k_edm_chunked<tiles::LtmRuns, RHO, D, SHIFT>;
    const uint32_t wmax = edm_chunk_wmax(d);
    const size_t smax = edm_chunk_smem(d, wmax);
    td_status s = set_dynamic_smem_once(reinterpret_cast<const void *>(k), smax);
    if (s != TD_OK) return s;
    const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, smax, ~0ull) * kWarps;
    const ChunkPlan cp = chunked_plan(blocks, RHO, resident, wmax, wmax);
    const uint32_t R = cp.S < cp.rcap ? cp.S : cp.rcap;
    if (R == 1) return launch_tiles<tiles::Ltm, RHO, D, SHIFT>(tiles::ltm_source(p), x, n, d, out, st, ctas);
    const tiles::LtmRuns t = tiles::ltm_runs_source(p, R);
    const uint32_t sl = cp.W + kPad;
    const size_t smem = edm_chunk_smem(d, cp.W);
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 32 * kWarps, smem, (t.units + kWarps - 1) / kWarps);
    k<<<dim3(static_cast<uint32_t>(g)), 32 * kWarps, smem, st>>>(t, n, 1u, R, sl, x, d, out);
    *ctas += g;
    return launch_status("td_edm chunked kernel (runs)");
}

template <int RHO, int D>
td_status launch_rho(td_mapping m, const float *x, uint32_t n, uint32_t d, float *out, const Plan &p, bool strict,
                     cudaStream_t st, uint64_t *ctas)
{
    if (strict) {  // the strict triangle of n points = the packed triangle of side n - 1, rows shifted
        if (m == TD_MAP_LTM) return launch_ltm_runs<RHO, D, 1>(p, x, n - 1, d, out, st, ctas);
        if (m == TD_MAP_BB)
            return launch_tiles<tiles::Bb, RHO, D, 1>(tiles::Bb{uint64_t(p.nb) * p.nb, p.nb}, x, n - 1, d, out, st, ctas);
        return fail(TD_ERR_UNSUPPORTED, "the block-mapped strict distance map serves LTM and BB");
    }
    switch (m) {
    case TD_MAP_LTM: return launch_ltm_runs<RHO, D>(p, x, n, d, out, st, ctas);
    case TD_MAP_UTM_BLOCK:
        return launch_tiles<tiles::UtmBlk, RHO, D>(tiles::UtmBlk{tri(p.nb), p.nb}, x, n, d, out, st, ctas);
    case TD_MAP_BB:
        return launch_tiles<tiles::Bb, RHO, D>(tiles::bb_source(p), x, n, d, out, st, ctas);
    case TD_MAP_REC: {
        for (uint32_t l = 1; l <= p.rec_k; ++l) {
            const uint32_t sb = (n >> l) / RHO, gx = n / (2 * RHO);
            const td_status s =
                launch_tiles<tiles::RecLevel, RHO, D>(tiles::RecLevel{uint64_t(gx) * sb, sb, gx}, x, n, d, out, st, ctas);
            if (s != TD_OK) return s;
        }
        const uint32_t mb = p.rec_m / RHO, gx = n / RHO;
        return launch_tiles<tiles::RecDiag, RHO, D>(tiles::RecDiag{uint64_t(gx) * mb, mb, gx}, x, n, d, out, st, ctas);
    }
    default:
        return fail(TD_ERR_UNSUPPORTED, "the chunked schedule serves the block strategies LTM, BB and REC");
    }
}

template <int D>
td_status launch_d(td_mapping m, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out, const Plan &p,
                   bool strict, cudaStream_t st, uint64_t *ctas)
{
    switch (rho) {
    case 8: return launch_rho<8, D>(m, x, n, d, out, p, strict, st, ctas);
    case 16: return launch_rho<16, D>(m, x, n, d, out, p, strict, st, ctas);
    case 32: return launch_rho<32, D>(m, x, n, d, out, p, strict, st, ctas);
    default: return fail(TD_ERR_INVALID_ARG, "the chunked distance map needs rho 8, 16 or 32 (got %u)", rho);
    }
}

}  // namespace

td_status launch_edm_chunked(td_mapping m, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out,
                             const Plan &p, bool strict, cudaStream_t st, uint64_t *ctas)
{
    if (d == 0 || d > kMaxD)
        return fail(TD_ERR_UNSUPPORTED, "the chunked distance map serves d <= %u (got %u); use rho 64/128", kMaxD, d);
    switch (d) {
    case 1: return launch_d<1>(m, x, n, d, rho, out, p, strict, st, ctas);
    case 2: return launch_d<2>(m, x, n, d, rho, out, p, strict, st, ctas);
    case 3: return launch_d<3>(m, x, n, d, rho, out, p, strict, st, ctas);
    case 4: return launch_d<4>(m, x, n, d, rho, out, p, strict, st, ctas);
    default: return launch_d<0>(m, x, n, d, rho, out, p, strict, st, ctas);
    }
}

}  // namespace td
