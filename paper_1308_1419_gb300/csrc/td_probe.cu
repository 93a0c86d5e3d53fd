// td_probe.cu -- the five strategies' launch spaces (td_strategies.cuh) driving the probe body
// (the paper's dummy kernel of Sec. III-A, made to write every in-domain element) or the
// coverage body (one atomic increment per in-domain thread), plus the mapping dump and the
// exhaustive self-check of g(lambda).
#include "td_strategies.cuh"
#include "td_tiles.cuh"

namespace td {
namespace {

struct ProbeBody {
    uint32_t *out;
    uint32_t N;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t j) const
    {
        out[tri(i) + j] = splitmix32(i * N + j);
    }
};

// The dummy kernel of Sec. III-A / IV test 1 as a map-only body: the thread's (i, j) feeds a store
// that no in-domain pair reaches (i + j <= 2N - 2 < 2^32 - 1), so the mapping cannot be
// optimised away, yet nothing is written (the paper's store of i + j to one fixed address
// would serialise every thread of the launch on one L2 line here).
struct DummyBody {
    uint32_t *sink;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t j) const
    {
        if (i + j == 0xFFFFFFFFu) *sink = i;
    }
};

struct CoverBody {
    uint32_t *count;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t j) const
    {
        atomicAdd(&count[tri(i) + j], 1u);
    }
};

// ---------------------------------------------------------------- chunked probe (block strategies)
// Persistent warps walk the launch space in strips of S consecutive units (chunked_plan: W / rho
// for large launches, W a power of two chosen per launch, or an even share per warp for small
// ones).  Units that continue one block row -- blocks (bi, bj), (bi, bj+1), ..., at most W / rho
// of them -- cover, in each element row i of that block row, one contiguous flat range [s, e) of
// the packed output (s = T(i) + bj rho), at most W elements long.  The flat output is cut into aligned 4-element (16-byte) chunks,
// and chunk c is written by the block row range holding its first element 4c: the blocks of
// every block strategy cover each element exactly once, so each chunk has exactly one writer.
// All 32 lanes of a warp work on the same element row, lane l on chunks l, l + 32, ... of [s, e),
// so one store instruction writes up to 512 contiguous bytes; the stores are streaming
// (st.global.cs), since every line is written once and never read back by the kernel.  A chunk that runs past e continues in
// the same packed row or, at a row end, into the first elements of the next row(s); the probe
// value is a function of (i, j) alone, so the writer computes it wherever the element lies.
// splitmix32 with its right shifts taken as high halves of multiplications
// (z >> s = umulhi(z, 2^(32-s))): the same function, but the shifts issue on the FMA pipe
// instead of the integer ALU pipe, which the xors and the index arithmetic already load.
__device__ __forceinline__ uint32_t xor_shr(uint32_t z, uint32_t pow2) { return z ^ __umulhi(z, pow2); }

__device__ __forceinline__ uint32_t splitmix32_mulshift(uint32_t x)
{
    uint32_t z = x + 0x9E3779B9u;
    z = xor_shr(z, 1u << 16) * 0x85EBCA6Bu;
    z = xor_shr(z, 1u << 19) * 0xC2B2AE35u;
    return xor_shr(z, 1u << 16);
}

__device__ __forceinline__ uint4 probe4(uint32_t key)
{
    return make_uint4(splitmix32_mulshift(key), splitmix32_mulshift(key + 1), splitmix32_mulshift(key + 2),
                      splitmix32_mulshift(key + 3));
}

// The chunk of 4 elements starting at row-local j of row i (flat T(i) + j, a multiple of 4).
// COVER: add 1 to each element's count instead of writing its probe value.
template <bool COVER>
__device__ __forceinline__ void probe_chunk(uint32_t *__restrict__ out, uint32_t N, uint32_t i, uint64_t ti,
                                            uint32_t j)
{
    if (j + 3 <= i) {
        if (COVER) {
            for (uint32_t k = 0; k < 4; ++k) atomicAdd(out + ti + j + k, 1u);
        } else {
            __stcs(reinterpret_cast<uint4 *>(out + ti + j), probe4(i * N + j));
        }
    } else {  // the chunk runs past the end of row i into the next row(s)
        uint32_t ii = i;
        uint64_t tii = ti;
        for (uint32_t k = 0; k < 4; ++k) {
            const uint64_t P = ti + j + k;
            while (P > tii + ii) {
                tii += ii + 1;
                ++ii;
            }
            if (ii >= N) break;
            if (COVER) atomicAdd(out + P, 1u);
            else out[P] = splitmix32_mulshift(ii * N + static_cast<uint32_t>(P - tii));
        }
    }
}

// CPL > 0: strips at most 128 CPL elements wide, each lane's chunks of a row in a fully unrolled
// loop; CPL = 0: any width, a runtime loop (the wide strips of large launches).  COVER: the
// coverage count under the same schedule (every element must be reached exactly once).
template <class Tiles, int RHO, int CPL, bool COVER>
__global__ void __launch_bounds__(256) k_probe_chunked(Tiles tiles, uint32_t N, uint32_t S, uint32_t rcap,
                                                     uint32_t *__restrict__ out)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
    const uint64_t strips = (tiles.units + S - 1) / S;
    for (uint64_t z = uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); z < strips; z += warps) {
        const uint64_t uend = min(tiles.units, (z + 1) * S);
        for (uint64_t u = z * S; u < uend;) {
            uint32_t bi, bj;
            const bool ok = tiles(u, bi, bj);
            const uint32_t run = tiles.run(u, ok, bi, bj, static_cast<uint32_t>(min(uend - u, uint64_t(rcap))));
            u += run;
            if (!ok) continue;
            const uint32_t jlo = bj * RHO;
            for (uint32_t r = 0; r < uint32_t(RHO); ++r) {
                const uint32_t i = bi * RHO + r;
                if (i >= N) break;
                const uint32_t jhi = min((bj + run) * RHO, i + 1);  // row-local end (exclusive)
                const uint64_t ti = tri(i);
                // first row-local j >= jlo whose flat index T(i) + j is a multiple of 4
                const uint32_t c0 = jlo + ((4u - ((static_cast<uint32_t>(ti) + jlo) & 3u)) & 3u);
                if (CPL > 0) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const uint32_t j = c0 + 4 * (lane + 32 * c);
                        if (j >= jhi) break;
                        probe_chunk<COVER>(out, N, i, ti, j);
                    }
                } else {
#pragma unroll 2
                    for (uint32_t j = c0 + 4 * lane; j < jhi; j += 128) probe_chunk<COVER>(out, N, i, ti, j);
                }
            }
        }
    }
}

// Strip width: longer contiguous row segments per warp raise the write bandwidth at large N
// (more of each DRAM page is written by one warp), but fewer strips balance worse over the
// resident warps.  Default: the widest power of two in [256, kStripMax] that still leaves four
// strips per resident warp (chunked_plan); the library option overrides it.
constexpr uint32_t kStripMax = 2048;


template <class Tiles, int RHO, bool COVER>
td_status launch_chunked_tiles(const Tiles &t, uint32_t N, uint32_t *out, cudaStream_t st, uint64_t *ctas)
{
    if (t.units == 0) return TD_OK;
    auto wide = k_probe_chunked<Tiles, RHO, 0, COVER>;
    auto narrow = k_probe_chunked<Tiles, RHO, 2, COVER>;
    const uint64_t resident = persistent_ctas(reinterpret_cast<const void *>(wide), 256, 0, ~0ull) * 8;
    const ChunkPlan cp = chunked_plan(t.units, RHO, resident, kStripMax, 8192);
    const auto k = cp.W <= 256 ? narrow : wide;
    const uint64_t strips = (t.units + cp.S - 1) / cp.S;
    const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 256, 0, (strips + 7) / 8);
    k<<<dim3(static_cast<uint32_t>(g)), 256, 0, st>>>(t, N, cp.S, cp.rcap, out);
    *ctas += g;
    return launch_status("td probe chunked kernel");
}

template <int RHO, bool COVER>
td_status launch_chunked_rho(td_mapping m, uint32_t N, uint32_t *out, const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    switch (m) {
    case TD_MAP_LTM: return launch_chunked_tiles<tiles::Ltm, RHO, COVER>(tiles::ltm_source(p), N, out, st, ctas);
    case TD_MAP_UTM_BLOCK:
        return launch_chunked_tiles<tiles::UtmBlk, RHO, COVER>(tiles::UtmBlk{tri(p.nb), p.nb}, N, out, st, ctas);
    case TD_MAP_BB:
        return launch_chunked_tiles<tiles::Bb, RHO, COVER>(tiles::bb_source(p), N, out, st, ctas);
    case TD_MAP_REC: {
        for (uint32_t l = 1; l <= p.rec_k; ++l) {
            const uint32_t sb = (N >> l) / RHO, gx = N / (2 * RHO);
            const td_status s = launch_chunked_tiles<tiles::RecLevel, RHO, COVER>(
                tiles::RecLevel{uint64_t(gx) * sb, sb, gx}, N, out, st, ctas);
            if (s != TD_OK) return s;
        }
        const uint32_t mb = p.rec_m / RHO, gx = N / RHO;
        return launch_chunked_tiles<tiles::RecDiag, RHO, COVER>(tiles::RecDiag{uint64_t(gx) * mb, mb, gx}, N, out,
                                                                st, ctas);
    }
    default:
        return fail(TD_ERR_UNSUPPORTED, "the chunked schedule serves the block strategies LTM, BB and REC");
    }
}

// ---------------------------------------------------------------- dump and self-check

__global__ void k_map_dump(int m, uint32_t N, uint32_t W, uint64_t u0, uint64_t count, uint32_t *ij)
{
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const uint64_t u = u0 + q;
        uint32_t i, j;
        if (m == TD_MAP_LTM) {
            ltm_g(u, i, j);
        } else if (m == TD_MAP_LTM_X) {
            LtmSqrt{}(u, i, j);
        } else if (m == TD_MAP_LTM_N) {
            LtmNewton{}(u, i, j);
        } else if (m == TD_MAP_LTM_N_FMA) {
            LtmNewtonFma{}(u, i, j);
        } else if (m == TD_MAP_LTM_R) {
            LtmRsqrtEps{}(u, i, j);
        } else if (m == TD_MAP_UTM_BLOCK) {
            UtmBlock{N}(u, i, j);
        } else if (m == TD_MAP_UTM) {
            utm_map(u, N, i, j);
        } else {
            const uint32_t y = static_cast<uint32_t>(u / W), x = static_cast<uint32_t>(u - uint64_t(y) * W);
            rb_map(N, x, y, i, j);
        }
        ij[2 * q] = i;
        ij[2 * q + 1] = j;
    }
}

// Counts the lambda whose (i, j) from Map breaks T(i) <= lambda <= T(i) + i, j = lambda - T(i)
// (exact 64-bit arithmetic), and the smallest such lambda.
template <class Map>
__global__ void k_ltm_check(uint64_t lam0, uint64_t count, unsigned long long *res)
{
    unsigned long long bad = 0, first = ~0ull;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t q = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const uint64_t lam = lam0 + q;
        uint32_t i, j;
        Map{}(lam, i, j);
        const uint64_t t = tri(i);
        const bool ok = t <= lam && lam - t <= i && uint64_t(j) == lam - t;
        if (!ok) {
            ++bad;
            first = first < lam ? first : lam;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        const unsigned long long f = __shfl_xor_sync(0xffffffffu, first, o);
        first = f < first ? f : first;
    }
    if ((threadIdx.x & 31) == 0 && bad) {
        atomicAdd(&res[0], bad);
        atomicMin(&res[1], first);
    }
}

// The Sec. III-A evaluations of g in the paper-style LTM kernel (one CTA or grid-stride step per
// block, one element per thread).
template <class Map, class Body>
td_status launch_variant_map(bool P, uint32_t N, uint32_t rho, Body body, const Plan &p, cudaStream_t st,
                             uint64_t *ctas)
{
    switch (rho) {
    case 8: strat::launch_ltm<8, Body, Map>(P, N, body, p, st, ctas); break;
    case 16: strat::launch_ltm<16, Body, Map>(P, N, body, p, st, ctas); break;
    case 32: strat::launch_ltm<32, Body, Map>(P, N, body, p, st, ctas); break;
    default: return fail(TD_ERR_INVALID_ARG, "rho must be 8, 16 or 32 (got %u)", rho);
    }
    return launch_status("td probe/cover kernel (LTM variant)");
}

template <class Body>
td_status launch_variant(td_mapping m, bool P, uint32_t N, uint32_t rho, Body body, const Plan &p, cudaStream_t st,
                         uint64_t *ctas)
{
    switch (m) {
    case TD_MAP_LTM_X: return launch_variant_map<LtmSqrt>(P, N, rho, body, p, st, ctas);
    case TD_MAP_LTM_N: return launch_variant_map<LtmNewton>(P, N, rho, body, p, st, ctas);
    case TD_MAP_LTM_N_FMA: return launch_variant_map<LtmNewtonFma>(P, N, rho, body, p, st, ctas);
    case TD_MAP_LTM_R: return launch_variant_map<LtmRsqrtEps>(P, N, rho, body, p, st, ctas);
    default: return fail(TD_ERR_INVALID_ARG, "not an LTM variant (%d)", int(m));
    }
}

}  // namespace

ChunkPlan chunked_plan(uint64_t units, uint32_t rho, uint64_t resident_warps, uint32_t wauto, uint32_t wlimit)
{
    const int forced = option(TD_OPT_PROBE_STRIP);
    uint32_t w = wauto < 256 ? wauto : 256;
    if (forced > 0) {
        w = uint32_t(forced) < wlimit ? uint32_t(forced) : wlimit;
    } else {
        while (w < wauto && units * rho / (2 * w) >= 4 * resident_warps) w *= 2;
    }
    ChunkPlan p;
    p.W = w < rho ? rho : w;
    p.rcap = p.W / rho;
    if (resident_warps == 0) resident_warps = 1;
    if (units >= 4 * resident_warps * p.rcap) {
        p.S = p.rcap;
    } else {
        const uint64_t share = (units + resident_warps - 1) / resident_warps;
        p.S = static_cast<uint32_t>(share ? share : 1);
    }
    return p;
}

td_status launch_dummy(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, uint32_t *sink, const Plan &p,
                       cudaStream_t st, uint64_t *ctas)
{
    if (s == TD_SCHED_CHUNKED) return fail(TD_ERR_UNSUPPORTED, "the dummy kernel uses the GRID or PERSISTENT schedule");
    if (ltm_variant(m)) return launch_variant(m, s == TD_SCHED_PERSISTENT, N, rho, DummyBody{sink}, p, st, ctas);
    return strat::launch_body(m, s, N, rho, DummyBody{sink}, p, st, ctas);
}

td_status launch_probe(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, uint32_t *out, bool cover,
                       const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    if (s == TD_SCHED_CHUNKED) {
        switch (rho) {
        case 8: return cover ? launch_chunked_rho<8, true>(m, N, out, p, st, ctas)
                             : launch_chunked_rho<8, false>(m, N, out, p, st, ctas);
        case 16: return cover ? launch_chunked_rho<16, true>(m, N, out, p, st, ctas)
                              : launch_chunked_rho<16, false>(m, N, out, p, st, ctas);
        case 32: return cover ? launch_chunked_rho<32, true>(m, N, out, p, st, ctas)
                              : launch_chunked_rho<32, false>(m, N, out, p, st, ctas);
        default: return fail(TD_ERR_INVALID_ARG, "rho must be 8, 16 or 32");
        }
    }
    if (ltm_variant(m)) {
        const bool P = s == TD_SCHED_PERSISTENT;
        if (cover) return launch_variant(m, P, N, rho, CoverBody{out}, p, st, ctas);
        return launch_variant(m, P, N, rho, ProbeBody{out, N}, p, st, ctas);
    }
    if (cover) return strat::launch_body(m, s, N, rho, CoverBody{out}, p, st, ctas);
    return strat::launch_body(m, s, N, rho, ProbeBody{out, N}, p, st, ctas);
}

td_status launch_map_dump(td_mapping m, uint32_t N, uint64_t u0, uint64_t count, uint32_t *ij, cudaStream_t st)
{
    uint32_t W = 1, H = 1;
    if (m == TD_MAP_RB) rb_dims(N, W, H);
    const uint64_t blocks = (count + 255) / 256;
    const uint32_t g = static_cast<uint32_t>(blocks < uint64_t(sm_count()) * 16 ? blocks : uint64_t(sm_count()) * 16);
    k_map_dump<<<g, 256, 0, st>>>(int(m), N, W, u0, count, ij);
    return launch_status("td_map_dump kernel");
}

td_status launch_ltm_check(td_mapping m, uint64_t lam0, uint64_t count, uint64_t *result, cudaStream_t st)
{
    const uint64_t blocks = (count + 255) / 256;
    const uint32_t g = static_cast<uint32_t>(blocks < uint64_t(sm_count()) * 16 ? blocks : uint64_t(sm_count()) * 16);
    auto *res = reinterpret_cast<unsigned long long *>(result);
    switch (m) {
    case TD_MAP_LTM: k_ltm_check<LtmExact><<<g, 256, 0, st>>>(lam0, count, res); break;
    case TD_MAP_LTM_X: k_ltm_check<LtmSqrt><<<g, 256, 0, st>>>(lam0, count, res); break;
    case TD_MAP_LTM_N: k_ltm_check<LtmNewton><<<g, 256, 0, st>>>(lam0, count, res); break;
    case TD_MAP_LTM_N_FMA: k_ltm_check<LtmNewtonFma><<<g, 256, 0, st>>>(lam0, count, res); break;
    case TD_MAP_LTM_R: k_ltm_check<LtmRsqrtEps><<<g, 256, 0, st>>>(lam0, count, res); break;
    default: return fail(TD_ERR_UNSUPPORTED, "td_ltm_variant_check takes LTM, LTM_X, LTM_N, LTM_N_FMA or LTM_R");
    }
    return launch_status("td_ltm_check kernel");
}

}  // namespace td
