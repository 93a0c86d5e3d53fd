// td_edm_tile.cu -- td_edm for many features (rho = 64 or 128): the register-tiled block body
// of td_edm_tile.cuh issued by g(lambda), BB or REC (td_tiles.cuh), under the grid or the
// persistent schedule.
#include "td_edm_tile.cuh"
#include "td_internal.h"
#include "td_sm100.cuh"
#include "td_tiles.cuh"

namespace td {

// Bounded waits of the TMA-staged body that ran out since the last td_wait_status with clear.
__device__ unsigned int g_wait_error;

namespace {

template <class Tiles, int RHO, bool X2, bool P>
__global__ void __launch_bounds__(edm_tile_threads(RHO), edm_tile_min_ctas(RHO))
    k_edm_tiled(Tiles tiles, const float *__restrict__ x, uint32_t n, uint32_t d, float *__restrict__ out)
{
    using Tile = typename EdmTileFor<RHO, X2>::type;
    __shared__ __align__(16) float sm[Tile::SMEM_FLOATS];
    const uint64_t stride = P ? gridDim.x : tiles.units;
    for (uint64_t u = blockIdx.x; u < tiles.units; u += stride) {
        uint32_t bi, bj;
        if (!tiles(u, bi, bj)) continue;
        Tile::run(x, n, d, bi * RHO, bj * RHO, out, sm);
    }
}

// TMA-staged form of the point-major body (d % 4 == 0, 16-byte aligned points), for many features.
// Per 16-feature chunk, one thread loads the block's row and column points as two boxes of
// RHO points x 64 bytes (cp.async.bulk.tensor; zero fill past n and d) into one stage of a
// two-stage ring, completing on that stage's mbarrier; the next chunk's boxes are issued before
// the current one is read.  The boxes use the 64-byte swizzle: granule g (features 4g .. 4g + 3)
// of point row r lands at granule g ^ ((r >> 1) & 3) of its 64-byte row, so the column threads of
// a warp (rows tc, tc + CT, ...) read 16 different rows without bank conflicts.  The sums are
// those of run_pm: each accumulator takes the features in order, so the output is bit-identical
// to the cp.async staging.  Every wait is bounded; one that runs out sets g_wait_error, the CTA
// waits (bounded) for the copies it issued and stops.
constexpr int kTmaFeatures = 16;

__device__ __forceinline__ float4 box_f4(const float *box, int r, int g)
{
    return *reinterpret_cast<const float4 *>(box + r * kTmaFeatures + ((g ^ ((r >> 1) & 3)) << 2));
}

template <class Tiles, int RHO>
__global__ void __launch_bounds__(edm_tile_threads(RHO), edm_tile_min_ctas(RHO))
    k_edm_tiled_tma(Tiles tiles, const __grid_constant__ CUtensorMap tmap, uint32_t n, uint32_t d,
                    float *__restrict__ out)
{
    using namespace sm100;
    using Tile = typename EdmTileFor<RHO, false>::type;
    constexpr int TM = edm_tile_tm(RHO), TN = edm_tile_tn(RHO), RT = RHO / TM, CT = RHO / TN;
    constexpr uint32_t BOXB = RHO * kTmaFeatures * 4;  // bytes of one box
    __shared__ __align__(1024) float sbox[2][2][RHO * kTmaFeatures];  // stage, rows / columns
    __shared__ __align__(8) uint64_t full[2];
    const int tid = threadIdx.x, tr = tid / CT, tc = tid % CT;
    const uint32_t bar0 = smem_u32(&full[0]);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t nch = (d + kTmaFeatures - 1) / kTmaFeatures;
    uint64_t g = 0;  // chunks this CTA has started: stage g & 1, that stage's use g >> 1
    for (uint64_t u = blockIdx.x; u < tiles.units; u += gridDim.x) {
        uint32_t bi, bj;
        if (!tiles(u, bi, bj)) continue;
        const uint32_t i0 = bi * RHO, j0 = bj * RHO;
        const bool diag = i0 == j0;
        auto issue = [&](uint32_t c, uint64_t gg) {  // thread 0: chunk c into stage gg & 1
            const uint32_t st = uint32_t(gg & 1), bar = bar0 + 8 * st;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, diag ? BOXB : 2 * BOXB);
            tma_load_2d(smem_u32(sbox[st][0]), &tmap, int32_t(c * kTmaFeatures), int32_t(i0), bar);
            if (!diag) tma_load_2d(smem_u32(sbox[st][1]), &tmap, int32_t(c * kTmaFeatures), int32_t(j0), bar);
        };
        float acc[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = 0.0f;
        if (tid == 0) issue(0, g);
        for (uint32_t c = 0; c < nch; ++c, ++g) {
            const bool next = c + 1 < nch;
            if (tid == 0 && next) issue(c + 1, g + 1);  // its stage was last read two chunks ago
            const uint32_t st = uint32_t(g & 1);
            const bool got = mbar_wait(bar0 + 8 * st, uint32_t(g >> 1) & 1u);
            if (__syncthreads_or(!got)) {  // a wait ran out: record it, let the copies land, stop
                if (tid == 0) {
                    atomicOr(&g_wait_error, 1u);
                    mbar_wait(bar0 + 8 * st, uint32_t(g >> 1) & 1u);
                    if (next) mbar_wait(bar0 + 8 * (st ^ 1u), uint32_t((g + 1) >> 1) & 1u);
                }
                return;
            }
            const float *A = sbox[st][0], *B = diag ? A : sbox[st][1];
            const int kc = d - c * kTmaFeatures < uint32_t(kTmaFeatures) ? int(d - c * kTmaFeatures) : kTmaFeatures;
            for (int g4 = 0; g4 < kc / 4; ++g4) {
                float4 av[TM];
#pragma unroll
                for (int a = 0; a < TM; ++a) av[a] = box_f4(A, tr + RT * a, g4);
#pragma unroll
                for (int b = 0; b < TN; ++b) {
                    const float4 bv = box_f4(B, tc + CT * b, g4);
                    float t[TM];  // one feature's differences for the TM rows first, then their FMAs
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].x - bv.x;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].y - bv.y;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].z - bv.z;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].w - bv.w;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
                }
            }
            __syncthreads();  // this stage is refilled two chunks from now
        }
        Tile::store(n, i0, j0, out, acc);
    }
}

template <class Tiles, int RHO>
td_status launch_tiles_tma(const Tiles &t, bool P, const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st,
                           uint64_t *ctas)
{
    constexpr int NT = edm_tile_threads(RHO);
    if (t.units == 0) return TD_OK;
    CUtensorMap tmap;
    const td_status s = encode_tiled_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, x, d, n, uint64_t(d) * 4, kTmaFeatures,
                                        RHO, CU_TENSOR_MAP_SWIZZLE_64B);
    if (s != TD_OK) return s;
    auto k = k_edm_tiled_tma<Tiles, RHO>;
    const uint64_t g = P ? persistent_ctas(reinterpret_cast<const void *>(k), NT, 0, t.units) : t.units;
    k<<<dim3(static_cast<uint32_t>(g)), NT, 0, st>>>(t, tmap, n, d, out);
    *ctas += g;
    return launch_status("td_edm tiled kernel (TMA staging)");
}

template <class Tiles, int RHO, bool X2>
td_status launch_tiles(const Tiles &t, bool P, const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st,
                       uint64_t *ctas)
{
    const int tma = option(TD_OPT_EDM_TMA);  // 0: for d >= 64, 1: always, 2: never
    if (!X2 && d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0 && (tma == 1 || (tma == 0 && d >= 64)))
        return launch_tiles_tma<Tiles, RHO>(t, P, x, n, d, out, st, ctas);
    constexpr int NT = EdmTileFor<RHO, X2>::type::NT;
    if (t.units == 0) return TD_OK;
    if (P) {
        auto k = k_edm_tiled<Tiles, RHO, X2, true>;
        const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), NT, 0, t.units);
        k<<<dim3(static_cast<uint32_t>(g)), NT, 0, st>>>(t, x, n, d, out);
        *ctas += g;
    } else {
        k_edm_tiled<Tiles, RHO, X2, false><<<dim3(static_cast<uint32_t>(t.units)), NT, 0, st>>>(t, x, n, d, out);
        *ctas += t.units;
    }
    return launch_status("td_edm tiled kernel");
}

template <int RHO, bool X2>
td_status launch_rho(td_mapping m, bool P, const float *x, uint32_t n, uint32_t d, float *out, const Plan &p,
                     cudaStream_t st, uint64_t *ctas)
{
    switch (m) {
    case TD_MAP_LTM:
        return launch_tiles<tiles::Ltm, RHO, X2>(tiles::ltm_source(p), P, x, n, d, out, st, ctas);
    case TD_MAP_UTM_BLOCK:
        return launch_tiles<tiles::UtmBlk, RHO, X2>(tiles::UtmBlk{tri(p.nb), p.nb}, P, x, n, d, out, st, ctas);
    case TD_MAP_BB:
        return launch_tiles<tiles::Bb, RHO, X2>(tiles::bb_source(p), P, x, n, d, out, st, ctas);
    case TD_MAP_REC: {
        for (uint32_t l = 1; l <= p.rec_k; ++l) {
            const uint32_t sb = (n >> l) / RHO, gx = n / (2 * RHO);
            const td_status s = launch_tiles<tiles::RecLevel, RHO, X2>(tiles::RecLevel{uint64_t(gx) * sb, sb, gx}, P, x,
                                                                       n, d, out, st, ctas);
            if (s != TD_OK) return s;
        }
        const uint32_t mb = p.rec_m / RHO, gx = n / RHO;
        return launch_tiles<tiles::RecDiag, RHO, X2>(tiles::RecDiag{uint64_t(gx) * mb, mb, gx}, P, x, n, d, out, st,
                                                     ctas);
    }
    default:
        return fail(TD_ERR_UNSUPPORTED, "tiled EDM (rho 64/128) supports LTM, BB and REC");
    }
}

}  // namespace

td_status launch_edm_tiled(td_mapping m, td_schedule s, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                           float *out, const Plan &p, bool x2, cudaStream_t st, uint64_t *ctas)
{
    const bool P = s == TD_SCHED_PERSISTENT;
    if (rho == 64) return x2 ? launch_rho<64, true>(m, P, x, n, d, out, p, st, ctas)
                             : launch_rho<64, false>(m, P, x, n, d, out, p, st, ctas);
    if (rho == 128) return x2 ? launch_rho<128, true>(m, P, x, n, d, out, p, st, ctas)
                              : launch_rho<128, false>(m, P, x, n, d, out, p, st, ctas);
    return fail(TD_ERR_INVALID_ARG, "tiled EDM needs rho 64 or 128");
}

td_status read_wait_status(bool clear, uint32_t *code, cudaStream_t st)
{
    uint32_t h = 0;
    td_status s = cuda_status(cudaMemcpyFromSymbolAsync(&h, g_wait_error, 4, 0, cudaMemcpyDeviceToHost, st),
                              "td_wait_status read");
    if (s == TD_OK && clear) {
        static const uint32_t zero = 0;
        s = cuda_status(cudaMemcpyToSymbolAsync(g_wait_error, &zero, 4, 0, cudaMemcpyHostToDevice, st),
                        "td_wait_status clear");
    }
    if (s == TD_OK) s = cuda_status(cudaStreamSynchronize(st), "td_wait_status sync");
    *code = h;
    return s;
}

}  // namespace td
