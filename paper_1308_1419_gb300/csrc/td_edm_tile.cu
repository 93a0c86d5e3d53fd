// td_edm_tile.cu -- td_edm for many features (rho = 64 or 128): the register-tiled block body
// of td_edm_tile.cuh issued by g(lambda), BB or REC (td_tiles.cuh), under the grid or the
// persistent schedule.
#include "td_edm_tile.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
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

template <class Tiles, int RHO, bool X2>
td_status launch_tiles(const Tiles &t, bool P, const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st,
                       uint64_t *ctas)
{
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

}  // namespace td
