// td_strategies.cuh -- the five launch spaces compared in arXiv:1308.1419 (Sec. II-A g(lambda);
// Sec. III-B BB, UTM, RB, REC), as kernel templates over a per-element body.
//
// Every kernel uses rho x rho threads per block (UTM: rho^2 threads over its thread index).
// Every body call is guarded by 0 <= j <= i < N, so a mapping error can only show up as a
// missed or doubled element, never as a store outside the triangle.
// GRID schedule: one CTA per block of the strategy's launch space, as in the paper.
// PERSISTENT schedule: (SMs x resident CTAs) CTAs walk the same launch space with a
// grid-stride loop, so a wasted block costs one loop test instead of one CTA launch.
//
// A body is a functor `void operator()(uint32_t i, uint32_t j) const` run by the thread that
// the strategy maps to element (i, j).
#pragma once

#include "td_device.cuh"
#include "td_internal.h"

namespace td {
namespace strat {

// ---------------------------------------------------------------- LTM, Sec. II-A
// Block lambda in [0, T(n)) -> (block row, block column) = g(lambda); diagonal blocks filter
// their upper threads, edge blocks their threads beyond N.
// Map: the evaluation of g -- LtmExact, or one of the Sec. III-A variants (td_device.cuh).
template <int RHO, bool P, class Body, class Map = LtmExact>
__global__ void __launch_bounds__(RHO * RHO) k_ltm(uint32_t N, uint64_t units, Body body, Map map)
{
    const uint32_t ty = threadIdx.x / RHO, tx = threadIdx.x % RHO;
    const uint64_t stride = P ? gridDim.x : units;
    for (uint64_t lam = blockIdx.x; lam < units; lam += stride) {
        uint32_t bi, bj;
        map(lam, bi, bj);
        const uint32_t i = bi * RHO + ty, j = bj * RHO + tx;
        if (j <= i && i < N) body(i, j);
    }
}

// ---------------------------------------------------------------- BB, Sec. III-B
// n x n grid; a block with B_x > B_y returns before computing any thread coordinate.
template <int RHO, class Body>
__global__ void __launch_bounds__(RHO * RHO) k_bb_grid(uint32_t N, Body body)
{
    const uint32_t bx = blockIdx.x, by = blockIdx.y;
    if (bx > by) return;
    const uint32_t i = by * RHO + threadIdx.x / RHO, j = bx * RHO + threadIdx.x % RHO;
    if (j <= i && i < N) body(i, j);
}

template <int RHO, class Body>
__global__ void __launch_bounds__(RHO * RHO) k_bb_persist(uint32_t N, uint32_t nb, Body body)
{
    const uint32_t ty = threadIdx.x / RHO, tx = threadIdx.x % RHO;
    const uint32_t units = nb * nb;
    for (uint32_t u = blockIdx.x; u < units; u += gridDim.x) {
        const uint32_t by = u / nb, bx = u - by * nb;
        if (bx > by) continue;
        const uint32_t i = by * RHO + ty, j = bx * RHO + tx;
        if (j <= i && i < N) body(i, j);
    }
}

// ---------------------------------------------------------------- UTM, Sec. III-B
// Thread-level: thread index k = block * rho^2 + threadIdx < T(N).
template <int RHO, bool P, class Body>
__global__ void __launch_bounds__(RHO * RHO) k_utm(uint32_t N, uint64_t total, uint64_t nblk, Body body)
{
    const uint64_t stride = P ? gridDim.x : nblk;
    for (uint64_t b = blockIdx.x; b < nblk; b += stride) {
        const uint64_t k = b * (RHO * RHO) + threadIdx.x;
        if (k < total) {
            uint32_t i, j;
            utm_map(k, N, i, j);
            if (j <= i && i < N) body(i, j);
        }
    }
}

// ---------------------------------------------------------------- RB, Sec. III-B
template <int RHO, class Body>
__global__ void __launch_bounds__(RHO * RHO) k_rb_grid(uint32_t N, uint32_t W, uint32_t H, Body body)
{
    const uint32_t x = blockIdx.x * RHO + threadIdx.x % RHO;
    const uint32_t y = blockIdx.y * RHO + threadIdx.x / RHO;
    if (x < W && y < H) {
        uint32_t i, j;
        rb_map(N, x, y, i, j);
        if (j <= i && i < N) body(i, j);
    }
}

template <int RHO, class Body>
__global__ void __launch_bounds__(RHO * RHO)
    k_rb_persist(uint32_t N, uint32_t W, uint32_t H, uint32_t gx, uint64_t units, Body body)
{
    const uint32_t ty = threadIdx.x / RHO, tx = threadIdx.x % RHO;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const uint32_t by = static_cast<uint32_t>(u / gx), bx = static_cast<uint32_t>(u - uint64_t(by) * gx);
        const uint32_t x = bx * RHO + tx, y = by * RHO + ty;
        if (x < W && y < H) {
            uint32_t i, j;
            rb_map(N, x, y, i, j);
            if (j <= i && i < N) body(i, j);
        }
    }
}

// ---------------------------------------------------------------- REC, Sec. III-B
// Level l (one launch): 2^(l-1) squares of side s = N / 2^l laid side by side along x;
// square q covers rows [(2q+1)s, (2q+2)s) and columns [2qs, (2q+1)s).  gx = N/(2 rho)
// blocks along x, s/rho along y.
template <int RHO, bool P, class Body>
__global__ void __launch_bounds__(RHO * RHO)
    k_rec_level(uint32_t N, uint32_t s, uint32_t sb, uint32_t gx, uint64_t units, Body body)
{
    const uint32_t ty = threadIdx.x / RHO, tx = threadIdx.x % RHO;
    const uint64_t stride = P ? gridDim.x : units;
    for (uint64_t u = P ? blockIdx.x : 0; u < units; u += stride) {
        uint32_t bx, by;
        if (P) { by = static_cast<uint32_t>(u / gx); bx = static_cast<uint32_t>(u - uint64_t(by) * gx); }
        else   { bx = blockIdx.x; by = blockIdx.y; }
        const uint32_t q = bx / sb, cb = bx - q * sb;
        const uint32_t i = (2 * q + 1) * s + by * RHO + ty;
        const uint32_t j = 2 * q * s + cb * RHO + tx;
        if (j <= i && i < N) body(i, j);
    }
}

// Final pass: 2^k diagonal triangles of side m, each covered bounding-box style.
template <int RHO, bool P, class Body>
__global__ void __launch_bounds__(RHO * RHO)
    k_rec_diag(uint32_t N, uint32_t m, uint32_t mb, uint32_t gx, uint64_t units, Body body)
{
    const uint32_t ty = threadIdx.x / RHO, tx = threadIdx.x % RHO;
    const uint64_t stride = P ? gridDim.x : units;
    for (uint64_t u = P ? blockIdx.x : 0; u < units; u += stride) {
        uint32_t bx, by;
        if (P) { by = static_cast<uint32_t>(u / gx); bx = static_cast<uint32_t>(u - uint64_t(by) * gx); }
        else   { bx = blockIdx.x; by = blockIdx.y; }
        const uint32_t t = bx / mb, lb = bx - t * mb;
        if (lb > by) continue;
        const uint32_t i = t * m + by * RHO + ty, j = t * m + lb * RHO + tx;
        if (j <= i && i < N) body(i, j);
    }
}

// ---------------------------------------------------------------- launchers

template <class K>
uint64_t grid_for(K kernel, bool P, int threads, uint64_t units)
{
    return P ? persistent_ctas(reinterpret_cast<const void *>(kernel), threads, 0, units) : units;
}

// Blocks lambda < T(nb) mapped by `map` (g(lambda), one of its FP32 variants, or block-level UTM).
template <int RHO, class Body, class Map>
void launch_ltm(bool P, uint32_t N, Body body, const Plan &p, cudaStream_t st, uint64_t *ctas, Map map = Map{})
{
    constexpr int threads = RHO * RHO;
    const uint64_t units = tri(p.nb);
    if (P) {
        auto k = k_ltm<RHO, true, Body, Map>;
        const uint64_t g = grid_for(k, true, threads, units);
        k<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, units, body, map);
        *ctas += g;
    } else {
        k_ltm<RHO, false, Body, Map><<<dim3(static_cast<uint32_t>(units)), threads, 0, st>>>(N, units, body, map);
        *ctas += units;
    }
}

template <int RHO, class Body>
td_status launch_rho(td_mapping m, bool P, uint32_t N, Body body, const Plan &p, cudaStream_t st,
                     uint64_t *ctas)
{
    constexpr int threads = RHO * RHO;
    switch (m) {
    case TD_MAP_LTM:
        launch_ltm<RHO, Body, LtmExact>(P, N, body, p, st, ctas);
        break;
    case TD_MAP_UTM_BLOCK:
        launch_ltm<RHO, Body, UtmBlock>(P, N, body, p, st, ctas, UtmBlock{p.nb});
        break;
    case TD_MAP_BB: {
        if (P) {
            auto k = k_bb_persist<RHO, Body>;
            const uint64_t g = grid_for(k, true, threads, uint64_t(p.nb) * p.nb);
            k<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, p.nb, body);
            *ctas += g;
        } else {
            k_bb_grid<RHO, Body><<<dim3(p.nb, p.nb), threads, 0, st>>>(N, body);
            *ctas += uint64_t(p.nb) * p.nb;
        }
        break;
    }
    case TD_MAP_UTM: {
        const uint64_t total = tri(N), nblk = (total + threads - 1) / threads;
        if (P) {
            auto k = k_utm<RHO, true, Body>;
            const uint64_t g = grid_for(k, true, threads, nblk);
            k<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, total, nblk, body);
            *ctas += g;
        } else {
            k_utm<RHO, false, Body><<<dim3(static_cast<uint32_t>(nblk)), threads, 0, st>>>(N, total, nblk, body);
            *ctas += nblk;
        }
        break;
    }
    case TD_MAP_RB: {
        uint32_t W, H;
        rb_dims(N, W, H);
        const uint32_t gx = (W + RHO - 1) / RHO, gy = (H + RHO - 1) / RHO;
        if (P) {
            auto k = k_rb_persist<RHO, Body>;
            const uint64_t units = uint64_t(gx) * gy;
            const uint64_t g = grid_for(k, true, threads, units);
            k<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, W, H, gx, units, body);
            *ctas += g;
        } else {
            k_rb_grid<RHO, Body><<<dim3(gx, gy), threads, 0, st>>>(N, W, H, body);
            *ctas += uint64_t(gx) * gy;
        }
        break;
    }
    case TD_MAP_REC: {
        const uint32_t k = p.rec_k, mside = p.rec_m;
        for (uint32_t l = 1; l <= k; ++l) {
            const uint32_t s = N >> l, sb = s / RHO, gx = N / (2 * RHO);
            const uint64_t units = uint64_t(gx) * sb;
            if (P) {
                auto kk = k_rec_level<RHO, true, Body>;
                const uint64_t g = grid_for(kk, true, threads, units);
                kk<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, s, sb, gx, units, body);
                *ctas += g;
            } else {
                k_rec_level<RHO, false, Body><<<dim3(gx, sb), threads, 0, st>>>(N, s, sb, gx, 1, body);
                *ctas += units;
            }
        }
        const uint32_t mb = mside / RHO, gx = N / RHO;
        const uint64_t units = uint64_t(gx) * mb;
        if (P) {
            auto kk = k_rec_diag<RHO, true, Body>;
            const uint64_t g = grid_for(kk, true, threads, units);
            kk<<<dim3(static_cast<uint32_t>(g)), threads, 0, st>>>(N, mside, mb, gx, units, body);
            *ctas += g;
        } else {
            k_rec_diag<RHO, false, Body><<<dim3(gx, mb), threads, 0, st>>>(N, mside, mb, gx, 1, body);
            *ctas += units;
        }
        break;
    }
    default:
        return fail(TD_ERR_INVALID_ARG, "unknown mapping %d", int(m));
    }
    return launch_status("td probe/cover kernel");
}

template <class Body>
td_status launch_body(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, Body body, const Plan &p,
                      cudaStream_t st, uint64_t *ctas)
{
    const bool P = s == TD_SCHED_PERSISTENT;
    switch (rho) {
    case 8: return launch_rho<8>(m, P, N, body, p, st, ctas);
    case 16: return launch_rho<16>(m, P, N, body, p, st, ctas);
    case 32: return launch_rho<32>(m, P, N, body, p, st, ctas);
    default: return fail(TD_ERR_INVALID_ARG, "rho must be 8, 16 or 32 (got %u)", rho);
    }
}

}  // namespace strat
}  // namespace td
