// td_edm_tile.cu -- the Euclidean distance map of Sec. IV of arXiv:1308.1419 for many features:
// one CTA of 256 threads per rho x rho block (rho = 64 or 128) of the packed lower triangle,
// blocks issued by g(lambda), BB or REC (td_tiles.cuh).
//
// The block's rho row points and rho column points are staged in shared memory, KC features
// at a time, feature-major; each thread keeps a TM x TM register tile of partial sums
// (TM = rho / 16) for rows {tr + 16 a} and columns {tc + 16 b}, so that every feature step is
// two 128-bit shared loads and TM^2 subtract/FMA pairs.  The shared-memory slot of row r is
// (r mod 16) TM + floor(r / 16): the TM rows a thread owns sit side by side.  With X2, two
// columns are processed per instruction by the packed sub.rn.f32x2 / fma.rn.f32x2 of sm_100+,
// which round every lane exactly like the scalar instructions.
//
// Summation order is the one of every EDM kernel in libtd: t = x_i[k] - x_j[k], s = fma(t, t, s)
// for k = 0 .. d-1 from s = 0, then sqrtf.  Features past d are staged as zeros, and
// fma(0, 0, s) = s, so the result is bit-identical to the one-thread-per-element kernel.
#include "td_device.cuh"
#include "td_internal.h"
#include "td_tiles.cuh"

namespace td {
namespace {

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long sub_f32x2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

template <int RHO, int KC, bool X2>
struct EdmTile {
    static constexpr int TM = RHO / 16;
    static constexpr int LD = RHO + 4;  // padded row of a feature plane, keeps 16-byte alignment
    static constexpr int SMEM_FLOATS = 2 * KC * LD;
    static_assert(TM % 4 == 0, "TM must be a multiple of 4");

    __device__ static __forceinline__ int slot(int r) { return (r & 15) * TM + (r >> 4); }

    __device__ static void run(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0, uint32_t j0,
                               float *__restrict__ out, float *sm)
    {
        const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
        float *sA = sm, *sB = sm + KC * LD;
        const bool diag = i0 == j0;
        float acc[TM][TM];
        unsigned long long acc2[TM][TM / 2];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) acc[a][b] = 0.0f;
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM / 2; ++b) acc2[a][b] = 0ull;

        for (uint32_t k0 = 0; k0 < d; k0 += KC) {
            for (int e = tid; e < RHO * KC; e += 256) {
                const int r = e % RHO, kk = e / RHO;
                const uint32_t k = k0 + kk;
                const uint32_t i = i0 + r, j = j0 + r;
                sA[kk * LD + slot(r)] = (i < n && k < d) ? __ldg(x + uint64_t(i) * d + k) : 0.0f;
                if (!diag) sB[kk * LD + slot(r)] = (j < n && k < d) ? __ldg(x + uint64_t(j) * d + k) : 0.0f;
            }
            __syncthreads();
            const float *B = diag ? sA : sB;
#pragma unroll 2
            for (int kk = 0; kk < KC; ++kk) {
                float av[TM], bv[TM];
#pragma unroll
                for (int q = 0; q < TM; q += 4) {
                    const float4 va = *reinterpret_cast<const float4 *>(sA + kk * LD + tr * TM + q);
                    const float4 vb = *reinterpret_cast<const float4 *>(B + kk * LD + tc * TM + q);
                    av[q] = va.x; av[q + 1] = va.y; av[q + 2] = va.z; av[q + 3] = va.w;
                    bv[q] = vb.x; bv[q + 1] = vb.y; bv[q + 2] = vb.z; bv[q + 3] = vb.w;
                }
                if (X2) {
                    unsigned long long b2[TM / 2];
#pragma unroll
                    for (int q = 0; q < TM / 2; ++q) b2[q] = pack2(bv[2 * q], bv[2 * q + 1]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) {
                        const unsigned long long a2 = pack2(av[a], av[a]);
#pragma unroll
                        for (int q = 0; q < TM / 2; ++q) {
                            const unsigned long long t = sub_f32x2(a2, b2[q]);
                            acc2[a][q] = fma_f32x2(t, t, acc2[a][q]);
                        }
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < TM; ++a)
#pragma unroll
                        for (int b = 0; b < TM; ++b) {
                            const float t = av[a] - bv[b];
                            acc[a][b] = fmaf(t, t, acc[a][b]);
                        }
                }
            }
            __syncthreads();
        }
        if (X2) {
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int q = 0; q < TM / 2; ++q) unpack2(acc2[a][q], acc[a][2 * q], acc[a][2 * q + 1]);
        }
        // Thread (tr, tc) owns rows i0 + tr + 16a and columns j0 + tc + 16b; for fixed (a, b)
        // a warp writes two 64-byte runs of two packed rows.
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            const uint32_t i = i0 + tr + 16 * a;
            if (i >= n) continue;
            float *row = out + tri(i);
#pragma unroll
            for (int b = 0; b < TM; ++b) {
                const uint32_t j = j0 + tc + 16 * b;
                if (j <= i) row[j] = sqrtf(acc[a][b]);
            }
        }
    }
};

constexpr int KC = 16;

template <class Tiles, int RHO, bool X2, bool P>
__global__ void __launch_bounds__(256) k_edm_tiled(Tiles tiles, const float *__restrict__ x, uint32_t n, uint32_t d,
                                                   float *__restrict__ out)
{
    using Tile = EdmTile<RHO, KC, X2>;
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
    if (t.units == 0) return TD_OK;
    if (P) {
        auto k = k_edm_tiled<Tiles, RHO, X2, true>;
        const uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), 256, 0, t.units);
        k<<<dim3(static_cast<uint32_t>(g)), 256, 0, st>>>(t, x, n, d, out);
        *ctas += g;
    } else {
        k_edm_tiled<Tiles, RHO, X2, false><<<dim3(static_cast<uint32_t>(t.units)), 256, 0, st>>>(t, x, n, d, out);
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
        return launch_tiles<tiles::Ltm, RHO, X2>(tiles::Ltm{tri(p.nb)}, P, x, n, d, out, st, ctas);
    case TD_MAP_BB:
        return launch_tiles<tiles::Bb, RHO, X2>(tiles::Bb{uint64_t(p.nb) * p.nb, p.nb}, P, x, n, d, out, st, ctas);
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
