// td_strict.cu -- td-problems without the diagonal (Eq. (theorem_nodiag) of arXiv:1308.1419):
// the strict lower triangle i > j of side n, n(n-1)/2 elements, packed row-major at
// k = i(i-1)/2 + j, mapped at the element level -- each thread takes packed indices k and finds
// its (i, j) with the strict g (ltm_g_strict), so consecutive threads own consecutive outputs.
//
//   k_edm_strict     distance map: a thread computes 4 consecutive k (one strict-g evaluation,
//                    then a row walk) and writes them with one 16-byte store.
//   k_collide_strict collision bits: bit k of a uint32 array (word k / 32, LSB first) is
//                    c(i, j); a warp takes one word, lane l the pair k = 32 w + l, and the
//                    word is a __ballot_sync of the 32 exact predicates.
//
// The EDM sums in the order of every EDM kernel of libtd (t = x_i[k] - x_j[k], s = fma(t, t, s)
// for k = 0 .. d-1 from s = 0, then sqrtf), so out[k] equals the with-diagonal map at (i, j) bit
// for bit.
#include "td_collide.cuh"
#include "td_internal.h"
#include "td_dist.cuh"

namespace td {
namespace {

template <int D>
__device__ __forceinline__ float distance(const float *__restrict__ x, uint32_t d, uint32_t i, uint32_t j)
{
    const uint32_t dd = D ? D : d;
    const float *a = x + uint64_t(i) * dd, *b = x + uint64_t(j) * dd;
    float s = 0.0f;
    if (D) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float t = __ldg(a + k) - __ldg(b + k);
            s = fmaf(t, t, s);
        }
    } else {
        for (uint32_t k = 0; k < dd; ++k) {
            const float t = __ldg(a + k) - __ldg(b + k);
            s = fmaf(t, t, s);
        }
    }
    return dist_sqrt(s);
}

template <int D>
__global__ void __launch_bounds__(256) k_edm_strict(const float *__restrict__ x, uint32_t d, uint64_t total,
                                                    float *__restrict__ out)
{
    const uint64_t chunks = (total + 3) / 4, stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < chunks; c += stride) {
        const uint64_t k0 = 4 * c;
        uint32_t i, j;
        ltm_g_strict(k0, i, j);
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = k0 + q < total ? distance<D>(x, d, i, j) : 0.0f;
            if (++j == i) {  // next strict row
                ++i;
                j = 0;
            }
        }
        if (k0 + 4 <= total) {
            __stcs(reinterpret_cast<float4 *>(out + k0), make_float4(v[0], v[1], v[2], v[3]));
        } else {
            for (int q = 0; k0 + q < total; ++q) out[k0 + q] = v[q];
        }
    }
}

__global__ void __launch_bounds__(256) k_collide_strict(const int32_t *__restrict__ c, const int32_t *__restrict__ r,
                                                        uint64_t total, uint32_t *__restrict__ bits)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t words = (total + 31) / 32, stride = uint64_t(gridDim.x) * (blockDim.x >> 5);
    for (uint64_t w = uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); w < words; w += stride) {
        const uint64_t k = 32 * w + lane;
        bool hit = false;
        if (k < total) {
            uint32_t i, j;
            ltm_g_strict(k, i, j);
            const int4 p = make_int4(__ldg(c + 3 * uint64_t(i)), __ldg(c + 3 * uint64_t(i) + 1),
                                     __ldg(c + 3 * uint64_t(i) + 2), __ldg(r + i));
            const int4 q = make_int4(__ldg(c + 3 * uint64_t(j)), __ldg(c + 3 * uint64_t(j) + 1),
                                     __ldg(c + 3 * uint64_t(j) + 2), __ldg(r + j));
            hit = collide_exact(p, q);
        }
        const uint32_t word = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) bits[w] = word;
    }
}

uint64_t grid_for_units(const void *kernel, uint64_t units_per_cta_work)
{
    return persistent_ctas(kernel, 256, 0, units_per_cta_work);
}

}  // namespace

td_status launch_edm_strict(const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st)
{
    const uint64_t total = uint64_t(n) * (n - 1) / 2;
    if (total == 0) return TD_OK;
    const uint64_t chunks = (total + 3) / 4, ctas = (chunks + 255) / 256;
    switch (d) {
#define TD_STRICT_CASE(DD)                                                                                      \
    case DD: {                                                                                                  \
        auto k = k_edm_strict<DD>;                                                                              \
        k<<<dim3(static_cast<uint32_t>(grid_for_units(reinterpret_cast<const void *>(k), ctas))), 256, 0, st>>>( \
            x, d, total, out);                                                                                  \
        break;                                                                                                  \
    }
        TD_STRICT_CASE(1)
        TD_STRICT_CASE(2)
        TD_STRICT_CASE(3)
        TD_STRICT_CASE(4)
#undef TD_STRICT_CASE
    default: {
        auto k = k_edm_strict<0>;
        k<<<dim3(static_cast<uint32_t>(grid_for_units(reinterpret_cast<const void *>(k), ctas))), 256, 0, st>>>(
            x, d, total, out);
    }
    }
    return launch_status("td_edm_strict kernel");
}

td_status launch_collide_strict(const int32_t *c, const int32_t *r, uint32_t n, uint32_t *bits, cudaStream_t st)
{
    const uint64_t total = uint64_t(n) * (n - 1) / 2;
    if (total == 0) return TD_OK;
    const uint64_t words = (total + 31) / 32, ctas = (words + 7) / 8;
    const uint64_t g = grid_for_units(reinterpret_cast<const void *>(k_collide_strict), ctas);
    k_collide_strict<<<dim3(static_cast<uint32_t>(g)), 256, 0, st>>>(c, r, total, bits);
    return launch_status("td_collide_strict kernel");
}

}  // namespace td
