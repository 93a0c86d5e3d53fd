// td_edm_pair.cu -- the Euclidean distance map of Sec. IV of arXiv:1308.1419,
//     f(i, j) = sqrt(sum_k (a_i^k - a_j^k)^2),  0 <= j <= i < n,
// one element per thread, under each of the five launch spaces (td_strategies.cuh).  This is
// the paper's EDM kernel: each thread reads its two points straight from global memory (L1
// cached) and writes one float of the packed lower triangle.
//
// Summation order (shared by every EDM kernel in libtd, so all strategies, block sides and
// schedules give bit-identical results): t = x_i[k] - x_j[k] rounded to FP32, then
// s = fma(t, t, s) for k = 0, 1, ..., d-1 starting from s = 0, then sqrt rounded to nearest.
#include "td_strategies.cuh"
#include "td_dist.cuh"

namespace td {
namespace {

template <int D>  // D = 0: d given at run time
struct EdmPairBody {
    const float *x;
    uint32_t d;
    float *out;
    __device__ __forceinline__ void operator()(uint32_t i, uint32_t j) const
    {
        const uint32_t dd = D ? D : d;
        const float *a = x + uint64_t(i) * dd;
        const float *b = x + uint64_t(j) * dd;
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
        out[tri(i) + j] = dist_sqrt(s);
    }
};

}  // namespace

td_status launch_edm_pair(td_mapping m, td_schedule s, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                          float *out, const Plan &p, cudaStream_t st, uint64_t *ctas)
{
    switch (d) {
    case 1: return strat::launch_body(m, s, n, rho, EdmPairBody<1>{x, d, out}, p, st, ctas);
    case 2: return strat::launch_body(m, s, n, rho, EdmPairBody<2>{x, d, out}, p, st, ctas);
    case 3: return strat::launch_body(m, s, n, rho, EdmPairBody<3>{x, d, out}, p, st, ctas);
    case 4: return strat::launch_body(m, s, n, rho, EdmPairBody<4>{x, d, out}, p, st, ctas);
    default: return strat::launch_body(m, s, n, rho, EdmPairBody<0>{x, d, out}, p, st, ctas);
    }
}

}  // namespace td
