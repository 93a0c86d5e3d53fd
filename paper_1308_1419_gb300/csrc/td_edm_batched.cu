// td_edm_batched.cu -- many independent distance maps (Sec. IV of arXiv:1308.1419) of uneven
// sizes in one persistent launch.
//
// The problems' block triangles are concatenated into one launch space: problem p owns the
// global block indices [P[p], P[p] + T(nb_p)) with P the exclusive prefix sum of T(nb_q),
// nb_q = ceil(n_q / rho).  A CTA takes a global index u, finds its problem by an upper-bound
// binary search over P (staged in shared memory), and maps the local index u - P[p] to a block
// with g(lambda) (Sec. II-A); the block body is the register-tiled one of td_edm_tile.cuh, so
// every problem's output is bit-identical to a td_edm call on that problem alone.  Problems
// are laid into the launch space heaviest first (by T(nb) * d), so the grid-stride walk meets
// the expensive blocks early and the tail is made of light ones.
//
// The plan (prefix sums and per-problem offsets) lives in a caller-provided workspace; the run
// step is a single kernel launch, so it can be captured in a CUDA graph.
#include <algorithm>
#include <numeric>
#include <vector>

#include "td_edm_tile.cuh"
#include "td_internal.h"

namespace td {

size_t batched_workspace_bytes(uint32_t nprob)
{
    return sizeof(BatchHeader) + (size_t(nprob) + 1) * sizeof(uint64_t) + size_t(nprob) * sizeof(BatchMeta);
}

uint64_t batched_weight(uint32_t n, uint32_t d, uint32_t rho) { return tri((n + rho - 1) / rho) * d; }

uint64_t batched_fill_image(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho, const uint32_t *order,
                            uint64_t *x_off, uint64_t *out_off, unsigned char *img)
{
    uint64_t xacc = 0, oacc = 0;
    for (uint32_t q = 0; q < nprob; ++q) {  // offsets in input (concatenation) order
        x_off[q] = xacc;
        out_off[q] = oacc;
        xacc += uint64_t(n[q]) * d[q];
        oacc += tri(n[q]);
    }
    auto *hdr = reinterpret_cast<BatchHeader *>(img);
    auto *prefix = reinterpret_cast<uint64_t *>(img + sizeof(BatchHeader));
    auto *meta = reinterpret_cast<BatchMeta *>(img + sizeof(BatchHeader) + (size_t(nprob) + 1) * sizeof(uint64_t));
    uint64_t acc = 0;
    for (uint32_t s = 0; s < nprob; ++s) {
        const uint32_t q = order[s];
        prefix[s] = acc;
        acc += tri((n[q] + rho - 1) / rho);
        meta[s] = BatchMeta{x_off[q], out_off[q], n[q], d[q], 0, 0};
    }
    prefix[nprob] = acc;
    hdr->magic = kBatchMagic;
    hdr->total_blocks = acc;
    hdr->nprob = nprob;
    hdr->rho = rho;
    return acc;
}

namespace {

constexpr int kSmemPrefix = 1024;  // prefix entries staged in shared memory (larger batches search global)

template <int RHO, bool X2>
__global__ void __launch_bounds__(edm_tile_threads(RHO), edm_tile_min_ctas(RHO))
    k_edm_batched(const uint64_t *__restrict__ prefix, const BatchMeta *__restrict__ meta, uint32_t nprob,
                  uint64_t total, const float *__restrict__ x, float *__restrict__ out)
{
    using Tile = typename EdmTileFor<RHO, X2>::type;
    __shared__ __align__(16) float sm[Tile::SMEM_FLOATS];
    __shared__ uint64_t sp[kSmemPrefix + 1];
    const bool staged = nprob <= kSmemPrefix;
    if (staged)
        for (uint32_t q = threadIdx.x; q <= nprob; q += blockDim.x) sp[q] = prefix[q];
    __syncthreads();
    const uint64_t *P = staged ? sp : prefix;
    for (uint64_t u = blockIdx.x; u < total; u += gridDim.x) {
        // largest p with P[p] <= u (P[0] = 0 <= u < P[nprob] = total)
        uint32_t lo = 0, hi = nprob;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (P[mid] <= u) lo = mid;
            else hi = mid;
        }
        const BatchMeta m = meta[lo];
        uint32_t bi, bj;
        ltm_g(u - P[lo], bi, bj);
        Tile::template run<true>(x + m.x_off, m.n, m.d, bi * RHO, bj * RHO, out + m.out_off, sm);
    }
}

template <int RHO, bool X2>
td_status launch_rho(const uint64_t *prefix, const BatchMeta *meta, uint32_t nprob, uint64_t total, const float *x,
                     float *out, uint32_t ctas_per_sm, cudaStream_t st, uint64_t *ctas)
{
    constexpr int NT = EdmTileFor<RHO, X2>::type::NT;
    auto k = k_edm_batched<RHO, X2>;
    uint64_t g = persistent_ctas(reinterpret_cast<const void *>(k), NT, 0, total);
    if (ctas_per_sm > 0) {
        const uint64_t want = uint64_t(ctas_per_sm) * sm_count();
        g = std::min<uint64_t>(std::min(g, want), total);
        if (g == 0) g = 1;
    }
    k<<<dim3(static_cast<uint32_t>(g)), NT, 0, st>>>(prefix, meta, nprob, total, x, out);
    if (ctas) *ctas = g;
    return launch_status("td_edm_batched kernel");
}

}  // namespace

td_status batched_plan(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho, void *ws, size_t ws_bytes,
                       cudaStream_t st, std::vector<unsigned char> &host, uint64_t *total_out)
{
    if (rho != 64 && rho != 128) return fail(TD_ERR_INVALID_ARG, "batched rho must be 64 or 128 (got %u)", rho);
    if (ws_bytes < batched_workspace_bytes(nprob)) return fail(TD_ERR_INVALID_ARG, "workspace too small");
    std::vector<uint64_t> xo(nprob), oo(nprob), weight(nprob);
    for (uint32_t q = 0; q < nprob; ++q) {
        if (n[q] == 0 || d[q] == 0) return fail(TD_ERR_INVALID_ARG, "problem %u has n = 0 or d = 0", q);
        weight[q] = batched_weight(n[q], d[q], rho);
    }
    std::vector<uint32_t> order(nprob);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return weight[a] > weight[b]; });
    host.assign(batched_workspace_bytes(nprob), 0);
    const uint64_t acc = batched_fill_image(nprob, n, d, rho, order.data(), xo.data(), oo.data(), host.data());
    *total_out = acc;
    return cuda_status(cudaMemcpyAsync(ws, host.data(), host.size(), cudaMemcpyHostToDevice, st),
                       "td_edm_batched_plan upload");
}

td_status batched_run(uint32_t nprob, uint32_t rho, uint64_t total, const float *x, float *out, const void *ws,
                      uint32_t ctas_per_sm, bool x2, cudaStream_t st, uint64_t *ctas)
{
    if (total == 0) return TD_OK;
    const auto *base = static_cast<const unsigned char *>(ws);
    const auto *prefix = reinterpret_cast<const uint64_t *>(base + sizeof(BatchHeader));
    const auto *meta = reinterpret_cast<const BatchMeta *>(base + sizeof(BatchHeader) + (size_t(nprob) + 1) * 8);
    if (rho == 64)
        return x2 ? launch_rho<64, true>(prefix, meta, nprob, total, x, out, ctas_per_sm, st, ctas)
                  : launch_rho<64, false>(prefix, meta, nprob, total, x, out, ctas_per_sm, st, ctas);
    return x2 ? launch_rho<128, true>(prefix, meta, nprob, total, x, out, ctas_per_sm, st, ctas)
              : launch_rho<128, false>(prefix, meta, nprob, total, x, out, ctas_per_sm, st, ctas);
}

}  // namespace td

using namespace td;

static bool batched_args_ok(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x, float *out,
                            const void *ws)
{
    if (nprob == 0) return true;
    if (!n || !d) return fail(TD_ERR_INVALID_ARG, "n and d (host arrays) must be non-NULL"), false;
    if (!x || !out || !ws) return fail(TD_ERR_INVALID_ARG, "x_cat, out_cat and workspace must be non-NULL"), false;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(ws)) & 15u)
        return fail(TD_ERR_INVALID_ARG, "x_cat, out_cat and workspace must be 16-byte aligned"), false;
    return true;
}

extern "C" {

size_t td_edm_batched_workspace(uint32_t nprob) { return batched_workspace_bytes(nprob); }

td_status td_edm_batched_plan(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho, void *ws,
                              size_t ws_bytes, uint64_t *total_blocks, void *stream)
{
    fail(TD_OK, "");
    if (!total_blocks) return fail(TD_ERR_INVALID_ARG, "total_blocks is NULL");
    *total_blocks = 0;
    if (nprob == 0) return TD_OK;
    if (!n || !d || !ws) return fail(TD_ERR_INVALID_ARG, "n, d and workspace must be non-NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 15u) return fail(TD_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    std::vector<unsigned char> host;
    return batched_plan(nprob, n, d, rho, ws, ws_bytes, static_cast<cudaStream_t>(stream), host, total_blocks);
}

td_status td_edm_batched_run(uint32_t nprob, uint32_t rho, uint64_t total_blocks, const float *x_cat, float *out_cat,
                             const void *ws, uint32_t ctas_per_sm, void *stream)
{
    fail(TD_OK, "");
    if (nprob == 0 || total_blocks == 0) return TD_OK;
    if (rho != 64 && rho != 128) return fail(TD_ERR_INVALID_ARG, "batched rho must be 64 or 128 (got %u)", rho);
    if (!x_cat || !out_cat || !ws) return fail(TD_ERR_INVALID_ARG, "x_cat, out_cat and workspace must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(x_cat) | reinterpret_cast<uintptr_t>(out_cat) | reinterpret_cast<uintptr_t>(ws)) & 15u)
        return fail(TD_ERR_INVALID_ARG, "x_cat, out_cat and workspace must be 16-byte aligned");
    return batched_run(nprob, rho, total_blocks, x_cat, out_cat, ws, ctas_per_sm, option(TD_OPT_EDM_F32X2) != 0,
                       static_cast<cudaStream_t>(stream), nullptr);
}

td_status td_edm_batched(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat, float *out_cat,
                         void *ws, size_t ws_bytes, const td_batched_config *cfg, td_launch_stats *stats, void *stream)
{
    fail(TD_OK, "");
    if (stats) *stats = td_launch_stats{0, 0, 0, 0, 0};
    if (nprob == 0) return TD_OK;
    if (!batched_args_ok(nprob, n, d, x_cat, out_cat, ws)) return TD_ERR_INVALID_ARG;
    const uint32_t rho = cfg ? cfg->rho : 128;
    const uint32_t cps = cfg ? cfg->ctas_per_sm : 0;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<unsigned char> host;
    uint64_t total = 0;
    td_status s = batched_plan(nprob, n, d, rho, ws, ws_bytes, st, host, &total);
    if (s != TD_OK) return s;
    uint64_t ctas = 0;
    s = batched_run(nprob, rho, total, x_cat, out_cat, ws, cps, option(TD_OPT_EDM_F32X2) != 0, st, &ctas);
    if (stats) *stats = td_launch_stats{total, total, 0, 1, ctas};
    return s;
}

td_status td_edm_batched_autotune(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat,
                                  float *out_cat, void *ws, size_t ws_bytes, td_batched_config *best, float *best_ms,
                                  void *stream)
{
    fail(TD_OK, "");
    if (!best) return fail(TD_ERR_INVALID_ARG, "best is NULL");
    *best = td_batched_config{128, 0};
    if (best_ms) *best_ms = 0.0f;
    if (nprob == 0) return TD_OK;
    if (!batched_args_ok(nprob, n, d, x_cat, out_cat, ws)) return TD_ERR_INVALID_ARG;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool x2 = option(TD_OPT_EDM_F32X2) != 0;
    cudaEvent_t e0, e1;
    td_status s = cuda_status(cudaEventCreate(&e0), "autotune event");
    if (s != TD_OK) return s;
    s = cuda_status(cudaEventCreate(&e1), "autotune event");
    if (s != TD_OK) {
        cudaEventDestroy(e0);
        return s;
    }
    float best_t = -1.0f;
    const uint32_t rhos[2] = {64, 128};
    const uint32_t cpss[5] = {0, 1, 2, 3, 4};
    for (uint32_t rho : rhos) {
        std::vector<unsigned char> host;
        uint64_t total = 0;
        s = batched_plan(nprob, n, d, rho, ws, ws_bytes, st, host, &total);
        if (s != TD_OK) break;
        for (uint32_t cps : cpss) {
            s = batched_run(nprob, rho, total, x_cat, out_cat, ws, cps, x2, st, nullptr);  // warm-up
            if (s != TD_OK) break;
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 3 && s == TD_OK; ++rep)
                s = batched_run(nprob, rho, total, x_cat, out_cat, ws, cps, x2, st, nullptr);
            cudaEventRecord(e1, st);
            if (s != TD_OK) break;
            s = cuda_status(cudaEventSynchronize(e1), "autotune timing");
            if (s != TD_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.0f;
            if (best_t < 0.0f || ms < best_t) {
                best_t = ms;
                *best = td_batched_config{rho, cps};
            }
        }
        if (s != TD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != TD_OK) return s;
    if (best_ms) *best_ms = best_t;
    // leave the workspace planned for the winner
    std::vector<unsigned char> host;
    uint64_t total = 0;
    return batched_plan(nprob, n, d, best->rho, ws, ws_bytes, st, host, &total);
}

}  // extern "C"
