// td_edm_batched_noalloc.cu -- td_edm_batched for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose memory pool already holds every
// byte of device memory it may use, a plugin hosted by a framework that owns all device
// allocations, or a latency-bound loop where an allocation (and the device synchronisation it can
// bring) is not acceptable.  td_edm_batched needs a small device workspace for its launch plan;
// this variant keeps that plan in a fixed array of device memory that is part of the library
// itself, so the call allocates nothing -- no cudaMalloc, no cudaFree, no host allocation.
//
// The array holds the plan of at most kMaxProblems problems (about 40 KB).  Every GPU that
// loads the library holds it until the process exits.  All calls share it and it keeps the last
// call's plan; the plan is rewritten in full by each call, so nothing in it needs clearing.
// Calls whose work overlaps on the GPU (different streams, or different host threads on the
// same device) race on the array: order them on one stream.
//
// In host code the array's name is only a host-side stand-in for the symbol, not a device
// address.  The device address is obtained with cudaGetSymbolAddress, once per device, with that
// device current, by the first call on that device; make that first call before any stream
// capture begins.
#include <cstring>
#include <mutex>

#include "td_device.cuh"
#include "td_internal.h"

namespace td {

// launch of the batched distance map on an already planned workspace (td_edm_batched.cu)
td_status batched_run(uint32_t nprob, uint32_t rho, uint64_t total, const float *x, float *out, const void *ws,
                      uint32_t ctas_per_sm, bool x2, cudaStream_t st, uint64_t *ctas);

namespace {

constexpr uint32_t kMaxProblems = 1024;
constexpr size_t kScratchBytes =
    sizeof(BatchHeader) + (size_t(kMaxProblems) + 1) * sizeof(uint64_t) + size_t(kMaxProblems) * sizeof(BatchMeta);

static __device__ __align__(256) unsigned char g_plan_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;                                   // guards the host staging and the address cache
void *g_scratch_addr[kMaxDevices] = {};            // device address of g_plan_scratch, per device
alignas(16) unsigned char g_stage[kScratchBytes];  // host image of the plan
uint32_t g_order[kMaxProblems];
uint64_t g_xoff[kMaxProblems], g_ooff[kMaxProblems];

td_status scratch_address(void **out)
{
    int dev = 0;
    td_status s = cuda_status(cudaGetDevice(&dev), "td_edm_batched_noalloc: cudaGetDevice");
    if (s != TD_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return fail(TD_ERR_UNSUPPORTED, "device index %d too large", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        s = cuda_status(cudaGetSymbolAddress(&p, g_plan_scratch), "td_edm_batched_noalloc: cudaGetSymbolAddress");
        if (s != TD_OK) return s;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TD_OK;
}

// Host image of the plan (the layout td_edm_batched_run reads), problems laid heaviest first with
// ties in input order -- td_edm_batched's order -- by a stable insertion sort, which needs no
// allocation.
uint64_t stage_plan(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho)
{
    for (uint32_t q = 0; q < nprob; ++q) {
        uint32_t k = q;
        const uint64_t w = batched_weight(n[q], d[q], rho);
        while (k > 0 && batched_weight(n[g_order[k - 1]], d[g_order[k - 1]], rho) < w) {
            g_order[k] = g_order[k - 1];
            --k;
        }
        g_order[k] = q;
    }
    std::memset(g_stage, 0, batched_workspace_bytes(nprob));
    return batched_fill_image(nprob, n, d, rho, g_order, g_xoff, g_ooff, g_stage);
}

}  // namespace
}  // namespace td

using namespace td;

extern "C" td_status td_edm_batched_noalloc(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat,
                                            float *out_cat, const td_batched_config *cfg, td_launch_stats *stats,
                                            void *stream)
{
    fail(TD_OK, "");
    if (stats) *stats = td_launch_stats{0, 0, 0, 0, 0};
    if (nprob == 0) return TD_OK;
    if (nprob > kMaxProblems)
        return fail(TD_ERR_INVALID_ARG, "td_edm_batched_noalloc takes at most %u problems (got %u)", kMaxProblems,
                    nprob);
    if (!n || !d) return fail(TD_ERR_INVALID_ARG, "n and d (host arrays) must be non-NULL");
    if (!x_cat || !out_cat) return fail(TD_ERR_INVALID_ARG, "x_cat and out_cat must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(x_cat) | reinterpret_cast<uintptr_t>(out_cat)) & 15u)
        return fail(TD_ERR_INVALID_ARG, "x_cat and out_cat must be 16-byte aligned");
    for (uint32_t q = 0; q < nprob; ++q)
        if (n[q] == 0 || d[q] == 0) return fail(TD_ERR_INVALID_ARG, "problem %u has n = 0 or d = 0", q);
    const uint32_t rho = cfg ? cfg->rho : 128;
    const uint32_t cps = cfg ? cfg->ctas_per_sm : 0;
    if (rho != 64 && rho != 128) return fail(TD_ERR_INVALID_ARG, "batched rho must be 64 or 128 (got %u)", rho);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_mu);
    void *ws = nullptr;
    td_status s = scratch_address(&ws);
    if (s != TD_OK) return s;
    const uint64_t total = stage_plan(nprob, n, d, rho);
    const size_t bytes = batched_workspace_bytes(nprob);
    // a pageable source: the copy returns once g_stage has been read, so the next call may reuse it
    s = cuda_status(cudaMemcpyAsync(ws, g_stage, bytes, cudaMemcpyHostToDevice, st),
                    "td_edm_batched_noalloc plan upload");
    if (s != TD_OK) return s;
    uint64_t ctas = 0;
    s = batched_run(nprob, rho, total, x_cat, out_cat, ws, cps, option(TD_OPT_EDM_F32X2) != 0, st, &ctas);
    if (stats) *stats = td_launch_stats{total, total, 0, 1, ctas};
    return s;
}
