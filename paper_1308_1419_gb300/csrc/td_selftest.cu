// td_selftest.cu -- the failure path of the bounded waits, taken on purpose.  One CTA waits on an
// mbarrier with the same bounded wait the Gram pipeline uses (sm100::mbar_wait); when nothing
// arrives on the barrier the wait gives up after its limit, the kernel records that and returns,
// and the host reads the record.  Nothing traps, faults or spins without a limit, and the context
// stays usable afterwards.
#include "td_internal.h"
#include "td_sm100.cuh"

namespace td {
namespace {

// rec[0] = 0 if the wait saw the phase complete, 1 if it ran out; rec[1] = its duration in ns.
__global__ void k_wait_selftest(uint32_t arrive, uint64_t limit_ns, uint64_t *rec)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = sm100::smem_u32(&bar);
    if (threadIdx.x == 0) {
        sm100::mbar_init(b, 1);
        sm100::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive) sm100::mbar_arrive(b);
        const uint64_t t0 = sm100::global_ns();
        const bool ok = sm100::mbar_wait(b, 0, limit_ns);
        const uint64_t t1 = sm100::global_ns();
        rec[0] = ok ? 0 : 1;
        rec[1] = t1 - t0;
    }
}

}  // namespace

td_status launch_wait_selftest(uint32_t arrive, uint64_t limit_ns, uint64_t *rec, uint64_t out[2], cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(arrive, limit_ns, rec);
    td_status s = launch_status("k_wait_selftest");
    if (s != TD_OK) return s;
    s = cuda_status(cudaMemcpyAsync(out, rec, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st), "td_wait_selftest copy");
    if (s != TD_OK) return s;
    return cuda_status(cudaStreamSynchronize(st), "td_wait_selftest sync");
}

}  // namespace td
