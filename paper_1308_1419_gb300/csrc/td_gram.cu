// td_gram.cu -- Euclidean distance map (Sec. IV of arXiv:1308.1419) for many features in Gram
// form on the tcgen05 tensor cores:
//     D(i, j)^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j>,
// with <x_i, x_j> from BF16 copies of the points accumulated in FP32 (TMEM), the squared norms in
// FP32 from the FP32 points.  The subtraction cancels when D^2 is small next to the norms, so
// every pair with D^2 < 1e-2 (|x_i|^2 + |x_j|^2) -- the diagonal included -- is recomputed in the
// direct FP32 form sum_k (x_i[k] - x_j[k])^2 from the FP32 points.
//
// Layout of the work: 128 x 128 blocks of the packed lower triangle, issued by g(lambda) over the
// tile triangle of side ceil(n / 128) (Sec. II-A), one persistent CTA per SM.  Per block:
//   1. thread 0 issues TMA loads of the block's 128 row points and 128 column points (BF16,
//      64-feature boxes of 128 rows x 128 bytes, 128-byte swizzle) -- one set for a diagonal block;
//   2. one thread issues d/16 tcgen05.mma (M = N = 128, K = 16) into a 128-column FP32 TMEM
//      accumulator and commits to an mbarrier;
//   3. eight epilogue warps read the accumulator (warp w: TMEM lanes 32 (w mod 4) .., columns
//      64 (w / 4) ..), form D^2, queue the cancelling pairs in shared memory, take the square
//      root of the rest, and write rows through a per-warp shared-memory transpose so that each
//      store instruction covers 32 consecutive floats of one packed row;
//   4. the warps recompute the queued pairs, one warp per pair, lanes striding the features,
//      partial sums combined in a fixed butterfly order.
// Every mbarrier wait is bounded; a timeout records an error code in the workspace status word,
// releases the tensor memory and ends the CTA.
#include <cuda.h>
#include <cuda_bf16.h>

#include "td_device.cuh"
#include "td_internal.h"
#include "td_sm100.cuh"

namespace td {
namespace {

constexpr uint32_t BM = 128;          // block side (rows and columns)
constexpr uint32_t BK = 64;           // features per TMA box (128 bytes of BF16)
constexpr uint32_t MAXKB = 4;         // boxes per operand: d <= 256
constexpr uint32_t BOX = BM * BK * 2; // 16 KB
constexpr uint32_t THREADS = 256;
constexpr uint32_t SLD = 33;          // padded row of the transpose stage

// shared-memory layout (offsets from a 1024-byte aligned base)
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_B = OFF_A + MAXKB * BOX;
constexpr uint32_t OFF_STAGE = OFF_B + MAXKB * BOX;
constexpr uint32_t OFF_QUEUE = OFF_STAGE + (THREADS / 32) * 32 * SLD * 4;
constexpr uint32_t OFF_NROW = OFF_QUEUE + BM * BM * 2;
constexpr uint32_t OFF_NCOL = OFF_NROW + BM * 4;
constexpr uint32_t OFF_CTRL = OFF_NCOL + BM * 4;
constexpr uint32_t SMEM_USED = OFF_CTRL + 64;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack for aligning the base
static_assert(OFF_STAGE % 1024 == 0 && OFF_B % 1024 == 0, "operand tiles must be 1024-byte aligned");
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

constexpr uint32_t TMEM_COLS = 128;
constexpr float kCancel = 1e-2f;  // recompute when D^2 < kCancel (|x_i|^2 + |x_j|^2)

// workspace status words (uint32): [0] error code, [1] reserved, [2..3] fallback pairs (uint64)
enum : uint32_t { kErrNone = 0, kErrTmaWait = 1, kErrMmaWait = 2 };

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// BF16 copy of the points and FP32 squared norms; one warp per point.
__global__ void __launch_bounds__(256) k_gram_prep(const float *__restrict__ x, uint32_t n, uint32_t d,
                                                   __nv_bfloat16 *__restrict__ xb, float *__restrict__ norms)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float *xi = x + uint64_t(warp) * d;
    __nv_bfloat16 *bi = xb + uint64_t(warp) * d;
    float s = 0.0f;
    for (uint32_t k = lane; k < d; k += 32) {
        const float v = xi[k];
        bi[k] = __float2bfloat16_rn(v);
        s = fmaf(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) norms[warp] = s;
}

__global__ void __launch_bounds__(THREADS, 1)
    k_gram(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ x, const float *__restrict__ norms,
           uint32_t n, uint32_t d, uint32_t nt, float *__restrict__ out, uint32_t *__restrict__ status)
{
    using namespace sm100;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t base = smem_u32(sm);
    float *stage_all = reinterpret_cast<float *>(sm + OFF_STAGE);
    uint16_t *queue = reinterpret_cast<uint16_t *>(sm + OFF_QUEUE);
    float *nrow = reinterpret_cast<float *>(sm + OFF_NROW);
    float *ncol = reinterpret_cast<float *>(sm + OFF_NCOL);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(sm + OFF_CTRL);
    const uint32_t tma_bar = base + OFF_CTRL, mma_bar = base + OFF_CTRL + 8;
    uint32_t *tmem_slot = ctrl + 4;
    uint32_t *qcount = ctrl + 6;  // two counters, alternating by block
    uint32_t *abort_flag = ctrl + 8;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nkb = (d + BK - 1) / BK;
    const uint32_t idesc = umma_idesc_bf16_f32(BM, BM);

    if (tid == 0) {
        mbar_init(tma_bar, 1);
        mbar_init(mma_bar, 1);
        fence_mbar_init();
        qcount[0] = 0;
        qcount[1] = 0;
        *abort_flag = 0;
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    uint32_t phase = 0, it = 0;
    uint64_t fallback = 0;
    const uint64_t tiles = tri(nt);
    for (uint64_t lam = blockIdx.x; lam < tiles; lam += gridDim.x, ++it) {
        uint32_t bi, bj;
        ltm_g(lam, bi, bj);
        const bool diag = bi == bj;
        uint32_t *qc = qcount + (it & 1);
        if (tid < BM) {
            const uint32_t r = bi * BM + tid;
            nrow[tid] = r < n ? norms[r] : 0.0f;
        } else {
            const uint32_t c = bj * BM + (tid - BM);
            ncol[tid - BM] = c < n ? norms[c] : 0.0f;
        }
        if (tid == 0) {
            qcount[(it + 1) & 1] = 0;  // counter of the next block; its last readers passed the previous barrier
            mbar_arrive_expect_tx(tma_bar, nkb * BOX * (diag ? 1u : 2u));
            for (uint32_t kb = 0; kb < nkb; ++kb) {
                tma_load_2d(base + OFF_A + kb * BOX, &tmap, int32_t(kb * BK), int32_t(bi * BM), tma_bar);
                if (!diag) tma_load_2d(base + OFF_B + kb * BOX, &tmap, int32_t(kb * BK), int32_t(bj * BM), tma_bar);
            }
        }
        __syncthreads();
        if (warp == 0) {
            const bool ok = mbar_wait(tma_bar, phase);
            if (!ok && lane == 0) {
                atomicCAS(status, kErrNone, kErrTmaWait);  // keep the first error
                *abort_flag = 1;
            }
            if (ok && lane == 0) {
                tc_fence_after();
                const uint32_t bsrc = diag ? OFF_A : OFF_B;
                for (uint32_t kb = 0; kb < nkb; ++kb)
#pragma unroll
                    for (uint32_t k = 0; k < BK / 16; ++k) {
                        if (kb * BK + k * 16 >= d) break;
                        const uint64_t a = umma_desc_sw128(base + OFF_A + kb * BOX + k * 32);
                        const uint64_t b = umma_desc_sw128(base + bsrc + kb * BOX + k * 32);
                        umma_bf16(tmem, a, b, idesc, (kb | k) != 0);
                    }
                umma_commit(mma_bar);
            }
            __syncwarp();
        }
        // warp-uniform, since the tensor-memory loads below are .sync.aligned
        const bool mma_ok = __all_sync(0xffffffffu, mbar_wait(mma_bar, phase));
        if (!mma_ok && lane == 0) {
            atomicCAS(status, kErrNone, kErrMmaWait);
            *abort_flag = 1;
        }
        phase ^= 1;
        tc_fence_after();
        if (mma_ok) {
            // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +32, columns 64 (w / 4) .. +64
            const uint32_t q = warp & 3, h = warp >> 2;
            const uint32_t rl = 32 * q + lane, i = bi * BM + rl;
            const float ni = nrow[rl];
            float *st = stage_all + warp * 32 * SLD;
#pragma unroll 1
            for (uint32_t c = 0; c < 2; ++c) {
                const uint32_t c0 = 64 * h + 32 * c;
                float v[32];
                tmem_ld_32x32b_x32(tmem + ((32 * q) << 16) + c0, v);
#pragma unroll
                for (uint32_t cc = 0; cc < 32; ++cc) {
                    const uint32_t jl = c0 + cc, j = bj * BM + jl;
                    const float s = ni + ncol[jl];
                    const float d2 = fmaf(-2.0f, v[cc], s);
                    const bool cancel = d2 < kCancel * s;
                    if (cancel && i < n && j <= i) {
                        const uint32_t slot = atomicAdd(qc, 1u);
                        queue[slot] = static_cast<uint16_t>((rl << 7) | jl);
                    }
                    st[lane * SLD + cc] = cancel ? 0.0f : sqrt_approx(d2);
                }
                __syncwarp();
                const uint32_t j2 = bj * BM + c0 + lane;
#pragma unroll 4
                for (uint32_t rr = 0; rr < 32; ++rr) {
                    const uint32_t i2 = bi * BM + 32 * q + rr;
                    if (i2 < n && j2 <= i2) out[tri(i2) + j2] = st[rr * SLD + lane];
                }
                __syncwarp();
            }
        }
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
        // ---- direct FP32 recompute of the cancelling pairs, one warp per pair
        const uint32_t Q = *qc;
        for (uint32_t e = warp; e < Q; e += THREADS / 32) {
            const uint32_t code = queue[e];
            const uint32_t i = bi * BM + (code >> 7), j = bj * BM + (code & 127u);
            const float *xi = x + uint64_t(i) * d, *xj = x + uint64_t(j) * d;
            float s = 0.0f;
            for (uint32_t k = lane; k < d; k += 32) {
                const float t = __ldg(xi + k) - __ldg(xj + k);
                s = fmaf(t, t, s);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) out[tri(i) + j] = sqrtf(s);
        }
        fallback += Q;
        __syncthreads();
    }
    if (tid == 0 && fallback) atomicAdd(reinterpret_cast<unsigned long long *>(status + 2), fallback);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

struct GramLayout {
    size_t norms, xb, total;
};

GramLayout gram_layout(uint32_t n, uint32_t d)
{
    GramLayout L;
    L.norms = 256;
    L.xb = (L.norms + size_t(n) * 4 + 1023) & ~size_t(1023);
    L.total = L.xb + size_t(n) * d * 2;
    return L;
}

}  // namespace

size_t gram_workspace_bytes(uint32_t n, uint32_t d) { return gram_layout(n, d).total; }

td_status launch_gram(const float *x, uint32_t n, uint32_t d, float *out, void *ws, cudaStream_t st)
{
    const GramLayout L = gram_layout(n, d);
    auto *base = static_cast<unsigned char *>(ws);
    auto *status = reinterpret_cast<uint32_t *>(base);
    auto *norms = reinterpret_cast<float *>(base + L.norms);
    auto *xb = reinterpret_cast<__nv_bfloat16 *>(base + L.xb);
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    td_status s = cuda_status(cudaMemsetAsync(status, 0, 16, st), "td_edm_gram status reset");
    if (s != TD_OK) return s;
    k_gram_prep<<<(n + 7) / 8, 256, 0, st>>>(x, n, d, xb, norms);
    s = launch_status("td_edm_gram prep kernel");
    if (s != TD_OK) return s;
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {d, n};
    const cuuint64_t gstride[1] = {cuuint64_t(d) * 2};
    const cuuint32_t box[2] = {BK, BM};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xb, gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    s = cuda_status(cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                    "td_edm_gram shared memory attribute");
    if (s != TD_OK) return s;
    const uint32_t nt = (n + BM - 1) / BM;
    const uint64_t tiles = tri(nt);
    const uint64_t grid = tiles < uint64_t(sm_count()) ? tiles : uint64_t(sm_count());
    k_gram<<<dim3(static_cast<uint32_t>(grid)), THREADS, SMEM_BYTES, st>>>(tmap, x, norms, n, d, nt, out, status);
    return launch_status("td_edm_gram kernel");
}

td_status read_gram_status(const void *ws, uint32_t *err, uint64_t *fallback, cudaStream_t st)
{
    uint32_t h[4] = {0, 0, 0, 0};
    td_status s = cuda_status(cudaMemcpyAsync(h, ws, 16, cudaMemcpyDeviceToHost, st), "td_edm_gram_status copy");
    if (s != TD_OK) return s;
    s = cuda_status(cudaStreamSynchronize(st), "td_edm_gram_status sync");
    if (s != TD_OK) return s;
    *err = h[0];
    *fallback = uint64_t(h[2]) | (uint64_t(h[3]) << 32);
    return TD_OK;
}

}  // namespace td
