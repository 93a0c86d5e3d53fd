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
//   3. sixteen epilogue warps read the accumulator (warp w: TMEM lanes 32 (w mod 4) .., columns
//      32 (w / 4) ..), form D^2, queue the cancelling pairs in shared memory, take the square
//      root of the rest, and write rows through a per-warp shared-memory transpose so that each
//      store instruction covers 32 consecutive floats of one packed row;
//   4. the block's FP32 row and column points are staged by TMA into the (now free) operand
//      region, 128 features at a time, and the warps recompute the queued pairs from shared
//      memory -- up to 32 pairs per warp per round, lanes striding the features, partial sums
//      combined in a fixed butterfly order.
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
constexpr uint32_t BK = 64;           // features per BF16 TMA box (128 bytes)
constexpr uint32_t MAXKB = 4;         // BF16 boxes per operand: d <= 256
constexpr uint32_t BOX = BM * BK * 2; // 16 KB
constexpr uint32_t KF = 128;          // features per FP32 staging phase of the recompute (512 bytes)
constexpr uint32_t THREADS = 512;     // 16 warps
constexpr uint32_t WARPS = THREADS / 32;
constexpr uint32_t SLD = 33;          // padded row of the transpose stage
constexpr uint32_t PAIRS_PER_WARP = 32;  // recomputed pairs a warp holds per round

// Shared-memory layout (offsets from a 1024-byte aligned base).  The 128 KB operand region is
// used three ways in turn within a block: BF16 operands (TMA -> MMA), then the epilogue's
// transpose stage, then FP32 point features for the recompute (rows at 0, columns at 64 KB).
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_B = OFF_A + MAXKB * BOX;
constexpr uint32_t OFF_STAGE = 0;
constexpr uint32_t OFF_FROW = 0;
constexpr uint32_t OFF_FCOL = BM * KF * 4;
constexpr uint32_t OFF_QUEUE = OFF_B + MAXKB * BOX;
constexpr uint32_t OFF_NROW = OFF_QUEUE + BM * BM * 2;
constexpr uint32_t OFF_NCOL = OFF_NROW + BM * 4;
constexpr uint32_t OFF_CTRL = OFF_NCOL + BM * 4;
constexpr uint32_t SMEM_USED = OFF_CTRL + 64;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack for aligning the base
static_assert(OFF_B % 1024 == 0, "operand tiles must be 1024-byte aligned");
static_assert(WARPS * 32 * SLD * 4 <= 2 * MAXKB * BOX, "transpose stage must fit the operand region");
static_assert(2 * BM * KF * 4 <= 2 * MAXKB * BOX, "recompute staging must fit the operand region");
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

constexpr uint32_t TMEM_COLS = 128;
constexpr float kCancel = 1e-2f;  // recompute when D^2 < kCancel (|x_i|^2 + |x_j|^2)

// workspace status words (uint32): [0] error code, [1] reserved, [2..3] recomputed pairs (uint64)
enum : uint32_t { kErrNone = 0, kErrTmaWait = 1, kErrMmaWait = 2, kErrStageWait = 3 };

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
    k_gram(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap fmap,
           const float *__restrict__ norms, uint32_t n, uint32_t d, uint32_t nt, float *__restrict__ out,
           uint32_t *__restrict__ status)
{
    using namespace sm100;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t base = smem_u32(sm);
    float *stage_all = reinterpret_cast<float *>(sm + OFF_STAGE);
    const float *frow = reinterpret_cast<const float *>(sm + OFF_FROW);
    uint16_t *queue = reinterpret_cast<uint16_t *>(sm + OFF_QUEUE);
    float *nrow = reinterpret_cast<float *>(sm + OFF_NROW);
    float *ncol = reinterpret_cast<float *>(sm + OFF_NCOL);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(sm + OFF_CTRL);
    const uint32_t tma_bar = base + OFF_CTRL, mma_bar = base + OFF_CTRL + 8, stage_bar = base + OFF_CTRL + 16;
    uint32_t *tmem_slot = ctrl + 6;
    uint32_t *qcount = ctrl + 8;  // two counters, alternating by block
    uint32_t *abort_flag = ctrl + 10;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nkb = (d + BK - 1) / BK;
    const uint32_t nph = (d + KF - 1) / KF;
    const uint32_t idesc = umma_idesc_bf16_f32(BM, BM);

    if (tid == 0) {
        mbar_init(tma_bar, 1);
        mbar_init(mma_bar, 1);
        mbar_init(stage_bar, 1);
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

    uint32_t phase = 0, sphase = 0, it = 0;
    uint64_t recomputed = 0;
    const uint64_t tiles = tri(nt);
    for (uint64_t lam = blockIdx.x; lam < tiles; lam += gridDim.x, ++it) {
        uint32_t bi, bj;
        ltm_g(lam, bi, bj);
        const bool diag = bi == bj;
        uint32_t *qc = qcount + (it & 1);
        if (tid < BM) {
            const uint32_t r = bi * BM + tid;
            nrow[tid] = r < n ? norms[r] : 0.0f;
        } else if (tid < 2 * BM) {
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
            // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +32, columns 32 (w / 4) .. +32;
            // the operand region is free now and holds the per-warp transpose stages
            const uint32_t q = warp & 3, c0 = 32 * (warp >> 2);
            const uint32_t rl = 32 * q + lane, i = bi * BM + rl;
            const float ni = nrow[rl];
            float *st = stage_all + warp * 32 * SLD;
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
        }
        fence_proxy_async_smem();  // the stage's generic accesses precede the staging TMA below
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
        // ---- direct FP32 recompute of the cancelling pairs.  The block's row and column points
        // are staged by TMA, KF features per phase, into the operand region; each warp holds up
        // to 32 pairs per round, its lanes striding the features, and the per-lane partial sums
        // are combined in a fixed butterfly order at the end.
        const uint32_t Q = *qc;
        bool stage_ok = true;
        for (uint32_t r0 = 0; r0 < Q && stage_ok; r0 += WARPS * PAIRS_PER_WARP) {
            const uint32_t e0 = r0 + warp * PAIRS_PER_WARP;
            const uint32_t cnt = e0 < Q ? min(PAIRS_PER_WARP, Q - e0) : 0u;
            float part[PAIRS_PER_WARP];
#pragma unroll
            for (uint32_t t = 0; t < PAIRS_PER_WARP; ++t) part[t] = 0.0f;
            for (uint32_t ph = 0; ph < nph; ++ph) {
                if (tid == 0) {
                    mbar_arrive_expect_tx(stage_bar, BM * KF * 4 * (diag ? 1u : 2u));
                    tma_load_2d(base + OFF_FROW, &fmap, int32_t(ph * KF), int32_t(bi * BM), stage_bar);
                    if (!diag) tma_load_2d(base + OFF_FCOL, &fmap, int32_t(ph * KF), int32_t(bj * BM), stage_bar);
                }
                const bool got = mbar_wait(stage_bar, sphase);
                sphase ^= 1;
                stage_ok = __syncthreads_and(got) != 0;  // CTA-uniform: every thread leaves together
                if (!stage_ok) {
                    if (tid == 0) atomicCAS(status, kErrNone, kErrStageWait);
                    break;
                }
                const float *fcol = reinterpret_cast<const float *>(sm + (diag ? OFF_FROW : OFF_FCOL));
#pragma unroll
                for (uint32_t t = 0; t < PAIRS_PER_WARP; ++t) {
                    if (t < cnt) {
                        const uint32_t code = queue[e0 + t];
                        const float *xi = frow + (code >> 7) * KF, *xj = fcol + (code & 127u) * KF;
                        float acc = part[t];
#pragma unroll
                        for (uint32_t k = lane; k < KF; k += 32) {
                            const float tdiff = xi[k] - xj[k];
                            acc = fmaf(tdiff, tdiff, acc);
                        }
                        part[t] = acc;
                    }
                }
                fence_proxy_async_smem();
                __syncthreads();  // every warp is done with this phase before a TMA overwrites it
            }
            if (!stage_ok) break;
#pragma unroll
            for (uint32_t t = 0; t < PAIRS_PER_WARP; ++t) {
                if (t < cnt) {
                    float s = part[t];
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) {
                        const uint32_t code = queue[e0 + t];
                        const uint32_t i = bi * BM + (code >> 7), j = bj * BM + (code & 127u);
                        out[tri(i) + j] = sqrtf(s);
                    }
                }
            }
        }
        recomputed += Q;
        if (!stage_ok) {
            if (tid == 0) *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) break;
    }
    if (tid == 0 && recomputed) atomicAdd(reinterpret_cast<unsigned long long *>(status + 2), recomputed);
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
    // FP32 points for the direct recompute: KF-feature boxes of 128 rows, no swizzle
    CUtensorMap fmap;
    const cuuint64_t fstride[1] = {cuuint64_t(d) * 4};
    const cuuint32_t fbox[2] = {KF, BM};
    const CUresult r2 = enc(&fmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(x), gdim, fstride, fbox,
                            estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r2 != CUDA_SUCCESS) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled (FP32 points) failed (%d)", int(r2));
    s = cuda_status(cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES),
                    "td_edm_gram shared memory attribute");
    if (s != TD_OK) return s;
    const uint32_t nt = (n + BM - 1) / BM;
    const uint64_t tiles = tri(nt);
    const uint64_t grid = tiles < uint64_t(sm_count()) ? tiles : uint64_t(sm_count());
    k_gram<<<dim3(static_cast<uint32_t>(grid)), THREADS, SMEM_BYTES, st>>>(tmap, fmap, norms, n, d, nt, out, status);
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
