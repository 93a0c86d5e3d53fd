// td_gram.cu -- Euclidean distance map (Sec. IV of arXiv:1308.1419) for many features in Gram
// form on the tcgen05 tensor cores:
//     D(i, j)^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j>,
// with <x_i, x_j> from BF16 copies of the points accumulated in FP32 (TMEM), the squared norms in
// FP32 from the FP32 points.  The subtraction cancels when D^2 is small next to the norms, so
// every pair with D^2 < 1e-2 (|x_i|^2 + |x_j|^2) -- the diagonal included -- is recomputed in the
// direct FP32 form sum_k (x_i[k] - x_j[k])^2 from the FP32 points.
//
// Three kernels, stream-ordered:
//   k_gram_prep  BF16 copy of the points and FP32 squared norms.
//   k_gram       persistent, warp-specialised, one CTA per SM; 128 x 128 blocks of the packed lower
//                triangle issued by g(lambda) over the block triangle of side ceil(n / 128)
//                (Sec. II-A), every role walking the same block sequence:
//                  warp 0    TMA producer: 64-feature boxes (128 rows x 128 bytes, 128-byte swizzle)
//                            of the block's row and column points into a 4-stage ring;
//                  warp 1    MMA issuer: tcgen05.mma (M = N = 128, K = 16) into one of two FP32 TMEM
//                            accumulators, each ring stage released by tcgen05.commit;
//                  warps 2-17 epilogue: read the accumulator (warp w: TMEM lanes 32 (w mod 4) ..,
//                            columns 32 ((w - 2) / 4) ..) and release it at once, form D^2, append
//                            the cancelling pairs to this CTA's segment of the queue (one
//                            shared-memory atomic per warp and 32 columns), take the square root
//                            and write packed rows through a per-warp transpose in shared memory.
//                The two accumulators let the next block's loads and MMAs run under the epilogue.
//   k_gram_fix   recomputes the queued pairs in the direct form: one pair per 8-lane group, 16-byte
//                loads (a whole 128-byte line of each point per group load), lanes striding the
//                features, partial sums combined in a fixed butterfly order; 32 warps per queue
//                segment.
// If a segment is full, the epilogue recomputes the extra pairs itself.  Every mbarrier wait is
// bounded; a timeout records an error code in the workspace status word and the roles wind down,
// the tensor memory is released and the CTA ends.
#include <cuda.h>
#include <cuda_bf16.h>

#include "td_device.cuh"
#include "td_internal.h"
#include "td_sm100.cuh"
#include "td_dist.cuh"

namespace td {
namespace {

constexpr uint32_t BM = 128;           // block side (rows and columns)
constexpr uint32_t BK = 64;            // features per BF16 TMA box (128 bytes)
constexpr uint32_t BOX = BM * BK * 2;  // 16 KB
constexpr uint32_t STAGES = 4;         // ring stages, one box of rows and one of columns each
constexpr uint32_t EPI_WARPS = 16;
constexpr uint32_t THREADS = 32 * (2 + EPI_WARPS);
constexpr uint32_t SLD = 36;           // padded row of the transpose stage (16-byte rows)
constexpr uint32_t TMEM_COLS = 256;    // two 128-column FP32 accumulators
constexpr float kCancel = 1e-2f;       // recompute when D^2 < kCancel (|x_i|^2 + |x_j|^2)

constexpr uint32_t OFF_RING = 0;
constexpr uint32_t OFF_STAGE = OFF_RING + STAGES * 2 * BOX;
constexpr uint32_t OFF_BAR = OFF_STAGE + EPI_WARPS * 32 * SLD * 4;
constexpr uint32_t SMEM_USED = OFF_BAR + 128;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack for aligning the base
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

// workspace status words (uint32): [0] error code, [1] reserved, [2..3] recomputed pairs (uint64)
enum : uint32_t { kErrNone = 0, kErrProducer = 1, kErrMma = 2, kErrEpilogue = 3 };

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// BF16 copy of the points and FP32 squared norms; one warp per point.  The norms are padded
// with zeros up to npad (a whole number of blocks), so the epilogue reads them unchecked.
__global__ void __launch_bounds__(256) k_gram_prep(const float *__restrict__ x, uint32_t n, uint32_t npad,
                                                   uint32_t d, __nv_bfloat16 *__restrict__ xb,
                                                   float *__restrict__ norms)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) {
        if (warp < npad && lane == 0) norms[warp] = 0.0f;
        return;
    }
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

// Direct FP32 distance of one pair, sequential over the features (the epilogue's overflow path).
__device__ float direct_distance(const float *__restrict__ x, uint32_t d, uint32_t i, uint32_t j)
{
    const float *xi = x + uint64_t(i) * d, *xj = x + uint64_t(j) * d;
    float s = 0.0f;
    for (uint32_t k = 0; k < d; ++k) {
        const float t = __ldg(xi + k) - __ldg(xj + k);
        s = fmaf(t, t, s);
    }
    return dist_sqrt(s);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_gram(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ x, const float *__restrict__ norms,
           uint32_t n, uint32_t d, uint32_t nt, float *__restrict__ out, uint2 *__restrict__ queue, uint32_t seg,
           uint32_t *__restrict__ seg_count, uint32_t *__restrict__ status)
{
    using namespace sm100;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t base = smem_u32(sm);
    const uint32_t bar = base + OFF_BAR;  // full[4], empty[4], tfull[2], tempty[2], then tmem slot, abort
    auto full_bar = [&](uint32_t s) { return bar + 8 * s; };
    auto empty_bar = [&](uint32_t s) { return bar + 8 * (STAGES + s); };
    auto tfull_bar = [&](uint32_t a) { return bar + 8 * (2 * STAGES + a); };
    auto tempty_bar = [&](uint32_t a) { return bar + 8 * (2 * STAGES + 2 + a); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 8 * (2 * STAGES + 4));
    volatile uint32_t *abort_flag = tmem_slot + 1;
    unsigned long long *qcount = reinterpret_cast<unsigned long long *>(status + 2);
    uint32_t *scount = tmem_slot + 2;  // pairs this CTA has recomputed or queued (shared memory)
    uint2 *qseg = queue + uint64_t(blockIdx.x) * seg;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nkb = (d + BK - 1) / BK;
    const uint64_t tiles = tri(nt);

    if (tid == 0) {
        for (uint32_t s2 = 0; s2 < STAGES; ++s2) {
            mbar_init(full_bar(s2), 1);
            mbar_init(empty_bar(s2), 1);
        }
        for (uint32_t a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), EPI_WARPS);
        }
        fence_mbar_init();
        *abort_flag = 0;
        *scount = 0;
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto fail_role = [&](uint32_t code) {
        atomicCAS(status, kErrNone, code);  // keep the first error
        *abort_flag = 1;
    };

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            uint64_t g = 0;  // boxes issued so far: stage g % STAGES, round g / STAGES
            for (uint64_t lam = blockIdx.x; lam < tiles && !*abort_flag; lam += gridDim.x) {
                uint32_t bi, bj;
                ltm_g(lam, bi, bj);
                const bool diag = bi == bj;
                for (uint32_t kb = 0; kb < nkb; ++kb, ++g) {
                    const uint32_t s2 = uint32_t(g % STAGES), round = uint32_t(g / STAGES);
                    if (!mbar_wait(empty_bar(s2), (round & 1u) ^ 1u)) {
                        fail_role(kErrProducer);
                        break;
                    }
                    const uint32_t dstA = base + OFF_RING + s2 * 2 * BOX, dstB = dstA + BOX;
                    mbar_arrive_expect_tx(full_bar(s2), diag ? BOX : 2 * BOX);
                    tma_load_2d(dstA, &tmap, int32_t(kb * BK), int32_t(bi * BM), full_bar(s2));
                    if (!diag) tma_load_2d(dstB, &tmap, int32_t(kb * BK), int32_t(bj * BM), full_bar(s2));
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_bf16_f32(BM, BM);
            uint64_t g = 0, t = 0;
            for (uint64_t lam = blockIdx.x; lam < tiles && !*abort_flag; lam += gridDim.x, ++t) {
                uint32_t bi, bj;
                ltm_g(lam, bi, bj);
                const bool diag = bi == bj;
                const uint32_t a = uint32_t(t & 1), use = uint32_t(t >> 1);
                if (!mbar_wait(tempty_bar(a), (use & 1u) ^ 1u)) {
                    fail_role(kErrMma);
                    break;
                }
                tc_fence_after();
                const uint32_t dacc = tmem + a * BM;
                bool ok = true;
                for (uint32_t kb = 0; kb < nkb; ++kb, ++g) {
                    const uint32_t s2 = uint32_t(g % STAGES), round = uint32_t(g / STAGES);
                    if (!mbar_wait(full_bar(s2), round & 1u)) {
                        fail_role(kErrMma);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t srcA = base + OFF_RING + s2 * 2 * BOX, srcB = diag ? srcA : srcA + BOX;
#pragma unroll
                    for (uint32_t k = 0; k < BK / 16; ++k) {
                        if (kb * BK + k * 16 >= d) break;
                        umma_bf16(dacc, umma_desc_sw128(srcA + k * 32), umma_desc_sw128(srcB + k * 32), idesc,
                                  (kb | k) != 0);
                    }
                    umma_commit(empty_bar(s2));  // the stage is free once these MMAs complete
                }
                if (!ok) break;
                umma_commit(tfull_bar(a));  // the accumulator is ready once all MMAs complete
            }
        }
    } else {
        // ---------------- epilogue warps
        const uint32_t ew = warp - 2, q = warp & 3, c0 = 32 * (ew >> 2);
        float *st = reinterpret_cast<float *>(sm + OFF_STAGE) + ew * 32 * SLD;
        uint64_t t = 0;
        for (uint64_t lam = blockIdx.x; lam < tiles; lam += gridDim.x, ++t) {
            if (*abort_flag) break;
            uint32_t bi, bj;
            ltm_g(lam, bi, bj);
            const uint32_t a = uint32_t(t & 1), use = uint32_t(t >> 1);
            // this warp's 32 x 32 chunk: rows i0 + lane (TMEM lanes 32 q ..), columns jb + cc.  The
            // norms do not depend on the accumulator: their loads go out before the wait for it
            // (the norms are zero-padded to whole blocks, so the 16-byte loads need no bounds)
            const uint32_t i0 = bi * BM + 32 * q, i = i0 + lane, jb = bj * BM + c0;
            const float ni = __ldg(norms + i);
            float4 nq[8];
            const float4 *nj4 = reinterpret_cast<const float4 *>(norms + jb);
#pragma unroll
            for (uint32_t c4 = 0; c4 < 8; ++c4) nq[c4] = __ldg(nj4 + c4);
            const bool ready = __all_sync(0xffffffffu, mbar_wait(tfull_bar(a), use & 1u));
            if (!ready) {
                if (lane == 0) fail_role(kErrEpilogue);
                break;
            }
            tc_fence_after();
            // interior: every row below n and every column left of every row (then also below n)
            const bool interior = bi > bj && i0 + 32 <= n;
            float v[32];
            tmem_ld_32x32b_x32(tmem + a * BM + ((32 * q) << 16) + c0, v);
            // the accumulator is in registers: hand it back to the MMA warp before the arithmetic
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(a));
            // D^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j> and the cancellation test.  The sign of
            // d2 - kCancel s2 is shifted into `neg` (column cc at bit 31 - cc).  A pair with
            // d2 < 0 always cancels, so the NaN its square root gives is rewritten later.
            uint32_t neg = 0;
#pragma unroll
            for (uint32_t c4 = 0; c4 < 8; ++c4) {
                const float nj[4] = {nq[c4].x, nq[c4].y, nq[c4].z, nq[c4].w};
                float w[4];
#pragma unroll
                for (uint32_t k = 0; k < 4; ++k) {
                    const float s2 = ni + nj[k];
                    const float d2 = fmaf(-2.0f, v[4 * c4 + k], s2);
                    neg = __funnelshift_l(__float_as_uint(fmaf(-kCancel, s2, d2)), neg, 1);
                    w[k] = sqrt_approx(d2);
                }
                *reinterpret_cast<float4 *>(st + lane * SLD + 4 * c4) = make_float4(w[0], w[1], w[2], w[3]);
            }
            uint32_t mask = __brev(neg);  // bit cc: pair (i, jb + cc) cancels
            if (!interior) {  // keep pairs with i < n and j <= i (then j < n too)
                const uint32_t lim = i < n ? i + 1 : 0u;
                const uint32_t nv = lim > jb ? min(lim - jb, 32u) : 0u;
                mask &= nv >= 32u ? 0xffffffffu : ((1u << nv) - 1u);
            }
            if (__any_sync(0xffffffffu, mask != 0)) {
                // append this warp's cancelling pairs with one atomic: an exclusive scan of the
                // per-lane counts gives each lane its slots
                const uint32_t cnt = __popc(mask);
                uint32_t pre = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= uint32_t(o)) pre += y;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, pre, 31);
                pre -= cnt;
                unsigned long long slot0 = 0;
                if (lane == 31) slot0 = atomicAdd(scount, total);
                slot0 = __shfl_sync(0xffffffffu, slot0, 31);
                uint64_t slot = slot0 + pre;
                for (uint32_t m = mask; m; m &= m - 1, ++slot) {
                    const uint32_t cc = __ffs(m) - 1, j = jb + cc;
                    if (slot < seg) qseg[slot] = make_uint2(i, j);
                    else st[lane * SLD + cc] = direct_distance(x, d, i, j);  // segment full: recompute here
                }
            }
            __syncwarp();
            // transposed write-out: row i0 + rr, lane = column, 128 contiguous bytes per row
            const uint32_t jl = jb + lane;
            if (interior) {
                float *p = out + tri(i0) + jl;
                uint32_t step = i0 + 1;  // T(r + 1) - T(r) = r + 1
#pragma unroll 8
                for (uint32_t rr = 0; rr < 32; ++rr, ++step) {
                    *p = st[rr * SLD + lane];
                    p += step;
                }
            } else {
#pragma unroll 4
                for (uint32_t rr = 0; rr < 32; ++rr) {
                    const uint32_t i2 = i0 + rr;
                    if (i2 < n && jl <= i2) out[tri(i2) + jl] = st[rr * SLD + lane];
                }
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
    if (tid == 0) {
        const uint32_t cnt = *scount;
        seg_count[blockIdx.x] = cnt < seg ? cnt : seg;
        if (cnt) atomicAdd(qcount, (unsigned long long)cnt);
    }
}

// Direct FP32 recompute of the queued pairs: FIX_WARPS warps per queue segment, each warp in
// groups of FIX_LPP lanes, one pair per group (FIX_PPW pairs per warp step).  Lane r of a group
// reads float4 r, r + FIX_LPP, ... of both points, so each load of the group covers one whole
// 128-byte line of each point; its partial sums are combined in a fixed butterfly order within
// the group.  d is a multiple of 4.  Launched with gsize * FIX_WARPS / 8 CTAs of 256 threads.
// (A whole warp per pair spent a 5-level butterfly per pair and ran about 4x the instructions;
// walking all segments as one list balances better but ran 1.7x slower on the clustered
// workload: every warp then works in the same few blocks at once.)
constexpr uint32_t FIX_WARPS = 32;
constexpr uint32_t FIX_LPP = 8;
constexpr uint32_t FIX_PPW = 32 / FIX_LPP;

__global__ void __launch_bounds__(256, 4) k_gram_fix(const float *__restrict__ x, uint32_t d,
                                                     const uint2 *__restrict__ queue,
                                                     const uint32_t *__restrict__ seg_count, uint32_t seg,
                                                     uint32_t gsize, float *__restrict__ out)
{
    const uint32_t lane = threadIdx.x & 31, d4 = d / 4, grp = lane / FIX_LPP, sub = lane % FIX_LPP;
    const uint32_t wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t c = wid % gsize, kw = wid / gsize;  // segment, and this warp's rank in it
    if (kw >= FIX_WARPS) return;
    const uint32_t cnt = seg_count[c];
    const uint64_t total = cnt < seg ? cnt : seg;
    const uint2 *qs = queue + uint64_t(c) * seg;
    for (uint64_t e0 = uint64_t(kw) * FIX_PPW; e0 < total; e0 += FIX_WARPS * FIX_PPW) {  // warp-uniform
        const uint64_t e = e0 + grp;
        const bool live = e < total;
        const uint2 pr = live ? qs[e] : make_uint2(0u, 0u);
        const float4 *xi = reinterpret_cast<const float4 *>(x + uint64_t(pr.x) * d);
        const float4 *xj = reinterpret_cast<const float4 *>(x + uint64_t(pr.y) * d);
        float part = 0.0f;
#pragma unroll 4
        for (uint32_t k4 = sub; k4 < d4; k4 += FIX_LPP) {
            const float4 a = __ldg(xi + k4), b = __ldg(xj + k4);
            float t = a.x - b.x;
            part = fmaf(t, t, part);
            t = a.y - b.y;
            part = fmaf(t, t, part);
            t = a.z - b.z;
            part = fmaf(t, t, part);
            t = a.w - b.w;
            part = fmaf(t, t, part);
        }
#pragma unroll
        for (uint32_t o = FIX_LPP / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (live && sub == 0) out[tri(pr.x) + pr.y] = dist_sqrt(part);
    }
}

struct GramLayout {
    size_t norms, xb, queue, counts, total;
    uint32_t gsize, seg;
};

// status (256 B) | norms (n floats, zero-padded to whole blocks) | BF16 points | pair queue: one
// segment of seg pairs (8 B) per k_gram CTA, T(n)/32 + 65536 pairs in all (twice the 1/64
// fraction of clustered data, plus slack) | pairs queued per segment (uint32)
GramLayout gram_layout(uint32_t n, uint32_t d)
{
    GramLayout L;
    L.norms = 256;
    const size_t npad = size_t((n + BM - 1) / BM) * BM;
    L.xb = (L.norms + npad * 4 + 1023) & ~size_t(1023);
    L.queue = (L.xb + size_t(n) * d * 2 + 1023) & ~size_t(1023);
    const uint64_t tiles = tri((n + BM - 1) / BM), sms = uint64_t(sm_count());
    L.gsize = static_cast<uint32_t>(tiles < sms ? (tiles ? tiles : 1) : sms);
    const uint64_t seg = (tri(n) / 32 + 65536 + L.gsize - 1) / L.gsize;
    L.seg = static_cast<uint32_t>(seg < 0xffffffffull ? seg : 0xffffffffull);
    L.counts = (L.queue + size_t(L.gsize) * L.seg * 8 + 1023) & ~size_t(1023);
    L.total = L.counts + size_t(L.gsize) * 4;
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
    auto *queue = reinterpret_cast<uint2 *>(base + L.queue);
    auto *seg_count = reinterpret_cast<uint32_t *>(base + L.counts);
    td_status s = cuda_status(cudaMemsetAsync(status, 0, 16, st), "td_edm_gram status reset");
    if (s != TD_OK) return s;
    const uint32_t npad = (n + BM - 1) / BM * BM;
    k_gram_prep<<<(npad + 7) / 8, 256, 0, st>>>(x, n, npad, d, xb, norms);
    s = launch_status("td_edm_gram prep kernel");
    if (s != TD_OK) return s;
    CUtensorMap tmap;
    s = encode_tiled_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, xb, d, n, uint64_t(d) * 2, BK, BM,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != TD_OK) return s;
    s = set_dynamic_smem_once(reinterpret_cast<const void *>(k_gram), SMEM_BYTES);
    if (s != TD_OK) return s;
    const uint32_t nt = (n + BM - 1) / BM;
    k_gram<<<dim3(L.gsize), THREADS, SMEM_BYTES, st>>>(tmap, x, norms, n, d, nt, out, queue, L.seg, seg_count, status);
    s = launch_status("td_edm_gram kernel");
    if (s != TD_OK) return s;
    k_gram_fix<<<dim3(L.gsize * (FIX_WARPS / 8)), 256, 0, st>>>(x, d, queue, seg_count, L.seg, L.gsize, out);
    return launch_status("td_edm_gram recompute kernel");
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
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

td_status encode_tiled_2d(CUtensorMap *map, CUtensorMapDataType type, const void *base, uint64_t inner, uint64_t outer,
                          uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swizzle)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t gdim[2] = {inner, outer};
    const cuuint64_t gstride[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = enc(map, type, 2, const_cast<void *>(base), gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return TD_OK;
}

}  // namespace td
