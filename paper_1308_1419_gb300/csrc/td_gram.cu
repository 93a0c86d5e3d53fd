// td_gram.cu -- Euclidean distance map (Sec. IV of arXiv:1308.1419) for many features in Gram
// form on the tcgen05 tensor cores:
//     D(i, j)^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j>,
// with <x_i, x_j> from BF16 copies of the points accumulated in FP32 (TMEM), the squared norms in
// FP32 from the FP32 points.  The subtraction cancels when D^2 is small next to the norms, so
// every pair with D^2 < 1e-2 (|x_i|^2 + |x_j|^2) -- the diagonal included -- is recomputed in the
// direct FP32 form sum_k (x_i[k] - x_j[k])^2 from the FP32 points.
//
// Three kernels, stream-ordered:
//   k_gram_prep  BF16 copy of the points and FP32 squared norms; clears the queue counters and the
//                status block.
//   k_gram       persistent, warp-specialised, one CTA per SM; 128 x 128 blocks of the packed lower
//                triangle issued by g(lambda) over the block triangle of side ceil(n / 128)
//                (Sec. II-A), every role walking the same block sequence:
//                  warp 0    TMA producer: 64-feature boxes (128 rows x 128 bytes, 128-byte swizzle)
//                            of the block's row and column points into a 4-stage ring;
//                  warp 1    MMA issuer: tcgen05.mma (M = N = 128, K = 16) into one of two FP32 TMEM
//                            accumulators, each ring stage released by tcgen05.commit;
//                  warps 2-17 epilogue: read the accumulator (warp w: TMEM lanes 32 (w mod 4) ..,
//                            columns 32 ((w - 2) / 4) ..) and release it at once, form D^2, take
//                            the square root and write the packed rows; reserve queue slots for
//                            the cancelling pairs (one global atomic per warp and 32 x 32 chunk,
//                            in the queue region of the block's 32-row quarter) and write them
//                            one block later, when the reservation has come back.  The MMA takes
//                            the column block's points as A, so the accumulator is D transposed:
//                            a lane holds one column for 32 rows, and each row's 32 columns
//                            leave as one 128-byte store, with no transpose through shared memory.
//                The two accumulators let the next block's loads and MMAs run under the epilogue.
//   k_gram_fix   recomputes the queued pairs in the direct form, one CTA per quarter of a run of
//                blocks of one block row: the pairs are sorted by row in shared memory, a warp
//                holds a row point in registers and streams its column points four at a time.
// If a region is full, the epilogue recomputes the extra pairs itself.  Every mbarrier wait is
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
constexpr uint32_t TMEM_COLS = 256;    // two 128-column FP32 accumulators
constexpr float kCancel = 1e-2f;       // recompute when D^2 < kCancel (|x_i|^2 + |x_j|^2)

constexpr uint32_t OFF_RING = 0;
constexpr uint32_t OFF_BAR = OFF_RING + STAGES * 2 * BOX;
constexpr uint32_t SMEM_USED = OFF_BAR + 128;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack for aligning the base
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

// Recompute queue: one region of QQ pairs per 32-row quarter of a BM x BM block (quarter r of
// block lambda at (4 lambda + r) QQ), 1/32 of the quarter's pairs, twice the 1/64 that cancels in
// clustered data, with one counter per region.  A pair that finds its region full is recomputed
// by the epilogue itself.
constexpr uint32_t QQ = 32 * BM / 32;

// The recompute takes the blocks of block row b (lambda = T(b) .. T(b) + b) in runs of FIX_R, so
// the row has b / FIX_R + 1 parts (its work grows with b); fix_units(b) = the parts of block rows
// 0 .. b - 1 = b + FIX_R q (q - 1) / 2 + r q, b = q FIX_R + r.
constexpr uint32_t FIX_R = 16;
__host__ __device__ __forceinline__ uint64_t fix_units(uint32_t b)
{
    const uint64_t q = b / FIX_R, r = b % FIX_R;
    return b + FIX_R * q * (q - (q ? 1 : 0)) / 2 + r * q;
}

// workspace status words (uint32): [0] error code, [1] reserved, [2..3] recomputed pairs (uint64)
enum : uint32_t { kErrNone = 0, kErrProducer = 1, kErrMma = 2, kErrEpilogue = 3 };

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// BF16 copy of the points and FP32 squared norms; one warp per point.  The norms are padded
// with zeros up to npad (a whole number of blocks), so the epilogue reads them unchecked.  Also
// clears the counters of the recompute queue's regions and the status block (the first kernel of
// the call, so no separate memset is needed).
__global__ void __launch_bounds__(256) k_gram_prep(const float *__restrict__ x, uint32_t n, uint32_t npad,
                                                   uint32_t d, __nv_bfloat16 *__restrict__ xb,
                                                   float *__restrict__ norms, uint32_t *__restrict__ qcount,
                                                   uint64_t regions, uint32_t *__restrict__ status)
{
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x, warp = gid >> 5, lane = threadIdx.x & 31;
    if (gid < 4) status[gid] = 0;  // error word, reserved word, recomputed pairs
    for (uint64_t k = gid; k < regions; k += uint64_t(gridDim.x) * blockDim.x) qcount[k] = 0;
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

// kOneStep (d <= 64, one k-step per block): the block's MMA is short, and the epilogue would wait
// on its norm loads, so the next block's norm lines are prefetched into L1 one block ahead, and an
// interior block's rows are stored after all 32 distances are formed.  With more k-steps the MMA
// covers the norm loads, and the rows are stored as they are formed, interleaved with the square
// roots.  (Each choice measured faster in its own range: n = 16384, d = 64 and d = 256.)
template <bool kOneStep>
__global__ void __launch_bounds__(THREADS, 1)
    k_gram(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ x, const float *__restrict__ norms,
           uint32_t n, uint32_t d, uint32_t nt, float *__restrict__ out, uint2 *__restrict__ queue,
           uint32_t *__restrict__ qcount, uint32_t *__restrict__ status)
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
                    // the accumulator is D transposed: A = the column block's points (TMEM lanes = columns),
                    // B = the row block's (TMEM columns = rows)
                    const uint32_t rowsb = base + OFF_RING + s2 * 2 * BOX, colsb = diag ? rowsb : rowsb + BOX;
                    const uint32_t srcA = colsb, srcB = rowsb;
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
        // The previous block's cancelling pairs wait here until the next block has been written:
        // by then the reservation of their queue slots (a global atomic) has long come back.
        bool p_any = false;
        uint32_t p_mask = 0, p_pre = 0, p_slot = 0, p_ib = 0, p_j = 0;
        uint64_t p_reg = 0;
        auto flush = [&]() {  // warp-uniform
            if (!p_any) return;
            uint32_t slot = __shfl_sync(0xffffffffu, p_slot, 31) + p_pre;
            uint2 *qr = queue + p_reg * QQ;
            for (uint32_t m = p_mask; m; m &= m - 1, ++slot) {
                const uint32_t i = p_ib + __ffs(m) - 1;
                if (slot < QQ) qr[slot] = make_uint2(i, p_j);
                else out[tri(i) + p_j] = direct_distance(x, d, i, p_j);  // region full: recompute here (after its store)
            }
            p_any = false;
        };
        uint64_t t = 0;
        for (uint64_t lam = blockIdx.x; lam < tiles; lam += gridDim.x, ++t) {
            if (*abort_flag) break;
            uint32_t bi, bj;
            ltm_g(lam, bi, bj);
            const uint32_t a = uint32_t(t & 1), use = uint32_t(t >> 1);
            // this warp's 32 x 32 chunk of the transposed accumulator: TMEM lane 32 q + lane is column
            // j = jb + lane, TMEM columns c0 .. c0 + 31 are rows ib .. ib + 31, so this lane holds
            // D(ib + c, j) for c = 0 .. 31 and a row's 32 columns lie in the warp's 32 lanes.  The
            // norms do not depend on the accumulator: their loads go out before the wait for it (the
            // norms are zero-padded to whole blocks, so the 16-byte loads need no bounds)
            const uint32_t jb = bj * BM + 32 * q, j = jb + lane, ib = bi * BM + c0;
            if (kOneStep && lam + gridDim.x < tiles && lane < 2) {  // the next block's norm lines
                uint32_t bi2, bj2;
                ltm_g(lam + gridDim.x, bi2, bj2);
                const float *nl = norms + (lane ? bi2 * BM + c0 : bj2 * BM + 32 * q);
                asm volatile("prefetch.global.L1 [%0];" ::"l"(nl));
            }
            const float nj = __ldg(norms + j);
            float4 nq[8];
            const float4 *ni4 = reinterpret_cast<const float4 *>(norms + ib);
#pragma unroll
            for (uint32_t c4 = 0; c4 < 8; ++c4) nq[c4] = __ldg(ni4 + c4);
            const bool ready = __all_sync(0xffffffffu, mbar_wait(tfull_bar(a), use & 1u));
            if (!ready) {
                if (lane == 0) fail_role(kErrEpilogue);
                break;
            }
            tc_fence_after();
            // interior: every row below n and every column left of every row (then also below n)
            const bool interior = bi > bj && ib + 32 <= n;
            float v[32];
            tmem_ld_32x32b_x32(tmem + a * BM + ((32 * q) << 16) + c0, v);
            // the accumulator is in registers: hand it back to the MMA warp before the arithmetic
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(a));
            // D^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j> and the cancellation test.  The sign of
            // d2 - kCancel s2 is shifted into `neg` (row c at bit 31 - c).  A pair with d2 < 0 always
            // cancels, so the NaN its square root gives is rewritten later.
            uint32_t neg = 0;
            if constexpr (!kOneStep) {
                // each interior row's 128 bytes leave as soon as they are formed
                float *p = out + tri(ib) + j;  // row ib + c at p, then p += ib + c + 1
                uint32_t step = ib + 1;
#pragma unroll
                for (uint32_t c4 = 0; c4 < 8; ++c4) {
                    const float ni[4] = {nq[c4].x, nq[c4].y, nq[c4].z, nq[c4].w};
#pragma unroll
                    for (uint32_t k = 0; k < 4; ++k) {
                        const float s2 = ni[k] + nj;
                        const float d2 = fmaf(-2.0f, v[4 * c4 + k], s2);
                        neg = __funnelshift_l(__float_as_uint(fmaf(-kCancel, s2, d2)), neg, 1);
                        v[4 * c4 + k] = sqrt_approx(d2);
                        if (interior) {
                            *p = v[4 * c4 + k];
                            p += step++;
                        }
                    }
                }
            } else {
#pragma unroll
                for (uint32_t c4 = 0; c4 < 8; ++c4) {
                    const float ni[4] = {nq[c4].x, nq[c4].y, nq[c4].z, nq[c4].w};
#pragma unroll
                    for (uint32_t k = 0; k < 4; ++k) {
                        const float s2 = ni[k] + nj;
                        const float d2 = fmaf(-2.0f, v[4 * c4 + k], s2);
                        neg = __funnelshift_l(__float_as_uint(fmaf(-kCancel, s2, d2)), neg, 1);
                        v[4 * c4 + k] = sqrt_approx(d2);
                    }
                }
            }
            uint32_t mask = __brev(neg);  // bit c: pair (ib + c, j) cancels
            if (!interior) {  // keep rows below n with j <= i
                const uint32_t lo = j > ib ? j - ib : 0u, hi = n > ib ? min(n - ib, 32u) : 0u;
                const uint32_t below = hi >= 32u ? 0xffffffffu : ((1u << hi) - 1u);
                mask &= lo >= 32u ? 0u : (below & (0xffffffffu << lo));
            }
            // write-out (the rest): row ib + c, lane = column, 128 contiguous bytes per row and store instruction
            if (kOneStep && interior) {
                float *p = out + tri(ib) + j;
                uint32_t step = ib + 1;  // T(r + 1) - T(r) = r + 1
#pragma unroll
                for (uint32_t c = 0; c < 32; ++c, ++step) {
                    *p = v[c];
                    p += step;
                }
            } else if (!interior) {
#pragma unroll
                for (uint32_t c = 0; c < 32; ++c) {
                    const uint32_t i2 = ib + c;
                    if (i2 < n && j <= i2) out[tri(i2) + j] = v[c];
                }
            }
            flush();
            if (__any_sync(0xffffffffu, mask != 0)) {
                // reserve queue slots for this warp's cancelling pairs with one atomic (written at the
                // next flush): an exclusive scan of the per-lane counts gives each lane its slots
                const uint32_t cnt = __popc(mask);
                uint32_t pre = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= uint32_t(o)) pre += y;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, pre, 31);
                pre -= cnt;
                const uint64_t reg = 4 * lam + (ew >> 2);  // this warp's rows are quarter c0 / 32 of the block
                p_slot = 0;
                if (lane == 31) p_slot = atomicAdd(qcount + reg, total);
                p_any = true;
                p_mask = mask;
                p_pre = pre;
                p_ib = ib;
                p_j = j;
                p_reg = reg;
            }
        }
        flush();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// Direct FP32 recompute of the queued pairs.  CTA 4k + r takes quarter r (rows i0 .. i0 + 31,
// i0 = 128 b + 32 r) of part p of block row b (the parts of the top block rows, the longest, get
// the lowest k): the quarter-r regions of blocks T(b) + p FIX_R .. T(b) + min(p FIX_R + FIX_R,
// b + 1) - 1.  Set-up, one round trip: the region counters and every slot of the regions (those
// past a counter are never read) are loaded together; the valid pairs are then sorted by row in
// shared memory (a 32-bin counting sort).  Then each warp takes rows, holds the row point in
// registers (two float4 per lane for up to 256 features) and streams the row's column points
// four at a time, lane l reading float4 l and l + 32 of each (512 contiguous bytes per load), so
// only the column points pass through L1.  Two features go through each packed sub.rn.f32x2 /
// fma.rn.f32x2, and the four sums are combined across the warp in six shuffles (two halving
// exchanges, then three butterfly steps), a fixed order.  For d > 256 the features go in chunks
// of 256 and the row point's chunk is reloaded (from L1) per four pairs.  d is a multiple of 4.
// (One pair per 8-lane group, with both points loaded per pair or the row point staged in shared
// memory, moved both points through L1 for every pair and ran about 2x the instructions.)  Each
// CTA adds its regions' counts, overflow included, to the status block's recomputed-pairs word.
constexpr uint32_t FIX_THREADS = 256;
constexpr uint32_t FIX_SPT = FIX_R * QQ / FIX_THREADS;  // region slots per thread
static_assert(FIX_R * QQ % FIX_THREADS == 0 && FIX_R <= 32, "fix set-up shape");

// One chunk of 64 float4 for four pairs (row point a0, a1 = float4 lane and lane + 32 of the
// chunk; column points jj): loads the column points' float4 and accumulates the squared
// differences into packed (even, odd) feature sums.  A lane outside the features (in0 / in1
// false) reads nothing and adds (0 - 0)^2.
template <bool kWhole>
__device__ __forceinline__ void fix_chunk(const ulonglong2 &a0, const ulonglong2 &a1, const ulonglong2 *xl,
                                          const uint32_t (&jj)[4], uint32_t d4, uint32_t kc, bool in0, bool in1,
                                          unsigned long long (&acc)[4])
{
    ulonglong2 c0[4], c1[4];
#pragma unroll
    for (uint32_t p = 0; p < 4; ++p) {
        const ulonglong2 *xj = xl + uint64_t(jj[p]) * d4 + kc;
        c0[p] = (kWhole || in0) ? __ldg(xj) : make_ulonglong2(0ull, 0ull);
        c1[p] = (kWhole || in1) ? __ldg(xj + 32) : make_ulonglong2(0ull, 0ull);
    }
#pragma unroll
    for (uint32_t p = 0; p < 4; ++p) {
        unsigned long long t = sub_f32x2(a0.x, c0[p].x);
        acc[p] = fma_f32x2(t, t, acc[p]);
        t = sub_f32x2(a0.y, c0[p].y);
        acc[p] = fma_f32x2(t, t, acc[p]);
        t = sub_f32x2(a1.x, c1[p].x);
        acc[p] = fma_f32x2(t, t, acc[p]);
        t = sub_f32x2(a1.y, c1[p].y);
        acc[p] = fma_f32x2(t, t, acc[p]);
    }
}

template <bool kOne>  // d <= 256: the row point is loaded once per row
__global__ void __launch_bounds__(FIX_THREADS, 4)
    k_gram_fix(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t nb, const uint2 *__restrict__ queue,
               const uint32_t *__restrict__ qcount, float *__restrict__ out,
               unsigned long long *__restrict__ fallback)
{
    __shared__ uint32_t s_cnt[FIX_R], s_hist[32], s_start[33];
    __shared__ uint32_t s_col[FIX_R * QQ + 4];  // column of each valid pair, grouped by row, then 4 pads
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t u = fix_units(nb) - 1 - blockIdx.x / 4;
    const uint32_t qtr = blockIdx.x % 4;
    uint32_t b = 0, hi = nb - 1;  // the block row: fix_units(b) <= u < fix_units(b + 1)
    while (b < hi) {
        const uint32_t mid = (b + hi + 1) / 2;
        if (fix_units(mid) <= u) b = mid;
        else hi = mid - 1;
    }
    const uint32_t k0 = uint32_t(u - fix_units(b)) * FIX_R, nk = min(FIX_R, b + 1 - k0);
    const uint64_t reg0 = 4 * (tri(b) + k0) + qtr;  // region of block k: reg0 + 4 k
    const uint32_t i0 = b * BM + 32 * qtr;          // a queued pair of these regions has its row in i0 .. i0 + 31
    if (tid < 32) s_hist[tid] = 0;
    uint32_t cv = 0;
    uint2 qv[FIX_SPT];
    if (tid < nk) cv = qcount[reg0 + 4 * tid];
#pragma unroll
    for (uint32_t w = 0; w < FIX_SPT; ++w) {
        const uint32_t sl = tid + w * FIX_THREADS, k = sl / QQ;
        qv[w] = k < nk ? queue[(reg0 + 4 * k) * QQ + sl % QQ] : make_uint2(0u, 0u);
    }
    if (tid < nk) s_cnt[tid] = cv;
    __syncthreads();
    uint32_t rk[FIX_SPT];  // rank of the pair among its row's, or ~0 for a slot past its counter
#pragma unroll
    for (uint32_t w = 0; w < FIX_SPT; ++w) {
        const uint32_t sl = tid + w * FIX_THREADS, k = sl / QQ;
        rk[w] = ~0u;
        if (k < nk && sl % QQ < min(s_cnt[k], QQ) && qv[w].x - i0 < 32u)  // (the row test always holds)
            rk[w] = atomicAdd(&s_hist[qv[w].x - i0], 1u);
    }
    if (tid == 0) {
        unsigned long long all = 0;
        for (uint32_t k = 0; k < nk; ++k) all += s_cnt[k];
        if (all) atomicAdd(fallback, all);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the row counts
        uint32_t v = s_hist[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= uint32_t(o)) v += y;
        }
        s_start[lane + 1] = v;
        if (lane == 0) s_start[0] = 0;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t w = 0; w < FIX_SPT; ++w)
        if (rk[w] != ~0u) s_col[s_start[qv[w].x - i0] + rk[w]] = qv[w].y;
    if (tid < 4) s_col[s_start[32] + tid] = i0;  // a row's last group of four may read past the list
    __syncthreads();

    const uint32_t d4 = d / 4;
    const bool whole = d4 == 64;  // d = 256: each lane holds float4 lane and lane + 32 of a point, no bounds
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    const uint32_t mine = (hi16 ? 2u : 0u) + (hi8 ? 1u : 0u);  // the pair whose sum this lane ends with
    const ulonglong2 *xl = reinterpret_cast<const ulonglong2 *>(x) + lane;  // a float4 as two packed pairs
    for (uint32_t r = warp; r < 32; r += FIX_THREADS / 32) {
        const uint32_t beg = s_start[r], end = s_start[r + 1];
        if (beg == end) continue;
        const uint32_t i = i0 + r;
        const ulonglong2 *xi = xl + uint64_t(i) * d4;
        ulonglong2 h0 = make_ulonglong2(0ull, 0ull), h1 = h0;
        if (kOne) {
            if (lane < d4) h0 = __ldg(xi);
            if (lane + 32 < d4) h1 = __ldg(xi + 32);
        }
        const uint64_t ti = tri(i);
        for (uint32_t e = beg; e < end; e += 4) {
            uint32_t jj[4];
#pragma unroll
            for (uint32_t p = 0; p < 4; ++p) jj[p] = s_col[e + p];  // past the row: other valid columns
            unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};  // packed (even, odd) feature sums
            if (kOne && whole) {
                fix_chunk<true>(h0, h1, xl, jj, d4, 0, true, true, acc);
            } else if (kOne) {
                fix_chunk<false>(h0, h1, xl, jj, d4, 0, lane < d4, lane + 32 < d4, acc);
            } else {
                for (uint32_t kc = 0; kc < d4; kc += 64) {
                    const bool in0 = kc + lane < d4, in1 = kc + lane + 32 < d4;
                    const ulonglong2 a0 = in0 ? __ldg(xi + kc) : make_ulonglong2(0ull, 0ull);
                    const ulonglong2 a1 = in1 ? __ldg(xi + kc + 32) : make_ulonglong2(0ull, 0ull);
                    fix_chunk<false>(a0, a1, xl, jj, d4, kc, in0, in1, acc);
                }
            }
            float sum[4];
#pragma unroll
            for (uint32_t p = 0; p < 4; ++p) {
                float lo, hi2;
                unpack2(acc[p], lo, hi2);
                sum[p] = lo + hi2;
            }
            // four sums over 32 lanes: lanes 0-15 keep pairs 0 and 1 and lanes 16-31 pairs 2 and 3,
            // each adding the partner's (lane ^ 16) share; then lanes with bit 3 clear keep the
            // first of the two, the others the second, adding lane ^ 8's; then an 8-lane butterfly
            float k0 = hi16 ? sum[2] : sum[0], k1 = hi16 ? sum[3] : sum[1];
            const float g0 = hi16 ? sum[0] : sum[2], g1 = hi16 ? sum[1] : sum[3];
            k0 += __shfl_xor_sync(0xffffffffu, g0, 16);
            k1 += __shfl_xor_sync(0xffffffffu, g1, 16);
            float v = hi8 ? k1 : k0;
            v += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            const uint32_t jm = mine == 0 ? jj[0] : mine == 1 ? jj[1] : mine == 2 ? jj[2] : jj[3];
            if ((lane & 7) == 0 && e + mine < end) out[ti + jm] = dist_sqrt(v);
        }
    }
}

struct GramLayout {
    size_t norms, xb, queue, counts, total;
    uint32_t gsize, nb;
    uint64_t regions;
};

// status (256 B) | norms (n floats, zero-padded to whole blocks) | BF16 points | recompute queue:
// QQ pairs (8 B) per quarter of a block | pairs queued per quarter (uint32)
GramLayout gram_layout(uint32_t n, uint32_t d)
{
    GramLayout L;
    L.nb = (n + BM - 1) / BM;
    L.norms = 256;
    const size_t npad = size_t(L.nb) * BM;
    L.xb = (L.norms + npad * 4 + 1023) & ~size_t(1023);
    L.queue = (L.xb + size_t(n) * d * 2 + 1023) & ~size_t(1023);
    const uint64_t tiles = tri(L.nb), sms = uint64_t(sm_count());
    L.gsize = static_cast<uint32_t>(tiles < sms ? (tiles ? tiles : 1) : sms);
    L.regions = 4 * tiles;
    L.counts = (L.queue + L.regions * QQ * 8 + 1023) & ~size_t(1023);
    L.total = L.counts + L.regions * 4;
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
    auto *qcount = reinterpret_cast<uint32_t *>(base + L.counts);
    const uint32_t npad = (n + BM - 1) / BM * BM;
    k_gram_prep<<<(npad + 7) / 8, 256, 0, st>>>(x, n, npad, d, xb, norms, qcount, L.regions, status);
    td_status s = launch_status("td_edm_gram prep kernel");
    if (s != TD_OK) return s;
    CUtensorMap tmap;
    s = encode_tiled_2d(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, xb, d, n, uint64_t(d) * 2, BK, BM,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (s != TD_OK) return s;
    const bool ahead = d <= BK;
    s = set_dynamic_smem_once(ahead ? reinterpret_cast<const void *>(k_gram<true>)
                                    : reinterpret_cast<const void *>(k_gram<false>),
                              SMEM_BYTES);
    if (s != TD_OK) return s;
    const uint32_t nt = (n + BM - 1) / BM;
    if (ahead)
        k_gram<true><<<dim3(L.gsize), THREADS, SMEM_BYTES, st>>>(tmap, x, norms, n, d, nt, out, queue, qcount, status);
    else
        k_gram<false><<<dim3(L.gsize), THREADS, SMEM_BYTES, st>>>(tmap, x, norms, n, d, nt, out, queue, qcount, status);
    s = launch_status("td_edm_gram kernel");
    if (s != TD_OK) return s;
    auto *fallback = reinterpret_cast<unsigned long long *>(status + 2);
    const dim3 fgrid(static_cast<uint32_t>(4 * fix_units(L.nb)));
    if (d <= 256) k_gram_fix<true><<<fgrid, FIX_THREADS, 0, st>>>(x, n, d, L.nb, queue, qcount, out, fallback);
    else k_gram_fix<false><<<fgrid, FIX_THREADS, 0, st>>>(x, n, d, L.nb, queue, qcount, out, fallback);
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
