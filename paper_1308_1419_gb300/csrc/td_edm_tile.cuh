// td_edm_tile.cuh -- the register-tiled block body of the Euclidean distance map (Sec. IV of
// arXiv:1308.1419), shared by td_edm (rho 64/128) and the batched distance map.
//
// One CTA computes one rho x rho block of the packed lower triangle.  The block's rho row points
// and rho column points are staged in shared memory by asynchronous copies, KC features at a
// time, double-buffered (chunk c + 1 loads while chunk c is consumed); each thread keeps a
// TM x TN register tile of partial sums.  Two staging layouts:
//   point-major (d a multiple of 4): 16-byte copies of 4 features of one point, rows padded to
//     KC + 4 floats; a thread reads 4 features of a point per 128-bit shared load (two, and a
//     register shift, when the points start off a 16-byte boundary) and applies them to its tile
//     in feature order;
//   feature-major (any d, and the X2 form): 4-byte copies into one plane per feature, a feature
//     step being a few 128-bit shared loads of TM row and TN column values.
// With X2, two columns go through each packed sub.rn.f32x2 / fma.rn.f32x2 (sm_100+), which
// round every lane like the scalar instructions.
//
// Summation order is the one of every EDM kernel in libtd: t = x_i[k] - x_j[k],
// s = fma(t, t, s) for k = 0 .. d-1 from s = 0, then sqrtf -- so the output is bit-identical to
// the one-thread-per-element kernel.
#pragma once

#include "td_device.cuh"
#include "td_dist.cuh"

namespace td {

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero without reading.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
// 16-byte asynchronous global -> shared copy (L2 only); src_bytes = 0 writes zeros without reading.
__device__ __forceinline__ void cp_async16(float *dst, const float *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// TM x TN register tile per thread: NT = (RHO / TM) (RHO / TN) threads.  Thread (tr, tc) owns rows
// tr + (RHO / TM) a, a < TM, and columns tc + (RHO / TN) b, b < TN; consecutive threads take
// consecutive tc, so a warp reads consecutive 16-byte column granules (no bank conflicts) and,
// when RHO / TN = 32, shares one tr (row values by broadcast) and stores 32 consecutive floats of
// one packed row per instruction.
template <int RHO, int KC, int TM, int TN, bool X2>
struct EdmTile {
    static constexpr int RT = RHO / TM, CT = RHO / TN;  // row threads, column threads
    static constexpr int NT = RT * CT;
    static constexpr int LD = RHO + 4;  // padded row of a feature plane, keeps 16-byte alignment
    static constexpr int PLD = KC + 4;  // padded point row of the point-major layout (conflict-free reads)
    static constexpr int FM_STAGE = 2 * KC * LD;   // feature-major rows and columns of one chunk
    static constexpr int PM_STAGE = 2 * RHO * PLD;  // point-major rows and columns of one chunk
    static constexpr int STAGE_FLOATS = FM_STAGE > PM_STAGE ? FM_STAGE : PM_STAGE;
    static constexpr int SMEM_FLOATS = 2 * STAGE_FLOATS;  // double-buffered
    static_assert(TM % 4 == 0 && TN % 4 == 0, "TM and TN must be multiples of 4");
    static_assert(KC % 4 == 0 && (PLD * 4) % 16 == 0, "point-major rows must stay 16-byte aligned");

    // Slot of row r = tr + RT a in the row plane: thread tr reads granules tr, tr + RT, ...;
    // granule g holds a = 4 (g / RT) .. +3.  Same scheme with CT, b for columns.
    __device__ static __forceinline__ int slot_row(int r)
    {
        const int t = r % RT, a = r / RT;
        return ((a >> 2) * RT + t) * 4 + (a & 3);
    }
    __device__ static __forceinline__ int slot_col(int c)
    {
        const int t = c % CT, b = c / CT;
        return ((b >> 2) * CT + t) * 4 + (b & 3);
    }
    static constexpr bool SAME_LAYOUT = TM == TN;  // a diagonal block may read columns from the row plane

    // Issues the asynchronous copies of features [k0, k0 + kc) of the block's rows and columns.
    __device__ static __forceinline__ void stage(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0,
                                                 uint32_t j0, bool diag, uint32_t k0, int kc, float *buf)
    {
        float *sA = buf, *sB = buf + KC * LD;
        const bool need_b = !(diag && SAME_LAYOUT);
        for (int e = threadIdx.x; e < RHO * kc; e += NT) {
            const int r = e % RHO, kk = e / RHO;
            const uint32_t i = i0 + r, j = j0 + r, k = k0 + kk;
            cp_async4(sA + kk * LD + slot_row(r), i < n ? x + uint64_t(i) * d + k : x, i < n ? 4u : 0u);
            if (need_b) cp_async4(sB + kk * LD + slot_col(r), j < n ? x + uint64_t(j) * d + k : x, j < n ? 4u : 0u);
        }
        cp_async_commit();
    }

    // Point-major staging of features [k0, k0 + kc) (kc a multiple of 4).  The points sit DELTA
    // floats past a 16-byte boundary (the same for every point, d being a multiple of 4), so the
    // copies take the aligned 16-byte groups from feature k0 - DELTA on: feature k0 + kk of point r
    // lands at float DELTA + kk of row r of the row (A) or column (B) plane.  A group's bytes past
    // the point's last feature are not read (zero-filled); the DELTA floats before feature 0 of a
    // point belong to the preceding point or problem of the same input array.
    template <int DELTA>
    __device__ static __forceinline__ void stage_pm(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0,
                                                    uint32_t j0, bool diag, uint32_t k0, int kc, float *buf)
    {
        float *sA = buf, *sB = buf + RHO * PLD;
        if (DELTA == 0) {
            for (int e = threadIdx.x; e < RHO * (KC / 4); e += NT) {
                const int r = e / (KC / 4), f = e % (KC / 4);
                if (4 * f >= kc) continue;
                const uint32_t i = i0 + r, j = j0 + r, k = k0 + 4 * f;
                cp_async16(sA + r * PLD + 4 * f, i < n ? x + uint64_t(i) * d + k : x, i < n ? 16u : 0u);
                if (!diag) cp_async16(sB + r * PLD + 4 * f, j < n ? x + uint64_t(j) * d + k : x, j < n ? 16u : 0u);
            }
        } else {
            constexpr int G = KC / 4 + 1;  // 16-byte groups per point row
            const int groups = (DELTA + kc + 3) / 4;
            for (int e = threadIdx.x; e < RHO * G; e += NT) {
                const int r = e / G, f = e % G;
                if (f >= groups) continue;
                const uint32_t k = k0 + 4 * f;  // the group holds features k - DELTA .. k - DELTA + 3
                // bytes of the point from feature k - DELTA on (d + DELTA - k >= 1 for every used group)
                const uint32_t bytes = min(16u, 4 * (d + DELTA - k));
                const uint32_t i = i0 + r, j = j0 + r;
                cp_async16(sA + r * PLD + 4 * f, i < n ? x + uint64_t(i) * d + k - DELTA : x, i < n ? bytes : 0u);
                if (!diag)
                    cp_async16(sB + r * PLD + 4 * f, j < n ? x + uint64_t(j) * d + k - DELTA : x, j < n ? bytes : 0u);
            }
        }
        cp_async_commit();
    }

    // Four consecutive features of a staged point row: the aligned group at float offset `at` of
    // the plane, shifted DELTA floats into the next group.
    template <int DELTA>
    __device__ static __forceinline__ float4 features4(const float *plane, int at)
    {
        const float4 lo = *reinterpret_cast<const float4 *>(plane + at);
        if (DELTA == 0) return lo;
        const float4 hi = *reinterpret_cast<const float4 *>(plane + at + 4);
        if (DELTA == 1) return make_float4(lo.y, lo.z, lo.w, hi.x);
        if (DELTA == 2) return make_float4(lo.z, lo.w, hi.x, hi.y);
        return make_float4(lo.w, hi.x, hi.y, hi.z);
    }

    // Point-major form of run(): the same sums, each accumulator taking features in order.
    template <int DELTA>
    __device__ static void run_pm(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0, uint32_t j0,
                                  float *__restrict__ out, float *sm)
    {
        const int tid = threadIdx.x, tr = tid / CT, tc = tid % CT;
        const bool diag = i0 == j0;
        float acc[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = 0.0f;
        const uint32_t nchunks = (d + KC - 1) / KC;
        stage_pm<DELTA>(x, n, d, i0, j0, diag, 0, d < uint32_t(KC) ? int(d) : KC, sm);
        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint32_t k0 = c * KC;
            const int kc = d - k0 < uint32_t(KC) ? int(d - k0) : KC;
            if (c + 1 < nchunks) {
                const uint32_t k1 = k0 + KC;
                stage_pm<DELTA>(x, n, d, i0, j0, diag, k1, d - k1 < uint32_t(KC) ? int(d - k1) : KC,
                                sm + ((c + 1) & 1) * STAGE_FLOATS);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float *A = sm + (c & 1) * STAGE_FLOATS;
            const float *B = diag ? A : A + RHO * PLD;
            for (int kk = 0; kk < kc; kk += 4) {
                float4 av[TM];
#pragma unroll
                for (int a = 0; a < TM; ++a) av[a] = features4<DELTA>(A, (tr + RT * a) * PLD + kk);
#pragma unroll
                for (int b = 0; b < TN; ++b) {
                    const float4 bv = features4<DELTA>(B, (tc + CT * b) * PLD + kk);
                    float t[TM];  // one feature's differences for the TM rows first, then their FMAs
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].x - bv.x;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].y - bv.y;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].z - bv.z;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) t[a] = av[a].w - bv.w;
#pragma unroll
                    for (int a = 0; a < TM; ++a) acc[a][b] = fmaf(t[a], t[a], acc[a][b]);
                }
            }
            __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
        }
        store(n, i0, j0, out, acc);
    }

    // The misaligned point-major bodies, kept out of line so that each gets its own register
    // allocation instead of adding to the caller's.
    __device__ static __noinline__ void run_pm_shifted(uint32_t delta, const float *__restrict__ x, uint32_t n,
                                                       uint32_t d, uint32_t i0, uint32_t j0, float *__restrict__ out,
                                                       float *sm)
    {
        if (delta == 1) run_pm<1>(x, n, d, i0, j0, out, sm);
        else if (delta == 2) run_pm<2>(x, n, d, i0, j0, out, sm);
        else run_pm<3>(x, n, d, i0, j0, out, sm);
    }

    __device__ static __forceinline__ void store(uint32_t n, uint32_t i0, uint32_t j0, float *__restrict__ out,
                                                 const float (&acc)[TM][TN])
    {
        const int tid = threadIdx.x, tr = tid / CT, tc = tid % CT;
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            const uint32_t i = i0 + tr + RT * a;
            if (i >= n) continue;
            float *row = out + tri(i);
#pragma unroll
            for (int b = 0; b < TN; ++b) {
                const uint32_t j = j0 + tc + CT * b;
                if (j <= i) row[j] = dist_sqrt(acc[a][b]);
            }
        }
    }

    // sm: SMEM_FLOATS floats.  All NT threads of the CTA call it together.  ANY_ALIGN: the points
    // may start at any 4-byte boundary of a larger array (the batched form's concatenated input);
    // otherwise d % 4 == 0 implies 16-byte aligned points.
    template <bool ANY_ALIGN = false>
    __device__ static void run(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0, uint32_t j0,
                               float *__restrict__ out, float *sm)
    {
        if (!X2 && d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
            run_pm<0>(x, n, d, i0, j0, out, sm);
            return;
        }
        if (ANY_ALIGN && !X2 && d % 4 == 0) {
            const uint32_t delta = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(x) >> 2) & 3u;
            run_pm_shifted(delta, x, n, d, i0, j0, out, sm);
            return;
        }
        run_fm(x, n, d, i0, j0, out, sm);
    }

    // Feature-major form (any d).
    __device__ static void run_fm(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t i0, uint32_t j0,
                                  float *__restrict__ out, float *sm)
    {
        const int tid = threadIdx.x, tr = tid / CT, tc = tid % CT;
        const bool diag = i0 == j0;
        const bool b_from_a = diag && SAME_LAYOUT;
        float acc[TM][TN];
        unsigned long long acc2[TM][TN / 2];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = 0.0f;
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN / 2; ++b) acc2[a][b] = 0ull;

        const uint32_t nchunks = (d + KC - 1) / KC;
        stage(x, n, d, i0, j0, diag, 0, d < uint32_t(KC) ? int(d) : KC, sm);
        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint32_t k0 = c * KC;
            const int kc = d - k0 < uint32_t(KC) ? int(d - k0) : KC;  // features in this chunk
            if (c + 1 < nchunks) {
                const uint32_t k1 = k0 + KC;
                stage(x, n, d, i0, j0, diag, k1, d - k1 < uint32_t(KC) ? int(d - k1) : KC,
                      sm + ((c + 1) & 1) * STAGE_FLOATS);
                cp_async_wait<1>();  // chunk c has landed; chunk c + 1 may still be in flight
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float *sA = sm + (c & 1) * STAGE_FLOATS;
            const float *B = b_from_a ? sA : sA + KC * LD;
#pragma unroll 2
            for (int kk = 0; kk < kc; ++kk) {
                float av[TM], bv[TN];
#pragma unroll
                for (int h = 0; h < TM / 4; ++h) {
                    const float4 va = *reinterpret_cast<const float4 *>(sA + kk * LD + (h * RT + tr) * 4);
                    av[4 * h] = va.x; av[4 * h + 1] = va.y; av[4 * h + 2] = va.z; av[4 * h + 3] = va.w;
                }
#pragma unroll
                for (int h = 0; h < TN / 4; ++h) {
                    const float4 vb = *reinterpret_cast<const float4 *>(B + kk * LD + (h * CT + tc) * 4);
                    bv[4 * h] = vb.x; bv[4 * h + 1] = vb.y; bv[4 * h + 2] = vb.z; bv[4 * h + 3] = vb.w;
                }
                if (X2) {
                    unsigned long long b2[TN / 2];
#pragma unroll
                    for (int q = 0; q < TN / 2; ++q) b2[q] = pack2(bv[2 * q], bv[2 * q + 1]);
#pragma unroll
                    for (int a = 0; a < TM; ++a) {
                        const unsigned long long a2 = pack2(av[a], av[a]);
#pragma unroll
                        for (int q = 0; q < TN / 2; ++q) {
                            const unsigned long long t = sub_f32x2(a2, b2[q]);
                            acc2[a][q] = fma_f32x2(t, t, acc2[a][q]);
                        }
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < TM; ++a) {
                        float t[TN];  // the row's differences first, then their FMAs
#pragma unroll
                        for (int b = 0; b < TN; ++b) t[b] = av[a] - bv[b];
#pragma unroll
                        for (int b = 0; b < TN; ++b) acc[a][b] = fmaf(t[b], t[b], acc[a][b]);
                    }
                }
            }
            __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
        }
        if (X2) {
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int q = 0; q < TN / 2; ++q) unpack2(acc2[a][q], acc[a][2 * q], acc[a][2 * q + 1]);
        }
        store(n, i0, j0, out, acc);
    }
};

// The block bodies used for each block side: rho = 64 -> 4 x 4 tiles, rho = 128 -> 8 x 8 tiles,
// 256 threads each.
__host__ __device__ constexpr int edm_tile_tm(int rho) { return rho / 16; }
__host__ __device__ constexpr int edm_tile_tn(int rho) { return rho / 16; }
__host__ __device__ constexpr int edm_tile_threads(int rho) { return (rho / edm_tile_tm(rho)) * (rho / edm_tile_tn(rho)); }
// resident CTAs asked of the compiler (the 8 x 8 tile keeps its 128 registers: measured faster
// than 8 x 4 tiles with twice the warps)
__host__ __device__ constexpr int edm_tile_min_ctas(int rho) { return rho == 128 ? 2 : 4; }

template <int RHO, bool X2>
struct EdmTileFor {
    using type = EdmTile<RHO, 16, edm_tile_tm(RHO), edm_tile_tn(RHO), X2>;
};

}  // namespace td
