// td_tiles.cuh -- block-level launch spaces as "tile sources": a unit index u -> the block
// (bi, bj), bj <= bi, that a CTA (or warp) processes, for the strategies whose unit is a whole
// square block: g(lambda) (Sec. II-A), BB and REC (Sec. III-B).  Used by the kernels whose
// block body needs the whole tile at once (shared-memory staging, warp ballots).
#pragma once

#include "td_device.cuh"
#include "td_internal.h"

namespace td {
namespace tiles {

// Each source also answers run(u, ok, bi, bj, cap): how many consecutive units from u (at most
// cap) continue the same block row -- (bi, bj), (bi, bj+1), ... when unit u is a block (ok) --
// or are consecutive wasted units (when it is not).

// Sources with a unit offset u0 (LTM and BB) can walk a slice of their launch space: units
// u0 .. u0 + units - 1.  A slice that starts and ends on block-row boundaries covers whole block
// rows, which is how a triangle is split into the contiguous pieces of a partition.

// g(lambda): unit = block index lambda = u0 + u < T(nb).
struct Ltm {
    static constexpr bool kRuns = false;  // a unit is one block
    uint64_t units;
    uint64_t u0 = 0;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        ltm_g(u0 + u, bi, bj);
        return true;
    }
    __device__ __forceinline__ uint32_t run(uint64_t, bool, uint32_t bi, uint32_t bj, uint32_t cap) const
    {
        return min(cap, bi - bj + 1);  // the rest of block row bi
    }
};

// Block-level UTM: unit = block index lambda < T(nb), mapped by the UTM formula with the
// reciprocal-square-root trick; consecutive units continue a block row from its first block.
struct UtmBlk {
    static constexpr bool kRuns = false;  // a unit is one block
    uint64_t units;
    uint32_t nb;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        UtmBlock{nb}(u, bi, bj);
        return true;
    }
    __device__ __forceinline__ uint32_t run(uint64_t, bool, uint32_t bi, uint32_t bj, uint32_t cap) const
    {
        return min(cap, bi - bj + 1);  // the rest of block row bi
    }
};

// BB: unit = by * nb + bx = u0 + u over the n x n bounding box; blocks above the diagonal are
// skipped.
struct Bb {
    static constexpr bool kRuns = false;  // a unit is one block
    uint64_t units;
    uint32_t nb;
    uint64_t u0 = 0;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        const uint64_t v = u0 + u;
        const uint32_t by = static_cast<uint32_t>(v / nb), bx = static_cast<uint32_t>(v - uint64_t(by) * nb);
        bi = by;
        bj = bx;
        return bx <= by;
    }
    __device__ __forceinline__ uint32_t run(uint64_t, bool ok, uint32_t bi, uint32_t bj, uint32_t cap) const
    {
        return ok ? min(cap, bi - bj + 1) : min(cap, nb - bj);  // to the diagonal / to the box edge
    }
};

// REC level: squares of sb x sb blocks laid along x (gx = N / (2 rho) blocks); square q covers
// block rows [(2q+1) sb, (2q+2) sb) and block columns [2q sb, (2q+1) sb).
struct RecLevel {
    static constexpr bool kRuns = false;  // a unit is one block
    uint64_t units;
    uint32_t sb, gx;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        const uint32_t by = static_cast<uint32_t>(u / gx), bx = static_cast<uint32_t>(u - uint64_t(by) * gx);
        const uint32_t q = bx / sb, cb = bx - q * sb;
        bi = (2 * q + 1) * sb + by;
        bj = 2 * q * sb + cb;
        return true;
    }
    __device__ __forceinline__ uint32_t run(uint64_t u, bool, uint32_t, uint32_t, uint32_t cap) const
    {
        const uint32_t bx = static_cast<uint32_t>(u % gx);
        return min(cap, sb - bx % sb);  // to the right edge of the square
    }
};

// REC diagonal pass: 2^k triangles of mb x mb blocks, each covered bounding-box style.
struct RecDiag {
    static constexpr bool kRuns = false;  // a unit is one block
    uint64_t units;
    uint32_t mb, gx;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        const uint32_t by = static_cast<uint32_t>(u / gx), bx = static_cast<uint32_t>(u - uint64_t(by) * gx);
        const uint32_t t = bx / mb, lb = bx - t * mb;
        bi = t * mb + by;
        bj = t * mb + lb;
        return lb <= by;
    }
    __device__ __forceinline__ uint32_t run(uint64_t u, bool ok, uint32_t bi, uint32_t bj, uint32_t cap) const
    {
        const uint32_t lb = static_cast<uint32_t>(u % gx) % mb;
        return ok ? min(cap, bi - bj + 1) : min(cap, mb - lb);  // to the diagonal / to the triangle's edge
    }
};

// g(lambda) over runs: the block triangle cut into runs of at most R consecutive blocks of one
// block row, numbered row by row; row b holds ceil((b + 1) / R) runs.  Rows QR .. QR + R - 1 hold
// Q + 1 runs each, so the runs before row QR number R T(Q): the group Q of run v is the row of
// floor(v / R) under g (T(Q) <= floor(v / R) < T(Q + 1)), and within the group
// v - R T(Q) = (b - QR)(Q + 1) + k for the k-th run of row b, which starts at block k R.  Unit = one
// run (u0 + u = v); no run crosses the end of a row.
struct LtmRuns {
    static constexpr bool kRuns = true;
    uint64_t units;
    uint32_t R;
    uint64_t u0 = 0;
    __device__ __forceinline__ bool operator()(uint64_t u, uint32_t &bi, uint32_t &bj) const
    {
        const uint64_t v = u0 + u;
        uint32_t Q, rem;
        ltm_g(v / R, Q, rem);
        const uint64_t w = v - uint64_t(R) * tri(Q);
        bi = Q * R + static_cast<uint32_t>(w / (Q + 1));
        bj = static_cast<uint32_t>(w % (Q + 1)) * R;
        return true;
    }
    __device__ __forceinline__ uint32_t run(uint64_t, bool, uint32_t bi, uint32_t bj, uint32_t) const
    {
        return min(R, bi + 1 - bj);  // the run's blocks: R, or the rest of the row
    }
};

// Runs of LtmRuns before block row b.
__host__ __device__ __forceinline__ uint64_t ltm_runs_before(uint32_t b, uint32_t R)
{
    const uint64_t Q = b / R;
    return uint64_t(R) * tri(Q) + (b - Q * R) * (Q + 1);
}

// The LTM and BB sources of a plan: its whole launch space, or the slice of block rows it was
// planned for (td_internal.h, Plan::sliced).
inline Ltm ltm_source(const Plan &p) { return p.sliced ? Ltm{p.slice_units, p.slice_u0} : Ltm{tri(p.nb), 0}; }
// The runs of at most R blocks of the plan's block rows (the whole triangle or its slice).
inline LtmRuns ltm_runs_source(const Plan &p, uint32_t R)
{
    const uint32_t b0 = p.sliced ? p.slice_br0 : 0u, b1 = p.sliced ? p.slice_br1 : p.nb;
    const uint64_t r0 = ltm_runs_before(b0, R);
    return LtmRuns{ltm_runs_before(b1, R) - r0, R, r0};
}
inline Bb bb_source(const Plan &p)
{
    return p.sliced ? Bb{p.slice_units, p.nb, p.slice_u0} : Bb{uint64_t(p.nb) * p.nb, p.nb, 0};
}

}  // namespace tiles
}  // namespace td
