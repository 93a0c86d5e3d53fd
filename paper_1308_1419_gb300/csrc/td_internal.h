// td_internal.h -- host-side declarations shared by the translation units of libtd.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "td.h"

namespace td {

// Records a formatted message for td_last_error() and returns `st`.
td_status fail(td_status st, const char *fmt, ...);
// Maps a CUDA error to TD_ERR_CUDA (recording `what`), or TD_OK.
td_status cuda_status(cudaError_t e, const char *what);
// Checks cudaGetLastError() after a launch.
td_status launch_status(const char *what);

// SM count of the current device (cached per device).
int sm_count();
// Persistent grid for a kernel: SM count x resident CTAs per SM (cached per device/kernel),
// capped at `units` (at least 1).
uint64_t persistent_ctas(const void *kernel, int threads, size_t smem, uint64_t units);
// Raises a kernel's dynamic shared memory limit to `bytes` on the current device, once: later
// calls (a stream capture among them) make no CUDA call.
td_status set_dynamic_smem_once(const void *kernel, size_t bytes);

// Launch space of a strategy (host closed forms; mirrors what the launchers issue).
struct Plan {
    uint64_t blocks = 0, useful = 0, launches = 0, ctas = 0;
    uint32_t nb = 0;          // blocks per side, ceil(N / rho)
    uint32_t rec_k = 0;       // REC levels
    uint32_t rec_m = 0;       // REC diagonal triangle side
    // a slice of the launch space (LTM and BB): units [slice_u0, slice_u0 + slice_units), the
    // blocks of block rows [br0, br1) (plan_rows)
    bool sliced = false;
    uint64_t slice_u0 = 0, slice_units = 0;
    uint32_t slice_br0 = 0, slice_br1 = 0;
};
td_status plan_strategy(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, Plan &p);
// Narrows a plan of LTM or BB to block rows [br0, br1), 0 <= br0 < br1 <= nb: LTM's units
// [T(br0), T(br1)), BB's [br0 nb, br1 nb); blocks / useful / wasted become the slice's own.
td_status plan_rows(td_mapping m, uint32_t br0, uint32_t br1, Plan &p);

// Launchers (stream-ordered, no synchronisation).
td_status launch_probe(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, uint32_t *out,
                       bool cover, const Plan &p, cudaStream_t st, uint64_t *ctas);
// Shape of a chunked launch.  W: the widest run (consecutive blocks of one block row), in elements
// of one packed row: the widest power of two in [min(256, wauto), wauto] leaving at least four
// runs of W per resident warp, or the TD_OPT_PROBE_STRIP value (capped at wlimit); never below rho.
// rcap = W / rho units.  S: units per strip (one warp's contiguous share): rcap while there are at
// least four strips per resident warp, else the launch split evenly, ceil(units / warps) -- with
// only a few strips per warp, whole strips would leave most warps idle for the last round.
struct ChunkPlan {
    uint32_t W, rcap, S;
};
ChunkPlan chunked_plan(uint64_t units, uint32_t rho, uint64_t resident_warps, uint32_t wauto, uint32_t wlimit);
td_status launch_edm_strict(const float *x, uint32_t n, uint32_t d, float *out, cudaStream_t st);
td_status launch_collide_strict(const int32_t *c, const int32_t *r, uint32_t n, uint32_t *bits, cudaStream_t st);
// strict: the strict lower triangle of the n points, as the packed triangle of side n - 1 whose
// row i' pairs point i' + 1 with j <= i' (p planned for side n - 1; LTM and BB).
td_status launch_edm_chunked(td_mapping m, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out,
                             const Plan &p, bool strict, cudaStream_t st, uint64_t *ctas);
// Strict-lower collision bits under the chunked schedule of the block strategies (LTM, BB), p
// planned for side n - 1.
td_status launch_collide_chunked(td_mapping m, const int32_t *c, const int32_t *r, uint32_t n, uint32_t rho,
                                 uint32_t *bits, const Plan &p, cudaStream_t st, uint64_t *ctas);
// Strict-lower collision bits (`words` of them) by the 64 x 64 blocks of td_collide over the
// n-point triangle, p planned as for td_collide: the array is cleared, then each block's nonzero
// row pieces are ORed in (LTM and BB).
td_status launch_collide_strict64(td_mapping m, const int32_t *c, const int32_t *r, uint32_t n, uint32_t *bits,
                                  uint64_t words, const Plan &p, cudaStream_t st, uint64_t *ctas);
td_status launch_edm_pair(td_mapping m, td_schedule s, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                          float *out, const Plan &p, cudaStream_t st, uint64_t *ctas);
td_status launch_edm_tiled(td_mapping m, td_schedule s, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                           float *out, const Plan &p, bool x2, cudaStream_t st, uint64_t *ctas);
// p: the tile plan (nb = ceil(n / 32) tiles per side, possibly sliced to tile rows).
td_status launch_collide(td_mapping m, td_schedule s, const int32_t *c, const int32_t *r, uint32_t n,
                         uint32_t *table, const Plan &p, cudaStream_t st, uint64_t *ctas);
// Plan of the batched distance map, as td_edm_batched_run reads it from device memory: a
// BatchHeader, the nprob + 1 exclusive prefix sums (uint64) of the problems' block counts
// T(ceil(n/rho)) in launch-space order, then one BatchMeta per problem in that order.
struct BatchMeta {     // one problem, in launch-space order
    uint64_t x_off;    // first float of the problem's points in x_cat
    uint64_t out_off;  // first float of the problem's packed triangle in out_cat
    uint32_t n, d;
    uint32_t pad0, pad1;
};
static_assert(sizeof(BatchMeta) == 32, "BatchMeta layout");
struct BatchHeader {   // first 64 bytes of the plan
    uint64_t magic;
    uint64_t total_blocks;
    uint32_t nprob, rho;
    uint32_t pad[10];
};
static_assert(sizeof(BatchHeader) == 64, "BatchHeader layout");
constexpr uint64_t kBatchMagic = 0x7464626174636831ull;  // "tdbatch1"
size_t batched_workspace_bytes(uint32_t nprob);
// Launch-space weight of a problem (block count times features): problems are laid heaviest first.
uint64_t batched_weight(uint32_t n, uint32_t d, uint32_t rho);
// Writes the plan image (batched_workspace_bytes(nprob) bytes at img, zeroed by the caller) for
// the problems taken in launch-space order order[0 .. nprob); returns the total block count.
// x_off / out_off: scratch of nprob entries each.  Allocates nothing.
uint64_t batched_fill_image(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho, const uint32_t *order,
                            uint64_t *x_off, uint64_t *out_off, unsigned char *img);
size_t gram_workspace_bytes(uint32_t n, uint32_t d);
// A 2-D tiled tensor map over a row-major array of `outer` rows of `inner` elements, rows
// row_bytes apart (a multiple of 16), boxes of box_inner x box_outer elements, zero fill outside.
td_status encode_tiled_2d(CUtensorMap *map, CUtensorMapDataType type, const void *base, uint64_t inner, uint64_t outer,
                          uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swizzle);
// Device word recording a bounded wait that ran out in a kernel without a workspace (the TMA
// staging of the register-tiled distance map); read and cleared by td_wait_status.
td_status read_wait_status(bool clear, uint32_t *code, cudaStream_t st);
td_status launch_gram(const float *x, uint32_t n, uint32_t d, float *out, void *ws, cudaStream_t st);
td_status read_gram_status(const void *ws, uint32_t *err, uint64_t *fallback, cudaStream_t st);
// One bounded mbarrier wait (arrive: whether its phase completes); copies {ran out, ns} to out
// after synchronising st.
td_status launch_wait_selftest(uint32_t arrive, uint64_t limit_ns, uint64_t *rec, uint64_t out[2], cudaStream_t st);
// Library options (td_set_option).
int option(td_option opt);
td_status launch_map_dump(td_mapping m, uint32_t N, uint64_t u0, uint64_t count, uint32_t *ij,
                          cudaStream_t st);
td_status launch_dummy(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, uint32_t *sink, const Plan &p,
                       cudaStream_t st, uint64_t *ctas);
td_status launch_ltm_check(td_mapping m, uint64_t lam0, uint64_t count, uint64_t *result, cudaStream_t st);
// The FP32 evaluations of g timed in Sec. III-A (probe, cover and dump only).
inline bool ltm_variant(td_mapping m)
{
    return m == TD_MAP_LTM_X || m == TD_MAP_LTM_N || m == TD_MAP_LTM_N_FMA || m == TD_MAP_LTM_R;
}
// Strategies whose unit is a whole square block and that have a tile source (td_tiles.cuh).
inline bool block_strategy(td_mapping m)
{
    return m == TD_MAP_LTM || m == TD_MAP_BB || m == TD_MAP_REC || m == TD_MAP_UTM_BLOCK;
}

}  // namespace td
