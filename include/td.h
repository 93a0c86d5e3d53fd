/*
 * td.h -- C ABI of libtd, the GB300 (sm_103a) implementation of the block-level
 * triangular-domain mapping g(lambda) of Navarro & Hitschfeld, "Improving the GPU space of
 * computation under triangular domain problems" (arXiv:1308.1419), fused with the kernels
 * it drives, plus the four strategies the paper compares it with.
 *
 * Common conventions
 *   - T(m) = m(m+1)/2.  A lower triangle of side N *with* its diagonal is stored packed,
 *     row-major: element (i, j), 0 <= j <= i < N, lives at offset T(i) + j (Sec. II-A,
 *     Eq. (matrix_indexing) numbers blocks the same way).
 *   - Device pointers are plain CUDA device addresses owned by the caller; every buffer the
 *     library writes must be 16-byte aligned.  The library allocates no device memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is asynchronous
 *     with respect to the host: it validates its arguments, enqueues its kernel(s) on
 *     `stream` and returns.  Nothing synchronises.
 *   - Errors: argument errors return TD_ERR_INVALID_ARG or TD_ERR_UNSUPPORTED before any
 *     launch; a CUDA error at launch returns TD_ERR_CUDA.  td_last_error() gives the message
 *     of the last failing call on the calling thread.  Nothing aborts or traps.
 *   - rho is the side of a square block of the domain ("dimensional blocksize", Sec. II-A):
 *     n = ceil(N / rho) blocks per side.
 */
#ifndef TD_H
#define TD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TD_OK = 0,
    TD_ERR_INVALID_ARG = 1,
    TD_ERR_UNSUPPORTED = 2,
    TD_ERR_CUDA = 3,
    TD_ERR_TIMEOUT = 4
} td_status;

/* Mapping strategies (Sec. III-B): bounding box, upper-triangular mapping (Avril et al.),
 * rectangular box (Jung et al.), recursive partition (Ries et al.), and the paper's
 * lower-triangular mapping g(lambda) (Sec. II-A).
 * TD_MAP_LTM evaluates i = floor(sqrt(1/4 + 2 lambda) - 1/2) with an FP32 reciprocal-square-root
 * estimate and an exact integer +-1 fix-up (exact for lambda < 2^40).  The LTM_* values are
 * the single-precision evaluations Sec. III-A times in its dummy kernel, with no fix-up; with
 * x = 1/4 + 2 lambda rounded to FP32 and every operation rounded to nearest (a fused
 * multiply-add, where written, rounded once):
 *   TD_MAP_LTM_X  i = trunc(sqrt(x) - 1/2)                      (LTM-X);
 *   TD_MAP_LTM_N  y = bits^-1(0x5f3759df - (bits(x) >> 1)), three steps y = y (3/2 - ((x/2) y) y),
 *                 i = trunc(x y - 1/2 + 1e-4)                   (LTM-N, the paper's epsilon);
 *   TD_MAP_LTM_R  i = trunc(x rsqrtf(x) - 1/2 + 1e-4)           (LTM-R, the paper's epsilon);
 *   TD_MAP_LTM_N_FMA  LTM-N as a CUDA compiler contracts it by default: each step rounds
 *                 t = (x/2) y and takes y = y fma(-t, y, 3/2); i = trunc(fma(x, y, -1/2) + 1e-4)
 *                 (exact for lambda < T(1920), i.e. N <= 30720 at rho = 16, as Sec. III-A states);
 * all with j = lambda - T(i).  They are exact only while FP32 resolves the row boundaries
 * (td_ltm_variant_check finds where each stops); they serve td_map_probe, td_map_cover and
 * td_map_dump under GRID or PERSISTENT, and every other call rejects them (TD_ERR_UNSUPPORTED).
 * TD_MAP_UTM_BLOCK is the conjecture that closes the paper: the UTM formula applied to block
 * indices lambda < T(nb) over the block triangle (rows reversed into the lower triangle, so
 * consecutive lambda continue a block row), its square root taken as y rsqrtf(y), with UTM's
 * integer fix-up; it is a block strategy like TD_MAP_LTM and is accepted wherever LTM is. */
typedef enum {
    TD_MAP_BB = 0,
    TD_MAP_UTM = 1,
    TD_MAP_RB = 2,
    TD_MAP_REC = 3,
    TD_MAP_LTM = 4,
    TD_MAP_LTM_X = 5,
    TD_MAP_LTM_N = 6,
    TD_MAP_LTM_R = 7,
    TD_MAP_UTM_BLOCK = 8,
    TD_MAP_LTM_N_FMA = 9
} td_mapping;

/* How the strategy's blocks are issued.
 *   GRID: one CTA per block of the strategy's launch space, one element per thread, as in
 *     the paper.
 *   PERSISTENT: a grid of (SM count x resident CTAs per SM) CTAs walks the same launch space
 *     with a grid-stride loop, one element per thread.
 *   CHUNKED (probe only; block strategies LTM, BB, REC): persistent warps walk the rows of the
 *     strategy's blocks and write the packed output in aligned 16-byte chunks; a chunk belongs
 *     to the block holding its first element, so each element is still written exactly once. */
typedef enum {
    TD_SCHED_GRID = 0,
    TD_SCHED_PERSISTENT = 1,
    TD_SCHED_CHUNKED = 2
} td_schedule;

/* Launch-space accounting of one call (Sec. II-A: BB wastes n(n-1)/2 blocks, g(lambda)
 * needs only n(n+1)/2).  `blocks` counts the strategy's blocks over all its launches,
 * `useful_blocks` those holding at least one in-domain element, `wasted_blocks` the rest,
 * `launches` the kernel launches, `ctas` the CTAs actually started (equal to `blocks`
 * under TD_SCHED_GRID). */
typedef struct {
    uint64_t blocks;
    uint64_t useful_blocks;
    uint64_t wasted_blocks;
    uint64_t launches;
    uint64_t ctas;
} td_launch_stats;

/* Library-wide options (process global; set them before launching work). */
typedef enum {
    /* 1: the tiled distance-map kernels use the packed FP32 pair instructions
     * (sub.rn.f32x2 / fma.rn.f32x2); 0 (default): scalar FP32, measured no slower on GB300.
     * Both round identically, so the output does not depend on it. */
    TD_OPT_EDM_F32X2 = 0,
    /* Strip width of the CHUNKED probe schedule: the elements of one packed row a warp writes per
     * strip of consecutive blocks.  0 (default): chosen per launch from its size (wider strips
     * write longer contiguous runs; narrower ones balance better when there are few blocks);
     * otherwise a power of two in [128, 8192].  Output does not depend on it. */
    TD_OPT_PROBE_STRIP = 1,
    /* How the register-tiled distance map (td_edm, rho 64 / 128, and its slices) stages the
     * block's points when d % 4 == 0 and x is 16-byte aligned: tensor-memory-accelerator box loads
     * (cp.async.bulk.tensor, 16 features x rho points, issued by one thread into a two-stage
     * mbarrier ring) or per-thread asynchronous 16-byte copies.  0 (default): TMA for d >= 64
     * (measured a few per cent faster there; at d = 4 a box moves four times the bytes used and
     * is slower); 1: TMA wherever possible; 2: per-thread copies only.  Same sums, bit-identical
     * output. */
    TD_OPT_EDM_TMA = 2,
    TD_OPT_COUNT = 3
} td_option;

/* ------------------------------------------------------------------ host-only helpers */

/* Library version (major * 10000 + minor * 100 + patch). */
int td_version(void);

/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
const char *td_last_error(void);

/* Sets / reads a library option.  Unknown option or a value outside the option's range:
 * TD_ERR_INVALID_ARG, option unchanged (td_get_option of an unknown option: 0). */
td_status td_set_option(td_option opt, int value);
int td_get_option(td_option opt);

/* T(N) = N(N+1)/2 if with_diag, else N(N-1)/2 (Sec. II-A). */
uint64_t td_tri_size(uint32_t N, int with_diag);

/* Words of the collision table for n spheres: T(ceil(n/32)) * 32 (see td_collide). */
uint64_t td_collide_words(uint32_t n);

/* Fills *stats with the launch space td_map_probe / td_edm (m, sched, N, rho, ...) would use,
 * without touching a GPU.  rho in {8, 16, 32, 64, 128}.  REC needs N to be a positive multiple of rho
 * (Sec. III-B: N = m 2^k, m a multiple of rho; k is taken as large as possible), else
 * TD_ERR_UNSUPPORTED. */
td_status td_plan(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, td_launch_stats *stats);

/* Host-only partition of a triangle of side N (block side rho) over G ranks: rank r gets the
 * contiguous block rows [*br0, *br1) -- the g(lambda) blocks lambda in [T(*br0), T(*br1)) -- and
 * with them the contiguous slice [*off0, *off1) of the packed output.  Boundaries are the first
 * block rows holding at least ceil(k T(N) / G) elements, so slices are balanced to within one
 * block row; the G slices are disjoint and cover [0, T(N)).  Every (i, j) output is
 * independent, so sharded ranks need no exchange beyond, optionally, gathering the slices. */
td_status td_partition(uint32_t N, uint32_t rho, uint32_t G, uint32_t r, uint32_t *br0, uint32_t *br1, uint64_t *off0,
                       uint64_t *off1);

/* Slices of whole block rows, the units of a partition over several GPUs (td_partition).  Block
 * rows [br0, br1) of a triangle of side N with block side rho hold the g(lambda) blocks
 * lambda in [T(br0), T(br1)) (Sec. II-A, Eq. (matrix_indexing): block rows are contiguous in
 * lambda) and, in the packed output, the contiguous elements [e0, e1) with
 * e0 = T(min(br0 rho, N)), e1 = T(min(br1 rho, N)).  Each call below computes only its slice: it
 * issues the slice's blocks (m = TD_MAP_LTM: lambda in [T(br0), T(br1)); TD_MAP_BB: the bounding
 * box rows br0 .. br1 - 1) and writes out[e - e0] for every element e of the slice, exactly the
 * values the whole-triangle call writes there -- so slices [b_0, b_1), [b_1, b_2), ... written one
 * after another into consecutive buffers reproduce the whole packed output byte for byte.
 * rho is a multiple of 8, so e0 and (unless e1 = T(N)) e1 are multiples of 4 and the chunked
 * kernels' aligned 16-byte chunks never straddle two slices.  0 <= br0 < br1 <= ceil(N / rho),
 * else TD_ERR_INVALID_ARG; other mappings: TD_ERR_UNSUPPORTED.  out: device, e1 - e0 elements,
 * 16-byte aligned.  stats (host, may be NULL): the slice's blocks.  Asynchronous on `stream`.
 *
 * td_map_probe_rows: the probe of td_map_probe under TD_SCHED_CHUNKED; rho in {8, 16, 32}.
 * td_edm_rows: the distance map of td_edm (same summation order, bit-identical values) under
 *   TD_SCHED_CHUNKED with rho in {8, 16, 32} and d <= 8, or under TD_SCHED_GRID / PERSISTENT with
 *   rho in {64, 128} (the register-tiled body); x as in td_edm (all n points).
 * td_collide_rows: the collision table of td_collide over its block rows [br0, br1) (rho = 64: 64
 *   spheres, two rows of 32 x 32 bit tiles, per block row): the tile rows [t0, t1),
 *   t0 = min(2 br0, nt), t1 = min(2 br1, nt), nt = ceil(n / 32), i.e. the words [32 T(t0), 32 T(t1))
 *   of the whole table, written to table[w - 32 T(t0)]; 0 <= br0 < br1 <= ceil(n / 64); sched GRID
 *   or PERSISTENT. */
td_status td_map_probe_rows(td_mapping m, uint32_t N, uint32_t rho, uint32_t br0, uint32_t br1, uint32_t *out,
                            td_launch_stats *stats, void *stream);
td_status td_edm_rows(td_mapping m, td_schedule sched, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                      uint32_t br0, uint32_t br1, float *out, td_launch_stats *stats, void *stream);
td_status td_collide_rows(td_mapping m, td_schedule sched, const int32_t *centers, const int32_t *radii, uint32_t n,
                          uint32_t br0, uint32_t br1, uint32_t *table, td_launch_stats *stats, void *stream);

/* ------------------------------------------------------------------ mapping kernels */

/* Probe: the paper's dummy kernel (Sec. III-A, Sec. IV test (1)) made to write the whole
 * domain.  Every in-domain thread of strategy m writes
 *     out[T(i) + j] = splitmix32((uint32_t)(i * N + j)),   0 <= j <= i < N,
 * where splitmix32(x) = fmix32(x + 0x9E3779B9) and fmix32 is the MurmurHash3 32-bit
 * finaliser.  out: device, uint32[T(N)], 16-byte aligned.  rho in {8, 16, 32} (rho x rho
 * threads per block; UTM uses rho^2-thread blocks over its thread index).  stats: host,
 * may be NULL.  N = 0 is a no-op. */
td_status td_map_probe(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho,
                       uint32_t *out, td_launch_stats *stats, void *stream);

/* Euclidean distance map (Sec. IV): for every 0 <= j <= i < n,
 *     out[T(i) + j] = sqrt(sum_{k<d} (x[i][k] - x[j][k])^2)     in FP32,
 * evaluated as t = x[i][k] - x[j][k], s = fma(t, t, s) for k = 0 .. d-1 from s = 0, then the
 * hardware square root sqrt.approx.f32 (within 2 units in the last place of the correctly
 * rounded one) -- the same order and square root in every kernel, so every strategy, schedule
 * and rho gives bit-identical output.  x: device, float[n][d] row-major, 16-byte aligned;
 * out: device, float[T(n)], 16-byte aligned.  d >= 1.
 * rho in {8, 16, 32}, sched GRID or PERSISTENT: rho x rho threads per block, one element per
 *   thread, every strategy (the paper's EDM kernel).
 * rho in {8, 16, 32}, sched CHUNKED (TD_MAP_LTM, TD_MAP_BB, TD_MAP_REC; d <= 8, else
 *   TD_ERR_UNSUPPORTED): the same blocks walked by warps in strips of consecutive blocks of a
 *   block row, column points staged in shared memory, aligned 16-byte stores -- the form for
 *   few features, where the map is store-bound.
 * rho in {64, 128}, sched GRID or PERSISTENT: one 256-thread CTA per rho x rho block with
 *   shared-memory coordinate tiles and register tiles, for large d; TD_MAP_LTM, TD_MAP_BB and
 *   TD_MAP_REC only (CHUNKED: TD_ERR_UNSUPPORTED).
 * stats: host, may be NULL.  n = 0 is a no-op. */
td_status td_edm(td_mapping m, td_schedule sched, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                 float *out, td_launch_stats *stats, void *stream);

/* td-problems without the diagonal (Eq. (theorem_nodiag)), mapped at the element level: the
 * strict lower triangle i > j of side n has n(n-1)/2 elements, packed row-major at
 * k = i(i-1)/2 + j, and a thread finds the (i, j) of its k with the strict g,
 *     i = floor(sqrt(1/4 + 2k) + 1/2),  j = k - i(i-1)/2
 * (the printed j = k - i(i+1)/2 would give j = -1 at k = 0), evaluated as an FP32 reciprocal-
 * square-root estimate with an exact integer +-1 row fix-up.  n(n-1)/2 < 2^40.
 *
 * td_edm_strict: out[k] = D(i, j) in the summation order of td_edm (so out[k] equals td_edm's
 *   out[T(i) + j] bit for bit).  x: device, float[n][d], 16-byte aligned; out: device,
 *   float[n(n-1)/2], 16-byte aligned; d >= 1.  n < 2: no-op.
 * td_collide_strict: bit k (word k / 32, bit k % 32, LSB first) of bits is 1 iff spheres i and
 *   j collide, decided exactly (same predicate and input domain as td_collide); the unused
 *   bits of the last word are 0.  centers: device int32[n][3]; radii: device int32[n];
 *   bits: device uint32[td_collide_strict_words(n)]; all 4-byte aligned.  n < 2: no-op. */
uint64_t td_collide_strict_words(uint32_t n); /* ceil(n(n-1)/2 / 32) */
td_status td_edm_strict(const float *x, uint32_t n, uint32_t d, float *out, void *stream);
td_status td_collide_strict(const int32_t *centers, const int32_t *radii, uint32_t n, uint32_t *bits, void *stream);

/* The same two strict outputs (same layout, bit-identical) mapped at the block level, the fast
 * form: the pairs (i, j), j < i < n, packed at i(i-1)/2 + j, are the with-diagonal packed
 * triangle of side n - 1 whose row i' holds the pairs of point i' + 1 (pair (i' + 1, j) at
 * T(i') + j, j <= i').  Its rho x rho blocks are issued by g(lambda) (m = TD_MAP_LTM) or by BB
 * (TD_MAP_BB) under the chunked schedule: warps walk strips of consecutive blocks of a block row
 * and write aligned 16-byte chunks (distances) or whole 32-bit words (collision bits, one
 * __ballot_sync per word).  rho: 8, 16 or 32.  stats (host, may be NULL): the block counts of
 * the triangle of side n - 1.
 * td_collide_strict_blocks also takes rho = 64: the 64 x 64 blocks of td_collide over the
 * triangle of the n points (its kernel and predicate, issued by g(lambda) or BB, persistent),
 * after clearing the bit array on `stream`; each block's nonzero 32-pair row pieces are ORed
 * into the one or two words they straddle (atomically: pieces of neighbouring blocks share
 * words).  The fast form when collisions are sparse; stats: the blocks of that triangle.
 * td_edm_strict_blocks: 1 <= d <= 8 (larger d: td_edm_strict); x and out 16-byte aligned.
 * td_collide_strict_blocks: centers, radii and bits 4-byte aligned.
 * n < 2: no-op.  Other errors as td_edm_strict / td_collide_strict. */
td_status td_edm_strict_blocks(td_mapping m, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out,
                               td_launch_stats *stats, void *stream);
td_status td_collide_strict_blocks(td_mapping m, const int32_t *centers, const int32_t *radii, uint32_t n,
                                   uint32_t rho, uint32_t *bits, td_launch_stats *stats, void *stream);

/* Collision table (collision detection is a td-problem named in the abstract and Sec. I):
 * spheres i > j collide iff |c_i - c_j|^2 <= (r_i + r_j)^2, decided exactly.  The table is
 * bit-packed in 32 x 32 bit-tiles over the tile triangle of side nt = ceil(n / 32): tile
 * (ti, tj), tj <= ti, is tile number T(ti) + tj and owns words [32 (T(ti)+tj), +32); word r of
 * it holds row i = 32 ti + r and its bit c (LSB first) holds column j = 32 tj + c.  Bits with
 * i <= j, i >= n or j >= n are 0.  Every word of the table is written.
 * The launch space is the triangle of 64 x 64 blocks (four tiles each, three on the diagonal),
 * m: TD_MAP_LTM (blocks issued by g(lambda)), TD_MAP_BB (their bounding box) or TD_MAP_UTM_BLOCK;
 * sched: GRID or PERSISTENT.  One warp computes one block; stats count these blocks.
 * centers: device, int32[n][3]; radii: device, int32[n]; any int32 values (the test is exact
 * for all of them: 32-bit arithmetic for blocks whose coordinates lie in [-2^30, 2^30) and radii
 * in [0, 2^14], 64/128-bit arithmetic otherwise; a negative radius enters only through
 * (r_i + r_j)^2).  Both 4-byte aligned.  table: device, uint32[td_collide_words(n)], 16-byte
 * aligned.  n = 0: no-op. */
td_status td_collide(td_mapping m, td_schedule sched, const int32_t *centers, const int32_t *radii, uint32_t n,
                     uint32_t *table, td_launch_stats *stats, void *stream);

/* ------------------------------------------------------------------ Gram-form distance map */

/* Bytes of device workspace td_edm_gram needs: a status block, n FP32 squared norms, a BF16
 * copy of the n x d points, and the recompute queue (room for 1/32 of the pairs of every
 * 128 x 128 block, 8 bytes a pair, with a counter per 32-row quarter of a block). */
size_t td_edm_gram_workspace(uint32_t n, uint32_t d);

/* Euclidean distance map in Gram form on the tensor cores: D(i,j)^2 = |x_i|^2 + |x_j|^2 -
 * 2 <x_i, x_j>, the inner products from BF16 copies of the points accumulated in FP32
 * (tcgen05.mma, 128 x 128 blocks issued by g(lambda) over the block triangle), the squared
 * norms in FP32 from the FP32 points.  A pair whose D^2 falls below 1e-2 (|x_i|^2 + |x_j|^2)
 * (the diagonal included) is recomputed in the direct FP32 form sum_k (x_i[k] - x_j[k])^2, since
 * the Gram subtraction cancels there.  Other pairs carry the BF16 error of the inner product.
 * Same output layout as td_edm.  x: device, float[n][d], d a multiple of 8 in [8, 8192], 16-byte
 * aligned; out: device, float[T(n)], 16-byte aligned; ws: device, td_edm_gram_workspace(n, d)
 * bytes, 1024-byte aligned.  Asynchronous; the pipeline's waits are bounded, and a wait that
 * runs out is reported by td_edm_gram_status. */
td_status td_edm_gram(const float *x, uint32_t n, uint32_t d, float *out, void *ws, size_t ws_bytes, void *stream);

/* Synchronises `stream` and reads the status block of the last td_edm_gram that used ws:
 * TD_ERR_TIMEOUT if a pipeline wait ran out, else TD_OK; *fallback_pairs (host, may be NULL)
 * gets the number of pairs recomputed in the direct form. */
td_status td_edm_gram_status(const void *ws, uint64_t *fallback_pairs, void *stream);

/* Synchronises `stream` and reports whether a bounded wait of a kernel without a workspace (the
 * TMA staging of td_edm, TD_OPT_EDM_TMA) ran out since the last call with clear = 1: TD_ERR_TIMEOUT
 * if one did (that call's output is incomplete), else TD_OK.  clear: 1 resets the record. */
td_status td_wait_status(int clear, void *stream);

/* Self-test of the failure path of the bounded waits (the Gram pipeline's mbarrier waits): one
 * thread initialises an mbarrier expecting one arrival, arrives on it if `arrive` is 1, then
 * waits for its first phase with the same bounded wait the pipeline uses, limited to limit_ns.
 * With arrive = 0 nothing completes the phase, so the wait must run out; the kernel records that
 * and returns (no trap, no unbounded spin) and the context stays usable.
 * arrive: 0 or 1; limit_ns: in [1e3, 1e9]; ws: device, uint64[2], 8-byte aligned, scratch;
 * waited_ns: host, may be NULL, gets the wait's duration read from the device's global timer.
 * Synchronises `stream`.  Returns TD_ERR_TIMEOUT if the wait ran out, TD_OK if it completed,
 * TD_ERR_INVALID_ARG for arguments outside the ranges above (nothing launched). */
td_status td_wait_selftest(uint32_t arrive, uint64_t limit_ns, uint64_t *ws, uint64_t *waited_ns, void *stream);

/* ------------------------------------------------------------------ batched distance maps */

/* Launch configuration of the batched distance map: block side rho (64 or 128) and CTAs per
 * SM of the persistent grid (0 = as many as fit). */
typedef struct {
    uint32_t rho;
    uint32_t ctas_per_sm;
} td_batched_config;

/* Bytes of device workspace td_edm_batched* needs for nprob problems (plan: prefix sums of
 * the block counts and per-problem offsets). */
size_t td_edm_batched_workspace(uint32_t nprob);

/* Batched Euclidean distance maps: nprob independent problems, problem p with n[p] >= 1
 * points of d[p] >= 1 features.  x_cat: device, the row-major n[p] x d[p] float blocks
 * concatenated in problem order; out_cat: device, the packed triangles T(n[p]) concatenated in
 * problem order (each exactly as td_edm would write it -- bit-identical).  All blocks of all
 * problems form one launch space (problem p owns [P[p], P[p] + T(ceil(n[p]/rho))), P the
 * prefix sum, problems laid heaviest first); one persistent launch walks it, finding each
 * block's problem by binary search over P and its position by g(lambda) (Sec. II-A).
 * n, d: host arrays.  ws: device workspace of td_edm_batched_workspace(nprob) bytes, 16-byte
 * aligned (x_cat and out_cat too).  cfg: NULL = {128, 0} (the faster block side on mixed batches
 * of 3 to 64 features; td_edm_batched_autotune chooses per batch).  The plan upload uses a
 * pageable host-to-device copy (it orders with `stream` but cannot be graph-captured); use
 * td_edm_batched_plan + td_edm_batched_run to capture the launch. */
td_status td_edm_batched(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat, float *out_cat,
                         void *ws, size_t ws_bytes, const td_batched_config *cfg, td_launch_stats *stats,
                         void *stream);

/* Split form of td_edm_batched: _plan writes the plan for block side rho into ws and returns the
 * launch-space size in *total_blocks (host); _run is a single kernel launch reading that plan
 * (capturable in a CUDA graph; the plan must stay in ws). */
td_status td_edm_batched_plan(uint32_t nprob, const uint32_t *n, const uint32_t *d, uint32_t rho, void *ws,
                              size_t ws_bytes, uint64_t *total_blocks, void *stream);
td_status td_edm_batched_run(uint32_t nprob, uint32_t rho, uint64_t total_blocks, const float *x_cat, float *out_cat,
                             const void *ws, uint32_t ctas_per_sm, void *stream);

/* Allocation-free form of td_edm_batched, for callers that cannot allocate device memory: a
 * serving process whose memory pool already holds all the device memory it may use, a plugin
 * hosted by a framework that owns every device allocation, or a latency-bound loop where an
 * allocation (and the device synchronisation it can bring) is not acceptable.  The paper has no
 * counterpart; this is a packaging of td_edm_batched.
 * Instead of a caller workspace, the launch plan lives in a fixed array of device memory inside
 * the library, sized for at most 1024 problems (about 40 KB; every GPU that loads the library
 * holds it until the process exits).  The call performs no cudaMalloc, cudaFree or other
 * allocation, on the device or the host.  More than 1024 problems: TD_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture begins.  Every call
 * rewrites the whole plan (nothing in the array needs clearing) and the array keeps the last
 * call's plan.  All calls share the one array: calls whose work overlaps on the GPU (different
 * streams) race on it, so issue them on one stream.  The plan upload is a pageable host-to-device
 * copy, which orders with `stream` and returns once the host image has been read.
 * Other arguments and the result are those of td_edm_batched (bit-identical output). */
td_status td_edm_batched_noalloc(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat,
                                 float *out_cat, const td_batched_config *cfg, td_launch_stats *stats, void *stream);

/* Autotuner: times every rho in {64, 128} and CTAs-per-SM in {max, 1, 2, 3, 4} (one warm-up and
 * three timed runs each, CUDA events on `stream`; synchronises), returns the fastest in *best and
 * its time per run in *best_ms (host, may be NULL), and leaves ws planned for it.  out_cat is
 * written (with the correct result). */
td_status td_edm_batched_autotune(uint32_t nprob, const uint32_t *n, const uint32_t *d, const float *x_cat,
                                  float *out_cat, void *ws, size_t ws_bytes, td_batched_config *best, float *best_ms,
                                  void *stream);

/* Coverage check of a strategy: every in-domain thread adds 1 to count[T(i) + j]
 * (atomically).  A bijective mapping leaves every entry at exactly its previous value + 1.
 * Same arguments and launch space as td_map_probe; count: device, uint32[T(N)].  Under
 * TD_SCHED_CHUNKED the chunked probe's own walk adds 1 to each element it would write (chunk
 * ownership, runs and the chunks that cross row ends included), so a double or missed write of
 * that schedule shows as a count other than 1. */
td_status td_map_cover(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho,
                       uint32_t *count, void *stream);

/* The dummy kernel of Sec. III-A (the timing of a mapping alone): the launch of td_map_probe,
 * each in-domain thread computing its (i, j) through strategy m, and a store to sink[0] guarded
 * by i + j == 2^32 - 1, which no in-domain pair meets, so the mapping cannot be optimised away
 * and nothing is written.  (The paper stores i + j to one fixed address; on this GPU that
 * would serialise every thread on one memory line.)  sched: GRID or PERSISTENT; every mapping,
 * the LTM_* variants included.  sink: device, uint32[1], 4-byte aligned, left unchanged. */
td_status td_map_dummy(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, uint32_t *sink,
                       td_launch_stats *stats, void *stream);

/* Dump of a mapping function for unit indices u0 .. u0+count-1 into ij (device,
 * uint32[2*count], pairs (i, j)):
 *   TD_MAP_LTM: unit = block index lambda, (i, j) = g(lambda) of Eq. (theorem); N unused.
 *   TD_MAP_LTM_X, TD_MAP_LTM_N, TD_MAP_LTM_N_FMA, TD_MAP_LTM_R: the same with that FP32 evaluation
 *               (lambda < 2^48).
 *   TD_MAP_UTM_BLOCK: unit = block index lambda < T(N), (i, j) = its block for a block triangle of
 *               side N (N < 2^30).
 *   TD_MAP_UTM: unit = thread index k < T(N), (i, j) = the UTM pair of Sec. III-B for the
 *               strict upper triangle of side N+1, rows reversed into the lower triangle:
 *               i = N - a, j = b - a - 1.
 *   TD_MAP_RB:  unit = y * W + x over the RB thread rectangle (W = N/2, H = N+1 for even N;
 *               W = N/2 + 1, H = N for odd N).
 * Other strategies: TD_ERR_UNSUPPORTED. */
td_status td_map_dump(td_mapping m, uint32_t N, uint64_t u0, uint64_t count, uint32_t *ij,
                      void *stream);

/* Exhaustive self-check of the fast g(lambda) (FP32 reciprocal square root plus an integer
 * +-1 fix-up) over lambda in [lam0, lam0 + count), lam0 + count <= 2^48: counts the lambda
 * whose (i, j) breaks T(i) <= lambda < T(i+1).  The fix-up is proven sufficient for
 * lambda < 2^40; beyond that this call measures where it stops being enough.
 * result: device, uint64[2], must hold {0, UINT64_MAX} on entry;
 * on exit result[0] = number of failures, result[1] = smallest failing lambda. */
td_status td_ltm_check(uint64_t lam0, uint64_t count, uint64_t *result, void *stream);

/* The same count for any evaluation of g: m in {TD_MAP_LTM, TD_MAP_LTM_X, TD_MAP_LTM_N,
 * TD_MAP_LTM_N_FMA, TD_MAP_LTM_R} (td_ltm_check is m = TD_MAP_LTM).  Same result convention and range limit;
 * other m: TD_ERR_UNSUPPORTED. */
td_status td_ltm_variant_check(td_mapping m, uint64_t lam0, uint64_t count, uint64_t *result, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TD_H */
