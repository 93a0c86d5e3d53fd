// td_api.cu -- the C ABI of libtd (declared in include/td.h): argument validation, launch
// planning and dispatch.  Nothing here allocates device memory or synchronises a stream.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "td_device.cuh"
#include "td_internal.h"

namespace td {

static thread_local char g_err[512] = "";

td_status fail(td_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

td_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TD_OK;
    return fail(TD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

td_status launch_status(const char *what) { return cuda_status(cudaGetLastError(), what); }

int sm_count()
{
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    cache[dev] = n;
    return n;
}

td_status set_dynamic_smem_once(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::unordered_map<uint64_t, size_t> done;  // key: device ^ kernel address
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t key = reinterpret_cast<uint64_t>(kernel) ^ (uint64_t(dev) << 56);
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return TD_OK;
    const td_status s = cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)),
                                    "dynamic shared memory attribute");
    if (s == TD_OK) done[key] = bytes;
    return s;
}

uint64_t persistent_ctas(const void *kernel, int threads, size_t smem, uint64_t units)
{
    static std::mutex mu;
    static std::unordered_map<uint64_t, int> cache;  // key: device ^ kernel address ^ smem
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t key = reinterpret_cast<uint64_t>(kernel) ^ (uint64_t(dev) << 56) ^ (uint64_t(smem) << 40);
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) per_sm = it->second;
    }
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm <= 0)
            per_sm = 1;
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = per_sm;
    }
    const uint64_t g = uint64_t(per_sm) * uint64_t(sm_count());
    if (units == 0) return 1;
    return units < g ? units : g;
}

static int rec_levels(uint32_t N, uint32_t rho, uint32_t &m)
{
    if (rho == 0 || N == 0 || N % rho != 0) return -1;
    int k = 0;
    uint32_t mm = N;
    while (mm % (2 * rho) == 0) {
        mm /= 2;
        ++k;
    }
    m = mm;
    return k;
}

static const uint64_t kMaxGridX = 0x7fffffffull, kMaxGridY = 65535ull;

td_status plan_strategy(td_mapping m, td_schedule s, uint32_t N, uint32_t rho, Plan &p)
{
    if (rho != 8 && rho != 16 && rho != 32 && rho != 64 && rho != 128)
        return fail(TD_ERR_INVALID_ARG, "rho must be 8, 16, 32, 64 or 128 (got %u)", rho);
    if (s != TD_SCHED_GRID && s != TD_SCHED_PERSISTENT && s != TD_SCHED_CHUNKED)
        return fail(TD_ERR_INVALID_ARG, "unknown schedule %d", int(s));
    if (s == TD_SCHED_CHUNKED && !block_strategy(m))
        return fail(TD_ERR_UNSUPPORTED, "the chunked schedule serves the block strategies LTM, BB, REC and UTM-BLOCK");
    const bool grid = s == TD_SCHED_GRID;
    p = Plan{};
    p.nb = (N + rho - 1) / rho;
    const uint64_t nb = p.nb, per = uint64_t(rho) * rho;
    p.launches = 1;
    switch (m) {
    case TD_MAP_BB:
        p.blocks = nb * nb;
        p.useful = tri(nb);
        if (nb > kMaxGridY) return fail(TD_ERR_UNSUPPORTED, "BB needs ceil(N/rho) <= 65535");
        break;
    case TD_MAP_LTM:
    case TD_MAP_LTM_X:
    case TD_MAP_LTM_N:
    case TD_MAP_LTM_N_FMA:
    case TD_MAP_LTM_R:
    case TD_MAP_UTM_BLOCK:
        p.blocks = p.useful = tri(nb);
        if (grid && p.blocks > kMaxGridX) return fail(TD_ERR_UNSUPPORTED, "LTM grid launch needs T(n) < 2^31");
        break;
    case TD_MAP_UTM:
        p.blocks = p.useful = (tri(N) + per - 1) / per;
        if (grid && p.blocks > kMaxGridX) return fail(TD_ERR_UNSUPPORTED, "UTM grid launch needs T(N)/rho^2 < 2^31");
        if (N >= (1u << 30)) return fail(TD_ERR_UNSUPPORTED, "UTM needs N < 2^30");
        break;
    case TD_MAP_RB: {
        uint32_t W, H;
        rb_dims(N, W, H);
        const uint64_t gx = (W + rho - 1) / rho, gy = (uint64_t(H) + rho - 1) / rho;
        p.blocks = p.useful = gx * gy;
        if (grid && gy > kMaxGridY) return fail(TD_ERR_UNSUPPORTED, "RB grid launch needs ceil((N+1)/rho) <= 65535");
        break;
    }
    case TD_MAP_REC: {
        uint32_t mside = 0;
        const int k = rec_levels(N, rho, mside);
        if (k < 0) return fail(TD_ERR_UNSUPPORTED, "REC needs N = m 2^k with m a multiple of rho (N=%u, rho=%u)", N, rho);
        p.rec_k = uint32_t(k);
        p.rec_m = mside;
        p.launches = uint64_t(k) + 1;
        for (int l = 1; l <= k; ++l) {
            const uint64_t sb = (N >> l) / rho, gx = N / (2 * rho);
            p.blocks += gx * sb;
            p.useful += gx * sb;
            if (grid && sb > kMaxGridY) return fail(TD_ERR_UNSUPPORTED, "REC level grid exceeds 65535 rows");
        }
        const uint64_t mb = mside / rho;
        p.blocks += (uint64_t(N) / rho) * mb;
        p.useful += (uint64_t(1) << k) * tri(mb);
        if (grid && mb > kMaxGridY) return fail(TD_ERR_UNSUPPORTED, "REC diagonal grid exceeds 65535 rows");
        break;
    }
    default:
        return fail(TD_ERR_INVALID_ARG, "unknown mapping %d", int(m));
    }
    return TD_OK;
}

td_status plan_rows(td_mapping m, uint32_t br0, uint32_t br1, Plan &p)
{
    if (m != TD_MAP_LTM && m != TD_MAP_BB) return fail(TD_ERR_UNSUPPORTED, "block-row slices serve LTM and BB");
    if (br0 >= br1 || br1 > p.nb)
        return fail(TD_ERR_INVALID_ARG, "block rows [%u, %u) must satisfy br0 < br1 <= %u", br0, br1, p.nb);
    const uint64_t useful = tri(br1) - tri(br0);
    p.sliced = true;
    p.slice_br0 = br0;
    p.slice_br1 = br1;
    if (m == TD_MAP_LTM) {
        p.slice_u0 = tri(br0);
        p.slice_units = useful;
    } else {
        p.slice_u0 = uint64_t(br0) * p.nb;
        p.slice_units = uint64_t(br1 - br0) * p.nb;
    }
    p.blocks = p.slice_units;
    p.useful = useful;
    return TD_OK;
}

static int g_options[TD_OPT_COUNT] = {0};

int option(td_option opt) { return (opt >= 0 && opt < TD_OPT_COUNT) ? g_options[opt] : 0; }

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static void fill_stats(td_launch_stats *st, const Plan &p, uint64_t ctas)
{
    if (!st) return;
    st->blocks = p.blocks;
    st->useful_blocks = p.useful;
    st->wasted_blocks = p.blocks - p.useful;
    st->launches = p.launches;
    st->ctas = ctas;
}

// The strict lower triangle of n points as the with-diagonal triangle of side n - 1.
static td_status plan_strict_blocks(td_mapping m, uint32_t n, uint32_t rho, Plan &p)
{
    if (m != TD_MAP_LTM && m != TD_MAP_BB) return fail(TD_ERR_UNSUPPORTED, "the block-mapped strict forms serve LTM and BB");
    if (rho != 8 && rho != 16 && rho != 32) return fail(TD_ERR_INVALID_ARG, "the block-mapped strict forms need rho 8, 16 or 32 (got %u)", rho);
    return plan_strategy(m, TD_SCHED_CHUNKED, n < 2 ? 0 : n - 1, rho, p);
}

// Packed offset of the first element of block row b: T(min(b rho, N)).  For rho a multiple of 8 it
// is a multiple of 4 (T(8k) = 4k (8k + 1)), so a slice of whole block rows starts and (unless it
// ends at T(N)) ends on the 16-byte grid of the whole packed array: the aligned chunks of the
// chunked kernels never cross a slice boundary, and the slice is the whole-triangle kernel
// restricted to the slice's blocks, writing through a base pointer moved back by this offset
// (integer arithmetic on the address; only addresses inside the slice are formed in the kernel).
uint64_t row_offset(uint32_t b, uint32_t rho, uint32_t N)
{
    const uint64_t r = uint64_t(b) * rho;
    return tri(r < N ? r : N);
}

template <class T>
T *slice_base(T *out, uint64_t e0)
{
    return reinterpret_cast<T *>(reinterpret_cast<uintptr_t>(out) - e0 * sizeof(T));
}

}  // namespace td

using namespace td;

extern "C" {

int td_version(void) { return 100; }

const char *td_last_error(void) { return g_err; }

uint64_t td_tri_size(uint32_t N, int with_diag)
{
    const uint64_t n = N;
    return with_diag ? n * (n + 1) / 2 : n * (n ? n - 1 : 0) / 2;
}

uint64_t td_collide_words(uint32_t n)
{
    const uint64_t nt = (uint64_t(n) + 31) / 32;
    return nt * (nt + 1) / 2 * 32;
}

td_status td_plan(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, td_launch_stats *stats)
{
    g_err[0] = 0;
    if (!stats) return fail(TD_ERR_INVALID_ARG, "stats is NULL");
    Plan p;
    const td_status st = plan_strategy(m, sched, N, rho, p);
    if (st != TD_OK) return st;
    fill_stats(stats, p, sched == TD_SCHED_GRID ? p.blocks : 0);
    return TD_OK;
}

td_status td_set_option(td_option opt, int value)
{
    g_err[0] = 0;
    if (opt < 0 || opt >= TD_OPT_COUNT) return fail(TD_ERR_INVALID_ARG, "unknown option %d", int(opt));
    if (opt == TD_OPT_PROBE_STRIP && value != 0 && (value < 128 || value > 8192 || (value & (value - 1)) != 0))
        return fail(TD_ERR_INVALID_ARG, "probe strip width must be 0 or a power of two in [128, 8192] (got %d)", value);
    if (opt == TD_OPT_EDM_F32X2 && value != 0 && value != 1)
        return fail(TD_ERR_INVALID_ARG, "TD_OPT_EDM_F32X2 takes 0 or 1 (got %d)", value);
    if (opt == TD_OPT_EDM_TMA && (value < 0 || value > 2))
        return fail(TD_ERR_INVALID_ARG, "TD_OPT_EDM_TMA takes 0, 1 or 2 (got %d)", value);
    g_options[opt] = value;
    return TD_OK;
}

int td_get_option(td_option opt) { return option(opt); }

static td_status probe_or_cover(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, uint32_t *out,
                                td_launch_stats *stats, void *stream, bool cover)
{
    g_err[0] = 0;
    if (rho > 32) return fail(TD_ERR_INVALID_ARG, "the probe needs rho 8, 16 or 32 (got %u)", rho);
    Plan p;
    td_status st = plan_strategy(m, sched, N, rho, p);
    if (st != TD_OK) return st;
    if (N == 0) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!out) return fail(TD_ERR_INVALID_ARG, "output pointer is NULL");
    if (!aligned16(out)) return fail(TD_ERR_INVALID_ARG, "output pointer must be 16-byte aligned");
    uint64_t ctas = 0;
    st = launch_probe(m, sched, N, rho, out, cover, p, static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_map_probe(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, uint32_t *out,
                       td_launch_stats *stats, void *stream)
{
    return probe_or_cover(m, sched, N, rho, out, stats, stream, false);
}

td_status td_map_cover(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, uint32_t *count, void *stream)
{
    return probe_or_cover(m, sched, N, rho, count, nullptr, stream, true);
}

td_status td_map_dummy(td_mapping m, td_schedule sched, uint32_t N, uint32_t rho, uint32_t *sink,
                       td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (rho > 32) return fail(TD_ERR_INVALID_ARG, "the dummy kernel needs rho 8, 16 or 32 (got %u)", rho);
    Plan p;
    td_status st = plan_strategy(m, sched, N, rho, p);
    if (st != TD_OK) return st;
    if (N == 0) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!sink) return fail(TD_ERR_INVALID_ARG, "sink is NULL");
    if (reinterpret_cast<uintptr_t>(sink) & 3u) return fail(TD_ERR_INVALID_ARG, "sink must be 4-byte aligned");
    uint64_t ctas = 0;
    st = launch_dummy(m, sched, N, rho, sink, p, static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_edm(td_mapping m, td_schedule sched, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out,
                 td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (ltm_variant(m)) return fail(TD_ERR_UNSUPPORTED, "the FP32 LTM variants serve the probe only");
    Plan p;
    td_status st = plan_strategy(m, sched, n, rho, p);
    if (st != TD_OK) return st;
    if (rho > 32 && !block_strategy(m))
        return fail(TD_ERR_UNSUPPORTED, "rho 64/128 (tiled EDM) supports LTM, BB, REC and UTM-BLOCK only");
    if (d == 0) return fail(TD_ERR_INVALID_ARG, "d must be at least 1");
    if (n == 0) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!x || !out) return fail(TD_ERR_INVALID_ARG, "x and out must be non-NULL");
    if (!aligned16(x) || !aligned16(out)) return fail(TD_ERR_INVALID_ARG, "x and out must be 16-byte aligned");
    uint64_t ctas = 0;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (sched == TD_SCHED_CHUNKED && rho > 32)
        return fail(TD_ERR_UNSUPPORTED, "the chunked distance map needs rho 8, 16 or 32 (rho 64/128 is the tiled body)");
    if (sched == TD_SCHED_CHUNKED)
        st = launch_edm_chunked(m, x, n, d, rho, out, p, false, cs, &ctas);
    else
        st = rho <= 32 ? launch_edm_pair(m, sched, x, n, d, rho, out, p, cs, &ctas)
                       : launch_edm_tiled(m, sched, x, n, d, rho, out, p, option(TD_OPT_EDM_F32X2) != 0, cs, &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_collide(td_mapping m, td_schedule sched, const int32_t *centers, const int32_t *radii, uint32_t n,
                     uint32_t *table, td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (m != TD_MAP_LTM && m != TD_MAP_BB && m != TD_MAP_UTM_BLOCK)
        return fail(TD_ERR_UNSUPPORTED, "td_collide supports LTM, BB and UTM-BLOCK");
    if (sched != TD_SCHED_GRID && sched != TD_SCHED_PERSISTENT)
        return fail(TD_ERR_INVALID_ARG, "td_collide takes the GRID or PERSISTENT schedule");
    const uint64_t nb = (uint64_t(n) + 63) / 64;  // the launch space: 64 x 64 blocks of four 32 x 32 bit tiles
    Plan p;
    p.nb = static_cast<uint32_t>(nb);
    p.blocks = m == TD_MAP_BB ? nb * nb : tri(nb);
    p.useful = tri(nb);
    p.launches = 1;
    if (n == 0) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!centers || !radii || !table) return fail(TD_ERR_INVALID_ARG, "centers, radii and table must be non-NULL");
    if (!aligned16(table)) return fail(TD_ERR_INVALID_ARG, "table must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(centers) | reinterpret_cast<uintptr_t>(radii)) & 3u)
        return fail(TD_ERR_INVALID_ARG, "centers and radii must be 4-byte aligned");
    if (sched == TD_SCHED_GRID && (p.blocks + 7) / 8 > kMaxGridX)
        return fail(TD_ERR_UNSUPPORTED, "grid launch too large; use the persistent schedule");
    uint64_t ctas = 0;
    const td_status st = launch_collide(m, sched, centers, radii, n, table, p, static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

uint64_t td_collide_strict_words(uint32_t n) { return (uint64_t(n) * (n ? n - 1 : 0) / 2 + 31) / 32; }

td_status td_edm_strict(const float *x, uint32_t n, uint32_t d, float *out, void *stream)
{
    g_err[0] = 0;
    if (d == 0) return fail(TD_ERR_INVALID_ARG, "d must be at least 1");
    if (n < 2) return TD_OK;
    if (uint64_t(n) * (n - 1) / 2 >= (uint64_t(1) << 40))
        return fail(TD_ERR_UNSUPPORTED, "td_edm_strict: the strict g is exact for n(n-1)/2 < 2^40");
    if (!x || !out) return fail(TD_ERR_INVALID_ARG, "x and out must be non-NULL");
    if (!aligned16(x) || !aligned16(out)) return fail(TD_ERR_INVALID_ARG, "x and out must be 16-byte aligned");
    return launch_edm_strict(x, n, d, out, static_cast<cudaStream_t>(stream));
}

td_status td_collide_strict(const int32_t *centers, const int32_t *radii, uint32_t n, uint32_t *bits, void *stream)
{
    g_err[0] = 0;
    if (n < 2) return TD_OK;
    if (uint64_t(n) * (n - 1) / 2 >= (uint64_t(1) << 40))
        return fail(TD_ERR_UNSUPPORTED, "td_collide_strict: the strict g is exact for n(n-1)/2 < 2^40");
    if (!centers || !radii || !bits) return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(centers) | reinterpret_cast<uintptr_t>(radii) | reinterpret_cast<uintptr_t>(bits)) & 3u)
        return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be 4-byte aligned");
    return launch_collide_strict(centers, radii, n, bits, static_cast<cudaStream_t>(stream));
}


td_status td_edm_strict_blocks(td_mapping m, const float *x, uint32_t n, uint32_t d, uint32_t rho, float *out,
                               td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    Plan p;
    td_status st = td::plan_strict_blocks(m, n, rho, p);
    if (st != TD_OK) return st;
    if (d == 0) return fail(TD_ERR_INVALID_ARG, "d must be at least 1");
    if (d > 8) return fail(TD_ERR_UNSUPPORTED, "td_edm_strict_blocks serves d <= 8 (got %u); use td_edm_strict", d);
    if (n < 2) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!x || !out) return fail(TD_ERR_INVALID_ARG, "x and out must be non-NULL");
    if (!aligned16(x) || !aligned16(out)) return fail(TD_ERR_INVALID_ARG, "x and out must be 16-byte aligned");
    uint64_t ctas = 0;
    st = launch_edm_chunked(m, x, n, d, rho, out, p, true, static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_collide_strict_blocks(td_mapping m, const int32_t *centers, const int32_t *radii, uint32_t n,
                                   uint32_t rho, uint32_t *bits, td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (rho == 64) {  // td_collide's 64 x 64 blocks over the n-point triangle, bits ORed into a cleared array
        if (m != TD_MAP_LTM && m != TD_MAP_BB)
            return fail(TD_ERR_UNSUPPORTED, "the block-mapped strict forms serve LTM and BB");
        const uint64_t nb = (uint64_t(n) + 63) / 64;
        Plan q;
        q.nb = static_cast<uint32_t>(nb);
        q.blocks = m == TD_MAP_BB ? nb * nb : tri(nb);
        q.useful = tri(nb);
        q.launches = 1;
        if (n < 2) {
            fill_stats(stats, q, 0);
            return TD_OK;
        }
        if (!centers || !radii || !bits) return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be non-NULL");
        if ((reinterpret_cast<uintptr_t>(centers) | reinterpret_cast<uintptr_t>(radii) | reinterpret_cast<uintptr_t>(bits)) & 3u)
            return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be 4-byte aligned");
        uint64_t ctas = 0;
        const td_status s64 = launch_collide_strict64(m, centers, radii, n, bits, td_collide_strict_words(n), q,
                                                      static_cast<cudaStream_t>(stream), &ctas);
        fill_stats(stats, q, ctas);
        return s64;
    }
    Plan p;
    td_status st = td::plan_strict_blocks(m, n, rho, p);
    if (st != TD_OK) return st;
    if (n < 2) {
        fill_stats(stats, p, 0);
        return TD_OK;
    }
    if (!centers || !radii || !bits) return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(centers) | reinterpret_cast<uintptr_t>(radii) | reinterpret_cast<uintptr_t>(bits)) & 3u)
        return fail(TD_ERR_INVALID_ARG, "centers, radii and bits must be 4-byte aligned");
    uint64_t ctas = 0;
    st = launch_collide_chunked(m, centers, radii, n, rho, bits, p, static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

size_t td_edm_gram_workspace(uint32_t n, uint32_t d) { return gram_workspace_bytes(n, d); }

td_status td_edm_gram(const float *x, uint32_t n, uint32_t d, float *out, void *ws, size_t ws_bytes, void *stream)
{
    g_err[0] = 0;
    if (n == 0) return TD_OK;
    if (d == 0 || d % 8 != 0 || d > 8192)
        return fail(TD_ERR_UNSUPPORTED, "td_edm_gram needs d a multiple of 8 in [8, 8192] (got %u)", d);
    if (!x || !out || !ws) return fail(TD_ERR_INVALID_ARG, "x, out and workspace must be non-NULL");
    if (!aligned16(x) || !aligned16(out)) return fail(TD_ERR_INVALID_ARG, "x and out must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(ws) & 1023u) return fail(TD_ERR_INVALID_ARG, "workspace must be 1024-byte aligned");
    if (ws_bytes < gram_workspace_bytes(n, d)) return fail(TD_ERR_INVALID_ARG, "workspace too small");
    return launch_gram(x, n, d, out, ws, static_cast<cudaStream_t>(stream));
}

td_status td_edm_gram_status(const void *ws, uint64_t *fallback_pairs, void *stream)
{
    g_err[0] = 0;
    if (!ws) return fail(TD_ERR_INVALID_ARG, "workspace is NULL");
    uint32_t err = 0;
    uint64_t fb = 0;
    const td_status s = read_gram_status(ws, &err, &fb, static_cast<cudaStream_t>(stream));
    if (s != TD_OK) return s;
    if (fallback_pairs) *fallback_pairs = fb;
    if (err != 0) return fail(TD_ERR_TIMEOUT, "td_edm_gram: a pipeline wait timed out (code %u)", err);
    return TD_OK;
}

td_status td_wait_status(int clear, void *stream)
{
    g_err[0] = 0;
    uint32_t code = 0;
    const td_status s = read_wait_status(clear != 0, &code, static_cast<cudaStream_t>(stream));
    if (s != TD_OK) return s;
    if (code != 0) return fail(TD_ERR_TIMEOUT, "a bounded wait of the TMA-staged distance map ran out");
    return TD_OK;
}

td_status td_wait_selftest(uint32_t arrive, uint64_t limit_ns, uint64_t *ws, uint64_t *waited_ns, void *stream)
{
    g_err[0] = 0;
    if (arrive > 1) return fail(TD_ERR_INVALID_ARG, "arrive must be 0 or 1 (got %u)", arrive);
    if (limit_ns < 1000 || limit_ns > 1000000000ull)
        return fail(TD_ERR_INVALID_ARG, "limit_ns must lie in [1e3, 1e9] (got %llu)", (unsigned long long)limit_ns);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 7u)) return fail(TD_ERR_INVALID_ARG, "ws must be non-NULL and 8-byte aligned");
    uint64_t rec[2] = {0, 0};
    const td_status s = launch_wait_selftest(arrive, limit_ns, ws, rec, static_cast<cudaStream_t>(stream));
    if (s != TD_OK) return s;
    if (waited_ns) *waited_ns = rec[1];
    if (rec[0] != 0) return fail(TD_ERR_TIMEOUT, "td_wait_selftest: the wait ran out after %llu ns", (unsigned long long)rec[1]);
    return TD_OK;
}

td_status td_map_probe_rows(td_mapping m, uint32_t N, uint32_t rho, uint32_t br0, uint32_t br1, uint32_t *out,
                            td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (rho != 8 && rho != 16 && rho != 32) return fail(TD_ERR_INVALID_ARG, "the probe needs rho 8, 16 or 32 (got %u)", rho);
    Plan p;
    td_status st = plan_strategy(m, TD_SCHED_CHUNKED, N, rho, p);
    if (st != TD_OK) return st;
    st = plan_rows(m, br0, br1, p);
    if (st != TD_OK) return st;
    if (!out) return fail(TD_ERR_INVALID_ARG, "output pointer is NULL");
    if (!aligned16(out)) return fail(TD_ERR_INVALID_ARG, "output pointer must be 16-byte aligned");
    uint64_t ctas = 0;
    st = launch_probe(m, TD_SCHED_CHUNKED, N, rho, slice_base(out, row_offset(br0, rho, N)), false, p,
                      static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_edm_rows(td_mapping m, td_schedule sched, const float *x, uint32_t n, uint32_t d, uint32_t rho,
                      uint32_t br0, uint32_t br1, float *out, td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    const bool chunked = sched == TD_SCHED_CHUNKED;
    if (chunked ? (rho != 8 && rho != 16 && rho != 32) : (rho != 64 && rho != 128))
        return fail(TD_ERR_UNSUPPORTED, "td_edm_rows: rho 8, 16 or 32 under CHUNKED, 64 or 128 under GRID/PERSISTENT");
    if (d == 0) return fail(TD_ERR_INVALID_ARG, "d must be at least 1");
    Plan p;
    td_status st = plan_strategy(m, sched, n, rho, p);
    if (st != TD_OK) return st;
    st = plan_rows(m, br0, br1, p);
    if (st != TD_OK) return st;
    if (!x || !out) return fail(TD_ERR_INVALID_ARG, "x and out must be non-NULL");
    if (!aligned16(x) || !aligned16(out)) return fail(TD_ERR_INVALID_ARG, "x and out must be 16-byte aligned");
    float *base = slice_base(out, row_offset(br0, rho, n));
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    uint64_t ctas = 0;
    st = chunked ? launch_edm_chunked(m, x, n, d, rho, base, p, false, cs, &ctas)
                 : launch_edm_tiled(m, sched, x, n, d, rho, base, p, option(TD_OPT_EDM_F32X2) != 0, cs, &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_collide_rows(td_mapping m, td_schedule sched, const int32_t *centers, const int32_t *radii, uint32_t n,
                          uint32_t br0, uint32_t br1, uint32_t *table, td_launch_stats *stats, void *stream)
{
    g_err[0] = 0;
    if (m != TD_MAP_LTM && m != TD_MAP_BB) return fail(TD_ERR_UNSUPPORTED, "td_collide_rows supports LTM and BB");
    if (sched != TD_SCHED_GRID && sched != TD_SCHED_PERSISTENT)
        return fail(TD_ERR_INVALID_ARG, "td_collide_rows takes the GRID or PERSISTENT schedule");
    Plan p;
    p.nb = static_cast<uint32_t>((uint64_t(n) + 63) / 64);
    p.launches = 1;
    td_status st = plan_rows(m, br0, br1, p);
    if (st != TD_OK) return st;
    if (!centers || !radii || !table) return fail(TD_ERR_INVALID_ARG, "centers, radii and table must be non-NULL");
    if (!aligned16(table)) return fail(TD_ERR_INVALID_ARG, "table must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(centers) | reinterpret_cast<uintptr_t>(radii)) & 3u)
        return fail(TD_ERR_INVALID_ARG, "centers and radii must be 4-byte aligned");
    if (sched == TD_SCHED_GRID && (p.blocks + 7) / 8 > kMaxGridX)
        return fail(TD_ERR_UNSUPPORTED, "grid launch too large; use the persistent schedule");
    uint64_t ctas = 0;
    const uint64_t nt = (uint64_t(n) + 31) / 32, t0 = 2 * uint64_t(br0) < nt ? 2 * uint64_t(br0) : nt;
    st = launch_collide(m, sched, centers, radii, n, slice_base(table, 32 * tri(t0)), p,
                        static_cast<cudaStream_t>(stream), &ctas);
    fill_stats(stats, p, ctas);
    return st;
}

td_status td_partition(uint32_t N, uint32_t rho, uint32_t G, uint32_t r, uint32_t *br0, uint32_t *br1, uint64_t *off0,
                       uint64_t *off1)
{
    g_err[0] = 0;
    if (rho == 0 || G == 0 || r >= G) return fail(TD_ERR_INVALID_ARG, "need rho >= 1 and rank < G");
    if (!br0 || !br1 || !off0 || !off1) return fail(TD_ERR_INVALID_ARG, "output pointers must be non-NULL");
    const uint64_t nb = (uint64_t(N) + rho - 1) / rho, total = tri(N);
    // elements in block rows [0, b)
    auto elems = [&](uint64_t b) { return tri(b * rho < N ? b * rho : N); };
    // first block row b with elems(b) >= ceil(k total / G)
    auto boundary = [&](uint64_t k) {
        if (k >= G) return nb;
        const uint64_t target = (k * total + G - 1) / G;
        uint64_t lo = 0, hi = nb;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (elems(mid) >= target) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    const uint64_t b0 = boundary(r), b1 = boundary(uint64_t(r) + 1);
    *br0 = static_cast<uint32_t>(b0);
    *br1 = static_cast<uint32_t>(b1);
    *off0 = elems(b0);
    *off1 = elems(b1);
    return TD_OK;
}

td_status td_map_dump(td_mapping m, uint32_t N, uint64_t u0, uint64_t count, uint32_t *ij, void *stream)
{
    g_err[0] = 0;
    if (m != TD_MAP_LTM && m != TD_MAP_UTM && m != TD_MAP_RB && m != TD_MAP_UTM_BLOCK && !ltm_variant(m))
        return fail(TD_ERR_UNSUPPORTED, "td_map_dump supports LTM (and its FP32 variants), UTM, UTM-BLOCK and RB");
    if (m == TD_MAP_UTM_BLOCK && (N >= (1u << 30) || u0 + count > tri(N)))
        return fail(TD_ERR_INVALID_ARG, "UTM-BLOCK block index must be < T(N)");
    if (count == 0) return TD_OK;
    if (!ij) return fail(TD_ERR_INVALID_ARG, "ij is NULL");
    if (!aligned16(ij)) return fail(TD_ERR_INVALID_ARG, "ij must be 16-byte aligned");
    if (m == TD_MAP_LTM && u0 + count > (uint64_t(1) << 40))
        return fail(TD_ERR_UNSUPPORTED, "LTM dump is exact for lambda < 2^40");
    if (ltm_variant(m) && (u0 + count < u0 || u0 + count > (uint64_t(1) << 48)))
        return fail(TD_ERR_UNSUPPORTED, "LTM variant dump covers lambda < 2^48");
    if (m == TD_MAP_UTM && (N >= (1u << 30) || u0 + count > tri(N)))
        return fail(TD_ERR_INVALID_ARG, "UTM thread index must be < T(N)");
    if (m == TD_MAP_RB) {
        if (N == 0 || u0 + count > tri(N)) return fail(TD_ERR_INVALID_ARG, "RB unit must be < T(N)");
    }
    return launch_map_dump(m, N, u0, count, ij, static_cast<cudaStream_t>(stream));
}

td_status td_ltm_variant_check(td_mapping m, uint64_t lam0, uint64_t count, uint64_t *result, void *stream)
{
    g_err[0] = 0;
    if (m != TD_MAP_LTM && !ltm_variant(m))
        return fail(TD_ERR_UNSUPPORTED, "td_ltm_variant_check takes LTM, LTM_X, LTM_N, LTM_N_FMA or LTM_R");
    if (!result) return fail(TD_ERR_INVALID_ARG, "result is NULL");
    if (!aligned16(result)) return fail(TD_ERR_INVALID_ARG, "result must be 16-byte aligned");
    if (lam0 + count < lam0 || lam0 + count > (uint64_t(1) << 48))
        return fail(TD_ERR_UNSUPPORTED, "td_ltm_check covers lambda < 2^48");
    if (count == 0) return TD_OK;
    return launch_ltm_check(m, lam0, count, result, static_cast<cudaStream_t>(stream));
}

td_status td_ltm_check(uint64_t lam0, uint64_t count, uint64_t *result, void *stream)
{
    return td_ltm_variant_check(TD_MAP_LTM, lam0, count, result, stream);
}

}  // extern "C"
