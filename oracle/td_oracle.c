/*
 * td_oracle.c -- plain, slow, obviously-correct CPU oracle for the triangular-domain
 * (td-problem) mappings and kernels of Navarro & Hitschfeld, "Improving the GPU space of
 * computation under triangular domain problems" (arXiv:1308.1419).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code.  It is used
 * by tests/, by __graft_entry__.smoke() (to check one small GPU run) and by the cpu_baseline
 * / reference leg of bench.py.  It shares no source, header, table or helper with the CUDA
 * library under paper_1308_1419_gb300/csrc, and it never reads a value produced there.
 *
 * Conventions (fixed by the paper, Sec. II-A, Eq. (matrix_indexing)):
 *   T(m) = m(m+1)/2.  A lower triangle of side N including the diagonal is stored packed,
 *   row-major: element (i, j), 0 <= j <= i < N, lives at offset T(i) + j.  The same numbering
 *   is the paper's block numbering: block lambda = T(i) + j.
 *
 * Arithmetic: integers are exact (64-bit, or 128-bit where sums of squared int32 differences
 * exceed 64 bits); real values are computed in double.
 * Every function is a direct statement of its definition; nothing is blocked, fused or
 * reordered.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

/* ---------------------------------------------------------------- basic helpers */

/* T(m) = m(m+1)/2: size of a triangle of side m including the diagonal
 * (Sec. II-A: "n(n+1)/2 blocks are sufficient to cover the problem domain"). */
uint64_t or_tri(uint64_t m) { return m * (m + 1) / 2; }

/* Exact floor(sqrt(x)) for any uint64 x: the textbook digit-by-digit (base 4) method.
 * Used so that the oracle's g(lambda) involves no floating point at all. */
uint64_t or_isqrt(uint64_t x)
{
    uint64_t rem = x, root = 0, bit = (uint64_t)1 << 62;
    while (bit > rem) bit >>= 2;
    while (bit != 0) {
        if (rem >= root + bit) {
            rem -= root + bit;
            root = (root >> 1) + bit;
        } else {
            root >>= 1;
        }
        bit >>= 2;
    }
    return root;
}

/* ---------------------------------------------------------------- g(lambda), Sec. II-A */

/* Eq. (theorem): g(lambda) = (i, j) with i = floor(sqrt(1/4 + 2 lambda) - 1/2) and
 * j = lambda - i(i+1)/2.  sqrt(1/4 + 2 lambda) - 1/2 = (sqrt(8 lambda + 1) - 1) / 2 (the
 * proof's positive root of x^2 + x - 2 lambda = 0), and for an integer c and real y,
 * floor((y - c)/2) = floor((floor(y) - c)/2), so i = (isqrt(8 lambda + 1) - 1) / 2 exactly.
 * Valid for 8 lambda + 1 < 2^64. */
void or_ltm(uint64_t lam, uint32_t *i, uint32_t *j)
{
    uint64_t r = or_isqrt(8 * lam + 1);
    uint64_t ii = (r - 1) / 2;
    *i = (uint32_t)ii;
    *j = (uint32_t)(lam - ii * (ii + 1) / 2);
}

/* Eq. (theorem_nodiag), strict lower triangle (j < i): i = floor(sqrt(1/4 + 2 lambda) + 1/2).
 * Row i of the strict triangle starts at i(i-1)/2, so j = lambda - i(i-1)/2.  (The printed
 * j = lambda - i(i+1)/2 would give j = -1 at lambda = 0; the strict triangle's own row start
 * is the reading taken here.) */
void or_ltm_nodiag(uint64_t lam, uint32_t *i, uint32_t *j)
{
    uint64_t r = or_isqrt(8 * lam + 1);
    uint64_t ii = (r + 1) / 2;
    *i = (uint32_t)ii;
    *j = (uint32_t)(lam - ii * (ii - 1) / 2);
}

void or_ltm_many(const uint64_t *lam, uint64_t count, uint32_t *ij)
{
    for (uint64_t q = 0; q < count; ++q) or_ltm(lam[q], &ij[2 * q], &ij[2 * q + 1]);
}

void or_ltm_nodiag_many(const uint64_t *lam, uint64_t count, uint32_t *ij)
{
    for (uint64_t q = 0; q < count; ++q) or_ltm_nodiag(lam[q], &ij[2 * q], &ij[2 * q + 1]);
}

/* ---------------------------------------------------------------- FP32 evaluations of g (Sec. III-A)
 * Sec. III-A times ways of evaluating i = floor(sqrt(1/4 + 2 lambda) - 1/2) in single precision
 * in its dummy kernel.  Two of them are fully specified by IEEE single-precision arithmetic and
 * are written out here (this file is built with -ffp-contract=off, and C evaluates float
 * expressions in float on the targets it is built for, so every operation below rounds to
 * nearest exactly once):
 *   variant 1 (LTM-X): x = 0.25f + 2.0f * (float)lambda;  i = trunc(sqrtf(x) - 0.5f);
 *   variant 2 (LTM-N): the same x; y0 = the float whose bits are 0x5f3759df - (bits(x) >> 1)
 *     (the bit-level inverse-square-root estimate analysed by Lomont), three Newton steps
 *     y = y * (1.5f - ((0.5f * x) * y) * y), then i = trunc((x * y - 0.5f) + 1e-4f): the paper
 *     adds epsilon = 1e-4 to the computation of i here to repair the rounding at row starts.
 * j = lambda - T(i).  The third variant (LTM-R: x * rsqrtf(x) - 0.5 + 1e-4) depends on the
 * device's reciprocal-square-root approximation and has no host definition.
 *
 * The paper does not say how its compiler evaluated these expressions.  CUDA's compiler fuses a
 * product feeding an addition or subtraction into one fused multiply-add (rounded once) unless
 * told not to, so the two variants are also given in that contracted form:
 *   variant 3 (LTM-N, contracted): the same seed; each Newton step rounds t = (0.5f * x) * y, then
 *     y = y * fmaf(-t, y, 1.5f) (the product t * y is not rounded before the subtraction); then
 *     i = trunc(fmaf(x, y, -0.5f) + 1e-4f).
 *   variant 4 (LTM-X, contracted): x = fmaf(2.0f, (float)lambda, 0.25f); i = trunc(sqrtf(x) - 0.5f).
 *     2 * (float)lambda is exact in binary floating point, so this x equals variant 1's and the two
 *     variants agree everywhere; it is kept so that the claim is checked rather than assumed.
 * fmaf is C99's fused multiply-add, correctly rounded. */

static float bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* The inverse-square-root estimate refined by `steps` Newton steps (variant 2's core). */
float or_fast_rsqrt(float x, int steps)
{
    const float h = 0.5f * x;
    float y = bits_to_float(0x5f3759dfu - (float_to_bits(x) >> 1));
    for (int k = 0; k < steps; ++k) y = y * (1.5f - (h * y) * y);
    return y;
}

static uint32_t trunc_u32(float v) { return v <= 0.0f ? 0u : (uint32_t)v; }

/* The inverse-square-root estimate refined by `steps` Newton steps, each in variant 3's
 * contracted form. */
float or_fast_rsqrt_fma(float x, int steps)
{
    const float h = 0.5f * x;
    float y = bits_to_float(0x5f3759dfu - (float_to_bits(x) >> 1));
    for (int k = 0; k < steps; ++k) {
        const float t = h * y;
        y = y * fmaf(-t, y, 1.5f);
    }
    return y;
}

void or_ltm_variant(int variant, uint64_t lam, uint32_t *i, uint32_t *j)
{
    const float x = 0.25f + 2.0f * (float)lam;
    uint32_t r = 0;
    if (variant == 1) r = trunc_u32(sqrtf(x) - 0.5f);
    if (variant == 2) r = trunc_u32((x * or_fast_rsqrt(x, 3) - 0.5f) + 1e-4f);
    if (variant == 3) r = trunc_u32(fmaf(x, or_fast_rsqrt_fma(x, 3), -0.5f) + 1e-4f);
    if (variant == 4) r = trunc_u32(sqrtf(fmaf(2.0f, (float)lam, 0.25f)) - 0.5f);
    *i = r;
    *j = (uint32_t)(lam - or_tri(r));
}

/* Smallest lambda in [lam0, lam1) whose variant (i, j) differs from the exact g(lambda), or
 * lam1 if there is none: a plain scan. */
uint64_t or_ltm_variant_first_fail(int variant, uint64_t lam0, uint64_t lam1)
{
    for (uint64_t lam = lam0; lam < lam1; ++lam) {
        uint32_t i, j, ei, ej;
        or_ltm_variant(variant, lam, &i, &j);
        or_ltm(lam, &ei, &ej);
        if (i != ei || j != ej) return lam;
    }
    return lam1;
}

/* ---------------------------------------------------------------- UTM, Sec. III-B */

/* UTM (Avril et al.), as given in Sec. III-B: for a strict upper triangle of side n and a
 * thread index k in [0, n(n-1)/2), a = floor((-(2n+1) + sqrt(4n^2 - 4n - 8k + 1)) / -2) and
 * b = (a+1) + k - (a-1)(2n-a)/2, with 1 <= a < b <= n.  Here the floor is taken exactly:
 * with D = 4n^2 - 4n - 8k + 1 and c = 2n+1, (-c + sqrt D)/(-2) = (c - sqrt D)/2 and
 * floor((c - y)/2) = floor((c - ceil(y))/2) for real y. */
void or_utm_ab(uint64_t n, uint64_t k, uint64_t *a, uint64_t *b)
{
    uint64_t D = 4 * n * n - 4 * n - 8 * k + 1;
    uint64_t r = or_isqrt(D);
    uint64_t ceil_sqrt = (r * r == D) ? r : r + 1;
    uint64_t aa = (2 * n + 1 - ceil_sqrt) / 2;
    *a = aa;
    *b = (aa + 1) + k - (aa - 1) * (2 * n - aa) / 2;
}

/* The definition UTM computes: the k-th pair (a, b), 1 <= a < b <= n, in row-major order. */
void or_utm_enum(uint64_t n, uint64_t *ab)
{
    uint64_t k = 0;
    for (uint64_t a = 1; a < n; ++a)
        for (uint64_t b = a + 1; b <= n; ++b) {
            ab[2 * k] = a;
            ab[2 * k + 1] = b;
            ++k;
        }
}

/* UTM used for a lower triangle of side N with its diagonal (Sec. III-B: an upper mapping
 * also serves lower domains): the strict upper triangle of side n = N + 1 has exactly
 * T(N) pairs; pair (a, b) is sent to row i = N - a, column j = b - a - 1 (rows reversed, so
 * consecutive k stay on consecutive j of one row). */
void or_utm_lower(uint32_t N, uint64_t k, uint32_t *i, uint32_t *j)
{
    uint64_t a, b;
    or_utm_ab((uint64_t)N + 1, k, &a, &b);
    *i = (uint32_t)((uint64_t)N - a);
    *j = (uint32_t)(b - a - 1);
}

void or_utm_lower_many(uint32_t N, const uint64_t *k, uint64_t count, uint32_t *ij)
{
    for (uint64_t q = 0; q < count; ++q) or_utm_lower(N, k[q], &ij[2 * q], &ij[2 * q + 1]);
}

/* ---------------------------------------------------------------- RB, Sec. III-B */

/* RB (Jung et al.) as a thread rectangle.  Even N: H = N + 1 rows, W = N/2 columns; a thread
 * (x, y) below the diagonal (x < y) takes i = y - 1, j = x; on/above it takes
 * i = N - 1 - y, j = N - 1 - x (the folded part, columns j >= N/2).  Odd N: partition at
 * m = floor(N/2): H = N rows, W = m + 1 columns; y >= x takes (y, x), else (N-1-y, N-x). */
void or_rb_dims(uint32_t N, uint64_t *W, uint64_t *H)
{
    if (N % 2 == 0) { *W = N / 2; *H = (uint64_t)N + 1; }
    else            { *W = N / 2 + 1; *H = N; }
}

void or_rb_map(uint32_t N, uint64_t x, uint64_t y, uint32_t *i, uint32_t *j)
{
    if (N % 2 == 0) {
        if (x < y) { *i = (uint32_t)(y - 1); *j = (uint32_t)x; }
        else       { *i = (uint32_t)(N - 1 - y); *j = (uint32_t)(N - 1 - x); }
    } else {
        if (y >= x) { *i = (uint32_t)y; *j = (uint32_t)x; }
        else        { *i = (uint32_t)(N - 1 - y); *j = (uint32_t)(N - x); }
    }
}

/* ---------------------------------------------------------------- REC, Sec. III-B */

/* REC (Ries et al.): N = m 2^k with m a multiple of rho; k is taken as large as possible.
 * Returns k (and m), or -1 if N is not a positive multiple of rho. */
int or_rec_levels(uint32_t N, uint32_t rho, uint32_t *m)
{
    if (rho == 0 || N == 0 || N % rho != 0) return -1;
    int k = 0;
    uint32_t mm = N;
    while (mm % (2 * rho) == 0) { mm /= 2; ++k; }
    *m = mm;
    return k;
}

/* ---------------------------------------------------------------- coverage / launch space */

enum { OR_BB = 0, OR_UTM = 1, OR_RB = 2, OR_REC = 3, OR_LTM = 4, OR_UTM_BLOCK = 8 };

static void cover_one(uint32_t *count, uint32_t N, uint64_t i, uint64_t j, uint64_t *outside)
{
    if (j <= i && i < N) count[or_tri(i) + j] += 1;
    else ++*outside;
}

/* Walk every thread each strategy launches for a td-problem of side N with rho x rho blocks
 * (Sec. II-A: n = ceil(N / rho) blocks per side; Sec. III-B: the four compared strategies)
 * and add 1 to count[T(i) + j] for every thread that lands inside the triangle.
 * stats[0] = blocks launched, stats[1] = blocks with at least one in-domain thread,
 * stats[2] = kernel launches, stats[3] = in-domain thread hits.
 * Returns 0, or -1 for an unsupported (strategy, N, rho). */
int or_cover(int strategy, uint32_t N, uint32_t rho, uint32_t *count, uint64_t stats[4])
{
    uint64_t nb = (N + (uint64_t)rho - 1) / rho;
    uint64_t launched = 0, useful = 0, launches = 1, hits = 0, outside = 0;
    memset(count, 0, sizeof(uint32_t) * or_tri(N));
    if (strategy == OR_BB) {
        /* n x n grid; a block with B_x > B_y returns at once; inside diagonal blocks the
         * thread test keeps j <= i (Sec. III-B). */
        for (uint64_t by = 0; by < nb; ++by)
            for (uint64_t bx = 0; bx < nb; ++bx) {
                ++launched;
                if (bx > by) continue;
                uint64_t before = outside;
                for (uint64_t ty = 0; ty < rho; ++ty)
                    for (uint64_t tx = 0; tx < rho; ++tx)
                        cover_one(count, N, by * rho + ty, bx * rho + tx, &outside);
                if (outside - before < (uint64_t)rho * rho) ++useful;
            }
    } else if (strategy == OR_LTM) {
        /* n(n+1)/2 blocks, block lambda -> g(lambda) = (block row, block column). */
        for (uint64_t lam = 0; lam < or_tri(nb); ++lam) {
            uint32_t bi, bj;
            or_ltm(lam, &bi, &bj);
            ++launched;
            uint64_t before = outside;
            for (uint64_t ty = 0; ty < rho; ++ty)
                for (uint64_t tx = 0; tx < rho; ++tx)
                    cover_one(count, N, (uint64_t)bi * rho + ty, (uint64_t)bj * rho + tx, &outside);
            if (outside - before < (uint64_t)rho * rho) ++useful;
        }
    } else if (strategy == OR_UTM_BLOCK) {
        /* block-level UTM (the paper's closing conjecture): block lambda < T(nb) -> the UTM
         * pair of the block triangle of side nb, rows reversed into the lower triangle. */
        for (uint64_t lam = 0; lam < or_tri(nb); ++lam) {
            uint32_t bi, bj;
            or_utm_lower((uint32_t)nb, lam, &bi, &bj);
            ++launched;
            uint64_t before = outside;
            for (uint64_t ty = 0; ty < rho; ++ty)
                for (uint64_t tx = 0; tx < rho; ++tx)
                    cover_one(count, N, (uint64_t)bi * rho + ty, (uint64_t)bj * rho + tx, &outside);
            if (outside - before < (uint64_t)rho * rho) ++useful;
        }
    } else if (strategy == OR_UTM) {
        /* thread-level: block b of rho^2 threads, thread k = b rho^2 + t, k < T(N). */
        uint64_t per = (uint64_t)rho * rho, total = or_tri(N);
        uint64_t nblk = (total + per - 1) / per;
        for (uint64_t b = 0; b < nblk; ++b) {
            ++launched;
            uint64_t before = outside;
            for (uint64_t t = 0; t < per; ++t) {
                uint64_t k = b * per + t;
                if (k >= total) { ++outside; continue; }
                uint32_t i, j;
                or_utm_lower(N, k, &i, &j);
                cover_one(count, N, i, j, &outside);
            }
            if (outside - before < per) ++useful;
        }
    } else if (strategy == OR_RB) {
        uint64_t W, H;
        or_rb_dims(N, &W, &H);
        uint64_t gx = (W + rho - 1) / rho, gy = (H + rho - 1) / rho;
        for (uint64_t by = 0; by < gy; ++by)
            for (uint64_t bx = 0; bx < gx; ++bx) {
                ++launched;
                uint64_t before = outside;
                for (uint64_t ty = 0; ty < rho; ++ty)
                    for (uint64_t tx = 0; tx < rho; ++tx) {
                        uint64_t x = bx * rho + tx, y = by * rho + ty;
                        if (x >= W || y >= H) { ++outside; continue; }
                        uint32_t i, j;
                        or_rb_map(N, x, y, &i, &j);
                        cover_one(count, N, i, j, &outside);
                    }
                if (outside - before < (uint64_t)rho * rho) ++useful;
            }
    } else if (strategy == OR_REC) {
        uint32_t m;
        int k = or_rec_levels(N, rho, &m);
        if (k < 0) return -1;
        launches = (uint64_t)k + 1;
        /* level l = 1..k: 2^(l-1) full squares of side s = N / 2^l, square q covering rows
         * [(2q+1)s, (2q+2)s) and columns [2qs, (2q+1)s); one launch per level. */
        for (int l = 1; l <= k; ++l) {
            uint64_t s = (uint64_t)N >> l;
            uint64_t sq = (uint64_t)1 << (l - 1);
            for (uint64_t q = 0; q < sq; ++q)
                for (uint64_t r = 0; r < s; r += rho)
                    for (uint64_t c = 0; c < s; c += rho) {
                        ++launched;
                        uint64_t before = outside;
                        for (uint64_t ty = 0; ty < rho; ++ty)
                            for (uint64_t tx = 0; tx < rho; ++tx)
                                cover_one(count, N, (2 * q + 1) * s + r + ty, 2 * q * s + c + tx, &outside);
                        if (outside - before < (uint64_t)rho * rho) ++useful;
                    }
        }
        /* final pass: the 2^k diagonal triangles of side m, each covered BB-style. */
        uint64_t nt = (uint64_t)1 << k, mb = m / rho;
        for (uint64_t t = 0; t < nt; ++t)
            for (uint64_t by = 0; by < mb; ++by)
                for (uint64_t bx = 0; bx < mb; ++bx) {
                    ++launched;
                    if (bx > by) continue;
                    uint64_t before = outside;
                    for (uint64_t ty = 0; ty < rho; ++ty)
                        for (uint64_t tx = 0; tx < rho; ++tx)
                            cover_one(count, N, t * m + by * rho + ty, t * m + bx * rho + tx, &outside);
                    if (outside - before < (uint64_t)rho * rho) ++useful;
                }
    } else {
        return -1;
    }
    for (uint64_t p = 0; p < or_tri(N); ++p) hits += count[p];
    stats[0] = launched;
    stats[1] = useful;
    stats[2] = launches;
    stats[3] = hits;
    return 0;
}

/* ---------------------------------------------------------------- probe (dummy kernel) */

/* The probe hash: a golden-ratio increment followed by the MurmurHash3 32-bit finaliser,
 * all in wrap-around uint32 arithmetic. */
uint32_t or_splitmix32(uint32_t x)
{
    uint32_t z = x + 0x9E3779B9u;
    z = (z ^ (z >> 16)) * 0x85EBCA6Bu;
    z = (z ^ (z >> 13)) * 0xC2B2AE35u;
    z = z ^ (z >> 16);
    return z;
}

/* The probe (the paper's dummy kernel of Sec. III-A / IV made to write the whole domain):
 * for every (i, j), j <= i < N, out[T(i) + j] = splitmix32((uint32)(i N + j)).
 * Rows [i0, i1) are written; out[0] is element (i0, 0). */
void or_probe(uint32_t N, uint32_t i0, uint32_t i1, uint32_t *out)
{
    uint64_t base = or_tri(i0);
    for (uint64_t i = i0; i < i1; ++i)
        for (uint64_t j = 0; j <= i; ++j)
            out[or_tri(i) + j - base] = or_splitmix32((uint32_t)(i * (uint64_t)N + j));
}

/* ---------------------------------------------------------------- EDM, Sec. IV */

/* Euclidean distance map (Sec. IV): f(i, j) = sqrt(sum_k (a_i^k - a_j^k)^2), for every
 * j <= i < n; x is n x d row-major float32, arithmetic in double.  Rows [i0, i1) are
 * written; out[0] is (i0, 0). */
void or_edm(const float *x, uint32_t n, uint32_t d, uint32_t i0, uint32_t i1, double *out)
{
    (void)n;
    uint64_t base = or_tri(i0);
    for (uint64_t i = i0; i < i1; ++i)
        for (uint64_t j = 0; j <= i; ++j) {
            double s = 0.0;
            for (uint64_t k = 0; k < d; ++k) {
                double diff = (double)x[i * d + k] - (double)x[j * d + k];
                s += diff * diff;
            }
            out[or_tri(i) + j - base] = sqrt(s);
        }
}

/* The same definition at a list of (i, j) pairs. */
void or_edm_pairs(const float *x, uint32_t d, const uint32_t *ii, const uint32_t *jj,
                  uint64_t count, double *out)
{
    for (uint64_t q = 0; q < count; ++q) {
        double s = 0.0;
        for (uint64_t k = 0; k < d; ++k) {
            double diff = (double)x[(uint64_t)ii[q] * d + k] - (double)x[(uint64_t)jj[q] * d + k];
            s += diff * diff;
        }
        out[q] = sqrt(s);
    }
}

/* ---------------------------------------------------------------- collision table */

/* Collision detection, a td-problem named in the abstract and Sec. I: spheres i and j
 * (i != j) collide iff |c_i - c_j|^2 <= (r_i + r_j)^2, evaluated exactly.  With int32 inputs a
 * coordinate difference reaches 2^32 and the sum of three squares 3 * 2^64, beyond int64, so
 * the squares are summed in unsigned 128-bit integers. */
int or_collides(const int32_t *c, const int32_t *r, uint32_t i, uint32_t j)
{
    unsigned __int128 s = 0;
    for (int k = 0; k < 3; ++k) {
        int64_t dk = (int64_t)c[3 * (uint64_t)i + k] - c[3 * (uint64_t)j + k];
        uint64_t ak = (uint64_t)(dk < 0 ? -dk : dk);
        s += (unsigned __int128)ak * ak;
    }
    int64_t R = (int64_t)r[i] + r[j];
    return s <= (unsigned __int128)(R < 0 ? -R : R) * (unsigned __int128)(R < 0 ? -R : R);
}

/* Bit position of strict-lower pair (i, j), j < i, in the packed table: the table is
 * split into 32 x 32 bit-tiles over the tile triangle of side ceil(n / 32); tile
 * (bi, bj), bj <= bi, is tile number T(bi) + bj and holds 32 words, word r for row
 * i = 32 bi + r, bit c (LSB first) for column j = 32 bj + c. */
void or_collide_bitpos(uint32_t i, uint32_t j, uint64_t *word, uint32_t *bit)
{
    uint64_t bi = i / 32, bj = j / 32;
    *word = (or_tri(bi) + bj) * 32 + (i % 32);
    *bit = j % 32;
}

uint64_t or_collide_words(uint32_t n) { return or_tri((n + 31) / 32) * 32; }

/* Full table for n spheres: every strict pair j < i < n evaluated one by one. */
void or_collide(const int32_t *c, const int32_t *r, uint32_t n, uint32_t *table)
{
    memset(table, 0, sizeof(uint32_t) * or_collide_words(n));
    for (uint32_t i = 1; i < n; ++i)
        for (uint32_t j = 0; j < i; ++j)
            if (or_collides(c, r, i, j)) {
                uint64_t w;
                uint32_t b;
                or_collide_bitpos(i, j, &w, &b);
                table[w] |= (uint32_t)1 << b;
            }
}

/* ---------------------------------------------------------------- td-problems without the diagonal
 * The strict lower triangle i > j of side n, packed row-major: pair (i, j) at k = i(i-1)/2 + j
 * (the numbering of Eq. (theorem_nodiag), with the strict row start).  Plain double loops. */

/* EDM over the strict triangle: out[k] = sqrt(sum (x_i - x_j)^2) in double. */
void or_edm_strict(const float *x, uint32_t n, uint32_t d, double *out)
{
    uint64_t k = 0;
    for (uint64_t i = 1; i < n; ++i)
        for (uint64_t j = 0; j < i; ++j, ++k) {
            double s = 0.0;
            for (uint64_t f = 0; f < d; ++f) {
                double diff = (double)x[i * d + f] - (double)x[j * d + f];
                s += diff * diff;
            }
            out[k] = sqrt(s);
        }
}

/* Collision bits over the strict triangle: bit k % 32 (LSB first) of word k / 32 is the exact
 * predicate for the pair at k; the words must hold ceil(n(n-1)/2 / 32) entries. */
void or_collide_strict(const int32_t *c, const int32_t *r, uint32_t n, uint32_t *bits)
{
    uint64_t total = (uint64_t)n * (n ? n - 1 : 0) / 2;
    memset(bits, 0, sizeof(uint32_t) * ((total + 31) / 32));
    uint64_t k = 0;
    for (uint32_t i = 1; i < n; ++i)
        for (uint32_t j = 0; j < i; ++j, ++k)
            if (or_collides(c, r, i, j)) bits[k / 32] |= (uint32_t)1 << (k % 32);
}

void or_collide_pairs(const int32_t *c, const int32_t *r, const uint32_t *ii, const uint32_t *jj,
                      uint64_t count, uint8_t *out)
{
    for (uint64_t q = 0; q < count; ++q) out[q] = (uint8_t)or_collides(c, r, ii[q], jj[q]);
}
