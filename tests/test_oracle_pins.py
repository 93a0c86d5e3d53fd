"""Pins for the CPU oracle: each oracle function is checked against something other than
itself -- the block numbering the paper prints, brute-force enumeration, library routines
(math.isqrt, scipy's pdist), closed forms and invariants.  No GPU is involved.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1308_1419_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ integer square root

def test_isqrt_matches_math_isqrt():
    rng = np.random.default_rng(7)
    vals = [0, 1, 2, 3, 4, 15, 16, 17, 2**32 - 1, 2**32, 2**62, 2**63 - 1, 2**64 - 1]
    for r in [1, 2, 3, 1000, 2**20 + 5, 2**31 - 1, 2**32 - 1]:
        vals += [r * r - 1, r * r, r * r + 1]
    vals += [int(v) for v in rng.integers(0, 2**63, 2000, dtype=np.uint64)]
    for v in vals:
        assert oracle.isqrt(v) == math.isqrt(v), v


# ------------------------------------------------------------------ g(lambda), Eq. (theorem)

def _golden_rows():
    rows, lasts = [], []
    with open(os.path.join(GOLDEN, "ltm_block_numbering.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            if p[0] == "last":
                lasts.append(int(p[1]))
            else:
                rows.append(tuple(int(v) for v in p))
    return rows, lasts


def test_ltm_printed_numbering():
    rows, lasts = _golden_rows()
    for lam, i, j in rows:
        assert tuple(oracle.ltm(lam)[0]) == (i, j)
    for n in lasts:
        first = n * (n - 1) // 2
        assert tuple(oracle.ltm(first)[0]) == (n - 1, 0)
        assert tuple(oracle.ltm(first + 1)[0]) == (n - 1, 1)
        assert tuple(oracle.ltm(n * (n + 1) // 2 - 1)[0]) == (n - 1, n - 1)


def _enumerate_lower(nb, diag=True):
    """Row-major walk of the block triangle: the numbering g must invert."""
    counts = np.arange(nb, dtype=np.int64) + (1 if diag else 0)
    i = np.repeat(np.arange(nb, dtype=np.int64), counts)
    starts = np.repeat(np.cumsum(counts) - counts, counts)
    j = np.arange(i.size, dtype=np.int64) - starts
    return i, j


def test_ltm_is_inverse_of_rowmajor_walk_up_to_nb_4096():
    # g does not depend on n, so one walk over lambda in [0, T(4096)) covers every nb <= 4096.
    i, j = _enumerate_lower(4096)
    lam = np.arange(i.size, dtype=np.uint64)
    ij = oracle.ltm(lam)
    assert np.array_equal(ij[:, 0], i) and np.array_equal(ij[:, 1], j)


def test_ltm_row_boundaries_up_to_2_40():
    rng = np.random.default_rng(11)
    rows = list(range(1, 5000)) + [int(v) for v in rng.integers(5000, 1_500_000, 20000)]
    rows += [1_482_910, 1_482_911, 1_482_912]  # T(i) straddles 2^40 near here
    lam, want = [], []
    for r in rows:
        start = r * (r + 1) // 2
        lam += [start - 1, start, start + r]
        want += [(r - 1, r - 1), (r, 0), (r, r)]
    ij = oracle.ltm(np.array(lam, dtype=np.uint64))
    assert [tuple(v) for v in ij.tolist()] == want


# ------------------------------------------------------------------ FP32 evaluations of g (Sec. III-A)

def test_fast_rsqrt_error_matches_lomont():
    """The bit-level estimate with 0x5f3759df has a maximum relative error of about 3.44%, and
    0.175% after one Newton step (Lomont's analysis of the constant); each further step about
    squares the error.  The relative error repeats with period 4 in x, and the estimate of 4x is
    exactly half the estimate of x (the exponent field moves by one)."""
    xs = [float(np.float32(x)) for x in np.linspace(1.0, 4.0, 20001)]
    errs = [max(abs(oracle.fast_rsqrt(x, s) * math.sqrt(x) - 1.0) for x in xs) for s in range(4)]
    assert 0.0340 < errs[0] < 0.0345
    assert 0.00174 < errs[1] < 0.001753
    assert errs[2] < 5e-6 and errs[3] < 3e-7
    for x in (1.0, 1.3, 2.7, 3.9, 1e3, 7e5):
        xf = float(np.float32(x))
        assert oracle.fast_rsqrt(4.0 * xf, 0) == oracle.fast_rsqrt(xf, 0) / 2.0


def _row(lam):
    return (math.isqrt(8 * lam + 1) - 1) // 2   # exact row of lambda, independent of the oracle


def test_ltm_x_exact_while_fp32_resolves_row_starts():
    """LTM-X: below T(2048), x = 2 lambda + 1/4 is exact in FP32 (two fraction bits, below 2^22)
    and sqrtf is correctly rounded, so a row start T(r), where sqrt(x) = r + 1/2 exactly, lands
    on the right row: no failure there.  The first failure lies on a row boundary and is genuine."""
    f = oracle.ltm_variant_first_fail(oracle.LTM_X, 0, 1 << 26)
    assert oracle.tri(2048) <= f < 1 << 26
    r = _row(f)
    assert f in (oracle.tri(r), oracle.tri(r + 1) - 1)
    assert oracle.ltm_variant(oracle.LTM_X, f)[0] != r
    for lam in (0, 1, 2, 3, 5, 6, oracle.tri(2047), oracle.tri(2048) - 1, f - 1):
        assert oracle.ltm_variant(oracle.LTM_X, lam) == (_row(lam), lam - oracle.tri(_row(lam)))


def test_ltm_n_with_epsilon():
    """LTM-N: after three Newton steps y is within 3e-7 of 1/sqrt(x), so at a row start the
    computed x y - 1/2 is at most (r + 1/2) 3e-7 below r, which the epsilon 1e-4 covers while
    r < 300.  The first failure lies on a row boundary and is genuine."""
    f = oracle.ltm_variant_first_fail(oracle.LTM_N, 0, 1 << 26)
    assert oracle.tri(300) <= f < 1 << 26
    r = _row(f)
    assert f in (oracle.tri(r), oracle.tri(r + 1) - 1)
    assert oracle.ltm_variant(oracle.LTM_N, f)[0] != r
    for lam in (0, 1, 2, 3, 4, 5, oracle.tri(299), f - 1):
        assert oracle.ltm_variant(oracle.LTM_N, lam) == (_row(lam), lam - oracle.tri(_row(lam)))


def test_fast_rsqrt_fma_error_matches_lomont():
    """The Newton steps with their product fused into the subtraction (one rounding fewer) keep
    Lomont's error figures: 3.44% for the seed, 0.175% after one step, then about squared per
    step.  A wrong sign or a dropped factor in the fused step breaks the one-step figure."""
    xs = [float(np.float32(x)) for x in np.linspace(1.0, 4.0, 20001)]
    errs = [max(abs(oracle.fast_rsqrt_fma(x, s) * math.sqrt(x) - 1.0) for x in xs) for s in range(4)]
    assert 0.0340 < errs[0] < 0.0345
    assert 0.00174 < errs[1] < 0.001753
    assert errs[2] < 5e-6 and errs[3] < 3e-7
    assert any(oracle.fast_rsqrt_fma(x, 3) != oracle.fast_rsqrt(x, 3) for x in xs)   # a distinct rounding


def test_ltm_n_fma_exact_over_the_papers_range():
    """Sec. III-A: with the epsilon 1e-4, LTM-N computes i exactly for N in [0, 30720], i.e. (rho = 16)
    for every block index lambda < T(1920) = 1 844 160.  The contracted evaluation, the one a CUDA
    compiler emits unless told otherwise, meets that claim; the evaluation that rounds every
    product on its own does not (it first fails inside the range, at the start of a row).  The
    contracted variant's own first failure lies on a row boundary and is genuine."""
    end = oracle.tri(30720 // 16)
    f = oracle.ltm_variant_first_fail(oracle.LTM_N_FMA, 0, 1 << 26)
    assert end <= f < 1 << 26
    r = _row(f)
    assert f in (oracle.tri(r), oracle.tri(r + 1) - 1)
    assert oracle.ltm_variant(oracle.LTM_N_FMA, f)[0] != r
    for lam in (0, 1, 2, 3, 4, 5, oracle.tri(1919), end - 1, f - 1):
        assert oracle.ltm_variant(oracle.LTM_N_FMA, lam) == (_row(lam), lam - oracle.tri(_row(lam)))
    assert oracle.ltm_variant_first_fail(oracle.LTM_N, 0, end) < end


def test_ltm_x_contraction_changes_nothing():
    """LTM-X has no product to fuse but 2 lambda + 1/4, and 2 (float)lambda is exact in binary
    floating point, so the fused radicand is the rounded one: both evaluations share their first
    failure and agree on a dense sample around it and over the whole range below it."""
    f = oracle.ltm_variant_first_fail(oracle.LTM_X, 0, 1 << 26)
    assert oracle.ltm_variant_first_fail(oracle.LTM_X_FMA, 0, 1 << 26) == f
    lams = list(range(f - 2000, f + 2000)) + list(range(1 << 25, (1 << 25) + 2000))
    for lam in lams:
        assert oracle.ltm_variant(oracle.LTM_X_FMA, lam) == oracle.ltm_variant(oracle.LTM_X, lam)


def test_ltm_nodiag_is_inverse_of_strict_walk():
    # strict walk: row i holds i blocks (row 0 is empty)
    i, j = _enumerate_lower(3000, diag=False)
    ij = oracle.ltm_nodiag(np.arange(i.size, dtype=np.uint64))
    assert np.array_equal(ij[:, 0], i) and np.array_equal(ij[:, 1], j)
    assert np.all(ij[:, 1] < ij[:, 0])


# ------------------------------------------------------------------ UTM (Sec. III-B)

@pytest.mark.parametrize("n", [2, 3, 4, 5, 16, 17, 100, 257])
def test_utm_formula_matches_rowmajor_enumeration(n):
    ab = oracle.utm_enum(n)
    for k in range(ab.shape[0]):
        assert oracle.utm_ab(n, k) == (int(ab[k, 0]), int(ab[k, 1])), (n, k)


def test_utm_formula_large_n_sampled():
    # n = 65537 is the side used for a lower triangle of N = 65536 with its diagonal.
    rng = np.random.default_rng(3)
    for n in [5000, 65537]:
        total = n * (n - 1) // 2
        row_start = np.concatenate([[0], np.cumsum(n - np.arange(1, n, dtype=np.int64))])
        ks = [0, 1, total - 1, total - 2] + [int(v) for v in rng.integers(0, total, 3000)]
        ks += [int(row_start[a]) + o for a in rng.integers(0, n - 1, 500) for o in (-1, 0) if row_start[a] + o >= 0]
        for k in ks:
            a, b = oracle.utm_ab(n, k)
            assert 1 <= a < b <= n
            assert row_start[a - 1] + (b - a - 1) == k


def test_utm_lower_covers_triangle():
    for N in [1, 2, 7, 64, 129]:
        ij = oracle.utm_lower(N, np.arange(N * (N + 1) // 2, dtype=np.uint64))
        assert np.all(ij[:, 1] <= ij[:, 0]) and np.all(ij[:, 0] < N)
        pos = ij[:, 0].astype(np.int64) * (ij[:, 0] + 1) // 2 + ij[:, 1]
        assert np.array_equal(np.sort(pos), np.arange(N * (N + 1) // 2))


# ------------------------------------------------------------------ all strategies: bijection

@pytest.mark.parametrize("strategy", ["BB", "LTM", "UTM", "RB", "UTM-BLOCK"])
def test_strategy_bijection_small_all_N(strategy):
    for rho in (8, 16):
        for N in range(1, 97):
            count, st = oracle.cover(strategy, N, rho)
            assert np.all(count == 1), (strategy, N, rho)
            assert st["hits"] == N * (N + 1) // 2


@pytest.mark.parametrize("strategy", ["BB", "LTM", "UTM", "RB", "REC", "UTM-BLOCK"])
@pytest.mark.parametrize("N,rho", [(1024, 8), (1024, 16), (1024, 32), (1000, 8), (2048, 32), (768, 16), (1536, 8)])
def test_strategy_bijection_sizes(strategy, N, rho):
    if strategy == "REC" and N % rho:
        with pytest.raises(ValueError):
            oracle.cover(strategy, N, rho)
        return
    count, st = oracle.cover(strategy, N, rho)
    assert np.all(count == 1)


@pytest.mark.slow
@pytest.mark.parametrize("strategy", ["UTM", "RB", "REC"])
def test_strategy_bijection_every_side_to_4096(strategy):
    """UTM, RB and REC depend on the triangle's side, so each is walked for every side N = 1 .. 4096
    (about 1.15e10 mapped elements per strategy) at the element level (rho = 1: REC then splits
    N = m 2^k with m odd), and every element of the triangle must be reached exactly once.
    Block-level UTM is the same formula applied to the block triangle of side nb, so the UTM walk
    covers it for every nb <= 4096; g(lambda) does not depend on the side at all (walked over
    every lambda < T(4096) above).  The sides are spread over the host's cores; each call into
    the C walk runs with the interpreter lock released."""
    import concurrent.futures as cf
    import os

    def check(N):
        count, st = oracle.cover(strategy, N, 1)
        return N, bool(count.min() == 1 and count.max() == 1 and st["hits"] == N * (N + 1) // 2)

    sides = range(4096, 0, -1)  # largest first, so the threads finish together
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        bad = [N for N, ok in ex.map(check, sides) if not ok]
    assert not bad, (strategy, bad[:10])


def test_rec_levels_and_launch_count():
    # N = m 2^k with m a multiple of rho and k as large as possible (Sec. III-B)
    assert oracle.rec_levels(1024, 16) == (6, 16)
    assert oracle.rec_levels(65536, 8) == (13, 8)
    assert oracle.rec_levels(768, 16) == (4, 48)
    assert oracle.rec_levels(1000, 8) == (0, 1000)
    assert oracle.rec_levels(100, 8) is None
    for N, rho in [(1024, 16), (768, 16), (512, 32)]:
        k, m = oracle.rec_levels(N, rho)
        _, st = oracle.cover("REC", N, rho)
        assert st["launches"] == k + 1
        # useful blocks: k levels of full squares plus the diagonal triangles' lower blocks
        mb = m // rho
        assert st["useful"] == sum((N >> l) ** 2 // rho ** 2 * 2 ** (l - 1) for l in range(1, k + 1)) \
            + 2 ** k * mb * (mb + 1) // 2


def test_rb_shape():
    # even N: (N+1) x N/2 threads, odd N: N x (floor(N/2)+1) threads; both equal T(N)
    for N in range(1, 200):
        W, H = oracle.rb_dims(N)
        assert W * H == N * (N + 1) // 2
    # rows below the fold keep their column; the folded part comes from columns >= N/2
    assert oracle.rb_map(8, 0, 1) == (0, 0)
    assert oracle.rb_map(8, 3, 8) == (7, 3)
    assert oracle.rb_map(8, 0, 0) == (7, 7)
    assert oracle.rb_map(8, 3, 0) == (7, 4)
    assert oracle.rb_map(8, 3, 3) == (4, 4)


@pytest.mark.parametrize("N,rho", [(1024, 16), (1000, 8), (4096, 32), (33, 8)])
def test_block_counts_closed_forms(N, rho):
    """Sec. II-A: BB launches n^2 blocks of which n(n-1)/2 are wasted; n(n+1)/2 suffice."""
    nb = -(-N // rho)
    _, bb = oracle.cover("BB", N, rho)
    assert bb["launched"] == nb * nb and bb["useful"] == nb * (nb + 1) // 2
    assert bb["launched"] - bb["useful"] == nb * (nb - 1) // 2
    _, lt = oracle.cover("LTM", N, rho)
    assert lt["launched"] == lt["useful"] == nb * (nb + 1) // 2


# ------------------------------------------------------------------ probe hash and layout

def _fmix_inverse(z):
    M = 0xFFFFFFFF
    z ^= z >> 16
    z = (z * pow(0xC2B2AE35, -1, 2**32)) & M
    z ^= (z >> 13) ^ (z >> 26)
    z = (z * pow(0x85EBCA6B, -1, 2**32)) & M
    z ^= z >> 16
    return (z - 0x9E3779B9) & M


def test_splitmix32_round_trips_through_inverse():
    rng = np.random.default_rng(5)
    for x in [0, 1, 2, 0xFFFFFFFF, 0x9E3779B9] + [int(v) for v in rng.integers(0, 2**32, 5000)]:
        assert _fmix_inverse(oracle.splitmix32(x)) == x
    # the finaliser maps 0 to 0, so the input that cancels the increment hashes to 0
    assert oracle.splitmix32((-0x9E3779B9) & 0xFFFFFFFF) == 0


def test_probe_layout():
    for N in [1, 2, 5, 64, 300]:
        out = oracle.probe(N)
        assert out.size == N * (N + 1) // 2
        # positions from a cumulative count of row lengths, independent of T()
        starts = np.concatenate([[0], np.cumsum(np.arange(1, N + 1))])
        for i in range(N):
            for j in sorted({0, i // 2, i}):
                assert out[starts[i] + j] == oracle.splitmix32(i * N + j)
    full = oracle.probe(300)
    part = oracle.probe(300, 100, 200)
    assert np.array_equal(part, full[oracle.tri(100): oracle.tri(200)])


# ------------------------------------------------------------------ EDM (Sec. IV)

@pytest.mark.parametrize("n,d", [(1, 3), (2, 1), (37, 3), (200, 4), (129, 16), (65, 64)])
def test_edm_matches_scipy_pdist(n, d):
    from scipy.spatial.distance import pdist, squareform
    x = synth.uniform_points(n, d, 99 + n + d)
    full = squareform(pdist(x.astype(np.float64))) if n > 1 else np.zeros((1, 1))
    ii, jj = np.tril_indices(n)   # row-major (i, j), j <= i
    assert np.allclose(oracle.edm(x), full[ii, jj], rtol=1e-14, atol=0)


def test_edm_exact_cases():
    # d = 1: |a_i - a_j| exactly
    x = synth.uniform_points(50, 1, 4)
    D = oracle.edm(x)
    ii, jj = np.tril_indices(50)
    assert np.array_equal(D, np.abs(x[ii, 0].astype(np.float64) - x[jj, 0]))
    # integer lattice points: D^2 is an integer, D = sqrt of it
    pts = np.array([[0, 0, 0], [3, 4, 0], [1, 2, 2], [6, 8, 0], [-1, -2, -2]], dtype=np.float32)
    D = oracle.edm(pts)
    assert D[oracle.tri(1) + 0] == 5.0 and D[oracle.tri(2) + 0] == 3.0
    assert D[oracle.tri(3) + 1] == 5.0 and D[oracle.tri(4) + 2] == 6.0
    assert D[oracle.tri(3) + 0] == 10.0


def test_edm_invariants():
    x = synth.uniform_points(120, 3, 17)
    D = oracle.edm(x)
    diag = np.array([oracle.tri(i) + i for i in range(120)])
    assert np.all(D[diag] == 0.0) and np.all(D >= 0)
    def dist(i, j):
        return D[oracle.tri(max(i, j)) + min(i, j)]
    rng = np.random.default_rng(2)
    for a, b, c in rng.integers(0, 120, (2000, 3)):
        assert dist(a, c) <= dist(a, b) + dist(b, c) + 1e-12
    # permuting the points permutes the map
    perm = rng.permutation(120)
    Dp = oracle.edm(x[perm])
    for _ in range(300):
        i, j = rng.integers(0, 120, 2)
        assert Dp[oracle.tri(max(i, j)) + min(i, j)] == dist(perm[i], perm[j])
    # pairs and row ranges agree with the full map
    ii, jj = np.tril_indices(120)
    assert np.array_equal(oracle.edm_pairs(x, ii, jj), D)
    assert np.array_equal(oracle.edm(x, 30, 70), D[oracle.tri(30): oracle.tri(70)])


def test_edm_batched_is_problem_by_problem():
    ns, ds, xcat = synth.batched_problems(nprob=6, nmin=3, ratio=10.0)
    out = oracle.edm_batched(xcat, ns, ds)
    off_x, off_o = 0, 0
    for n, d in zip(ns, ds):
        n, d = int(n), int(d)
        x = xcat[off_x: off_x + n * d].reshape(n, d)
        assert np.array_equal(out[off_o: off_o + n * (n + 1) // 2], oracle.edm(x))
        off_x += n * d
        off_o += n * (n + 1) // 2
    assert off_o == out.size


# ------------------------------------------------------------------ collision table

def _brute_collisions(c, r):
    c = c.astype(np.int64)
    r = r.astype(np.int64)
    d2 = ((c[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    R = r[:, None] + r[None, :]
    return d2 <= R * R


def _decode_table(table, n):
    """Read every strict pair back out of the table by walking tiles in numbering order."""
    nt = -(-n // 32)
    M = np.zeros((n, n), dtype=bool)
    t = 0
    for bi in range(nt):
        for bj in range(bi + 1):
            for r in range(32):
                w = int(table[t * 32 + r])
                for c in range(32):
                    i, j = 32 * bi + r, 32 * bj + c
                    bit = (w >> c) & 1
                    if i < n and j < i:
                        M[i, j] = bool(bit)
                    else:
                        assert bit == 0, (i, j)
            t += 1
    assert t * 32 == table.size
    return M


@pytest.mark.parametrize("n,bits,rmax", [(1, 8, 4), (31, 6, 20), (33, 6, 20), (100, 10, 64), (130, 20, 2048)])
def test_collide_matches_brute_force(n, bits, rmax):
    c, r = synth.spheres(n, seed=40 + n, coord_bits=bits, rmin=0, rmax=rmax)
    table = oracle.collide(c, r)
    assert table.size == oracle.collide_words(n) == (-(-n // 32)) * (-(-n // 32) + 1) // 2 * 32
    want = np.tril(_brute_collisions(c, r), -1)
    assert np.array_equal(_decode_table(table, n), want)


def test_collide_edge_cases():
    # all centres equal: every strict pair collides; nothing on or above the diagonal
    n = 70
    c = np.zeros((n, 3), dtype=np.int32)
    r = np.zeros(n, dtype=np.int32)
    M = _decode_table(oracle.collide(c, r), n)
    assert np.array_equal(M, np.tril(np.ones((n, n), dtype=bool), -1))
    # touching exactly counts (<=); one unit further does not
    c = np.array([[0, 0, 0], [300, 400, 0], [0, 0, 0], [301, 400, 0]], dtype=np.int32)
    r = np.array([200, 300, 200, 300], dtype=np.int32)
    assert oracle.collide_pairs(c, r, [1, 3], [0, 2]).tolist() == [1, 0]
    # large coordinates need 64-bit squares
    c = np.array([[0, 0, 0], [2**30 - 1, 2**30 - 1, 2**30 - 1]], dtype=np.int32)
    r = np.array([2**30, 2**29], dtype=np.int32)             # R^2 = 2.25 * 2^60 < 3 (2^30 - 1)^2
    assert oracle.collide_pairs(c, r, [1], [0]).tolist() == [0]
    r = np.array([2**30 - 1, 2**29 + 2**28], dtype=np.int32)  # R^2 = (1.75 * 2^30 - 1)^2 >= 3 (2^30 - 1)^2
    assert oracle.collide_pairs(c, r, [1], [0]).tolist() == [1]


def test_collide_exact_for_full_int32_range():
    """The predicate stays exact where int64 squares would overflow: compared with Python
    integers on pairs spanning the whole int32 range."""
    rng = np.random.default_rng(12)
    lo, hi = -2**31, 2**31 - 1
    c = rng.integers(lo, hi + 1, (300, 3)).astype(np.int32)
    c[0] = [lo, lo, lo]
    c[1] = [hi, hi, hi]
    r = rng.integers(0, 2**31, 300).astype(np.int32)
    r[0], r[1] = 2**31 - 1, 2**31 - 1
    ii, jj = np.tril_indices(300, -1)
    got = oracle.collide_pairs(c, r, ii, jj)
    cc = [[int(v) for v in row] for row in c]
    rr = [int(v) for v in r]
    want = [int(sum((cc[i][k] - cc[j][k]) ** 2 for k in range(3)) <= (rr[i] + rr[j]) ** 2)
            for i, j in zip(ii.tolist(), jj.tolist())]
    assert got.tolist() == want
    assert got[0] == 0  # (1, 0): |d|^2 = 3 (2^32 - 1)^2 > (2^32 - 2)^2


def test_collide_bitpos_layout():
    assert oracle.collide_bitpos(1, 0) == (1, 0)
    assert oracle.collide_bitpos(31, 30) == (31, 30)
    assert oracle.collide_bitpos(32, 0) == (32 * 1 + 0, 0)      # tile (1,0) is tile 1
    assert oracle.collide_bitpos(33, 32) == (32 * 2 + 1, 0)     # tile (1,1) is tile 2
    assert oracle.collide_bitpos(64, 33) == (32 * 4 + 0, 1)     # tile (2,1) is tile 4


# ------------------------------------------------------------------ synthetic inputs

def test_synth_streams():
    s1 = synth.Stream(1)
    a = s1.u64(10)
    b = s1.u64(5)
    assert np.array_equal(np.concatenate([a, b]), synth.Stream(1).u64(15))
    # SplitMix64 with seed 0 (published reference output of the generator)
    assert int(synth.Stream(0).u64(1)[0]) == 0xE220A8397B1DCDAF
    u = synth.uniform_points(100000, 1, 3)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    z = synth.Stream(9).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    c, r = synth.spheres(10000)
    assert c.min() >= 0 and c.max() < 2**20 and r.min() >= 256 and r.max() <= 2048
    ns, ds, x = synth.batched_problems()
    assert ns.size == 512 and ns.min() >= 64 and ns.max() < 8192
    assert set(ds.tolist()) <= {3, 16, 64} and x.size == int((ns.astype(np.int64) * ds).sum())


# ------------------------------------------------------------------ td-problems without the diagonal

@pytest.mark.parametrize("n,d", [(2, 1), (3, 3), (40, 2), (129, 4), (300, 7)])
def test_edm_strict_matches_scipy_pdist(n, d):
    """pdist lists the pairs j < i in its own order (row j of the upper triangle); the strict
    packed index k = i(i-1)/2 + j of the same pair picks the same distance."""
    from scipy.spatial.distance import pdist
    x = synth.uniform_points(n, d, 77 + n)
    got = oracle.edm_strict(x)
    ref = pdist(x.astype(np.float64))
    i, j = np.tril_indices(n, -1)                   # row-major strict lower: (1,0), (2,0), (2,1), ...
    k = i * (i - 1) // 2 + j
    assert np.array_equal(k, np.arange(k.size))
    pos = n * j - j * (j + 1) // 2 + (i - j - 1)     # pdist's index of the pair (j, i)
    assert np.allclose(got, ref[pos], rtol=1e-15, atol=0)


@pytest.mark.parametrize("n,bits,rmax", [(2, 4, 8), (33, 6, 20), (100, 10, 64), (257, 12, 2048)])
def test_collide_strict_matches_brute_force(n, bits, rmax):
    c, r = synth.spheres(n, seed=90 + n, coord_bits=bits, rmin=0, rmax=rmax)
    words = oracle.collide_strict(c, r)
    total = n * (n - 1) // 2
    assert words.size == -(-total // 32)
    flags = np.unpackbits(words.view(np.uint8), bitorder="little")
    assert not flags[total:].any()                   # unused bits of the last word are zero
    i, j = np.tril_indices(n, -1)
    assert np.array_equal(flags[:total].astype(bool), _brute_collisions(c, r)[i, j])
