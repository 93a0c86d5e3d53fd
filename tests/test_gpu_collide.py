"""GPU parity of the bit-packed collision table (a td-problem of the abstract and Sec. I):
bit-exact against the oracle's int64 definition, for g(lambda) and BB tiles and both
schedules."""
import numpy as np
import pytest

import oracle
from paper_1308_1419_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402

VARIANTS = [("LTM", "grid"), ("LTM", "persistent"), ("BB", "grid"), ("BB", "persistent")]


def _table(c, r, mapping, sched):
    ct = torch.from_numpy(np.ascontiguousarray(c, dtype=np.int32)).cuda()
    rt = torch.from_numpy(np.ascontiguousarray(r, dtype=np.int32)).cuda()
    words = td.td_collide_words(r.size)
    table = torch.full((max(words, 4),), -1, dtype=torch.int32, device="cuda")
    table, st = td.td_collide(mapping, sched, ct, rt, table)
    return table[:words].cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("mapping,sched", VARIANTS)
def test_collide_benchmark_config_full_table(mapping, sched):
    """n = 32768 spheres, centres U[0,2^20)^3, radii U[256,2048]: the whole table."""
    c, r = synth.spheres()
    got, st = _table(c, r, mapping, sched)
    want = oracle.collide(c, r)
    assert np.array_equal(got, want), int(np.count_nonzero(got != want))
    assert st["useful_blocks"] == 512 * 513 // 2  # 64 x 64 blocks of four bit tiles


@pytest.mark.parametrize("mapping,sched", VARIANTS)
def test_collide_dense_and_ragged(mapping, sched):
    for n in [1, 2, 31, 32, 33, 63, 100, 1000, 4097]:
        c, r = synth.spheres(n, seed=500 + n, coord_bits=12, rmin=0, rmax=600)
        got, _ = _table(c, r, mapping, sched)
        want = oracle.collide(c, r)
        assert np.array_equal(got, want), (n, int(np.count_nonzero(got != want)))
        assert want.any() or n < 100


def test_collide_edge_cases():
    n = 70
    c = np.zeros((n, 3), dtype=np.int32)
    r = np.zeros(n, dtype=np.int32)
    got, _ = _table(c, r, "LTM", "persistent")
    assert np.array_equal(got, oracle.collide(c, r))
    assert sum(bin(int(w)).count("1") for w in got) == n * (n - 1) // 2
    # exactly touching collides, one unit further does not; extreme allowed ranges
    c = np.array([[0, 0, 0], [300, 400, 0], [0, 0, 0], [301, 400, 0],
                  [-2**30, -2**30, -2**30], [2**30 - 1, 2**30 - 1, 2**30 - 1],
                  [5, 5, 5], [5 + 16384 * 2, 5, 5]], dtype=np.int32)
    r = np.array([200, 300, 200, 300, 16384, 16384, 16384, 16384], dtype=np.int32)
    got, _ = _table(c, r, "LTM", "grid")
    assert np.array_equal(got, oracle.collide(c, r))
    w, b = oracle.collide_bitpos(1, 0)
    assert (got[w] >> b) & 1 == 1
    w, b = oracle.collide_bitpos(7, 6)
    assert (got[w] >> b) & 1 == 1


def test_collide_rejects():
    c = torch.zeros(10, 3, dtype=torch.int32, device="cuda")
    r = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(td.TDError):
        td.td_collide("UTM", "grid", c, r)
    with pytest.raises(td.TDError):
        td.td_collide("LTM", "chunked", c, r)


def test_collide_many_exact_ties():
    """Small integer cube and radii: s - R^2 is often exactly 0 or +-1, so most tiles take the FP32
    band and the exact re-test (tiled table and block-mapped strict bits)."""
    rng = np.random.default_rng(77)
    for n in (100, 1000, 3000):
        c = rng.integers(0, 16, (n, 3)).astype(np.int32)
        r = rng.integers(0, 16, n).astype(np.int32)
        s = ((c[:, None, :].astype(np.int64) - c[None, :, :]) ** 2).sum(-1)
        R2 = (r[:, None].astype(np.int64) + r[None, :]) ** 2
        assert np.count_nonzero(np.abs(s - R2) <= 1) > n // 8  # the case really is tie-heavy
        ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
        got, _ = _table(c, r, "LTM", "persistent")
        assert np.array_equal(got, oracle.collide(c, r)), n
        words = td.td_collide_strict_words(n)
        for rho in (8, 32):
            bits, _ = td.td_collide_strict_blocks("LTM", ct, rt, rho)
            assert np.array_equal(bits[:words].cpu().numpy().view(np.uint32), oracle.collide_strict(c, r)), (n, rho)


def _full_range_cases(seed):
    """Coordinates and radii over the whole int32 range: squared distances and (r_i + r_j)^2 up to
    about 2^64, exact ties and one-off misses at large magnitudes, negative radii (they enter only
    through (r_i + r_j)^2), and the extreme corners where |r_i + r_j| = 2^32."""
    rng = np.random.default_rng(seed)
    lo, hi = -2**31, 2**31 - 1
    c = [rng.integers(lo, hi, (160, 3), endpoint=True)]
    r = [rng.integers(lo, hi, 160, endpoint=True)]
    k = 2**28  # (3k, 4k, 0) at distance exactly 5k
    c.append(np.array([[0, 0, 0], [3 * k, 4 * k, 0], [3 * k + 1, 4 * k, 0], [-3 * k, -4 * k, 7]]))
    r.append(np.array([2 * k, 3 * k, 3 * k, -7 * k]))
    c.append(np.array([[lo, lo, lo], [hi, hi, hi], [lo, hi, 0], [hi, lo, 0], [lo, lo, lo]]))
    r.append(np.array([lo, lo, hi, hi, 0]))
    base = rng.integers(-2**30, 2**30, 3)  # a cluster with radii of 2^29..2^30: many near-ties
    c.append(base + rng.integers(-2**30, 2**30, (120, 3)))
    r.append(rng.integers(2**29, 2**30, 120))
    c = np.concatenate(c).clip(lo, hi).astype(np.int32)
    r = np.concatenate(r).clip(lo, hi).astype(np.int32)
    return c, r


@pytest.mark.parametrize("seed", [1, 2])
def test_collide_full_int32_range(seed):
    """Every kernel form decides any int32 input exactly: the tiled table (both mappings, both
    schedules), the element-level strict bits and the block-mapped strict bits."""
    c, r = _full_range_cases(seed)
    want = oracle.collide(c, r)
    assert want.any()
    for mapping, sched in VARIANTS:
        got, _ = _table(c, r, mapping, sched)
        assert np.array_equal(got, want), (mapping, sched, int(np.count_nonzero(got != want)))
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    words = td.td_collide_strict_words(r.size)
    want_s = oracle.collide_strict(c, r)
    got = td.td_collide_strict(ct, rt)[:words].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want_s)
    for rho in (8, 32):
        bits, _ = td.td_collide_strict_blocks("LTM", ct, rt, rho)
        assert np.array_equal(bits[:words].cpu().numpy().view(np.uint32), want_s), rho
