"""GPU parity of the td-problems without the diagonal (Eq. (theorem_nodiag), strict g at the
element level): the packed strict-lower distance map against the FP64 oracle (2e-6) and bit for
bit against td_edm's with-diagonal map, and the strict-lower collision bits bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1308_1419_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402

RTOL = 2e-6


def _check_rel(got, want, ctx):
    err = np.abs(np.asarray(got, np.float64) - want)
    assert not (err > RTOL * want + 1e-30).any(), ctx


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 16])
def test_edm_strict_small(d):
    for n in [2, 3, 4, 5, 7, 100, 513, 1000]:
        xh = synth.uniform_points(n, d, 300 + n + d)
        x = torch.from_numpy(xh).cuda()
        total = n * (n - 1) // 2
        got = td.td_edm_strict(x)[:total].cpu().numpy()
        _check_rel(got, oracle.edm_strict(xh), (n, d))
        full, _ = td.td_edm("LTM", "persistent", x, 16)
        i, j = np.tril_indices(n, -1)
        ref = full.cpu().numpy()[i * (i + 1) // 2 + j]
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (n, d)


def test_edm_strict_large_sampled():
    n, d = 32768, 3
    xh = synth.uniform_points(n, d, 4243)
    x = torch.from_numpy(xh).cuda()
    out = td.td_edm_strict(x)
    total = n * (n - 1) // 2
    rng = np.random.default_rng(3)
    k = np.concatenate([rng.integers(0, total, 200000), np.arange(64), np.arange(total - 64, total)])
    i = ((np.sqrt(8 * k.astype(np.float64) + 1) + 1) // 2).astype(np.int64)
    i -= (i * (i - 1) // 2 > k)                       # exact row from the row starts
    i += ((i + 1) * i // 2 <= k)
    j = k - i * (i - 1) // 2
    assert np.all((j >= 0) & (j < i))
    got = out[torch.from_numpy(k).cuda()].cpu().numpy()
    _check_rel(got, oracle.edm_pairs(xh, i.astype(np.uint32), j.astype(np.uint32)), "n32768")


@pytest.mark.parametrize("n,bits,rmax", [(2, 4, 8), (33, 6, 20), (100, 10, 64), (1000, 12, 256), (3001, 14, 2048)])
def test_collide_strict_matches_oracle(n, bits, rmax):
    c, r = synth.spheres(n, seed=700 + n, coord_bits=bits, rmin=0, rmax=rmax)
    got = td.td_collide_strict(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda())
    words = td.td_collide_strict_words(n)
    want = oracle.collide_strict(c, r)
    assert np.array_equal(got[:words].cpu().numpy().view(np.uint32), want), n


def test_collide_strict_workload():
    """The collision workload (n = 32768, centres in [0, 2^20)^3, radii in [256, 2048])."""
    c, r = synth.spheres(32768)
    got = td.td_collide_strict(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda())
    words = td.td_collide_strict_words(32768)
    assert np.array_equal(got[:words].cpu().numpy().view(np.uint32), oracle.collide_strict(c, r))


def test_strict_errors_and_no_ops():
    x = torch.zeros(10, 3, device="cuda")
    with pytest.raises(td.TDError):
        td.td_edm_strict(torch.zeros(10, 0, device="cuda"))
    one = torch.zeros(1, 3, device="cuda")
    td.td_edm_strict(one)                                # n < 2: nothing to do
    assert td.td_collide_strict_words(0) == 0 and td.td_collide_strict_words(2) == 1
    assert td.td_collide_strict_words(33) == -(-33 * 32 // 2 // 32)
    td.td_edm_strict(x)


# ---- the block-mapped strict forms: the strict triangle of n points as the packed triangle of
# side n - 1 (row i' pairs point i' + 1 with j <= i'), blocks issued by g(lambda) or BB


@pytest.mark.parametrize("mapping", ["LTM", "BB"])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_edm_strict_blocks_bit_identical(mapping, rho):
    for d in (1, 2, 3, 4, 5, 8):
        for n in (2, 3, 9, 33, 100, 517, 1000, 2049):
            xh = synth.uniform_points(n, d, 900 + n + d)
            x = torch.from_numpy(xh).cuda()
            total = n * (n - 1) // 2
            got, st = td.td_edm_strict_blocks(mapping, x, rho)
            ref = td.td_edm_strict(x)
            assert torch.equal(got[:total].view(torch.int32), ref[:total].view(torch.int32)), (mapping, rho, d, n)
            nb = -(-(n - 1) // rho)
            assert st["useful_blocks"] == nb * (nb + 1) // 2
            if n in (100, 1000):
                _check_rel(got[:total].cpu().numpy(), oracle.edm_strict(xh), (mapping, rho, d, n))


def test_edm_strict_blocks_large_sampled():
    n, d = 32768, 3
    xh = synth.uniform_points(n, d, 4243)
    x = torch.from_numpy(xh).cuda()
    got, _ = td.td_edm_strict_blocks("LTM", x, 16)
    ref = td.td_edm_strict(x)
    total = n * (n - 1) // 2
    assert torch.equal(got[:total].view(torch.int32), ref[:total].view(torch.int32))


@pytest.mark.parametrize("mapping", ["LTM", "BB"])
@pytest.mark.parametrize("rho", [8, 16, 32, 64])
def test_collide_strict_blocks_matches_oracle(mapping, rho):
    for n, bits, rmax in [(2, 4, 8), (3, 4, 8), (33, 6, 20), (34, 6, 20), (100, 10, 64), (1000, 12, 256),
                          (3001, 14, 2048)]:
        c, r = synth.spheres(n, seed=800 + n + rho, coord_bits=bits, rmin=0, rmax=rmax)
        got, st = td.td_collide_strict_blocks(mapping, torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), rho)
        words = td.td_collide_strict_words(n)
        assert np.array_equal(got[:words].cpu().numpy().view(np.uint32), oracle.collide_strict(c, r)), (mapping, rho, n)


def test_collide_strict_blocks_exact_paths():
    """Exactly touching pairs (the FP32 band) and coordinates beyond 2^23 (the integer path)."""
    c = np.array([[0, 0, 0], [300, 400, 0], [0, 0, 0], [301, 400, 0],
                  [-2**30, -2**30, -2**30], [2**30 - 1, 2**30 - 1, 2**30 - 1],
                  [5, 5, 5], [5 + 16384 * 2, 5, 5]], dtype=np.int32)
    r = np.array([200, 300, 200, 300, 16384, 16384, 16384, 16384], dtype=np.int32)
    c = np.tile(c, (40, 1))
    r = np.tile(r, 40)
    small = c[:, :] % 1000
    for cc in (c, small.astype(np.int32)):
        for rho in (8, 32, 64):
            got, _ = td.td_collide_strict_blocks("LTM", torch.from_numpy(cc).cuda(), torch.from_numpy(r).cuda(), rho)
            words = td.td_collide_strict_words(len(r))
            assert np.array_equal(got[:words].cpu().numpy().view(np.uint32), oracle.collide_strict(cc, r)), rho


def test_collide_strict_blocks_workload():
    """The collision workload (n = 32768): identical to the element-level strict bits."""
    c, r = synth.spheres(32768)
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    words = td.td_collide_strict_words(32768)
    ref = td.td_collide_strict(ct, rt)[:words]
    for mapping, rho in (("LTM", 32), ("BB", 32), ("LTM", 16), ("LTM", 64), ("BB", 64)):
        got, _ = td.td_collide_strict_blocks(mapping, ct, rt, rho)
        assert torch.equal(got[:words], ref), (mapping, rho)
    assert np.array_equal(ref.cpu().numpy().view(np.uint32), oracle.collide_strict(c, r))


def test_collide_strict_blocks64_dense():
    """Every pair collides (all centres equal): with rho = 64 every word of the array is set by the
    OR of the row pieces of neighbouring blocks, including the words shared across block and row
    boundaries.  The array is cleared by the call: a buffer full of ones gives the same result."""
    for n in (2, 31, 33, 64, 65, 1000, 3001):
        c = np.zeros((n, 3), dtype=np.int32)
        r = np.full(n, 5, dtype=np.int32)
        ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
        words = td.td_collide_strict_words(n)
        want = oracle.collide_strict(c, r)
        for mapping in ("LTM", "BB"):
            bits = torch.full((max(words, 4),), -1, dtype=torch.int32, device="cuda")
            got, st = td.td_collide_strict_blocks(mapping, ct, rt, 64, bits)
            assert np.array_equal(got[:words].cpu().numpy().view(np.uint32), want), (n, mapping)
            nb = -(-n // 64)
            assert st["useful_blocks"] == nb * (nb + 1) // 2


def test_strict_blocks_errors_and_no_ops():
    x = torch.zeros(10, 3, device="cuda")
    c = torch.zeros(10, 3, dtype=torch.int32, device="cuda")
    r = torch.zeros(10, dtype=torch.int32, device="cuda")
    for bad in (("UTM", 16), ("RB", 16), ("LTM", 12), ("LTM", 128), ("UTM-BLOCK", 64)):
        with pytest.raises(td.TDError):
            td.td_edm_strict_blocks(bad[0], x, bad[1])
        with pytest.raises(td.TDError):
            td.td_collide_strict_blocks(bad[0], c, r, bad[1])
    with pytest.raises(td.TDError):
        td.td_edm_strict_blocks("LTM", x, 64)  # 64 x 64 blocks: the collision bits only
    td.td_collide_strict_blocks("LTM", c[:1], r[:1], 64)
    with pytest.raises(td.TDError):
        td.td_edm_strict_blocks("LTM", torch.zeros(10, 9, device="cuda"), 16)  # d > 8: td_edm_strict
    td.td_edm_strict_blocks("LTM", torch.zeros(1, 3, device="cuda"), 16)
    td.td_collide_strict_blocks("LTM", c[:1], r[:1], 32)


def test_collide_strict_blocks_random_shapes():
    """Seeded random sizes and radii ranges: the block-mapped strict bits equal the element-level ones."""
    rng = np.random.default_rng(77)
    for _ in range(12):
        n = int(rng.integers(2, 6000))
        bits_ = int(rng.integers(4, 21))
        c, r = synth.spheres(n, seed=int(rng.integers(1, 1 << 30)), coord_bits=bits_, rmin=0,
                             rmax=int(rng.integers(1, 2049)))
        ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
        words = td.td_collide_strict_words(n)
        ref = td.td_collide_strict(ct, rt)[:words].clone()
        for mapping in ("LTM", "BB"):
            for rho in (8, 16, 32, 64):
                got, _ = td.td_collide_strict_blocks(mapping, ct, rt, rho)
                assert torch.equal(got[:words], ref), (n, bits_, mapping, rho)
