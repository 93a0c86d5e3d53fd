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
