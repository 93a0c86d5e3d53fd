"""GPU checks of the block-row slices a partition hands to each GPU (td_partition, then
td_map_probe_rows / td_edm_rows / td_collide_rows), run on one GPU one slice after another.

Block rows are contiguous in g(lambda) (Sec. II-A, Eq. (matrix_indexing)), so a rank's share of a
triangle is one contiguous range of lambda and one contiguous slice of the packed output.  For
G in {2, 3, 8}, every rank's slice is written into its place of one buffer; the result must equal
the whole-triangle call byte for byte, and the oracle (bit-exact for the probe and the collision
table, within 2e-6 for the distances)."""
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


def _tri(m):
    return m * (m + 1) // 2


def _slices(N, rho, G):
    parts = [td.td_partition(N, rho, G, r) for r in range(G)]
    for k, (br0, br1, off0, off1) in enumerate(parts):
        assert off0 == _tri(min(br0 * rho, N)) and off1 == _tri(min(br1 * rho, N))
        assert off0 % 4 == 0 and (off1 % 4 == 0 or off1 == _tri(N))  # slices keep the 16-byte grid
        if k:
            assert parts[k - 1][1] == br0 and parts[k - 1][3] == off0
    assert parts[0][2] == 0 and parts[-1][3] == _tri(N)
    return [p for p in parts if p[1] > p[0]]  # ranks with no block row get nothing to do


@pytest.mark.parametrize("mapping", ["LTM", "BB"])
@pytest.mark.parametrize("N,rho", [(16384, 8), (16384, 16), (5000, 16), (3001, 32)])
def test_probe_slices_rebuild_the_triangle(mapping, N, rho):
    whole, _ = td.td_map_probe(mapping, "chunked", N, rho)
    want = oracle.probe(N)
    for G in (2, 3, 8):
        full = torch.full((_tri(N),), -1, dtype=torch.int32, device="cuda")
        for br0, br1, off0, off1 in _slices(N, rho, G):
            _, st = td.td_map_probe_rows(mapping, N, rho, br0, br1, full[off0:off1])
            assert st["useful_blocks"] == _tri(br1) - _tri(br0)
            assert st["blocks"] == (st["useful_blocks"] if mapping == "LTM" else (br1 - br0) * (-(-N // rho)))
        assert torch.equal(full, whole[: _tri(N)]), (mapping, N, rho, G)
        assert np.array_equal(full.cpu().numpy().view(np.uint32), want)


def test_probe_slices_full_size():
    """The N = 65536 triangle of the benchmark (8.6 GB), 8 slices, against the whole launch."""
    N, rho = 65536, 16
    whole, _ = td.td_map_probe("LTM", "chunked", N, rho)
    full = torch.empty(_tri(N), dtype=torch.int32, device="cuda")
    for br0, br1, off0, off1 in _slices(N, rho, 8):
        td.td_map_probe_rows("LTM", N, rho, br0, br1, full[off0:off1])
    assert torch.equal(full, whole[: _tri(N)])
    del full, whole


@pytest.mark.parametrize("sched,rho,d", [("chunked", 16, 3), ("chunked", 8, 1), ("persistent", 128, 16),
                                         ("grid", 64, 64)])
@pytest.mark.parametrize("mapping", ["LTM", "BB"])
def test_edm_slices_rebuild_the_map(mapping, sched, rho, d):
    n = 5000
    xh = synth.uniform_points(n, d, 8100 + d)
    x = torch.from_numpy(xh).cuda()
    whole, _ = td.td_edm(mapping, sched, x, rho)
    want = oracle.edm(xh)
    for G in (2, 3, 8):
        full = torch.full((_tri(n),), float("nan"), dtype=torch.float32, device="cuda")
        for br0, br1, off0, off1 in _slices(n, rho, G):
            td.td_edm_rows(mapping, sched, x, rho, br0, br1, full[off0:off1])
        assert torch.equal(full, whole[: _tri(n)]), (mapping, sched, rho, d, G)
    got = full.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - want) <= RTOL * want + 1e-30)


@pytest.mark.parametrize("mapping", ["LTM", "BB"])
def test_collision_slices_rebuild_the_table(mapping):
    c, r = synth.spheres(3000, seed=17, coord_bits=12, rmin=0, rmax=200)
    ct, rt = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    n = r.size
    words = td.td_collide_words(n)
    whole, _ = td.td_collide(mapping, "persistent", ct, rt)
    want = oracle.collide(c, r)
    assert np.array_equal(whole[:words].cpu().numpy().view(np.uint32), want)
    nt = -(-n // 32)
    for G in (2, 3, 8):
        full = torch.full((words,), -1, dtype=torch.int32, device="cuda")
        for br0, br1, _, _ in _slices(n, 64, G):   # block rows of 64 spheres: two tile rows each
            w0, w1 = 32 * _tri(min(2 * br0, nt)), 32 * _tri(min(2 * br1, nt))
            td.td_collide_rows(mapping, "persistent", ct, rt, br0, br1, full[w0:w1])
        assert torch.equal(full, whole[:words]), (mapping, G)


def test_slice_arguments_rejected():
    out = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    for args in [("LTM", 1024, 16, 3, 3), ("LTM", 1024, 16, 5, 2), ("LTM", 1024, 16, 0, 65), ("UTM", 1024, 16, 0, 1),
                 ("REC", 1024, 16, 0, 1), ("LTM", 1024, 64, 0, 1)]:
        with pytest.raises(td.TDError):
            td.td_map_probe_rows(*args, out=out)
    x = torch.zeros(100, 4, device="cuda")
    with pytest.raises(td.TDError):
        td.td_edm_rows("LTM", "chunked", x, 128, 0, 1)     # the chunked body takes rho <= 32
    with pytest.raises(td.TDError):
        td.td_edm_rows("LTM", "persistent", x, 16, 0, 1)   # one element per thread: no slices
