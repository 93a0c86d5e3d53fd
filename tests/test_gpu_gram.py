"""GPU checks of the Gram-form distance map (BF16 inner products on tcgen05, FP32 norms, FP32
direct recompute of cancelling pairs) against the FP64 oracle.

Error model of the Gram path: with BF16 rounding |delta| <= 2^-9 on each coordinate and FP32
accumulation, |D_gram^2 - D^2| <= 2^-7 sum_k |x_ik x_jk| + 2^-20 (|x_i|^2 + |x_j|^2) for every
pair; pairs with D^2 < 1e-2 (|x_i|^2 + |x_j|^2) are recomputed in the direct form and held to
the FP32 tolerance 2e-6."""
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


def _check_pairs(xh, out, ii, jj):
    x64 = xh.astype(np.float64)
    want = oracle.edm_pairs(xh, ii, jj)
    pos = torch.from_numpy(ii.astype(np.int64) * (ii.astype(np.int64) + 1) // 2 + jj).cuda()
    got = out[pos].cpu().numpy().astype(np.float64)
    nsum = (x64[ii] ** 2).sum(1) + (x64[jj] ** 2).sum(1)
    absdot = np.abs(x64[ii] * x64[jj]).sum(1)
    bound_d2 = 2.0 ** -7 * absdot + 2.0 ** -20 * nsum
    # a bound on |D_gram - D| from the bound on the squares: |a - b| <= |a^2 - b^2| / (a + b)
    err = np.abs(got - want)
    gram_ok = err * (got + want) <= bound_d2 * 1.0001 + 1e-30
    direct_ok = err <= RTOL * want + 1e-30
    assert np.all(gram_ok | direct_ok), int((~(gram_ok | direct_ok)).sum())
    surely_recomputed = want ** 2 < 1e-3 * nsum
    assert np.all(direct_ok[surely_recomputed])
    rel = err / np.maximum(want, 1e-30)
    return float(rel.max()), float(np.sqrt((rel ** 2).mean()))


@pytest.mark.parametrize("n,d", [(1, 8), (37, 8), (128, 64), (300, 64), (257, 200), (640, 256), (300, 520), (200, 1024),
                                 (130, 8192)])
def test_gram_small_all_pairs(n, d):
    xh = synth.uniform_points(n, d, 7000 + n + d)
    xh[n // 3] = xh[n // 5]  # a duplicated point: distance exactly 0 through the recompute
    x = torch.from_numpy(xh).cuda()
    out, ws = td.td_edm_gram(x)
    fb = td.td_edm_gram_status(ws)
    ii, jj = np.tril_indices(n)
    _check_pairs(xh, out, ii.astype(np.uint32), jj.astype(np.uint32))
    diag = torch.arange(n, device="cuda", dtype=torch.int64)
    assert bool((out[diag * (diag + 1) // 2 + diag] == 0).all())
    assert fb >= n  # the diagonal always takes the direct form


def test_gram_precision_workload():
    """n = 16384, d = 256, 64 Gaussian clusters: sampled pairs against the FP64 oracle, the
    recomputed fraction (~1/64 of the pairs: the same-cluster ones), and the diagonal."""
    xh = synth.clustered_points()
    n = xh.shape[0]
    x = torch.from_numpy(xh).cuda()
    out, ws = td.td_edm_gram(x)
    fb = td.td_edm_gram_status(ws)
    total = n * (n + 1) // 2
    assert 0.5 / 64 * total < fb < 2.0 / 64 * total, fb
    rng = np.random.default_rng(31)
    ii = rng.integers(0, n, 300000).astype(np.uint32)
    jj = (rng.random(300000) * (ii + 1)).astype(np.uint32)
    mx, rms = _check_pairs(xh, out, ii, jj)
    assert mx < 1e-2
    diag = torch.arange(n, device="cuda", dtype=torch.int64)
    assert bool((out[diag * (diag + 1) // 2 + diag] == 0).all())
    # where the Gram form cancels, the recomputed value agrees with the FP32 direct kernel
    ref, _ = td.td_edm("LTM", "persistent", x, 128)
    close = (ref < 0.1 * torch.sqrt(torch.tensor(2.0 * 256)))
    assert torch.allclose(out[close], ref[close], rtol=4e-6, atol=0)


@pytest.mark.parametrize("n,d", [(4096, 64), (2048, 256)])
def test_gram_queue_regions_half_full(n, d):
    """16 clusters: 1/16 of the pairs cancel, twice what a queue region holds (1/32 of its block
    quarter's pairs).  In the same warp some cancelling pairs then land in the queue and the rest
    are recomputed by the epilogue itself; both must meet the FP32 tolerance.  d = 64 and d = 256
    run the two forms of the main pass."""
    xh = synth.clustered_points(n, d, clusters=16, sigma=0.05, seed=9100 + d)
    x = torch.from_numpy(xh).cuda()
    out, ws = td.td_edm_gram(x)
    fb = td.td_edm_gram_status(ws)
    total = n * (n + 1) // 2
    assert 0.5 / 16 * total < fb < 2.0 / 16 * total, fb
    rng = np.random.default_rng(d)
    ii = rng.integers(0, n, 200000).astype(np.uint32)
    jj = (rng.random(200000) * (ii + 1)).astype(np.uint32)
    _check_pairs(xh, out, ii, jj)
    # every pair that cancels takes the direct form, queued or not: against the FP32 direct kernel
    ref, _ = td.td_edm("LTM", "persistent", x, 128)
    close = ref < 0.1 * torch.sqrt(torch.tensor(2.0 * d))
    assert int(close.sum()) > 0.5 / 16 * total
    assert torch.allclose(out[: total][close[: total]], ref[: total][close[: total]], rtol=4e-6, atol=0)


def test_gram_rejects():
    x = torch.zeros(10, 12, device="cuda")
    with pytest.raises(td.TDError):
        td.td_edm_gram(x)                                  # d not a multiple of 8
    x = torch.zeros(10, 8200, device="cuda")
    with pytest.raises(td.TDError):
        td.td_edm_gram(x)                                  # d > 8192


def test_gram_queue_overflow_identical_points():
    """Every pair of identical points cancels: far more pairs than the recompute queue holds, so
    the epilogue recomputes the overflow itself.  All distances must be exactly 0."""
    n, d = 2048, 64
    row = synth.uniform_points(1, d, 5)
    x = torch.from_numpy(np.repeat(row, n, axis=0)).cuda()
    out, ws = td.td_edm_gram(x)
    fb = td.td_edm_gram_status(ws)
    assert fb == n * (n + 1) // 2
    assert bool((out[: n * (n + 1) // 2] == 0).all())
