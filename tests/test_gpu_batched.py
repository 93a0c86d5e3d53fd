"""GPU parity of the batched distance map: every problem's slice equals a stand-alone td_edm
call bit for bit and the FP64 oracle within 2e-6; the split plan/run form captures in a CUDA
graph; the autotuner returns a working configuration."""
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


def _offsets(ns, ds):
    xo = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * ds)])
    oo = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * (ns.astype(np.int64) + 1) // 2)])
    return xo, oo


def _check_rel(got, want, ctx):
    err = np.abs(np.asarray(got, np.float64) - want)
    assert not (err > RTOL * want + 1e-30).any(), ctx


@pytest.mark.parametrize("rho", [64, 128])
def test_batched_small_against_oracle_and_td_edm(rho):
    ns, ds, xh = synth.batched_problems(nprob=23, nmin=1, ratio=400.0, dims=(1, 3, 5, 16, 64), seed=99)
    x = torch.from_numpy(xh).cuda()
    out, ws, st = td.td_edm_batched(ns, ds, x, config=(rho, 0))
    xo, oo = _offsets(ns, ds)
    want = oracle.edm_batched(xh, ns, ds)
    got = out[: oo[-1]].cpu().numpy()
    _check_rel(got, want, rho)
    for p, (n, d) in enumerate(zip(ns, ds)):
        xp = x[xo[p]: xo[p + 1]].view(int(n), int(d)).clone()
        ref, _ = td.td_edm("LTM", "persistent", xp, 16)
        assert torch.equal(out[oo[p]: oo[p + 1]], ref[: oo[p + 1] - oo[p]]), p


def test_batched_workload_512_problems():
    """512 problems, n log-uniform in [64, 8192), d in {3, 16, 64}: the batched workload."""
    ns, ds, xh = synth.batched_problems()
    x = torch.from_numpy(xh).cuda()
    out, ws, st = td.td_edm_batched(ns, ds, x)
    xo, oo = _offsets(ns, ds)
    assert st["launches"] == 1
    rng = np.random.default_rng(0)
    for p in range(0, 512, 7):
        n, d = int(ns[p]), int(ds[p])
        xp = x[xo[p]: xo[p + 1]].view(n, d).clone()
        ref, _ = td.td_edm("LTM", "persistent", xp, 16 if d < 16 else 128)
        assert torch.equal(out[oo[p]: oo[p + 1]], ref[: oo[p + 1] - oo[p]]), p
        ii = rng.integers(0, n, 2000).astype(np.uint32)
        jj = (rng.random(2000) * (ii + 1)).astype(np.uint32)
        pos = torch.from_numpy(oo[p] + ii.astype(np.int64) * (ii + 1) // 2 + jj).cuda()
        _check_rel(out[pos].cpu().numpy(), oracle.edm_pairs(xh[xo[p]: xo[p + 1]].reshape(n, d), ii, jj), p)


def test_batched_graph_capture_and_autotune():
    ns, ds, xh = synth.batched_problems(nprob=64, seed=7)
    x = torch.from_numpy(xh).cuda()
    xs, os_ = td.batched_sizes(ns, ds)
    ref, ws, _ = td.td_edm_batched(ns, ds, x, config=(64, 0))
    (rho, cps), ms = td.td_edm_batched_autotune(ns, ds, x, torch.empty_like(ref), ws)
    assert rho in (64, 128) and 0 <= cps <= 4 and ms > 0
    total = td.td_edm_batched_plan(ns, ds, rho, ws)
    out = torch.zeros_like(ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        td.td_edm_batched_run(len(ns), rho, total, x, out, ws, cps, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert torch.equal(out[:os_], ref[:os_])
    g = torch.cuda.CUDAGraph()
    out.zero_()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        td.td_edm_batched_run(len(ns), rho, total, x, out, ws, cps)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out[:os_], ref[:os_])


def test_batched_default_config_matches_both_block_sides():
    """cfg NULL (rho = 128) and an explicit rho = 64 give the same bits: the block side changes
    the schedule, never a sum."""
    ns, ds, xh = synth.batched_problems(nprob=48, seed=11)
    x = torch.from_numpy(xh).cuda()
    _, os_ = td.batched_sizes(ns, ds)
    dflt, _, st = td.td_edm_batched(ns, ds, x)
    r64, _, _ = td.td_edm_batched(ns, ds, x, config=(64, 0))
    r128, _, _ = td.td_edm_batched(ns, ds, x, config=(128, 0))
    torch.cuda.synchronize()
    assert torch.equal(dflt[:os_], r128[:os_]) and torch.equal(dflt[:os_], r64[:os_])


def test_batched_rejects():
    x = torch.zeros(16, device="cuda")
    with pytest.raises(td.TDError):
        td.td_edm_batched([2, 0], [3, 3], x)           # empty problem
    with pytest.raises(td.TDError):
        td.td_edm_batched([2], [3], x, config=(32, 0))  # rho must be 64 or 128
