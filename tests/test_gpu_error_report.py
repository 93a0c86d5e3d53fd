"""Max and RMS relative error against the FP64 oracle for every floating-point workload (plain
EDM, the FP32 direct form at d = 256, the Gram form, the batched form, the chunked and strict
forms), each held to its bound and printed as one JSON line (visible with pytest -s)."""
import json

import numpy as np
import pytest

import oracle
from paper_1308_1419_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402


def _rel(got, want):
    got = np.asarray(got, dtype=np.float64)
    rel = np.abs(got - want) / np.maximum(want, 1e-30)
    rel[want == 0] = np.abs(got[want == 0])
    return float(rel.max()), float(np.sqrt((rel ** 2).mean()))


def _sample(n, count, seed):
    rng = np.random.default_rng(seed)
    ii = rng.integers(0, n, count).astype(np.uint32)
    jj = (rng.random(count) * (ii.astype(np.float64) + 1)).astype(np.uint32)
    return ii, jj


def _report(name, mx, rms, bound):
    print(json.dumps({"workload": name, "max_rel": mx, "rms_rel": rms, "bound": bound}))
    assert mx <= bound, (name, mx)


def test_plain_edm_errors():
    xh = synth.plain_edm()
    x = torch.from_numpy(xh).cuda()
    want = oracle.edm(xh)
    for sched in ("grid", "chunked"):
        got, _ = td.td_edm("LTM", sched, x, 16)
        _report(f"plain EDM n=2048 d=3 LTM {sched}", *_rel(got[: want.size].cpu().numpy(), want), 2e-6)


def test_precision_workload_errors():
    xh = synth.clustered_points()
    n = xh.shape[0]
    x = torch.from_numpy(xh).cuda()
    ii, jj = _sample(n, 300000, 41)
    want = oracle.edm_pairs(xh, ii, jj)
    pos = torch.from_numpy(ii.astype(np.int64) * (ii.astype(np.int64) + 1) // 2 + jj).cuda()
    direct, _ = td.td_edm("LTM", "persistent", x, 128)
    _report("precision n=16384 d=256 FP32 direct", *_rel(direct[pos].cpu().numpy(), want), 2e-6)
    gram, _ = td.td_edm_gram(x)
    _report("precision n=16384 d=256 BF16 Gram + FP32 recompute", *_rel(gram[pos].cpu().numpy(), want), 1e-2)


def test_batched_errors():
    ns, ds, xh = synth.batched_problems()
    x = torch.from_numpy(xh).cuda()
    out, _, _ = td.td_edm_batched(ns, ds, x)
    xo = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * ds)])
    oo = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * (ns.astype(np.int64) + 1) // 2)])
    mx, sq, cnt = 0.0, 0.0, 0
    for p in range(0, len(ns), 5):
        n, d = int(ns[p]), int(ds[p])
        ii, jj = _sample(n, 4000, p)
        want = oracle.edm_pairs(xh[xo[p]: xo[p + 1]].reshape(n, d), ii, jj)
        pos = torch.from_numpy(oo[p] + ii.astype(np.int64) * (ii.astype(np.int64) + 1) // 2 + jj).cuda()
        m, r = _rel(out[pos].cpu().numpy(), want)
        mx, sq, cnt = max(mx, m), sq + r * r * ii.size, cnt + ii.size
    _report("batched 512 problems (every 5th, 4000 pairs each)", mx, float(np.sqrt(sq / cnt)), 2e-6)


def test_store_bound_forms_errors():
    n, d = 32768, 3
    xh = synth.uniform_points(n, d, 4244)
    x = torch.from_numpy(xh).cuda()
    ii, jj = _sample(n, 300000, 43)
    want = oracle.edm_pairs(xh, ii, jj)
    pos = torch.from_numpy(ii.astype(np.int64) * (ii.astype(np.int64) + 1) // 2 + jj).cuda()
    got, _ = td.td_edm("LTM", "chunked", x, 16)
    _report("EDM n=32768 d=3 chunked", *_rel(got[pos].cpu().numpy(), want), 2e-6)
    keep = ii > jj
    strict = td.td_edm_strict(x)
    k = torch.from_numpy(ii[keep].astype(np.int64) * (ii[keep].astype(np.int64) - 1) // 2 + jj[keep]).cuda()
    _report("strict EDM n=32768 d=3", *_rel(strict[k].cpu().numpy(), want[keep]), 2e-6)
