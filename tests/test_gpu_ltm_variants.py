"""GPU parity of the FP32 evaluations of g that Sec. III-A times (LTM-X, LTM-N, LTM-R): the
device dump of LTM-X and LTM-N (rounded per operation, and as a compiler contracts it into fused
multiply-adds) equals the oracle's FP32 definitions bit for bit, the device
check finds the oracle's first failing lambda, and the probe driven by a variant is exact below
that lambda and misses elements above it.  LTM-R rests on the device's reciprocal square root,
so its first failure is checked for consistency: a genuine failure, with none before it."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402

VARIANT = {"LTM-X": oracle.LTM_X, "LTM-N": oracle.LTM_N, "LTM-N-FMA": oracle.LTM_N_FMA}


def _row(lam):
    return (math.isqrt(8 * lam + 1) - 1) // 2


def _dump(mapping, lams):
    out = np.empty((0, 2), dtype=np.uint32)
    for a, b in lams:
        ij = td.td_map_dump(mapping, 0, a, b - a)[: 2 * (b - a)].cpu().numpy().view(np.uint32).reshape(-1, 2)
        out = np.concatenate([out, ij])
    return out


def _check(mapping, lam0, count):
    r = td.td_ltm_variant_check(mapping, lam0, count).cpu().tolist()
    return int(r[0]), int(r[1]) & (2**64 - 1)


@pytest.mark.parametrize("mapping", ["LTM-X", "LTM-N", "LTM-N-FMA"])
def test_variant_dump_matches_oracle_fp32(mapping):
    v = VARIANT[mapping]
    first = oracle.ltm_variant_first_fail(v, 0, 1 << 26)
    ranges = [(0, 1 << 16), (first - 5000, first + 5000), (oracle.tri(3000) - 3000, oracle.tri(3000) + 3000)]
    got = _dump(mapping, ranges)
    lams = [lam for a, b in ranges for lam in range(a, b)]
    want = np.array([oracle.ltm_variant(v, lam) for lam in lams], dtype=np.uint32)
    assert np.array_equal(got, want), mapping


@pytest.mark.parametrize("mapping", ["LTM-X", "LTM-N", "LTM-N-FMA"])
def test_variant_check_finds_oracle_first_failure(mapping):
    first = oracle.ltm_variant_first_fail(VARIANT[mapping], 0, 1 << 26)
    bad, f = _check(mapping, 0, 1 << 26)
    assert f == first and bad >= 1
    assert _check(mapping, 0, first) == (0, 2**64 - 1)


def test_exact_g_and_ltm_r_checks():
    assert _check("LTM", 0, 1 << 32) == (0, 2**64 - 1)      # the fix-up: exact throughout
    bad, f = _check("LTM-R", 0, 1 << 32)
    if bad:                                                 # a genuine failure, none before it
        i, j = (int(v) for v in _dump("LTM-R", [(f, f + 1)])[0])
        r = _row(f)
        assert (i, j) != (r, f - oracle.tri(r))
        assert _check("LTM-R", 0, f) == (0, 2**64 - 1)


@pytest.mark.parametrize("mapping", ["LTM-X", "LTM-N", "LTM-N-FMA", "LTM-R"])
def test_variant_probe_exact_below_first_failure(mapping):
    N, rho = 4096, 16                                       # lambda < T(256): below every failure
    want = oracle.probe(N)
    for sched in ("grid", "persistent"):
        out, st = td.td_map_probe(mapping, sched, N, rho)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want), (mapping, sched)
        assert st["blocks"] == oracle.tri(N // rho) and st["wasted_blocks"] == 0


def test_variant_probe_misses_elements_past_first_failure():
    """N = 16384, rho = 8: lambda reaches T(2048) - 1, past LTM-N's first failure; the blocks it
    maps to the wrong row leave their elements unwritten (the kernels' guards keep every store
    inside the triangle), while the exact g writes every element."""
    N, rho = 16384, 8
    assert oracle.ltm_variant_first_fail(oracle.LTM_N, 0, oracle.tri(N // rho)) < oracle.tri(N // rho)
    sentinel = -559038737
    exact = torch.full((oracle.tri(N),), sentinel, dtype=torch.int32, device="cuda")
    td.td_map_probe("LTM", "grid", N, rho, exact)
    assert int((exact == sentinel).sum()) == 0
    variant = torch.full((oracle.tri(N),), sentinel, dtype=torch.int32, device="cuda")
    td.td_map_probe("LTM-N", "grid", N, rho, variant)
    assert int((variant == sentinel).sum()) > 0


def test_variants_rejected_elsewhere():
    x = torch.zeros(64, 3, device="cuda")
    for mapping in ("LTM-X", "LTM-N", "LTM-N-FMA", "LTM-R"):
        with pytest.raises(td.TDError):
            td.td_edm(mapping, "grid", x, 16)
        with pytest.raises(td.TDError):
            td.td_map_probe(mapping, "chunked", 1024, 16)


@pytest.mark.parametrize("mapping", ["BB", "UTM", "RB", "REC", "LTM", "LTM-X", "LTM-N", "LTM-N-FMA", "LTM-R"])
def test_dummy_kernel_maps_and_writes_nothing(mapping):
    """The map-only dummy kernel: every strategy launches its plan's blocks and leaves the sink."""
    sentinel = 12345
    for N, rho in ((1024, 16), (3000, 8)):
        if mapping == "REC" and N % rho:
            continue
        for sched in ("grid", "persistent"):
            sink = torch.full((4,), sentinel, dtype=torch.int32, device="cuda")
            _, st = td.td_map_dummy(mapping, sched, N, rho, sink)
            torch.cuda.synchronize()
            assert int(sink[0]) == sentinel, (mapping, sched)
            assert st == td.td_plan(mapping, sched, N, rho) | {"ctas": st["ctas"]}


def test_ltm_n_fma_probe_exact_over_the_papers_range():
    """Sec. III-A: LTM-N with its epsilon is exact for N up to 30720 at rho = 16.  The contracted
    evaluation writes that whole triangle correctly through the probe, under both schedules, and
    the device check finds no failure over its block indices; the per-operation rounding fails there."""
    N, rho = 30720, 16
    want = oracle.probe(N)
    for sched in ("grid", "persistent"):
        out, _ = td.td_map_probe("LTM-N-FMA", sched, N, rho)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want), sched
    assert _check("LTM-N-FMA", 0, oracle.tri(N // rho)) == (0, 2**64 - 1)
    assert _check("LTM-N", 0, oracle.tri(N // rho))[0] > 0
