"""GPU parity of the mapping kernels (Sec. II-A g(lambda); Sec. III-B BB, UTM, RB, REC)
against the CPU oracle: the probe output must be bit-exact, identical across all five
strategies (Sec. IV: "the output for each strategy ... always correct and the same"), and
every in-domain element must be hit exactly once."""
import functools

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402

STRATS = ["BB", "UTM", "RB", "REC", "LTM", "UTM-BLOCK"]
SCHEDS = ["grid", "persistent"]
SENTINEL = -559038737  # 0xDEADBEEF


@functools.lru_cache(maxsize=None)
def _oracle_probe(N):
    return oracle.probe(N)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _supported(strategy, N, rho, sched="grid"):
    if sched == "chunked" and strategy not in ("LTM", "BB", "REC", "UTM-BLOCK"):
        return False
    return not (strategy == "REC" and (N == 0 or N % rho))


def _first_diff(a, b):
    idx = np.flatnonzero(a != b)
    return None if idx.size == 0 else (int(idx[0]), int(a[idx[0]]), int(b[idx[0]]), int(idx.size))


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("sched", SCHEDS + ["chunked"])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_probe_matches_oracle_small(strategy, sched, rho):
    if not _supported(strategy, 1024, rho, sched):
        with pytest.raises(td.TDError):
            td.td_map_probe(strategy, sched, 1024, rho)
        return
    for N in [1, 2, 3, 4, 5, 7, 8, 33, 100, 255, 256, 1000, 1024, 3000, 4096]:
        if not _supported(strategy, N, rho, sched):
            continue
        out = torch.full((td.td_tri_size(N),), SENTINEL, dtype=torch.int32, device="cuda")
        _, st = td.td_map_probe(strategy, sched, N, rho, out)
        got = _u32(out)
        assert _first_diff(got, _oracle_probe(N)) is None, (strategy, sched, rho, N, _first_diff(got, _oracle_probe(N)))
        ref = td.td_plan(strategy, sched, N, rho)
        assert st["blocks"] == ref["blocks"] and st["useful_blocks"] == ref["useful_blocks"]
        if sched == "grid":
            assert st["ctas"] == st["blocks"]


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("sched", SCHEDS + ["chunked"])
def test_cover_exactly_once_small(strategy, sched):
    for rho in [8, 16, 32]:
        for N in [1, 5, 64, 129, 1000, 2048]:
            if not _supported(strategy, N, rho, sched):
                continue
            cnt = td.td_map_cover(strategy, sched, N, rho)
            c = cnt.cpu().numpy()
            assert c.size == td.td_tri_size(N) and np.all(c == 1), (strategy, sched, rho, N)


@pytest.mark.parametrize("sched", ["persistent", "chunked"])
def test_probe_full_size_ltm_against_oracle(sched):
    """N = 65536, the largest probe size: the full triangle (8.6 GB) against the oracle."""
    N = 65536
    out = torch.full((td.td_tri_size(N),), SENTINEL, dtype=torch.int32, device="cuda")
    td.td_map_probe("LTM", sched, N, 16, out)
    torch.cuda.synchronize()
    rows = 4096
    for i0 in range(0, N, rows):
        a, b = td.td_tri_size(i0), td.td_tri_size(i0 + rows)
        got = out[a:b].cpu().numpy().view(np.uint32)
        want = oracle.probe(N, i0, i0 + rows)
        assert _first_diff(got, want) is None, (i0, _first_diff(got, want))


@pytest.mark.parametrize("rho", [8, 16, 32])
def test_probe_full_size_all_strategies_identical(rho):
    """Every strategy and schedule writes the same 8.6 GB triangle at N = 65536; sampled
    rows are checked against the oracle and the whole array against the g(lambda) output."""
    N = 65536
    total = td.td_tri_size(N)
    ref = torch.empty(total, dtype=torch.int32, device="cuda")
    td.td_map_probe("LTM", "grid", N, rho, ref)
    rng = np.random.default_rng(rho)
    for i in list(rng.integers(0, N, 16)) + [0, N - 1]:
        i = int(i)
        got = ref[td.td_tri_size(i): td.td_tri_size(i + 1)].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.probe(N, i, i + 1)), i
    out = torch.empty_like(ref)
    for strategy in STRATS:
        for sched in SCHEDS + ["chunked"]:
            if not _supported(strategy, N, rho, sched):
                continue
            out.fill_(SENTINEL)
            td.td_map_probe(strategy, sched, N, rho, out)
            assert torch.equal(out, ref), (strategy, sched, rho)


@pytest.mark.parametrize("strategy", STRATS)
def test_cover_full_size(strategy):
    N, rho = 65536, 16
    cnt = td.td_map_cover(strategy, "persistent", N, rho)
    assert bool((cnt == 1).all()), strategy


@pytest.mark.parametrize("strategy,rho", [("LTM", 8), ("LTM", 16), ("LTM", 32), ("BB", 16), ("UTM-BLOCK", 16),
                                          ("REC", 16)])
def test_cover_chunked_full_size(strategy, rho):
    """The chunked schedule at N = 65536 (wide strips, runs capped at W / rho): each element once."""
    cnt = td.td_map_cover(strategy, "chunked", 65536, rho)
    assert bool((cnt == 1).all()), (strategy, rho)
    del cnt
    torch.cuda.empty_cache()


@pytest.mark.parametrize("strategy", ["LTM", "BB", "UTM-BLOCK"])
def test_cover_chunked_ragged(strategy):
    for rho in [8, 16, 32]:
        for N in [4097, 12345, 30001]:
            cnt = td.td_map_cover(strategy, "chunked", N, rho)
            assert bool((cnt == 1).all()), (strategy, rho, N)


def test_ltm_fast_g_exhaustive_below_2_32():
    res = td.td_ltm_check(0, 2**32)
    r = res.cpu().numpy().view(np.uint64)
    assert r[0] == 0, f"first failing lambda {r[1]}"


def test_ltm_fast_g_windows_up_to_2_40():
    for lo in [2**33, 2**36, 2**38, 2**39, 2**40 - 2**32]:
        r = td.td_ltm_check(lo, 2**32).cpu().numpy().view(np.uint64)
        assert r[0] == 0, (lo, r[1])


def test_ltm_dump_matches_exact_g():
    rng = np.random.default_rng(1)
    lam = np.unique(np.concatenate([
        rng.integers(0, 2**40, 200000, dtype=np.uint64),
        np.array([r * (r + 1) // 2 + o for r in rng.integers(1, 1_482_900, 20000) for o in (-1, 0)], dtype=np.uint64),
    ]))
    # contiguous windows
    for u0, cnt in [(0, 1 << 20), (2**40 - (1 << 20), 1 << 20), (123456789012, 1 << 16)]:
        ij = td.td_map_dump("LTM", 0, u0, cnt)
        got = ij[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
        want = oracle.ltm(np.arange(u0, u0 + cnt, dtype=np.uint64))
        assert np.array_equal(got, want), u0
    # scattered values, one dump call per value block
    for v in lam[::997]:
        got = td.td_map_dump("LTM", 0, int(v), 1)[:2].cpu().numpy().view(np.uint32)
        assert tuple(got) == tuple(oracle.ltm(int(v))[0]), int(v)


def test_utm_dump_matches_oracle():
    for N in [1, 2, 100, 1023, 65536]:
        total = td.td_tri_size(N)
        rng = np.random.default_rng(N)
        cnt = min(total, 1 << 20)
        for u0 in {0, max(0, total - cnt), int(rng.integers(0, max(total - cnt, 1)))}:
            ij = td.td_map_dump("UTM", N, u0, cnt)
            got = ij[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
            want = oracle.utm_lower(N, np.arange(u0, u0 + cnt, dtype=np.uint64))
            assert np.array_equal(got, want), (N, u0)


def test_rb_dump_matches_oracle():
    for N in [1, 2, 3, 8, 101, 1024]:
        W, H = oracle.rb_dims(N)
        cnt = W * H
        got = td.td_map_dump("RB", N, 0, cnt)[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
        for u in range(0, cnt, max(1, cnt // 5000)):
            assert tuple(got[u]) == oracle.rb_map(N, u % W, u // W), (N, u)


def test_utm_block_dump_matches_oracle_formula():
    """Block-level UTM (rsqrt estimate + integer fix-up) equals the exact UTM formula of the
    oracle at every block index of several block triangles, and on random indices of large ones."""
    rng = np.random.default_rng(5)
    for nb in [1, 2, 3, 17, 64, 1000, 1920, 8192]:
        total = nb * (nb + 1) // 2
        cnt = min(total, 1 << 21)
        got = td.td_map_dump("UTM-BLOCK", nb, 0, cnt)[: 2 * cnt].cpu().numpy().view(np.uint32).reshape(-1, 2)
        assert np.array_equal(got, oracle.utm_lower(nb, np.arange(cnt, dtype=np.uint64))), nb
    for nb in [65535, 1 << 20, (1 << 30) - 1]:
        total = nb * (nb + 1) // 2
        for u0 in [0, total // 3, total - 4096] + [int(v) for v in rng.integers(0, total - 4096, 4)]:
            got = td.td_map_dump("UTM-BLOCK", nb, u0, 4096)[: 8192].cpu().numpy().view(np.uint32).reshape(-1, 2)
            want = oracle.utm_lower(nb, np.arange(u0, u0 + 4096, dtype=np.uint64))
            assert np.array_equal(got, want), (nb, u0)


def test_utm_thread_dump_large_n():
    """Thread-level UTM near its limit N < 2^30, where the FP32 estimate can be rows off."""
    rng = np.random.default_rng(9)
    for N in [1 << 22, (1 << 26) + 3, (1 << 30) - 1]:
        total = N * (N + 1) // 2
        for u0 in [0, total - 4096] + [int(v) for v in rng.integers(0, total - 4096, 4)]:
            got = td.td_map_dump("UTM", N, u0, 4096)[: 8192].cpu().numpy().view(np.uint32).reshape(-1, 2)
            want = oracle.utm_lower(N, np.arange(u0, u0 + 4096, dtype=np.uint64))
            assert np.array_equal(got, want), (N, u0)
