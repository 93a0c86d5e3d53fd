"""CPU checks of the C ABI: the library builds and loads, exports every entry point the
header declares, and its host-only logic (sizes, launch planning, argument validation)
agrees with the oracle's closed forms -- all without a GPU."""
import ctypes as C
import os
import re

import pytest

import oracle
from paper_1308_1419_gb300.build import INCLUDE, build_libtd

build_libtd()
from paper_1308_1419_gb300 import td  # noqa: E402

HEADER = os.path.join(INCLUDE, "td.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(td_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported():
    names = _declared_functions()
    assert "td_map_probe" in names and "td_last_error" in names
    for name in names:
        assert hasattr(td.lib, name), f"{name} declared in td.h but not exported"


def test_sizes():
    for N in [0, 1, 2, 3, 1000, 65536, 2**32 - 1]:
        assert td.td_tri_size(N, True) == N * (N + 1) // 2
        assert td.td_tri_size(N, False) == N * (N - 1) // 2 if N else td.td_tri_size(N, False) == 0
    for n in [0, 1, 31, 32, 33, 32768, 100000]:
        assert td.td_collide_words(n) == oracle.collide_words(n)


@pytest.mark.parametrize("strategy", ["BB", "LTM", "UTM", "RB", "REC", "UTM-BLOCK"])
@pytest.mark.parametrize("N,rho", [(1, 8), (100, 8), (1024, 16), (1000, 8), (768, 16), (2048, 32)])
def test_plan_matches_oracle_launch_space(strategy, N, rho):
    if strategy == "REC" and N % rho:
        with pytest.raises(td.TDError) as e:
            td.td_plan(strategy, "grid", N, rho)
        assert e.value.status == 2
        return
    _, ref = oracle.cover(strategy, N, rho)
    got = td.td_plan(strategy, "grid", N, rho)
    assert got["blocks"] == ref["launched"]
    assert got["useful_blocks"] == ref["useful"]
    assert got["wasted_blocks"] == ref["launched"] - ref["useful"]
    assert got["launches"] == ref["launches"]
    assert got["ctas"] == got["blocks"]


def test_plan_paper_waste_counts():
    # Sec. II-A: BB wastes n(n-1)/2 blocks; g(lambda) launches exactly n(n+1)/2 (none idle).
    for N, rho in [(65536, 16), (30720, 16), (65536, 8)]:
        n = -(-N // rho)
        bb = td.td_plan("BB", "grid", N, rho)
        lt = td.td_plan("LTM", "grid", N, rho)
        assert bb["blocks"] == n * n and bb["wasted_blocks"] == n * (n - 1) // 2
        assert lt["blocks"] == n * (n + 1) // 2 and lt["wasted_blocks"] == 0


def test_argument_errors_return_before_launch():
    st = td.td_launch_stats()
    assert td._c_map_probe(4, 1, 1024, 7, 256, C.byref(st), None) == 1       # bad rho
    assert "rho" in td._c_last_error().decode()
    assert td._c_map_probe(4, 1, 1024, 16, None, C.byref(st), None) == 1     # NULL output
    assert td._c_map_probe(4, 1, 1024, 16, 8, C.byref(st), None) == 1        # misaligned
    assert td._c_map_probe(3, 1, 100, 8, 256, C.byref(st), None) == 2        # REC needs N % rho == 0
    assert td._c_map_probe(10, 1, 100, 8, 256, C.byref(st), None) == 1       # unknown mapping
    assert td._c_map_probe(4, 5, 100, 8, 256, C.byref(st), None) == 1        # unknown schedule
    assert td._c_map_probe(4, 1, 0, 16, None, C.byref(st), None) == 0        # N = 0 is a no-op
    assert td._c_map_dump(0, 100, 0, 10, 256, None) == 2                     # BB has no dump
    assert td._c_ltm_check(0, 10, None, None) == 1
    assert td._c_ltm_check(2**50, 10, 256, None) == 2
    ns = C.c_uint64()
    assert td._c_wait_selftest(2, 10**6, 256, C.byref(ns), None) == 1         # arrive not 0/1
    assert td._c_wait_selftest(0, 999, 256, C.byref(ns), None) == 1           # limit below 1 us
    assert td._c_wait_selftest(0, 10**9 + 1, 256, C.byref(ns), None) == 1     # limit above 1 s
    assert td._c_wait_selftest(0, 10**6, None, C.byref(ns), None) == 1        # NULL record
    assert td._c_wait_selftest(0, 10**6, 260, C.byref(ns), None) == 1         # misaligned record


def test_options_validated():
    assert td.td_get_option("probe_strip") == 0                              # chosen per launch
    for bad in (-1, 1, 64, 300, 16384):
        assert td._c_set_option(1, bad) == 1 and "strip" in td._c_last_error().decode()
        assert td.td_get_option("probe_strip") == 0                          # unchanged
    td.td_set_option("probe_strip", 1024)
    assert td.td_get_option("probe_strip") == 1024
    td.td_set_option("probe_strip", 0)
    assert td._c_set_option(7, 0) == 1 and td.td_get_option(7) == 0          # unknown option
    for bad in (-1, 3):
        assert td._c_set_option(2, bad) == 1                                   # TMA staging: 0, 1 or 2
    for v in (1, 2, 0):
        td.td_set_option("edm_tma", v)
        assert td.td_get_option("edm_tma") == v


def test_oracle_not_imported_by_product():
    import glob
    pkg = os.path.dirname(td.__file__)
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        src = open(path, errors="ignore").read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
        assert "td_oracle" not in src and "liboracle" not in src, path


def test_slice_arguments_rejected_before_launch():
    """The block-row slice entry points validate on the host: empty or out-of-range row ranges,
    strategies without contiguous block rows, wrong block sides and misaligned outputs return an
    error before any launch (no GPU needed)."""
    st = td.td_launch_stats()
    probe = td._c_map_probe_rows
    assert probe(4, 1024, 16, 3, 3, 256, C.byref(st), None) == 1          # empty range
    assert probe(4, 1024, 16, 5, 2, 256, C.byref(st), None) == 1          # reversed
    assert probe(4, 1024, 16, 0, 65, 256, C.byref(st), None) == 1         # past ceil(N / rho) = 64
    assert probe(1, 1024, 16, 0, 1, 256, C.byref(st), None) == 2          # UTM: not a block strategy
    assert probe(3, 1024, 16, 0, 1, 256, C.byref(st), None) == 2          # REC: block rows not contiguous
    assert probe(4, 1024, 64, 0, 1, 256, C.byref(st), None) == 1          # the probe takes rho <= 32
    assert probe(4, 1024, 16, 0, 1, 8, C.byref(st), None) == 1            # misaligned output
    assert probe(4, 1024, 16, 0, 1, None, C.byref(st), None) == 1         # NULL output
    edm = td._c_edm_rows
    assert edm(4, 2, 256, 100, 4, 128, 0, 1, 256, C.byref(st), None) == 2  # chunked needs rho <= 32
    assert edm(4, 1, 256, 100, 4, 16, 0, 1, 256, C.byref(st), None) == 2   # tiled needs rho 64 / 128
    assert edm(4, 2, 256, 100, 0, 16, 0, 1, 256, C.byref(st), None) == 1   # d = 0
    col = td._c_collide_rows
    assert col(4, 1, 256, 256, 100, 2, 2, 256, C.byref(st), None) == 1    # empty tile-row range
    assert col(4, 1, 256, 256, 100, 0, 5, 256, C.byref(st), None) == 1    # past ceil(100 / 32) = 4
    assert col(8, 1, 256, 256, 100, 0, 1, 256, C.byref(st), None) == 2    # UTM-BLOCK not sliced
    assert col(4, 2, 256, 256, 100, 0, 1, 256, C.byref(st), None) == 1    # CHUNKED not a collision schedule



def test_empty_inputs_are_noops():
    """Every entry point documents an empty input (N = 0, n = 0, n < 2 for the strict forms,
    nprob = 0) as a no-op: it returns TD_OK before any check of the (here NULL) buffers and before
    any launch, so it needs no GPU, and its stats report no launched CTA."""
    st = td.td_launch_stats()
    for m in ("LTM", "BB", "UTM", "RB"):
        for sched in (0, 1):
            st.ctas = 7
            assert td._c_map_probe(td.MAPPINGS[m], sched, 0, 16, None, C.byref(st), None) == 0, (m, sched)
            assert st.ctas == 0 and st.useful_blocks == 0
            st.ctas = 7
            assert td._c_edm(td.MAPPINGS[m], sched, None, 0, 3, 16, None, C.byref(st), None) == 0, (m, sched)
            assert st.ctas == 0
    assert td._c_map_probe(td.MAPPINGS["LTM"], 2, 0, 16, None, C.byref(st), None) == 0        # chunked
    assert td._c_edm(td.MAPPINGS["LTM"], 1, None, 0, 64, 128, None, C.byref(st), None) == 0   # tiled
    for m in ("LTM", "BB"):
        st.ctas = 7
        assert td._c_collide(td.MAPPINGS[m], 0, None, None, 0, None, C.byref(st), None) == 0
        assert st.ctas == 0
    for n in (0, 1):
        assert td._c_edm_strict(None, n, 3, None, None) == 0
        assert td._c_collide_strict(None, None, n, None, None) == 0
        assert td._c_edm_strict_blocks(td.MAPPINGS["LTM"], None, n, 3, 16, None, C.byref(st), None) == 0
        assert td._c_collide_strict_blocks(td.MAPPINGS["LTM"], None, None, n, 32, None, C.byref(st), None) == 0
    assert td._c_gram(None, 0, 256, None, None, 0, None) == 0
    cfg = td.td_batched_config(128, 0)
    assert td._c_batched(0, None, None, None, None, None, 0, C.byref(cfg), C.byref(st), None) == 0
    assert td._c_batched_noalloc(0, None, None, None, None, C.byref(cfg), C.byref(st), None) == 0
    assert st.ctas == 0
