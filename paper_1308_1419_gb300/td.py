"""Thin Python binding of libtd (include/td.h).

Argument marshalling only: every function has the name of the C entry point it calls,
checks that tensors live on a CUDA device with the right dtype and size, passes raw device
pointers and the current torch stream, and raises TDError on a non-zero status.  Torch only
provides device memory and streams; all computation happens in libtd's kernels.  There is
no fallback: if libtd.so is missing, importing this module fails.
"""
import ctypes as C
import os

import torch

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtd.so")
if not os.path.exists(_PATH):
    raise ImportError(f"{_PATH} is missing; build it first (python -m paper_1308_1419_gb300.build, "
                      "needs nvcc with sm_103a support)")
lib = C.CDLL(_PATH)

MAPPINGS = {"BB": 0, "UTM": 1, "RB": 2, "REC": 3, "LTM": 4, "LTM-X": 5, "LTM-N": 6, "LTM-R": 7, "UTM-BLOCK": 8,
            "LTM-N-FMA": 9}
SCHEDULES = {"grid": 0, "persistent": 1, "chunked": 2}
STATUS = {0: "TD_OK", 1: "TD_ERR_INVALID_ARG", 2: "TD_ERR_UNSUPPORTED", 3: "TD_ERR_CUDA", 4: "TD_ERR_TIMEOUT"}


class TDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class td_launch_stats(C.Structure):
    _fields_ = [("blocks", C.c_uint64), ("useful_blocks", C.c_uint64), ("wasted_blocks", C.c_uint64),
                ("launches", C.c_uint64), ("ctas", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _sig(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_vp, _u32, _u64, _int = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
_stats_p = C.POINTER(td_launch_stats)
_c_version = _sig("td_version", _int)
_c_last_error = _sig("td_last_error", C.c_char_p)
_c_tri_size = _sig("td_tri_size", _u64, _u32, _int)
_c_collide_words = _sig("td_collide_words", _u64, _u32)
_c_plan = _sig("td_plan", _int, _int, _int, _u32, _u32, _stats_p)
_c_map_probe = _sig("td_map_probe", _int, _int, _int, _u32, _u32, _vp, _stats_p, _vp)
_c_edm = _sig("td_edm", _int, _int, _int, _vp, _u32, _u32, _u32, _vp, _stats_p, _vp)
_c_collide = _sig("td_collide", _int, _int, _int, _vp, _vp, _u32, _vp, _stats_p, _vp)
_c_set_option = _sig("td_set_option", _int, _int, _int)
_c_get_option = _sig("td_get_option", _int, _int)
class td_batched_config(C.Structure):
    _fields_ = [("rho", C.c_uint32), ("ctas_per_sm", C.c_uint32)]


_c_batched_ws = _sig("td_edm_batched_workspace", C.c_size_t, _u32)
_c_batched = _sig("td_edm_batched", _int, _u32, _vp, _vp, _vp, _vp, _vp, C.c_size_t,
                  C.POINTER(td_batched_config), _stats_p, _vp)
_c_batched_plan = _sig("td_edm_batched_plan", _int, _u32, _vp, _vp, _u32, _vp, C.c_size_t,
                       C.POINTER(C.c_uint64), _vp)
_c_batched_run = _sig("td_edm_batched_run", _int, _u32, _u32, _u64, _vp, _vp, _vp, _u32, _vp)
_c_batched_tune = _sig("td_edm_batched_autotune", _int, _u32, _vp, _vp, _vp, _vp, _vp, C.c_size_t,
                       C.POINTER(td_batched_config), C.POINTER(C.c_float), _vp)
_c_gram_ws = _sig("td_edm_gram_workspace", C.c_size_t, _u32, _u32)
_c_gram = _sig("td_edm_gram", _int, _vp, _u32, _u32, _vp, _vp, C.c_size_t, _vp)
_c_gram_status = _sig("td_edm_gram_status", _int, _vp, C.POINTER(C.c_uint64), _vp)
_c_batched_noalloc = _sig("td_edm_batched_noalloc", _int, _u32, _vp, _vp, _vp, _vp,
                          C.POINTER(td_batched_config), _stats_p, _vp)
_c_partition = _sig("td_partition", _int, _u32, _u32, _u32, _u32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                    C.POINTER(C.c_uint64), C.POINTER(C.c_uint64))
_c_map_cover = _sig("td_map_cover", _int, _int, _int, _u32, _u32, _vp, _vp)
_c_map_dump = _sig("td_map_dump", _int, _int, _u32, _u64, _u64, _vp, _vp)
_c_ltm_check = _sig("td_ltm_check", _int, _u64, _u64, _vp, _vp)
_c_ltm_variant_check = _sig("td_ltm_variant_check", _int, _int, _u64, _u64, _vp, _vp)
_c_map_dummy = _sig("td_map_dummy", _int, _int, _int, _u32, _u32, _vp, _vp, _vp)
_c_collide_strict_words = _sig("td_collide_strict_words", _u64, _u32)
_c_edm_strict = _sig("td_edm_strict", _int, _vp, _u32, _u32, _vp, _vp)
_c_collide_strict = _sig("td_collide_strict", _int, _vp, _vp, _u32, _vp, _vp)
_c_edm_strict_blocks = _sig("td_edm_strict_blocks", _int, _int, _vp, _u32, _u32, _u32, _vp, _stats_p, _vp)
_c_collide_strict_blocks = _sig("td_collide_strict_blocks", _int, _int, _vp, _vp, _u32, _u32, _vp, _stats_p, _vp)
_c_wait_selftest = _sig("td_wait_selftest", _int, _u32, _u64, _vp, C.POINTER(C.c_uint64), _vp)
_c_wait_status = _sig("td_wait_status", _int, _int, _vp)
_c_map_probe_rows = _sig("td_map_probe_rows", _int, _int, _u32, _u32, _u32, _u32, _vp, _stats_p, _vp)
_c_edm_rows = _sig("td_edm_rows", _int, _int, _int, _vp, _u32, _u32, _u32, _u32, _u32, _vp, _stats_p, _vp)
_c_collide_rows = _sig("td_collide_rows", _int, _int, _int, _vp, _vp, _u32, _u32, _u32, _vp, _stats_p, _vp)


def _check(status):
    if status != 0:
        raise TDError(status, _c_last_error().decode())


def _mapping(m):
    return MAPPINGS[m] if isinstance(m, str) else int(m)


def _schedule(s):
    return SCHEDULES[s] if isinstance(s, str) else int(s)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t, dtype, numel, name, host_ok=False):
    """Device address of t.  host_ok: a pinned host tensor is accepted too -- its address is
    valid on the device (unified addressing), so a kernel writes it in place over the host link."""
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise TypeError(f"{name} must be a CUDA tensor" + (" or a pinned host tensor" if host_ok else ""))
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")
    return t.data_ptr()


# ---------------------------------------------------------------- host-only helpers

def td_version() -> int:
    return int(_c_version())


OPTIONS = {"edm_f32x2": 0, "probe_strip": 1, "edm_tma": 2}


def td_set_option(opt, value: int):
    _check(_c_set_option(OPTIONS[opt] if isinstance(opt, str) else int(opt), int(value)))


def td_get_option(opt) -> int:
    return int(_c_get_option(OPTIONS[opt] if isinstance(opt, str) else int(opt)))


def td_tri_size(N: int, with_diag: bool = True) -> int:
    return int(_c_tri_size(N, int(bool(with_diag))))


def td_collide_words(n: int) -> int:
    return int(_c_collide_words(n))


def td_plan(mapping, schedule, N: int, rho: int) -> dict:
    st = td_launch_stats()
    _check(_c_plan(_mapping(mapping), _schedule(schedule), N, rho, C.byref(st)))
    return st.as_dict()


def td_partition(N: int, rho: int, G: int, r: int):
    """Rank r's block rows [br0, br1) and packed-output slice [off0, off1) (host only)."""
    b0, b1, o0, o1 = C.c_uint32(), C.c_uint32(), C.c_uint64(), C.c_uint64()
    _check(_c_partition(N, rho, G, r, C.byref(b0), C.byref(b1), C.byref(o0), C.byref(o1)))
    return int(b0.value), int(b1.value), int(o0.value), int(o1.value)


# ---------------------------------------------------------------- mapping kernels

def td_map_probe(mapping, schedule, N: int, rho: int, out: torch.Tensor = None, stream=None):
    """Probe output (int32 tensor holding the uint32 bit patterns) and launch stats.  out may be
    a device tensor or a pinned host tensor (written in place by the kernel)."""
    total = td_tri_size(N)
    if out is None:
        out = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    ptr = _dev(out, torch.int32, total, "out", host_ok=True)
    st = td_launch_stats()
    _check(_c_map_probe(_mapping(mapping), _schedule(schedule), N, rho, ptr, C.byref(st), _stream(stream)))
    return out, st.as_dict()


def _row_offset(b: int, rho: int, N: int) -> int:
    r = min(b * rho, N)
    return r * (r + 1) // 2


def td_map_probe_rows(mapping, N: int, rho: int, br0: int, br1: int, out: torch.Tensor = None, stream=None):
    """Probe of block rows [br0, br1) only (chunked schedule): the packed elements
    [T(br0 rho), T(min(br1 rho, N))) of the whole output; returns (slice, stats)."""
    size = _row_offset(br1, rho, N) - _row_offset(br0, rho, N)
    if out is None:
        out = torch.empty(max(size, 4), dtype=torch.int32, device="cuda")
    op = _dev(out, torch.int32, size, "out")
    st = td_launch_stats()
    _check(_c_map_probe_rows(_mapping(mapping), N, rho, br0, br1, op, C.byref(st), _stream(stream)))
    return out, st.as_dict()


def td_edm_rows(mapping, schedule, x: torch.Tensor, rho: int, br0: int, br1: int, out: torch.Tensor = None,
                stream=None):
    """Distance map of block rows [br0, br1) of the points x (n x d); returns (slice, stats)."""
    n, d = x.shape
    xp = _dev(x, torch.float32, n * d, "x")
    size = _row_offset(br1, rho, n) - _row_offset(br0, rho, n)
    if out is None:
        out = torch.empty(max(size, 4), dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, size, "out")
    st = td_launch_stats()
    _check(_c_edm_rows(_mapping(mapping), _schedule(schedule), xp, n, d, rho, br0, br1, op, C.byref(st),
                       _stream(stream)))
    return out, st.as_dict()


def td_collide_rows(mapping, schedule, centers: torch.Tensor, radii: torch.Tensor, br0: int, br1: int,
                    table: torch.Tensor = None, stream=None):
    """Collision-table words of block rows [br0, br1) (64 spheres each): tile rows
    [t0, t1) = [min(2 br0, nt), min(2 br1, nt)), words [32 T(t0), 32 T(t1)); returns (slice, stats)."""
    n = radii.numel()
    cp = _dev(centers, torch.int32, 3 * n, "centers")
    rp = _dev(radii, torch.int32, n, "radii")
    nt = (n + 31) // 32
    t0, t1 = min(2 * br0, nt), min(2 * br1, nt)
    words = 32 * (t1 * (t1 + 1) // 2 - t0 * (t0 + 1) // 2)
    if table is None:
        table = torch.empty(max(words, 4), dtype=torch.int32, device=radii.device)
    tp = _dev(table, torch.int32, words, "table")
    st = td_launch_stats()
    _check(_c_collide_rows(_mapping(mapping), _schedule(schedule), cp, rp, n, br0, br1, tp, C.byref(st),
                           _stream(stream)))
    return table, st.as_dict()


def td_map_dummy(mapping, schedule, N: int, rho: int, sink: torch.Tensor = None, stream=None):
    """The map-only dummy kernel (Sec. III-A): launch stats; sink (int32[1]) is left unchanged."""
    if sink is None:
        sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    ptr = _dev(sink, torch.int32, 1, "sink")
    st = td_launch_stats()
    _check(_c_map_dummy(_mapping(mapping), _schedule(schedule), N, rho, ptr, C.byref(st), _stream(stream)))
    return sink, st.as_dict()


def td_collide_strict_words(n: int) -> int:
    return int(_c_collide_strict_words(n))


def td_edm_strict(x: torch.Tensor, out: torch.Tensor = None, stream=None):
    """Packed strict-lower distance map (no diagonal): float32[n(n-1)/2], k = i(i-1)/2 + j."""
    if x.dim() != 2:
        raise ValueError("x must be a 2-D (n, d) tensor")
    n, d = x.shape
    xp = _dev(x, torch.float32, n * d, "x")
    total = n * (n - 1) // 2
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, total, "out")
    _check(_c_edm_strict(xp, n, d, op, _stream(stream)))
    return out


def td_collide_strict(centers: torch.Tensor, radii: torch.Tensor, bits: torch.Tensor = None, stream=None):
    """Strict-lower collision bits (int32 tensor of uint32 words): bit k for pair k = i(i-1)/2 + j."""
    n = radii.numel()
    cp = _dev(centers, torch.int32, 3 * n, "centers")
    rp = _dev(radii, torch.int32, n, "radii")
    words = td_collide_strict_words(n)
    if bits is None:
        bits = torch.empty(max(words, 4), dtype=torch.int32, device=radii.device)
    bp = _dev(bits, torch.int32, words, "bits")
    _check(_c_collide_strict(cp, rp, n, bp, _stream(stream)))
    return bits


def td_edm_strict_blocks(mapping, x: torch.Tensor, rho: int, out: torch.Tensor = None, stream=None):
    """td_edm_strict's output mapped at the block level (LTM or BB, rho 8/16/32, d <= 8), and stats."""
    if x.dim() != 2:
        raise ValueError("x must be a 2-D (n, d) tensor")
    n, d = x.shape
    xp = _dev(x, torch.float32, n * d, "x")
    total = n * (n - 1) // 2
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, total, "out")
    st = td_launch_stats()
    _check(_c_edm_strict_blocks(_mapping(mapping), xp, n, d, rho, op, C.byref(st), _stream(stream)))
    return out, st.as_dict()


def td_collide_strict_blocks(mapping, centers: torch.Tensor, radii: torch.Tensor, rho: int = 32,
                             bits: torch.Tensor = None, stream=None):
    """td_collide_strict's bits mapped at the block level (LTM or BB, rho 8/16/32 strips, or 64:
    td_collide's 64 x 64 blocks ORing the rare set bits into a cleared array), and stats."""
    n = radii.numel()
    cp = _dev(centers, torch.int32, 3 * n, "centers")
    rp = _dev(radii, torch.int32, n, "radii")
    words = td_collide_strict_words(n)
    if bits is None:
        bits = torch.empty(max(words, 4), dtype=torch.int32, device=radii.device)
    bp = _dev(bits, torch.int32, words, "bits")
    st = td_launch_stats()
    _check(_c_collide_strict_blocks(_mapping(mapping), cp, rp, n, rho, bp, C.byref(st), _stream(stream)))
    return bits, st.as_dict()


def td_edm(mapping, schedule, x: torch.Tensor, rho: int, out: torch.Tensor = None, stream=None):
    """Packed FP32 Euclidean distance map of the rows of x (n x d, float32) and launch stats."""
    if x.dim() != 2:
        raise ValueError("x must be a 2-D (n, d) tensor")
    n, d = x.shape
    xp = _dev(x, torch.float32, n * d, "x")
    total = td_tri_size(n)
    if out is None:
        out = torch.empty(max(total, 1), dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, total, "out")
    st = td_launch_stats()
    _check(_c_edm(_mapping(mapping), _schedule(schedule), xp, n, d, rho, op, C.byref(st), _stream(stream)))
    return out, st.as_dict()


def td_collide(mapping, schedule, centers: torch.Tensor, radii: torch.Tensor, table: torch.Tensor = None,
               stream=None):
    """Bit-packed collision table (int32 tensor holding uint32 words) and launch stats."""
    n = radii.numel()
    cp = _dev(centers, torch.int32, 3 * n, "centers")
    rp = _dev(radii, torch.int32, n, "radii")
    words = td_collide_words(n)
    if table is None:
        table = torch.empty(max(words, 4), dtype=torch.int32, device=radii.device)
    tp = _dev(table, torch.int32, words, "table")
    st = td_launch_stats()
    _check(_c_collide(_mapping(mapping), _schedule(schedule), cp, rp, n, tp, C.byref(st), _stream(stream)))
    return table, st.as_dict()


def _host_u32(a, count, name):
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    if arr.size != count:
        raise ValueError(f"{name} must hold {count} values")
    return arr, arr.ctypes.data_as(C.c_void_p)


def td_edm_batched_workspace(nprob: int) -> int:
    return int(_c_batched_ws(nprob))


def batched_sizes(ns, ds):
    """(x floats, out floats) of a batch: sum n_p d_p and sum T(n_p)."""
    return (sum(int(n) * int(d) for n, d in zip(ns, ds)), sum(td_tri_size(int(n)) for n in ns))


def td_edm_batched(ns, ds, x_cat: torch.Tensor, out_cat: torch.Tensor = None, ws: torch.Tensor = None,
                   config=None, stream=None):
    """All problems' packed distance maps in one persistent launch; returns (out_cat, ws, stats)."""
    nprob = len(ns)
    nh, npp = _host_u32(ns, nprob, "ns")
    dh, dp = _host_u32(ds, nprob, "ds")
    xs, os_ = batched_sizes(nh, dh)
    xp = _dev(x_cat, torch.float32, xs, "x_cat")
    if out_cat is None:
        out_cat = torch.empty(max(os_, 4), dtype=torch.float32, device=x_cat.device)
    op = _dev(out_cat, torch.float32, os_, "out_cat")
    wsb = td_edm_batched_workspace(nprob)
    if ws is None:
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=x_cat.device)
    wp = _dev(ws, torch.uint8, wsb, "ws")
    cfg = None if config is None else C.byref(td_batched_config(*config))
    st = td_launch_stats()
    _check(_c_batched(nprob, npp, dp, xp, op, wp, ws.numel(), cfg, C.byref(st), _stream(stream)))
    return out_cat, ws, st.as_dict()


def td_edm_batched_noalloc(ns, ds, x_cat: torch.Tensor, out_cat: torch.Tensor, config=None, stream=None):
    """td_edm_batched without a workspace: the plan lives in the library's own fixed device
    array (at most 1024 problems), so the call allocates nothing.  out_cat must be given."""
    nprob = len(ns)
    nh, npp = _host_u32(ns, nprob, "ns")
    dh, dp = _host_u32(ds, nprob, "ds")
    xs, os_ = batched_sizes(nh, dh)
    cfg = None if config is None else C.byref(td_batched_config(*config))
    st = td_launch_stats()
    _check(_c_batched_noalloc(nprob, npp, dp, _dev(x_cat, torch.float32, xs, "x_cat"),
                              _dev(out_cat, torch.float32, os_, "out_cat"), cfg, C.byref(st), _stream(stream)))
    return out_cat, st.as_dict()


def td_edm_batched_plan(ns, ds, rho: int, ws: torch.Tensor, stream=None) -> int:
    nprob = len(ns)
    nh, npp = _host_u32(ns, nprob, "ns")
    dh, dp = _host_u32(ds, nprob, "ds")
    wp = _dev(ws, torch.uint8, td_edm_batched_workspace(nprob), "ws")
    total = C.c_uint64()
    _check(_c_batched_plan(nprob, npp, dp, rho, wp, ws.numel(), C.byref(total), _stream(stream)))
    return int(total.value)


def td_edm_batched_run(nprob: int, rho: int, total_blocks: int, x_cat: torch.Tensor, out_cat: torch.Tensor,
                       ws: torch.Tensor, ctas_per_sm: int = 0, stream=None):
    _check(_c_batched_run(nprob, rho, total_blocks, _dev(x_cat, torch.float32, 1, "x_cat"),
                          _dev(out_cat, torch.float32, 1, "out_cat"), _dev(ws, torch.uint8, 1, "ws"),
                          ctas_per_sm, _stream(stream)))


def td_edm_batched_autotune(ns, ds, x_cat: torch.Tensor, out_cat: torch.Tensor, ws: torch.Tensor, stream=None):
    """Returns ((rho, ctas_per_sm), ms per run) of the fastest configuration."""
    nprob = len(ns)
    nh, npp = _host_u32(ns, nprob, "ns")
    dh, dp = _host_u32(ds, nprob, "ds")
    xs, os_ = batched_sizes(nh, dh)
    best = td_batched_config()
    ms = C.c_float()
    _check(_c_batched_tune(nprob, npp, dp, _dev(x_cat, torch.float32, xs, "x_cat"),
                           _dev(out_cat, torch.float32, os_, "out_cat"),
                           _dev(ws, torch.uint8, td_edm_batched_workspace(nprob), "ws"), ws.numel(),
                           C.byref(best), C.byref(ms), _stream(stream)))
    return (int(best.rho), int(best.ctas_per_sm)), float(ms.value)


def td_edm_gram_workspace(n: int, d: int) -> int:
    return int(_c_gram_ws(n, d))


def td_edm_gram(x: torch.Tensor, out: torch.Tensor = None, ws: torch.Tensor = None, stream=None):
    """Gram-form (BF16 tensor-core) packed distance map with FP32 direct recompute of
    cancelling pairs; returns (out, ws)."""
    n, d = x.shape
    xp = _dev(x, torch.float32, n * d, "x")
    total = td_tri_size(n)
    if out is None:
        out = torch.empty(max(total, 4), dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, total, "out")
    wsb = td_edm_gram_workspace(n, d)
    if ws is None:
        ws = torch.empty(wsb + 1024, dtype=torch.uint8, device=x.device)
    base = ws.data_ptr()
    off = (-base) % 1024  # the workspace must be 1024-byte aligned
    if ws.numel() - off < wsb:
        raise ValueError("workspace too small")
    _check(_c_gram(xp, n, d, op, base + off, ws.numel() - off, _stream(stream)))
    return out, ws


def td_edm_gram_status(ws: torch.Tensor, stream=None) -> int:
    """Synchronises; returns the number of pairs recomputed in the direct form (raises on a timeout)."""
    off = (-ws.data_ptr()) % 1024
    fb = C.c_uint64()
    _check(_c_gram_status(ws.data_ptr() + off, C.byref(fb), _stream(stream)))
    return int(fb.value)


def td_wait_status(clear: bool = True, stream=None):
    """Synchronises; raises TDError (TD_ERR_TIMEOUT) if a bounded wait of the TMA-staged distance
    map ran out since the last clearing call."""
    _check(_c_wait_status(1 if clear else 0, _stream(stream)))


def td_wait_selftest(arrive: bool, limit_ns: int, ws: torch.Tensor = None, stream=None) -> int:
    """One bounded mbarrier wait whose phase completes (arrive) or never does; synchronises and
    returns the wait's duration in ns, raising TDError (status TD_ERR_TIMEOUT) if it ran out."""
    if ws is None:
        ws = torch.zeros(2, dtype=torch.int64, device="cuda")
    ptr = _dev(ws, torch.int64, 2, "ws")
    ns = C.c_uint64()
    _check(_c_wait_selftest(1 if arrive else 0, int(limit_ns), ptr, C.byref(ns), _stream(stream)))
    return int(ns.value)


def td_map_cover(mapping, schedule, N: int, rho: int, count: torch.Tensor = None, stream=None):
    total = td_tri_size(N)
    if count is None:
        count = torch.zeros(max(total, 1), dtype=torch.int32, device="cuda")
    ptr = _dev(count, torch.int32, total, "count")
    _check(_c_map_cover(_mapping(mapping), _schedule(schedule), N, rho, ptr, _stream(stream)))
    return count


def td_map_dump(mapping, N: int, u0: int, count: int, ij: torch.Tensor = None, stream=None):
    if ij is None:
        ij = torch.empty(max(2 * count, 2), dtype=torch.int32, device="cuda")
    ptr = _dev(ij, torch.int32, 2 * count, "ij")
    _check(_c_map_dump(_mapping(mapping), N, u0, count, ptr, _stream(stream)))
    return ij


def td_ltm_check(lam0: int, count: int, result: torch.Tensor = None, stream=None):
    if result is None:
        result = torch.tensor([0, -1], dtype=torch.int64, device="cuda")
    ptr = _dev(result, torch.int64, 2, "result")
    _check(_c_ltm_check(lam0, count, ptr, _stream(stream)))
    return result


def td_ltm_variant_check(mapping, lam0: int, count: int, result: torch.Tensor = None, stream=None):
    """(failures, first failing lambda or -1) of an evaluation of g over [lam0, lam0 + count)."""
    if result is None:
        result = torch.tensor([0, -1], dtype=torch.int64, device="cuda")
    ptr = _dev(result, torch.int64, 2, "result")
    _check(_c_ltm_variant_check(_mapping(mapping), lam0, count, ptr, _stream(stream)))
    return result
