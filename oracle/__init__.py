"""CPU oracle for the triangular-domain mappings and kernels (arXiv:1308.1419).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg are the only callers.  The product path (paper_1308_1419_gb300) never
imports this package, and this package never imports the product or reads its output.

Each wrapper calls the plain C definition in td_oracle.c through ctypes; arrays are numpy.
Paper references: Sec. II-A Eq. (matrix_indexing), Eq. (theorem), Eq. (theorem_nodiag)
for g; Sec. III-B for BB, RB, REC and UTM; Sec. IV for the dummy kernel and the EDM.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

_lib = C.CDLL(build_oracle())

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_tri = _sig("or_tri", C.c_uint64, C.c_uint64)
_isqrt = _sig("or_isqrt", C.c_uint64, C.c_uint64)
_ltm_many = _sig("or_ltm_many", None, _u64p, C.c_uint64, _u32p)
_ltm_nd_many = _sig("or_ltm_nodiag_many", None, _u64p, C.c_uint64, _u32p)
_utm_ab = _sig("or_utm_ab", None, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64))
_utm_enum = _sig("or_utm_enum", None, C.c_uint64, _u64p)
_utm_lower_many = _sig("or_utm_lower_many", None, C.c_uint32, _u64p, C.c_uint64, _u32p)
_rb_dims = _sig("or_rb_dims", None, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64))
_rb_map = _sig("or_rb_map", None, C.c_uint32, C.c_uint64, C.c_uint64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32))
_rec_levels = _sig("or_rec_levels", C.c_int, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint32))
_cover = _sig("or_cover", C.c_int, C.c_int, C.c_uint32, C.c_uint32, _u32p, _u64p)
_splitmix32 = _sig("or_splitmix32", C.c_uint32, C.c_uint32)
_probe = _sig("or_probe", None, C.c_uint32, C.c_uint32, C.c_uint32, _u32p)
_edm = _sig("or_edm", None, _f32p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _f64p)
_edm_pairs = _sig("or_edm_pairs", None, _f32p, C.c_uint32, _u32p, _u32p, C.c_uint64, _f64p)
_collide = _sig("or_collide", None, _i32p, _i32p, C.c_uint32, _u32p)
_collide_pairs = _sig("or_collide_pairs", None, _i32p, _i32p, _u32p, _u32p, C.c_uint64, _u8p)
_collide_words = _sig("or_collide_words", C.c_uint64, C.c_uint32)
_collide_bitpos = _sig("or_collide_bitpos", None, C.c_uint32, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32))
_edm_strict = _sig("or_edm_strict", None, _f32p, C.c_uint32, C.c_uint32, _f64p)
_collide_strict = _sig("or_collide_strict", None, _i32p, _i32p, C.c_uint32, _u32p)
_fast_rsqrt = _sig("or_fast_rsqrt", C.c_float, C.c_float, C.c_int)
_fast_rsqrt_fma = _sig("or_fast_rsqrt_fma", C.c_float, C.c_float, C.c_int)
_ltm_variant = _sig("or_ltm_variant", None, C.c_int, C.c_uint64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32))
_ltm_variant_first_fail = _sig("or_ltm_variant_first_fail", C.c_uint64, C.c_int, C.c_uint64, C.c_uint64)

# strategy ids used by or_cover (same numbering as the public enum, by choice, not by sharing)
BB, UTM, RB, REC, LTM, UTM_BLOCK = 0, 1, 2, 3, 4, 8
STRATEGIES = {"BB": BB, "UTM": UTM, "RB": RB, "REC": REC, "LTM": LTM, "UTM-BLOCK": UTM_BLOCK}


def tri(m: int) -> int:
    """T(m) = m(m+1)/2 (Sec. II-A)."""
    return int(_tri(m))


def isqrt(x: int) -> int:
    return int(_isqrt(x))


def ltm(lam) -> np.ndarray:
    """Eq. (theorem), exact: returns an (count, 2) uint32 array of (i, j)."""
    lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lam, dtype=np.uint64)))
    ij = np.empty(2 * lam.size, dtype=np.uint32)
    _ltm_many(lam, lam.size, ij)
    return ij.reshape(-1, 2)


# the FP32 evaluations of g that Sec. III-A times (the two with a host definition)
# 1, 2: every operation rounded once; 3, 4: the products feeding an addition fused (one rounding)
LTM_X, LTM_N, LTM_N_FMA, LTM_X_FMA = 1, 2, 3, 4


def fast_rsqrt(x: float, steps: int) -> float:
    """The bit-level inverse-square-root estimate after `steps` Newton steps, in FP32."""
    return float(_fast_rsqrt(x, steps))


def fast_rsqrt_fma(x: float, steps: int) -> float:
    """The same estimate with each Newton step's product fused into its subtraction (FP32)."""
    return float(_fast_rsqrt_fma(x, steps))


def ltm_variant(variant: int, lam: int):
    """(i, j) of LTM-X (variants 1, 4) or LTM-N (variants 2, 3) at lambda, in FP32 as defined in
    td_oracle.c (3 and 4: the fused multiply-add evaluations)."""
    i, j = C.c_uint32(), C.c_uint32()
    _ltm_variant(variant, lam, C.byref(i), C.byref(j))
    return i.value, j.value


def ltm_variant_first_fail(variant: int, lam0: int, lam1: int) -> int:
    """Smallest lambda in [lam0, lam1) where the variant differs from the exact g (lam1 if none)."""
    return int(_ltm_variant_first_fail(variant, lam0, lam1))


def ltm_nodiag(lam) -> np.ndarray:
    """Eq. (theorem_nodiag) with the strict triangle's own row start (see td_oracle.c)."""
    lam = np.ascontiguousarray(np.atleast_1d(np.asarray(lam, dtype=np.uint64)))
    ij = np.empty(2 * lam.size, dtype=np.uint32)
    _ltm_nd_many(lam, lam.size, ij)
    return ij.reshape(-1, 2)


def utm_ab(n: int, k: int):
    """UTM formula of Sec. III-B, exact: (a, b) with 1 <= a < b <= n."""
    a, b = C.c_uint64(), C.c_uint64()
    _utm_ab(n, k, C.byref(a), C.byref(b))
    return int(a.value), int(b.value)


def utm_enum(n: int) -> np.ndarray:
    """Row-major enumeration of the strict upper pairs (a, b) of side n."""
    cnt = n * (n - 1) // 2
    ab = np.empty(2 * max(cnt, 1), dtype=np.uint64)
    _utm_enum(n, ab)
    return ab[: 2 * cnt].reshape(-1, 2)


def utm_lower(N: int, k) -> np.ndarray:
    """UTM thread index k -> lower-with-diagonal (i, j) of side N (rows reversed)."""
    k = np.ascontiguousarray(np.atleast_1d(np.asarray(k, dtype=np.uint64)))
    ij = np.empty(2 * k.size, dtype=np.uint32)
    _utm_lower_many(N, k, k.size, ij)
    return ij.reshape(-1, 2)


def rb_dims(N: int):
    W, H = C.c_uint64(), C.c_uint64()
    _rb_dims(N, C.byref(W), C.byref(H))
    return int(W.value), int(H.value)


def rb_map(N: int, x: int, y: int):
    i, j = C.c_uint32(), C.c_uint32()
    _rb_map(N, x, y, C.byref(i), C.byref(j))
    return int(i.value), int(j.value)


def rec_levels(N: int, rho: int):
    """(k, m) with N = m 2^k, m a multiple of rho, k maximal; None if N % rho != 0."""
    m = C.c_uint32()
    k = _rec_levels(N, rho, C.byref(m))
    return None if k < 0 else (int(k), int(m.value))


def cover(strategy, N: int, rho: int):
    """Per-element hit counts of every thread a strategy launches, plus launch counts.

    Returns (count uint32[T(N)], dict(launched, useful, launches, hits)).
    """
    sid = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
    count = np.zeros(max(tri(N), 1), dtype=np.uint32)
    st = np.zeros(4, dtype=np.uint64)
    rc = _cover(sid, N, rho, count, st)
    if rc != 0:
        raise ValueError(f"unsupported strategy {strategy} for N={N}, rho={rho}")
    return count[: tri(N)], dict(launched=int(st[0]), useful=int(st[1]), launches=int(st[2]), hits=int(st[3]))


def splitmix32(x: int) -> int:
    return int(_splitmix32(x & 0xFFFFFFFF))


def probe(N: int, i0: int = 0, i1: int = None) -> np.ndarray:
    """Probe output rows [i0, i1): out[T(i)+j - T(i0)] = splitmix32(i N + j)."""
    i1 = N if i1 is None else i1
    out = np.empty(max(tri(i1) - tri(i0), 1), dtype=np.uint32)
    _probe(N, i0, i1, out)
    return out[: tri(i1) - tri(i0)]


def edm(x: np.ndarray, i0: int = 0, i1: int = None) -> np.ndarray:
    """FP64 EDM of x (n x d float32), packed lower triangle with diagonal, rows [i0, i1)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    i1 = n if i1 is None else i1
    out = np.empty(max(tri(i1) - tri(i0), 1), dtype=np.float64)
    _edm(x, n, d, i0, i1, out)
    return out[: tri(i1) - tri(i0)]


def edm_pairs(x: np.ndarray, ii, jj) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    ii = np.ascontiguousarray(ii, dtype=np.uint32)
    jj = np.ascontiguousarray(jj, dtype=np.uint32)
    out = np.empty(max(ii.size, 1), dtype=np.float64)
    _edm_pairs(x, x.shape[1], ii, jj, ii.size, out)
    return out[: ii.size]


def edm_batched(xs, ns, ds):
    """Batched EDM: the per-problem definition applied to each problem in turn.

    xs is the concatenation of the row-major n_p x d_p blocks; the result is the
    concatenation of the packed triangles, problem by problem.
    """
    outs, off = [], 0
    for n, d in zip(ns, ds):
        x = np.asarray(xs[off: off + n * d], dtype=np.float32).reshape(n, d)
        outs.append(edm(x))
        off += n * d
    return np.concatenate(outs) if outs else np.zeros(0)


def collide_words(n: int) -> int:
    return int(_collide_words(n))


def collide(centers: np.ndarray, radii: np.ndarray) -> np.ndarray:
    """Exact int64 collision table in the 32x32 bit-tile layout."""
    c = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1)
    r = np.ascontiguousarray(radii, dtype=np.int32)
    n = r.size
    out = np.empty(max(collide_words(n), 1), dtype=np.uint32)
    _collide(c, r, n, out)
    return out[: collide_words(n)]


def collide_pairs(centers, radii, ii, jj) -> np.ndarray:
    c = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1)
    r = np.ascontiguousarray(radii, dtype=np.int32)
    ii = np.ascontiguousarray(ii, dtype=np.uint32)
    jj = np.ascontiguousarray(jj, dtype=np.uint32)
    out = np.empty(max(ii.size, 1), dtype=np.uint8)
    _collide_pairs(c, r, ii, jj, ii.size, out)
    return out[: ii.size]


def collide_bitpos(i: int, j: int):
    w, b = C.c_uint64(), C.c_uint32()
    _collide_bitpos(i, j, C.byref(w), C.byref(b))
    return int(w.value), int(b.value)


def edm_strict(x: np.ndarray) -> np.ndarray:
    """Strict-lower distance map (no diagonal) in double: pair (i, j), i > j, at k = i(i-1)/2 + j."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    out = np.empty(n * (n - 1) // 2, dtype=np.float64)
    _edm_strict(x.reshape(-1), n, d, out)
    return out


def collide_strict(c: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Strict-lower collision bits: bit k % 32 of word k / 32 for the pair at k = i(i-1)/2 + j."""
    c = np.ascontiguousarray(c, dtype=np.int32).reshape(-1)
    r = np.ascontiguousarray(r, dtype=np.int32)
    n = r.size
    bits = np.zeros(max((n * (n - 1) // 2 + 31) // 32, 1), dtype=np.uint32)
    _collide_strict(c, r, n, bits)
    return bits[: (n * (n - 1) // 2 + 31) // 32]
