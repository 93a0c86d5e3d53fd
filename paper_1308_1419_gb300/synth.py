"""Seeded synthetic inputs for the triangular-domain workloads.

This module only draws random inputs; it holds none of the mapping or kernel arithmetic,
so the CUDA path and the CPU oracle can both use it.  Everything derives from one
counter-based SplitMix64 stream (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): value k of stream s is mix64(s + (k + 1) * 0x9E3779B97F4A7C15).

Derived draws:
  * uniform float32 in [0, 1):   (u >> 40) * 2^-24            (exact in float32)
  * uniform integer in [lo, hi]:  lo + (((u >> 32) * (hi - lo + 1)) >> 32)  (multiply-shift)
  * standard normal (float64):   Box-Muller cosine branch from two draws,
                                 u1 = ((u_a >> 11) + 1) 2^-53, u2 = (u_b >> 11) 2^-53.

Workload recipes (each seed is 1308 + the workload's number):
  1 plain EDM      n = 2048, d = 3, x ~ U[0,1)^3 float32.
  2 probe sweep    N in {1024, 4096, 16384, 65536}, rho in {8, 16, 32}; no input array.
  3 collision      n = 32768, centres int32 U[0, 2^20)^3, radii int32 U[256, 2048].
  4 precision EDM  n = 16384, d = 256, 64 cluster centres ~ N(0,1)^256, labels U{0..63},
                   point = centre[label] + N(0, 0.05^2) per coordinate, float32.
  5 batched EDM    512 problems, n_p = floor(64 * 128^U) (U ~ U[0,1)), d_p U{3,16,64},
                   x ~ U[0,1) float32, concatenated problem after problem.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
SEED_BASE = 1308


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Stream:
    """A SplitMix64 stream; successive draws continue the counter."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed)
        self.k = 0

    def u64(self, count: int) -> np.ndarray:
        k = np.arange(self.k + 1, self.k + 1 + count, dtype=np.uint64)
        self.k += count
        with np.errstate(over="ignore"):
            return _mix64(self.seed + k * GAMMA)

    def uniform_f32(self, count: int) -> np.ndarray:
        return ((self.u64(count) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)

    def uniform_f64(self, count: int) -> np.ndarray:
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

    def randint(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers in [lo, hi] inclusive."""
        span = np.uint64(hi - lo + 1)
        with np.errstate(over="ignore"):
            v = ((self.u64(count) >> np.uint64(32)) * span) >> np.uint64(32)
        return (v.astype(np.int64) + lo)

    def normal(self, count: int) -> np.ndarray:
        ua = self.u64(count)
        ub = self.u64(count)
        u1 = ((ua >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (ub >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def seed_for(workload: int) -> int:
    return SEED_BASE + workload


def uniform_points(n: int, d: int, seed: int) -> np.ndarray:
    """n x d float32 points, coordinates U[0,1)."""
    return Stream(seed).uniform_f32(n * d).reshape(n, d)


def plain_edm(n: int = 2048, d: int = 3) -> np.ndarray:
    return uniform_points(n, d, seed_for(1))


def spheres(n: int = 32768, seed: int = None, coord_bits: int = 20, rmin: int = 256, rmax: int = 2048):
    """Centres int32 (n, 3) uniform in [0, 2^coord_bits), radii int32 uniform in [rmin, rmax]."""
    s = Stream(seed_for(3) if seed is None else seed)
    centres = s.randint(0, (1 << coord_bits) - 1, 3 * n).astype(np.int32).reshape(n, 3)
    radii = s.randint(rmin, rmax, n).astype(np.int32)
    return centres, radii


def clustered_points(n: int = 16384, d: int = 256, clusters: int = 64, sigma: float = 0.05,
                     seed: int = None) -> np.ndarray:
    """Gaussian clusters: centres N(0,1)^d, random labels, per-coordinate noise N(0, sigma^2)."""
    s = Stream(seed_for(4) if seed is None else seed)
    centres = s.normal(clusters * d).reshape(clusters, d)
    labels = s.randint(0, clusters - 1, n)
    noise = s.normal(n * d).reshape(n, d)
    return (centres[labels] + sigma * noise).astype(np.float32)


def batched_problems(nprob: int = 512, nmin: int = 64, ratio: float = 128.0, dims=(3, 16, 64),
                     seed: int = None):
    """Problem sizes n_p = floor(nmin * ratio^U), dimensions from `dims`, uniform x.

    Returns (ns uint32[nprob], ds uint32[nprob], x_cat float32[sum n_p d_p]).
    """
    s = Stream(seed_for(5) if seed is None else seed)
    u = s.uniform_f64(nprob)
    ns = np.floor(nmin * ratio ** u).astype(np.uint32)
    ds = np.asarray(dims, dtype=np.uint32)[s.randint(0, len(dims) - 1, nprob)]
    total = int(np.sum(ns.astype(np.int64) * ds.astype(np.int64)))
    x = s.uniform_f32(total)
    return ns, ds, x
