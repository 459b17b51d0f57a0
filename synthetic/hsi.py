"""Seeded synthetic hyperspectral cubes with the paper's noise model.

The paper's datasets (Pavia Centre 200x200x80, Washington DC Mall
256x256x191, Indian Pines 145x145x220; Section IV-A) are not available, so
cubes of those shapes are synthesised:

* clean cube = sum_k A_k(x, y) s_k(band): abundances A_k piecewise constant on
  seeded Voronoi cells, normalised to sum to one per pixel; spectra s_k a sum
  of three seeded Gaussians over the band index, scaled to max 1;
* noise (Section IV-B, noise cases 1-9): zero-mean Gaussian with a per-band
  standard deviation (the paper's "variance" is a standard deviation: its
  noisy PSNR of 20.001 dB at 0.1 is 20 log10(1/0.1)), salt-and-pepper
  impulses on a fraction of voxels, stripes (a constant offset on 10% of the
  columns of chosen bands) and dead lines (3-10 columns of width 1-3 set to 0
  on chosen bands).

Every random number comes from one counter-based generator (SplitMix64's
output mix applied to key + counter * golden-gamma, the published
definition by Steele, Lea and Flood, 2014), so a cube is a pure function of
its recipe and seed on any machine and numpy version.

Cubes are numpy float64 arrays of shape (n1, n2, n3); the library and the
oracle both use the flat order i + n1*(j + n2*k), i.e. Fortran order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Stream", "Recipe", "RECIPES", "BATCH_SHAPES", "batch_recipes", "make_cube", "mpsnr",
           "flat", "unflat"]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def _fnv1a(s: str) -> int:
    h = 0xCBF29CE484222325
    for b in s.encode():
        h = ((h ^ b) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Stream:
    """Counter-based random stream: value i = mix(key + (i + 1) * gamma)."""

    def __init__(self, seed: int, tag: str):
        k = np.array([(int(seed) * 0x9E3779B97F4A7C15 + _fnv1a(tag)) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        self.key = _mix(k)[0]
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi)."""
        return lo + np.floor(self.uniform(n) * (hi - lo)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller from pairs of uniforms (u1 in (0, 1])."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
        return z[:n]


@dataclasses.dataclass(frozen=True)
class Recipe:
    """Shape, mixture and noise of one synthetic cube."""
    n1: int
    n2: int
    n3: int
    endmembers: int = 4
    cells: int = 12
    sigma: tuple = (0.1, 0.1)        # per-band Gaussian std drawn from U[lo, hi]
    impulse: float = 0.1             # salt-and-pepper fraction of voxels
    stripe_bands: float = 0.0        # fraction of bands with stripes
    deadline_bands: float = 0.0      # fraction of bands with dead lines

    @property
    def shape(self):
        return (self.n1, self.n2, self.n3)


RECIPES = {
    # 32x32x16, 4 endmembers, 12 cells, sigma 0.1 + 10% salt-and-pepper
    "c1": Recipe(32, 32, 16, 4, 12, (0.1, 0.1), 0.10),
    # Pavia-shaped 200x200x80, mixed noise of noise case 9 style
    "c2": Recipe(200, 200, 80, 6, 40, (0.1, 0.2), 0.20, 0.30, 0.10),
    # Washington-DC-shaped 256x256x191
    "c3": Recipe(256, 256, 191, 8, 48, (0.1, 0.2), 0.20, 0.30, 0.10),
    # 64x64x31 pairs for the unrolled form
    "c5": Recipe(64, 64, 31, 4, 12, (0.1, 0.1), 0.10),
}


BATCH_SHAPES = ((64, 64, 31), (128, 128, 64), (145, 145, 220), (200, 200, 80))


def batch_recipes(count: int, seed: int):
    """`count` recipes for a batch of uneven cubes: shapes drawn by seed from
    the Indian-Pines, Pavia and smaller shapes above, each cube with its own
    Gaussian level U[0.05, 0.2] and impulse fraction U[0, 0.3]."""
    st = Stream(seed, "batch")
    pick = st.integers(count, 0, len(BATCH_SHAPES))
    sig = st.uniform(count, 0.05, 0.2)
    imp = st.uniform(count, 0.0, 0.3)
    return [Recipe(*BATCH_SHAPES[int(k)], 6, 24, (float(s_), float(s_)), float(p_))
            for k, s_, p_ in zip(pick, sig, imp)]


def make_cube(recipe: Recipe, seed: int):
    """Returns (clean, noisy) float64 cubes of shape (n1, n2, n3)."""
    n1, n2, n3 = recipe.shape
    K = recipe.endmembers
    # Voronoi abundances
    st = Stream(seed, "voronoi")
    cx = st.uniform(recipe.cells, 0.0, n1)
    cy = st.uniform(recipe.cells, 0.0, n2)
    ab = st.uniform(recipe.cells * K).reshape(recipe.cells, K) + 1e-3
    ab /= ab.sum(axis=1, keepdims=True)
    ii, jj = np.meshgrid(np.arange(n1, dtype=np.float64), np.arange(n2, dtype=np.float64),
                         indexing="ij")
    d2 = (ii[..., None] - cx) ** 2 + (jj[..., None] - cy) ** 2
    cell = np.argmin(d2, axis=-1)                       # (n1, n2)
    A = ab[cell]                                        # (n1, n2, K)
    # Spectra: three Gaussians each, scaled to max 1
    ss = Stream(seed, "spectra")
    band = np.arange(n3, dtype=np.float64)
    S = np.zeros((K, n3))
    for k in range(K):
        c = ss.uniform(3, 0.0, n3)
        w = ss.uniform(3, max(n3 / 20.0, 0.5), max(n3 / 4.0, 1.0))
        a = ss.uniform(3, 0.2, 1.0)
        S[k] = (a[:, None] * np.exp(-((band - c[:, None]) ** 2) / (2 * w[:, None] ** 2))).sum(0)
        S[k] /= S[k].max()
    clean = np.einsum("ijk,kb->ijb", A, S)
    # Noise
    noisy = clean.copy()
    sn = Stream(seed, "noise")
    sig = sn.uniform(n3, recipe.sigma[0], recipe.sigma[1])
    noisy += sn.normal(clean.size).reshape(n3, n2, n1).transpose(2, 1, 0) * sig
    if recipe.impulse > 0:
        hit = sn.uniform(clean.size).reshape(n3, n2, n1).transpose(2, 1, 0) < recipe.impulse
        val = (sn.uniform(clean.size).reshape(n3, n2, n1).transpose(2, 1, 0) < 0.5).astype(float)
        noisy[hit] = val[hit]
    if recipe.stripe_bands > 0:
        ns = int(round(recipe.stripe_bands * n3))
        bands = np.sort(sn.integers(ns, 0, n3))
        for b in bands:
            ncol = max(1, int(round(0.1 * n2)))
            cols = sn.integers(ncol, 0, n2)
            off = sn.uniform(ncol, -0.25, 0.25)
            noisy[:, cols, b] += off[None, :]
    if recipe.deadline_bands > 0:
        nd = int(round(recipe.deadline_bands * n3))
        bands = np.sort(sn.integers(nd, 0, n3))
        for b in bands:
            nl = int(sn.integers(1, 3, 11)[0])
            starts = sn.integers(nl, 0, n2)
            widths = sn.integers(nl, 1, 4)
            for s0, wd in zip(starts, widths):
                noisy[:, s0:min(n2, s0 + wd), b] = 0.0
    return clean, noisy


def flat(cube: np.ndarray, dtype=np.float32) -> np.ndarray:
    """Cube (n1, n2, n3) -> flat vector in i + n1*(j + n2*k) order."""
    return np.ascontiguousarray(np.asarray(cube).reshape(-1, order="F").astype(dtype))


def unflat(v: np.ndarray, shape) -> np.ndarray:
    return np.asarray(v).reshape(shape, order="F")


def mpsnr(x, clean) -> float:
    """Mean over bands of PSNR = 10 log10(1 / MSE_band) on [0, 1] data
    (Section IV-A's evaluation index)."""
    x = np.asarray(x, np.float64)
    clean = np.asarray(clean, np.float64)
    n3 = x.shape[-1]
    mse = ((x - clean) ** 2).reshape(-1, n3, order="F").mean(axis=0)
    return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-300))))
