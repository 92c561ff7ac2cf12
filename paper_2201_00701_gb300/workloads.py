"""Seeded synthetic inputs for the EmbedSOM projection (points X, landmarks L and l).

This module only draws random numbers; it holds none of the projection's
arithmetic.  Both the CUDA path and the FP64 oracle are fed from it, so a
test can hand the very same arrays to each side.

The paper benchmarks on synthetic data only: n = 2^20 points with every
coordinate drawn from one uniform distribution (Section 4.1).  The named
workloads below are the mixture shapes this project is measured on; every
one is drawn with numpy's PCG64 from an explicit seed, in float32, row-major:

* ``mixture10_d8``      n=10,000, d=8, 10 isotropic Gaussians (sigma 0.5,
  means ~U[-5,5]^d); L=100 landmarks drawn from the same mixture; 2-D
  positions are the cells of a 10x10 grid in seeded order; k=10, boost=1,
  adjust=1.
* ``mixture30_d16``     n=1,000,000, d=16, 30 anisotropic Gaussians (random
  rotation from a sign-fixed QR, per-axis sigma ~U[0.2,1.5]) plus 5% points
  uniform over the bounding box of the mixture sample; L=1024 landmarks from
  the mixture (no outliers) on a 32x32 grid; k=20, boost=2, adjust=1.
* ``student50_d32``     n=10,000,000, d=32, 50 components with Student-t
  (nu=4) noise of scale 0.5 per axis; L=4096 on a 64x64 grid; k=30, boost=1,
  adjust=1.
* ``uniform_d16`` / ``uniform_d32``  the paper's own shape (Section 4.1 and
  the real-time figure of Section 5.1): n=2^20, every coordinate U[0,1],
  L=256 landmarks drawn the same way on a 16x16 grid, k=16.
* ``serve8``            8 resident sessions for the frame server, d=24,
  k=20, n in {2e5, 1e6, 5e6}, L in {256, 1024}, SOM step per frame.
* ``batch64``           64 independent datasets with n log-uniform in
  [1e3, 2e6], d in {8,16,32,48}, L in {100,400,1024,2500}, k in {10,20,30},
  each a 10-40 component Gaussian mixture.

Grid spacing is 1 with the origin at 0, so the layout extent (the largest
range of l over both axes) is side-1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray        # n x d float32, row-major
    hi: np.ndarray       # L x d float32 (high-dimensional landmarks)
    lo: np.ndarray       # L x 2 float32 (2-D landmarks)
    k: int
    boost: float
    adjust: float

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.hi.shape[1])

    @property
    def L(self) -> int:
        return int(self.hi.shape[0])

    @property
    def extent(self) -> float:
        """Largest range of the 2-D landmark layout over both axes."""
        rng = self.lo.max(axis=0) - self.lo.min(axis=0)
        return float(rng.max())


def _streams(seed: int, count: int) -> list[np.random.Generator]:
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(count)]


def grid_layout(L: int, rng: np.random.Generator) -> np.ndarray:
    """Cells of a side x side grid (spacing 1, origin 0) in seeded order."""
    side = int(round(math.sqrt(L)))
    if side * side != L:
        raise ValueError(f"L={L} is not a square")
    cells = np.stack([np.arange(L) % side, np.arange(L) // side], axis=1)
    return cells[rng.permutation(L)].astype(np.float32)


def _rotation(d: int, rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((d, d)))
    return q * np.sign(np.diag(r))[None, :]


class Mixture:
    """A Gaussian (or Student-t) mixture with equal weights."""

    def __init__(self, d: int, comps: int, rng: np.random.Generator, *,
                 kind: str = "iso", sigma: float = 0.5, nu: float = 4.0,
                 sigma_range=(0.2, 1.5)):
        self.d, self.comps, self.kind, self.nu = d, comps, kind, nu
        self.means = rng.uniform(-5.0, 5.0, (comps, d))
        if kind == "aniso":
            self.scales = [(_rotation(d, rng) * rng.uniform(*sigma_range, d)[None, :]).T
                           for _ in range(comps)]
        else:
            self.scales = [np.eye(d) * sigma for _ in range(comps)]

    def sample(self, n: int, seed: int) -> np.ndarray:
        streams = _streams(seed, self.comps + 1)
        comp = streams[0].integers(0, self.comps, n)
        out = np.empty((n, self.d), np.float32)
        for c in range(self.comps):
            sel = np.nonzero(comp == c)[0]
            if sel.size == 0:
                continue
            g = streams[c + 1]
            if self.kind == "student":
                z = g.standard_t(self.nu, (sel.size, self.d))
            else:
                z = g.standard_normal((sel.size, self.d))
            out[sel] = (self.means[c] + z @ self.scales[c]).astype(np.float32)
        return out


def mixture10_d8(seed: int = 0, n: int = 10_000) -> Workload:
    s = _streams(seed, 4)
    mix = Mixture(8, 10, s[0], kind="iso", sigma=0.5)
    X = mix.sample(n, seed * 1000 + 1)
    hi = mix.sample(100, seed * 1000 + 2)
    lo = grid_layout(100, s[1])
    return Workload("mixture10_d8", X, hi, lo, k=10, boost=1.0, adjust=1.0)


def mixture30_d16(seed: int = 0, n: int = 1_000_000, shard: int = 0) -> Workload:
    """`shard` > 0 draws a different set of points (same mixture, landmarks
    and layout), so ranks of a sharded run hold distinct points."""
    s = _streams(seed, 4)
    mix = Mixture(16, 30, s[0], kind="aniso")
    n_out = int(round(0.05 * n))
    ps = seed * 1000 + 1 + 7919 * shard
    Xm = mix.sample(n - n_out, ps)
    lo_box, hi_box = Xm.min(axis=0), Xm.max(axis=0)
    t = _streams(ps, 2) if shard else s[2:4]
    Xo = t[0].uniform(lo_box, hi_box, (n_out, 16)).astype(np.float32)
    X = np.concatenate([Xm, Xo])[t[1].permutation(n)]
    hi = mix.sample(1024, seed * 1000 + 2)
    lo = grid_layout(1024, s[1])
    return Workload("mixture30_d16", np.ascontiguousarray(X), hi, lo,
                    k=20, boost=2.0, adjust=1.0)


def student50_d32(seed: int = 0, n: int = 10_000_000) -> Workload:
    s = _streams(seed, 4)
    mix = Mixture(32, 50, s[0], kind="student", sigma=0.5, nu=4.0)
    X = mix.sample(n, seed * 1000 + 1)
    hi = mix.sample(4096, seed * 1000 + 2)
    lo = grid_layout(4096, s[1])
    return Workload("student50_d32", X, hi, lo, k=30, boost=1.0, adjust=1.0)


def uniform(d: int, seed: int = 0, n: int = 1 << 20, L: int = 256,
            k: int = 16) -> Workload:
    s = _streams(seed, 3)
    X = s[0].random((n, d), dtype=np.float32)
    hi = s[1].random((L, d), dtype=np.float32)
    lo = grid_layout(L, s[2])
    return Workload(f"uniform_d{d}", X, hi, lo, k=k, boost=1.0, adjust=1.0)


def batch64(seed: int = 0, count: int = 64, n_max: float = 2e6):
    """Parameters and lazy generators of the 64-dataset batch."""
    s = _streams(seed, count + 1)
    out = []
    for i in range(count):
        g = s[i + 1]
        n = int(round(10 ** g.uniform(3.0, math.log10(n_max))))
        d = int(g.choice([8, 16, 32, 48]))
        L = int(g.choice([100, 400, 1024, 2500]))
        k = int(g.choice([10, 20, 30]))
        comps = int(g.integers(10, 41))
        out.append(dict(index=i, n=n, d=d, L=L, k=k, comps=comps,
                        seed=seed * 100_000 + i))
    return out


def batch_member(p: dict, n: int | None = None) -> Workload:
    s = _streams(p["seed"], 3)
    mix = Mixture(p["d"], p["comps"], s[0], kind="iso",
                  sigma=float(s[2].uniform(0.3, 1.2)))
    nn = p["n"] if n is None else n
    X = mix.sample(nn, p["seed"] * 10 + 1)
    hi = mix.sample(p["L"], p["seed"] * 10 + 2)
    lo = grid_layout(p["L"], s[1])
    return Workload(f"batch64[{p['index']}]", X, hi, lo, k=p["k"],
                    boost=1.0, adjust=1.0)


def serve8(seed: int = 0, sessions: int = 8, n_scale: float = 1.0):
    """Parameters of the resident sessions of the serving workload: d=24,
    k=20, n from {2e5, 1e6, 5e6} (each size on every third session, in a
    seeded order), L from {256, 1024} alternating, a 10-40 component
    mixture each.  Frames: one SOM step (rate 0.05, neighbourhood sigma 1.5
    grid cells, 4096-point minibatch) and a full reprojection, arriving as a
    Poisson process of 60 frames/s per session.  `n_scale` shrinks n for
    tests."""
    s = _streams(seed, sessions + 1)
    sizes = [200_000, 1_000_000, 5_000_000]
    order = s[0].permutation(sessions)
    out = []
    for i in range(sessions):
        g = s[i + 1]
        n = max(1, int(round(sizes[int(order[i]) % 3] * n_scale)))
        out.append(dict(index=i, n=n, d=24, L=[256, 1024][i % 2], k=20,
                        comps=int(g.integers(10, 41)), seed=seed * 100_000 + 50_000 + i,
                        alpha=0.05, sigma=1.5, minibatch=4096, rate=60.0))
    return out


def serve_member(p: dict) -> Workload:
    w = batch_member(p)
    w.name = f"serve8[{p['index']}]"
    return w


NAMED = {
    "mixture10_d8": mixture10_d8,
    "mixture30_d16": mixture30_d16,
    "student50_d32": student50_d32,
    "uniform_d16": lambda seed=0, n=1 << 20: uniform(16, seed, n),
    "uniform_d32": lambda seed=0, n=1 << 20: uniform(32, seed, n),
}


def make(name: str, seed: int = 0, n: int | None = None) -> Workload:
    f = NAMED[name]
    return f(seed) if n is None else f(seed, n=n)


def random_case(rng: np.random.Generator, n: int, d: int, L: int, k: int,
                boost: float = 1.0, adjust: float = 1.0,
                scale: float = 3.0) -> Workload:
    """Small unstructured case for edge tests: uniform points and landmarks,
    2-D landmarks uniform in [0, 10)^2."""
    X = (rng.standard_normal((n, d)) * scale).astype(np.float32)
    hi = (rng.standard_normal((L, d)) * scale).astype(np.float32)
    lo = rng.uniform(0.0, 10.0, (L, 2)).astype(np.float32)
    return Workload("random", X, hi, lo, k=k, boost=boost, adjust=adjust)
