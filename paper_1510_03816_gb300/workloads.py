"""Seeded synthetic landmark workloads.

Both the CUDA library's tests/benchmark and the CPU oracle take their inputs
from here.  The module holds no arithmetic of the method (no kernel, no
right-hand side, no gain): it only draws landmark sets X, targets Y and, where
a configuration asks for one, a starting momentum, with numpy's PCG64 from a
fixed seed.  The shapes mirror the paper's experiments (closed planar curves
of landmarks, Sec. 7 Examples 1-2), scaled into the unit square/cube.

Workloads (all positions (n, dim) float64):
  circle_to_ellipse   N points on a circle r=0.3 about (0.5, 0.5); target the
                      same angles on an ellipse with semi-axes 0.35, 0.22
                      plus seeded radial noise U(-0.01, 0.01).  Tent sigma=0.25.
  fourier_curve_warp  N points equispaced in arc length on the closed curve
                      r(t) = 0.3 + sum_{k=1..8} a_k cos(k t + f_k),
                      a_k ~ N(0, (0.02/k)^2), f_k ~ U[0, 2 pi); target under the
                      warp (x + 0.05 sin 2 pi y, y + 0.05 sin 2 pi x).  Gaussian
                      sigma = 0.1.
  jittered_grid       a side x side grid in [0,1]^2 with each point uniform in
                      its cell; target X + u(X), u = sum of 16 Fourier modes
                      with integer wave vectors 1 <= |k|_inf <= 4, random unit
                      directions and phases, scaled so max |u(X_i)| = 0.02.
                      Tent with sigma = sqrt(32 / (pi N)) (32 neighbours on
                      average).
  star_surface_3d     N directions on a Fibonacci sphere, radius
                      0.3 + 0.03 g(w) with g a seeded polynomial of degree <= 6
                      on the sphere (the span of spherical harmonics l <= 6),
                      max|g| = 1, centred at (0.5, 0.5, 0.5); target the cyclic
                      sine warp x_a + 0.02 sin(2 pi x_{a+1}) plus N(0, 0.005^2)
                      noise; starting momentum p0 = h0 (Y - X).  Gaussian
                      sigma = 0.05, lambda = 100.
  batched_curves      512 problems, N_b = round(exp(U(ln 32, ln 8192))); each a
                      circle_to_ellipse pair with N_b points; even b tent
                      sigma = 0.2, odd b Gaussian sigma = 0.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 1510

GAUSS, TENT, EXPCONE = 0, 1, 2


@dataclass
class Problem:
    name: str
    X: np.ndarray
    Y: np.ndarray
    kernel: int
    sigma: float
    steps: int
    eps: float = 1e-6
    maxit: int = 200
    lam: float = 0.0
    p0: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def dim(self) -> int:
        return int(self.X.shape[1])


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, stream]))


def circle_to_ellipse(n: int = 64, seed: int = SEED, stream: int = 1, sigma: float = 0.25,
                      kernel: int = TENT, steps: int = 50) -> Problem:
    rng = _rng(seed, stream)
    th = 2.0 * np.pi * np.arange(n) / n
    X = np.stack([0.5 + 0.3 * np.cos(th), 0.5 + 0.3 * np.sin(th)], axis=1)
    xi = rng.uniform(-0.01, 0.01, size=n)
    Y = np.stack([0.5 + (0.35 + xi) * np.cos(th), 0.5 + (0.22 + xi) * np.sin(th)], axis=1)
    return Problem("circle_to_ellipse", X, Y, kernel, sigma, steps)


def _arclength_curve(n: int, radius_fn, dense: int) -> np.ndarray:
    """n points equispaced in arc length on the closed polar curve r(t)."""
    t = np.linspace(0.0, 2.0 * np.pi, dense + 1)
    r = radius_fn(t)
    x = r * np.cos(t)
    y = r * np.sin(t)
    seg = np.hypot(np.diff(x), np.diff(y))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    targets = np.arange(n) * (s[-1] / n)
    tt = np.interp(targets, s, t)
    rr = radius_fn(tt)
    return np.stack([rr * np.cos(tt), rr * np.sin(tt)], axis=1)


def fourier_curve_warp(n: int = 4096, seed: int = SEED, stream: int = 2, sigma: float = 0.1,
                       steps: int = 100) -> Problem:
    rng = _rng(seed, stream)
    k = np.arange(1, 9)
    a = rng.normal(0.0, 0.02 / k)
    f = rng.uniform(0.0, 2.0 * np.pi, size=8)

    def radius(t):
        return 0.3 + np.sum(a[:, None] * np.cos(k[:, None] * t[None, :] + f[:, None]), axis=0)

    X = _arclength_curve(n, radius, dense=max(64 * n, 4096)) + 0.5
    Y = np.stack([X[:, 0] + 0.05 * np.sin(2 * np.pi * X[:, 1]),
                  X[:, 1] + 0.05 * np.sin(2 * np.pi * X[:, 0])], axis=1)
    return Problem("fourier_curve_warp", X, Y, GAUSS, sigma, steps)


def jittered_grid(side: int = 512, seed: int = SEED, stream: int = 3, steps: int = 100) -> Problem:
    rng = _rng(seed, stream)
    n = side * side
    ix, iy = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    jit = rng.uniform(0.0, 1.0, size=(n, 2))
    X = np.stack([(ix.ravel() + jit[:, 0]) / side, (iy.ravel() + jit[:, 1]) / side], axis=1)
    # 16 Fourier modes with integer wave vectors, 1 <= |k|_inf <= 4
    ks = []
    while len(ks) < 16:
        kk = rng.integers(-4, 5, size=2)
        if np.max(np.abs(kk)) >= 1:
            ks.append(kk)
    ks = np.array(ks, dtype=np.float64)
    ang = rng.uniform(0.0, 2.0 * np.pi, size=16)
    dirs = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=16)
    arg = 2.0 * np.pi * (X @ ks.T) + ph[None, :]
    u = np.sin(arg) @ dirs
    u *= 0.02 / np.max(np.hypot(u[:, 0], u[:, 1]))
    sigma = math.sqrt(32.0 / (math.pi * n))
    return Problem("jittered_grid", X, X + u, TENT, sigma, steps)


def _fibonacci_sphere(n: int) -> np.ndarray:
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    th = golden * i
    return np.stack([rxy * np.cos(th), rxy * np.sin(th), z], axis=1)


def star_surface_3d(n: int = 16384, seed: int = SEED, stream: int = 4, sigma: float = 0.05,
                    steps: int = 100, lam: float = 100.0, h0: float = 0.004) -> Problem:
    rng = _rng(seed, stream)
    w = _fibonacci_sphere(n)
    # random polynomial of degree <= 6 in (x, y, z); on the unit sphere these
    # span exactly the spherical harmonics of degree <= 6
    g = np.zeros(n)
    for a in range(7):
        for b in range(7 - a):
            for c in range(7 - a - b):
                g += rng.normal() * w[:, 0] ** a * w[:, 1] ** b * w[:, 2] ** c
    g /= np.max(np.abs(g))
    r = 0.3 + 0.03 * g
    X = 0.5 + r[:, None] * w
    Y = X + 0.02 * np.sin(2.0 * np.pi * np.roll(X, -1, axis=1))
    Y = Y + rng.normal(0.0, 0.005, size=Y.shape)
    p0 = h0 * (Y - X)
    return Problem("star_surface_3d", X, Y, GAUSS, sigma, steps, lam=lam, p0=p0)


def batched_sizes(count: int = 512, seed: int = SEED, stream: int = 5, nmin: int = 32,
                  nmax: int = 8192) -> np.ndarray:
    rng = _rng(seed, stream)
    return np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))).astype(np.int64)


def batched_curves(count: int = 512, seed: int = SEED, nmin: int = 32, nmax: int = 8192,
                   steps: int = 50) -> list[Problem]:
    sizes = batched_sizes(count, seed, nmin=nmin, nmax=nmax)
    probs = []
    for b, nb in enumerate(sizes):
        if b % 2 == 0:
            pr = circle_to_ellipse(int(nb), seed=seed, stream=1000 + b, sigma=0.2, kernel=TENT, steps=steps)
        else:
            pr = circle_to_ellipse(int(nb), seed=seed, stream=1000 + b, sigma=0.1, kernel=GAUSS, steps=steps)
        pr.name = f"batched_curves[{b}]"
        probs.append(pr)
    return probs


def concentric_circles(n: int, r0: float, r1: float, center=(0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """n equispaced points on circles of radius r0 (X) and r1 (Y) at the same angles."""
    th = 2.0 * np.pi * np.arange(n) / n
    c = np.asarray(center, dtype=np.float64)
    X = c + r0 * np.stack([np.cos(th), np.sin(th)], axis=1)
    Y = c + r1 * np.stack([np.cos(th), np.sin(th)], axis=1)
    return X, Y


def random_cloud(n: int, dim: int, seed: int = SEED, stream: int = 7, scale: float = 1.0,
                 pscale: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """Uniform positions in [0, scale]^dim and N(0, pscale^2) momenta (test inputs)."""
    rng = _rng(seed, stream)
    q = rng.uniform(0.0, scale, size=(n, dim))
    p = rng.normal(0.0, pscale, size=(n, dim))
    return q, p


def by_name(name: str, **kw) -> Problem:
    return {
        "circle_to_ellipse": circle_to_ellipse,
        "fourier_curve_warp": fourier_curve_warp,
        "jittered_grid": jittered_grid,
        "star_surface_3d": star_surface_3d,
    }[name](**kw)
