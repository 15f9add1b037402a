"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the stencil method's arithmetic: it only draws grids and
weight cubes.  Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used counter-style:
z_i = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15).

  * uniform [0, 1) FP32  = (z >> 40) * 2^-24   (exact in FP32)
  * uniform [-1, 1) FP32 = 2 * u - 1           (exact in FP32)

Weight recipes (the paper's workloads, Table 2, with the benchmark workloads' weights):
  * 'heat'      — Heat-2D/3D: centre 0.5, each axis neighbour 0.5 / (2 * ndim) ... for 2D
                  this is centre 0.5 and four neighbours 0.125 (exact in FP16/BF16).
  * 'random'    — seeded positive U[0.05, 1) per stencil point, normalised to sum 1 in
                  FP64, then rounded to FP32.
  * 'gaussian'  — w(o) proportional to exp(-|o|^2 / (2 sigma^2)), sigma = 1.5, normalised
                  in FP64, rounded to FP32 (for a star, |o| is the axis distance).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n consecutive splitmix64 outputs (uint64) of stream `seed`, from index `start`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, shape) -> np.ndarray:
    """FP32 grid, uniform on [0, 1), exactly representable."""
    n = int(np.prod(shape))
    z = splitmix64(seed, n)
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32).reshape(shape)


def uniform_pm1(seed: int, shape) -> np.ndarray:
    """FP32 grid, uniform on [-1, 1), exactly representable."""
    return (2.0 * uniform01(seed, shape).astype(np.float64) - 1.0).astype(np.float32)


def stencil_mask(shape: str, ndim: int, radius: int) -> np.ndarray:
    """Boolean cube of side 2r+1: 'box' = all points, 'star' = centre plus the axes."""
    side = 2 * radius + 1
    if shape == "box":
        return np.ones((side,) * ndim, dtype=bool)
    if shape == "star":
        m = np.zeros((side,) * ndim, dtype=bool)
        c = (radius,) * ndim
        for a in range(ndim):
            for o in range(-radius, radius + 1):
                idx = list(c)
                idx[a] = radius + o
                m[tuple(idx)] = True
        return m
    raise ValueError(shape)


def stencil_weights(shape: str, ndim: int, radius: int, recipe: str, seed: int = 0,
                    sigma: float = 1.5) -> np.ndarray:
    """FP32 weight cube of side 2r+1 (offset-indexed, [z][y][x] order, centre at r)."""
    mask = stencil_mask(shape, ndim, radius)
    side = 2 * radius + 1
    w = np.zeros((side,) * ndim, dtype=np.float64)
    pts = np.argwhere(mask)
    if recipe == "heat":
        if shape != "star" or radius != 1:
            raise ValueError("the heat recipe is the radius-1 star")
        w[mask] = 0.5 / (2 * ndim)
        w[(radius,) * ndim] = 0.5
    elif recipe == "random":
        z = splitmix64(seed, len(pts), start=1 << 40)
        v = 0.05 + 0.95 * ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)
        for p, val in zip(pts, v):
            w[tuple(p)] = val
        w /= w.sum()
    elif recipe == "gaussian":
        for p in pts:
            o = p - radius
            d2 = float(np.sum(o.astype(np.float64) ** 2))
            w[tuple(p)] = np.exp(-d2 / (2.0 * sigma * sigma))
        w /= w.sum()
    else:
        raise ValueError(recipe)
    return w.astype(np.float32)


# The paper's workloads restated as single-run configurations (Table 2 shapes).
CONFIGS = {
    "heat1d": dict(name="Heat-1D 3-point 10240000, periodic, 10000 steps", shape="star", ndim=1, radius=1,
                   recipe="heat", dims=(10240000,), steps=10000, bc="periodic", grid="u01", seed=6),
    "1d5p": dict(name="1D5P 5-point 10240000, periodic, 10000 steps", shape="box", ndim=1, radius=2,
                 recipe="random", dims=(10240000,), steps=10000, bc="periodic", grid="u01", seed=7),
    "heat2d_512": dict(name="Heat-2D 5-point star 512^2, Dirichlet zero, 8 steps", shape="star", ndim=2, radius=1,
                       recipe="heat", dims=(512, 512), steps=8, bc="dirichlet", grid="u01", seed=1),
    "box2d9p_4096": dict(name="Box-2D 9-point 4096^2, periodic, 100 steps", shape="box", ndim=2, radius=1,
                         recipe="random", dims=(4096, 4096), steps=100, bc="periodic", grid="u01", seed=2),
    "heat3d_512": dict(name="Heat-3D 7-point star 512^3, Dirichlet zero, 50 steps", shape="star", ndim=3, radius=1,
                       recipe="random", dims=(512, 512, 512), steps=50, bc="dirichlet", grid="upm1", seed=3),
    "heat3d_256": dict(name="Heat-3D 7-point star 256^3, Dirichlet zero", shape="star", ndim=3, radius=1,
                       recipe="random", dims=(256, 256, 256), steps=50, bc="dirichlet", grid="upm1", seed=3),
    "box3d27p_256": dict(name="Box-3D 27-point 256^3, Dirichlet zero, 50 steps", shape="box", ndim=3, radius=1,
                         recipe="random", dims=(256, 256, 256), steps=50, bc="dirichlet", grid="upm1", seed=3),
    "star2d13p_8192": dict(name="Star-2D 13-point 8192^2, 200 steps", shape="star", ndim=2, radius=3,
                           recipe="gaussian", dims=(8192, 8192), steps=200, bc="periodic", grid="u01", seed=4),
    "box2d49p_8192": dict(name="Box-2D 49-point 8192^2, 200 steps", shape="box", ndim=2, radius=3,
                          recipe="gaussian", dims=(8192, 8192), steps=200, bc="periodic", grid="u01", seed=4),
}


def make_grid(kind: str, seed: int, dims) -> np.ndarray:
    if kind == "u01":
        return uniform01(seed, dims)
    if kind == "upm1":
        return uniform_pm1(seed, dims)
    raise ValueError(kind)
