"""FP64 oracle for the SparStencil hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import, call, link or execute anything in this package.  The
product path (``paper_2506_22969_gb300``) never does, and this package never
imports the product.  The two share no code; the only thing both sides consume is
the seeded input generator, which holds none of the method's arithmetic.

Contents
  * :func:`run` / :func:`point` — the plain direct-loop stencil in FP64 (C, OpenMP over
    the slowest axis), following the stencil definition of Sec. 2.2 (correlation
    orientation fixed by the Box-2D9P pseudo-code: out[i][j] = sum c_ab in[i+a][j+b]).
  * :mod:`oracle.morph` — the paper's matrix formulation written out literally:
    flattening, the horizontal/vertical duplicate crush (Sec. 3.1, Eq. 3-4), the conflict
    graph (Def. 1), Algorithm 1 (hierarchical two-level matching), a brute-force solver
    for Problem 1, the 2:4 rule (Eq. 2) and the dense stencil matrix.

Where the paper is silent this oracle takes these readings: the stencil is a correlation
(offsets not flipped); a Dirichlet boundary is a zero halo re-imposed after every step, a
periodic one wraps indices; T steps are taken one by one in FP64 with no intermediate
rounding.  Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (closed forms, invariants, brute force, textbook special cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_stencil.so")
_lib = None

DIRICHLET = 0
PERIODIC = 1


def build(force: bool = False) -> str:
    """Compile stencil_ref.c into oracle/_build/liboracle_stencil.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "stencil_ref.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_stencil_run.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int64,
                                           dp, dp, dp, ctypes.c_int]
        lib.oracle_stencil_run.restype = ctypes.c_int
        lib.oracle_stencil_point.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int64,
                                             dp, i64p, dp]
        lib.oracle_stencil_point.restype = ctypes.c_int
        _lib = lib
    return _lib


def _bc_code(bc) -> int:
    if isinstance(bc, str):
        return {"dirichlet": DIRICHLET, "periodic": PERIODIC}[bc]
    return int(bc)


def _prep(u0, weights):
    u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    ndim = u.ndim
    if w.ndim != ndim or any(s != w.shape[0] for s in w.shape) or w.shape[0] % 2 != 1:
        raise ValueError("weights must be a (2r+1)^ndim cube matching the grid's dimensionality")
    return u, w, ndim, (w.shape[0] - 1) // 2


def run(u0, weights, bc, T: int, threads: int = 0) -> np.ndarray:
    """T stencil steps in FP64 on the whole grid (Sec. 2.2).

    u0: grid (any float dtype, promoted exactly to FP64); weights: dense cube of side
    2r+1 indexed by offset (+r), same axis order as the grid; bc: 'dirichlet' (zero
    outside the grid at every step) or 'periodic'.  Returns a new FP64 array.
    """
    lib = _load()
    u, w, ndim, r = _prep(u0, weights)
    dims = np.array(u.shape, dtype=np.int64)
    out = np.empty_like(u)
    scratch = np.empty_like(u)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_stencil_run(ndim, dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), r,
                                w.ctypes.data_as(dp), _bc_code(bc), int(T), u.ctypes.data_as(dp),
                                out.ctypes.data_as(dp), scratch.ctypes.data_as(dp), int(threads))
    if rc != 0:
        raise ValueError("oracle_stencil_run rejected its arguments")
    return out


def point(u0, weights, bc, T: int, index) -> float:
    """Value of one grid point after T steps, from its dependence cone only."""
    lib = _load()
    u, w, ndim, r = _prep(u0, weights)
    dims = np.array(u.shape, dtype=np.int64)
    idx = np.array(index, dtype=np.int64)
    val = ctypes.c_double(0.0)
    dp = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    rc = lib.oracle_stencil_point(ndim, dims.ctypes.data_as(i64p), r, w.ctypes.data_as(dp), _bc_code(bc), int(T),
                                  u.ctypes.data_as(dp), idx.ctypes.data_as(i64p), ctypes.byref(val))
    if rc != 0:
        raise ValueError("oracle_stencil_point rejected its arguments")
    return float(val.value)


def points(u0, weights, bc, T: int, indices, threads: int = 0) -> np.ndarray:
    """:func:`point` at many grid points, evaluated concurrently on host threads (the C
    routine keeps no shared state, and ctypes releases the GIL while it runs)."""
    from concurrent.futures import ThreadPoolExecutor
    u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64))  # converted once, shared
    n = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=n) as ex:
        return np.array(list(ex.map(lambda p: point(u, weights, bc, T, p), list(indices))), dtype=np.float64)


def rel_errors(x, ref):
    """rel-L2 = ||x-ref||_2/||ref||_2 and rel-Linf = max|x-ref|/max|ref|, in FP64."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = x - ref
    l2 = float(np.sqrt(np.sum(d * d)) / max(np.sqrt(np.sum(ref * ref)), 1e-300))
    linf = float(np.max(np.abs(d)) / max(np.max(np.abs(ref)), 1e-300)) if ref.size else 0.0
    return l2, linf


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
