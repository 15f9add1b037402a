"""Pins for the FP64 stencil oracle: closed forms, invariants, brute force, library special cases.

Each test fixes the oracle to something other than itself, chosen so that a plausible
mistake (a dropped term, a wrong sign or axis, a transposed offset, a wrong boundary)
fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import morph
from paper_2506_22969_gb300 import inputs


def _rng(seed):
    return np.random.default_rng(seed)


def test_orientation_is_correlation(oracle_mod):
    """Sec. 2.2 (Box-2D9P pseudo-code): out[i][j] = sum_ab c_ab * in[i+a][j+b].
    A unit impulse at x* therefore produces w[o] at x* - o (no kernel flip)."""
    w = np.arange(1, 10, dtype=np.float64).reshape(3, 3) / 16.0
    u = np.zeros((7, 9))
    u[3, 4] = 1.0
    out = oracle_mod.run(u, w, "periodic", 1)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            assert out[3 - a, 4 - b] == w[a + 1, b + 1]
    assert np.count_nonzero(out) == 9


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_quadratic_field_exact(oracle_mod, bc):
    """Quadratic field, asymmetric dyadic weights: every interior value after one step equals
    the exact rational sum_o w[o] u(x+o) (Python Fractions, written from the polynomial)."""
    a, b, c, d, e, f = 3, -2, 5, 7, -11, 13
    H, W = 12, 14
    y, x = np.mgrid[0:H, 0:W]
    u = a * y * y + b * x * x + c * x * y + d * y + e * x + f
    w = np.array([[1, 2, 3], [4, 20, 5], [6, 7, 8]], dtype=np.float64) / 64.0
    out = oracle_mod.run(u.astype(np.float64), w, bc, 1)
    for yy in range(1, H - 1):
        for xx in range(1, W - 1):
            exact = Fraction(0)
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    Y, X = yy + oy, xx + ox
                    val = a * Y * Y + b * X * X + c * X * Y + d * Y + e * X + f
                    exact += Fraction(int(w[oy + 1, ox + 1] * 64), 64) * val
            assert out[yy, xx] == float(exact)


def test_heat2d_laplacian_on_quadratic(oracle_mod):
    """Heat-2D (centre 0.5, axis neighbours 0.125) on u = a y^2 + b x^2 + ... adds exactly
    0.25 (a + b) per step at interior points (the discrete Laplacian of a quadratic)."""
    w = inputs.stencil_weights("star", 2, 1, "heat").astype(np.float64)
    H, W = 10, 11
    y, x = np.mgrid[0:H, 0:W]
    a, b = 4, -3
    u = a * y * y + b * x * x + 2 * x * y - y + 5 * x + 1.0
    out = oracle_mod.run(u, w, "dirichlet", 1)
    np.testing.assert_array_equal(out[1:-1, 1:-1], u[1:-1, 1:-1] + 0.25 * (a + b))


@pytest.mark.parametrize("T", [1, 7, 40])
def test_fourier_mode_periodic(oracle_mod, T):
    """Periodic: u = Re(exp(i theta.x)) is an eigenvector; u_T = Re(lambda^T exp(i theta.x)),
    lambda(theta) = sum_o w[o] exp(i theta.o) (correlation sign)."""
    w = inputs.stencil_weights("box", 2, 2, "random", seed=9).astype(np.float64)
    H, W = 24, 20
    p, q = 3, 5
    th = np.array([2 * np.pi * p / H, 2 * np.pi * q / W])
    y, x = np.mgrid[0:H, 0:W]
    phase = th[0] * y + th[1] * x
    lam = 0j
    for oy in range(-2, 3):
        for ox in range(-2, 3):
            lam += w[oy + 2, ox + 2] * np.exp(1j * (th[0] * oy + th[1] * ox))
    u0 = np.cos(phase)
    ref = np.real(lam ** T * np.exp(1j * phase))
    out = oracle_mod.run(u0, w, "periodic", T)
    assert np.max(np.abs(out - ref)) < 1e-12


@pytest.mark.parametrize("ndim,T", [(2, 5), (2, 60), (3, 9)])
def test_sine_mode_dirichlet(oracle_mod, ndim, T):
    """Dirichlet zero, symmetric radius-1 star: prod_i sin(pi p_i (x_i+1)/(N_i+1)) is an
    eigenvector with lambda = w0 + sum_i 2 w_i cos(pi p_i/(N_i+1))."""
    dims = (13, 17, 11)[:ndim]
    ps = (2, 3, 4)[:ndim]
    w = np.zeros((3,) * ndim)
    c = (1,) * ndim
    w[c] = 0.4
    axis_w = [0.11, 0.07, 0.12][:ndim]
    for a in range(ndim):
        for o in (-1, 1):
            idx = list(c)
            idx[a] += o
            w[tuple(idx)] = axis_w[a]
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    u0 = np.ones(dims)
    lam = 0.4
    for a in range(ndim):
        u0 = u0 * np.sin(np.pi * ps[a] * (grids[a] + 1) / (dims[a] + 1))
        lam += 2 * axis_w[a] * np.cos(np.pi * ps[a] / (dims[a] + 1))
    out = oracle_mod.run(u0, w, "dirichlet", T)
    assert np.max(np.abs(out - lam ** T * u0)) < 1e-12


def test_dense_matrix_pinned_by_fft():
    """Periodic S is block-circulant: S u = ifft2(fft2(u) * conj(fft2(w wrapped)))
    (numpy FFT as an independent routine); Dirichlet S equals periodic S on a grid padded
    with r zero cells, restricted to the interior."""
    rng = _rng(3)
    H, W, r = 6, 7, 1
    w = rng.random((3, 3))
    u = rng.random((H, W))
    S = morph.dense_stencil_matrix((H, W), w, "periodic")
    wp = np.zeros((H, W))
    for oy in range(-r, r + 1):
        for ox in range(-r, r + 1):
            wp[oy % H, ox % W] += w[oy + r, ox + r]
    ref = np.real(np.fft.ifft2(np.fft.fft2(u) * np.conj(np.fft.fft2(wp))))
    np.testing.assert_allclose((S @ u.ravel()).reshape(H, W), ref, atol=1e-13)
    Sd = morph.dense_stencil_matrix((H, W), w, "dirichlet")
    up = np.zeros((H + 2 * r, W + 2 * r))
    up[r:-r, r:-r] = u
    Sp = morph.dense_stencil_matrix(up.shape, w, "periodic")
    ref_d = (Sp @ up.ravel()).reshape(up.shape)[r:-r, r:-r]
    np.testing.assert_allclose((Sd @ u.ravel()).reshape(H, W), ref_d, atol=1e-13)


@pytest.mark.parametrize("dims,r,bc,T", [((5, 6), 1, "dirichlet", 4), ((5, 6), 1, "periodic", 5),
                                         ((7, 5), 2, "dirichlet", 3), ((4, 5, 3), 1, "periodic", 3),
                                         ((3, 4, 5), 1, "dirichlet", 4), ((11,), 2, "periodic", 6),
                                         # the widest cubes the planner accepts: 2D radius 9, 1D radius 60
                                         ((23, 25), 9, "periodic", 2), ((21, 22), 9, "dirichlet", 2),
                                         ((150,), 60, "periodic", 2), ((130,), 60, "dirichlet", 2)])
def test_brute_force_matrix_power(oracle_mod, dims, r, bc, T):
    """Tiny grids: the oracle equals S^T u with S the dense stencil matrix."""
    rng = _rng(sum(dims) + r + T)
    w = rng.random((2 * r + 1,) * len(dims)) - 0.3
    u = rng.random(dims)
    S = morph.dense_stencil_matrix(dims, w, bc)
    ref = np.linalg.matrix_power(S, T) @ u.ravel()
    np.testing.assert_allclose(oracle_mod.run(u, w, bc, T).ravel(), ref, rtol=1e-12, atol=1e-12)


def test_constant_field_invariant(oracle_mod):
    """Weights summing to s: a constant c maps to c s^T (periodic everywhere; Dirichlet at
    points farther than T*r from every edge)."""
    w = inputs.stencil_weights("box", 2, 1, "random", seed=4).astype(np.float64)
    s = float(np.sum(w))
    u = np.full((20, 22), 0.75)
    T = 5
    outp = oracle_mod.run(u, w, "periodic", T)
    np.testing.assert_allclose(outp, 0.75 * s ** T, rtol=1e-14)
    outd = oracle_mod.run(u, w, "dirichlet", T)
    np.testing.assert_allclose(outd[T:-T, T:-T], 0.75 * s ** T, rtol=1e-14)
    assert np.all(outd[0, :] < 0.75 * s ** T)


@pytest.mark.parametrize("ndim,bc", [(1, "periodic"), (1, "dirichlet"), (2, "periodic"), (2, "dirichlet"),
                                     (3, "dirichlet"), (3, "periodic")])
def test_point_oracle_matches_full(oracle_mod, ndim, bc):
    """The dependence-cone point oracle equals the full-grid oracle (both boundaries; the
    cone's half-width T*r exceeds the grid, so periodic windows wrap more than once)."""
    rng = _rng(11 + ndim)
    dims = {1: (37,), 2: (19, 23), 3: (9, 10, 11)}[ndim]
    r, T = {1: (3, 9), 2: (2, 7), 3: (1, 6)}[ndim]
    w = rng.random((2 * r + 1,) * ndim)
    u = rng.random(dims)
    full = oracle_mod.run(u, w, bc, T)
    pts = [tuple(rng.integers(0, d) for d in dims) for _ in range(12)] + [tuple([0] * ndim),
                                                                          tuple(d - 1 for d in dims)]
    for p in pts:
        assert abs(oracle_mod.point(u, w, bc, T, p) - full[p]) <= 1e-13 * max(1.0, abs(full[p]))


def test_zero_steps_is_identity(oracle_mod):
    u = _rng(5).random((6, 7))
    w = _rng(6).random((3, 3))
    np.testing.assert_array_equal(oracle_mod.run(u, w, "dirichlet", 0), u)


def _shifted(u, axis, step, bc):
    """u translated so that out[i] = u[i + step * e_axis]; zero where that leaves the grid
    under a Dirichlet boundary."""
    if bc == "periodic":
        return np.roll(u, -step, axis=axis)
    out = np.zeros_like(u)
    n = u.shape[axis]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if step >= 0:
        src[axis], dst[axis] = slice(step, n), slice(0, max(n - step, 0))
    else:
        src[axis], dst[axis] = slice(0, max(n + step, 0)), slice(-step, n)
    out[tuple(dst)] = u[tuple(src)]
    return out


@pytest.mark.parametrize("ndim,dims", [(1, (23,)), (2, (9, 11)), (3, (5, 6, 7))])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_degenerate_stencils_are_exact(oracle_mod, ndim, dims, bc):
    """Degenerate stencils of Sec. 2.2's update: all weights zero gives zeros; the centre
    weight alone gives the input back; a single unit weight at offset +-1 along one axis
    translates the grid by T cells per T steps (a plain array shift, zeros entering under a
    Dirichlet boundary).  Every value is exact in FP64.  A wrong axis, offset sign or
    boundary rule moves cells and fails this."""
    u = _rng(9).random(dims)
    T = 4
    zero = np.zeros((3,) * ndim)
    assert np.all(oracle_mod.run(u, zero, bc, T) == 0.0)
    ident = zero.copy()
    ident[(1,) * ndim] = 1.0
    np.testing.assert_array_equal(oracle_mod.run(u, ident, bc, T), u)
    for axis in range(ndim):
        for sign in (1, -1):
            w = zero.copy()
            idx = [1] * ndim
            idx[axis] = 1 + sign
            w[tuple(idx)] = 1.0
            np.testing.assert_array_equal(oracle_mod.run(u, w, bc, T), _shifted(u, axis, sign * T, bc))


def test_rel_errors(oracle_mod):
    ref = np.array([1.0, -2.0, 2.0])
    x = np.array([1.0, -2.0, 2.5])
    l2, linf = oracle_mod.rel_errors(x, ref)
    assert abs(l2 - 0.5 / 3.0) < 1e-15 and abs(linf - 0.25) < 1e-15


def test_input_generator_exact_and_seeded():
    a = inputs.uniform01(7, (5, 6))
    b = inputs.uniform01(7, (5, 6))
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.float32 and np.all(a >= 0) and np.all(a < 1)
    # exact: every value is a multiple of 2^-24
    assert np.all((a.astype(np.float64) * 2 ** 24) % 1 == 0)
    # splitmix64 reference value: first output of seed 0 (published test vector)
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    w = inputs.stencil_weights("box", 2, 3, "gaussian")
    assert abs(float(np.sum(w.astype(np.float64))) - 1.0) < 1e-6
    h = inputs.stencil_weights("star", 2, 1, "heat")
    assert h[1, 1] == 0.5 and h[0, 1] == 0.125 and h[0, 0] == 0.0
