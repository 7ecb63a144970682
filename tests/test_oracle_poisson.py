"""Pins of the oracle's Poisson solver (Sect. 2.12).

* The three-point Laplacian on a non-uniform axis is the second derivative of
  the parabola through the three points, so it is exact on quadratics; the
  central gravity formula is exact on them too.
* The multipole boundary values approach the exact point-mass potential
  with distance at the rate of the first omitted order (monopole about the
  centre of mass: relative error ~ R^-2; with the quadrupole ~ R^-3; with the
  octupole ~ R^-4).
* BiCGSTAB converges to the discrete solution of a direct sparse solve of
  the same operator (assembled by applying the oracle to unit vectors).
* The paper's accuracy test (Eqs. coll1, coll2): the potential of the
  (1 - r^2/r0^2)^2 sphere on the (eta + eta^5)/4 stretched grid converges to
  the closed form at second order.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def centres(xf):
    return [0.5 * (a[1:] + a[:-1]) for a in xf]


def ghost_centres(xf):
    """Mirror images of the first and last centres in the boundary faces."""
    out = []
    for a in xf:
        c = 0.5 * (a[1:] + a[:-1])
        out.append((2 * a[0] - c[0], 2 * a[-1] - c[-1]))
    return out


def ghost_array(xf, f):
    """Ghost potentials of a function f(x, y, z) in the oracle's layout."""
    xc, gc = centres(xf), ghost_centres(xf)
    parts = []
    for side in (0, 1):   # x faces [nz][ny]
        z, y = np.meshgrid(xc[2], xc[1], indexing="ij")
        parts.append(f(np.full(z.shape, gc[0][side]), y, z).ravel())
    for side in (0, 1):   # y faces [nz][nx]
        z, x = np.meshgrid(xc[2], xc[0], indexing="ij")
        parts.append(f(x, np.full(z.shape, gc[1][side]), z).ravel())
    for side in (0, 1):   # z faces [ny][nx]
        y, x = np.meshgrid(xc[1], xc[0], indexing="ij")
        parts.append(f(x, y, np.full(y.shape, gc[2][side])).ravel())
    return np.concatenate(parts)


def cell_grid(xf):
    xc = centres(xf)
    z, y, x = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    return x, y, z


XF = [W.random_faces(9, 1), W.random_faces(7, 2, spread=0.6), W.random_faces(6, 3)]
QUAD = (0.7, -1.3, 0.4, 0.2, -0.5, 0.9, 2.0)


def quad(x, y, z):
    a, b, c, d, e, f, k = QUAD
    return a * x * x + b * y * y + c * z * z + d * x + e * y + f * z + k


def test_laplacian_exact_on_quadratics():
    P = O.Poisson(XF)
    x, y, z = cell_grid(XF)
    out = P.apply(quad(x, y, z), ghost_array(XF, quad))
    a, b, c = QUAD[:3]
    assert np.allclose(out, 2 * (a + b + c), rtol=0, atol=1e-10 * 2 * (abs(a) + abs(b) + abs(c)))
    # a cubic is not reproduced on a stretched axis (first order on non-uniform spacing)
    cub = lambda x, y, z: x ** 3
    err = np.abs(P.apply(cub(x, y, z), ghost_array(XF, cub)) - 6 * x).max()
    assert err > 1e-6


def test_gravity_exact_on_quadratics():
    P = O.Poisson(XF)
    x, y, z = cell_grid(XF)
    g = P.gravity(quad(x, y, z), ghost_array(XF, quad))
    a, b, c, d, e, f, _ = QUAD
    for got, want in zip(g, (-(2 * a * x + d), -(2 * b * y + e), -(2 * c * z + f))):
        assert np.abs(got - want).max() <= 1e-11


def direct_potential(xf, rho, pts, G=1.0):
    """-G sum m / |r - r'| over the cell masses m = rho V at their centres."""
    x, y, z = cell_grid(xf)
    V = np.einsum("k,j,i->kji", np.diff(xf[2]), np.diff(xf[1]), np.diff(xf[0]))
    m = (rho * V).ravel()
    r = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    return np.array([-G * np.sum(m / np.linalg.norm(r - p, axis=1)) for p in pts])


@pytest.mark.parametrize("lmax,order", [(0, 2), (2, 3), (3, 4)])
def test_multipole_error_falls_with_the_first_omitted_order(lmax, order):
    xf = [W.random_faces(10, 11), W.random_faces(9, 12), W.random_faces(8, 13)]
    rho = W.lumpy_density(xf, seed=5, floor=0.0)
    P = O.Poisson(xf, G=1.0, lmax=lmax)
    mom = P.moments(rho)
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(12, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    errs = []
    for R in (3.0, 6.0):
        pts = mom[1] + R * dirs
        exact = direct_potential(xf, rho, pts)
        errs.append(np.abs(P.multipole_phi(mom, pts) - exact).max() / np.abs(exact).max())
    rate = math.log2(errs[0] / errs[1])
    assert rate > order - 0.35, (lmax, errs, rate)


def test_multipole_moments_of_a_point_pair():
    """Two equal masses on the x axis: M = 2m, centre of mass between them,
    Q = m d^2 diag(4, -2, -2) for separation 2d, and the octupole vanishes
    by symmetry."""
    xf = [np.linspace(-0.5, 0.5, 11)] * 3
    rho = np.zeros((10, 10, 10))
    rho[5, 5, 2] = rho[5, 5, 7] = 3.0
    P = O.Poisson(xf)
    M, X, Q, Oc = P.moments(rho)
    m = 3.0 * 0.1 ** 3
    assert abs(M - 2 * m) < 1e-15
    assert np.allclose(X, [0.0, 0.05, 0.05], atol=1e-15)
    d = 0.25
    assert np.allclose(Q, m * d * d * np.diag([4.0, -2.0, -2.0]), atol=1e-15)
    assert np.abs(Oc).max() < 1e-15


def test_bicgstab_matches_a_direct_solve():
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    xf = [W.random_faces(6, 21), W.random_faces(5, 22), W.random_faces(4, 23)]
    rho = W.lumpy_density(xf, seed=9)
    P = O.Poisson(xf, G=0.7, lmax=3, criterion="relative", tol=1e-12, max_iter=500)
    phi, gh, its, res, st = P.solve(rho)
    assert st == 0 and res < 1e-12 and its > 3
    n = rho.size
    cols = []
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        cols.append(P.apply(e.reshape(rho.shape)).ravel())
    A = sp.csc_matrix(np.array(cols).T)
    b = 4 * np.pi * 0.7 * rho.ravel() - P.apply(np.zeros_like(rho), gh).ravel()
    ref = spla.spsolve(A, b)
    assert np.abs(phi.ravel() - ref).max() <= 1e-10 * np.abs(ref).max()
    # the ghost potentials are the multipole expansion at the ghost centres
    assert np.array_equal(gh, P.boundary(rho))


def sphere_phi(r, r0=0.25, rho0=1.0):
    M = 32 * np.pi * rho0 * r0 ** 3 / 105
    inner = -2 / 3 * np.pi * rho0 * r0 ** 2 + 4 * np.pi * rho0 * (r ** 2 / 6 - r ** 4 / (10 * r0 ** 2)
                                                                    + r ** 6 / (42 * r0 ** 4))
    return np.where(r <= r0, inner, -M / np.maximum(r, 1e-300))


def sphere_gr(r, r0=0.25, rho0=1.0):
    M = 32 * np.pi * rho0 * r0 ** 3 / 105
    inner = -4 * np.pi * rho0 * (r / 3 - 2 * r ** 3 / (5 * r0 ** 2) + r ** 5 / (7 * r0 ** 4))
    return np.where(r <= r0, inner, -M / np.maximum(r, 1e-300) ** 2)


def test_sphere_potential_converges_at_second_order():
    """The paper's accuracy test: monopole boundary values, absolute RMS
    residual below 1e-10, zero initial guess; L1 of phi and of the radial
    gravity against Eqs. coll1 / coll2."""
    errs, gerrs = [], []
    for n in (16, 32, 64):
        xf = [W.stretched_faces(n)] * 3
        rho = W.sphere_density(xf)
        P = O.Poisson(xf, G=1.0, lmax=0, criterion="absolute", tol=1e-10, max_iter=5000)
        phi, gh, its, res, st = P.solve(rho)
        assert st == 0 and res < 1e-10
        x, y, z = cell_grid(xf)
        r = np.sqrt(x * x + y * y + z * z)
        errs.append(np.abs(phi - sphere_phi(r)).mean())
        gx, gy, gz = P.gravity(phi, gh)
        gr = (gx * x + gy * y + gz * z) / r
        gerrs.append(np.abs(gr - sphere_gr(r)).mean())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    gorder = np.log2(np.array(gerrs[:-1]) / np.array(gerrs[1:]))
    assert order[-1] > 1.8 and gorder[-1] > 1.5, (errs, order, gerrs, gorder)
    assert errs[-1] < 1e-3 * abs(sphere_phi(np.array(0.0)))


def test_sphere_mass_converges_to_the_printed_closed_form():
    """The monopole of the paper's sphere: the cell masses rho V sum to
    M = 32 pi rho0 r0^3 / 105 (the closed form the paper prints with Eq.
    coll1), at second order on the stretched grid (midpoint rule), with the
    centre of mass at the origin and vanishing octupole by symmetry."""
    M_exact = 32 * np.pi * 1.0 * 0.25 ** 3 / 105
    errs = []
    for n in (16, 32, 64):
        xf = [W.stretched_faces(n)] * 3
        M, X, Q, Oc = O.Poisson(xf).moments(W.sphere_density(xf))
        errs.append(abs(M - M_exact) / M_exact)
        assert np.abs(X).max() < 1e-15
        assert np.abs(Oc).max() < 1e-15 * M
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3 and np.all(order > 1.8), (errs, order)
