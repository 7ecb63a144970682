"""The seeded synthetic inputs follow their stated recipes: the stratified
magnetoconvection box (the benchmark's workload), the Orszag-Tang vortex, the
ensemble's box sizes, and the stretched axis and sphere of the paper's
Poisson test.  Each is checked against its definition, not against stored
output, so a change to a generator that would silently change a workload
fails here."""
import math

import numpy as np

import workloads as W


def test_stratified_box_recipe():
    n = 32
    pr = W.stratified_box(n, n, n)
    assert pr.n == (n, n, n) and pr.lo == (0.0, 0.0, 0.0) and pr.hi == (1.0, 1.0, 1.0)
    assert pr.bc == ((W.PERIODIC,) * 2, (W.PERIODIC,) * 2, (W.REFLECT,) * 2)
    assert pr.g == (0.0, 0.0, -1.0) and pr.gamma == 5.0 / 3.0 and pr.cfl == 0.4
    # polytrope n = 1.5 with rho(0) = 1, rho(1) = 0.1, P = K rho^(1 + 1/n), hydrostatic under g = 1
    z = np.linspace(0.0, 1.0, 11)
    rho_hat, p_hat, K = W.polytrope_profile(z)
    assert abs(rho_hat[0] - 1.0) < 1e-15 and abs(rho_hat[-1] - 0.1) < 1e-15
    assert np.allclose(p_hat, K * rho_hat ** (1.0 + 1.0 / 1.5), rtol=1e-14, atol=0)
    h = 1e-5
    dpdz = (W.polytrope_profile(z + h)[1] - W.polytrope_profile(z - h)[1]) / (2 * h)
    assert np.allclose(dpdz, -rho_hat, rtol=1e-9, atol=0)
    # background point values at centres and faces, three ghost layers each side
    dz = 1.0 / n
    zc = (np.arange(-3, n + 3) + 0.5) * dz
    zf = np.arange(-3, n + 4) * dz
    bg = pr.bg
    assert np.array_equal(bg["rho_c"], W.polytrope_profile(zc)[0])
    assert np.array_equal(bg["p_f"], W.polytrope_profile(zf)[1])
    # isobaric density noise of amplitude 1e-3, at rest
    rho = pr.cons[0]
    rel = rho / bg["rho_c"][3:3 + n][:, None, None] - 1.0
    assert 0.99e-3 < np.abs(rel).max() <= 1e-3 * (1 + 1e-12) and abs(rel.mean()) < 1e-4
    assert not pr.cons[1:4].any()
    # uniform B_x with beta = 2 P_hat(1/2) / B^2 = 1e6; E = P/(gamma - 1) + B^2/2
    b0 = pr.bx[0, 0, 0]
    assert np.all(pr.bx == b0) and not pr.by.any() and not pr.bz.any()
    p_mid = W.polytrope_profile(np.array([0.5]))[1][0]
    assert math.isclose(2.0 * p_mid / b0 ** 2, 1e6, rel_tol=1e-12)
    p = bg["p_c"][3:3 + n][:, None, None]
    assert np.allclose(pr.cons[4], p / (pr.gamma - 1.0) + 0.5 * b0 ** 2, rtol=1e-14, atol=0)
    # heating uniform in z < 0.1, sized so (q 0.1 / rho_b)^(1/3) = 1e-3 c_s(z = 0)
    q = pr.heat
    zcell = (np.arange(n) + 0.5) / n
    assert q[0] > 0 and np.all(q[zcell < 0.1] == q[0]) and not q[zcell >= 0.1].any()
    cs0 = math.sqrt(pr.gamma * W.polytrope_profile(np.array([0.0]))[1][0] / 1.0)
    assert math.isclose((q[0] * 0.1 / 1.0) ** (1.0 / 3.0), 1e-3 * cs0, rel_tol=1e-12)
    # seeded: the same seed gives the same state, another seed another noise
    assert np.array_equal(W.stratified_box(n, n, n).cons, pr.cons)
    assert not np.array_equal(W.stratified_box(n, n, n, seed=1235).cons[0], rho)


def test_orszag_tang_recipe():
    n = 64
    pr = W.orszag_tang(n)
    assert pr.n == (n, n, 1) and pr.gamma == 5.0 / 3.0
    assert np.all(pr.cons[0] == 25.0 / (36.0 * math.pi))
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = 25.0 / (36.0 * math.pi)
    assert np.allclose(pr.cons[1][0], -rho * np.sin(2 * np.pi * Y), rtol=0, atol=1e-15)
    assert np.allclose(pr.cons[2][0], rho * np.sin(2 * np.pi * X), rtol=0, atol=1e-15)
    # face B from the discrete curl of A_z at the corners: divergence-free to
    # round-off, and close to B0 (-sin 2 pi y, sin 4 pi x) with B0 = 1/sqrt(4 pi)
    bx, by = pr.bx[0], pr.by[0]
    div = (bx[:, 1:] - bx[:, :-1]) * n + (by[1:, :] - by[:-1, :]) * n
    assert np.abs(div).max() < 1e-12
    b0 = 1.0 / math.sqrt(4 * math.pi)
    yc = (np.arange(n) + 0.5) / n
    assert np.allclose(bx, -b0 * np.sin(2 * np.pi * yc)[:, None] * np.ones(n + 1), atol=5e-3 * b0)
    assert np.allclose(by, b0 * np.sin(4 * np.pi * x)[None, :] * np.ones((n + 1, 1)), atol=5e-3 * b0)
    # E = p/(gamma - 1) + rho u^2/2 + B_c^2/2 with p = 5/(12 pi)
    bcx = 0.5 * (bx[:, 1:] + bx[:, :-1])
    bcy = 0.5 * (by[1:, :] + by[:-1, :])
    kin = 0.5 * (pr.cons[1][0] ** 2 + pr.cons[2][0] ** 2) / rho
    E = 5.0 / (12.0 * math.pi) / (2.0 / 3.0) + kin + 0.5 * (bcx ** 2 + bcy ** 2)
    assert np.allclose(pr.cons[4][0], E, rtol=1e-14, atol=0)


def test_ensemble_box_sizes():
    dims = W.ensemble_dims()
    assert len(dims) == 24 and all(e in (64, 96, 128, 160, 192) for d in dims for e in d)
    assert dims == W.ensemble_dims()                  # seeded
    cells = sum(a * b * c for a, b, c in dims)
    assert 4.0e7 < cells < 6.0e7 and cells == 47_906_816, cells


def test_paper_poisson_inputs():
    n = 64
    xf = W.stretched_faces(n)
    eta = -1.0 + 2.0 * np.arange(n + 1) / n
    assert np.allclose(xf, 0.25 * (eta + eta ** 5), rtol=0, atol=1e-16)
    assert xf[0] == -0.5 and xf[-1] == 0.5 and np.allclose(xf, -xf[::-1], atol=1e-16)
    dxf = np.diff(xf)
    # dx/deta = (1 + 5 eta^4)/4: cells about six times wider at the edges than at the centre
    assert math.isclose(dxf.max() / dxf.min(), 6.0, rel_tol=0.1)
    rho = W.sphere_density([xf] * 3)
    xc = 0.5 * (xf[1:] + xf[:-1])
    z, y, x = np.meshgrid(xc, xc, xc, indexing="ij")
    r2 = x * x + y * y + z * z
    assert np.array_equal(rho > 0, r2 < 0.25 ** 2)
    inside = r2 < 0.25 ** 2
    assert np.allclose(rho[inside], (1 - r2[inside] / 0.0625) ** 2, rtol=1e-15, atol=0)
    assert np.array_equal(rho, rho[::-1]) and np.array_equal(rho, rho.transpose(2, 1, 0))


def test_stellar_box_recipe():
    n = 32
    pr = W.stellar_box(n, n, n)
    L = W.STELLAR_L
    assert pr.hi == (L, L, L) and pr.eos == "stellar" and pr.nspec == 2
    assert W.STELLAR_RHO_BASE == 1e7 and W.STELLAR_RHO_TOP == 1e5
    assert list(W.STELLAR_X) == [0.5, 0.5] and list(W.STELLAR_A) == [16.0, 28.0]
    bg = pr.bg
    dz = L / n
    # the polytrope starts at rho_base at z = 0 and reaches rho_top at L (1 + 4/n), so the
    # three ghost layers above the box stay inside [rho_top, rho_base]
    assert math.isclose(bg["rho_f"][3], 1e7, rel_tol=1e-14)
    assert bg["rho_f"].min() > 1e5 and bg["rho_f"].max() < 1e8 and bg["rho_c"].min() > 1e5
    K = bg["p_f"][3] / bg["rho_f"][3] ** (5.0 / 3.0)
    assert np.allclose(bg["p_f"], K * bg["rho_f"] ** (5.0 / 3.0), rtol=1e-13, atol=0)
    # hydrostatic under the stored g: d P / dz = -rho g on the faces' closed form
    g0 = -pr.g[2]
    rho_f13 = bg["rho_f"] ** (1.0 / 1.5)
    assert np.allclose(np.diff(rho_f13), -g0 * dz / (K * 2.5), rtol=1e-9, atol=0)
    z_top = L * (1 + 4.0 / n)
    assert math.isclose((1e7 ** (1 / 1.5) - g0 * z_top / (K * 2.5)) ** 1.5, 1e5, rel_tol=1e-10)
    # composition, rest, isobaric noise, uniform B_x with beta 1e6 at mid-height
    prim = pr.meta["prim"]
    assert np.all(prim["X"] == 0.5) and not prim["vel"].any()
    rel = prim["rho"] / bg["rho_c"][3:3 + n][:, None, None] - 1.0
    assert np.abs(rel).max() <= 1e-3 * (1 + 1e-12)
    b0 = pr.bx[0, 0, 0]
    p_mid = K * ((1e7 ** (1 / 1.5) - g0 * 0.5 * L / (K * 2.5)) ** 1.5) ** (5.0 / 3.0)
    assert np.all(pr.bx == b0) and math.isclose(2 * p_mid / b0 ** 2, 1e6, rel_tol=1e-10)
