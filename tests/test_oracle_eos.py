"""Pins of the oracle's stellar EOS and temperature-guess network.

The e-/e+ gas is checked against closed forms (complete Fermi-Dirac integrals
as polylogarithms, the non-degenerate and completely degenerate limits), an
independent quadrature library, thermodynamic identities, and round trips of
the Newton inversion; the network's gradient against finite differences.
"""
import math

import numpy as np
import pytest

import oracle as O

K_B = 1.380649e-16
ME_C2 = 8.1871057769e-7
N_A = 6.02214076e23
H = 6.62607015e-27
C_L = 2.99792458e10
A_RAD = 7.565733250e-15
X = [0.5, 0.5]
A, Z = [16.0, 28.0], [8.0, 14.0]


@pytest.fixture(scope="module")
def table():
    return O.EosTable(nrho=321, nT=241)   # 80 nodes per decade in rho Y_e and T


@pytest.mark.parametrize("k", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("eta", [-30.0, -5.0, 0.0, 3.0, 20.0, 200.0, 1000.0, 2500.0])
def test_fd_integral_nonrelativistic_polylog(k, eta):
    """b -> 0: F_k(eta) = -Gamma(k + 1) Li_{k+1}(-e^eta), up to the strongly
    degenerate electrons at the cold, dense corner of the table (eta ~ 2000)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    exact = float(mpmath.re(-mpmath.gamma(k + 1) * mpmath.polylog(k + 1, -mpmath.exp(mpmath.mpf(eta)))))
    got = O.fd(k, eta, 1e-22)
    assert abs(got - exact) <= 1e-13 * abs(exact), (got, exact)


@pytest.mark.parametrize("beta", [0.1, 1.0, 5.0])
@pytest.mark.parametrize("eta", [-3.0, 2.0, 30.0])
def test_fd_integral_relativistic_vs_quadrature_library(beta, eta):
    integrate = pytest.importorskip("scipy.integrate")
    for k in (0.5, 1.5, 2.5):
        f = lambda x: x ** k * math.sqrt(1 + 0.5 * beta * x) / (math.exp(min(x - eta, 700)) + 1)
        pts = [max(eta, 0.0)] if eta > 0 else None
        ref, _ = integrate.quad(f, 0, max(eta, 0) + 200, points=pts, epsabs=0, epsrel=1e-13, limit=500)
        got = O.fd(k, eta, beta)
        assert abs(got - ref) <= 1e-11 * ref, (k, got, ref)


def test_nondegenerate_limit():
    # P = n k T for a non-degenerate gas at any temperature (no pairs here)
    rho, ye, T = 1e-2, 0.5, 1e8
    r = O.ep_direct(rho, ye, T)
    n = rho * ye * N_A
    assert abs(r["P"] / (n * K_B * T) - 1) < 1e-6
    # kinetic energy 3/2 n k T once k T << m_e c^2 (b = 1.7e-6 here)
    rho, T = 1e-8, 1e4
    r = O.ep_direct(rho, ye, T)
    n = rho * ye * N_A
    assert abs(r["e"] * rho / (1.5 * n * K_B * T) - 1) < 1e-5


@pytest.mark.parametrize("rho,T", [(1e8, 1e7), (3e7, 1e7), (1e8, 3e7)])
def test_degenerate_entropy_sommerfeld(rho, T):
    """Strong degeneracy: s = (pi^2 / 3) k^2 T g(E_F), g = 8 pi p_F E_F / (c^2 h^3)
    the density of states at the Fermi surface; the next term of the
    expansion is O((pi / eta)^2) relative."""
    n = rho * N_A
    pf = H * (3 * n / (8 * math.pi)) ** (1 / 3)
    ef = math.sqrt((pf * C_L) ** 2 + ME_C2 ** 2)
    g = 8 * math.pi * pf * ef / (C_L ** 2 * H ** 3)
    s_vol = math.pi ** 2 / 3 * K_B ** 2 * T * g
    r = O.ep_direct(rho, 1.0, T)
    assert r["eta"] > 500
    assert abs(r["s"] * rho / s_vol - 1) <= 10 * (math.pi / r["eta"]) ** 2, (r["s"] * rho, s_vol)


def test_complete_degeneracy_chandrasekhar():
    rho, ye, T = 1e8, 1.0, 1e6
    n = rho * ye * N_A
    me = ME_C2 / C_L ** 2
    x = (3 * n / (8 * math.pi)) ** (1 / 3) * H / (me * C_L)
    p_chandra = math.pi * me ** 4 * C_L ** 5 / (3 * H ** 3) * (
        x * (2 * x * x - 3) * math.sqrt(1 + x * x) + 3 * math.asinh(x))
    r = O.ep_direct(rho, ye, T)
    assert abs(r["P"] / p_chandra - 1) < 1e-5, (r["P"], p_chandra)


def _points():
    """The stellar box's range on a grid, plus seeded points over the table."""
    pts = [(rho, T) for rho in (1e5, 3e5, 1e6, 3e6, 1e7) for T in (1.1e8, 4e8, 1.3e9, 3e9)]
    rng = np.random.default_rng(1)
    pts += [(10 ** rng.uniform(4.3, 7.9), 10 ** rng.uniform(7.2, 9.95)) for _ in range(24)]
    return pts


def test_table_vs_direct_quadrature(table):
    """Biquintic Hermite interpolation of the free energy (Sect. 2.2) at 80
    nodes per decade against the exact derivatives of the integrals at the
    same points: first-derivative quantities O(h^5), second-derivative ones
    (c_v, gamma_c, dP/drho, dP/dT) O(h^4)."""
    cfg = O.stellar_cfg(A, Z, table)
    cfgd = O.stellar_cfg(A, Z, None)
    worst = {}
    for rho, T in _points():
        a, b = O.eos_rt(cfg, rho, T, X), O.eos_rt(cfgd, rho, T, X)
        for k in ("P", "e", "gamma_e", "gamma_c", "cv", "dPdT", "dPdr"):
            worst[k] = max(worst.get(k, 0), abs(a[k] - b[k]) / abs(b[k]))
    assert worst["P"] < 1e-8 and worst["e"] < 1e-8 and worst["gamma_e"] < 1e-8, worst
    for k in ("cv", "gamma_c", "dPdT", "dPdr"):
        assert worst[k] < 1e-6, worst


def test_interpolation_order():
    """Halving the node spacing divides the interpolation error of first-
    derivative quantities by ~2^5 and of second-derivative ones by ~2^4 (a
    bicubic table would give 2^3 and 2^2)."""
    cfgd = O.stellar_cfg(A, Z, None)
    rng = np.random.default_rng(3)
    pts = [(10 ** rng.uniform(5.2, 6.8) / 0.5, 10 ** rng.uniform(8.6, 9.4)) for _ in range(12)]
    ref = [O.eos_rt(cfgd, r, T, X) for r, T in pts]
    err = []
    for per in (20, 40):
        tb = O.EosTable(lrhoye=(5.0, 7.0), nrho=2 * per + 1, lT=(8.5, 9.5), nT=per + 1)
        cfg = O.stellar_cfg(A, Z, tb)
        w = {}
        for (r, T), b in zip(pts, ref):
            a = O.eos_rt(cfg, r, T, X)
            for k in ("e", "gamma_e", "cv", "gamma_c"):
                w[k] = max(w.get(k, 0), abs(a[k] - b[k]) / abs(b[k]))
        err.append(w)
    for k in ("e", "gamma_e"):
        assert err[0][k] / err[1][k] > 16, (k, err)
    for k in ("cv", "gamma_c"):
        assert err[0][k] / err[1][k] > 11, (k, err)


def test_table_reproduces_direct_values_at_nodes():
    """At a node the interpolant takes the node's f and its derivatives, so
    the EOS there equals the direct evaluation to rounding."""
    tb = O.EosTable(lrhoye=(5.0, 7.0), nrho=21, lT=(8.5, 9.5), nT=11)
    cfg, cfgd = O.stellar_cfg(A, Z, tb), O.stellar_cfg(A, Z, None)
    ye = 0.5
    for i, j in ((3, 2), (10, 5), (17, 9)):
        rho = 10 ** (5.0 + 0.1 * i) / ye
        T = 10 ** (8.5 + 0.1 * j)
        a, b = O.eos_rt(cfg, rho, T, X), O.eos_rt(cfgd, rho, T, X)
        for k in ("P", "e", "cv", "dPdT", "dPdr", "gamma_c"):
            assert abs(a[k] - b[k]) <= 1e-11 * abs(b[k]), (k, a[k], b[k])


@pytest.mark.parametrize("rho,T", [(1e5, 1e8), (3e6, 1.3e9), (1e7, 3e9), (2e4, 1e10), (2e8, 1e8)])
def test_taylor_derivatives_match_direct_combinations(rho, T):
    """The table's node values come from truncated Taylor arithmetic; f,
    f_x = n eta k T, f_y = -T s and f_xy = n k T (eta + d eta/d ln T) also
    follow from their own combinations of the integrals (P, E, s and
    dn/db).  For degenerate electrons f_y and f_xy are small differences
    (relative size (pi / eta)^2) of terms of size |f| + |f_x|: there the
    rounding of those terms bounds the agreement."""
    n = rho * 0.5 * N_A
    d, f = O.ep_derivs(n, T), O.ep_first(n, T)
    big = abs(f[0]) + abs(f[1])
    for i, j in ((0, 0), (1, 1), (2, 2), (5, 3)):
        assert abs(d[i] - f[j]) <= 1e-12 * abs(f[j]) + 1e-14 * big, (i, d[i], f[j])


@pytest.mark.parametrize("rho,T", [(1e5, 1e8), (3e6, 1.3e9), (1e7, 3e9), (2e4, 1e10)])
def test_taylor_higher_derivatives_vs_finite_differences(rho, T):
    """f_xx, f_yy, f_xxy, f_xyy, f_xxyy against fourth-order central
    differences (step 0.002 in ln n or ln T, truncation error ~1e-10) of the
    lower derivatives."""
    n = rho * 0.5 * N_A
    h = 2e-3
    d = O.ep_derivs(n, T)

    def fd(fun):
        return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)

    dx = lambda k: fd(lambda s: O.ep_derivs(n * math.exp(s), T)[k])
    dy = lambda k: fd(lambda s: O.ep_derivs(n, T * math.exp(s))[k])
    # (index, finite difference): f_xx = d_x f_x, f_yy = d_y f_y,
    # f_xxy = d_x f_xy, f_xyy = d_y f_xy, f_xxyy = d_y f_xxy
    for i, v in ((3, dx(1)), (4, dy(2)), (6, dx(5)), (7, dy(5)), (8, dy(6))):
        assert abs(d[i] - v) <= 5e-9 * abs(d[i]), (i, d[i], v)


def test_thermodynamic_consistency_of_the_table(table):
    """(de/drho)_T = (P - T (dP/dT)_rho) / rho^2 holds for the interpolated EOS."""
    cfg = O.stellar_cfg(A, Z, table)
    for rho, T in ((2e5, 3.3e8), (5e6, 2.1e9), (1e7, 1.2e9)):
        h = 1e-5
        ep = O.eos_rt(cfg, rho * (1 + h), T, X)["e"]
        em = O.eos_rt(cfg, rho * (1 - h), T, X)["e"]
        r = O.eos_rt(cfg, rho, T, X)
        lhs = (ep - em) / (2 * h * rho)
        rhs = (r["P"] - T * r["dPdT"]) / rho ** 2
        assert abs(lhs - rhs) <= 1e-5 * abs(r["P"] / rho ** 2), (lhs, rhs)


def test_gamma_c_is_the_adiabatic_sound_speed(table):
    """c_s^2 = (dP/drho)_s from an explicit adiabat de = P / rho^2 drho."""
    cfg = O.stellar_cfg(A, Z, table)
    for rho, T in ((3e5, 5e8), (4e6, 2.5e9)):
        r0 = O.eos_rt(cfg, rho, T, X)
        d = 1e-5 * rho
        target = r0["e"] + r0["P"] / rho ** 2 * d
        r1 = O.eos_invert(cfg, rho + d, target, X, T)
        cs2_fd = (r1["P"] - r0["P"]) / d
        cs2 = r0["gamma_c"] * r0["P"] / rho
        assert abs(cs2_fd / cs2 - 1) < 1e-4, (cs2_fd, cs2)


def test_newton_round_trip_and_guess_independence(table):
    """T -> e -> T; the attainable accuracy is the rounding of e amplified by
    the condition number e / (c_v T) (large for degenerate electrons)."""
    cfg = O.stellar_cfg(A, Z, table)
    for rho in (1e5, 1e6, 1e7):
        for T in (1.2e8, 7e8, 2.9e9):
            r = O.eos_rt(cfg, rho, T, X)
            cond = max(1.0, r["e"] / (r["cv"] * T))
            tol = max(1e-12, 2e-14 * cond) * T
            ts = [O.eos_invert(cfg, rho, r["e"], X, g)["T"] for g in (1.05e8, 1e9, 8e9)]
            for t in ts:
                assert abs(t - T) <= tol, (rho, T, t, cond)
            assert max(ts) - min(ts) <= tol


def test_radiation_dominated_limit(table):
    cfg = O.stellar_cfg(A, Z, table)
    rho, T = 1e4 * 2, 9e9     # rho Y_e = 1e4, radiation- and pair-dominated
    r = O.eos_rt(cfg, rho, T, X)
    assert r["P"] > A_RAD * T ** 4 / 3


# ---------------------------------------------------------------------------
# temperature-guess network (3 -> 64 -> 64 -> 1, tanh)
# ---------------------------------------------------------------------------

def _nparams(nin, nh):
    return nh * nin + nh + nh * nh + nh + nh + 1


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nin, nh = 3, 8
    w = rng.normal(scale=0.5, size=_nparams(nin, nh))
    x = rng.normal(size=(20, nin))
    t = rng.normal(size=20)
    loss, g = O.mlp_loss_grad(w, nin, nh, x, t)
    for i in rng.choice(len(w), 25, replace=False):
        e = np.zeros_like(w)
        e[i] = 1e-6
        lp, _ = O.mlp_loss_grad(w + e, nin, nh, x, t)
        lm, _ = O.mlp_loss_grad(w - e, nin, nh, x, t)
        fdg = (lp - lm) / 2e-6
        assert abs(fdg - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fdg, g[i])


def test_mlp_forward_hand_computed():
    nin, nh = 1, 1
    # W1, b1, W2, b2, W3, b3
    w = np.array([2.0, -0.5, 1.5, 0.25, -3.0, 0.1])
    x = np.array([[0.3]])
    h1 = math.tanh(2.0 * 0.3 - 0.5)
    h2 = math.tanh(1.5 * h1 + 0.25)
    assert abs(O.mlp_forward(w, nin, nh, x)[0] - (-3.0 * h2 + 0.1)) < 1e-15
