"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties part of the oracle to something other than itself: a textbook
exact solution, a convergence order, a conservation law or symmetry, a closed
form, or a special case that reduces to a textbook solver.  The aim is that a
plausible slip anywhere in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from exact_riemann import sample, star_state

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        out[parts[0]] = float(parts[1])
    return out


# ---------------------------------------------------------------------------
# whole scheme, hydrodynamic limit: Sod vs the exact Riemann solution
# ---------------------------------------------------------------------------

def test_exact_solver_matches_textbook_star_state():
    g = _gold("sod_star_state.txt")
    p, u, rl, rr = star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(p - g["p_star"]) < 1e-5
    assert abs(u - g["u_star"]) < 1e-5
    assert abs(rl - g["rho_star_left"]) < 1e-5
    assert abs(rr - g["rho_star_right"]) < 1e-5


def test_sod_converges_to_exact_solution():
    errs = []
    for n in (100, 200, 400):
        pr = W.sod(n)
        st, t, _ = O.Oracle(pr).run_to(0.2)
        x = (np.arange(n) + 0.5) / n
        ex = sample(x, t, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
        rho = st["cons"][0, 0, 0]
        u = st["cons"][1, 0, 0] / rho
        errs.append(np.abs(rho - ex[0]).mean())
        assert np.abs(u - ex[1]).mean() < 0.02
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert errs[-1] < 2.0e-3, errs
    assert np.all(order > 0.75), order


# ---------------------------------------------------------------------------
# smooth MHD: linear Alfven waves converge at second order; CT keeps div B
# ---------------------------------------------------------------------------

def _alfven_err(pr, comp):
    st, t, _ = O.Oracle(pr).run_to(pr.meta["period"])
    return np.abs(st["cons"][comp] - pr.cons[comp]).mean() / pr.meta["amp"], st


def test_alfven_1d_second_order():
    errs = [_alfven_err(W.alfven_1d(n), 2)[0] for n in (64, 128, 256)]
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.9), order


def test_alfven_2d_oblique_second_order_and_divb():
    errs = []
    for n in (32, 64):
        pr = W.alfven_2d(n)
        e, st = _alfven_err(pr, 1)
        errs.append(e)
        o = O.Oracle(pr)
        bmax = max(np.abs(st["bx"]).max(), np.abs(st["by"]).max())
        assert o.divb(st) <= 1e-13 * bmax
    assert math.log2(errs[0] / errs[1]) > 1.75, errs


# ---------------------------------------------------------------------------
# Contact-CT structure: a grid-aligned 1D problem embedded in 2D reduces to 1D
# (the corner EMF must collapse to the face EMF; a sign slip in the upwind
# derivative terms gives the cell average instead)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("solver", ["lhlld", "hll"])
def test_ct_reduces_to_1d_for_plane_parallel_flow(solver):
    n, ny = 64, 4
    pr = W.brio_wu(n)
    pr2 = pr.copy()
    pr2.n, pr2.ndim, pr2.hi = (n, ny, 1), 2, (1.0, ny / n, 1.0)
    pr2.cons = np.repeat(pr.cons, ny, axis=2)
    pr2.bx = np.repeat(pr.bx, ny, axis=1)
    pr2.by = np.repeat(pr.by[:, :1], ny + 1, axis=1)
    pr2.bz = np.repeat(pr.bz, ny, axis=1)
    s1, _, _ = O.Oracle(pr, riemann=solver).run(20, dt_fixed=4e-4)
    s2, _, _ = O.Oracle(pr2, riemann=solver).run(20, dt_fixed=4e-4)
    for j in range(ny):
        np.testing.assert_allclose(s2["cons"][:, 0, j, :], s1["cons"][:, 0, 0, :], rtol=0, atol=1e-13)
        np.testing.assert_allclose(s2["by"][0, j, :], s1["by"][0, 0, :], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s2["bx"], 0.75, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# axis relabelling invariance (catches transposed operands / strides)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 0, 1)])
def test_brio_wu_along_every_axis(perm):
    n = 128
    s1, _, _ = O.Oracle(W.brio_wu(n)).run(30)
    q = W.permute_axes(W.brio_wu(n), list(perm))
    sq, _, _ = O.Oracle(q).run(30)
    xnew = perm.index(0)
    np.testing.assert_array_equal(sq["cons"][0].ravel(), s1["cons"][0].ravel())
    np.testing.assert_array_equal(sq["cons"][4].ravel(), s1["cons"][4].ravel())
    np.testing.assert_array_equal(sq["cons"][1 + xnew].ravel(), s1["cons"][1].ravel())
    ynew = perm.index(1)
    np.testing.assert_array_equal(sq["cons"][1 + ynew].ravel(), s1["cons"][2].ravel())
    faces = [sq["bx"], sq["by"], sq["bz"]]
    # B_y of the original (cell-like, 2 layers) -> the face array of axis ynew
    np.testing.assert_array_equal(np.sort(faces[ynew].ravel())[::2], np.sort(s1["by"].ravel())[::2])


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 0, 1)])
def test_orszag_tang_in_other_planes(perm):
    """OT in the (x,y) plane vs the same problem in the (z,x) or (y,z) plane."""
    n = 32
    s1, _, _ = O.Oracle(W.orszag_tang(n)).run(15)
    q = W.permute_axes(W.orszag_tang(n), list(perm))
    sq, _, _ = O.Oracle(q).run(15)
    ax_x, ax_y = perm.index(0), perm.index(1)    # new axes holding old x and old y

    def to_old(a):
        # a has array axes (z', y', x'); bring the old-x axis last, old-y before it
        arr_ax = {0: 2, 1: 1, 2: 0}
        return np.transpose(a, (arr_ax[3 - ax_x - ax_y], arr_ax[ax_y], arr_ax[ax_x]))[0]
    np.testing.assert_array_equal(to_old(sq["cons"][0]), s1["cons"][0, 0])
    np.testing.assert_array_equal(to_old(sq["cons"][1 + ax_x]), s1["cons"][1, 0])
    np.testing.assert_array_equal(to_old(sq["cons"][1 + ax_y]), s1["cons"][2, 0])
    np.testing.assert_array_equal(to_old(sq["cons"][4]), s1["cons"][4, 0])


# ---------------------------------------------------------------------------
# Orszag-Tang (C1): conservation, point symmetry, div B
# ---------------------------------------------------------------------------

def test_orszag_tang_conservation_symmetry_divb():
    n = 64
    pr = W.orszag_tang(n)
    o = O.Oracle(pr)
    st, _, _ = o.run(40)
    tot0 = pr.cons.sum(axis=(1, 2, 3))
    tot1 = st["cons"].sum(axis=(1, 2, 3))
    scale = np.abs(pr.cons).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale), (tot1 - tot0) / scale
    rho = st["cons"][0, 0]
    # 180-degree rotation about the box centre maps cell (i, j) -> (n-1-i, n-1-j)
    assert np.abs(rho - rho[::-1, ::-1]).max() < 1e-10 * rho.max()
    bmax = max(np.abs(st["bx"]).max(), np.abs(st["by"]).max())
    assert o.divb(st) <= 1e-13 * bmax
    # the solution has developed shocks: the flattener must have been active
    assert rho.max() / rho.min() > 1.5


# ---------------------------------------------------------------------------
# well-balancing (Sect. 2.8): hydrostatic states stay at rest to round-off,
# and without the deviation method they do not (negative control)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["polytrope", "isothermal"])
def test_well_balanced_rest(kind):
    if kind == "polytrope":
        pr = W.stratified_box(4, 4, 32, amp=0.0, heat=False)
    else:
        pr = W.isothermal_atmosphere(8, 32)
    st, _, _ = O.Oracle(pr).run(200)
    rho = st["cons"][0]
    cs = np.sqrt(pr.gamma * (pr.gamma - 1) * st["cons"][4] / rho)
    u = np.abs(st["cons"][1:4] / rho).max(axis=0)
    assert (u / cs).max() <= 1e-13
    rhohat = pr.bg["rho_c"][3:3 + pr.n[2]][:, None, None]
    assert np.abs((rho - rhohat) / rhohat).max() <= 1e-13
    st2, _, _ = O.Oracle(pr, wb=False).run(50)
    assert np.abs(st2["cons"][1:4] / st2["cons"][0]).max() > 1e-5


def test_reflecting_walls_keep_normal_field_zero():
    """Table bcs: B_n = 0 at a reflecting wall.  The wall faces carry no EMF, so
    the normal field there stays exactly zero while the interior field evolves."""
    pr = W.stratified_box(12, 10, 16, amp=5e-2)
    rng = np.random.default_rng(2)
    pr.cons[1:3] += 1e-3 * rng.standard_normal(pr.cons[1:3].shape)
    pr.bx[:] = 1e-2
    st, _, _ = O.Oracle(pr).run(15)
    assert np.all(st["bz"][0] == 0.0) and np.all(st["bz"][-1] == 0.0)
    assert np.abs(st["bz"][1:-1]).max() > 1e-9


def test_gravity_source_closed_form():
    """Uniform gas in a tall box with reflecting ends and no background: far from
    the walls the only force is rho*g, so m_z = rho*g*t and E gains rho*(g t)^2/2."""
    nz = 48
    pr = W.isothermal_atmosphere(4, nz, g0=0.0)
    pr.g = (0.0, 0.0, -0.5)
    pr.bg = None
    dt, nst = 2e-3, 3
    st, t, _ = O.Oracle(pr).run(nst, dt_fixed=dt)
    rho = pr.cons[0]
    mid = slice(nz // 2 - 8, nz // 2 + 8)
    np.testing.assert_allclose(st["cons"][3][mid], rho[mid] * (-0.5) * t, rtol=1e-12, atol=0)
    np.testing.assert_allclose(st["cons"][4][mid] - pr.cons[4][mid],
                               0.5 * rho[mid] * (0.5 * t) ** 2, rtol=1e-9, atol=0)


def test_heating_source_closed_form():
    """Uniform periodic gas with uniform heating q: E grows by q t exactly."""
    pr = W.orszag_tang(8)
    pr.cons[1:4] = 0.0
    pr.cons[4] = 1.0
    pr.bx[:] = 0.0
    pr.by[:] = 0.0
    q = 0.37
    pr.heat = np.array([q])
    st, t, _ = O.Oracle(pr).run(4, dt_fixed=1e-2)
    np.testing.assert_allclose(st["cons"][4], 1.0 + q * t, rtol=1e-14)
    assert np.abs(st["cons"][1:4]).max() == 0.0


# ---------------------------------------------------------------------------
# Riemann solver special cases (Sect. 2.6)
# ---------------------------------------------------------------------------

def _phys_flux(w, bn):
    rho, un, u1, u2, b1, b2, p, ge, _ = w[:9]
    b2s = bn * bn + b1 * b1 + b2 * b2
    pt = p + 0.5 * b2s
    e = p / (ge - 1) + 0.5 * rho * (un * un + u1 * u1 + u2 * u2) + 0.5 * b2s
    vb = un * bn + u1 * b1 + u2 * b2
    return np.array([rho * un, rho * un * un + pt - bn * bn, rho * un * u1 - bn * b1,
                     rho * un * u2 - bn * b2, (e + pt) * un - bn * vb,
                     un * b1 - u1 * bn, un * b2 - u2 * bn])


def _rand_state(rng, mag=True):
    g = 5.0 / 3.0
    return np.array([rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.normal(),
                     rng.normal() if mag else 0.0, rng.normal() if mag else 0.0,
                     rng.uniform(0.2, 2), g, g])


@pytest.mark.parametrize("solver", ["lhlld", "hlld", "hll"])
def test_equal_states_give_physical_flux(solver):
    rng = np.random.default_rng(7)
    for _ in range(50):
        w = _rand_state(rng)
        bn = rng.normal()
        f = O.riemann(w, w, bn, solver)
        fp = _phys_flux(w, bn)
        np.testing.assert_allclose(f, fp, rtol=1e-12, atol=1e-12 * np.abs(fp).max())


def _toro_hllc(wl, wr, gamma):
    """HLLC (Toro 1994) with the same Davis-type speeds, B = 0."""
    def parts(w):
        rho, u, v, ww, _, _, p = w[:7]
        e = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + ww * ww)
        U = np.array([rho, rho * u, rho * v, rho * ww, e])
        F = np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * ww, (e + p) * u])
        return rho, u, v, ww, p, e, U, F, math.sqrt(gamma * p / rho)
    rl, ul, vl, wl_, pl, el, Ul, Fl, cl = parts(wl)
    rr, ur, vr, wr_, prr, er, Ur, Fr, cr = parts(wr)
    sl = min(ul - cl, ur - cr)
    sr = max(ul + cl, ur + cr)
    ss = (prr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))
    def star(rho, u, v, ww, p, e, s):
        f = rho * (s - u) / (s - ss)
        return f * np.array([1.0, ss, v, ww, e / rho + (ss - u) * (ss + p / (rho * (s - u)))])
    if sl >= 0:
        return Fl
    if sr <= 0:
        return Fr
    if ss >= 0:
        return Fl + sl * (star(rl, ul, vl, wl_, pl, el, sl) - Ul)
    return Fr + sr * (star(rr, ur, vr, wr_, prr, er, sr) - Ur)


def test_hlld_without_field_is_hllc():
    rng = np.random.default_rng(11)
    g = 5.0 / 3.0
    for _ in range(200):
        wl, wr = _rand_state(rng, mag=False), _rand_state(rng, mag=False)
        f = O.riemann(wl, wr, 0.0, "hlld")
        ref = _toro_hllc(wl, wr, g)
        np.testing.assert_allclose(f[:5], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
        assert np.all(f[5:] == 0.0)


def test_lhlld_reduces_to_hlld_when_threshold_is_zero():
    rng = np.random.default_rng(3)
    for _ in range(100):
        wl, wr = _rand_state(rng), _rand_state(rng)
        bn = rng.normal()
        a = O.riemann(wl, wr, bn, "lhlld", mach_thr=0.0)
        b = O.riemann(wl, wr, bn, "hlld")
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mach", [1e-2, 1e-3, 1e-4])
def test_lhlld_scales_pressure_dissipation_by_mach(mach):
    """Eq. pstar with xi: the interface pressure's dissipative part is xi times
    that of HLLD, xi = max(M_L, M_R) below the 0.6 threshold (M = |u| / c_s)."""
    g = 5.0 / 3.0
    wl = np.array([1.0, mach, 0, 0, 0.1, 0.0, 1.0, g, g])
    wr = np.array([1.0, -mach, 0, 0, 0.1, 0.0, 1.0, g, g])
    bn = 0.2
    pt = 1.0 + 0.5 * (bn * bn + 0.01)
    fh = O.riemann(wl, wr, bn, "hlld")
    fl = O.riemann(wl, wr, bn, "lhlld")
    central = pt - bn * bn
    xi = mach / math.sqrt(g)
    np.testing.assert_allclose((fl[1] - central) / (fh[1] - central), xi, rtol=1e-6)
    # above the threshold nothing changes
    wl2, wr2 = wl.copy(), wr.copy()
    wl2[1], wr2[1] = 0.9, -0.9
    np.testing.assert_array_equal(O.riemann(wl2, wr2, bn, "lhlld"), O.riemann(wl2, wr2, bn, "hlld"))


def test_hlld_resolves_stationary_contact():
    g = 5.0 / 3.0
    bn, b1, b2, p = 0.7, 0.3, -0.2, 1.3
    wl = np.array([2.0, 0, 0, 0, b1, b2, p, g, g])
    wr = np.array([0.5, 0, 0, 0, b1, b2, p, g, g])
    for solver in ("hlld", "lhlld"):
        f = O.riemann(wl, wr, bn, solver)
        pt = p + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
        ref = np.array([0.0, pt - bn * bn, -bn * b1, -bn * b2, 0.0, 0.0, 0.0])
        np.testing.assert_allclose(f, ref, rtol=0, atol=1e-14)


def test_riemann_mirror_symmetry():
    """Reflecting the problem (u_n -> -u_n, swap L/R) mirrors the flux."""
    rng = np.random.default_rng(5)
    for solver in ("lhlld", "hlld", "hll"):
        for _ in range(100):
            wl, wr = _rand_state(rng), _rand_state(rng)
            bn = rng.normal()
            f = O.riemann(wl, wr, bn, solver)
            ml, mr = wr.copy(), wl.copy()
            ml[1] *= -1
            mr[1] *= -1
            fm = O.riemann(ml, mr, -bn, solver)
            # mass, transverse momenta, energy are odd; normal momentum even;
            # transverse B flux: u_n B_t - u_t B_n is odd under (u_n, B_n) -> -
            sign = np.array([-1, 1, -1, -1, -1, -1, -1])
            np.testing.assert_allclose(fm, sign * f, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_hlld_flux_is_continuous_across_fan_regions():
    g = 5.0 / 3.0
    wr = np.array([1.0, 0.0, 0.1, 0.0, 0.5, 0.2, 1.0, g, g])
    prev = None
    for ul in np.linspace(-2.5, 2.5, 4001):
        wl = np.array([1.2, ul, -0.1, 0.05, -0.3, 0.4, 0.8, g, g])
        f = O.riemann(wl, wr, 0.6, "hlld")
        if prev is not None:
            assert np.abs(f - prev).max() < 0.02
        prev = f


# ---------------------------------------------------------------------------
# shocks: Brio-Wu (Sect. 3.1)
# ---------------------------------------------------------------------------

def test_brio_wu_positions_match_fine_grid():
    g = _gold("paper_parameters.txt")
    pr = W.brio_wu(int(g["brio_wu_cells"]))
    assert pr.gamma == g["brio_wu_gamma"] and pr.bx[0, 0, 0] == g["brio_wu_bx"]
    assert pr.eps_sf == g["eps_sf"] and pr.mach_thr == g["mach_threshold"]
    assert pr.cfl == g["cfl_mhd_shocks"]
    s5, _, _ = O.Oracle(pr).run_to(g["brio_wu_t"])
    s20, _, _ = O.Oracle(W.brio_wu(2000)).run_to(g["brio_wu_t"])
    r5 = s5["cons"][0, 0, 0]
    r20 = s20["cons"][0, 0, 0].reshape(500, 4).mean(axis=1)
    assert np.abs(r5 - r20).mean() < 4e-3
    assert r5.min() > 0.1 and np.isfinite(s5["cons"]).all()


# ---------------------------------------------------------------------------
# low-Mach behaviour of LHLLD vs HLLD on the advected vortex (Sect. 3.2)
# ---------------------------------------------------------------------------

def test_vortex_dissipation_independent_of_mach_with_lhlld():
    def ekin_frac(solver, ut):
        pr = W.balsara_vortex(32, ut, 0.0)
        st, _, _ = O.Oracle(pr, riemann=solver, eps_sf=0.0).run_to(pr.meta["tau"] / 4)
        def ek(c):
            a = ut / math.sqrt(2)
            return (0.5 * ((c[1] / c[0] - a) ** 2 + (c[2] / c[0] - a) ** 2)).sum()
        return ek(st["cons"]) / ek(pr.cons)
    l1, l2 = ekin_frac("lhlld", 0.1), ekin_frac("lhlld", 0.02)
    h1, h2 = ekin_frac("hlld", 0.1), ekin_frac("hlld", 0.02)
    assert abs(l1 - l2) < 0.01 * l1
    assert h2 < 0.75 * h1
    assert l2 > h2 + 0.2


# ---------------------------------------------------------------------------
# PPH reconstruction (Sect. 2.5, item ii): third order on smooth flows; the
# structural properties of the scheme are unchanged (conservation, div B,
# well-balanced rest)
# ---------------------------------------------------------------------------

def _pph(pr):
    q = pr.copy()
    q.recon = "pph"
    return q


def test_flagged_cells_reconstruct_with_van_leer():
    """Shock flattening (Sect. 2.7): a flagged cell reconstructs with van Leer
    and its faces use HLL, whatever the scheme elsewhere.  With a threshold so
    small that every cell is flagged (the stratified box: pressure varies in
    every cell), PPH and van Leer give the same result bit for bit; with
    flattening off they differ."""
    base = W.stratified_box(6, 5, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    out = {}
    for eps in (1e-13, 0.0):
        for recon in ("vanleer", "pph", "pqh"):
            q = base.copy()
            q.recon, q.eps_sf = recon, eps
            st, _, _ = O.Oracle(q).run(2)
            out[(eps, recon)] = st["cons"]
    for r in ("pph", "pqh"):
        assert np.array_equal(out[(1e-13, "vanleer")], out[(1e-13, r)])
        assert not np.array_equal(out[(0.0, "vanleer")], out[(0.0, r)])


def test_alfven_1d_pph_third_order():
    """The parabola through three cell averages is exact for quadratics, so the
    linear Alfven wave converges at third order (SSP-RK3 in time), against
    second order with the van Leer slope."""
    errs = [_alfven_err(_pph(W.alfven_1d(n)), 2)[0] for n in (32, 64, 128)]
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 2.7), order
    vl = _alfven_err(W.alfven_1d(128), 2)[0]
    assert errs[-1] < 0.2 * vl, (errs[-1], vl)


def test_alfven_2d_pph_order_and_divb():
    """Oblique wave in 2D: the face-centred field is advanced by constrained
    transport, whose edge EMFs average face values (second order), so the
    order stays ~2 with PPH too; the error is smaller than with the van Leer
    slope, and div B stays at round-off."""
    errs = []
    for n in (32, 64):
        pr = _pph(W.alfven_2d(n))
        e, st = _alfven_err(pr, 1)
        errs.append(e)
        bmax = max(np.abs(st["bx"]).max(), np.abs(st["by"]).max())
        assert O.Oracle(pr).divb(st) <= 1e-13 * bmax
    assert math.log2(errs[0] / errs[1]) > 1.9, errs
    vl, _ = _alfven_err(W.alfven_2d(64), 1)
    assert errs[-1] < vl, (errs[-1], vl)


def test_pph_conserves_and_keeps_rest():
    """Orszag-Tang with PPH conserves mass and energy to round-off; a
    well-balanced polytrope with zero deviations stays exactly at rest."""
    pr = _pph(W.orszag_tang(32))
    st, _, _ = O.Oracle(pr).run(20, dt_fixed=2e-3)
    for v in (0, 4):
        t0 = pr.cons[v].sum()
        assert abs(st["cons"][v].sum() - t0) <= 1e-13 * abs(t0), v
    q = _pph(W.stratified_box(4, 4, 32, amp=0.0, heat=False))
    st, _, _ = O.Oracle(q).run(200)
    rho = st["cons"][0]
    cs = np.sqrt(q.gamma * (q.gamma - 1) * st["cons"][4] / rho)
    u = np.abs(st["cons"][1:4] / rho).max(axis=0)
    assert (u / cs).max() <= 1e-13
    rhohat = q.bg["rho_c"][3:3 + q.n[2]][:, None, None]
    assert np.abs((rho - rhohat) / rhohat).max() <= 1e-13


def test_pph_mass_fractions_stay_bounded():
    """Mass fractions take the limited parabola: two species in a step profile
    advected by a uniform flow (periodic, uniform rho and P) stay inside
    [0, 1] and sum to one, while the velocity field is reconstructed by
    unlimited parabolas."""
    n = 64
    x = (np.arange(n) + 0.5) / n
    X0 = np.where((x > 0.3) & (x < 0.6), 1.0, 0.0)[None, None, :]
    z = np.zeros((1, 1, n))
    pr = W._assemble("scalar_step", 1, (n, 1, 1), (0, 0, 0), (1, 1, 1), ((0, 0), (0, 0), (0, 0)), 1.4,
                     np.ones((1, 1, n)), [np.ones((1, 1, n)), z, z], np.ones((1, 1, n)),
                     np.zeros((1, 1, n + 1)), np.zeros((1, 2, n)), np.zeros((2, 1, n)),
                     nspec=2, X=[X0, 1.0 - X0], cfl=0.4)
    pr.meta.update(A=[16.0, 28.0], Z=[8.0, 14.0])
    pr.recon = "pph"
    st, _, _ = O.Oracle(pr).run(40)
    X = st["cons"][5:7] / st["cons"][0]
    assert X.min() >= -1e-13 and X.max() <= 1.0 + 1e-13, (X.min(), X.max())
    assert np.abs(X.sum(axis=0) - 1.0).max() <= 1e-13
    assert np.abs(X[0] - X0).max() > 0.1     # the profile did move



# ---------------------------------------------------------------------------
# Limited fifth-order reconstruction (Sect. 2.5, item iii)
# ---------------------------------------------------------------------------

def _pqh(pr):
    q = pr.copy()
    q.recon = "pqh"
    return q


def _cell_avgs(coef, centres):
    """Exact averages over unit cells of the polynomial sum coef[k] x^k."""
    P = np.polynomial.polynomial.Polynomial(coef).integ()
    return np.array([P(c + 0.5) - P(c - 0.5) for c in centres])


def test_pqh_face_values_exact_for_quartics():
    """The face value of the degree-4 polynomial through five cell averages is
    exact for any quartic; on smooth monotone data the limiter leaves it."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        coef = [rng.uniform(-1, 1), rng.uniform(2, 3), rng.uniform(-0.1, 0.1), rng.uniform(-0.02, 0.02),
                rng.uniform(-0.004, 0.004)]
        w = _cell_avgs(coef, [-2, -1, 0, 1, 2])
        fl, fr = O.recon_cell("pqh", w)
        p = np.polynomial.polynomial.Polynomial(coef)
        assert abs(fr - p(0.5)) <= 1e-13 and abs(fl - p(-0.5)) <= 1e-13, (fl, fr, p(-0.5), p(0.5))


def test_pqh_keeps_smooth_extrema_and_monotone_data():
    """At a smooth extremum (averages of cos) the limited value keeps its
    fifth-order accuracy instead of flattening to the cell value; on monotone
    data (steps, ramps) the face value stays between the two cells sharing
    the face."""
    h = 0.1
    x = np.arange(-2, 3) * h
    w = (np.sin(x + h / 2) - np.sin(x - h / 2)) / h            # averages of cos over the cells
    fl, fr = O.recon_cell("pqh", w)
    assert abs(fr - np.cos(h / 2)) < 1e-7 and abs(fl - np.cos(-h / 2)) < 1e-7
    rng = np.random.default_rng(9)
    for _ in range(200):
        w = np.sort(rng.uniform(-1, 1, 5)) * rng.choice([-1, 1])
        if rng.uniform() < 0.5:
            w = np.where(np.arange(5) < rng.integers(1, 5), w[0], w[-1])   # a step
        fl, fr = O.recon_cell("pqh", w)
        assert min(w[2], w[3]) - 1e-15 <= fr <= max(w[2], w[3]) + 1e-15
        assert min(w[1], w[2]) - 1e-15 <= fl <= max(w[1], w[2]) + 1e-15


def test_alfven_1d_pqh_more_accurate_than_pph():
    """Fifth-order space: the linear Alfven wave's error is an order of
    magnitude below PPH's at the same resolution; overall order three (SSP-RK3
    in time at a fixed CFL number)."""
    errs = [_alfven_err(_pqh(W.alfven_1d(n)), 2)[0] for n in (32, 64, 128)]
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 2.8), (errs, order)
    e_pph = _alfven_err(_pph(W.alfven_1d(64)), 2)[0]
    assert errs[1] < 0.1 * e_pph, (errs[1], e_pph)


def test_brio_wu_pqh_flattening_damps_oscillations():
    """The paper's Brio-Wu test (500 cells, t = 0.08, CFL 0.4): the limited
    fifth-order scheme alone oscillates behind the waves; with shock
    flattening (van Leer + HLL in a 5-cell band around flagged cells) the
    total variation of the density drops towards that of a converged
    solution (van Leer on 2000 cells), and both stay close to it."""
    def rho(recon, eps, n=500):
        q = W.brio_wu(n)
        q.recon, q.eps_sf = recon, eps
        st, t, _ = O.Oracle(q).run_to(0.08)
        return st["cons"][0].ravel()
    ref = rho("vanleer", 0.0, 2000).reshape(500, 4).mean(1)
    tv = lambda r: np.abs(np.diff(r)).sum()
    raw, flat = rho("pqh", 0.0), rho("pqh", 0.2)
    assert tv(raw) - tv(ref) > 1.5 * (tv(flat) - tv(ref)) > 0.0, (tv(raw), tv(flat), tv(ref))
    for r in (raw, flat):
        assert np.abs(r - ref).mean() < 3e-3


# ---------------------------------------------------------------------------
# Contact-CT upwinding of the corner EMF and its deadband (Sect. 2.4)
# ---------------------------------------------------------------------------

def _corner_weights(F, rho=1.0, smax=1.0, seed=0):
    """d E_corner / d E_cell for the four cells (E00, E10, E01, E11), by
    perturbing each cell's reference EMF (the corner EMF is linear in them)."""
    rng = np.random.default_rng(seed)
    Ef = rng.normal(size=4)
    Ec = rng.normal(size=4)
    e0 = O.ct_corner(Ef, Ec, F, rho, smax)
    w = []
    for q in range(4):
        d = Ec.copy()
        d[q] += 1.0
        w.append(O.ct_corner(Ef, d, F, rho, smax) - e0)
    return e0, np.array(w)


def test_ct_corner_rounding_level_mass_flux_has_no_direction():
    """A mass flux at the rounding level of the face's flux scale (here
    |F_rho| = 1e-14 rho max|S|, either sign) carries no direction: the corner
    EMF equals the one with exactly zero mass fluxes, and the four cells enter
    it symmetrically (weight -1/4 each, Gardiner & Stone's zero-flux case)."""
    e_zero, w_zero = _corner_weights(np.zeros(4))
    np.testing.assert_allclose(w_zero, -0.25, rtol=0, atol=1e-15)
    for signs in ((1, 1, 1, 1), (-1, 1, -1, 1), (1, -1, -1, 1), (-1, -1, -1, -1)):
        F = 1e-14 * np.array(signs, dtype=float)
        e, w = _corner_weights(F)
        assert e == e_zero, (signs, e, e_zero)
        np.testing.assert_array_equal(w, w_zero)


@pytest.mark.parametrize("scale", [1e-10, 1e-6, 1.0])
def test_ct_corner_takes_the_upwind_side(scale):
    """Above the deadband each half-cell derivative comes from the upwind
    cell of its face: with every mass flux positive (flow towards +a and +b)
    the corner EMF does not depend on the downwind cell (c_a, c_b) and does
    on the upwind one (c_a - 1, c_b - 1); negative fluxes swap them.  The
    density and signal speed set the band (1e-12 rho max|S|): the same flux
    below it has no direction."""
    for rho, smax in ((1.0, 1.0), (3e7, 2e8)):
        F = scale * rho * smax * np.ones(4)
        _, wp = _corner_weights(F, rho, smax)
        assert wp[3] == 0.0 and wp[0] != 0.0, wp
        _, wm = _corner_weights(-F, rho, smax)
        assert wm[0] == 0.0 and wm[3] != 0.0, wm
        # the mixed cells are upwind of one face each
        assert wp[1] != 0.0 and wp[2] != 0.0 and wm[1] != 0.0 and wm[2] != 0.0
    # just below the band the same configuration is direction-free
    _, w = _corner_weights(1e-13 * np.ones(4))
    np.testing.assert_allclose(w, -0.25, rtol=0, atol=1e-15)
