"""Pins of the oracle's thermal diffusion by RKL2 super-time-stepping
(Sect. 2.10): the RKL2 step is second order and stable over the interval its
stage count is designed for (and not beyond), the stage count follows the
paper's formula, a Gaussian pulse under constant conductivity converges to
the closed-form heat-equation solution at second order, and the operator
conserves the total energy with periodic sides and with walls.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("s", [3, 4, 8, 22, 65])
def test_rkl2_second_order_and_stable(s):
    L = O.lib()
    zmax = -(s * s + s - 2) / 2.0
    zs = np.linspace(zmax, 0.0, 4001)
    amp = np.array([L.ora_rkl2_amp(s, z) for z in zs])
    assert np.abs(amp).max() <= 1.0 + 1e-12
    assert abs(L.ora_rkl2_amp(s, 1.25 * zmax)) > 1.0          # the interval is (close to) the limit
    for z in (-1e-2, -1e-3):                                   # R(z) = 1 + z + z^2/2 + O(z^3)
        r = L.ora_rkl2_amp(s, z)
        assert abs((r - 1.0 - z) / z ** 2 - 0.5) < 0.2 * abs(z) + 1e-9, (s, z, r)


def test_stage_count_formula():
    L = O.lib()
    for ratio, n in ((0.1, 3), (1.0, 3), (2.5, 4), (10.0, 7), (13.5, 8), (100.0, 20), (1000.0, 63)):
        assert L.ora_sts_stages(ratio, 1.0) == n, ratio
        assert n == max(1 + math.floor(0.5 * (math.sqrt(9.0 + 16.0 * ratio) - 1.0)), 3)


def pulse(n, k0=1e-2, cv=1.5, T0=1.0, A=0.5, sigma=0.1, bc=0):
    """2D Gaussian temperature pulse at rest, rho = 1, no field (ideal gas,
    E = rho c_v T), on [-1/2, 1/2]^2."""
    x = (np.arange(n) + 0.5) / n - 0.5
    yy, xx = np.meshgrid(x, x, indexing="ij")
    T = T0 + A * np.exp(-(xx ** 2 + yy ** 2) / sigma ** 2)
    z = np.zeros((1, n, n))
    pr = W._assemble("pulse", 2, (n, n, 1), (-0.5, -0.5, 0.0), (0.5, 0.5, 1.0), ((bc, bc), (bc, bc), (0, 0)),
                     1.0 + 1.0 / cv, np.ones((1, n, n)), [z, z, z], T[None],
                     np.zeros((1, n, n + 1)), np.zeros((1, n + 1, n)), np.zeros((2, n, n)),
                     eint_density=cv * T[None])
    return pr, xx, yy


def test_pulse_converges_to_heat_equation():
    """Constant K: T obeys the heat equation with D = K / (rho c_v); the
    Gaussian keeps its shape, T - T0 = A s^2/(s^2 + 4Dt) exp(-r^2/(s^2 + 4Dt)).
    Steps of CFL_p = 10 (dt ~ dx^2, so the second-order time error stays below
    the spatial one); the L1 error falls at second order."""
    k0, cv, T0, A, sig = 1e-2, 1.5, 1.0, 0.5, 0.1
    D = k0 / cv
    t_end = sig ** 2 / (4 * D)            # the pulse's variance doubles
    errs = []
    for n in (32, 64, 128):
        pr, xx, yy = pulse(n, k0, cv, T0, A, sig)
        dtp = 0.5 / (2 * D * n * n)       # dt_p = 1/2 [sum_s D / dx^2]^-1
        nsteps = max(1, int(round(t_end / (10 * dtp))))
        dt = t_end / nsteps
        o = O.Oracle(pr)
        st = dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
        for _ in range(nsteps):
            st, ns = o.diffuse(dt, k0, cv=cv, state=st)
        T = st["cons"][4][0] / cv
        s2 = sig ** 2 + 4 * D * t_end
        exact = T0 + A * sig ** 2 / s2 * np.exp(-(xx ** 2 + yy ** 2) / s2)
        errs.append(np.abs(T - exact).mean())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.8), (errs, order)


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("nT,nR", [(0, 0), (3, 1)])
def test_diffusion_conserves_energy(bc, nT, nR):
    """Periodic sides, reflecting walls and outflow sides carry no net flux:
    the total energy is conserved to round-off, for constant and for
    radiative (T^3 / rho) conductivity, over a step of many stages."""
    rng = np.random.default_rng(3)
    pr, _, _ = pulse(24, bc=bc)
    pr.cons[0] *= 1.0 + 0.2 * rng.uniform(-1, 1, pr.cons[0].shape)
    E0 = pr.cons[4].sum()
    st, ns = O.Oracle(pr).diffuse(5e-3, 1e-2, nT=nT, nR=nR, cv=1.5)
    assert ns >= 3
    assert abs(st["cons"][4].sum() - E0) <= 1e-13 * abs(E0)
    assert np.array_equal(st["cons"][:4], pr.cons[:4])     # rho and momentum untouched


def test_insulating_cells_block_the_flux():
    """The face conductivity is the harmonic mean of the two cells' (Sect.
    2.10), which is the series conductance of two half cells: a face next to
    a cell of vanishing conductivity carries (almost) no heat.  Two columns of
    such cells (K = k0 / rho^2 with rho = 1e9) split a periodic box into two
    compartments at different temperatures; each compartment keeps its own
    energy while heat still spreads inside it.  (An arithmetic face mean
    would leak half the neighbour's conductance through those faces.)"""
    n, cv, k0 = 32, 1.5, 1e-2
    pr, xx, yy = pulse(n, k0, cv)
    ix = np.arange(n)
    inner = (ix > 8) & (ix < 24)
    T = np.where(inner[None, :], 2.0 + 0.5 * np.exp(-(xx ** 2 + yy ** 2) / 0.01), 1.0)
    rho = np.ones((n, n))
    rho[:, [8, 24]] = 1e9
    pr.cons[0][0] = rho
    pr.cons[4][0] = rho * cv * T
    st, ns = O.Oracle(pr).diffuse(0.2, k0, nT=0, nR=2, cv=cv)
    assert ns >= 4
    E0, E1 = pr.cons[4][0], st["cons"][4][0]
    for part in (inner, ~inner & (ix != 8) & (ix != 24)):
        a, b = E0[:, part].sum(), E1[:, part].sum()
        assert abs(b - a) <= 1e-12 * abs(a), (a, b)
    assert np.abs(E1[:, inner] - E0[:, inner]).max() > 1e-2     # heat does spread inside


def test_delta_T_option_leaves_the_background_alone():
    """Sect. 2.10's option: diffusing T - T_hat (the deviation from the
    hydrostatic background) leaves the background at rest untouched, whereas
    the full operator conducts heat down the background's temperature
    gradient; with a constant conductivity the option is the full operator
    minus its action on the background (linearity)."""
    rest = W.stratified_box(6, 5, 24, amp=0.0, heat=False)
    cv = 1.0 / (rest.gamma - 1.0)
    kw = dict(k0=3e-3, nT=0, nR=0, cv=cv)
    o = O.Oracle(rest)
    st_d, ns_d = o.diffuse(5e-3, delta_T=True, **kw)
    st_f, ns_f = o.diffuse(5e-3, **kw)
    assert ns_d == ns_f >= 3
    # at rest e_int = (E - B^2/2)/rho equals the background's P/((gamma-1) rho) up to rounding
    assert np.array_equal(st_d["cons"][:4], rest.cons[:4])
    assert np.abs(st_d["cons"][4] - rest.cons[4]).max() <= 1e-13 * np.abs(rest.cons[4]).max()
    assert np.abs(st_f["cons"][4] - rest.cons[4]).max() > 1e-6 * np.abs(rest.cons[4]).max()
    pert = rest.copy()                                  # a temperature perturbation, the same rho
    pert.cons = rest.cons.copy()
    rng = np.random.default_rng(4)
    pert.cons[4] = rest.cons[4] * (1.0 + 3e-2 * rng.uniform(-1, 1, rest.cons[4].shape))
    op = O.Oracle(pert)
    d_opt = op.diffuse(5e-3, delta_T=True, **kw)[0]["cons"][4] - pert.cons[4]
    d_full = op.diffuse(5e-3, **kw)[0]["cons"][4] - pert.cons[4]
    d_bg = st_f["cons"][4] - rest.cons[4]
    assert np.abs(d_opt - (d_full - d_bg)).max() <= 1e-9 * np.abs(d_full).max()
