"""Thermal diffusion by RKL2 super-time-stepping (Sect. 2.10) on the GPU
against the CPU oracle.

FP64 form (on FP64 grids, and on mixed grids when asked for): relative
L-infinity of the total energy <= 1e-11 after super steps of many stages.
Mixed form (float stages on the change of e_int): the change of the total
energy agrees to 1e-5 in relative L1 (and 1e-4 of its largest value cell by
cell).  Both: the same stage count, untouched density and momentum, energy
conserved, insulating cells block the flux; and at the benchmark's size
(256^3 stratified box, radiative conductivity, CFL_p = 100) the mixed form
against the oracle over the whole box.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_oracle_diffusion import pulse

pytestmark = pytest.mark.gpu

MIXED_L1 = 1e-5
MIXED_MAX = 1e-4


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def run_gpu(P, pr, steps, dt, grid="fp64", dprec="grid", **kw):
    g = P.Grid(pr, precision=grid)
    g.load()
    ns = [g.diffuse(dt, precision=dprec, **kw) for _ in range(steps)]
    g.check()
    st = g.get_state()
    g.close()
    return st, ns


def run_oracle(pr, steps, dt, **kw):
    o = O.Oracle(pr)
    ref = dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
    ns = []
    for _ in range(steps):
        ref, n = o.diffuse(dt, state=ref, **kw)
        ns.append(n)
    return ref, ns


def check_fp64(pr, st, ref):
    e = np.abs(st["cons"][4] - ref["cons"][4]).max() / np.abs(ref["cons"][4]).max()
    assert e <= 1e-11, e
    assert np.array_equal(st["cons"][:4], pr.cons[:4])


def check_mixed(pr, st, ref):
    dE, dR = st["cons"][4] - pr.cons[4], ref["cons"][4] - pr.cons[4]
    l1 = np.abs(dE - dR).sum() / np.abs(dR).sum()
    mx = np.abs(dE - dR).max() / np.abs(dR).max()
    assert l1 <= MIXED_L1 and mx <= MIXED_MAX, (l1, mx)
    assert np.array_equal(st["cons"][:4], pr.cons[:4])
    return l1, mx


FORMS = [("fp64", "grid", "fp64"), ("mixed", "fp64", "fp64"), ("mixed", "grid", "mixed"), ("fp64", "mixed", "mixed")]


@pytest.mark.parametrize("grid,dprec,form", FORMS)
def test_pulse_matches_oracle(P, grid, dprec, form):
    pr, _, _ = pulse(48)
    kw = dict(k0=1e-2, cv=1.5)
    st, ng = run_gpu(P, pr, 3, 0.2, grid, dprec, **kw)    # 7 stages per step
    ref, no = run_oracle(pr, 3, 0.2, **kw)
    assert ng == no and min(ng) > 3
    if form == "fp64":
        check_fp64(pr, st, ref)
        tol = 1e-13
    else:
        check_mixed(pr, st, ref)
        tol = 1e-6 * np.abs(st["cons"][4] - pr.cons[4]).sum() / abs(pr.cons[4].sum())
    assert abs(st["cons"][4].sum() - pr.cons[4].sum()) <= tol * abs(pr.cons[4].sum())


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_radiative_conductivity_in_a_stratified_box(P, form):
    """K = k0 T^3 / rho on the stratified box (noise, field, walls in z, a
    ragged 20 x 17 x 24 grid): nonlinear diffusion across a background
    temperature gradient."""
    pr = W.stratified_box(20, 17, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    kw = dict(k0=2e-3, nT=3, nR=1, cv=1.0 / (pr.gamma - 1.0))
    st, ng = run_gpu(P, pr, 2, 1e-3, form, "grid", **kw)
    ref, no = run_oracle(pr, 2, 1e-3, **kw)
    assert ng == no and min(ng) >= 3
    dE, dR = st["cons"][4] - pr.cons[4], ref["cons"][4] - pr.cons[4]
    assert np.abs(dR).max() > 1e-6 * np.abs(pr.cons[4]).max()   # the change is resolved
    if form == "fp64":
        check_fp64(pr, st, ref)
        assert np.abs(dE - dR).max() <= 1e-9 * np.abs(dR).max()
    else:
        check_mixed(pr, st, ref)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_insulating_cells_block_the_flux(P, form):
    """Harmonic-mean face conductivity: two columns of cells with vanishing
    K split a periodic box into compartments that keep their energies."""
    n, cv, k0 = 32, 1.5, 1e-2
    pr, xx, yy = pulse(n, k0, cv)
    ix = np.arange(n)
    inner = (ix > 8) & (ix < 24)
    T = np.where(inner[None, :], 2.0 + 0.5 * np.exp(-(xx ** 2 + yy ** 2) / 0.01), 1.0)
    rho = np.ones((n, n))
    rho[:, [8, 24]] = 1e9
    pr.cons[0][0] = rho
    pr.cons[4][0] = rho * cv * T
    st, ng = run_gpu(P, pr, 1, 0.2, form, "grid", k0=k0, nR=2, cv=cv)
    ref, no = run_oracle(pr, 1, 0.2, k0=k0, nR=2, cv=cv)
    assert ng == no
    E0, E1 = pr.cons[4][0], st["cons"][4][0]
    for part in (inner, ~inner & (ix != 8) & (ix != 24)):
        a, b = E0[:, part].sum(), E1[:, part].sum()
        moved = np.abs(E1[:, part] - E0[:, part]).sum()
        tol = 1e-12 * abs(a) if form == "fp64" else 1e-6 * moved
        assert abs(b - a) <= tol, (form, a, b, moved)
    assert np.abs(E1[:, inner] - E0[:, inner]).max() > 1e-2
    if form == "fp64":
        check_fp64(pr, st, ref)
    else:
        check_mixed(pr, st, ref)


def test_stage_limit_is_enforced(P):
    pr, _, _ = pulse(32)
    for grid in ("fp64", "mixed"):
        g = P.Grid(pr, precision=grid)
        g.load()
        with pytest.raises(P.PhlError):
            g.diffuse(10.0, 1.0, cv=1.5, max_stages=50)
        g.close()


def test_full_size_mixed_against_oracle(P):
    """The benchmark's super step: 256^3 stratified box, K = k0 T^3 / rho
    with k0 set so that the box's MHD step is 100 parabolic limits, dt = the
    MHD step; the mixed form on the mixed grid against the oracle over the
    whole box (one super step, the same stage count)."""
    n = 256
    pr = W.stratified_box(n, n, n)
    cv = 1.0 / (pr.gamma - 1.0)
    g = P.Grid(pr, precision="mixed")
    g.load()
    dt = g.compute_dt()
    rho = pr.cons[0]
    T = (pr.cons[4] - 0.5 * (pr.cons[1] ** 2 + pr.cons[2] ** 2 + pr.cons[3] ** 2) / rho) / rho / cv
    rate1 = (T ** 3 / rho / (rho * cv)).max() * 3 * n * n
    k0 = 100.0 / (2.0 * rate1 * dt)
    ns = g.diffuse(dt, k0, nT=3, nR=1, cv=cv)
    g.check()
    st = g.get_state()
    g.close()
    ref, no = run_oracle(pr, 1, dt, k0=k0, nT=3, nR=1, cv=cv, max_stages=1000)
    assert [ns] == no and ns >= 15
    check_mixed(pr, st, ref)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_delta_T_option_matches_oracle(P, form):
    """Sect. 2.10's option: diffusing only the deviation from the background
    temperature (radiative K of the full temperature) on the stratified box;
    a grid without a background rejects it."""
    pr = W.stratified_box(20, 17, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    kw = dict(k0=2e-3, nT=3, nR=1, cv=1.0 / (pr.gamma - 1.0), delta_T=True)
    st, ng = run_gpu(P, pr, 2, 1e-3, form, "grid", **kw)
    ref, no = run_oracle(pr, 2, 1e-3, **kw)
    assert ng == no
    dE, dR = st["cons"][4] - pr.cons[4], ref["cons"][4] - pr.cons[4]
    assert np.abs(dR).max() > 1e-7 * np.abs(pr.cons[4]).max()
    if form == "fp64":
        check_fp64(pr, st, ref)
        assert np.abs(dE - dR).max() <= 1e-9 * np.abs(dR).max()
    else:
        check_mixed(pr, st, ref)
    q, _, _ = pulse(16)
    g = P.Grid(q)
    g.load()
    with pytest.raises(P.PhlError):
        g.diffuse(0.1, 1e-2, cv=1.5, delta_T=True)
    g.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", [0, 1])
def test_one_dimensional_row(P, form, bc):
    """Edge case: a 1-D row (ny = nz = 1; the mixed stage kernel's 32 x 8 tile
    keeps one active row), periodic or walled, against the oracle."""
    n, cv, k0 = 77, 1.5, 1e-2
    x = (np.arange(n) + 0.5) / n - 0.5
    T = 1.0 + 0.5 * np.exp(-x ** 2 / 0.01)
    z = np.zeros((1, 1, n))
    pr = W._assemble("row", 1, (n, 1, 1), (-0.5, 0.0, 0.0), (0.5, 1.0, 1.0), ((bc, bc), (0, 0), (0, 0)),
                     1.0 + 1.0 / cv, np.ones((1, 1, n)), [z, z, z], T[None, None, :],
                     np.zeros((1, 1, n + 1)), np.zeros((1, 2, n)), np.zeros((2, 1, n)),
                     eint_density=cv * T[None, None, :])
    st, ng = run_gpu(P, pr, 2, 0.1, form, "grid", k0=k0, cv=cv)     # 6 stages per step
    ref, no = run_oracle(pr, 2, 0.1, k0=k0, cv=cv)
    assert ng == no and min(ng) > 3
    if form == "fp64":
        check_fp64(pr, st, ref)
    else:
        check_mixed(pr, st, ref)
