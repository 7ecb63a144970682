"""Thermal diffusion by RKL2 super-time-stepping (Sect. 2.10) on the GPU
against the CPU oracle: relative L-infinity of the total energy <= 1e-11
after super steps of many stages, the same stage count, untouched density and
momentum, and energy conservation; on FP64 and mixed-precision grids (the
diffusion works on the FP64 state of either)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_oracle_diffusion import pulse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def both(P, pr, steps, dt, precision="fp64", **kw):
    g = P.Grid(pr, precision=precision)
    g.load()
    ns_gpu = [g.diffuse(dt, **kw) for _ in range(steps)]
    g.check()
    st = g.get_state()
    g.close()
    o = O.Oracle(pr)
    ref = dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
    ns_ora = []
    for _ in range(steps):
        ref, ns = o.diffuse(dt, state=ref, **kw)
        ns_ora.append(ns)
    return st, ref, ns_gpu, ns_ora


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pulse_matches_oracle(P, precision):
    pr, _, _ = pulse(48)
    st, ref, ng, no = both(P, pr, 3, 0.2, precision, k0=1e-2, cv=1.5)   # 7 stages per step
    assert ng == no and min(ng) > 3
    e = np.abs(st["cons"][4] - ref["cons"][4]).max() / np.abs(ref["cons"][4]).max()
    assert e <= 1e-11, e
    assert np.array_equal(st["cons"][:4], pr.cons[:4])
    assert abs(st["cons"][4].sum() - pr.cons[4].sum()) <= 1e-13 * abs(pr.cons[4].sum())


def test_radiative_conductivity_in_a_stratified_box(P):
    """K = k0 T^3 / rho on the stratified box (noise, field, walls in z):
    nonlinear diffusion across a background temperature gradient."""
    pr = W.stratified_box(20, 17, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    cv = 1.0 / (pr.gamma - 1.0)
    st, ref, ng, no = both(P, pr, 2, 1e-3, k0=2e-3, nT=3, nR=1, cv=cv)
    assert ng == no and min(ng) >= 3
    e = np.abs(st["cons"][4] - ref["cons"][4]).max() / np.abs(ref["cons"][4]).max()
    assert e <= 1e-11, e
    # the change itself is resolved (not round-off): compare it too
    dE, dR = st["cons"][4] - pr.cons[4], ref["cons"][4] - pr.cons[4]
    assert np.abs(dR).max() > 1e-6 * np.abs(pr.cons[4]).max()
    assert np.abs(dE - dR).max() <= 1e-9 * np.abs(dR).max()


def test_stage_limit_is_enforced(P):
    pr, _, _ = pulse(32)
    g = P.Grid(pr)
    g.load()
    with pytest.raises(P.PhlError):
        g.diffuse(10.0, 1.0, cv=1.5, max_stages=50)
    g.close()
