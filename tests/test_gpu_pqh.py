"""Limited fifth-order (PQH) reconstruction (Sect. 2.5, item iii) on the GPU
against the oracle: the face value of the degree-4 polynomial through five
cell averages with the Suresh-Huynh monotonicity-preserving bounds, for every
variable; three ghost layers; van Leer in cells flagged by the shock
flattener.

FP64 form: relative L-infinity per field <= 1e-11 (the induced transverse
field against the field scale); mixed form (per-direction kernels; the fused
tile kernel stages two ghost layers and declines PQH): relative L1 of the
deviations <= 1e-5.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_gpu_parity import compare, run_both
from test_gpu_mixed import deviation_l1
from test_gpu_pph import _scalar_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def pqh(pr):
    q = pr.copy()
    q.recon = "pqh"
    return q


def compare_field_scale(st, ref, tol=1e-11):
    """Vector components that start at zero and are only driven (momentum
    from rest, the induced transverse field) against their vector's scale,
    the other fields against their own."""
    errs = {f"cons{v}": np.abs(st["cons"][v] - ref["cons"][v]).max() / np.abs(ref["cons"][v]).max()
            for v in (0, 4)}
    ms = np.abs(ref["cons"][1:4]).max()
    errs.update({f"cons{v}": np.abs(st["cons"][v] - ref["cons"][v]).max() / ms for v in (1, 2, 3)})
    bs = max(np.abs(ref[k]).max() for k in ("bx", "by", "bz"))
    errs.update({k: np.abs(st[k] - ref[k]).max() / bs for k in ("bx", "by", "bz")})
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, bad


def test_pqh_orszag_tang_fp64(P):
    st, ref = run_both(P, pqh(W.orszag_tang(64)), 60)
    compare(st, ref)


def test_pqh_brio_wu_fp64(P):
    """The paper's shock tube, 400 cells, 120 steps, with and without shock
    flattening."""
    for eps in (0.2, 0.0):
        pr = pqh(W.brio_wu(400))
        pr.eps_sf = eps
        st, ref = run_both(P, pr, 120)
        compare(st, ref)


def test_pqh_stratified_box_fp64(P):
    pr = pqh(W.stratified_box(20, 17, 24, amp=3e-2, beta=1e3, mach_heat=3e-2))
    dt = 0.5 * O.Oracle(pr).dt(dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz))
    st, ref = run_both(P, pr, 5, dt=dt)
    compare_field_scale(st, ref)


def test_pqh_mass_fractions_fp64(P):
    pr = _scalar_step()
    pr.recon = "pqh"
    st, ref = run_both(P, pr, 40)
    compare(st, ref)
    X = st["cons"][5:7] / st["cons"][0]
    assert X.min() >= -1e-13 and X.max() <= 1.0 + 1e-13


def test_pqh_mixed_stratified_box(P):
    pr = pqh(W.stratified_box(19, 13, 21, amp=3e-2, beta=1e3, mach_heat=3e-2))
    o = O.Oracle(pr)
    dt = 0.5 * o.dt(dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz))
    g = P.Grid(pr, precision="mixed")
    with pytest.raises(P.PhlError):
        g.set_fused(1)
    g.load()
    g.step(6, dt)
    st = g.get_state()
    g.close()
    ref, _, _ = o.run(6, dt_fixed=dt)
    l1 = deviation_l1(pr, st, ref)
    for k in ("rho", "mx", "my", "mz", "E", "bx"):
        assert l1[k] <= 1e-5, (k, l1[k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pqh_flagged_cells_reconstruct_with_van_leer(P, precision):
    base = W.stratified_box(16, 12, 24, amp=3e-2, beta=1e3, mach_heat=3e-2)
    out = {}
    for recon in ("vanleer", "pqh"):
        q = base.copy()
        q.recon, q.eps_sf = recon, 1e-13
        g = P.Grid(q, precision=precision)
        if precision == "mixed":
            g.set_fused(0)
        g.load()
        g.step(2, g.compute_dt())
        g.check()
        out[recon] = g.get_state()["cons"]
        g.close()
    assert np.array_equal(out["vanleer"], out["pqh"])
