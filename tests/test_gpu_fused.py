"""The fused mixed-precision stage (one TMA-staged tile kernel for the faces of
all three directions and the cell update) against the per-direction kernels
and against the FP64 CPU oracle.

Both GPU paths evaluate the same method in FP32 on the same deviations; the
default tile shape pairs the left and right states of a face on FP32x2
arithmetic with explicit FMAs, so the two agree to FP32 rounding (relative L1
of the deviations <= 1e-5, the mixed form's bar; the scalar tile shapes to
1e-6), and each is held to the same bar against the oracle.  Grid sizes are
not multiples of the 8^3 tile, so ragged tiles are exercised on every face.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from test_gpu_mixed import deviation_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def run(P, pr, fused, nsteps, dt):
    g = P.Grid(pr, precision="mixed")
    g.set_fused(fused)
    g.load()
    g.step(nsteps, dt)
    out = g.get_state()
    g.close()
    return out


BCS = {
    "periodic_xy": ((0, 0), (0, 0), (1, 1)),
    "outflow_x_reflect_y": ((2, 2), (1, 1), (1, 1)),
    "reflect_x_outflow_y": ((1, 1), (2, 2), (1, 1)),
}


@pytest.mark.parametrize("bc", list(BCS))
def test_fused_matches_per_direction_and_oracle(P, bc):
    pr = W.stratified_box(19, 13, 21, amp=3e-2, beta=1e3, mach_heat=3e-2)
    pr.bc = BCS[bc]
    o = O.Oracle(pr)
    dt = 0.5 * o.dt(dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz))
    nsteps = 6
    fu = run(P, pr, True, nsteps, dt)
    pd = run(P, pr, False, nsteps, dt)
    ref, _, _ = o.run(nsteps, dt_fixed=dt)
    l_fp = deviation_l1(pr, fu, pd)
    l_fo = deviation_l1(pr, fu, ref)
    print(bc, "fused vs per-direction", {k: f"{v:.1e}" for k, v in l_fp.items()})
    print(bc, "fused vs oracle", {k: f"{v:.1e}" for k, v in l_fo.items()})
    for k, v in l_fp.items():
        assert v <= 1e-5, ("fused vs per-direction", k, v)
    for k in ("rho", "mx", "my", "mz", "E", "bx"):
        assert l_fo[k] <= 1e-5, ("fused vs oracle", k, l_fo[k])


@pytest.mark.parametrize("shape", [2, 3, 4, 5, 6, 7, 8, 9])
def test_fused_launch_shapes_agree(P, shape):
    """Every launch shape of the tile kernel (phased faces, other CTA sizes,
    two faces per thread on FP32x2 arithmetic) gives the per-direction result
    to FP32 rounding: shapes 2-4 run the same scalar face code (agreement to
    1e-6 relative L1 of the deviations), shapes 5-7 the paired solver, whose
    explicit FMAs round differently (held to the mixed form's bar, 1e-5)."""
    pr = W.stratified_box(19, 13, 21, amp=3e-2, beta=1e3, mach_heat=3e-2)
    pr.bc = BCS["outflow_x_reflect_y"]
    dt = 0.5 * O.Oracle(pr).dt(dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz))
    a = run(P, pr, shape, 4, dt)
    b = run(P, pr, 0, 4, dt)
    tol = 1e-6 if shape <= 4 else 1e-5   # paired shapes round their explicit FMAs differently
    for k, v in deviation_l1(pr, a, b).items():
        assert v <= tol, (shape, k, v)


def blast(nx, ny, nz, seed=5):
    """Periodic box, uniform oblique field, random velocities and a pressure
    jump of 10 in a ball: shock-flagged (HLL) faces next to LHLLD faces."""
    pr = W.stratified_box(nx, ny, nz, amp=0.0, heat=False)
    pr.bc = ((0, 0), (0, 0), (0, 0))
    pr.g = (0.0, 0.0, 0.0)
    pr.bg, pr.heat = None, None
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny,
                          (np.arange(nx) + 0.5) / nx, indexing="ij")
    r2 = (x - 0.4) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2
    p = np.where(r2 < 0.2 ** 2, 10.0, 1.0)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, size=(nz, ny, nx))
    v = 0.2 * rng.standard_normal((3, nz, ny, nx))
    b = (0.3, 0.2, 0.1)
    pr.bx[:], pr.by[:], pr.bz[:] = b
    pr.cons[0] = rho
    pr.cons[1:4] = rho * v
    pr.cons[4] = p / (pr.gamma - 1.0) + 0.5 * rho * (v ** 2).sum(axis=0) + 0.5 * sum(c * c for c in b)
    return pr


def test_fused_blast_with_flags(P):
    pr = blast(21, 18, 11)
    dt = 2e-3
    fu = run(P, pr, True, 5, dt)
    pd = run(P, pr, False, 5, dt)
    ref, _, _ = O.Oracle(pr).run(5, dt_fixed=dt)
    for key in ("cons", "bx", "by", "bz"):
        a, b, c = fu[key], pd[key], ref[key]
        scale = np.abs(c).max()
        assert np.abs(a - b).max() <= 1e-5 * scale, key
    # against the oracle: the mixed form's measure, relative L1 per field (no
    # background here, so the deviation is the field; m and B as vectors)
    rel = lambda x, y: np.abs(x - y).sum() / np.abs(y).sum()
    l1 = {"rho": rel(fu["cons"][0], ref["cons"][0]), "m": rel(fu["cons"][1:4], ref["cons"][1:4]),
          "E": rel(fu["cons"][4], ref["cons"][4]),
          "B": (sum(np.abs(fu[k] - ref[k]).sum() for k in ("bx", "by", "bz")) /
                sum(np.abs(ref[k]).sum() for k in ("bx", "by", "bz")))}
    print("blast, fused vs oracle:", {k: f"{v:.2e}" for k, v in l1.items()})
    for k, v in l1.items():
        assert v <= 1e-5, (k, v)
    # total mass and energy: exactly conserved up to FP64 accumulation of FP32 increments
    for v_ in (0, 4):
        t0 = pr.cons[v_].sum()
        assert abs(fu["cons"][v_].sum() - t0) <= 1e-9 * abs(t0), v_


def test_fused_flag_vote_is_taken_every_stage(P):
    """The raw-flag kernel votes whether any cell is flagged; with no vote the
    dilation is skipped (its buffer keeps an older stage's flags) and the tile
    kernel stages zero flags.  One grid switched between a flagged state (the
    blast) and a flag-free one (the same box at uniform pressure) must give,
    after each switch, exactly what a fresh grid gives: no stale flag or vote
    leaks from one state into the other."""
    pr = blast(21, 18, 11)
    calm = pr.copy()   # uniform pressure 1: the internal energy of every cell replaced
    b = (0.3, 0.2, 0.1)
    rho, m = pr.cons[0], pr.cons[1:4]
    calm.cons[4] = 1.0 / (pr.gamma - 1.0) + 0.5 * (m ** 2).sum(axis=0) / rho + 0.5 * sum(c * c for c in b)

    def fresh(state_pr, nsteps):
        return run(P, state_pr, True, nsteps, 2e-3)

    ref_calm, ref_blast = fresh(calm, 2), fresh(pr, 2)
    g = P.Grid(pr, precision="mixed")
    g.set_fused(True)
    for src, ref in ((pr, ref_blast), (calm, ref_calm), (pr, ref_blast), (calm, ref_calm)):
        g.set_state(src.cons, src.bx, src.by, src.bz)
        g.step(2, 2e-3)
        got = g.get_state()
        for k in ("cons", "bx", "by", "bz"):
            assert np.array_equal(got[k], ref[k]), k
    g.close()
    # the two states really differ in their flags: the calm run is not the blast run
    assert not np.array_equal(ref_calm["cons"], ref_blast["cons"])


def test_fused_divergence_free(P):
    """Contact-CT on the fused path keeps div B at round-off (Eq. divb).  The
    mixed form adds FP32 face increments (each a discrete curl rounded once in
    FP32) to the FP64 field, so div B is bounded by FP32 rounding of the field's
    change, not of the field itself."""
    pr = blast(16, 12, 20, seed=8)
    st = run(P, pr, True, 8, 2e-3)
    n = pr.n
    dx = [1.0 / n[0], 1.0 / n[1], 1.0 / n[2]]

    def div(s):
        return ((s["bx"][:, :, 1:] - s["bx"][:, :, :-1]) / dx[0] + (s["by"][:, 1:, :] - s["by"][:, :-1, :]) / dx[1]
                + (s["bz"][1:] - s["bz"][:-1]) / dx[2])

    db = max(np.abs(st[k] - getattr(pr, k)).max() for k in ("bx", "by", "bz"))
    assert db > 0
    assert np.abs(div(st)).max() * min(dx) <= 1e-6 * db
    # the initial field is uniform: div B = 0 exactly at the start
    assert np.abs(div(dict(bx=pr.bx, by=pr.by, bz=pr.bz))).max() == 0.0


def test_fused_only_where_eligible(P):
    g = P.Grid(W.orszag_tang(32), precision="mixed")
    with pytest.raises(P.PhlError):
        g.set_fused(True)
    g.set_fused(False)
    g.close()


def _box_bc(bc, n=(21, 18, 27)):
    pr = W.stratified_box(*n, amp=3e-2, beta=1e3, mach_heat=3e-2)
    pr.bc = BCS[bc]
    return pr


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("shape", [1, 2])
def test_three_launch_stage_matches_six_launch_stage(P, bc, shape):
    """The stage in three launches (tile kernel with the flag dilation inside;
    Contact-CT with the face update; next primitives with their ghost images
    and the raw flags) against the same tile kernel in six launches, with the
    device CFL step (folded into the last stage on the three-launch path) and
    shock flags active, on ragged boxes with every boundary kind: the same
    arithmetic in other kernels, equal to FP32 rounding of the deviations."""
    pr = _box_bc(bc)
    pr.eps_sf = 0.02   # a low threshold: many flagged cells and HLL faces
    outs = []
    for on in (200 + shape, shape):
        g = P.Grid(pr, precision="mixed")
        g.set_fused(on)
        g.load()
        g.step(6)   # device CFL step each step
        outs.append(g.get_state())
        g.close()
    same = all(np.array_equal(outs[0][k], outs[1][k]) for k in ("cons", "bx", "by", "bz"))
    l1 = deviation_l1(pr, outs[0], outs[1])
    print(bc, shape, "bit-identical" if same else {k: f"{v:.1e}" for k, v in l1.items()})
    for k, v in l1.items():
        assert v <= 1e-6, (k, v)


def test_three_launch_stage_resumes_after_set_state(P):
    """The state set from outside between steps (as a restart does) is picked
    up: the next step forms the primitives, flags and CFL step again, and the
    run equals one that never stopped."""
    pr = _box_bc("periodic_xy", (16, 24, 20))
    g = P.Grid(pr, precision="mixed")
    g.set_fused(201)
    g.load()
    g.step(3)
    mid = g.get_state()
    g.step(3)
    ref = g.get_state()
    g.close()
    h = P.Grid(pr, precision="mixed")
    h.set_fused(201)
    h.load()
    h.step(1)                      # leaves W of a state about to be replaced
    h.set_state(mid["cons"], mid["bx"], mid["by"], mid["bz"])
    h.step(3)
    got = h.get_state()
    h.close()
    for k in ("cons", "bx", "by", "bz"):
        assert np.array_equal(got[k], ref[k]), k
