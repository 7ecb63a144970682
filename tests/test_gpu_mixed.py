"""Mixed-precision stage (FP32 deviations, FP64 background and accumulation)
against the FP64 CPU oracle.

Accuracy measure (stated per field): relative L1 error of the deviation from
the hydrostatic background,
    || dq_mixed - dq_oracle ||_1 / || dq_oracle ||_1,   dq = q - q_hat,
with q_hat = rho_hat, E_hat = P_hat / (gamma - 1) for density and energy, and
zero for momentum and the magnetic field.  The fields are rho, m, E and B;
momentum and B are vector fields, each one field whose norm sums its three
components (a component born from zero, such as B_y under a uniform B_x, is
held to the bar relative to its vector).  The per-component values are
printed beside the per-field ones.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def deviation_l1(pr, st, ref):
    nz = pr.n[2]
    rho_hat = pr.bg["rho_c"][3:3 + nz][:, None, None] if pr.bg else 0.0
    e_hat = (pr.bg["p_c"][3:3 + nz][:, None, None] / (pr.gamma - 1.0)) if pr.bg else 0.0
    out = {}
    hats = {0: rho_hat, 1: 0.0, 2: 0.0, 3: 0.0, 4: e_hat}
    names = {0: "rho", 1: "mx", 2: "my", 3: "mz", 4: "E"}
    for v in range(5):
        a = st["cons"][v] - hats[v]
        b = ref["cons"][v] - hats[v]
        den = np.abs(b).sum()
        if den > 0:
            out[names[v]] = np.abs(a - b).sum() / den
    for k in ("bx", "by", "bz"):
        den = np.abs(ref[k]).sum()
        if den > 0:
            out[k] = np.abs(st[k] - ref[k]).sum() / den
    # the vector fields as one field each
    a = np.abs(st["cons"][1:4] - ref["cons"][1:4]).sum()
    b = np.abs(ref["cons"][1:4]).sum()
    if b > 0:
        out["m"] = a / b
    a = sum(np.abs(st[k] - ref[k]).sum() for k in ("bx", "by", "bz"))
    b = sum(np.abs(ref[k]).sum() for k in ("bx", "by", "bz"))
    if b > 0:
        out["B"] = a / b
    return out


FIELDS = ("rho", "m", "E", "B")


def test_riemann_fp32_close_to_oracle(P):
    """The FP32 deviation-form LHLLD flux of single faces against the oracle's
    FP64 flux of the full states minus the flux of the background state
    (F - F_hat, Sect. 2.8): errors relative to each component's scale."""
    rng = np.random.default_rng(31)
    n = 3000
    g = 5.0 / 3.0
    bg = np.zeros((n, 4))
    bg[:, 0] = rng.uniform(0.1, 1.0, n)
    bg[:, 1] = rng.uniform(0.01, 1.0, n)
    bg[:, 2:] = g
    dl = np.zeros((n, 9))
    dr = np.zeros((n, 9))
    for d in (dl, dr):
        d[:, 0] = 1e-3 * rng.normal(size=n) * bg[:, 0]
        d[:, 1:4] = 1e-2 * rng.normal(size=(n, 3))
        d[:, 4:6] = 1e-3 * rng.normal(size=(n, 2))
        d[:, 6] = 1e-5 * rng.normal(size=n) * bg[:, 1]
    bn = 1e-3 * rng.normal(size=n)
    f32 = P.riemann_batch(dl, dr, bn, bg=bg, solver="lhlld", precision="mixed")
    ref = np.zeros((n, 7))
    for i in range(n):
        full = []
        for d in (dl[i], dr[i]):
            w = d.copy()
            w[0] += bg[i, 0]
            w[6] += bg[i, 1]
            w[7], w[8] = g, g   # gamma_e, gamma_c
            full.append(w)
        hat = np.array([bg[i, 0], 0, 0, 0, 0, 0, bg[i, 1], g, g])
        ref[i] = (O.riemann(full[0], full[1], bn[i], "lhlld") - O.riemann(hat, hat, 0.0, "lhlld"))[:7]
    scale = np.abs(ref).max(axis=0)
    err = (np.abs(f32 - ref) / scale).max(axis=0)
    assert np.all(err < 1e-4), err


@pytest.mark.parametrize("nsteps", [40])
def test_mixed_stratified_box_l1_deviations(P, nsteps):
    """Box with the C2 physics (polytrope, heating, noise 1e-3, beta 1e6, walls)."""
    pr = W.stratified_box(32, 32, 48)
    o = O.Oracle(pr)
    g = P.Grid(pr, precision="mixed")
    g.load()
    st = dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
    for _ in range(nsteps):
        dt = o.dt(st)
        st, _, _ = o.run(1, st, dt_fixed=dt)
        g.step(1, dt)
    out = g.get_state()
    g.close()
    l1 = deviation_l1(pr, out, st)
    print("mixed L1 of deviations after", nsteps, "steps:", {k: f"{v:.2e}" for k, v in l1.items()})
    for k in FIELDS:
        assert l1[k] <= 1e-5, (k, l1[k])


def test_mixed_long_run_c2_physics(P):
    """The box physics of the 256^3 benchmark (polytrope, heating, density noise
    1e-3, beta 1e6, walls) on 64^3 for the configuration's 500 steps against
    the oracle (its OpenMP build, bit-identical to the plain one), each step
    with the oracle's CFL step: the mixed form's error does not grow past the
    bar over a long run."""
    pr = W.stratified_box(64, 64, 64)
    O.set_parallel(True)
    try:
        o = O.Oracle(pr)
        g = P.Grid(pr, precision="mixed")
        g.load()
        st = dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
        worst = {}
        for n in range(1, 501):
            dt = o.dt(st)
            st, _, _ = o.run(1, st, dt_fixed=dt)
            g.step(1, dt)
            if n in (100, 250, 500):
                l1 = deviation_l1(pr, g.get_state(), st)
                print(f"step {n}:", {k: f"{v:.2e}" for k, v in l1.items()})
                for k in FIELDS:
                    worst[k] = max(worst.get(k, 0.0), l1[k])
        g.close()
    finally:
        O.set_parallel(False)
    for k in FIELDS:
        assert worst[k] <= 1e-5, (k, worst[k])


@pytest.mark.parametrize("bcx", [(0, 0), (1, 1), (2, 2)])
def test_prim_pairs_equal_single_cells(P, bcx):
    """Boxes of even n_x form the primitive deviations two cells of a row per
    thread from aligned FP64 pairs.  The pair form and the cell-by-cell form
    must give bit-identical W and auxiliary planes over the whole work box
    (interior cells and the ghost images of every boundary kind along x,
    mirrored along z), with and without the stage increments, and the same
    CFL rate in the first-stage forms."""
    pr = W.stratified_box(24, 14, 18, amp=3e-2, beta=1e3, mach_heat=3e-2)
    pr.bc = (bcx, (0, 0), (1, 1))
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(1)   # leaves nonzero stage increments behind
    for inc in (False, True):
        a, _ = g.test_prims(0, inc)
        b, _ = g.test_prims(1, inc)
        assert np.count_nonzero(a) > a.size // 4
        assert np.array_equal(a, b), inc
    a, ra = g.test_prims(2)
    b, rb = g.test_prims(3)
    c, _ = g.test_prims(0, False)
    assert ra > 0 and ra == rb
    assert np.array_equal(a, b) and np.array_equal(a, c)
    g.close()
    odd = W.stratified_box(23, 14, 18, amp=3e-2)
    h = P.Grid(odd, precision="mixed")
    with pytest.raises(P.PhlError):
        h.test_prims(1)
    h.close()


@pytest.mark.parametrize("bcx", [(0, 0), (1, 1), (2, 2)])
@pytest.mark.parametrize("eps", [0.5, 5.0])
def test_raw_flags_four_cells_equal_single_cells(P, bcx, eps):
    """Boxes with n_x a multiple of 4 take the raw shock flags four cells of a
    row per thread; the flags and the vote must equal the cell-by-cell
    kernel's bit for bit -- with flagged cells next to unflagged ones (on
    16 cells the stratification alone gives 0.25 at the bottom and 1.1 at
    the top; a slab of raised pressure adds jumps) and with none (a
    threshold above every cell's jump)."""
    pr = W.stratified_box(24, 12, 16, amp=3e-2, beta=1e3, mach_heat=3e-2)
    pr.bc = (bcx, (0, 0), (1, 1))
    pr.eps_sf = eps
    if eps < 1.0:   # a pressure jump across a slab: flagged cells next to unflagged ones
        pr.cons[4, :, :, 9:14] *= 1.5
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.test_prims(0, False)
    a, va = g.test_raw_flags(0)
    b, vb = g.test_raw_flags(1)
    assert np.array_equal(a, b)
    assert va == vb == int(a.any())
    if eps < 1.0:
        assert 0 < a.sum() < a.size
    else:
        assert a.sum() == 0
    g.close()


def test_mixed_orszag_tang_close_to_oracle(P):
    pr = W.orszag_tang(64)
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(30, 2e-3)
    out = g.get_state()
    g.close()
    ref, _, _ = O.Oracle(pr).run(30, dt_fixed=2e-3)
    l1 = deviation_l1(pr, out, ref)
    for k in FIELDS:
        assert l1[k] <= 1e-5, (k, l1[k])


def test_mixed_well_balanced_rest(P):
    pr = W.stratified_box(16, 16, 32, amp=0.0, heat=False)
    pr.bx[:] = 0.0
    pr.cons[4] = pr.bg["p_c"][3:3 + 32][:, None, None] * np.ones((32, 16, 16)) / (pr.gamma - 1.0)
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(100, 2e-3)
    out = g.get_state()
    g.close()
    u = np.abs(out["cons"][1:4] / out["cons"][0]).max()
    assert u <= 1e-12, u
    assert np.abs(out["cons"][0] - pr.cons[0]).max() <= 1e-13


def test_mixed_mass_conservation_periodic(P):
    """Periodic box without gravity: total mass changes only by the FP64
    rounding of the accumulation and the FP32 rounding of the increments."""
    n = 24
    rng = np.random.default_rng(9)
    pr = W.stratified_box(n, n, n, amp=0.0, heat=False)
    pr.bc = ((0, 0), (0, 0), (0, 0))
    pr.g = (0.0, 0.0, 0.0)
    pr.bg, pr.heat = None, None
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, size=(n, n, n))
    v = 0.05 * rng.standard_normal((3, n, n, n))
    p0 = 1.0
    pr.cons[0] = rho
    pr.cons[1:4] = rho * v
    b2 = 0.5 * pr.bx[:, :, :-1] ** 2
    pr.cons[4] = p0 / (pr.gamma - 1.0) + 0.5 * rho * (v ** 2).sum(axis=0) + b2
    g = P.Grid(pr, precision="mixed")
    g.load()
    g.step(50)
    out = g.get_state()
    g.close()
    for v_ in (0, 4):
        t0 = pr.cons[v_].sum()
        assert abs(out["cons"][v_].sum() - t0) <= 1e-10 * abs(t0), v_


def test_mixed_form_is_unit_invariant(P):
    """The FP32 quantities are held in power-of-two units near the
    background's scales: the same box in units where P ~ 2^80 (stellar CGS
    magnitudes, whose squares overflow FP32) steps to the exactly rescaled
    result of the unit box."""
    pr = W.stratified_box(16, 16, 32, amp=3e-2, beta=1e3, mach_heat=3e-2)
    s_rho, s_p, s_l = 2.0 ** 24, 2.0 ** 80, 2.0 ** 27
    s_v = 2.0 ** 28                      # sqrt(s_p / s_rho)
    s_b, s_t = 2.0 ** 40, s_l / s_v
    q = pr.copy()
    q.lo = tuple(x * s_l for x in pr.lo)
    q.hi = tuple(x * s_l for x in pr.hi)
    q.g = tuple(x * s_v * s_v / s_l for x in pr.g)
    q.cons = pr.cons.copy()
    q.cons[0] *= s_rho
    q.cons[1:4] *= s_rho * s_v
    q.cons[4] *= s_p
    q.bx, q.by, q.bz = pr.bx * s_b, pr.by * s_b, pr.bz * s_b
    q.bg = dict(rho_c=pr.bg["rho_c"] * s_rho, rho_f=pr.bg["rho_f"] * s_rho,
                p_c=pr.bg["p_c"] * s_p, p_f=pr.bg["p_f"] * s_p)
    q.heat = pr.heat * s_p / s_t
    out = []
    for prob in (pr, q):
        g = P.Grid(prob, precision="mixed")
        g.load()
        g.step(6)
        out.append(g.get_state())
        g.close()
    a, b = out
    assert np.array_equal(b["cons"][0], a["cons"][0] * s_rho)
    assert np.array_equal(b["cons"][1:4], a["cons"][1:4] * (s_rho * s_v))
    assert np.array_equal(b["cons"][4], a["cons"][4] * s_p)
    for k in ("bx", "by", "bz"):
        assert np.array_equal(b[k], a[k] * s_b)


@pytest.mark.parametrize("solver", ["lhlld", "hlld", "hll"])
@pytest.mark.parametrize("regime", ["low_mach", "strong"])
def test_riemann_fp32x2_pairs(P, solver, regime):
    """The fused kernel's paired ideal-gas solver (two faces per thread on
    packed FP32x2 arithmetic) against the FP64 solver and the scalar FP32 one,
    on independent random faces: low-Mach deviations from a background, and
    O(1) jumps with fields (every HLLD region, subsonic and supersonic)."""
    rng = np.random.default_rng(77 if regime == "low_mach" else 78)
    n = 4001                    # odd: the last pair repeats its face
    g = 5.0 / 3.0
    bg = np.zeros((n, 4))
    bg[:, 2:] = g
    dl = np.zeros((n, 9))
    dr = np.zeros((n, 9))
    if regime == "low_mach":
        bg[:, 0] = rng.uniform(0.1, 1.0, n)
        bg[:, 1] = rng.uniform(0.01, 1.0, n)
        for d in (dl, dr):
            d[:, 0] = 1e-3 * rng.normal(size=n) * bg[:, 0]
            d[:, 1:4] = 1e-2 * rng.normal(size=(n, 3))
            d[:, 4:6] = 1e-3 * rng.normal(size=(n, 2))
            d[:, 6] = 1e-5 * rng.normal(size=n) * bg[:, 1]
        bn = 1e-3 * rng.normal(size=n)
    else:
        for d in (dl, dr):
            d[:, 0] = rng.uniform(0.2, 2.0, n)
            d[:, 1:4] = rng.normal(size=(n, 3)) * rng.choice([0.1, 1.0, 3.0], size=(n, 1))
            d[:, 4:6] = rng.normal(size=(n, 2))
            d[:, 6] = rng.uniform(0.1, 2.0, n)
        bn = rng.normal(size=n) * rng.choice([0.0, 1e-3, 1.0], size=n)
    kw = dict(bg=bg, solver=solver)
    f32 = P.riemann_batch(dl, dr, bn, precision="mixed", **kw)
    f64 = P.riemann_batch(dl, dr, bn, precision="fp64", **kw)
    scale = np.abs(f64).max(axis=0) + 1e-300
    err32 = (np.abs(f32 - f64) / scale).max(axis=0)
    # both paired solvers (two faces per thread; left/right states of one face)
    # are as accurate as the scalar FP32 one (a few FP32 ulps of each
    # component's scale; the deviation form keeps low-Mach fluxes free of
    # cancellation)
    for prec in ("mixed_x2", "mixed_lr"):
        fp = P.riemann_batch(dl, dr, bn, precision=prec, **kw)
        assert np.all(np.isfinite(fp)), prec
        err = (np.abs(fp - f64) / scale).max(axis=0)
        assert np.all(err < np.maximum(4.0 * err32, 1e-5)), (prec, err, err32)
