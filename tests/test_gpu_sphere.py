"""The cubed-sphere shell on the GPU (phl_sphere_*, FP64) against the CPU
oracle (oracle/sphere.c), element by element, and at the full
6 x 256 x 256 x 384 shell through properties that hold at any size.

Bar: relative L-infinity error per field <= 1e-11,
    max |gpu - oracle| / max |oracle|
for rho, momentum (as one vector field), E and each face-flux array, after
the stated number of steps; both sides take their own CFL steps from their
own state unless a fixed dt is given.  Inputs come from workloads/ only."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def rel_linf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def errors(st, ref):
    e = dict(rho=rel_linf(st["cons"][0], ref["cons"][0]), m=rel_linf(st["cons"][1:4], ref["cons"][1:4]),
             E=rel_linf(st["cons"][4], ref["cons"][4]))
    for k in ("pa", "pb", "pr"):
        e[k] = rel_linf(st[k], ref[k])
    return e


def state0(pr):
    return dict(cons=pr.cons, pa=pr.pa, pb=pr.pb, pr=pr.pr)


def gpu_run(P, pr, nsteps, dt=0.0, wb=True, state=None):
    s = P.Sphere.from_problem(pr, wb=wb)
    st = state or state0(pr)
    s.set_state(*(np.ascontiguousarray(st[k]) for k in ("cons", "pa", "pb", "pr")))
    s.step(nsteps, dt=dt)
    out = s.get_state()
    s.close()
    return out


def oracle_run(pr, nsteps, dt=0.0, wb=True):
    o = O.Sphere(pr, riemann=pr.riemann, cfl=pr.cfl, mach_thr=pr.mach_thr, wb=wb)
    st, _ = o.run(nsteps, dt_fixed=dt)
    return st, o


CASES = [
    # name, shell_problem kwargs, steps, solver, wb
    ("polytrope_field_heat", dict(N=6, Nr=5, amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05), 8,
     "lhlld", True),
    ("no_background", dict(N=6, Nr=5, amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05), 8,
     "lhlld", False),
    ("hlld", dict(N=5, Nr=4, amp=2e-2, beta=30.0, vel_amp=0.1, heat_frac=0.0), 6, "hlld", True),
    ("hll", dict(N=5, Nr=4, amp=2e-2, beta=30.0, vel_amp=0.1, heat_frac=0.0), 6, "hll", True),
    ("smallest_shell", dict(N=2, Nr=2, amp=5e-2, beta=1e2, vel_amp=0.05, heat_frac=0.5), 6, "lhlld", True),
    ("odd_ragged", dict(N=7, Nr=3, amp=1e-2, beta=1e3, vel_amp=0.02, heat_frac=0.3), 5, "lhlld", True),
    ("uniform_medium", dict(N=6, Nr=4, uniform=True, amp=5e-2, beta=1e3, vel_amp=0.05, heat_frac=0.0), 8,
     "lhlld", True),
]


@pytest.mark.parametrize("name,kw,nsteps,solver,wb", CASES, ids=[c[0] for c in CASES])
def test_sphere_matches_oracle(P, name, kw, nsteps, solver, wb):
    kw = dict(kw)
    N, Nr = kw.pop("N"), kw.pop("Nr")
    pr = W.shell_problem(N, Nr, **kw)
    pr.riemann = solver
    ref, o = oracle_run(pr, nsteps, wb=wb)
    st = gpu_run(P, pr, nsteps, wb=wb)
    err = errors(st, ref)
    print(name, {k: f"{v:.2e}" for k, v in err.items()})
    assert all(v <= TOL for v in err.values()), err
    # the state moved: the comparison is not of two copies of the input
    assert np.abs(ref["cons"][1:4] - pr.cons[1:4]).max() > 0
    # every copy of a seam face carries the face's flux in its own orientation
    assert np.abs(o.divb(st)).max() <= 1e-13 * max(np.abs(st["pa"]).max(), np.abs(st["pr"]).max(), 1e-300)


def test_sphere_fixed_dt_and_counts(P):
    pr = W.shell_problem(5, 3, amp=1e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3)
    ref, o = oracle_run(pr, 4, dt=2e-3)
    s = P.Sphere.from_problem(pr)
    c, oc = s.counts(), o.counts()
    assert (c["cells"], c["faces"], c["edges"]) == (oc["cells"], oc["faces"], oc["edges"])
    s.set_state(pr.cons, pr.pa, pr.pb, pr.pr)
    dt_gpu = s.compute_dt()
    dt_ora = o.dt()
    assert abs(dt_gpu - dt_ora) <= 1e-13 * dt_ora
    s.step(4, dt=2e-3)
    st = s.get_state()
    err = errors(st, ref)
    assert all(v <= TOL for v in err.values()), err


def test_sphere_device_state_roundtrip(P):
    import torch
    pr = W.shell_problem(4, 3, amp=1e-2, beta=1e2, vel_amp=0.05)
    host = gpu_run(P, pr, 3)
    s = P.Sphere.from_problem(pr)
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in state0(pr).items()}
    s.set_state(dev["cons"], dev["pa"], dev["pb"], dev["pr"])
    s.step(3)
    out = {k: torch.empty_like(v) for k, v in dev.items()}
    s.get_state(out)
    torch.cuda.synchronize()
    for k in out:
        assert np.array_equal(out[k].cpu().numpy(), host[k]), k


def test_sphere_flags_negative_density(P):
    pr = W.shell_problem(3, 2, amp=0.0, beta=0.0)
    cons = pr.cons.copy()
    cons[0, 2, 1, 1, 1] = -1.0
    s = P.Sphere.from_problem(pr)
    s.set_state(cons, pr.pa, pr.pb, pr.pr)
    with pytest.raises(P.PhlError) as ei:
        s.compute_dt()
    assert ei.value.status == 4   # PHL_ENEGATIVE
    s.set_state(cons, pr.pa, pr.pb, pr.pr)
    s.step(1, dt=1e-6)
    with pytest.raises(P.PhlError) as ei:
        s.check()
    assert ei.value.status in (4, 5)   # the bad cell also poisons its faces' fluxes
    # set_state clears the flags
    s.set_state(pr.cons, pr.pa, pr.pb, pr.pr)
    s.step(1, dt=1e-6)
    s.check()


# ---------------------------------------------------------------------------
# the mixed form: FP32 deviations, fluxes, EMFs and stage increments around
# FP64 U^n and face fluxes


def deviation_l1(pr, st, ref):
    """Relative L1 errors of the deviations from the background (rho - rho_hat,
    E - P_hat / (gamma - 1); momentum and the face fluxes as vector fields)."""
    Nr = pr.Nr
    rho_hat = pr.bg["rho_c"][None, :, None, None] if pr.bg else 0.0
    e_hat = pr.bg["p_c"][None, :, None, None] / (pr.gamma - 1.0) if pr.bg else 0.0
    out = {}
    for name, v, hat in (("rho", 0, rho_hat), ("E", 4, e_hat)):
        a, b = st["cons"][v] - hat, ref["cons"][v] - hat
        out[name] = np.abs(a - b).sum() / np.abs(b).sum()
    out["m"] = np.abs(st["cons"][1:4] - ref["cons"][1:4]).sum() / np.abs(ref["cons"][1:4]).sum()
    out["B"] = sum(np.abs(st[k] - ref[k]).sum() for k in ("pa", "pb", "pr")) / \
        sum(np.abs(ref[k]).sum() for k in ("pa", "pb", "pr"))
    assert Nr == st["cons"].shape[2]
    return out


@pytest.mark.parametrize("nsteps", [40])
def test_sphere_mixed_l1_deviations(P, nsteps):
    """The shell physics of the benchmark (polytrope, radial gravity, heating,
    noise, poloidal field) on 6 x 12 x 12 x 12, each step with the oracle's
    CFL step: the mixed form within 1e-5 of the FP64 oracle in the L1 norm
    of the deviations, per field."""
    pr = W.shell_problem(12, 12, amp=1e-2, beta=1e3, vel_amp=0.02, mach_heat=0.02)
    o = O.Sphere(pr, riemann=pr.riemann, cfl=pr.cfl, mach_thr=pr.mach_thr)
    s = P.Sphere.from_problem(pr, precision="mixed")
    s.set_state(pr.cons, pr.pa, pr.pb, pr.pr)
    st = state0(pr)
    for _ in range(nsteps):
        dt = o.dt(st)
        st, _ = o.run(1, state=st, dt_fixed=dt)
        s.step(1, dt=dt)
    out = s.get_state()
    s.close()
    l1 = deviation_l1(pr, out, st)
    print("sphere mixed L1 of deviations after", nsteps, "steps:", {k: f"{v:.2e}" for k, v in l1.items()})
    for k in ("rho", "m", "E", "B"):
        assert l1[k] <= 1e-5, (k, l1[k])
    # the face fluxes advance in FP64 from the FP32 edge EMFs: div B at FP64
    # rounding, as in the FP64 form
    div = np.abs(o.divb(out)).max()
    scale = max(np.abs(out["pa"]).max(), np.abs(out["pr"]).max())
    print("max |div B| / flux scale:", div / scale)
    assert div <= 1e-13 * scale


def test_sphere_mixed_rest_and_cfl(P):
    """At the hydrostatic rest state every FP32 deviation is exactly zero, so
    the mixed form keeps the state bit for bit; its own CFL step agrees with
    the oracle's to FP32 rounding."""
    pr = W.shell_problem(6, 6, amp=0.0, beta=0.0, heat_frac=0.0)
    s = P.Sphere.from_problem(pr, precision="mixed")
    s.set_state(pr.cons, pr.pa, pr.pb, pr.pr)
    dt = s.compute_dt()
    o = O.Sphere(pr, riemann=pr.riemann, cfl=pr.cfl, mach_thr=pr.mach_thr)
    assert abs(dt - o.dt()) <= 1e-6 * o.dt()
    s.step(5)
    st = s.get_state()
    assert np.array_equal(st["cons"], pr.cons)
    q = W.shell_problem(6, 6, amp=1e-2, beta=1e3, vel_amp=0.05)
    s2 = P.Sphere.from_problem(q, precision="mixed")
    s2.set_state(q.cons, q.pa, q.pb, q.pr)
    o2 = O.Sphere(q, riemann=q.riemann, cfl=q.cfl, mach_thr=q.mach_thr)
    assert abs(s2.compute_dt() - o2.dt()) <= 1e-6 * o2.dt()


# ---------------------------------------------------------------------------
# the full 6 x 256 x 256 x 384 shell

FULL = dict(N=256, Nr=384)


def torch_divb(st):
    """Discrete divergence of every cell from the ABI face fluxes (sum of the
    outward fluxes: + on the upper face of each direction, - on the lower)."""
    pa, pb, prr = st["pa"], st["pb"], st["pr"]
    return (pa[..., 1:] - pa[..., :-1]) + (pb[..., 1:, :] - pb[..., :-1, :]) + (prr[:, 1:] - prr[:, :-1])


def shell_volumes(N, Nr, r):
    """Cell volumes (6, Nr, N, N): (r1^3 - r0^3) / 3 times the solid angle of
    the spherical quad (two triangles, Van Oosterom & Strackee)."""
    d = W.shell_dirs(N)
    a, b, c, e = d[:, :-1, :-1], d[:, :-1, 1:], d[:, 1:, 1:], d[:, 1:, :-1]

    def tri(x, y, z):
        num = np.abs(np.einsum("...i,...i->...", x, np.cross(y, z)))
        den = 1.0 + np.einsum("...i,...i->...", x, y) + np.einsum("...i,...i->...", y, z) + \
            np.einsum("...i,...i->...", z, x)
        return 2.0 * np.arctan2(num, den)
    om = tri(a, b, c) + tri(a, c, e)
    shell = (r[1:] ** 3 - r[:-1] ** 3) / 3.0
    return shell[None, :, None, None] * om[:, None]


def _full_run(P, nsteps, precision="fp64", **kw):
    import torch
    pr = W.shell_problem(FULL["N"], FULL["Nr"], device="cuda", **kw)
    torch.cuda.synchronize()
    s = P.Sphere.from_problem(pr, precision=precision)
    s.set_state(pr.cons, pr.pa, pr.pb, pr.pr)
    s.step(nsteps)
    out = {k: torch.empty_like(getattr(pr, k)) for k in ("cons", "pa", "pb", "pr")}
    s.get_state(out)
    torch.cuda.synchronize()
    s.close()
    return pr, out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_shell_well_balanced_rest(P, precision):
    import torch
    pr, st = _full_run(P, 3, precision, amp=0.0, beta=0.0, heat_frac=0.0)
    cs = math.sqrt(pr.gamma * pr.bg["p_c"].max() / pr.bg["rho_c"].min())
    u = st["cons"][1:4] / st["cons"][0]
    assert float(u.abs().max()) <= 1e-12 * cs
    assert float((st["cons"] - pr.cons).abs().max()) <= 1e-12 * float(pr.cons.abs().max())
    del st, pr
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision,cons_tol", [("fp64", 1e-13), ("mixed", 1e-9)])
def test_full_shell_divb_and_conservation(P, precision, cons_tol):
    """div B of every cell (both forms advance the face fluxes in FP64: FP64
    rounding) and the totals of mass and energy between the reflecting walls
    (the mixed form's cell increments are FP32: FP32 rounding of the fluxes)."""
    import torch
    pr, st = _full_run(P, 3, precision, uniform=True, amp=2e-2, beta=1e3, vel_amp=0.05, heat_frac=0.0)
    scale = max(float(pr.pa.abs().max()), float(pr.pr.abs().max()))
    div_tol = 1e-13
    print(precision, "max |div B| / scale:", float(torch_divb(st).abs().max()) / scale)
    assert float(torch_divb(st).abs().max()) <= div_tol * scale
    flux_scale = max(float(pr.pa.abs().max()), float(pr.pr.abs().max()))
    assert float(torch_divb(dict(pa=pr.pa, pb=pr.pb, pr=pr.pr)).abs().max()) <= 1e-13 * flux_scale
    vol = torch.from_numpy(shell_volumes(pr.N, pr.Nr, pr.meta["r"])).cuda()
    for v in (0, 4):   # mass and total energy between reflecting walls
        q0, q1 = float((vol * pr.cons[v]).sum()), float((vol * st["cons"][v]).sum())
        print(precision, "relative change of the total", ["mass", "", "", "", "energy"][v], abs(q1 - q0) / abs(q0))
        assert abs(q1 - q0) <= cons_tol * abs(q0), (v, q0, q1)
    assert float((st["cons"][1:4] - pr.cons[1:4]).abs().max()) > 0
    del st, pr
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# the stellar EOS on the shell (Sect. 2.2: ions, radiation, the e-/e+ table;
# 16O/28Si 0.5/0.5 everywhere).  The problem comes in primitives: the device
# and the oracle each build the energy and the temperatures with their own
# EOS table.


@pytest.fixture(scope="module")
def st_tables(P):
    return P.EosTable(), O.EosTable()


def stellar_pair(P, pr, tables, precision="fp64", mlp=None, wb=True):
    dtab, otab = tables
    o = O.Sphere(pr, riemann=pr.riemann, cfl=pr.cfl, mach_thr=pr.mach_thr, eos_table=otab, wb=wb)
    s = P.Sphere.from_problem(pr, precision=precision, eos_table=dtab, mlp=mlp, wb=wb)
    s.load(pr)
    return s, o


def temps(pr, T):
    return np.asarray(T).reshape(6, pr.Nr, pr.N, pr.N)


STELLAR_CASES = [
    ("polytrope_field_heat", dict(N=5, Nr=4, amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05), 5,
     "lhlld", True),
    ("no_background", dict(N=5, Nr=4, amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05), 4,
     "lhlld", False),
    ("hlld", dict(N=4, Nr=4, amp=2e-2, beta=30.0, vel_amp=0.1, heat_frac=0.0), 4, "hlld", True),
    ("uniform_medium", dict(N=4, Nr=3, uniform=True, amp=5e-2, beta=1e3, vel_amp=0.05, heat_frac=0.0), 5,
     "lhlld", True),
]


@pytest.mark.parametrize("name,kw,nsteps,solver,wb", STELLAR_CASES, ids=[c[0] for c in STELLAR_CASES])
def test_stellar_sphere_matches_oracle(P, st_tables, name, kw, nsteps, solver, wb):
    kw = dict(kw)
    N, Nr = kw.pop("N"), kw.pop("Nr")
    pr = W.shell_problem(N, Nr, eos="stellar", **kw)
    pr.riemann = solver
    s, o = stellar_pair(P, pr, st_tables, wb=wb)
    # the loaded state: E and T from the primitives by each side's EOS
    e0 = errors(s.get_state(), o.state0)
    assert all(v <= TOL for v in e0.values()), e0
    assert rel_linf(s.get_temperature(), temps(pr, o.state0["T"])) <= TOL
    ref, _ = o.run(nsteps)
    s.step(nsteps)
    st = s.get_state()
    err = errors(st, ref)
    err["T"] = rel_linf(s.get_temperature(), temps(pr, ref["T"]))
    s.close()
    print(name, {k: f"{v:.2e}" for k, v in err.items()})
    assert all(v <= TOL for v in err.values()), err
    assert np.abs(ref["cons"][1:4] - o.state0["cons"][1:4]).max() > 0
    assert np.abs(o.divb(st)).max() <= 1e-13 * max(np.abs(st["pa"]).max(), np.abs(st["pr"]).max(), 1e-300)


def stellar_e_hat(pr, otab):
    """The background's energy density rho_hat e(rho_hat, T_hat) per shell
    (code units), from the oracle's EOS."""
    cfg = O.stellar_cfg(pr.meta["A"], pr.meta["Z"], otab)
    ru, pu = pr.meta["rho_u"], pr.meta["p_u"]
    out = np.zeros(pr.Nr)
    T = 1e9
    for k in range(pr.Nr):
        rho, p = pr.bg["rho_c"][k] * ru, pr.bg["p_c"][k] * pu
        T = O.p_to_T(cfg, rho, p, pr.meta["X"], T)
        out[k] = pr.bg["rho_c"][k] * O.eos_rt(cfg, rho, T, pr.meta["X"])["e"] * ru / pu
    return out


def test_stellar_sphere_mixed_l1_deviations(P, st_tables):
    """The mixed form (FP32 deviations, FP64 inversion) of the stellar shell,
    each step with the oracle's CFL step: L1 of the deviations from the
    background per field within 1e-5 of the FP64 oracle."""
    pr = W.shell_problem(8, 8, eos="stellar", amp=1e-2, beta=1e3, vel_amp=0.02, mach_heat=0.02)
    s, o = stellar_pair(P, pr, st_tables, precision="mixed")
    st = o.state0
    for _ in range(20):
        dt = o.dt(st)
        st, _ = o.run(1, state=st, dt_fixed=dt)
        s.step(1, dt=dt)
    out = s.get_state()
    T = s.get_temperature()
    s.close()
    rho_hat = pr.bg["rho_c"][None, :, None, None]
    e_hat = stellar_e_hat(pr, st_tables[1])[None, :, None, None]
    l1 = {}
    for name, v, hat in (("rho", 0, rho_hat), ("E", 4, e_hat)):
        a, b = out["cons"][v] - hat, st["cons"][v] - hat
        l1[name] = np.abs(a - b).sum() / np.abs(b).sum()
    l1["m"] = np.abs(out["cons"][1:4] - st["cons"][1:4]).sum() / np.abs(st["cons"][1:4]).sum()
    l1["B"] = sum(np.abs(out[k] - st[k]).sum() for k in ("pa", "pb", "pr")) / \
        sum(np.abs(st[k]).sum() for k in ("pa", "pb", "pr"))
    print("stellar sphere mixed L1 of deviations:", {k: f"{v:.2e}" for k, v in l1.items()})
    for k, v in l1.items():
        assert v <= 1e-5, (k, v)
    assert rel_linf(T, temps(pr, st["T"])) <= 1e-6
    assert np.abs(o.divb(out)).max() <= 1e-13 * max(np.abs(out["pa"]).max(), np.abs(out["pr"]).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stellar_sphere_rest(P, st_tables, precision):
    """The stellar polytrope at rest stays at rest (both forms)."""
    pr = W.shell_problem(6, 6, eos="stellar", amp=0.0, beta=0.0, heat_frac=0.0)
    s, _ = stellar_pair(P, pr, st_tables, precision=precision)
    st0 = s.get_state()
    s.step(4)
    st = s.get_state()
    s.close()
    cs = math.sqrt(5.0 / 3.0 * pr.bg["p_c"].max() / pr.bg["rho_c"].min())
    assert np.abs(st["cons"][1:4] / st["cons"][0]).max() <= 1e-12 * cs
    assert np.abs(st["cons"][4] / st0["cons"][4] - 1.0).max() <= 1e-13


def test_stellar_sphere_cold_start_network_guess(P, st_tables):
    """A state loaded without temperatures: the first inversion starts from
    the network's guess (cold start) or from the shell background's
    temperature; both converge to the temperatures the loaded primitives
    gave, and the steps agree with the warm run to the Newton tolerance."""
    pr = W.shell_problem(5, 4, eos="stellar", amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05)
    m = P.Mlp(seed=11)
    m.train(st_tables[0], nsamples=2_000_000, epochs=4, batch=1024, lr=1e-2, seed=99)
    warm, _ = stellar_pair(P, pr, st_tables)
    st0 = warm.get_state()
    T0 = warm.get_temperature()
    warm.step(2, dt=1e-3)
    ref, Tref = warm.get_state(), warm.get_temperature()
    for mlp in (m, None):
        s = P.Sphere.from_problem(pr, eos_table=st_tables[0], mlp=mlp)
        s.set_state(st0["cons"], st0["pa"], st0["pb"], st0["pr"])
        s.step(2, dt=1e-3)
        out, T = s.get_state(), s.get_temperature()
        s.close()
        assert rel_linf(T, Tref) <= 1e-12
        err = errors(out, ref)
        assert all(v <= 1e-12 for v in err.values()), (mlp is not None, err)
    assert np.abs(T0 - Tref).max() > 0   # the temperatures did move


@pytest.mark.parametrize("eos", ["ideal", "stellar"])
def test_sphere_graph_steps_equal_direct_launches(P, st_tables, eos):
    """Steps replayed as a captured CUDA graph give the direct launches'
    results bit for bit, through a change of dt mode (device CFL step, then a
    fixed dt) and, for the stellar shell, after a cold start."""
    import torch
    pr = W.shell_problem(5, 4, eos=eos, amp=1e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05)
    outs = []
    for graph in (False, True):
        stream = torch.cuda.Stream()
        s = P.Sphere.from_problem(pr, precision="mixed", stream=stream.cuda_stream,
                                  eos_table=st_tables[0] if eos == "stellar" else None)
        s.set_graph(graph)
        s.load(pr)
        if eos == "stellar":   # reload without temperatures: a cold start
            st = s.get_state()
            s.set_state(st["cons"], st["pa"], st["pb"], st["pr"])
        s.step(3)
        s.step(2, dt=1e-3)
        s.step(2, dt=1e-3)
        outs.append(s.get_state())
        s.close()
    for k in ("cons", "pa", "pb", "pr"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_stellar_sphere_resume_with_record(P, st_tables):
    """The mixed stellar shell resumed from its state, temperatures and
    inversion record repeats the uninterrupted run bit for bit."""
    pr = W.shell_problem(4, 4, eos="stellar", amp=2e-2, beta=1e2, vel_amp=0.05, heat_frac=0.3, mach_heat=0.05)
    def fresh():
        s = P.Sphere.from_problem(pr, precision="mixed", eos_table=st_tables[0])
        s.load(pr)
        return s
    a = fresh()
    a.step(4, dt=1e-3)
    whole = a.get_state()
    a.close()
    b = fresh()
    b.step(2, dt=1e-3)
    mid, T, rec = b.get_state(), b.get_temperature(), b.get_eos_record()
    b.close()
    c = fresh()
    c.set_state(mid["cons"], mid["pa"], mid["pb"], mid["pr"])
    c.set_temperature(T)
    c.set_eos_record(rec)
    c.step(2, dt=1e-3)
    out = c.get_state()
    c.close()
    for k in ("cons", "pa", "pb", "pr"):
        assert np.array_equal(out[k], whole[k]), k
