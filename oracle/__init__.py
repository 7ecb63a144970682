"""ctypes front end of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It never touches the CUDA library; the CUDA library never
touches it.  Problems come from workloads/ (seeded inputs shared by both).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ORA_MAXSPEC = 4
_RIEMANN = {"lhlld": 0, "hlld": 1, "hll": 2}
_EOS = {"ideal": 0, "stellar": 1}
_RECON = {"vanleer": 0, "pph": 1, "pqh": 2}

_dp = C.POINTER(C.c_double)


class OraCfg(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", (C.c_int * 2) * 3), ("eos", C.c_int), ("gamma", C.c_double),
        ("nspec", C.c_int), ("A", C.c_double * ORA_MAXSPEC), ("Z", C.c_double * ORA_MAXSPEC),
        ("g", C.c_double * 3),
        ("bg_rho_c", _dp), ("bg_p_c", _dp), ("bg_rho_f", _dp), ("bg_p_f", _dp),
        ("bg_ge_c", _dp), ("bg_gc_c", _dp), ("bg_ge_f", _dp), ("bg_gc_f", _dp),
        ("heat", _dp), ("cfl", C.c_double), ("rk", C.c_int), ("riemann", C.c_int),
        ("eps_sf", C.c_double), ("mach_thr", C.c_double), ("newton_tol", C.c_double),
        ("newton_maxit", C.c_int), ("eos_table", C.c_void_p), ("recon", C.c_int),
    ]


class OraDiff(C.Structure):
    _fields_ = [("k0", C.c_double), ("nT", C.c_int), ("nR", C.c_int), ("cv", C.c_double), ("delta_T", C.c_int)]


class OraPoisson(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("xf", _dp * 3), ("G", C.c_double), ("lmax", C.c_int),
                ("criterion", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int)]


_CRITERION = {"relative": 0, "absolute": 1}


_lib = None
_libs = {}
_parallel = False


def set_parallel(on: bool) -> None:
    """Run the oracle's stage loops over all host cores (the -fopenmp build of
    the same sources, bit-identical results) or single-threaded (default)."""
    global _lib, _parallel
    _parallel = bool(on)
    _lib = None


def lib():
    global _lib
    if _lib is None:
        _build.build()
        path = _build.LIB_OMP if _parallel else _build.LIB
        if path in _libs:
            _lib = _libs[path]
            return _lib
        L = C.CDLL(path)
        L.ora_run.restype = C.c_int
        L.ora_run.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp, _dp, _dp, C.c_int, C.c_double, _dp, _dp]
        L.ora_dt.restype = C.c_double
        L.ora_dt.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp, _dp, _dp]
        L.ora_stage.restype = C.c_int
        L.ora_stage.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                C.c_double, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
        L.ora_riemann.restype = None
        L.ora_riemann.argtypes = [_dp, _dp, C.c_double, C.c_int, C.c_int, C.c_double, _dp]
        L.ora_divb.restype = C.c_double
        L.ora_divb.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp]
        L.ora_diffuse.restype = C.c_int
        L.ora_diffuse.argtypes = [C.POINTER(OraCfg), _dp, _dp, _dp, _dp, C.POINTER(OraDiff), C.c_double, C.c_int,
                                  C.POINTER(C.c_int)]
        L.ora_recon_cell.restype = None
        L.ora_recon_cell.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.ora_poisson_nghost.restype = C.c_long
        L.ora_poisson_nghost.argtypes = [C.POINTER(C.c_int)]
        L.ora_multipole_moments.restype = C.c_int
        L.ora_multipole_moments.argtypes = [C.POINTER(OraPoisson), _dp, _dp, _dp, _dp, _dp]
        L.ora_multipole_phi.restype = C.c_double
        L.ora_multipole_phi.argtypes = [C.c_double, C.c_int, C.c_double, _dp, _dp, _dp,
                                        C.c_double, C.c_double, C.c_double]
        L.ora_poisson_boundary.restype = C.c_int
        L.ora_poisson_boundary.argtypes = [C.POINTER(OraPoisson), _dp, _dp]
        L.ora_poisson_apply.restype = C.c_int
        L.ora_poisson_apply.argtypes = [C.POINTER(OraPoisson), _dp, _dp, _dp]
        L.ora_gravity.restype = C.c_int
        L.ora_gravity.argtypes = [C.POINTER(OraPoisson), _dp, _dp, _dp, _dp, _dp]
        L.ora_poisson_solve.restype = C.c_int
        L.ora_poisson_solve.argtypes = [C.POINTER(OraPoisson), _dp, _dp, _dp, C.POINTER(C.c_int), _dp]
        L.ora_rkl2_amp.restype = C.c_double
        L.ora_rkl2_amp.argtypes = [C.c_int, C.c_double]
        L.ora_sts_stages.restype = C.c_int
        L.ora_sts_stages.argtypes = [C.c_double, C.c_double]
        L.ora_eos_table_build.restype = C.c_void_p
        L.ora_eos_table_build.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
        L.ora_eos_table_free.restype = None
        L.ora_eos_table_free.argtypes = [C.c_void_p]
        L.ora_eos_table_size.restype = C.c_long
        L.ora_eos_table_size.argtypes = [C.c_void_p]
        L.ora_eos_table_export.restype = C.c_int
        L.ora_eos_table_export.argtypes = [C.c_void_p, _dp, C.c_long]
        L.ora_ep_direct.restype = C.c_int
        L.ora_ep_direct.argtypes = [C.c_double, C.c_double, C.c_double] + [_dp] * 5
        L.ora_ep_first.restype = C.c_int
        L.ora_ep_first.argtypes = [C.c_double, C.c_double, _dp]
        L.ora_ep_derivs.restype = C.c_int
        L.ora_ep_derivs.argtypes = [C.c_double, C.c_double, _dp]
        L.ora_sphere_create.restype = C.c_void_p
        L.ora_sphere_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double] + [_dp] * 6 + \
            [C.c_double, C.c_int, C.c_double]
        L.ora_sphere_free.restype = None
        L.ora_sphere_free.argtypes = [C.c_void_p]
        for nm in ("ncells", "nfaces", "nedges", "nabi_faces"):
            getattr(L, "ora_sphere_" + nm).restype = C.c_long
            getattr(L, "ora_sphere_" + nm).argtypes = [C.c_void_p]
        L.ora_sphere_geometry.restype = C.c_int
        L.ora_sphere_geometry.argtypes = [C.c_void_p] + [_dp] * 5
        L.ora_sphere_dt.restype = C.c_double
        L.ora_sphere_dt.argtypes = [C.c_void_p] + [_dp] * 4
        L.ora_sphere_run.restype = C.c_int
        L.ora_sphere_run.argtypes = [C.c_void_p] + [_dp] * 4 + [C.c_int, C.c_double, _dp]
        L.ora_sphere_divb.restype = C.c_int
        L.ora_sphere_divb.argtypes = [C.c_void_p] + [_dp] * 4
        L.ora_sphere_set_stellar.restype = C.c_int
        L.ora_sphere_set_stellar.argtypes = [C.c_void_p, C.POINTER(OraCfg), _dp, C.c_double, C.c_double]
        L.ora_sphere_from_prims.restype = C.c_int
        L.ora_sphere_from_prims.argtypes = [C.c_void_p] + [_dp] * 7
        L.ora_sphere_set_T.restype = C.c_int
        L.ora_sphere_set_T.argtypes = [C.c_void_p, _dp]
        L.ora_sphere_get_T.restype = C.c_int
        L.ora_sphere_get_T.argtypes = [C.c_void_p, _dp]
        L.ora_ct_corner.restype = C.c_double
        L.ora_ct_corner.argtypes = [_dp, _dp, _dp, C.c_double, C.c_double]
        L.ora_fd.restype = C.c_double
        L.ora_fd.argtypes = [C.c_double, C.c_double, C.c_double]
        L.ora_eos_rt.restype = C.c_int
        L.ora_eos_rt.argtypes = [C.POINTER(OraCfg), C.c_double, C.c_double, _dp] + [_dp] * 7
        L.ora_eos_invert.restype = C.c_int
        L.ora_eos_invert.argtypes = [C.POINTER(OraCfg), C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp,
                                     C.POINTER(C.c_int)]
        L.ora_mlp_forward.restype = None
        L.ora_mlp_forward.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_long, _dp]
        L.ora_mlp_loss_grad.restype = C.c_double
        L.ora_mlp_loss_grad.argtypes = [_dp, C.c_int, C.c_int, _dp, _dp, C.c_long, _dp]
        _libs[path] = L
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Oracle:
    """Holds a problem's configuration (and keeps its arrays alive)."""

    def __init__(self, pr, rk: int = 3, riemann: str | None = None, eps_sf: float | None = None,
                 cfl: float | None = None, wb: bool = True, newton_tol: float = 1e-11,
                 newton_maxit: int = 50, eos_table=None, mach_thr: float | None = None):
        self.pr = pr
        c = OraCfg()
        for d in range(3):
            c.n[d] = pr.n[d]
            c.lo[d] = pr.lo[d]
            c.hi[d] = pr.hi[d]
            c.bc[d][0], c.bc[d][1] = pr.bc[d]
            c.g[d] = pr.g[d]
        c.eos = _EOS[pr.eos]
        c.gamma = pr.gamma
        c.nspec = pr.nspec
        for l, (a, z) in enumerate(zip(pr.meta.get("A", []), pr.meta.get("Z", []))):
            c.A[l], c.Z[l] = a, z
        self._keep = []
        if pr.bg is not None and wb:
            for key in ("rho_c", "p_c", "rho_f", "p_f", "ge_c", "gc_c", "ge_f", "gc_f"):
                if key in pr.bg:
                    arr = np.ascontiguousarray(pr.bg[key], dtype=np.float64)
                    self._keep.append(arr)
                    setattr(c, "bg_" + key, _ptr(arr))
        if pr.heat is not None:
            h = np.ascontiguousarray(pr.heat, dtype=np.float64)
            self._keep.append(h)
            c.heat = _ptr(h)
        c.cfl = pr.cfl if cfl is None else cfl
        c.rk = rk
        c.riemann = _RIEMANN[riemann or pr.riemann]
        c.eps_sf = pr.eps_sf if eps_sf is None else eps_sf
        c.mach_thr = pr.mach_thr if mach_thr is None else mach_thr
        c.newton_tol = newton_tol
        c.newton_maxit = newton_maxit
        c.eos_table = eos_table
        c.recon = _RECON[pr.recon]
        self.cfg = c

    # ------------------------------------------------------------------
    def run(self, nsteps, state=None, dt_fixed=0.0):
        """Advance nsteps; returns (state dict, t, dt_last).  Input state untouched."""
        pr = self.pr
        st = state or dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz, T=pr.T)
        cons = np.ascontiguousarray(st["cons"], dtype=np.float64).copy()
        bx = np.ascontiguousarray(st["bx"], dtype=np.float64).copy()
        by = np.ascontiguousarray(st["by"], dtype=np.float64).copy()
        bz = np.ascontiguousarray(st["bz"], dtype=np.float64).copy()
        T = None if st.get("T") is None else np.ascontiguousarray(st["T"], dtype=np.float64).copy()
        t = C.c_double(0.0)
        dtl = C.c_double(0.0)
        rc = lib().ora_run(C.byref(self.cfg), _ptr(cons), _ptr(bx), _ptr(by), _ptr(bz), _ptr(T),
                           int(nsteps), float(dt_fixed), C.byref(t), C.byref(dtl))
        if rc != 0:
            raise RuntimeError(f"oracle run failed with code {rc}")
        return dict(cons=cons, bx=bx, by=by, bz=bz, T=T), t.value, dtl.value

    def run_to(self, t_end, state=None, max_steps=10 ** 7):
        """Advance to exactly t_end (last step shortened)."""
        st = state or dict(cons=self.pr.cons, bx=self.pr.bx, by=self.pr.by, bz=self.pr.bz, T=self.pr.T)
        t = 0.0
        steps = 0
        while t < t_end * (1 - 1e-14) and steps < max_steps:
            dt = self.dt(st)
            if t + dt > t_end:
                dt = t_end - t
            st, _, _ = self.run(1, st, dt_fixed=dt)
            t += dt
            steps += 1
        return st, t, steps

    def dt(self, state=None):
        pr = self.pr
        st = state or dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz, T=pr.T)
        T = None if st.get("T") is None else np.ascontiguousarray(st["T"]).copy()
        return lib().ora_dt(C.byref(self.cfg), _ptr(np.ascontiguousarray(st["cons"])),
                            _ptr(np.ascontiguousarray(st["bx"])), _ptr(np.ascontiguousarray(st["by"])),
                            _ptr(np.ascontiguousarray(st["bz"])), _ptr(T))

    def diffuse(self, dt, k0, nT=0, nR=0, cv=1.5, state=None, max_stages=100000, delta_T=False):
        """One RKL2 thermal-diffusion super step (diffusion.c); returns
        (state dict with the new total energy, number of stages)."""
        pr = self.pr
        st = state or dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz)
        cons = np.ascontiguousarray(st["cons"], dtype=np.float64).copy()
        p = OraDiff(k0=float(k0), nT=int(nT), nR=int(nR), cv=float(cv), delta_T=int(bool(delta_T)))
        ns = C.c_int(0)
        rc = lib().ora_diffuse(C.byref(self.cfg), _ptr(cons), *[_ptr(np.ascontiguousarray(st[k])) for k in ("bx", "by", "bz")],
                               C.byref(p), float(dt), int(max_stages), C.byref(ns))
        if rc != 0:
            raise RuntimeError(f"oracle diffusion failed with code {rc}")
        out = dict(st)
        out["cons"] = cons
        return out, ns.value

    def divb(self, state):
        return lib().ora_divb(C.byref(self.cfg), _ptr(np.ascontiguousarray(state["bx"])),
                              _ptr(np.ascontiguousarray(state["by"])), _ptr(np.ascontiguousarray(state["bz"])))

    def stage(self, state_in, state_base, a, b, dt):
        cons_o = np.empty_like(state_in["cons"])
        bo = [np.empty_like(state_in[k]) for k in ("bx", "by", "bz")]
        T = None if state_in.get("T") is None else np.ascontiguousarray(state_in["T"]).copy()
        rc = lib().ora_stage(C.byref(self.cfg), *[_ptr(np.ascontiguousarray(state_in[k])) for k in ("cons", "bx", "by", "bz")],
                             _ptr(T), *[_ptr(np.ascontiguousarray(state_base[k])) for k in ("cons", "bx", "by", "bz")],
                             a, b, dt, _ptr(cons_o), *[_ptr(x) for x in bo])
        if rc != 0:
            raise RuntimeError(f"oracle stage failed with code {rc}")
        return dict(cons=cons_o, bx=bo[0], by=bo[1], bz=bo[2], T=T)


class EosTable:
    """The oracle's own e-/e+ free-energy table (its own quadrature)."""

    def __init__(self, lrhoye=(4.0, 8.0), nrho=161, lT=(7.0, 10.0), nT=121):
        self.h = lib().ora_eos_table_build(lrhoye[0], lrhoye[1], nrho, lT[0], lT[1], nT)
        if not self.h:
            raise RuntimeError("oracle EOS table build failed")

    def export(self):
        n = lib().ora_eos_table_size(self.h)
        out = np.zeros(n)
        lib().ora_eos_table_export(self.h, _ptr(out), n)
        return out

    def __del__(self):
        try:
            lib().ora_eos_table_free(self.h)
        except Exception:
            pass


def stellar_cfg(A, Z, table=None, tol=1e-11, maxit=50):
    c = OraCfg()
    c.eos = 1
    c.nspec = len(A)
    for l, (a, z) in enumerate(zip(A, Z)):
        c.A[l], c.Z[l] = a, z
    c.newton_tol = tol
    c.newton_maxit = maxit
    c.eos_table = table.h if table is not None else None
    return c


def eos_rt(cfg, rho, T, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    o = [C.c_double() for _ in range(7)]
    rc = lib().ora_eos_rt(C.byref(cfg), rho, T, _ptr(X), *[C.byref(v) for v in o])
    if rc:
        raise RuntimeError(f"oracle EOS failed ({rc})")
    return dict(zip(("P", "e", "cv", "dPdr", "dPdT", "gamma_e", "gamma_c"), [v.value for v in o]))


def eos_invert(cfg, rho, eint, X, T_guess):
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = C.c_double(T_guess)
    P, ge, gc = C.c_double(), C.c_double(), C.c_double()
    it = C.c_int()
    rc = lib().ora_eos_invert(C.byref(cfg), rho, eint, _ptr(X), C.byref(T), C.byref(P), C.byref(ge), C.byref(gc),
                              C.byref(it))
    if rc:
        raise RuntimeError(f"oracle EOS inversion failed ({rc})")
    return dict(T=T.value, P=P.value, gamma_e=ge.value, gamma_c=gc.value, iters=it.value)


def p_to_T(cfg, rho, P, X, T0=1e9, tol=1e-14, maxit=100):
    """Temperature with P_EoS(rho, T, X) = P: Newton on P (bracketed)."""
    T, lo, hi = T0, 1e7, 1e10
    for _ in range(maxit):
        r = eos_rt(cfg, rho, T, X)
        dp = P - r["P"]
        if dp > 0:
            lo = T
        else:
            hi = T
        if abs(dp) <= tol * P:
            return T
        Tn = T + dp / r["dPdT"]
        T = Tn if lo < Tn < hi else 0.5 * (lo + hi)
    raise RuntimeError("P -> T inversion did not converge")


def prepare_stellar(pr, table):
    """The oracle's own completion of a stellar problem given in primitives:
    background gamma_e, gamma_c (centres and faces) and the cell temperature
    and total energy, all from the oracle EOS with P -> T inversions."""
    q = pr.copy()
    cfg = stellar_cfg(pr.meta["A"], pr.meta["Z"], table)
    bX = pr.meta["bg_X"]
    bg = dict(pr.bg)
    for loc in ("c", "f"):
        rho, P = bg["rho_" + loc], bg["p_" + loc]
        ge, gc = np.zeros_like(rho), np.zeros_like(rho)
        T = 1e9
        for i in range(rho.size):
            T = p_to_T(cfg, rho[i], P[i], bX, T)
            r = eos_rt(cfg, rho[i], T, bX)
            ge[i], gc[i] = r["gamma_e"], r["gamma_c"]
        bg["ge_" + loc], bg["gc_" + loc] = ge, gc
    q.bg = bg
    prim = pr.meta["prim"]
    nz, ny, nx = prim["rho"].shape
    Tc = np.zeros((nz, ny, nx))
    bcx = 0.5 * (pr.bx[:, :, :-1] + pr.bx[:, :, 1:])
    bcy = 0.5 * (pr.by[:, :-1, :] + pr.by[:, 1:, :])
    bcz = 0.5 * (pr.bz[:-1, :, :] + pr.bz[1:, :, :])
    E = np.zeros((nz, ny, nx))
    for k in range(nz):
        T = 1e9
        for j in range(ny):
            for i in range(nx):
                rho = prim["rho"][k, j, i]
                Xc = prim["X"][:, k, j, i]
                T = p_to_T(cfg, rho, prim["p"][k, j, i], Xc, T)
                e = eos_rt(cfg, rho, T, Xc)["e"]
                v = prim["vel"][:, k, j, i]
                Tc[k, j, i] = T
                E[k, j, i] = rho * e + 0.5 * rho * (v ** 2).sum() + 0.5 * (
                    bcx[k, j, i] ** 2 + bcy[k, j, i] ** 2 + bcz[k, j, i] ** 2)
    q.cons = pr.cons.copy()
    q.cons[4] = E
    q.T = Tc
    return q


def ep_direct(rho, ye, T):
    o = [C.c_double() for _ in range(5)]
    rc = lib().ora_ep_direct(rho, ye, T, *[C.byref(v) for v in o])
    if rc:
        raise RuntimeError("oracle e-/e+ evaluation failed")
    return dict(zip(("P", "e", "s", "eta", "npos"), [v.value for v in o]))


def fd(k, eta, beta):
    return lib().ora_fd(k, eta, beta)


def ct_corner(Ef, Ec, F, rho, smax):
    """Contact-CT corner EMF from four face EMFs, four cell EMFs and the four
    faces' mass fluxes (see oracle.h)."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (Ef, Ec, F)]
    return lib().ora_ct_corner(*[_ptr(v) for v in a], float(rho), float(smax))


class Sphere:
    """The oracle's cubed-sphere shell (sphere.c) for a problem from
    workloads.shell_problem: state arrays in the ABI layout.  A stellar
    problem (given in primitives) needs the oracle's EosTable; its energy and
    temperatures come from the oracle's EOS (self.state0)."""

    def __init__(self, pr, riemann="lhlld", cfl=0.4, mach_thr=0.6, wb=True, eos_table=None, newton_tol=1e-11,
                 newton_maxit=50):
        self.pr = pr
        bg = pr.bg if wb and pr.bg is not None else None
        keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return _ptr(a)
        self._keep = keep
        self.h = lib().ora_sphere_create(pr.N, pr.Nr, pr.r_in, pr.r_out, pr.gamma,
                                         arr(bg["rho_c"]) if bg else None, arr(bg["p_c"]) if bg else None,
                                         arr(bg["rho_f"]) if bg else None, arr(bg["p_f"]) if bg else None,
                                         arr(pr.g_c), arr(pr.heat), cfl, _RIEMANN[riemann], mach_thr)
        if not self.h:
            raise RuntimeError("oracle sphere creation failed")
        self.stellar = pr.meta.get("eos") == "stellar"
        self.state0 = dict(cons=pr.cons, pa=pr.pa, pb=pr.pb, pr=pr.pr)
        if self.stellar:
            if eos_table is None:
                raise ValueError("a stellar shell needs the oracle's EosTable")
            self._table = eos_table
            self.ecfg = stellar_cfg(pr.meta["A"], pr.meta["Z"], eos_table, tol=newton_tol, maxit=newton_maxit)
            X = np.ascontiguousarray(pr.meta["X"], dtype=np.float64)
            self._keep.append(X)
            if lib().ora_sphere_set_stellar(self.h, C.byref(self.ecfg), _ptr(X), pr.meta["rho_u"], pr.meta["p_u"]):
                raise RuntimeError("oracle sphere: stellar background failed")
            prim = pr.meta["prim"]
            a = {k: np.ascontiguousarray(prim[k], dtype=np.float64) for k in ("rho", "vel", "p")}
            st = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in self.state0.items()}
            cons = np.zeros_like(st["cons"])
            rc = lib().ora_sphere_from_prims(self.h, _ptr(a["rho"]), _ptr(a["vel"]), _ptr(a["p"]), _ptr(st["pa"]),
                                             _ptr(st["pb"]), _ptr(st["pr"]), _ptr(cons))
            if rc:
                raise RuntimeError(f"oracle sphere: primitives to conserved failed ({rc})")
            self.state0 = dict(st, cons=cons, T=self.get_T())

    def get_T(self):
        T = np.zeros(self.counts()["cells"])
        lib().ora_sphere_get_T(self.h, _ptr(T))
        return T

    def __del__(self):
        try:
            lib().ora_sphere_free(self.h)
        except Exception:
            pass

    def counts(self):
        L = lib()
        return dict(cells=L.ora_sphere_ncells(self.h), faces=L.ora_sphere_nfaces(self.h),
                    edges=L.ora_sphere_nedges(self.h), abi_faces=L.ora_sphere_nabi_faces(self.h))

    def geometry(self):
        n = self.counts()
        vol, xc, csum = np.zeros(n["cells"]), np.zeros((n["cells"], 3)), np.zeros((n["cells"], 3))
        S, xf = np.zeros((n["faces"], 3)), np.zeros((n["faces"], 3))
        lib().ora_sphere_geometry(self.h, _ptr(vol), _ptr(xc), _ptr(S), _ptr(xf), _ptr(csum))
        return dict(vol=vol, xc=xc, S=S, xf=xf, csum=csum)

    def _state(self, st):
        st = st or self.state0
        if self.stellar and st.get("T") is not None:   # the temperatures the state came with: Newton guesses
            lib().ora_sphere_set_T(self.h, _ptr(np.ascontiguousarray(st["T"], dtype=np.float64)))
        return {k: np.ascontiguousarray(st[k], dtype=np.float64).copy() for k in ("cons", "pa", "pb", "pr")}

    def dt(self, state=None):
        st = self._state(state)
        return lib().ora_sphere_dt(self.h, *[_ptr(st[k]) for k in ("cons", "pa", "pb", "pr")])

    def run(self, nsteps, state=None, dt_fixed=0.0):
        st = self._state(state)
        last = C.c_double()
        rc = lib().ora_sphere_run(self.h, *[_ptr(st[k]) for k in ("cons", "pa", "pb", "pr")], int(nsteps),
                                  float(dt_fixed), C.byref(last))
        if rc:
            raise RuntimeError(f"oracle sphere run failed ({rc})")
        if self.stellar:
            st["T"] = self.get_T()
        return st, last.value

    def divb(self, state=None):
        st = self._state(state)
        out = np.zeros(self.counts()["cells"])
        lib().ora_sphere_divb(self.h, *[_ptr(st[k]) for k in ("pa", "pb", "pr")], _ptr(out))
        return out


def ep_first(nnet, T):
    """f, f_x, f_y, f_xy of the e-/e+ free-energy density from the integrals'
    own combinations (x = ln n, y = ln T)."""
    out = np.zeros(4)
    if lib().ora_ep_first(nnet, T, _ptr(out)):
        raise RuntimeError("oracle e-/e+ evaluation failed")
    return out


def ep_derivs(nnet, T):
    """f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy (Taylor-mode)."""
    out = np.zeros(9)
    if lib().ora_ep_derivs(nnet, T, _ptr(out)):
        raise RuntimeError("oracle e-/e+ evaluation failed")
    return out


def riemann(wl, wr, bn, solver="lhlld", mach_thr=0.6, nspec=0):
    """Single-face flux in the normal frame (see oracle.h)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(7 + nspec)
    lib().ora_riemann(_ptr(wl), _ptr(wr), float(bn), int(nspec), _RIEMANN[solver], float(mach_thr), _ptr(f))
    return f


def mlp_forward(w, nin, nh, x):
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(x.shape[0])
    lib().ora_mlp_forward(_ptr(w), nin, nh, _ptr(x), x.shape[0], _ptr(y))
    return y


def mlp_loss_grad(w, nin, nh, x, t):
    w = np.ascontiguousarray(w, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros_like(w)
    loss = lib().ora_mlp_loss_grad(_ptr(w), nin, nh, _ptr(x), _ptr(t), x.shape[0], _ptr(g))
    return loss, g


class Poisson:
    """The oracle's Poisson solver (Sect. 2.12) on a grid given by its face
    coordinates xf = (xf_x, xf_y, xf_z), each n_d + 1 increasing values.
    Cell arrays are [nz][ny][nx]; ghost potentials are one flat array (x
    faces [2][nz][ny], y faces [2][nz][nx], z faces [2][ny][nx])."""

    def __init__(self, xf, G=1.0, lmax=0, criterion="relative", tol=1e-4, max_iter=10000):
        self.xf = [np.ascontiguousarray(a, dtype=np.float64) for a in xf]
        self.n = tuple(len(a) - 1 for a in self.xf)
        self.p = OraPoisson()
        for d in range(3):
            self.p.n[d] = self.n[d]
            self.p.xf[d] = _ptr(self.xf[d])
        self.p.G, self.p.lmax = float(G), int(lmax)
        self.p.criterion, self.p.tol, self.p.max_iter = _CRITERION[criterion], float(tol), int(max_iter)
        self.nghost = lib().ora_poisson_nghost(self.p.n)

    def _cells(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == self.n[::-1], (a.shape, self.n)
        return a

    def moments(self, rho):
        rho = self._cells(rho)
        M, X, Q, O = C.c_double(), np.zeros(3), np.zeros(9), np.zeros(27)
        assert lib().ora_multipole_moments(C.byref(self.p), _ptr(rho), C.byref(M), _ptr(X), _ptr(Q), _ptr(O)) == 0
        return M.value, X, Q.reshape(3, 3), O.reshape(3, 3, 3)

    def multipole_phi(self, moments, pts, lmax=None):
        M, X, Q, O = moments
        X, Q, O = (np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (X, Q, O))
        lm = self.p.lmax if lmax is None else lmax
        return np.array([lib().ora_multipole_phi(self.p.G, lm, M, _ptr(X), _ptr(Q), _ptr(O), *map(float, r))
                         for r in pts])

    def boundary(self, rho):
        gh = np.zeros(self.nghost)
        assert lib().ora_poisson_boundary(C.byref(self.p), _ptr(self._cells(rho)), _ptr(gh)) == 0
        return gh

    def apply(self, phi, ghost=None):
        out = np.zeros(self.n[::-1])
        gh = None if ghost is None else np.ascontiguousarray(ghost, dtype=np.float64)
        assert lib().ora_poisson_apply(C.byref(self.p), _ptr(self._cells(phi)),
                                       _ptr(gh) if gh is not None else None, _ptr(out)) == 0
        return out

    def gravity(self, phi, ghost):
        g = [np.zeros(self.n[::-1]) for _ in range(3)]
        gh = np.ascontiguousarray(ghost, dtype=np.float64)
        assert lib().ora_gravity(C.byref(self.p), _ptr(self._cells(phi)), _ptr(gh), *map(_ptr, g)) == 0
        return g

    def solve(self, rho, phi0=None):
        """Returns (phi, ghost, iterations, final residual RMS, status)."""
        rho = self._cells(rho)
        phi = np.zeros(self.n[::-1]) if phi0 is None else self._cells(phi0).copy()
        gh = np.zeros(self.nghost)
        it, res = C.c_int(), C.c_double()
        st = lib().ora_poisson_solve(C.byref(self.p), _ptr(rho), _ptr(phi), _ptr(gh), C.byref(it), C.byref(res))
        return phi, gh, it.value, res.value, st


def recon_cell(recon, w5, species=False):
    """(left, right) face values of the centre of five cell values."""
    w = np.ascontiguousarray(w5, dtype=np.float64)
    fl, fr = C.c_double(), C.c_double()
    lib().ora_recon_cell(_RECON[recon], int(bool(species)), _ptr(w), C.byref(fl), C.byref(fr))
    return fl.value, fr.value
