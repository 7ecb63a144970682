"""Host-side argument checks of the C-ABI (include/phl.h): every entry point
rejects a bad descriptor, a bad option or a null handle with PHL_EINVAL and a
message naming the problem, before it makes any CUDA call, so these run on a
machine without a GPU.  Each case starts from a valid descriptor and breaks
one field."""
import ctypes as C
import math

import numpy as np
import pytest

import workloads as W

EINVAL = 1


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as ge
    ge.build()
    import paper_2604_12672_gb300 as P
    return P


def status_and_message(P, st):
    return st, P.lib().phl_last_error().decode()


def create(P, d):
    h = C.c_void_p()
    st, msg = status_and_message(P, P.lib().phl_create_grid(C.byref(d), C.byref(h)))
    assert not h.value            # nothing is handed out on failure
    return st, msg


def set_n(d, n):
    for k in range(3):
        d.n[k] = n[k]


def set_bc(d, k, bc):
    d.bc[k][0], d.bc[k][1] = bc


def set_field(name, value):
    return lambda d: setattr(d, name, value)


GRID_CASES = [
    ("empty axis", lambda d: set_n(d, (0, 8, 8)), "n[0] = 0 < 1"),
    ("axis too short", lambda d: set_n(d, (8, 3, 8)), "active dimension 1 needs n >= 4"),
    ("empty extent", lambda d: d.hi.__setitem__(2, d.lo[2]), "hi[2] <= lo[2]"),
    ("unknown boundary", lambda d: set_bc(d, 0, (3, 3)), "bad boundary condition"),
    ("half-periodic axis", lambda d: set_bc(d, 2, (0, 1)), "periodic on both sides"),
    ("too many species", set_field("nspec", 99), "nspec out of range"),
    ("unknown EOS", set_field("eos", 7), "bad eos"),
    ("stellar EOS without a table", set_field("eos", 1), "needs an eos_table"),
    ("bad network mode", set_field("use_mlp", 3), "use_mlp must be 0, 1 or 2"),
    ("network on an ideal gas", set_field("use_mlp", 1), "use_mlp needs the stellar EOS"),
    ("gamma = 1", set_field("gamma", 1.0), "gamma must exceed 1"),
    ("CFL = 0", set_field("cfl", 0.0), "cfl must be positive"),
    ("CFL = NaN", set_field("cfl", math.nan), "cfl must be positive"),
    ("RK order 4", set_field("rk", 4), "rk must be 2 or 3"),
    ("unknown Riemann solver", set_field("riemann", 3), "bad riemann solver"),
    ("unknown reconstruction", set_field("recon", 3), "bad reconstruction"),
    ("unknown precision", set_field("precision", 5), "bad precision mode"),
    ("background without pressure", set_field("bg_p_c", None), "incomplete background profiles"),
    ("more than 2^31 cells", lambda d: set_n(d, (2048, 2048, 1024)), "grid too large"),
]


@pytest.mark.parametrize("name,breaker,words", GRID_CASES, ids=[c[0] for c in GRID_CASES])
def test_create_grid_rejects_bad_descriptors(P, name, breaker, words):
    pr = W.stratified_box(8, 8, 16)
    d, keep = P.make_desc(pr, precision="mixed")
    breaker(d)
    st, msg = create(P, d)
    assert st == EINVAL and words in msg, (name, st, msg)


def test_create_grid_rejects_null_arguments(P):
    h = C.c_void_p()
    assert status_and_message(P, P.lib().phl_create_grid(None, C.byref(h))) == (EINVAL, "null argument")
    pr = W.stratified_box(8, 8, 16)
    d, keep = P.make_desc(pr)
    assert P.lib().phl_create_grid(C.byref(d), None) == EINVAL


def test_calls_on_a_null_grid_are_rejected(P):
    L = P.lib()
    buf = np.zeros(8)
    p = buf.ctypes.data
    dt = C.c_double()
    diff = P.Diffusion(k0=1.0, nT=0, nR=0, cv=1.5)
    n = C.c_int()
    calls = {
        "phl_step": lambda: L.phl_step(None, 0.0, 1),
        "phl_set_state": lambda: L.phl_set_state(None, p, p, p, p, None, 0),
        "phl_get_state": lambda: L.phl_get_state(None, p, p, p, p, None, 0),
        "phl_compute_dt": lambda: L.phl_compute_dt(None, C.byref(dt)),
        "phl_check": lambda: L.phl_check(None),
        "phl_set_fused": lambda: L.phl_set_fused(None, 1),
        "phl_diffuse": lambda: L.phl_diffuse(None, C.byref(diff), 0.1, 100, C.byref(n)),
        "phl_test_prims": lambda: L.phl_test_prims(None, 0, 0, p, 8, None),
        "phl_test_prims_size": lambda: L.phl_test_prims_size(None, C.byref(C.c_long())),
        "phl_test_raw_flags": lambda: L.phl_test_raw_flags(None, 0, p, 8, None),
    }
    for name, call in calls.items():
        st, msg = status_and_message(P, call())
        assert st == EINVAL and "null" in msg, (name, st, msg)
    L.phl_destroy(None)           # a no-op


def poisson_desc(P, xf, **kw):
    d = P.PoissonDesc()
    for a in range(3):
        d.n[a] = len(xf[a]) - 1
        d.xf[a] = xf[a].ctypes.data
    d.G, d.lmax, d.criterion, d.tol, d.max_iter = 1.0, 0, 0, 1e-8, 100
    for k, v in kw.items():
        setattr(d, k, v)
    return d


POISSON_CASES = [
    ("one cell on an axis", dict(n=1), {}, "at least 2 cells"),
    ("faces not increasing", dict(swap=True), {}, "face coordinates must increase"),
    ("dipole boundary order", {}, dict(lmax=1), "lmax must be 0, 2 or 3"),
    ("unknown criterion", {}, dict(criterion=2), "bad convergence criterion"),
    ("zero tolerance", {}, dict(tol=0.0), "bad tol, max_iter or G"),
    ("no iterations", {}, dict(max_iter=0), "bad tol, max_iter or G"),
    ("G = 0", {}, dict(G=0.0), "bad tol, max_iter or G"),
]


@pytest.mark.parametrize("name,grid,fields,words", POISSON_CASES, ids=[c[0] for c in POISSON_CASES])
def test_poisson_create_rejects_bad_descriptors(P, name, grid, fields, words):
    xf = [np.linspace(-0.5, 0.5, 7), np.linspace(-0.5, 0.5, 6), np.linspace(-0.5, 0.5, 5)]
    if "n" in grid:
        xf[1] = np.array([-0.5, 0.5])
    if grid.get("swap"):
        xf[2] = xf[2].copy()
        xf[2][[1, 2]] = xf[2][[2, 1]]
    d = poisson_desc(P, xf, **fields)
    h = C.c_void_p()
    st, msg = status_and_message(P, P.lib().phl_poisson_create(C.byref(d), C.byref(h)))
    assert st == EINVAL and words in msg and not h.value, (name, st, msg)


def test_poisson_rejects_grids_beyond_32_bit_indexing(P):
    # 2^32 - 2^24 cells is the limit (checked before any allocation)
    xf = [np.linspace(0.0, 1.0, 2049), np.linspace(0.0, 1.0, 2049), np.linspace(0.0, 1.0, 1025)]
    d = poisson_desc(P, xf)
    h = C.c_void_p()
    st, msg = status_and_message(P, P.lib().phl_poisson_create(C.byref(d), C.byref(h)))
    assert st == 8 and "32 bits" in msg and not h.value, (st, msg)      # PHL_EUNSUPPORTED


def test_unit_entry_points_reject_bad_options(P):
    L = P.lib()
    x = np.zeros(4)
    # the conversion's power-of-two scale must stay inside the double range
    st = L.phl_convert_batch(4, x.ctypes.data, 900, x.ctypes.data, x.ctypes.data)
    assert status_and_message(P, st) == (EINVAL, "phl_convert_batch: n < 0 or scale exponent out of range")
    assert L.phl_convert_batch(-1, None, 0, None, None) == EINVAL
    assert status_and_message(P, L.phl_convert_batch(4, None, 0, None, None)) == \
        (EINVAL, "phl_convert_batch: null argument")
    # unknown solver, species on the FP32 paths, too many species
    for solver, nspec, prec, words in ((3, 0, 0, "bad n, nspec or solver"), (0, 1, 2, "take no species"),
                                       (0, 99, 0, "bad n, nspec or solver")):
        st = L.phl_riemann_batch(1, x.ctypes.data, x.ctypes.data, x.ctypes.data, x.ctypes.data,
                                 nspec, solver, 0.6, prec, x.ctypes.data)
        st, msg = status_and_message(P, st)
        assert st == EINVAL and words in msg, (solver, nspec, prec, msg)
    # empty batches succeed without touching the device
    assert L.phl_convert_batch(0, None, 0, None, None) == 0
    assert L.phl_riemann_batch(0, None, None, None, None, 0, 0, 0.6, 0, None) == 0


def test_status_names_cover_the_header(P):
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "phl.h")).read()
    codes = {int(v): k for k, v in re.findall(r"\b(PHL_E[A-Z]+|PHL_OK)\s*=\s*(\d+)", hdr)}
    assert codes == P.STATUS


def _sphere_desc(P, bg):
    d = P.SphereDesc()
    d.N, d.Nr, d.r_in, d.r_out, d.gamma, d.cfl, d.riemann, d.mach_thr = 4, 3, 0.2, 1.0, 5.0 / 3.0, 0.4, 0, 0.6
    for k in ("rho_c", "p_c", "rho_f", "p_f"):
        setattr(d, k, bg[k].ctypes.data)
    return d


SPHERE_CASES = [
    ("one angular cell", set_field("N", 1), "N, Nr >= 2"),
    ("one shell", set_field("Nr", 1), "N, Nr >= 2"),
    ("inner radius zero", set_field("r_in", 0.0), "0 < r_in < r_out"),
    ("inverted radii", set_field("r_out", 0.1), "0 < r_in < r_out"),
    ("gamma = 1", set_field("gamma", 1.0), "gamma > 1"),
    ("zero cfl", set_field("cfl", 0.0), "cfl > 0"),
    ("zero Mach threshold", set_field("mach_thr", 0.0), "mach_thr > 0"),
    ("unknown solver", set_field("riemann", 5), "bad solver"),
    ("unknown precision", set_field("precision", 7), "bad precision"),
    ("partial background", set_field("p_f", None), "all four profiles"),
    ("too many faces", lambda d: (setattr(d, "N", 8000), setattr(d, "Nr", 8000)), "2^31"),
    ("unknown eos", set_field("eos", 3), "bad eos"),
    ("stellar without a table", lambda d: (setattr(d, "eos", 1), setattr(d, "nspec", 1), setattr(d, "rho_unit", 1.0),
                                           setattr(d, "p_unit", 1.0)), "eos_table"),
]


@pytest.mark.parametrize("name,breaker,needle", SPHERE_CASES, ids=[c[0] for c in SPHERE_CASES])
def test_sphere_create_rejects(P, name, breaker, needle):
    bg = {k: np.ones(3 if k.endswith("_c") else 4) for k in ("rho_c", "p_c", "rho_f", "p_f")}
    d = _sphere_desc(P, bg)
    breaker(d)
    h = C.c_void_p()
    st, msg = status_and_message(P, P.lib().phl_sphere_create(C.byref(d), C.byref(h)))
    assert not h.value
    assert st == EINVAL and needle in msg, (st, msg)


def test_sphere_null_handles(P):
    L = P.lib()
    assert L.phl_sphere_create(None, None) == EINVAL
    assert L.phl_sphere_step(None, 0.0, 1) == EINVAL
    assert L.phl_sphere_check(None) == EINVAL
    assert L.phl_sphere_counts(None, None, None, None) == EINVAL
    assert L.phl_sphere_set_state(None, None, None, None, None, 0) == EINVAL
    assert L.phl_sphere_get_state(None, None, None, None, None, 0) == EINVAL
    assert L.phl_sphere_compute_dt(None, None) == EINVAL
    assert L.phl_sphere_set_prims(None, None, None, None, None, None, None, 0) == EINVAL
    assert L.phl_sphere_set_temperature(None, None, 0) == EINVAL
    assert L.phl_sphere_get_temperature(None, None, 0) == EINVAL
    assert L.phl_sphere_set_graph(None, 1) == EINVAL
    assert L.phl_sphere_get_eos_record(None, None, 0) == EINVAL
    assert L.phl_sphere_set_eos_record(None, None, 0) == EINVAL
    L.phl_sphere_destroy(None)
