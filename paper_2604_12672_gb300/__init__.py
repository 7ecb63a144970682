"""GB300-native explicit MHD stage (arXiv 2604.12672, Sect. 2): Python binding.

A thin ctypes layer over the C ABI of libphl.so (include/phl.h): it only
marshals arguments.  Every step of the scheme runs in the library's CUDA
kernels; there is no CPU fallback -- if libphl.so is missing or fails to load,
every entry point raises.  torch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphl.so")

PHL_MAXSPEC = 4
PERIODIC, REFLECT, OUTFLOW = 0, 1, 2
EOS = {"ideal": 0, "stellar": 1}
RIEMANN = {"lhlld": 0, "hlld": 1, "hll": 2}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_x2": 2, "mixed_lr": 3}
RECON = {"vanleer": 0, "pph": 1, "pqh": 2}
HOST, DEVICE = 0, 1
STATUS = {0: "PHL_OK", 1: "PHL_EINVAL", 2: "PHL_ECUDA", 3: "PHL_ENOMEM", 4: "PHL_ENEGATIVE",
          5: "PHL_ENAN", 6: "PHL_ENEWTON", 7: "PHL_ETIMEOUT", 8: "PHL_EUNSUPPORTED", 9: "PHL_ENOCONV"}

_dp = C.POINTER(C.c_double)


class PhlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", (C.c_int * 2) * 3), ("eos", C.c_int), ("gamma", C.c_double),
        ("nspec", C.c_int), ("A", C.c_double * PHL_MAXSPEC), ("Z", C.c_double * PHL_MAXSPEC),
        ("g", C.c_double * 3),
        ("bg_rho_c", _dp), ("bg_p_c", _dp), ("bg_rho_f", _dp), ("bg_p_f", _dp),
        ("bg_ge_c", _dp), ("bg_gc_c", _dp), ("bg_ge_f", _dp), ("bg_gc_f", _dp),
        ("heat", _dp), ("cfl", C.c_double), ("rk", C.c_int), ("riemann", C.c_int),
        ("eps_sf", C.c_double), ("mach_thr", C.c_double), ("precision", C.c_int),
        ("newton_tol", C.c_double), ("newton_maxit", C.c_int), ("use_mlp", C.c_int),
        ("stream", C.c_void_p),
        ("eos_table", C.c_void_p), ("mlp", C.c_void_p), ("bg_X", C.c_double * PHL_MAXSPEC),
        ("recon", C.c_int),
    ]


class Diffusion(C.Structure):
    _fields_ = [("k0", C.c_double), ("nT", C.c_int), ("nR", C.c_int), ("cv", C.c_double),
                ("precision", C.c_int), ("tile_z", C.c_int), ("delta_T", C.c_int)]


DIFF_PRECISION = {"grid": 0, "fp64": 1, "mixed": 2}


class Stats(C.Structure):
    _fields_ = [("steps", C.c_long), ("t", C.c_double), ("last_dt", C.c_double),
                ("device_flags", C.c_int), ("kernels_per_step", C.c_int), ("device_bytes", C.c_size_t),
                ("newton_iters", C.c_long)]


MLP_NPARAM = 4481
MLP_HIDDEN = 64


class MlpTrainCfg(C.Structure):
    _fields_ = [("nsamples", C.c_long), ("epochs", C.c_int), ("batch", C.c_long), ("lr", C.c_double),
                ("seed", C.c_ulonglong), ("lrho", C.c_double * 2), ("lT", C.c_double * 2),
                ("A", C.c_double * 2), ("Z", C.c_double * 2)]


class MlpTrainStats(C.Structure):
    _fields_ = [("final_loss", C.c_double), ("val_rms_log10T", C.c_double), ("val_max_log10T", C.c_double),
                ("steps", C.c_long), ("seconds", C.c_double)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_long), ("ms", C.c_double)]


_lib = None

# every exported symbol of include/phl.h with (restype, argtypes)
_SIGS = {
    "phl_create_grid": (C.c_int, [C.POINTER(GridDesc), C.POINTER(C.c_void_p)]),
    "phl_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_set_state_prim": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_compute_dt": (C.c_int, [C.c_void_p, _dp]),
    "phl_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "phl_check": (C.c_int, [C.c_void_p]),
    "phl_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "phl_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "phl_dt_device_ptr": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "phl_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_set_fused": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_diffuse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "phl_test_tile_wait_timeout": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_test_prims": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_long, C.POINTER(C.c_float)]),
    "phl_test_prims_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_long)]),
    "phl_test_raw_flags": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_long, C.POINTER(C.c_int)]),
    "phl_convert_batch": (C.c_int, [C.c_long, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "phl_kernel_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "phl_destroy": (None, [C.c_void_p]),
    "phl_last_error": (C.c_char_p, []),
    "phl_probe_alu": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "phl_cfl_dt_noalloc": (C.c_int, [C.POINTER(GridDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "phl_eos_table_create": (C.c_int, [C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                       C.POINTER(C.c_void_p)]),
    "phl_eos_table_destroy": (None, [C.c_void_p]),
    "phl_mlp_create": (C.c_int, [C.c_ulonglong, C.POINTER(C.c_void_p)]),
    "phl_mlp_destroy": (None, [C.c_void_p]),
    "phl_mlp_set_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "phl_mlp_get_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "phl_mlp_set_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "phl_mlp_get_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "phl_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_long, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                    C.c_void_p, C.c_int]),
    "phl_mlp_forward": (C.c_int, [C.c_void_p, C.c_long, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_mlp_guess_temperature": (C.c_int, [C.c_void_p, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int]),
    "phl_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(MlpTrainCfg), C.POINTER(MlpTrainStats)]),
    "phl_ensemble_create": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "phl_ensemble_grid": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "phl_ensemble_step": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_ensemble_check": (C.c_int, [C.c_void_p]),
    "phl_ensemble_set_shape": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "phl_ensemble_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "phl_ensemble_get_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "phl_ensemble_destroy": (None, [C.c_void_p]),
    "phl_eos_table_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_long]),
    "phl_eos": (C.c_int, [C.c_void_p, C.c_long] + [C.c_void_p] * 10 + [C.c_int, C.c_double, C.c_int, C.c_int,
                                                                          C.c_void_p]),
    "phl_riemann_batch": (C.c_int, [C.c_long, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_int, C.c_double, C.c_int, C.c_void_p]),
    "phl_poisson_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "phl_poisson_destroy": (C.c_int, [C.c_void_p]),
    "phl_poisson_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)]),
    "phl_poisson_ghost": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_poisson_gravity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "phl_sphere_destroy": (None, [C.c_void_p]),
    "phl_sphere_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long), C.POINTER(C.c_long)]),
    "phl_sphere_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_compute_dt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "phl_sphere_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "phl_sphere_check": (C.c_int, [C.c_void_p]),
    "phl_sphere_set_prims": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int]),
    "phl_sphere_set_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_sphere_get_eos_record": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_set_eos_record": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_get_eos_record": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_set_eos_record": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_set_temperature": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_get_temperature": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "phl_sphere_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "phl_sphere_kernel_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int]),
}


def lib():
    """Load libphl.so (in-tree build).  Raises if it is missing: no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise PhlError(st, lib().phl_last_error().decode())


def _ptr(a):
    """Raw pointer and location of a numpy array or a torch tensor."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "float64 C-contiguous array expected"
        return a.ctypes.data, HOST
    # torch tensor
    assert a.is_contiguous(), "contiguous tensor expected"
    return a.data_ptr(), (DEVICE if a.is_cuda else HOST)


def convert_batch(x, k):
    """Device FP64 -> FP32 conversion of x * 2^k and its exact way back
    (phl_convert_batch); returns (float32 array, float64 array)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.empty(x.shape, np.float32)
    back = np.empty(x.shape, np.float64)
    _check(lib().phl_convert_batch(x.size, x.ctypes.data, int(k), f.ctypes.data, back.ctypes.data))
    return f, back


def riemann_batch(wl, wr, bn, bg=None, nspec=0, solver="lhlld", mach_thr=0.6, precision="fp64"):
    """Device Riemann solver on n faces (see phl_riemann_batch in include/phl.h)."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    bn = np.ascontiguousarray(bn, dtype=np.float64)
    n = wl.shape[0]
    bg = np.zeros((n, 4)) if bg is None else np.ascontiguousarray(bg, dtype=np.float64)
    f = np.zeros((n, 7 + nspec))
    _check(lib().phl_riemann_batch(n, wl.ctypes.data, wr.ctypes.data, bn.ctypes.data, bg.ctypes.data, nspec,
                                   RIEMANN[solver], float(mach_thr), PRECISION[precision], f.ctypes.data))
    return f


def probe_alu(kind, stream=None):
    """Measured FMA throughput of the current GPU in TFLOP/s: kind "fp32" or
    "fp64" (phl_probe_alu)."""
    v = C.c_double()
    _check(lib().phl_probe_alu({"fp32": 0, "fp64": 1}[kind], C.byref(v), stream))
    return v.value


def cfl_dt_noalloc(grid_or_desc, cons, bx, by, bz, dt_out, stream=None):
    """CFL step without device allocation (phl_cfl_dt_noalloc in include/phl.h).

    For callers that cannot let the library allocate device memory.  All arrays
    are contiguous float64 CUDA tensors in the ABI layout, checked against the
    descriptor's sizes; dt_out is a one-element float64 CUDA tensor.  The call
    is asynchronous on `stream` (a cudaStream_t handle).  dt_out = 0 marks a
    state with rho <= 0, P <= 0 or a non-finite value.
    """
    d = grid_or_desc.desc if isinstance(grid_or_desc, Grid) else grid_or_desc
    nx, ny, nz = d.n[0], d.n[1], d.n[2]
    need = {"cons": (5 + d.nspec) * nx * ny * nz, "bx": (nx + 1) * ny * nz, "by": nx * (ny + 1) * nz,
            "bz": nx * ny * (nz + 1), "dt_out": 1}
    arrs = {"cons": cons, "bx": bx, "by": by, "bz": bz, "dt_out": dt_out}
    for name, a in arrs.items():
        import torch
        ok = isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
        if not ok:
            raise PhlError(1, f"phl_cfl_dt_noalloc: {name} must be a contiguous float64 CUDA tensor")
        if a.numel() < need[name]:
            raise PhlError(1, f"phl_cfl_dt_noalloc: {name} holds {a.numel()} values, the grid needs {need[name]}")
    ptrs = [arrs[k].data_ptr() for k in ("cons", "bx", "by", "bz", "dt_out")]
    _check(lib().phl_cfl_dt_noalloc(C.byref(d), *ptrs, stream))


class EosTable:
    """Stellar EOS table on the current device (phl_eos_table_create)."""

    def __init__(self, lrhoye=(4.0, 8.0), nrho=161, lT=(7.0, 10.0), nT=121):
        h = C.c_void_p()
        _check(lib().phl_eos_table_create(lrhoye[0], lrhoye[1], nrho, lT[0], lT[1], nT, C.byref(h)))
        self.h = h
        self.shape = (nrho, nT)

    def export(self):
        n = 6 + 9 * self.shape[0] * self.shape[1]
        out = np.zeros(n)
        _check(lib().phl_eos_table_export(self.h, out.ctypes.data, n))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().phl_eos_table_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eos(table, rho, eint, abar, ye, T_guess, precision="fp64", tol=1e-11, maxit=50):
    """Batch stellar EOS on host arrays; returns dict of T, P, gamma_e, gamma_c, cs, iters."""
    arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    rho, eint, abar, ye = arr(rho), arr(eint), arr(abar), arr(ye)
    T = arr(T_guess).copy()
    n = rho.size
    out = {k: np.zeros(n) for k in ("P", "gamma_e", "gamma_c", "cs")}
    it = np.zeros(n, dtype=np.int32)
    _check(lib().phl_eos(table.h, n, rho.ctypes.data, eint.ctypes.data, abar.ctypes.data, ye.ctypes.data,
                         T.ctypes.data, out["P"].ctypes.data, out["gamma_e"].ctypes.data,
                         out["gamma_c"].ctypes.data, out["cs"].ctypes.data, it.ctypes.data,
                         PRECISION[precision], tol, maxit, HOST, None))
    out["T"] = T
    out["iters"] = it
    return out


class Mlp:
    """Temperature-guess network on the current device (phl_mlp_* in include/phl.h)."""

    def __init__(self, seed=1):
        h = C.c_void_p()
        _check(lib().phl_mlp_create(int(seed), C.byref(h)))
        self.h = h

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == MLP_NPARAM
        _check(lib().phl_mlp_set_weights(self.h, w.ctypes.data))

    def get_weights(self):
        w = np.zeros(MLP_NPARAM, dtype=np.float32)
        _check(lib().phl_mlp_get_weights(self.h, w.ctypes.data))
        return w

    def set_norm(self, c, s):
        c = np.ascontiguousarray(c, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        _check(lib().phl_mlp_set_norm(self.h, c.ctypes.data, s.ctypes.data))

    def get_norm(self):
        c, s = np.zeros(4), np.zeros(4)
        _check(lib().phl_mlp_get_norm(self.h, c.ctypes.data, s.ctypes.data))
        return c, s

    def loss_grad(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = C.c_double()
        _check(lib().phl_mlp_loss_grad(self.h, t.size, x.ctypes.data, t.ctypes.data, C.byref(loss),
                                       g.ctypes.data, HOST))
        return loss.value, g

    def forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros(x.shape[0], dtype=np.float32)
        _check(lib().phl_mlp_forward(self.h, x.shape[0], x.ctypes.data, y.ctypes.data, HOST))
        return y

    def guess_T(self, table, rho, eint, X0):
        arr = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        rho, eint, X0 = arr(rho), arr(eint), arr(X0)
        T = np.zeros(rho.size)
        _check(lib().phl_mlp_guess_temperature(self.h, table.h, rho.size, rho.ctypes.data, eint.ctypes.data,
                                     X0.ctypes.data, T.ctypes.data, HOST))
        return T

    def train(self, table, nsamples=10_000_000, epochs=8, batch=8192, lr=3e-3, seed=2026,
              lrho=(5.0, 7.0), lT=(8.0, 9.477121254719663), A=(16.0, 28.0), Z=(8.0, 14.0)):
        c = MlpTrainCfg()
        c.nsamples, c.epochs, c.batch, c.lr, c.seed = int(nsamples), int(epochs), int(batch), float(lr), int(seed)
        c.lrho[0], c.lrho[1] = lrho
        c.lT[0], c.lT[1] = lT
        c.A[0], c.A[1] = A
        c.Z[0], c.Z[1] = Z
        st = MlpTrainStats()
        _check(lib().phl_mlp_train(self.h, table.h, C.byref(c), C.byref(st)))
        return {k: getattr(st, k) for k, _ in MlpTrainStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().phl_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(pr, precision="fp64", riemann=None, eps_sf=None, cfl=None, rk=3, wb=True, stream=None,
              mach_thr=None, eos_table=None, newton_tol=1e-11, newton_maxit=50, mlp=None, mlp_mode=2):
    """phl_grid_desc of a problem; returns (desc, arrays the desc points into)."""
    d = GridDesc()
    for k in range(3):
        d.n[k] = pr.n[k]
        d.lo[k] = pr.lo[k]
        d.hi[k] = pr.hi[k]
        d.bc[k][0], d.bc[k][1] = pr.bc[k]
        d.g[k] = pr.g[k]
    d.eos = EOS[pr.eos]
    d.gamma = pr.gamma
    d.nspec = pr.nspec
    if pr.eos == "stellar":
        if eos_table is None:
            raise ValueError("stellar problems need an EosTable")
        d.eos_table = eos_table.h
        for l in range(pr.nspec):
            d.A[l], d.Z[l] = pr.meta["A"][l], pr.meta["Z"][l]
            d.bg_X[l] = pr.meta["bg_X"][l]
    keep = []
    if pr.bg is not None and wb:
        for key in ("rho_c", "p_c", "rho_f", "p_f", "ge_c", "gc_c", "ge_f", "gc_f"):
            if key in pr.bg:
                arr = np.ascontiguousarray(pr.bg[key], dtype=np.float64)
                keep.append(arr)
                setattr(d, "bg_" + key, arr.ctypes.data_as(_dp))
    if pr.heat is not None:
        h = np.ascontiguousarray(pr.heat, dtype=np.float64)
        keep.append(h)
        d.heat = h.ctypes.data_as(_dp)
    d.cfl = pr.cfl if cfl is None else cfl
    d.rk = rk
    d.riemann = RIEMANN[riemann or pr.riemann]
    d.eps_sf = pr.eps_sf if eps_sf is None else eps_sf
    d.mach_thr = pr.mach_thr if mach_thr is None else mach_thr
    d.precision = PRECISION[precision]
    d.newton_tol = newton_tol
    d.newton_maxit = newton_maxit
    d.recon = RECON[getattr(pr, "recon", "vanleer")]
    d.use_mlp = int(mlp_mode) if mlp is not None else 0
    d.mlp = mlp.h if mlp is not None else None
    d.stream = stream
    return d, keep


class TuneEntry(C.Structure):
    _fields_ = [("mode", C.c_int), ("block", C.c_int), ("blocks_per_sm", C.c_int), ("streams", C.c_int),
                ("ms_per_step", C.c_double)]


class EnsembleInfo(C.Structure):
    _fields_ = [("nbox", C.c_int), ("cells", C.c_long), ("mode", C.c_int), ("block", C.c_int),
                ("blocks_per_sm", C.c_int), ("streams", C.c_int), ("graph", C.c_int),
                ("launches_per_step", C.c_int)]


class Ensemble:
    """Independent boxes of uneven sizes stepped together (phl_ensemble_* in
    include/phl.h): one persistent launch per RK stage, graph-captured step."""

    def __init__(self, problems, use_graph=True, stream=None):
        self.problems = list(problems)
        descs = (GridDesc * len(self.problems))()
        self._keep = []
        for i, pr in enumerate(self.problems):
            d, keep = make_desc(pr, precision="mixed", stream=stream)
            descs[i] = d
            self._keep += keep
        h = C.c_void_p()
        _check(lib().phl_ensemble_create(descs, len(self.problems), int(bool(use_graph)), C.byref(h)))
        self.h = h
        self.grids = []
        for i, pr in enumerate(self.problems):
            gh = C.c_void_p()
            _check(lib().phl_ensemble_grid(self.h, i, C.byref(gh)))
            self.grids.append(Grid(pr, _handle=gh))

    def load(self):
        for g in self.grids:
            g.load()

    def step(self, nsteps=1):
        _check(lib().phl_ensemble_step(self.h, int(nsteps)))

    def check(self):
        _check(lib().phl_ensemble_check(self.h))

    def set_shape(self, block=256, blocks_per_sm=0, mode=0, streams=0):
        _check(lib().phl_ensemble_set_shape(self.h, int(mode), int(block), int(blocks_per_sm), int(streams)))

    def autotune(self, trial_steps=2):
        out = (TuneEntry * 64)()
        n = C.c_int()
        _check(lib().phl_ensemble_autotune(self.h, int(trial_steps), out, 64, C.byref(n)))
        return [{"mode": out[i].mode, "block": out[i].block, "blocks_per_sm": out[i].blocks_per_sm,
                 "streams": out[i].streams, "ms_per_step": out[i].ms_per_step} for i in range(min(n.value, 64))]

    def info(self):
        i = EnsembleInfo()
        _check(lib().phl_ensemble_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in EnsembleInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            for g in self.grids:
                g.h = None
            lib().phl_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """One simulation box on the current CUDA device (see include/phl.h)."""

    def __init__(self, pr, precision="fp64", riemann=None, eps_sf=None, cfl=None, rk=3, wb=True,
                 stream=None, mach_thr=None, eos_table=None, newton_tol=1e-11, newton_maxit=50, mlp=None,
                 mlp_mode=2, _handle=None):
        self.pr = pr
        self.eos_table = eos_table
        self.mlp = mlp
        if _handle is not None:          # a box owned by an Ensemble
            self.h, self._owned, self._keep = _handle, False, []
            return
        d, self._keep = make_desc(pr, precision, riemann, eps_sf, cfl, rk, wb, stream, mach_thr, eos_table,
                                  newton_tol, newton_maxit, mlp, mlp_mode)
        self.desc = d
        h = C.c_void_p()
        _check(lib().phl_create_grid(C.byref(d), C.byref(h)))
        self.h = h
        self._owned = True

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib().phl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def set_state(self, cons, bx, by, bz, T=None):
        ptrs = [_ptr(a) for a in (cons, bx, by, bz, T)]
        where = ptrs[0][1]
        _check(lib().phl_set_state(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[4][0], where))

    def set_state_prim(self, prim, bx, by, bz):
        ptrs = [_ptr(a) for a in (prim, bx, by, bz)]
        _check(lib().phl_set_state_prim(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[0][1]))

    def load(self, st=None):
        pr = self.pr
        if st is None and pr.eos == "stellar" and np.isnan(pr.cons[4]).any():
            pm = pr.meta["prim"]
            prim = np.ascontiguousarray(np.concatenate(
                [pm["rho"][None], pm["vel"], pm["p"][None], pm["X"]], axis=0), dtype=np.float64)
            self.set_state_prim(prim, np.ascontiguousarray(pr.bx), np.ascontiguousarray(pr.by),
                                np.ascontiguousarray(pr.bz))
            return
        st = st or dict(cons=pr.cons, bx=pr.bx, by=pr.by, bz=pr.bz, T=pr.T)
        T = st.get("T")
        self.set_state(np.ascontiguousarray(st["cons"]), np.ascontiguousarray(st["bx"]),
                       np.ascontiguousarray(st["by"]), np.ascontiguousarray(st["bz"]),
                       None if T is None else np.ascontiguousarray(T))

    def get_state_into(self, cons, bx, by, bz, T=None):
        ptrs = [_ptr(a) for a in (cons, bx, by, bz, T)]
        _check(lib().phl_get_state(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[4][0], ptrs[0][1]))

    def get_state(self):
        pr = self.pr
        cons = np.empty_like(pr.cons)
        bx, by, bz = np.empty_like(pr.bx), np.empty_like(pr.by), np.empty_like(pr.bz)
        T = np.empty(cons.shape[1:]) if pr.eos == "stellar" else None
        self.get_state_into(cons, bx, by, bz, T)
        return dict(cons=cons, bx=bx, by=by, bz=bz, T=T)

    def get_eos_record(self):
        """The mixed stellar form's inversion record [8][nz][ny][nx]."""
        out = np.zeros((8,) + self.pr.cons.shape[1:])
        _check(lib().phl_get_eos_record(self.h, out.ctypes.data, HOST))
        return out

    def set_eos_record(self, rec):
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        _check(lib().phl_set_eos_record(self.h, rec.ctypes.data, HOST))

    def step(self, nsteps=1, dt=0.0):
        _check(lib().phl_step(self.h, float(dt), int(nsteps)))

    def compute_dt(self):
        v = C.c_double()
        _check(lib().phl_compute_dt(self.h, C.byref(v)))
        return v.value

    def check(self):
        _check(lib().phl_check(self.h))

    def set_stream(self, stream):
        _check(lib().phl_set_stream(self.h, stream))

    def stats(self):
        s = Stats()
        _check(lib().phl_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_timing(self, on=True):
        _check(lib().phl_set_timing(self.h, int(bool(on))))

    def diffuse(self, dt, k0, nT=0, nR=0, cv=1.5, max_stages=100000, precision="grid", tile_z=0, delta_T=False):
        """One RKL2 thermal-diffusion super step of length dt (phl_diffuse);
        precision "grid" (the grid's mode), "fp64" or "mixed"; tile_z: planes
        per CTA of the mixed stage kernel (0: default); returns the number of
        stages."""
        p = Diffusion(k0=float(k0), nT=int(nT), nR=int(nR), cv=float(cv),
                      precision=DIFF_PRECISION[precision], tile_z=int(tile_z), delta_T=int(bool(delta_T)))
        ns = C.c_int(0)
        _check(lib().phl_diffuse(self.h, C.byref(p), float(dt), int(max_stages), C.byref(ns)))
        return ns.value

    def test_tile_wait_timeout(self, on=True):
        """Make the fused tile kernel's bounded TMA wait run out (a test of the
        failure path; see phl_test_tile_wait_timeout)."""
        _check(lib().phl_test_tile_wait_timeout(self.h, int(bool(on))))

    def test_prims(self, form, increments=True):
        """The mixed stage's primitive deviations of the whole work box in one
        form (phl_test_prims): returns (W and auxiliary planes as float32,
        the CFL rate for forms 2 and 3)."""
        n = C.c_long(0)
        _check(lib().phl_test_prims_size(self.h, C.byref(n)))
        out = np.zeros(n.value, dtype=np.float32)
        rate = C.c_float(0.0)
        _check(lib().phl_test_prims(self.h, int(form), int(bool(increments)), out.ctypes.data, n.value,
                                    C.byref(rate)))
        return out, rate.value

    def test_raw_flags(self, form):
        """Raw shock flags of the W the last test_prims formed, in one form
        (phl_test_raw_flags): returns (flags as uint8 (nz, ny, nx), the vote)."""
        nx, ny, nz = self.pr.n
        out = np.zeros((nz, ny, nx), dtype=np.uint8)
        anyf = C.c_int(0)
        _check(lib().phl_test_raw_flags(self.h, int(form), out.ctypes.data, out.size, C.byref(anyf)))
        return out, anyf.value

    def set_fused(self, on=1):
        """Mixed-precision stage decomposition (phl_set_fused): 0/False = one
        face kernel per direction, 1/True = the fused tile kernel in its
        default launch shape (six launches per stage), 2..9 = other launch
        shapes of it, 201..209 = shapes 1..9 with the stage in three launches."""
        _check(lib().phl_set_fused(self.h, int(on)))

    def kernel_times(self, reset=True):
        """{kernel class: (launches, total ms)} since the last reset (synchronises)."""
        arr = (KernelTime * 32)()
        n = C.c_int()
        _check(lib().phl_kernel_times(self.h, arr, 32, C.byref(n), int(bool(reset))))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(min(n.value, 32))}

    def dt_device_ptr(self):
        p = C.c_void_p()
        _check(lib().phl_dt_device_ptr(self.h, C.byref(p)))
        return p.value


class PoissonDesc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("xf", C.c_void_p * 3), ("G", C.c_double), ("lmax", C.c_int),
                ("criterion", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("stream", C.c_void_p)]


POISSON_CRITERION = {"relative": 0, "absolute": 1}


class Poisson:
    """The device Poisson solver (phl_poisson_*, Sect. 2.12) on a grid given
    by its face coordinates xf = (xf_x, xf_y, xf_z).  Cell arrays are
    [nz][ny][nx] numpy float64 (host) or CUDA tensors (device)."""

    def __init__(self, xf, G=1.0, lmax=0, criterion="relative", tol=1e-4, max_iter=10000, stream=None):
        self._xf = [np.ascontiguousarray(a, dtype=np.float64) for a in xf]
        self.n = tuple(len(a) - 1 for a in self._xf)
        d = PoissonDesc()
        for a in range(3):
            d.n[a] = self.n[a]
            d.xf[a] = self._xf[a].ctypes.data
        d.G, d.lmax, d.criterion = float(G), int(lmax), POISSON_CRITERION[criterion]
        d.tol, d.max_iter, d.stream = float(tol), int(max_iter), stream
        h = C.c_void_p()
        _check(lib().phl_poisson_create(C.byref(d), C.byref(h)))
        self.h = h
        nx, ny, nz = self.n
        self.nghost = 2 * (ny * nz + nx * nz + nx * ny)

    def solve(self, rho, phi=None):
        """Returns (phi, iterations, residual); phi (optional) is the initial
        guess and, as an array of the same kind as rho, receives the result."""
        if phi is None:
            phi = np.zeros(self.n[::-1]) if isinstance(rho, np.ndarray) else rho.new_zeros(rho.shape)
        pr, wr = _ptr(rho)
        pp, wp = _ptr(phi)
        assert wr == wp, "rho and phi must live in the same memory"
        it, res = C.c_int(), C.c_double()
        _check(lib().phl_poisson_solve(self.h, pr, pp, wr, C.byref(it), C.byref(res)))
        return phi, it.value, res.value

    def ghost(self):
        g = np.zeros(self.nghost)
        _check(lib().phl_poisson_ghost(self.h, g.ctypes.data, HOST))
        return g

    def gravity(self, phi):
        if isinstance(phi, np.ndarray):
            g = [np.zeros(self.n[::-1]) for _ in range(3)]
        else:
            g = [phi.new_zeros(phi.shape) for _ in range(3)]
        pp, w = _ptr(phi)
        _check(lib().phl_poisson_gravity(self.h, pp, _ptr(g[0])[0], _ptr(g[1])[0], _ptr(g[2])[0], w))
        return g

    def close(self):
        if self.h:
            lib().phl_poisson_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SphereDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("Nr", C.c_int), ("r_in", C.c_double), ("r_out", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double), ("riemann", C.c_int), ("mach_thr", C.c_double),
                ("precision", C.c_int), ("rho_c", C.c_void_p), ("p_c", C.c_void_p), ("rho_f", C.c_void_p), ("p_f", C.c_void_p),
                ("g_c", C.c_void_p), ("heat", C.c_void_p), ("stream", C.c_void_p),
                ("eos", C.c_int), ("eos_table", C.c_void_p), ("nspec", C.c_int),
                ("A", C.c_double * 4), ("Z", C.c_double * 4), ("X", C.c_double * 4),
                ("rho_unit", C.c_double), ("p_unit", C.c_double), ("newton_tol", C.c_double),
                ("newton_maxit", C.c_int), ("mlp", C.c_void_p)]


class Sphere:
    """MHD on a cubed-sphere shell (phl_sphere_*): six equiangular patches of
    N x N angular cells times Nr radial cells, FP64 on the device.  The state
    is cons [5][6][Nr][N][N] and the face fluxes pa [6][Nr][N][N+1],
    pb [6][Nr][N+1][N], pr [6][Nr+1][N][N], as numpy float64 arrays (host)
    or CUDA tensors (device).  `bg` holds rho_c, p_c (Nr) and rho_f, p_f
    (Nr + 1), or is None for full-state fluxes.  `stellar` (a dict of
    eos_table, A, Z, X, rho_u, p_u, and optionally mlp, newton_tol) selects
    the stellar EOS with a uniform composition."""

    def __init__(self, N, Nr, r_in, r_out, gamma=5.0 / 3.0, cfl=0.4, riemann="lhlld", mach_thr=0.6, bg=None,
                 g_c=None, heat=None, stream=None, precision="fp64", stellar=None):
        self.N, self.Nr = int(N), int(Nr)
        keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data
        d = SphereDesc()
        d.N, d.Nr, d.r_in, d.r_out = self.N, self.Nr, float(r_in), float(r_out)
        d.gamma, d.cfl, d.riemann, d.mach_thr = float(gamma), float(cfl), RIEMANN[riemann], float(mach_thr)
        d.precision = PRECISION[precision]
        if bg is not None:
            d.rho_c, d.p_c, d.rho_f, d.p_f = (arr(bg[k]) for k in ("rho_c", "p_c", "rho_f", "p_f"))
        d.g_c, d.heat, d.stream = arr(g_c), arr(heat), stream
        self.stellar = stellar is not None
        if self.stellar:
            d.eos, d.eos_table = 1, stellar["eos_table"].h
            d.nspec = len(stellar["A"])
            for l in range(d.nspec):
                d.A[l], d.Z[l], d.X[l] = stellar["A"][l], stellar["Z"][l], stellar["X"][l]
            d.rho_unit, d.p_unit = float(stellar["rho_u"]), float(stellar["p_u"])
            d.newton_tol = float(stellar.get("newton_tol", 1e-11))
            d.newton_maxit = int(stellar.get("newton_maxit", 50))
            m = stellar.get("mlp")
            d.mlp = m.h if m is not None else None
            self._stellar_refs = (stellar["eos_table"], m)   # the handles must outlive the shell
        h = C.c_void_p()
        _check(lib().phl_sphere_create(C.byref(d), C.byref(h)))
        self.h = h

    @classmethod
    def from_problem(cls, pr, wb=True, stream=None, precision="fp64", eos_table=None, mlp=None):
        """From a workloads.ShellProblem (its solver, CFL, background, gravity
        and heating); wb=False drops the background.  A stellar problem needs
        an EosTable (and takes an optional Mlp for cold starts)."""
        stellar = None
        if pr.meta.get("eos") == "stellar":
            if eos_table is None:
                raise ValueError("a stellar shell needs an EosTable")
            stellar = dict(eos_table=eos_table, A=pr.meta["A"], Z=pr.meta["Z"], X=pr.meta["X"],
                           rho_u=pr.meta["rho_u"], p_u=pr.meta["p_u"], mlp=mlp)
        return cls(pr.N, pr.Nr, pr.r_in, pr.r_out, gamma=pr.gamma, cfl=pr.cfl, riemann=pr.riemann,
                   mach_thr=pr.mach_thr, bg=pr.bg if wb else None, g_c=pr.g_c, heat=pr.heat, stream=stream,
                   precision=precision, stellar=stellar)

    def load(self, pr):
        """The problem's initial state: set_state, or for a stellar problem
        (given in primitives) set_prims."""
        if pr.meta.get("eos") == "stellar":
            p = pr.meta["prim"]
            self.set_prims(p["rho"], p["vel"], p["p"], pr.pa, pr.pb, pr.pr)
        else:
            self.set_state(pr.cons, pr.pa, pr.pb, pr.pr)

    def shapes(self):
        N, Nr = self.N, self.Nr
        return dict(cons=(5, 6, Nr, N, N), pa=(6, Nr, N, N + 1), pb=(6, Nr, N + 1, N), pr=(6, Nr + 1, N, N))

    def counts(self):
        c, f, e = C.c_long(), C.c_long(), C.c_long()
        _check(lib().phl_sphere_counts(self.h, C.byref(c), C.byref(f), C.byref(e)))
        return dict(cells=c.value, faces=f.value, edges=e.value)

    def set_state(self, cons, pa, pb, pr):
        ptrs = [_ptr(a) for a in (cons, pa, pb, pr)]
        for (a, (p, w)), (k, shp) in zip(zip((cons, pa, pb, pr), ptrs), self.shapes().items()):
            assert tuple(a.shape) == shp, (k, tuple(a.shape), shp)
        assert len({w for _, w in ptrs}) == 1, "all state arrays must live in the same memory"
        _check(lib().phl_sphere_set_state(self.h, *[p for p, _ in ptrs], ptrs[0][1]))

    def set_prims(self, rho, vel, P, pa, pb, pr):
        """rho, P [6][Nr][N][N], vel [6][Nr][N][N][3] (code units) and the fluxes."""
        N, Nr = self.N, self.Nr
        arrs = (rho, vel, P, pa, pb, pr)
        shp = [(6, Nr, N, N), (6, Nr, N, N, 3), (6, Nr, N, N)] + [self.shapes()[k] for k in ("pa", "pb", "pr")]
        for a, s_ in zip(arrs, shp):
            assert tuple(a.shape) == s_, (tuple(a.shape), s_)
        ptrs = [_ptr(a) for a in arrs]
        assert len({w for _, w in ptrs}) == 1, "all arrays must live in the same memory"
        _check(lib().phl_sphere_set_prims(self.h, *[p for p, _ in ptrs], ptrs[0][1]))

    def set_temperature(self, T):
        p, w = _ptr(T)
        _check(lib().phl_sphere_set_temperature(self.h, p, w))

    def get_eos_record(self):
        """The mixed stellar shell's inversion record [8][6][Nr][N][N]."""
        out = np.zeros((8, 6, self.Nr, self.N, self.N))
        _check(lib().phl_sphere_get_eos_record(self.h, out.ctypes.data, HOST))
        return out

    def set_eos_record(self, rec):
        p, w = _ptr(np.ascontiguousarray(rec, dtype=np.float64) if isinstance(rec, np.ndarray) else rec)
        _check(lib().phl_sphere_set_eos_record(self.h, p, w))

    def get_temperature(self, out=None):
        """Cell temperatures [6][Nr][N][N] (K) of a stellar shell."""
        if out is None:
            out = np.zeros((6, self.Nr, self.N, self.N))
        p, w = _ptr(out)
        _check(lib().phl_sphere_get_temperature(self.h, p, w))
        return out

    def get_state(self, out=None):
        """Returns dict(cons, pa, pb, pr); `out` (a dict of arrays or tensors of
        the right shapes) receives them instead of new numpy arrays."""
        if out is None:
            out = {k: np.zeros(s) for k, s in self.shapes().items()}
        ptrs = [_ptr(out[k]) for k in ("cons", "pa", "pb", "pr")]
        _check(lib().phl_sphere_get_state(self.h, *[p for p, _ in ptrs], ptrs[0][1]))
        return out

    def step(self, nsteps=1, dt=0.0):
        _check(lib().phl_sphere_step(self.h, float(dt), int(nsteps)))

    def compute_dt(self):
        v = C.c_double()
        _check(lib().phl_sphere_compute_dt(self.h, C.byref(v)))
        return v.value

    def check(self):
        _check(lib().phl_sphere_check(self.h))

    def set_graph(self, on=True):
        """Replay each step as one captured CUDA graph (needs a stream)."""
        _check(lib().phl_sphere_set_graph(self.h, int(bool(on))))

    def set_timing(self, on=True):
        _check(lib().phl_sphere_set_timing(self.h, int(bool(on))))

    def kernel_times(self, reset=True):
        """{kernel class: (launches, summed ms)} since the last reset."""
        arr = (KernelTime * 32)()
        n = C.c_int()
        _check(lib().phl_sphere_kernel_times(self.h, arr, 32, C.byref(n), int(bool(reset))))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].ms) for i in range(min(n.value, 32))}

    def close(self):
        if self.h:
            lib().phl_sphere_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
