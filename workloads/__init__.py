"""Seeded synthetic workloads for the explicit MHD stage.

This module builds problem descriptions and initial data: grid sizes, boundary
conditions, gravity, the hydrostatic background profiles, and the conserved
state (rho, rho*u, rho*e, rho*X_l) plus the face-centred normal magnetic field.
It is the one module that both the CUDA path's tests/benchmarks and the CPU
oracle consume. It holds none of the scheme's arithmetic: no reconstruction, no
Riemann flux, no constrained transport, no EOS inversion. Conserved energy is
assembled from the primitive initial data with the definition of the total
energy density (Sect. 2.1, below Eq. energy), using the face-average cell field.

Array layout (the library's ABI layout, x fastest, no ghost cells):
  cons[v, k, j, i]   v = rho, mx, my, mz, E, rho*X_0, ...      shape (nv, nz, ny, nx)
  bx[k, j, i]        normal B on x-faces i-1/2, i = 0..nx          (nz, ny, nx+1)
  by[k, j, i]        normal B on y-faces j-1/2, j = 0..ny          (nz, ny+1, nx)
  bz[k, j, i]        normal B on z-faces k-1/2, k = 0..nz          (nz+1, ny, nx)
Inactive dimensions have one cell; their face arrays hold 2 equal layers.

Background profiles (well-balanced deviation method, Sect. 2.8) vary along z
only and are given with 3 ghost layers on each side:
  rho_c, p_c : cell centres k = -3 .. nz+2          (length nz+6, index k+3)
  rho_f, p_f : z-faces k-1/2, k = -3 .. nz+3        (length nz+7, index k+3)
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

PERIODIC, REFLECT, OUTFLOW = 0, 1, 2
NG_BG = 3  # ghost layers carried by background profiles


@dataclasses.dataclass
class Problem:
    name: str
    ndim: int
    n: tuple                      # (nx, ny, nz)
    lo: tuple
    hi: tuple
    bc: tuple                     # ((xlo, xhi), (ylo, yhi), (zlo, zhi))
    gamma: float
    cons: np.ndarray
    bx: np.ndarray
    by: np.ndarray
    bz: np.ndarray
    g: tuple = (0.0, 0.0, 0.0)
    bg: Optional[dict] = None     # rho_c, p_c, rho_f, p_f (see module doc)
    heat: Optional[np.ndarray] = None   # volumetric heating rate per z-cell (nz,)
    cfl: float = 0.4
    riemann: str = "lhlld"        # lhlld | hlld | hll
    recon: str = "vanleer"        # vanleer (limited linear) | pph (third-order parabolic)
    eps_sf: float = 0.2           # shock-flattening threshold; 0 switches it off
    mach_thr: float = 0.6
    nspec: int = 0
    eos: str = "ideal"
    T: Optional[np.ndarray] = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nv(self) -> int:
        return 5 + self.nspec

    @property
    def ncells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    def copy(self) -> "Problem":
        p = dataclasses.replace(self)
        p.cons = self.cons.copy()
        p.bx, p.by, p.bz = self.bx.copy(), self.by.copy(), self.bz.copy()
        p.T = None if self.T is None else self.T.copy()
        return p

    def dx(self):
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def _centres(lo, hi, n):
    d = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * d


def _faces(lo, hi, n):
    d = (hi - lo) / n
    return lo + np.arange(n + 1) * d


def _assemble(name, ndim, n, lo, hi, bc, gamma, rho, vel, p, bx, by, bz, **kw):
    """Build conserved variables from point values of the primitive fields.

    rho, p and vel[3] are cell-centred arrays of shape (nz, ny, nx); the cell
    magnetic field is the mean of the two face values (used only to form E).
    """
    nx, ny, nz = n
    bcx = 0.5 * (bx[:, :, :-1] + bx[:, :, 1:])
    bcy = 0.5 * (by[:, :-1, :] + by[:, 1:, :])
    bcz = 0.5 * (bz[:-1, :, :] + bz[1:, :, :])
    nspec = kw.get("nspec", 0)
    cons = np.zeros((5 + nspec, nz, ny, nx))
    cons[0] = rho
    for d in range(3):
        cons[1 + d] = rho * vel[d]
    kin = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    mag = 0.5 * (bcx ** 2 + bcy ** 2 + bcz ** 2)
    if "eint_density" in kw:
        cons[4] = kw.pop("eint_density") + kin + mag
    else:
        cons[4] = p / (gamma - 1.0) + kin + mag
    if nspec:
        X = kw.pop("X")
        for l in range(nspec):
            cons[5 + l] = rho * X[l]
    kw.pop("nspec", None)
    return Problem(name=name, ndim=ndim, n=tuple(n), lo=tuple(lo), hi=tuple(hi),
                   bc=tuple(tuple(b) for b in bc), gamma=gamma, cons=cons,
                   bx=bx, by=by, bz=bz, nspec=nspec, **kw)


def _faces_from_az(az_corner, dx, dy, nz):
    """Face normal fields of B = curl(A_z z^) from A_z at cell corners.

    az_corner[j, i] is A_z at (x_{i-1/2}, y_{j-1/2}), shape (ny+1, nx+1).
    Discrete curl: divergence-free to round-off by construction.
    """
    bx2 = (az_corner[1:, :] - az_corner[:-1, :]) / dy          # (ny, nx+1)
    by2 = -(az_corner[:, 1:] - az_corner[:, :-1]) / dx         # (ny+1, nx)
    bx = np.repeat(bx2[None], nz, axis=0)
    by = np.repeat(by2[None], nz, axis=0)
    return bx, by


# ----------------------------------------------------------------------------
# 1D problems
# ----------------------------------------------------------------------------

def shock_tube(n, left, right, gamma, bxn=0.0, x0=0.5, name="tube", cfl=0.4, **kw):
    """1D Riemann problem on x in [0,1]; left/right = (rho, vx, vy, vz, By, Bz, P)."""
    x = _centres(0.0, 1.0, n)
    sel = x < x0
    st = np.where(sel[None, :], np.array(left)[:, None], np.array(right)[:, None])
    rho, vx, vy, vz, byc, bzc, p = st
    shp = (1, 1, n)
    bx = np.full((1, 1, n + 1), float(bxn))
    by = np.repeat(byc.reshape(shp), 2, axis=1)
    bz = np.repeat(bzc.reshape(shp), 2, axis=0)
    return _assemble(name, 1, (n, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0),
                     ((OUTFLOW, OUTFLOW), (PERIODIC, PERIODIC), (PERIODIC, PERIODIC)),
                     gamma, rho.reshape(shp), [vx.reshape(shp), vy.reshape(shp), vz.reshape(shp)],
                     p.reshape(shp), bx, by, bz, cfl=cfl, **kw)


def sod(n, **kw):
    """Sod tube: (rho, p) = (1, 1) | (0.125, 0.1), gamma = 1.4, B = 0."""
    return shock_tube(n, (1.0, 0, 0, 0, 0, 0, 1.0), (0.125, 0, 0, 0, 0, 0, 0.1), 1.4,
                      name=f"sod{n}", **kw)


def brio_wu(n, **kw):
    """Brio-Wu tube (Sect. 3.1): gamma = 2, Bx = 0.75, By = +1 | -1."""
    return shock_tube(n, (1.0, 0, 0, 0, 1.0, 0, 1.0), (0.125, 0, 0, 0, -1.0, 0, 0.1), 2.0,
                      bxn=0.75, name=f"briowu{n}", **kw)


def alfven_1d(n, amp=1e-6, rho0=1.0, p0=0.1, b0=1.0, gamma=5.0 / 3.0, cfl=0.4):
    """Right-going linear Alfven wave along x, periodic on [0,1]: dB_y = -sqrt(rho) dv_y."""
    x = _centres(0.0, 1.0, n)
    xf = _faces(0.0, 1.0, n)
    shp = (1, 1, n)
    vy = amp * np.sin(2 * np.pi * x)
    rho = np.full(shp, rho0)
    p = np.full(shp, p0)
    bx = np.full((1, 1, n + 1), b0)
    byc = -math.sqrt(rho0) * vy
    by = np.repeat(byc.reshape(shp), 2, axis=1)
    bz = np.zeros((2, 1, n))
    pr = _assemble(f"alfven1d_{n}", 1, (n, 1, 1), (0, 0, 0), (1, 1, 1),
                   ((PERIODIC,) * 2,) * 3, gamma, rho, [np.zeros(shp), vy.reshape(shp), np.zeros(shp)],
                   p, bx, by, bz, cfl=cfl)
    pr.meta.update(period=1.0 / (b0 / math.sqrt(rho0)), amp=amp, xf=xf)
    return pr


# ----------------------------------------------------------------------------
# 2D problems
# ----------------------------------------------------------------------------

def orszag_tang(n, cfl=0.4, **kw):
    """Orszag-Tang vortex on [0,1]^2, gamma = 5/3 (configuration C1)."""
    gamma = 5.0 / 3.0
    dx = 1.0 / n
    x = _centres(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")          # [j, i]
    b0 = 1.0 / math.sqrt(4 * math.pi)
    xf = _faces(0.0, 1.0, n)
    XF, YF = np.meshgrid(xf, xf, indexing="xy")
    az = b0 * (np.cos(4 * np.pi * XF) / (4 * np.pi) + np.cos(2 * np.pi * YF) / (2 * np.pi))
    bx, by = _faces_from_az(az, dx, dx, 1)
    bz = np.zeros((2, n, n))
    rho = np.full((1, n, n), 25.0 / (36.0 * math.pi))
    p = np.full((1, n, n), 5.0 / (12.0 * math.pi))
    vx = (-np.sin(2 * np.pi * Y))[None]
    vy = (np.sin(2 * np.pi * X))[None]
    return _assemble(f"orszag_tang{n}", 2, (n, n, 1), (0, 0, 0), (1, 1, 1),
                     ((PERIODIC,) * 2,) * 3, gamma, rho, [vx, vy, np.zeros_like(vx)], p,
                     bx, by, bz, cfl=cfl, **kw)


def alfven_2d(n, amp=1e-6, cfl=0.4):
    """Linear Alfven wave along the diagonal of the periodic unit square.

    B0 = (1,1)/sqrt(2) (|B0| = 1), rho = 1, P = 0.1, gamma = 5/3; in-plane
    perturbation along (-1,1)/sqrt(2); wavelength 1/sqrt(2), period 1/sqrt(2).
    """
    gamma = 5.0 / 3.0
    dx = 1.0 / n
    x = _centres(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    xf = _faces(0.0, 1.0, n)
    XF, YF = np.meshgrid(xf, xf, indexing="xy")
    b = 1.0 / math.sqrt(2.0)
    az = b * (YF - XF) + amp * np.cos(2 * np.pi * (XF + YF)) / (2 * math.sqrt(2) * np.pi)
    bx, by = _faces_from_az(az, dx, dx, 1)
    bz = np.zeros((2, n, n))
    ph = 2 * np.pi * (X + Y)
    dbx = -amp / math.sqrt(2) * np.sin(ph)
    dby = amp / math.sqrt(2) * np.sin(ph)
    vx, vy = -dbx, -dby
    rho = np.ones((1, n, n))
    p = np.full((1, n, n), 0.1)
    pr = _assemble(f"alfven2d_{n}", 2, (n, n, 1), (0, 0, 0), (1, 1, 1),
                   ((PERIODIC,) * 2,) * 3, gamma, rho, [vx[None], vy[None], np.zeros((1, n, n))],
                   p, bx, by, bz, cfl=cfl)
    pr.meta.update(period=1.0 / math.sqrt(2.0), amp=amp)
    return pr


def balsara_vortex(n, u_tilde, beta_k, cfl=0.8, **kw):
    """Balsara (2004) MHD vortex on (-5,5)^2 advected along the diagonal (Sect. 3.2)."""
    gamma = 5.0 / 3.0
    dx = 10.0 / n
    x = _centres(-5.0, 5.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    xf = _faces(-5.0, 5.0, n)
    XF, YF = np.meshgrid(xf, xf, indexing="xy")
    b_tilde = u_tilde * math.sqrt(beta_k)
    az = b_tilde * np.exp(0.5 * (1.0 - (XF ** 2 + YF ** 2)))
    bx, by = _faces_from_az(az, dx, dx, 1)
    bz = np.zeros((2, n, n))
    r2 = X ** 2 + Y ** 2
    f = np.exp(0.5 * (1.0 - r2))
    vx = -u_tilde * f * Y + u_tilde / math.sqrt(2.0)
    vy = u_tilde * f * X + u_tilde / math.sqrt(2.0)
    p = 1.0 + (0.5 * b_tilde ** 2 * (1.0 - r2) - 0.5 * u_tilde ** 2) * np.exp(1.0 - r2)
    rho = np.ones((1, n, n))
    pr = _assemble(f"balsara{n}", 2, (n, n, 1), (-5, -5, 0), (5, 5, 1),
                   ((PERIODIC,) * 2,) * 3, gamma, rho, [vx[None], vy[None], np.zeros((1, n, n))],
                   p[None], bx, by, bz, cfl=cfl, **kw)
    pr.meta.update(tau=10.0 * math.sqrt(2.0) / u_tilde, b_tilde=b_tilde)
    return pr


# ----------------------------------------------------------------------------
# stratified 3D boxes (configurations C2 / C4)
# ----------------------------------------------------------------------------

def polytrope_profile(z, n_poly=1.5, g0=1.0, rho_b=1.0, rho_top=0.1, ztop=1.0):
    """Hydrostatic polytrope P = K rho^(1+1/n) under constant downward g0.

    rho^(1/n)(z) = rho_b^(1/n) - g0 z / (K (n+1)); K fixed by rho(ztop) = rho_top.
    """
    K = g0 * ztop / ((n_poly + 1.0) * (rho_b ** (1.0 / n_poly) - rho_top ** (1.0 / n_poly)))
    # beyond the polytrope's surface (z > 1.27 for the defaults: only the
    # top ghost layers of boxes with nz < 12 reach it) density and pressure
    # are zero
    base = np.maximum(rho_b ** (1.0 / n_poly) - g0 * z / (K * (n_poly + 1.0)), 0.0)
    rho = base ** n_poly
    return rho, K * rho ** (1.0 + 1.0 / n_poly), K


def background_profiles(nz, lo, hi, fn):
    dz = (hi - lo) / nz
    zc = lo + (np.arange(-NG_BG, nz + NG_BG) + 0.5) * dz
    zf = lo + np.arange(-NG_BG, nz + NG_BG + 1) * dz
    rc, pc = fn(zc)[:2]
    rf, pf = fn(zf)[:2]
    return dict(rho_c=np.ascontiguousarray(rc), p_c=np.ascontiguousarray(pc),
                rho_f=np.ascontiguousarray(rf), p_f=np.ascontiguousarray(pf))


def stratified_box(nx, ny, nz, seed=1234, amp=1e-3, beta=1e6, mach_heat=1e-3,
                   n_poly=1.5, rho_top=0.1, cfl=0.4, gamma=5.0 / 3.0, heat=True,
                   name=None, **kw):
    """3D stratified low-Mach magnetoconvection box (configuration C2 shape).

    Domain [0,1]^3, g = (0,0,-1), polytrope n = 1.5 with rho(0) = 1, rho(1) = 0.1,
    isobaric density noise rho = rho_hat (1 + amp U(-1,1)) from numpy PCG64(seed),
    uniform B_x with plasma beta 2 P_hat(1/2) / B^2 = beta, uniform heating in
    z < 0.1 sized so (q * 0.1 / rho_b)^(1/3) = mach_heat * c_s(z=0).
    Periodic x, y; reflecting z.
    """
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    fn = lambda z: polytrope_profile(z, n_poly=n_poly, rho_top=rho_top)
    bg = background_profiles(nz, 0.0, 1.0, fn)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    rho_c = bg["rho_c"][NG_BG:NG_BG + nz][:, None, None]
    p_c = bg["p_c"][NG_BG:NG_BG + nz][:, None, None]
    rho = rho_c * (1.0 + amp * noise)
    p = np.broadcast_to(p_c, (nz, ny, nx)).copy()
    _, p_mid, _ = fn(np.array([0.5]))
    b0 = math.sqrt(2.0 * float(p_mid[0]) / beta)
    bx = np.full((nz, ny, nx + 1), b0)
    by = np.zeros((nz, ny + 1, nx))
    bz = np.zeros((nz + 1, ny, nx))
    zero = np.zeros((nz, ny, nx))
    q = None
    if heat:
        cs_b = math.sqrt(gamma * float(fn(np.array([0.0]))[1][0]) / 1.0)
        qv = (mach_heat * cs_b) ** 3 * 1.0 / 0.1
        zc = (np.arange(nz) + 0.5) / nz
        q = np.where(zc < 0.1, qv, 0.0)
    pr = _assemble(name or f"box{nx}x{ny}x{nz}", 3, (nx, ny, nz), lo, hi,
                   ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (REFLECT, REFLECT)),
                   gamma, rho, [zero, zero, zero], p, bx, by, bz,
                   g=(0.0, 0.0, -1.0), bg=bg, heat=q, cfl=cfl, **kw)
    pr.meta.update(seed=seed, amp=amp, beta=beta, b0=b0)
    return pr


def isothermal_atmosphere(nx, nz, c2=1.0, g0=1.0, ndim=2, cfl=0.4, b0=0.0):
    """Isothermal hydrostatic atmosphere rho = exp(-g0 z / c2), P = c2 rho, at rest.

    2D (x, z-like second axis mapped to z via a 3D grid with ny = 1) would need
    z active; here the box is (nx, 1, nz) with x periodic and z reflecting.
    """
    fn = lambda z: (np.exp(-g0 * z / c2), c2 * np.exp(-g0 * z / c2))
    bg = background_profiles(nz, 0.0, 1.0, fn)
    rho = np.broadcast_to(bg["rho_c"][NG_BG:NG_BG + nz][:, None, None], (nz, 1, nx)).copy()
    p = c2 * rho
    bx = np.full((nz, 1, nx + 1), b0)
    by = np.zeros((nz, 2, nx))
    bz = np.zeros((nz + 1, 1, nx))
    zero = np.zeros((nz, 1, nx))
    return _assemble(f"isothermal{nx}x{nz}", 3, (nx, 1, nz), (0, 0, 0), (1, 1, 1),
                     ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (REFLECT, REFLECT)),
                     1.4, rho, [zero, zero, zero], p, bx, by, bz,
                     g=(0.0, 0.0, -g0), bg=bg, cfl=cfl)


# Stellar box (configuration C3 shape): CGS units, O/Si mixture.
STELLAR_A = (16.0, 28.0)
STELLAR_Z = (8.0, 14.0)
STELLAR_X = (0.5, 0.5)
# Base pressure of the polytrope: close to the stellar EOS at rho = 1e7 g/cc,
# T = 3e9 K for this mixture (ions + radiation + e-/e+ = 1.8e24 dyn/cm^2).
STELLAR_P_BASE = 1.8e24
STELLAR_RHO_BASE = 1.0e7
STELLAR_RHO_TOP = 1.0e5
STELLAR_L = 1.0e8          # box edge, cm


def stellar_box(nx, ny, nz, seed=1234, amp=1e-3, beta=1e6, mach_heat=1e-3, cfl=0.4, heat=True, name=None,
                vel_amp=0.0):
    """3D stratified box with the stellar EOS (configuration C3 shape).

    Given as primitive fields: the conserved energy and the temperature
    depend on the equation of state, so each implementation builds them from
    (rho, P, v, X, B) with its own EOS.  Background: n = 1.5 polytrope
    P = K rho^(5/3) under constant g from rho = 1e7 g/cc at z = 0, reaching
    1e5 g/cc at z = L (1 + 4/nz), K = P_base / rho_base^(5/3).  Isobaric density noise amp * U(-1, 1) from
    PCG64(seed); X(16O) = X(28Si) = 0.5; uniform B_x with beta = 2 P_hat(L/2)/B^2.
    vel_amp > 0 adds velocities vel_amp * c_s0 * U(-1, 1) per component (drawn
    after the density noise), c_s0 = sqrt(5/3 P_base / rho_base).
    """
    n_poly = 1.5
    K = STELLAR_P_BASE / STELLAR_RHO_BASE ** (1.0 + 1.0 / n_poly)
    # rho = rho_top is reached at z = L (1 + 4/nz), so the three ghost layers
    # above the box keep rho inside [rho_top, rho_base]
    z_end = STELLAR_L * (1.0 + 4.0 / nz)
    g0 = K * (n_poly + 1.0) * (STELLAR_RHO_BASE ** (1.0 / n_poly) - STELLAR_RHO_TOP ** (1.0 / n_poly)) / z_end

    def fn(z):
        base = STELLAR_RHO_BASE ** (1.0 / n_poly) - g0 * z / (K * (n_poly + 1.0))
        rho = base ** n_poly
        return rho, K * rho ** (1.0 + 1.0 / n_poly)

    L = STELLAR_L
    bg = background_profiles(nz, 0.0, L, fn)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    rho_c = bg["rho_c"][NG_BG:NG_BG + nz][:, None, None]
    p_c = bg["p_c"][NG_BG:NG_BG + nz][:, None, None]
    rho = rho_c * (1.0 + amp * noise)
    p = np.broadcast_to(p_c, (nz, ny, nx)).copy()
    _, p_mid = fn(np.array([0.5 * L]))
    b0 = math.sqrt(2.0 * float(p_mid[0]) / beta)
    bx = np.full((nz, ny, nx + 1), b0)
    by = np.zeros((nz, ny + 1, nx))
    bz = np.zeros((nz + 1, ny, nx))
    q = None
    if heat:
        cs_b = math.sqrt(1.4 * STELLAR_P_BASE / STELLAR_RHO_BASE)
        qv = (mach_heat * cs_b) ** 3 * STELLAR_RHO_BASE / (0.1 * L)
        zc = (np.arange(nz) + 0.5) / nz
        q = np.where(zc < 0.1, qv, 0.0)
    nspec = 2
    cons = np.full((5 + nspec, nz, ny, nx), np.nan)
    cons[0] = rho
    cons[1:4] = 0.0
    for l in range(nspec):
        cons[5 + l] = rho * STELLAR_X[l]
    vel = np.zeros((3, nz, ny, nx))
    if vel_amp > 0.0:
        cs0 = math.sqrt(5.0 / 3.0 * STELLAR_P_BASE / STELLAR_RHO_BASE)
        vel = vel_amp * cs0 * rng.uniform(-1.0, 1.0, size=(3, nz, ny, nx))
        cons[1:4] = rho * vel
    prim = dict(rho=rho, vel=vel, p=p,
                X=np.stack([np.full((nz, ny, nx), x) for x in STELLAR_X]))
    pr = Problem(name=name or f"stellar{nx}x{ny}x{nz}", ndim=3, n=(nx, ny, nz), lo=(0.0, 0.0, 0.0),
                 hi=(L, L, L), bc=((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (REFLECT, REFLECT)),
                 gamma=5.0 / 3.0, cons=cons, bx=bx, by=by, bz=bz, g=(0.0, 0.0, -g0), bg=bg, heat=q, cfl=cfl,
                 nspec=nspec, eos="stellar")
    pr.meta.update(seed=seed, amp=amp, beta=beta, b0=b0, A=list(STELLAR_A), Z=list(STELLAR_Z),
                   X=list(STELLAR_X), prim=prim, bg_X=list(STELLAR_X))
    return pr


def ensemble_dims(nbox=24, seed=2024, choices=(64, 96, 128, 160, 192)):
    """Box edge lengths of the batched ensemble (configuration C4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [tuple(int(c) for c in rng.choice(choices, size=3)) for _ in range(nbox)]


def ensemble(nbox=24, seed=2024, choices=(64, 96, 128, 160, 192), **kw):
    dims = ensemble_dims(nbox, seed, choices)
    return [stratified_box(nx, ny, nz, seed=seed + 1 + b, name=f"ens{b}_{nx}x{ny}x{nz}", **kw)
            for b, (nx, ny, nz) in enumerate(dims)]


def permute_axes(pr: Problem, perm) -> Problem:
    """Relabel the axes of a problem: new axis d is old axis perm[d].

    Used by invariance tests: a problem run along x, y or z must give the same
    (relabelled) result.  Backgrounds are only supported along z, so this is
    for problems without a background.
    """
    assert pr.bg is None and pr.heat is None
    inv = [perm.index(d) for d in range(3)]
    n = tuple(pr.n[perm[d]] for d in range(3))
    # array axis order is (z, y, x) = reversed dims
    def tr(a):
        # a has axes (z, y, x) -> old dims (2,1,0); new axes (z', y', x') = old (perm[2], perm[1], perm[0])
        return np.ascontiguousarray(np.transpose(a, [2 - perm[2], 2 - perm[1], 2 - perm[0]]))
    cons = np.empty((pr.nv,) + (n[2], n[1], n[0]))
    cons[0] = tr(pr.cons[0])
    cons[4:] = [tr(c) for c in pr.cons[4:]]
    for d in range(3):
        cons[1 + d] = tr(pr.cons[1 + perm[d]])
    faces_old = [pr.bx, pr.by, pr.bz]
    faces = [tr(faces_old[perm[d]]) for d in range(3)]
    q = dataclasses.replace(pr)
    q.n = n
    q.lo = tuple(pr.lo[perm[d]] for d in range(3))
    q.hi = tuple(pr.hi[perm[d]] for d in range(3))
    q.bc = tuple(pr.bc[perm[d]] for d in range(3))
    q.g = tuple(pr.g[perm[d]] for d in range(3))
    q.cons, q.bx, q.by, q.bz = cons, faces[0], faces[1], faces[2]
    q.ndim = 3 if min(n) > 1 else pr.ndim
    q.meta = dict(pr.meta, perm=tuple(perm), inv=tuple(inv))
    return q


# ---------------------------------------------------------------- Poisson
# Inputs of the Poisson solver (Sect. 2.12): face coordinates per axis and a
# cell density.  No solver arithmetic lives here.

def stretched_faces(n, lo=-0.5, hi=0.5):
    """n + 1 face coordinates of the paper's stretched axis for its Poisson
    test: x = (eta + eta^5) / 4 at eta = -1 + 2 i / n, i = 0..n, mapped onto
    [lo, hi] (the paper's domain is [-1/2, 1/2]): twice the uniform
    resolution at the origin."""
    eta = -1.0 + 2.0 * np.arange(n + 1) / n
    x = 0.25 * (eta + eta ** 5)
    return lo + (x + 0.5) * (hi - lo)


def random_faces(n, seed, lo=-0.5, hi=0.5, spread=0.5):
    """n + 1 increasing face coordinates on [lo, hi] with cell widths varying
    by up to a factor (1 + spread) / (1 - spread), smoothly (a random sum of
    a few sines), seeded."""
    rng = np.random.default_rng(seed)
    s = np.linspace(0.0, 1.0, n)
    w = np.ones(n)
    for k in range(1, 4):
        w += spread / 3.0 * np.sin(2 * np.pi * k * s + rng.uniform(0, 2 * np.pi))
    w = np.clip(w, 1.0 - spread, 1.0 + spread)
    f = np.concatenate([[0.0], np.cumsum(w)])
    return lo + (hi - lo) * f / f[-1]


def sphere_density(xf, rho0=1.0, r0=0.25):
    """The paper's Poisson test density rho0 (1 - r^2/r0^2)^2 inside r0, zero
    outside, at the cell centres (midpoints of the faces)."""
    xc = [0.5 * (a[1:] + a[:-1]) for a in xf]
    z, y, x = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    r2 = x * x + y * y + z * z
    return np.where(r2 <= r0 * r0, rho0 * (1.0 - r2 / (r0 * r0)) ** 2, 0.0)


def lumpy_density(xf, seed, nblob=5, floor=1e-3):
    """A positive density: a floor plus a few seeded Gaussian blobs of random
    centre, width and mass (off-centre, so every multipole is present)."""
    rng = np.random.default_rng(seed)
    xc = [0.5 * (a[1:] + a[:-1]) for a in xf]
    z, y, x = np.meshgrid(xc[2], xc[1], xc[0], indexing="ij")
    rho = np.full(x.shape, floor)
    for _ in range(nblob):
        c = rng.uniform(-0.25, 0.25, 3)
        w = rng.uniform(0.04, 0.12)
        rho += rng.uniform(0.2, 1.0) * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / w ** 2)
    return rho


# ---------------------------------------------------------------------------
# cubed-sphere shell: six equiangular patches of N x N angular cells times Nr
# radial cells between r_in and r_out (the layout of the library's phl_sphere
# calls and of the oracle's sphere.c):
#   cons[v, p, k, j, i]   (5, 6, Nr, N, N), v = rho, m_x, m_y, m_z, E
#   pa[p, k, j, i]        magnetic flux through alpha faces i = 0..N  (6, Nr, N, N+1)
#   pb[p, k, j, i]        ... beta faces j = 0..N                      (6, Nr, N+1, N)
#   pr[p, k, j, i]        ... radial faces k = 0..Nr                   (6, Nr+1, N, N)
# each flux in its patch's orientation (+alpha, +beta, +r).  Patch p has
# centre direction c_p and axes a_p (alpha), b_p (beta), a_p x b_p = c_p;
# the direction of (alpha, beta) is c_p + tan(alpha) a_p + tan(beta) b_p.
# ---------------------------------------------------------------------------

PATCH_C = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=float)
PATCH_A = np.array([[0, 1, 0], [-1, 0, 0], [0, -1, 0], [1, 0, 0], [0, 1, 0], [0, 1, 0]], dtype=float)
PATCH_B = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1], [-1, 0, 0], [1, 0, 0]], dtype=float)


@dataclasses.dataclass
class ShellProblem:
    name: str
    N: int
    Nr: int
    r_in: float
    r_out: float
    gamma: float
    cons: np.ndarray
    pa: np.ndarray
    pb: np.ndarray
    pr: np.ndarray
    bg: Optional[dict] = None      # rho_c, p_c (Nr, shell middles), rho_f, p_f (Nr + 1, shell radii)
    g_c: Optional[np.ndarray] = None   # inward gravity at the shell middles (Nr,)
    heat: Optional[np.ndarray] = None  # volumetric heating per shell (Nr,)
    cfl: float = 0.4
    riemann: str = "lhlld"
    mach_thr: float = 0.6
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def ncells(self):
        return 6 * self.N * self.N * self.Nr

    def copy(self):
        return dataclasses.replace(self, cons=self.cons.copy(), pa=self.pa.copy(), pb=self.pb.copy(),
                                   pr=self.pr.copy())


def _tline(m, N):
    q = 2 * m - N
    if q == N:
        return 1.0
    if q == -N:
        return -1.0
    t = math.tan(abs(q) * (math.pi / (4.0 * N)))
    return -t if q < 0 else t


def shell_dirs(N):
    """Unit directions of the angular vertices, shape (6, N+1, N+1, 3) [p, j, i]."""
    t = np.array([_tline(m, N) for m in range(N + 1)])
    d = (PATCH_C[:, None, None, :] + t[None, None, :, None] * PATCH_A[:, None, None, :]
         + t[None, :, None, None] * PATCH_B[:, None, None, :])
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def lane_emden(n_poly=1.5, nodes=100000):
    """Lane-Emden theta(xi), theta'(xi) of index n by RK4 on `nodes` steps up to
    the first zero (series start at xi = 1e-6)."""
    def f(x, y):
        th = max(y[0], 0.0)
        return np.array([y[1], -th ** n_poly - 2.0 * y[1] / x])
    xi1_guess = {1.0: math.pi, 1.5: 3.65375, 2.0: 4.35287, 3.0: 6.89685}.get(n_poly, 3.65375)
    x0 = 1e-6
    h = (xi1_guess - x0) / nodes
    xs = np.empty(nodes + 1)
    ys = np.empty((nodes + 1, 2))
    y = np.array([1.0 - x0 * x0 / 6.0, -x0 / 3.0])
    x = x0
    xs[0], ys[0] = x, y
    for q in range(nodes):
        k1 = f(x, y)
        k2 = f(x + 0.5 * h, y + 0.5 * h * k1)
        k3 = f(x + 0.5 * h, y + 0.5 * h * k2)
        k4 = f(x + h, y + h * k3)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        x += h
        xs[q + 1], ys[q + 1] = x, y
    return xs, ys


def shell_background(r_mid, r_faces, r_star=1.2, n_poly=1.5, rho_c=1.0, G=1.0):
    """A Lane-Emden polytrope of index n whose surface sits at r_star (beyond
    the shell): rho = rho_c theta^n, P = K rho_c^(1+1/n) theta^(n+1),
    g = 4 pi G rho_c alpha (-theta'), r = alpha xi (hydrostatic by
    construction), at the shell middles and the shell radii."""
    xs, ys = lane_emden(n_poly)
    xi1 = xs[np.argmax(ys[:, 0] <= 0.0)] if (ys[:, 0] <= 0.0).any() else xs[-1]
    alpha = r_star / xi1
    K = 4.0 * math.pi * G * alpha * alpha * rho_c ** (1.0 - 1.0 / n_poly) / (n_poly + 1.0)

    def at(r):
        xi = np.asarray(r) / alpha
        th = np.interp(xi, xs, ys[:, 0])
        dth = np.interp(xi, xs, ys[:, 1])
        rho = rho_c * th ** n_poly
        p = K * rho_c ** (1.0 + 1.0 / n_poly) * th ** (n_poly + 1.0)
        g = 4.0 * math.pi * G * rho_c * alpha * (-dth)
        return rho, p, g

    rc, pc, gc = at(r_mid)
    rf, pf, _ = at(r_faces)
    return dict(rho_c=rc, p_c=pc, rho_f=rf, p_f=pf), gc


def _gl(ng, dev):
    import torch
    gx, gw = np.polynomial.legendre.leggauss(ng)
    return torch.tensor(gx, dtype=torch.float64, device=dev), torch.tensor(gw, dtype=torch.float64, device=dev)


def _arc_integrals(A, u, w, r, gx, gw):
    """Line integrals of A along the great-circle arcs of radius r from the
    unit directions u to w (..., 3), Gauss-Legendre on the angle."""
    import torch
    c = torch.linalg.cross(u, w, dim=-1)
    th = torch.atan2(torch.linalg.norm(c, dim=-1), (u * w).sum(-1))
    wp = w - (w * u).sum(-1, keepdim=True) * u
    wp = wp / torch.linalg.norm(wp, dim=-1, keepdim=True)
    s = 0.5 * th[..., None] * (gx + 1.0)                                  # (..., ng)
    cs, sn = torch.cos(s)[..., None], torch.sin(s)[..., None]
    pts = r * (cs * u[..., None, :] + sn * wp[..., None, :])
    tang = r * (-sn * u[..., None, :] + cs * wp[..., None, :])
    return 0.5 * th * ((A(pts) * tang).sum(-1) * gw).sum(-1)


def _radial_integrals(A, d, r0, r1, gx, gw):
    """Line integrals of A along the radial segments r0 d -> r1 d."""
    t = 0.5 * (gx + 1.0)
    x0, dx = r0 * d, (r1 - r0) * d
    pts = x0[..., None, :] + t[:, None] * dx[..., None, :]
    return 0.5 * ((A(pts) * dx[..., None, :]).sum(-1) * gw).sum(-1)


def shell_fluxes_from_potential(N, Nr, r, A, device="cpu", ng=8):
    """Magnetic fluxes (pa, pb, pr) of B = curl A through every face, each the
    circulation of A around the face counter-clockwise about the patch's
    +alpha, +beta or +r direction, from the line integrals of A along the
    mesh's edges (Gauss-Legendre, ng points per edge; torch float64 on
    `device`, one shell at a time).  Each patch integrates its own edges; the
    two patches of a seam integrate a shared edge from the same end points,
    so the discrete divergence of every cell vanishes to rounding."""
    import torch
    dev = torch.device(device)
    d = torch.tensor(shell_dirs(N), dtype=torch.float64, device=dev)     # (6, N+1, N+1, 3) [p, j, i]
    gx, gw = _gl(ng, dev)
    rr = [float(x) for x in r]
    # arcs: Ea from (i, j) to (i+1, j), Eb from (i, j) to (i, j+1), per radius
    Ea = torch.stack([_arc_integrals(A, d[:, :, :-1], d[:, :, 1:], rr[k], gx, gw) for k in range(Nr + 1)], 1)
    Eb = torch.stack([_arc_integrals(A, d[:, :-1, :], d[:, 1:, :], rr[k], gx, gw) for k in range(Nr + 1)], 1)
    # radial segments at every vertex, per shell
    R = torch.stack([_radial_integrals(A, d, rr[k], rr[k + 1], gx, gw) for k in range(Nr)], 1)
    # Ea (6, Nr+1, N+1, N) [p, k, j, i]; Eb (6, Nr+1, N, N+1); R (6, Nr, N+1, N+1)
    pa = Eb[:, :-1] + R[:, :, 1:, :] - Eb[:, 1:] - R[:, :, :-1, :]
    pb = R[:, :, :, :-1] + Ea[:, 1:] - R[:, :, :, 1:] - Ea[:, :-1]
    prr = Ea[:, :, :-1, :] + Eb[:, :, :, 1:] - Ea[:, :, 1:, :] - Eb[:, :, :, :-1]
    return pa.contiguous(), pb.contiguous(), prr.contiguous()


def shell_problem(N, Nr, r_in=0.2, r_out=1.0, seed=1234, amp=1e-3, beta=1e5, heat_frac=0.3, mach_heat=1e-3,
                  gamma=5.0 / 3.0, vel_amp=0.0, background=True, gravity=True, cfl=0.4, name=None,
                  uniform=False, device="cpu", eos="ideal"):
    """The cubed-sphere shell of the spherical configuration: a Lane-Emden
    n = 1.5 polytrope (surface at 1.2, so the whole shell r in [0.2, 1] is
    inside the star) in hydrostatic balance under its own radial gravity,
    isobaric density noise amp U(-1, 1) (seeded torch generator on `device`),
    a seed field from the toroidal vector potential A = f(r) (z x r) / r with
    f vanishing at both walls (poloidal, dipole-like, no flux through the
    walls), plasma beta 2 P_hat(r_mid) / B^2 at the shell's middle radius,
    heating in the inner heat_frac of the radial span sized so
    (q dr / rho)^(1/3) ~ mach_heat c_s.  vel_amp > 0 adds a swirl
    u = vel_amp c_s (z x r) / r.  uniform: density and pressure of the shell's
    middle everywhere, no gravity and no background (a medium in which the
    total energy is conserved).  device "cpu": numpy arrays; otherwise the
    state arrays are torch tensors on that device (profiles stay numpy).

    eos "stellar": the same shell in code units whose density and pressure
    are rho_u = 1e7 g/cm^3 / rho_hat(r_in) and p_u = 1.8e24 erg/cm^3 /
    P_hat(r_in) times the stellar EOS's (the stellar box's base state at the
    inner wall, 1e7 -> 6.1e5 g/cm^3 across the shell), 16O/28Si mass fractions
    0.5/0.5 everywhere.  Given as primitives (meta["prim"]: rho, velocity
    (6, Nr, N, N, 3), P): the energy and temperature depend on the EOS, so
    cons[4] is NaN and each implementation builds it with its own EOS."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=dev)
    r = r_in + (r_out - r_in) * np.arange(Nr + 1) / Nr
    rm = 0.5 * (r[:-1] + r[1:])
    bg, g_c = shell_background(rm, r)
    if uniform:
        rmid = 0.5 * (r_in + r_out)
        rho0, p0 = float(np.interp(rmid, rm, bg["rho_c"])), float(np.interp(rmid, rm, bg["p_c"]))
        bg = dict(rho_c=np.full(Nr, rho0), p_c=np.full(Nr, p0), rho_f=np.full(Nr + 1, rho0), p_f=np.full(Nr + 1, p0))
        gravity, background = False, False
    if not gravity:
        g_c = np.zeros(Nr)
    d = torch.tensor(shell_dirs(N), **f64)
    dc = d[:, :-1, :-1] + d[:, 1:, :-1] + d[:, :-1, 1:] + d[:, 1:, 1:]    # cell centre directions [p, j, i]
    dc = dc / torch.linalg.norm(dc, dim=-1, keepdim=True)
    xc = torch.tensor(rm, **f64)[None, :, None, None, None] * dc[:, None]  # (6, Nr, N, N, 3)
    rho_hat = torch.tensor(bg["rho_c"], **f64)[None, :, None, None].expand(6, Nr, N, N)
    p = torch.tensor(bg["p_c"], **f64)[None, :, None, None].expand(6, Nr, N, N).contiguous()
    rho = rho_hat * (1.0 + amp * (2.0 * torch.rand((6, Nr, N, N), generator=gen, **f64) - 1.0))
    rmid = 0.5 * (r_in + r_out)
    p_mid = float(np.interp(rmid, rm, bg["p_c"]))
    cs_mid = math.sqrt(gamma * p_mid / float(np.interp(rmid, rm, bg["rho_c"])))
    vel = torch.zeros(xc.shape, **f64)
    if vel_amp > 0.0:
        zr = torch.stack([-xc[..., 1], xc[..., 0], torch.zeros(xc.shape[:-1], **f64)], -1)
        vel = vel_amp * cs_mid * zr / torch.linalg.norm(xc, dim=-1, keepdim=True)
    span = r_out - r_in
    bc = torch.zeros(xc.shape, **f64)
    if beta and beta > 0:
        b0 = math.sqrt(2.0 * p_mid / beta)

        def A(x):
            rr = torch.linalg.norm(x, dim=-1)
            fr = (rr - r_in) ** 2 * (r_out - rr) ** 2 / (0.25 * span) ** 4
            zx = torch.stack([-x[..., 1], x[..., 0], torch.zeros(x.shape[:-1], dtype=x.dtype, device=x.device)], -1)
            return (b0 * 0.25 * span * fr / rr)[..., None] * zx
        pa, pb, prr = shell_fluxes_from_potential(N, Nr, r, A, device=dev)
        # the energy takes the potential field's curl at the cell centres
        # (central differences); the method's own cell field differs at the
        # truncation level, a negligible share of E at beta >> 1
        eps = 1e-6 * span
        for a_ in range(3):
            e = torch.zeros(3, **f64)
            e[a_] = eps
            dA = (A(xc + e) - A(xc - e)) / (2 * eps)       # dA / dx_a
            if a_ == 0:
                bc[..., 1] -= dA[..., 2]; bc[..., 2] += dA[..., 1]
            elif a_ == 1:
                bc[..., 2] -= dA[..., 0]; bc[..., 0] += dA[..., 2]
            else:
                bc[..., 0] -= dA[..., 1]; bc[..., 1] += dA[..., 0]
    else:
        pa = torch.zeros((6, Nr, N, N + 1), **f64)
        pb = torch.zeros((6, Nr, N + 1, N), **f64)
        prr = torch.zeros((6, Nr + 1, N, N), **f64)
    heat = None
    if heat_frac and heat_frac > 0:
        rho_b = float(bg["rho_c"][0])
        q = rho_b * (mach_heat * cs_mid) ** 3 / (heat_frac * span)
        heat = np.where(rm < r_in + heat_frac * span, q, 0.0)
    cons = torch.empty((5, 6, Nr, N, N), **f64)
    cons[0] = rho
    cons[1:4] = torch.movedim(rho[..., None] * vel, -1, 0)
    meta = dict(seed=seed, amp=amp, beta=beta, r=r, r_mid=rm, eos=eos)
    if eos == "stellar":
        cons[4] = float("nan")
        meta.update(rho_u=STELLAR_RHO_BASE / float(bg["rho_f"][0]), p_u=STELLAR_P_BASE / float(bg["p_f"][0]),
                    A=list(STELLAR_A), Z=list(STELLAR_Z), X=list(STELLAR_X))
    else:
        cons[4] = p / (gamma - 1.0) + 0.5 * rho * (vel ** 2).sum(-1) + 0.5 * (bc ** 2).sum(-1)
    out = [cons, pa, pb, prr]
    prim = dict(rho=rho, vel=vel, p=p)
    if dev.type == "cpu":
        out = [t.numpy() for t in out]
        prim = {k: v.numpy() for k, v in prim.items()}
    if eos == "stellar":
        meta["prim"] = prim
    return ShellProblem(name=name or f"shell_{N}x{N}x{Nr}", N=N, Nr=Nr, r_in=r_in, r_out=r_out, gamma=gamma,
                        cons=out[0], pa=out[1], pb=out[2], pr=out[3], bg=bg if background else None, g_c=g_c,
                        heat=heat, cfl=cfl, meta=meta)
