// eos_stellar.cuh -- stellar equation of state on the device (Sect. 2.2, item ii).
//
// Ions (ideal gas), radiation (Eqs. prad, erad) and an electron-positron gas
// in pair equilibrium.  The e-/e+ part is a table of its Helmholtz
// free-energy density f over (x, y) = (ln n_e, ln T), n_e = rho Y_e N_A, with
// the derivatives f_x = n eta k T, f_y = -T s and f_xy at each node, built on
// the device from the generalised Fermi-Dirac integrals
//   F_k(eta, b) = int_0^inf x^k sqrt(1 + b x/2) / (exp(x - eta) + 1) dx,
// b = kT / m_e c^2.  Bicubic Hermite interpolation of f gives P = f_x - f,
// e = (f - f_y) / rho, c_v = (f_y - f_yy) / (rho T), dP/dT = (f_xy - f_y) / T,
// dP/drho = (f_xx - f_x) / rho -- all from one interpolant, so the
// thermodynamic identities hold for the interpolated EOS.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace phl {
namespace eos {

// CODATA 2018 (CGS)
constexpr double KB = 1.380649e-16;
constexpr double MEC2 = 8.1871057769e-7;
constexpr double HPL = 6.62607015e-27;
constexpr double CL = 2.99792458e10;
constexpr double NAV = 6.02214076e23;
constexpr double ARAD = 7.565733250e-15;
constexpr double ARAD_QUARTER = 2.9492579329135276e-04;   // ARAD^(1/4)
constexpr double RGAS = KB * NAV;
constexpr double PI_D = 3.14159265358979323846;

struct Table {
  int nx, ny;
  double x0, dx, y0, dy;      // x = ln n_e, y = ln T
  const double *v;            // [ny][nx][4]: f, f_x, f_y, f_xy (device)
  const float *vf;            // FP32 copy
  float x0f, dxf, y0f, dyf;
  double idx, idy;            // 1/dx, 1/dy: the evaluation multiplies (FP64 division
  float idxf, idyf;           // is a dozen FP64-pipe instructions on this GPU)
  double Tlo, Thi;            // the table's temperature range, exp(y0) and
  float Tlof, Thif;           // exp(y0 + (ny - 1) dy), set with the table
};

struct Mix {                   // composition-derived constants of a cell
  double abar, ye;
};

template <typename R> struct TV { R f, fx, fy, fxx, fyy, fxy; };

// x-part of the bicubic Hermite evaluation (x = ln n_e): cell, fraction and
// the cubic Hermite basis (value at 0, slope at 0, value at 1, slope at 1)
// with its first and second derivatives.  Constant during a Newton inversion
// (rho and the composition are fixed), so it is computed once per cell.
template <typename R> struct XB {
  int i;
  bool ok;
  R hu[4], du[4], eu[4];
};

template <typename R>
__device__ __forceinline__ XB<R> xbasis(const Table &t, R x) {
  XB<R> X;
  const R x0 = sizeof(R) == 8 ? (R)t.x0 : (R)t.x0f, idx = sizeof(R) == 8 ? (R)t.idx : (R)t.idxf;
  const R gx = (x - x0) * idx;
  X.ok = gx >= R(0) && gx <= R(t.nx - 1);
  int i = X.ok ? (int)gx : 0;
  if (i > t.nx - 2) i = t.nx - 2;
  X.i = i;
  const R u = gx - (R)i;
  const R u2 = u * u, u3 = u2 * u;
  X.hu[0] = R(2) * u3 - R(3) * u2 + R(1); X.hu[1] = u3 - R(2) * u2 + u;
  X.hu[2] = R(-2) * u3 + R(3) * u2;       X.hu[3] = u3 - u2;
  X.du[0] = R(6) * u2 - R(6) * u;          X.du[1] = R(3) * u2 - R(4) * u + R(1);
  X.du[2] = R(-6) * u2 + R(6) * u;         X.du[3] = R(3) * u2 - R(2) * u;
  X.eu[0] = R(12) * u - R(6);              X.eu[1] = R(6) * u - R(4);
  X.eu[2] = R(-12) * u + R(6);             X.eu[3] = R(6) * u - R(2);
  return X;
}

// Bicubic Hermite evaluation of the free energy and its derivatives at
// (x, y = ln T) given the x-part (FULL = false: only f, f_y, f_yy, which is
// what e and c_v need).
template <typename R, bool FULL = true>
__device__ __forceinline__ bool table_eval_xb(const Table &t, const XB<R> &X, R y, TV<R> &o) {
  const R dx = sizeof(R) == 8 ? (R)t.dx : (R)t.dxf, idx = sizeof(R) == 8 ? (R)t.idx : (R)t.idxf;
  const R y0 = sizeof(R) == 8 ? (R)t.y0 : (R)t.y0f, dy = sizeof(R) == 8 ? (R)t.dy : (R)t.dyf;
  const R idy = sizeof(R) == 8 ? (R)t.idy : (R)t.idyf;
  const R gy = (y - y0) * idy;
  if (!(X.ok && gy >= R(0) && gy <= R(t.ny - 1))) return false;
  const int i = X.i;
  int j = (int)gy;
  if (j > t.ny - 2) j = t.ny - 2;
  const R v = gy - (R)j;
  const R v2 = v * v, v3 = v2 * v;
  const R hv[4] = {R(2) * v3 - R(3) * v2 + R(1), v3 - R(2) * v2 + v, R(-2) * v3 + R(3) * v2, v3 - v2};
  const R dv[4] = {R(6) * v2 - R(6) * v, R(3) * v2 - R(4) * v + R(1), R(-6) * v2 + R(6) * v, R(3) * v2 - R(2) * v};
  const R ev[4] = {R(12) * v - R(6), R(6) * v - R(4), R(-12) * v + R(6), R(6) * v - R(2)};
  const R *hu = X.hu, *du = X.du, *eu = X.eu;
  R a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
#pragma unroll
  for (int cb = 0; cb < 2; ++cb)
#pragma unroll
    for (int ca = 0; ca < 2; ++ca) {
      const long k = ((long)(j + cb) * t.nx + (i + ca)) * 4;
      R q0, q1, q2, q3;
      if (sizeof(R) == 8) { q0 = (R)t.v[k]; q1 = (R)t.v[k + 1]; q2 = (R)t.v[k + 2]; q3 = (R)t.v[k + 3]; }
      else { q0 = (R)t.vf[k]; q1 = (R)t.vf[k + 1]; q2 = (R)t.vf[k + 2]; q3 = (R)t.vf[k + 3]; }
      const R c0 = q0, c1 = q1 * dx, c2 = q2 * dy, c3 = q3 * dx * dy;
      const int iv = 2 * ca, is = 2 * ca + 1, jv = 2 * cb, js = 2 * cb + 1;
      a0 += c0 * hu[iv] * hv[jv] + c1 * hu[is] * hv[jv] + c2 * hu[iv] * hv[js] + c3 * hu[is] * hv[js];
      a2 += c0 * hu[iv] * dv[jv] + c1 * hu[is] * dv[jv] + c2 * hu[iv] * dv[js] + c3 * hu[is] * dv[js];
      a4 += c0 * hu[iv] * ev[jv] + c1 * hu[is] * ev[jv] + c2 * hu[iv] * ev[js] + c3 * hu[is] * ev[js];
      if (FULL) {
        a1 += c0 * du[iv] * hv[jv] + c1 * du[is] * hv[jv] + c2 * du[iv] * hv[js] + c3 * du[is] * hv[js];
        a3 += c0 * eu[iv] * hv[jv] + c1 * eu[is] * hv[jv] + c2 * eu[iv] * hv[js] + c3 * eu[is] * hv[js];
        a5 += c0 * du[iv] * dv[jv] + c1 * du[is] * dv[jv] + c2 * du[iv] * dv[js] + c3 * du[is] * dv[js];
      }
    }
  o.f = a0;
  o.fx = a1 * idx;
  o.fy = a2 * idy;
  o.fxx = a3 * (idx * idx);
  o.fyy = a4 * (idy * idy);
  o.fxy = a5 * (idx * idy);
  return true;
}

template <typename R, bool FULL = true>
__device__ __forceinline__ bool table_eval(const Table &t, R x, R y, TV<R> &o) {
  return table_eval_xb<R, FULL>(t, xbasis<R>(t, x), y, o);
}

template <typename R> struct EosOut { R P, e, cv, Pr, PT, ge, gc; };

// Full EOS at (rho, T) for a mixture with mean mass number abar and Y_e
// (irho = 1/rho and iab = 1/abar: fixed during an inversion, formed once).
template <typename R>
__device__ __forceinline__ bool eos_rt_xy(const Table &t, const XB<R> &X, R rho, R irho, R T, R lnT, R iab,
                                          EosOut<R> &o) {
  TV<R> q;
  if (!table_eval_xb<R>(t, X, lnT, q)) return false;
  const R iT = R(1) / T;
  const R Pe = q.fx - q.f;
  const R ee = (q.f - q.fy) * irho;
  const R cve = (q.fy - q.fyy) * irho * iT;
  const R PeT = (q.fxy - q.fy) * iT;
  const R Per = (q.fxx - q.fx) * irho;
  const R Rg = R(RGAS);
  R aT4, aT3;   // radiation a T^4 and a T^3
  if (sizeof(R) == 8) {
    const R T3 = T * T * T;
    aT3 = R(ARAD) * T3;
    aT4 = aT3 * T;
  } else {   // T^4 overflows FP32 above 2^32 K: form (a^(1/4) T)^4 instead
    const R t = R(ARAD_QUARTER) * T, t2 = t * t;
    aT4 = t2 * t2;
    aT3 = aT4 * iT;
  }
  o.P = Pe + rho * Rg * T * iab + aT4 / R(3);
  o.e = ee + R(1.5) * Rg * T * iab + aT4 * irho;
  o.cv = cve + R(1.5) * Rg * iab + R(4) * aT3 * irho;
  o.PT = PeT + rho * Rg * iab + R(4) / R(3) * aT3;
  o.Pr = Per + Rg * T * iab;
  // auxiliary indices of Sect. 2.6: gamma_e = P / (rho e) + 1, gamma_c = rho c_s^2 / P;
  // c_s^2 = P_rho + T P_T^2 / (rho^2 c_v), grouped so no product leaves the FP32 range
  const R cs2 = o.Pr + (T * o.PT * irho) * (o.PT * irho / o.cv);
  o.ge = o.P / (rho * o.e) + R(1);
  o.gc = rho * cs2 / o.P;
  return true;
}

template <typename R>
__device__ __forceinline__ bool eos_rt(const Table &t, R rho, R T, R abar, R ye, EosOut<R> &o) {
  return eos_rt_xy<R>(t, xbasis<R>(t, log(rho * ye * R(NAV))), rho, R(1) / rho, T, log(T), R(1) / abar, o);
}

// Specific internal energy and c_v at (rho, T): what a Newton iteration needs.
template <typename R>
__device__ __forceinline__ bool eos_ecv_xy(const Table &t, const XB<R> &X, R irho, R T, R lnT, R iab, R &e, R &cv) {
  TV<R> q;
  if (!table_eval_xb<R, false>(t, X, lnT, q)) return false;
  const R iT = R(1) / T;
  const R Rg = R(RGAS);
  R aT4, aT3;
  if (sizeof(R) == 8) {
    aT3 = R(ARAD) * T * T * T;
    aT4 = aT3 * T;
  } else {
    const R tt = R(ARAD_QUARTER) * T, t2 = tt * tt;
    aT4 = t2 * t2;
    aT3 = aT4 * iT;
  }
  e = (q.f - q.fy) * irho + R(1.5) * Rg * T * iab + aT4 * irho;
  cv = (q.fy - q.fyy) * irho * iT + R(1.5) * Rg * iab + R(4) * aT3 * irho;
  return true;
}

template <typename R>
__device__ __forceinline__ bool eos_ecv(const Table &t, R rho, R T, R abar, R ye, R &e, R &cv) {
  return eos_ecv_xy<R>(t, xbasis<R>(t, log(rho * ye * R(NAV))), R(1) / rho, T, log(T), R(1) / abar, e, cv);
}

// ln Tn from ln T for a Newton step T -> Tn: with d = (Tn - T) / T below
// 2^-10, ln(1 + d) by its Taylor series to d^4 (truncation below d^5 / 5 <
// 2e-16, under the rounding of ln T ~ 16..23); otherwise the logarithm.
// Saves an FP64 logarithm per step once the iteration is close.
template <typename R>
__device__ __forceinline__ R next_lnT(R T, R lnT, R Tn) {
  const R d = (Tn - T) / T;
  if (!(fabs(d) < R(1.0 / 1024.0))) return log(Tn);
  return lnT + d * (R(1) - d * (R(0.5) - d * (R(1.0 / 3.0) - d * R(0.25))));
}

// Newton inversion e_int -> T (Sect. 2.2): T <- T + (e - e_EoS)/c_v until
// |de|/e < tol, then one more step; bracketed inside the table's T range.
// The iterations evaluate only e and c_v; the full EOS (P, gamma_e, gamma_c)
// is evaluated once, at the final T.  Returns the iteration count or -1.
template <typename R>
__device__ __forceinline__ int newton_loop(const Table &t, const XB<R> &X, R rho, R irho, R eint, R iab, R &T, R tol,
                                           int maxit, EosOut<R> &o, bool have, R e0, R cv0, R lnT0) {
  const R Tlo = sizeof(R) == 8 ? (R)t.Tlo : (R)t.Tlof, Thi = sizeof(R) == 8 ? (R)t.Thi : (R)t.Thif;
  R lo = Tlo, hi = Thi;
  if (!(T > Tlo && T < Thi)) { T = sqrt(Tlo * Thi); have = false; }
  R lnT = have ? lnT0 : log(T);   // e0, cv0 were evaluated at (T, lnT0)
  for (int it = 1; it <= maxit; ++it) {
    R e = e0, cv = cv0;   // the first iteration may come evaluated
    if (!(have && it == 1) && !eos_ecv_xy<R>(t, X, irho, T, lnT, iab, e, cv)) return -1;
    const R de = eint - e;
    if (fabs(de) < tol * fabs(eint)) {
      const R Tn = T + de / cv;
      lnT = next_lnT<R>(T, lnT, Tn);
      T = Tn;
      if (!eos_rt_xy<R>(t, X, rho, irho, T, lnT, iab, o)) return -1;
      return it;
    }
    if (de > R(0)) lo = T; else hi = T;
    R Tn = T + de / cv;
    if (!(Tn > lo && Tn < hi)) Tn = R(0.5) * (lo + hi);
    lnT = next_lnT<R>(T, lnT, Tn);
    T = Tn;
  }
  return -1;
}

template <typename R>
__device__ __forceinline__ int eos_invert(const Table &t, R rho, R eint, R abar, R ye, R &T, R tol, int maxit,
                                          EosOut<R> &o) {
  const XB<R> X = xbasis<R>(t, log(rho * ye * R(NAV)));   // rho and Y_e fixed
  return newton_loop<R>(t, X, rho, R(1) / rho, eint, R(1) / abar, T, tol, maxit, o, false, R(0), R(0), R(0));
}

// The FP32 phase of the mixed inversion: Newton on e and c_v only, until
// |de|/e < tol or maxit; T keeps the last bracketed iterate.
__device__ __forceinline__ int newton_fp32(const Table &t, float rho, float eint, float abar, float ye, float &T,
                                           float tol, int maxit) {
  const float Tlo = t.Tlof, Thi = t.Thif;
  float lo = Tlo, hi = Thi;
  if (!(T > Tlo && T < Thi)) T = sqrtf(Tlo * Thi);
  const XB<float> X = xbasis<float>(t, logf(rho * ye * float(NAV)));
  const float irho = 1.0f / rho, iab = 1.0f / abar;
  for (int it = 1; it <= maxit; ++it) {
    float e, cv;
    if (!eos_ecv_xy<float>(t, X, irho, T, logf(T), iab, e, cv)) return -1;
    const float de = eint - e;
    if (de > 0.0f) lo = T; else hi = T;
    float Tn = T + de / cv;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5f * (lo + hi);
    T = Tn;
    if (fabsf(de) < tol * fabsf(eint)) return it;
  }
  return -1;
}

// Mixed-precision inversion: from a guess farther than 1e-4 from the root,
// FP32 Newton iterations (e and c_v only) bring T within about 1e-5 of it (|de| / e; FP32 holds ln n_e ~ 70 and
// ln T ~ 20 only to ~1e-6, the floor of an FP32 table lookup); FP64 Newton
// then finishes with the FP64 path's stopping rule (|de|/e < tol, one more
// step, the full evaluation at the final T).  The low-Mach deviations need
// P to ~1e-12, so a single FP64 step from 1e-5 is not enough.  Returns the
// total iteration count, or -1 if the FP64 phase fails.
__device__ __forceinline__ int eos_invert_mixed(const Table &t, double rho, double eint, double abar, double ye,
                                                double &T, double tol, int maxit, EosOut<double> &o) {
  // a first guess already within 1e-4 of the root (the previous step's T in
  // a time step) goes straight to the FP64 iteration: the FP32 phase could
  // only degrade it to FP32's ~1e-6
  const XB<double> X = xbasis<double>(t, log(rho * ye * NAV));
  const double irho = 1.0 / rho, iab = 1.0 / abar;
  {
    double e, cv;
    if (T > t.Tlo && T < t.Thi) {
      const double lnT = log(T);
      if (eos_ecv_xy<double>(t, X, irho, T, lnT, iab, e, cv) && fabs(eint - e) < 1e-4 * fabs(eint))
        return newton_loop<double>(t, X, rho, irho, eint, iab, T, tol, maxit, o, true, e, cv, lnT);
    }
  }
  float Tf = (float)T;
  const int it32 = newton_fp32(t, (float)rho, (float)eint, (float)abar, (float)ye, Tf, 1e-5f, maxit < 12 ? maxit : 12);
  if (isfinite(Tf) && Tf > 0.0f) T = (double)Tf;
  const int it64 = newton_loop<double>(t, X, rho, irho, eint, iab, T, tol, maxit, o, false, 0.0, 0.0, 0.0);
  return it64 < 0 ? -1 : it64 + (it32 > 0 ? it32 : 12);
}

}  // namespace eos
}  // namespace phl
