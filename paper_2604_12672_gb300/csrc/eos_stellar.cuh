// eos_stellar.cuh -- stellar equation of state on the device (Sect. 2.2, item ii).
//
// Ions (ideal gas), radiation (Eqs. prad, erad) and an electron-positron gas
// in pair equilibrium.  The e-/e+ part is a table of its Helmholtz
// free-energy density f over (x, y) = (ln n_e, ln T), n_e = rho Y_e N_A,
// holding at each node f and its derivatives f_x, f_y, f_xx, f_yy, f_xy,
// f_xxy, f_xyy, f_xxyy (eos_nodes.cuh), interpolated biquintically as the
// paper does with its Helmholtz table: the tensor product of quintic Hermite
// polynomials, which takes f and its derivatives up to second order in each
// variable from the nodes.  P = f_x - f, e = (f - f_y) / rho,
// c_v = (f_y - f_yy) / (rho T), dP/dT = (f_xy - f_y) / T,
// dP/drho = (f_xx - f_x) / rho all come from one interpolant, so the
// thermodynamic identities hold for the interpolated EOS, and c_v, gamma_c
// are continuous.
//
// Evaluation in two parts.  rho and the composition are fixed during an
// inversion, so the x-direction is contracted once per table row pair: for
// the two y-nodes j, j+1 of the current cell and each y-order r = 0, 1, 2,
// g[m][b][r] = d^m/dx^m d^r/dy^r f at (x, y_(j+b)) by the quintic Hermite
// polynomial in x.  A Newton iteration then needs only the one-dimensional
// quintic in y on those six values (18 multiply-adds for f, f_y, f_yy), and
// redoes the contraction only when T leaves the current table interval.
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
constexpr int NQ = 9;          // node values: f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy

// node slot of d^(p + r) f / dx^p dy^r
__host__ __device__ __forceinline__ int qslot(int p, int r) {
  return p == 0 ? 2 * r : (p == 1 ? (r == 0 ? 1 : 3 + 2 * r) : (r == 0 ? 3 : 4 + 2 * r));
}

struct Table {
  int nx, ny;
  double x0, dx, y0, dy;      // x = ln n_e, y = ln T
  const double *v;            // [ny][nx][NQ] (device)
  const float *vf;            // FP32 copy
  const double *d;            // [ny-1][nx-1][NQ][4]: each table cell's corner values in difference
                              // form (D00, D10, D01, D11 below), each slot times dx^p dy^r (its
                              // derivative orders in units of the cell), formed once; null: formed
                              // per use.  With d the FP64 evaluation works in cell units and scales
                              // its results once (idx2 = idx^2, idy2 = idy^2, idxdy = idx idy).
  double idx2, idy2, idxdy;
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

// Quintic Hermite basis on [0, 1]: h[a][q] has q-th derivative 1 at end a and
// value, first and second derivative 0 otherwise at both ends; d, e are its
// first and second derivatives.  At end 1 the functions are (-1)^q times those
// of end 0 at 1 - u.  D selects what is formed: 0 values, 1 + first, 2 + second.
template <typename R, int D>
__device__ __forceinline__ void quintic(R u, R h[2][3], R d[2][3], R e[2][3]) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const R w = a == 0 ? u : R(1) - u;
    const R w2 = w * w, w3 = w2 * w;
    h[a][0] = R(1) + w3 * (R(-10) + w * (R(15) - R(6) * w));
    h[a][1] = w + w3 * (R(-6) + w * (R(8) - R(3) * w));
    h[a][2] = R(0.5) * w2 * (R(1) + w * (R(-3) + w * (R(3) - w)));
    if (D >= 1) {
      d[a][0] = w2 * (R(-30) + w * (R(60) - R(30) * w));
      d[a][1] = R(1) + w2 * (R(-18) + w * (R(32) - R(15) * w));
      d[a][2] = w * (R(1) + w * (R(-4.5) + w * (R(6) - R(2.5) * w)));
    }
    if (D >= 2) {
      e[a][0] = w * (R(-60) + w * (R(180) - R(120) * w));
      e[a][1] = w * (R(-36) + w * (R(96) - R(60) * w));
      e[a][2] = R(1) + w * (R(-9) + w * (R(18) - R(10) * w));
    }
    if (a == 1) {   // (-1)^q, and d/du = -d/dw on the first derivative
      h[1][1] = -h[1][1];
      if (D >= 1) { d[1][0] = -d[1][0]; d[1][2] = -d[1][2]; }
      if (D >= 2) e[1][1] = -e[1][1];
    }
  }
}

// Difference form of a tensor product.  The 2 x 2 corner values c[a][b] of
// a quantity enter as sum c[a][b] X_a Y_b = sum D[a][b] X~_a Y~_b with
// D00 = c00, D10 = c10 - c00, D01 = c01 - c00, D11 = (c11 - c10) - (c01 - c00),
// X~_0 = X_0 + X_1, X~_1 = X_1 (the same in y): an identity, in which the
// value functions' X~_0 is exactly 1 (value) or 0 (derivatives).  It keeps a
// derivative from cancelling two large node values (f_y from f alone would
// lose ~|f| / dy to rounding).
template <typename R>
__device__ __forceinline__ void diff_basis(R b[2][3], R first) {
  b[0][0] = first;
  b[0][1] += b[1][1];
  b[0][2] += b[1][2];
}

// x-part (x = ln n_e), fixed during an inversion: cell and the quintic basis
// in difference form, with dx^p folded into order p (value), dx^(p-1) (first
// derivative) and dx^(p-2) (second), so contracted values are physical
// derivatives.
template <typename R> struct XB {
  int i;
  bool ok;
  R h[2][3], d[2][3], e[2][3];
};

template <typename R>
__device__ __forceinline__ XB<R> xbasis(const Table &t, R x) {
  XB<R> X;
  const R x0 = sizeof(R) == 8 ? (R)t.x0 : (R)t.x0f, idx = sizeof(R) == 8 ? (R)t.idx : (R)t.idxf;
  const R dx = sizeof(R) == 8 ? (R)t.dx : (R)t.dxf;
  const R gx = (x - x0) * idx;
  X.ok = gx >= R(0) && gx <= R(t.nx - 1);
  int i = X.ok ? (int)gx : 0;
  if (i > t.nx - 2) i = t.nx - 2;
  X.i = i;
  quintic<R, 2>(gx - (R)i, X.h, X.d, X.e);
  diff_basis<R>(X.h, R(1));
  diff_basis<R>(X.d, R(0));
  diff_basis<R>(X.e, R(0));
  if (sizeof(R) == 8 && t.d) return X;   // cell units: the table's differences carry dx^p
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    X.h[a][1] *= dx; X.h[a][2] *= dx * dx;
    X.d[a][0] *= idx; X.d[a][2] *= dx;
    X.e[a][0] *= idx * idx; X.e[a][1] *= idx;
  }
  return X;
}

// The x-contracted values of one y-interval, in difference form along y:
// g[m][r] = d^m/dx^m d^r/dy^r f at (x, y_j) and dg[m][r] the same at y_(j+1)
// minus that at y_j (contracted from node differences), m < M.
template <typename R, int M> struct YC {
  int j;
  R g[M][3], dg[M][3];
};

template <typename R, int M, int M0 = 0>
__device__ __forceinline__ void contract(const Table &t, const XB<R> &X, int j, YC<R, M> &c) {
  c.j = j;
  const bool pre = sizeof(R) == 8 && t.d;   // the differences stored with the table
  const long k0 = ((long)j * t.nx + X.i) * NQ, k1 = k0 + (long)t.nx * NQ;
  const double *dc = pre ? t.d + ((long)j * (t.nx - 1) + X.i) * 4 * NQ : nullptr;
  R q[2][2][NQ];   // [b][a][slot]; with pre: [0][0] D00, [0][1] D10, [1][0] D01, [1][1] D11
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int s = 0; s < NQ; ++s) {
        const long k = (b ? k1 : k0) + a * NQ + s;
        q[b][a][s] = pre ? (R)dc[4 * s + 2 * b + a] : (sizeof(R) == 8 ? (R)t.v[k] : (R)t.vf[k]);
      }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    R g0 = R(0), g1 = R(0), g2 = R(0), d0 = R(0), d1 = R(0), d2 = R(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const int sl = qslot(p, r);
      const R D00 = q[0][0][sl];
      const R D10 = pre ? q[0][1][sl] : q[0][1][sl] - q[0][0][sl];
      const R D01 = pre ? q[1][0][sl] : q[1][0][sl] - q[0][0][sl];
      const R D11 = pre ? q[1][1][sl] : (q[1][1][sl] - q[0][1][sl]) - (q[1][0][sl] - q[0][0][sl]);
      if (M0 == 0) {
        g0 += D00 * X.h[0][p] + D10 * X.h[1][p];
        d0 += D01 * X.h[0][p] + D11 * X.h[1][p];
      }
      if (M > 1) {
        g1 += D00 * X.d[0][p] + D10 * X.d[1][p];
        d1 += D01 * X.d[0][p] + D11 * X.d[1][p];
      }
      if (M > 2) {
        g2 += D00 * X.e[0][p] + D10 * X.e[1][p];
        d2 += D01 * X.e[0][p] + D11 * X.e[1][p];
      }
    }
    if (M0 == 0) { c.g[0][r] = g0; c.dg[0][r] = d0; }
    if (M > 1) { c.g[1][r] = g1; c.dg[1][r] = d1; }
    if (M > 2) { c.g[2][r] = g2; c.dg[2][r] = d2; }
  }
}

// The full contraction of interval j, reusing the values of a Newton
// iteration's contraction c1 when it holds the same interval.
template <typename R>
__device__ __forceinline__ void contract_full(const Table &t, const XB<R> &X, int j, const YC<R, 1> *c1, YC<R, 3> &c) {
  if (c1 && c1->j == j) {
#pragma unroll
    for (int r = 0; r < 3; ++r) { c.g[0][r] = c1->g[0][r]; c.dg[0][r] = c1->dg[0][r]; }
    contract<R, 3, 1>(t, X, j, c);
  } else {
    contract<R, 3>(t, X, j, c);
  }
}

// Interval index of y and its fraction; false outside the table.
template <typename R>
__device__ __forceinline__ bool yloc(const Table &t, R y, int &j, R &v) {
  const R y0 = sizeof(R) == 8 ? (R)t.y0 : (R)t.y0f, idy = sizeof(R) == 8 ? (R)t.idy : (R)t.idyf;
  const R gy = (y - y0) * idy;
  if (!(gy >= R(0) && gy <= R(t.ny - 1))) return false;
  j = (int)gy;
  if (j > t.ny - 2) j = t.ny - 2;
  v = gy - (R)j;
  return true;
}

// f, f_y, f_yy (M = 1) and also f_x, f_xy (M >= 2), f_xx (M = 3) at fraction
// v of the interval the contraction holds.
template <typename R, int M>
__device__ __forceinline__ void yeval(const Table &t, const YC<R, M> &c, R v, TV<R> &o) {
  const R dy = sizeof(R) == 8 ? (R)t.dy : (R)t.dyf, idy = sizeof(R) == 8 ? (R)t.idy : (R)t.idyf;
  const bool pre = sizeof(R) == 8 && t.d;   // cell units: scale the results once
  R h[2][3], d[2][3], e[2][3];
  quintic<R, 2>(v, h, d, e);
  diff_basis<R>(h, R(1));
  diff_basis<R>(d, R(0));
  diff_basis<R>(e, R(0));
  R a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, c0 = 0;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const R sh[3] = {h[b][0], pre ? h[b][1] : h[b][1] * dy, pre ? h[b][2] : h[b][2] * dy * dy};
    const R sd[3] = {pre ? d[b][0] : d[b][0] * idy, d[b][1], pre ? d[b][2] : d[b][2] * dy};
    const R se[3] = {pre ? e[b][0] : e[b][0] * idy * idy, pre ? e[b][1] : e[b][1] * idy, e[b][2]};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const R g0 = b ? c.dg[0][r] : c.g[0][r];
      a0 += g0 * sh[r];
      a1 += g0 * sd[r];
      a2 += g0 * se[r];
      if (M > 1) {
        const R g1 = b ? c.dg[1][r] : c.g[1][r];
        b0 += g1 * sh[r];
        b1 += g1 * sd[r];
      }
      if (M > 2) c0 += (b ? c.dg[2][r] : c.g[2][r]) * sh[r];
    }
  }
  if (pre) {
    o.f = a0; o.fy = a1 * R(t.idy); o.fyy = a2 * R(t.idy2);
    o.fx = b0 * R(t.idx); o.fxy = b1 * R(t.idxdy); o.fxx = c0 * R(t.idx2);
  } else {
    o.f = a0; o.fy = a1; o.fyy = a2;
    o.fx = b0; o.fxy = b1; o.fxx = c0;
  }
}

// Biquintic evaluation of f and its derivatives up to second order at
// (x, y = ln T) given the x-part.
template <typename R>
__device__ __forceinline__ bool table_eval_xb(const Table &t, const XB<R> &X, R y, TV<R> &o,
                                              const YC<R, 1> *c1 = nullptr) {
  int j;
  R v;
  if (!(X.ok && yloc<R>(t, y, j, v))) return false;
  YC<R, 3> c;
  contract_full<R>(t, X, j, c1, c);
  yeval<R, 3>(t, c, v, o);
  return true;
}

template <typename R>
__device__ __forceinline__ bool table_eval(const Table &t, R x, R y, TV<R> &o) {
  return table_eval_xb<R>(t, xbasis<R>(t, x), y, o);
}

// er: de/drho at fixed T (the next inversion's first guess, eos_invert_pred)
template <typename R> struct EosOut { R P, e, cv, Pr, PT, ge, gc, er; };

// Full EOS at (rho, T) for a mixture with mean mass number abar and Y_e
// (irho = 1/rho and iab = 1/abar: fixed during an inversion, formed once).
template <typename R>
__device__ __forceinline__ bool eos_rt_xy(const Table &t, const XB<R> &X, R rho, R irho, R T, R lnT, R iab,
                                          EosOut<R> &o, const YC<R, 1> *c1 = nullptr) {
  TV<R> q;
  if (!table_eval_xb<R>(t, X, lnT, q, c1)) return false;
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
  // d/drho = (1/rho) d/dx at fixed T: ((f_x - f_xy) - (f - f_y)) / rho^2 and -a T^4 / rho^2
  o.er = ((q.fx - q.fxy) - (q.f - q.fy) - aT4) * irho * irho;
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
// c holds the x-contraction of the current table interval and is redone when
// T has left it.
template <typename R>
__device__ __forceinline__ bool eos_ecv_xy(const Table &t, const XB<R> &X, YC<R, 1> &c, R irho, R T, R lnT, R iab,
                                           R &e, R &cv) {
  int j;
  R v;
  if (!(X.ok && yloc<R>(t, lnT, j, v))) return false;
  if (j != c.j) contract<R, 1>(t, X, j, c);
  TV<R> q;
  yeval<R, 1>(t, c, v, q);
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
  YC<R, 1> c;
  c.j = -1;
  return eos_ecv_xy<R>(t, xbasis<R>(t, log(rho * ye * R(NAV))), c, R(1) / rho, T, log(T), R(1) / abar, e, cv);
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
__device__ __forceinline__ int newton_loop(const Table &t, const XB<R> &X, YC<R, 1> &c, R rho, R irho, R eint, R iab,
                                           R &T, R tol, int maxit, EosOut<R> &o, bool have, R e0, R cv0, R lnT0) {
  const R Tlo = sizeof(R) == 8 ? (R)t.Tlo : (R)t.Tlof, Thi = sizeof(R) == 8 ? (R)t.Thi : (R)t.Thif;
  R lo = Tlo, hi = Thi;
  if (!(T > Tlo && T < Thi)) { T = sqrt(Tlo * Thi); have = false; }
  R lnT = have ? lnT0 : log(T);   // e0, cv0 were evaluated at (T, lnT0), c may hold its interval
  for (int it = 1; it <= maxit; ++it) {
    R e = e0, cv = cv0;   // the first iteration may come evaluated
    if (!(have && it == 1) && !eos_ecv_xy<R>(t, X, c, irho, T, lnT, iab, e, cv)) return -1;
    const R de = eint - e;
    if (fabs(de) < tol * fabs(eint)) {
      const R Tn = T + de / cv;
      lnT = next_lnT<R>(T, lnT, Tn);
      T = Tn;
      if (!eos_rt_xy<R>(t, X, rho, irho, T, lnT, iab, o, &c)) return -1;
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
  YC<R, 1> c;
  c.j = -1;
  return newton_loop<R>(t, X, c, rho, R(1) / rho, eint, R(1) / abar, T, tol, maxit, o, false, R(0), R(0), R(0));
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
  YC<float, 1> c;
  c.j = -1;
  for (int it = 1; it <= maxit; ++it) {
    float e, cv;
    if (!eos_ecv_xy<float>(t, X, c, irho, T, logf(T), iab, e, cv)) return -1;
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
  YC<double, 1> c;
  c.j = -1;
  {
    double e, cv;
    if (T > t.Tlo && T < t.Thi) {
      const double lnT = log(T);
      if (eos_ecv_xy<double>(t, X, c, irho, T, lnT, iab, e, cv) && fabs(eint - e) < 1e-4 * fabs(eint)) {
        const double de = eint - e;
        // From |de|/e < 2e-6 one Newton step lands within ~(de/e)^2 < 1e-11
        // of the root (quadratic convergence; d ln e / d ln T is 1..4 here):
        // the full evaluation at that T1, carried to the root T1 + dT, dT =
        // (e - e(T1)) / c_v(T1), to first order in dT -- P by P_T dT (error
        // ~ dT^2), gamma_e = P / (rho e) + 1 from that P and e; gamma_c keeps
        // its value at T1 (relative error ~ dT / T < 1e-11, wave speeds
        // only).  The plain iteration would evaluate e, c_v at T1 once more
        // and then the full EOS at T1 + dT.
        if (fabs(de) >= tol * fabs(eint) && fabs(de) < 2e-6 * fabs(eint)) {
          const double T1 = T + de / cv;
          if (T1 > t.Tlo && T1 < t.Thi) {
            if (!eos_rt_xy<double>(t, X, rho, irho, T1, next_lnT<double>(T, lnT, T1), iab, o, &c)) return -1;
            const double dT = (eint - o.e) / o.cv;
            o.P = fma(o.PT, dT, o.P);
            o.e = eint;
            o.ge = o.P / (rho * eint) + 1.0;
            T = T1 + dT;
            return 2;
          }
        }
        return newton_loop<double>(t, X, c, rho, irho, eint, iab, T, tol, maxit, o, true, e, cv, lnT);
      }
    }
  }
  float Tf = (float)T;
  const int it32 = newton_fp32(t, (float)rho, (float)eint, (float)abar, (float)ye, Tf, 1e-5f, maxit < 12 ? maxit : 12);
  if (isfinite(Tf) && Tf > 0.0f) T = (double)Tf;
  const int it64 = newton_loop<double>(t, X, c, rho, irho, eint, iab, T, tol, maxit, o, false, 0.0, 0.0, 0.0);
  return it64 < 0 ? -1 : it64 + (it32 > 0 ? it32 : 12);
}

// The last inversion of a cell, for the next one's first guess: its rho,
// e_int, 1/c_v and de/drho|_T there, ln T and 1/T of the result, and
// x = ln(n_e N_A) and 1/n_e with n_e = rho Y_e.
struct Pred {
  double rho, e, icv, er, lnT, iT, x, ine;
};

// 1/(a (1 + d)) from ia = 1/a: the series 1 - d + d^2 - d^3 + d^4 below
// |d| = 2^-10 (truncation below 2^-50), else the division.
__device__ __forceinline__ double inv_step(double ia, double d, double a_new) {
  if (!(fabs(d) < 1.0 / 1024.0)) return 1.0 / a_new;
  return ia * (1.0 - d * (1.0 - d * (1.0 - d * (1.0 - d))));
}

// ln(a) from ln(a_p) for a = a_p (1 + d): the series of ln(1 + d) to d^4
// below |d| = 2^-10 (as next_lnT), else fall back.
__device__ __forceinline__ double ln_step(double lnp, double d, double fallback_arg) {
  if (!(fabs(d) < 1.0 / 1024.0)) return log(fallback_arg);
  return lnp + d * (1.0 - d * (0.5 - d * (1.0 / 3.0 - d * 0.25)));
}

// The full EOS at (rho, T) for the recorded mixed inversion: P, e, P_T,
// 1/c_v, de/drho|_T, c_s^2 and 1/T, the reciprocals formed once (gamma_e and
// gamma_c follow from the carried P in rec_carry).
struct EosC {
  double P, e, PT, icv, er, cs2, iT;
};
__device__ __forceinline__ bool eos_rt_c(const Table &t, const XB<double> &X, double rho, double irho, double T,
                                         double lnT, double iT, double iab, EosC &o, const YC<double, 1> *c1) {
  TV<double> q;
  if (!table_eval_xb<double>(t, X, lnT, q, c1)) return false;
  const double Rg = RGAS;
  const double aT3 = ARAD * T * T * T, aT4 = aT3 * T;
  o.P = (q.fx - q.f) + rho * Rg * T * iab + aT4 * (1.0 / 3.0);
  o.e = (q.f - q.fy) * irho + 1.5 * Rg * T * iab + aT4 * irho;
  o.icv = 1.0 / ((q.fy - q.fyy) * irho * iT + 1.5 * Rg * iab + 4.0 * aT3 * irho);
  o.PT = (q.fxy - q.fy) * iT + rho * Rg * iab + (4.0 / 3.0) * aT3;
  const double Pr = (q.fxx - q.fx) * irho + Rg * T * iab;
  o.cs2 = Pr + (T * o.PT * irho) * (o.PT * irho * o.icv);
  o.er = ((q.fx - q.fxy) - (q.f - q.fy) - aT4) * irho * irho;
  o.iT = iT;
  return true;
}

// The carry of a full evaluation c at T1 (within ~2e-6 of the root in e) to
// the root T1 + dT, dT = (e - e(T1)) / c_v, to first order: P + P_T dT;
// gamma_e = P / (rho e) + 1 from that P and e; gamma_c = rho c_s^2 / P
// (c_s^2 at T1: relative error ~dT/T, wave speeds only); one reciprocal for
// both.  Writes the record of the inversion.
__device__ __forceinline__ void rec_carry(double rho, double eint, double ine, double x, double T1, double lnT1,
                                          const EosC &c, EosOut<double> &o, double &T, Pred &pr) {
  const double dT = (eint - c.e) * c.icv;
  const double P = fma(c.PT, dT, c.P);
  const double re = rho * eint;
  const double inv = 1.0 / (P * re);   // 1/(rho e) = P inv, 1/P = rho e inv
  o.P = P;
  o.e = eint;
  o.ge = P * (P * inv) + 1.0;
  o.gc = rho * c.cs2 * (re * inv);
  o.cv = 0.0;   // not formed on this path
  o.er = c.er;
  T = T1 + dT;
  const double dd = dT * c.iT;
  pr = Pred{rho, eint, c.icv, c.er, lnT1 + dd * (1.0 - dd * (0.5 - dd * (1.0 / 3.0))), c.iT * (1.0 - dd), x, ine};
}

// Mixed-precision inversion with a per-cell record (rec: the record holds
// the cell's previous inversion).  With a record, the first-order guess
//   T1 = T + (e - e_p - (de/drho)_T (rho - rho_p)) / c_v
// lies within ~(relative change since then)^2 of the root: one full
// evaluation there and, where |e - e(T1)| / e < 2e-6, its carry to the root
// (rec_carry); ln(n_e N_A) and ln T1 follow from the record's by the series
// of ln(1 + d).  Without a record (or where the change was larger) the
// mixed inversion's own steps: e, c_v at T; from within 2e-6 one Newton
// step, the full evaluation and the carry; from within 1e-4 the FP64 Newton
// loop; else FP32 iterations first.  irho = 1/rho and iab = 1/Abar come
// with the arguments.  Writes the record; returns the count of evaluations
// at distinct temperatures (1 for the recorded path) or -1.
__device__ __forceinline__ int eos_invert_rec(const Table &t, double rho, double irho, double eint, double abar,
                                              double iab, double ye, double &T, double tol, int maxit,
                                              EosOut<double> &o, Pred &pr, bool rec) {
  const double ne = rho * ye;
  rec = rec && pr.ine > 0.0;
  const double dn = rec ? ne * pr.ine - 1.0 : 0.0;   // n_e = n_e,p (1 + dn)
  const double x = rec ? ln_step(pr.x, dn, ne * NAV) : log(ne * NAV);
  const double ine = rec ? inv_step(pr.ine, dn, ne) : 1.0 / ne;
  const XB<double> X = xbasis<double>(t, x);
  YC<double, 1> c;
  c.j = -1;
  EosC f;
  if (rec && pr.icv > 0.0 && T > t.Tlo && T < t.Thi) {
    const double T1 = T + (eint - pr.e - pr.er * (rho - pr.rho)) * pr.icv;
    if (T1 > t.Tlo && T1 < t.Thi) {
      const double dT = (T1 - T) * pr.iT;   // T1 = T (1 + dT)
      const double lnT1 = ln_step(pr.lnT, dT, T1);
      if (!eos_rt_c(t, X, rho, irho, T1, lnT1, inv_step(pr.iT, dT, T1), iab, f, nullptr)) return -1;
      if (fabs(eint - f.e) < 2e-6 * fabs(eint)) {
        rec_carry(rho, eint, ine, x, T1, lnT1, f, o, T, pr);
        return 1;
      }
      T = T1;   // a larger change: the steps below from T1
    }
  }
  int it0 = -2;   // -2: a far guess, FP32 iterations first
  if (T > t.Tlo && T < t.Thi) {
    const double lnT = log(T);
    double e, cv;
    if (eos_ecv_xy<double>(t, X, c, irho, T, lnT, iab, e, cv) && fabs(eint - e) < 1e-4 * fabs(eint)) {
      const double de = eint - e;
      if (fabs(de) < 2e-6 * fabs(eint)) {
        const double T1 = T + de / cv;
        if (T1 > t.Tlo && T1 < t.Thi) {
          const double lnT1 = next_lnT<double>(T, lnT, T1);
          if (!eos_rt_c(t, X, rho, irho, T1, lnT1, 1.0 / T1, iab, f, &c)) return -1;
          rec_carry(rho, eint, ine, x, T1, lnT1, f, o, T, pr);
          return 2;
        }
      }
      it0 = newton_loop<double>(t, X, c, rho, irho, eint, iab, T, tol, maxit, o, true, e, cv, lnT);
    }
  }
  if (it0 == -2) {
    float Tf = (float)T;
    const int it32 = newton_fp32(t, (float)rho, (float)eint, (float)abar, (float)ye, Tf, 1e-5f, maxit < 12 ? maxit : 12);
    if (isfinite(Tf) && Tf > 0.0f) T = (double)Tf;
    const int it64 = newton_loop<double>(t, X, c, rho, irho, eint, iab, T, tol, maxit, o, false, 0.0, 0.0, 0.0);
    it0 = it64 < 0 ? -1 : it64 + (it32 > 0 ? it32 : 12);
  }
  if (it0 > 0)   // the record of a Newton-loop result (the rare paths)
    pr = Pred{rho, eint, 1.0 / o.cv, o.er, log(T), 1.0 / T, x, ine};
  return it0;
}

}  // namespace eos
}  // namespace phl
