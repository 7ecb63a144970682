// riemann.cuh -- face fluxes of the MHD stage, written in deviation form.
//
// The flux is returned as F - F_hat, where F_hat is the flux of the hydrostatic
// background state at the face (Sect. 2.8, Eq. wb1).  The background has u = 0
// and B = 0, so F_hat = (0, P_hat, 0, ..., 0) in the normal frame and the
// subtraction is done algebraically: every quantity that would otherwise be a
// difference of two background-sized numbers is carried as a deviation
// (Delta p_T = Delta P + B^2/2, E* - E written with (S_M - u) factors, ...).
// In FP64 this is the same function as F(W_L, W_R) - F_hat up to rounding; in
// FP32 it never subtracts two background-sized values.
//
// Solvers (Sect. 2.6):
//   HLLD  five-wave solver of Miyoshi & Kusano (2005): outer fast waves S_L,
//         S_R (Davis-type estimates), contact S_M, Alfven waves S*_L, S*_R,
//         intermediate states from the jump conditions; region choice as in
//         Eq. flux-hlld.
//   LHLLD the interface total pressure carries its dissipative part, the
//         (u_R - u_L) term of the HLLD intermediate pressure, scaled by
//         xi = max(M_L, M_R) when that Mach number (|u| / c_s) is below the
//         threshold (Eq. pstar and the text after it); inside the fan the
//         normal-momentum flux and its pressure work in the energy flux take
//         the scaled value.
//   HLL   two-wave solver used on shock-flagged faces (Sect. 2.7).
// Species: mass fractions are rescaled by their sum (Sect. 2.9, consistent
// multi-fluid advection) and advected with the mass flux of the side of the
// contact the flux is taken from.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define PHL_NSPEC_MAX 4

namespace phl {

// normal-frame deviation state indices
enum { RD_RHO = 0, RD_UN, RD_UT1, RD_UT2, RD_BT1, RD_BT2, RD_P, RD_GE, RD_GC, RD_X0 };
// normal-frame flux indices
enum { RF_RHO = 0, RF_MN, RF_MT1, RF_MT2, RF_E, RF_BT1, RF_BT2, RF_X0 };
enum { SOLVER_LHLLD = 0, SOLVER_HLLD = 1, SOLVER_HLL = 2 };

__device__ __forceinline__ double rsqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return sqrtf(x); }

template <typename R>
struct Side {
  R rho, un, ut1, ut2, bt1, bt2, p, ge;  // full rho, P, gamma_e
  R dpt;    // p_T - P_hat
  R enth;   // E + p_T (full)
  R de;     // E - E_hat
  R cf;
  R m2;     // |u|^2 / c_s^2
  R vb;     // u . B
  R F[7];   // physical flux minus background flux
};

// Ideal-gas constants of the flux (gamma, 1/(gamma-1), gamma/(gamma-1)); with
// IDEAL the indices are these constants instead of reconstructed values.
template <typename R>
struct GasK { R g, igm1, ggm1; };

template <typename R, bool IDEAL>
__device__ __forceinline__ void side_init(Side<R> &s, const R *w, R bn, R rh, R ph, R geh, R gch, const GasK<R> &K) {
  s.rho = rh + w[RD_RHO];
  s.un = w[RD_UN]; s.ut1 = w[RD_UT1]; s.ut2 = w[RD_UT2];
  s.bt1 = w[RD_BT1]; s.bt2 = w[RD_BT2];
  const R dp = w[RD_P];
  s.p = ph + dp;
  const R irho = R(1) / s.rho;
  const R b2 = bn * bn + s.bt1 * s.bt1 + s.bt2 * s.bt2;
  const R u2 = s.un * s.un + s.ut1 * s.ut1 + s.ut2 * s.ut2;
  const R half = R(0.5);
  s.dpt = dp + half * b2;
  const R kin = half * s.rho * u2;
  R gc;
  if (IDEAL) {
    // P / (gamma - 1) relative to P_hat / (gamma - 1)
    s.ge = K.g;
    gc = K.g;
    s.de = dp * K.igm1 + kin + half * b2;
    s.enth = K.ggm1 * s.p + kin + b2;
  } else {
    s.ge = geh + w[RD_GE];
    gc = gch + w[RD_GC];
    const R gem1 = s.ge - R(1);
    // internal energy density P / (gamma_e - 1) relative to P_hat / (gamma_hat_e - 1)
    R deint;
    if (ph == R(0)) {
      deint = s.p / gem1;
    } else {
      const R gehm1 = geh - R(1);
      deint = (dp * gehm1 - ph * w[RD_GE]) / (gem1 * gehm1);
    }
    s.de = deint + kin + half * b2;
    s.enth = s.ge / gem1 * s.p + kin + b2;
  }
  const R a2 = gc * s.p * irho;
  const R bb = b2 * irho, bnn = bn * bn * irho;
  R disc = (a2 + bb) * (a2 + bb) - R(4) * a2 * bnn;
  if (disc < R(0)) disc = R(0);
  s.cf = rsqrt_t(half * (a2 + bb + rsqrt_t(disc)));
  s.m2 = u2 / a2;
  s.vb = s.un * bn + s.ut1 * s.bt1 + s.ut2 * s.bt2;
  s.F[RF_RHO] = s.rho * s.un;
  s.F[RF_MN] = s.rho * s.un * s.un + s.dpt - bn * bn;
  s.F[RF_MT1] = s.rho * s.un * s.ut1 - bn * s.bt1;
  s.F[RF_MT2] = s.rho * s.un * s.ut2 - bn * s.bt2;
  s.F[RF_E] = s.enth * s.un - bn * s.vb;
  s.F[RF_BT1] = s.un * s.bt1 - s.ut1 * bn;
  s.F[RF_BT2] = s.un * s.bt2 - s.ut2 * bn;
}

// Differences U* - U of one side's HLLD intermediate state, plus the
// intermediate transverse velocity / field needed by the double-star states.
template <typename R>
__device__ __forceinline__ void star_diff(const Side<R> &s, R S, R SM, R dpts, R bn, R *dU, R &rhos,
                                          R &vs1, R &vs2, R &bs1, R &bs2) {
  const R su = S - s.un;           // S - u   (nonzero)
  const R q = S - SM;              // S - S_M (nonzero)
  const R iq = R(1) / q;
  const R smu = SM - s.un;
  rhos = s.rho * su * iq;
  const R den = s.rho * su * q - bn * bn;
  const R scale = s.rho * su * su + bn * bn;
  // degenerate case (den ~ 0): the transverse values stay those of the side;
  // selected rather than branched so that a warp's faces take one path
  const bool deg = fabs(den) < R(1e-12) * scale;
  const R iden = R(1) / den;
  const R fv = deg ? R(0) : bn * smu * iden;
  const R dbf = deg ? R(0) : s.rho * su * smu * iden;   // (B*_t - B_t) / B_t
  vs1 = s.ut1 - s.bt1 * fv;
  vs2 = s.ut2 - s.bt2 * fv;
  bs1 = s.bt1 + s.bt1 * dbf;
  bs2 = s.bt2 + s.bt2 * dbf;
  const R vbs = SM * bn + vs1 * bs1 + vs2 * bs2;
  dU[RF_RHO] = s.rho * smu * iq;                         // rho* - rho
  dU[RF_MN] = rhos * SM - s.rho * s.un;
  dU[RF_MT1] = rhos * vs1 - s.rho * s.ut1;
  dU[RF_MT2] = rhos * vs2 - s.rho * s.ut2;
  dU[RF_E] = (smu * s.enth + (dpts - s.dpt) * SM + bn * (s.vb - vbs)) * iq;   // E* - E
  dU[RF_BT1] = s.bt1 * dbf;
  dU[RF_BT2] = s.bt2 * dbf;
}

// Direction of the contact for Contact-CT upwinding: sign of the mass flux,
// 0 when |F_rho| <= 1e-12 rho max|S| (a mass flux at the rounding level of the
// face's flux scale carries no direction; the zero-flux rule then applies).
template <typename R>
__device__ __forceinline__ int contact_dir(R frho, R rhol, R rhor, R SL, R SR) {
  const R scale = R(1e-12) * fmax(rhol, rhor) * fmax(fabs(SL), fabs(SR));
  return frho > scale ? 1 : (frho < -scale ? -1 : 0);
}

// wl, wr: normal-frame deviation states (RD_* order) with nspec mass fractions.
// Background at the face: rh, ph, geh, gch (all 0 without a background).
// f: F - F_hat in RF_* order (7 + nspec values).
// NS: compile-time capacity for mass fractions (loops unroll; nspec <= NS).
template <typename R, int NS, bool IDEAL = false>
__device__ __forceinline__ void riemann_dev(const R *wl, const R *wr, R bn, R rh, R ph, R geh, R gch, int nspec,
                                            int solver, R mthr, R *f, int &up, const GasK<R> &K = GasK<R>{}) {
  Side<R> L, R_;
  side_init<R, IDEAL>(L, wl, bn, rh, ph, geh, gch, K);
  side_init<R, IDEAL>(R_, wr, bn, rh, ph, geh, gch, K);
  const R SL = fmin(L.un - L.cf, R_.un - R_.cf);
  const R SR = fmax(L.un + L.cf, R_.un + R_.cf);
  R xl[NS > 0 ? NS : 1], xr[NS > 0 ? NS : 1];
  {
    R sl = R(0), sr = R(0);
#pragma unroll
    for (int l = 0; l < NS; ++l)
      if (l < nspec) { sl += wl[RD_X0 + l]; sr += wr[RD_X0 + l]; }
#pragma unroll
    for (int l = 0; l < NS; ++l)
      if (l < nspec) { xl[l] = wl[RD_X0 + l] / sl; xr[l] = wr[RD_X0 + l] / sr; }
  }

  if (solver == SOLVER_HLL) {
    if (SL >= R(0)) {
      for (int q = 0; q < 7; ++q) f[q] = L.F[q];
#pragma unroll
      for (int l = 0; l < NS; ++l)
        if (l < nspec) f[RF_X0 + l] = L.F[RF_RHO] * xl[l];
    } else if (SR <= R(0)) {
      for (int q = 0; q < 7; ++q) f[q] = R_.F[q];
#pragma unroll
      for (int l = 0; l < NS; ++l)
        if (l < nspec) f[RF_X0 + l] = R_.F[RF_RHO] * xr[l];
    } else {
      R dU[7];
      dU[RF_RHO] = wr[RD_RHO] - wl[RD_RHO];
      dU[RF_MN] = R_.rho * R_.un - L.rho * L.un;
      dU[RF_MT1] = R_.rho * R_.ut1 - L.rho * L.ut1;
      dU[RF_MT2] = R_.rho * R_.ut2 - L.rho * L.ut2;
      dU[RF_E] = R_.de - L.de;
      dU[RF_BT1] = R_.bt1 - L.bt1;
      dU[RF_BT2] = R_.bt2 - L.bt2;
      const R idn = R(1) / (SR - SL);
      for (int q = 0; q < 7; ++q) f[q] = (SR * L.F[q] - SL * R_.F[q] + SL * SR * dU[q]) * idn;
#pragma unroll
      for (int l = 0; l < NS; ++l)
        if (l < nspec)
          f[RF_X0 + l] = (SR * L.F[RF_RHO] * xl[l] - SL * R_.F[RF_RHO] * xr[l] +
                          SL * SR * (R_.rho * xr[l] - L.rho * xl[l])) * idn;
    }
    up = contact_dir(f[RF_RHO], L.rho, R_.rho, SL, SR);
    return;
  }

  R xi = R(1);
  if (solver == SOLVER_LHLLD) {   // xi = max(M_L, M_R) below the threshold, M = |u| / c_s
    const R m2 = L.m2 > R_.m2 ? L.m2 : R_.m2;
    xi = m2 < mthr * mthr ? rsqrt_t(m2) : R(1);
  }
  const R sR = SR - R_.un, sL = SL - L.un;
  const R D = sR * R_.rho - sL * L.rho;
  const R iD = R(1) / D;
  const R SM = (sR * R_.rho * R_.un - sL * L.rho * L.un - R_.dpt + L.dpt) * iD;
  const R pdis = L.rho * R_.rho * sR * sL * (R_.un - L.un) * iD;
  const R dpts = (sR * R_.rho * L.dpt - sL * L.rho * R_.dpt) * iD + pdis;   // p_T* - P_hat

  // Region of the face (Eq. flux-hlld): outside the fan (S_L >= 0 or S_R < 0),
  // single-star (S*_L >= 0 or S*_R < 0) or double-star.  The flux is always
  // F_X + [fan] S_X (U*_X - U_X) + [double star] S*_X (U**_X - U*_X) with X the
  // side the region belongs to; every region's terms are computed and the
  // face's are selected, so the faces of a warp follow one instruction path.
  R dUL[7], dUR[7], rhosL, rhosR, vL1, vL2, bL1, bL2, vR1, vR2, bR1, bR2;
  star_diff(L, SL, SM, dpts, bn, dUL, rhosL, vL1, vL2, bL1, bL2);
  star_diff(R_, SR, SM, dpts, bn, dUR, rhosR, vR1, vR2, bR1, bR2);
  const R sqL = rsqrt_t(rhosL), sqR = rsqrt_t(rhosR);
  const R abn = fabs(bn);
  const R SsL = SM - abn / sqL, SsR = SM + abn / sqR;
  const bool outL = SL >= R(0), outR = !outL && SR < R(0), fan = !outL && !outR;
  const bool starL = SsL >= R(0), starR = !starL && SsR < R(0), dbl = fan && !starL && !starR;
  const bool left = outL || (fan && (starL || (!starR && SM >= R(0))));
  const R sgn = bn >= R(0) ? R(1) : R(-1);
  const R isum = R(1) / (sqL + sqR);
  const R vss1 = (sqL * vL1 + sqR * vR1 + (bR1 - bL1) * sgn) * isum;
  const R vss2 = (sqL * vL2 + sqR * vR2 + (bR2 - bL2) * sgn) * isum;
  const R bss1 = (sqL * bR1 + sqR * bL1 + sqL * sqR * (vR1 - vL1) * sgn) * isum;
  const R bss2 = (sqL * bR2 + sqR * bL2 + sqL * sqR * (vR2 - vL2) * sgn) * isum;
  const R vbss = SM * bn + vss1 * bss1 + vss2 * bss2;
  // the chosen side's quantities
  const R S = left ? SL : SR, Ss = left ? SsL : SsR, rhos = left ? rhosL : rhosR;
  const R sqs = left ? -sqL : sqR;
  const R v1 = left ? vL1 : vR1, v2 = left ? vL2 : vR2, b1 = left ? bL1 : bR1, b2 = left ? bL2 : bR2;
  const R vbs = SM * bn + v1 * b1 + v2 * b2;
  R d2[7];
  d2[RF_RHO] = R(0); d2[RF_MN] = R(0);
  d2[RF_MT1] = rhos * (vss1 - v1); d2[RF_MT2] = rhos * (vss2 - v2);
  d2[RF_E] = sqs * (vbs - vbss) * sgn;
  d2[RF_BT1] = bss1 - b1; d2[RF_BT2] = bss2 - b2;
  R F[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const R fx = left ? L.F[q] : R_.F[q];
    const R dux = left ? dUL[q] : dUR[q];
    const R t1 = fan ? S * dux : R(0);
    const R t2 = dbl ? Ss * d2[q] : R(0);
    F[q] = fx + t1 + t2;
  }
  // LHLLD: inside the fan the dissipative part of p_T* is scaled by xi
  if (fan && xi != R(1) && SR > R(0)) {
    F[RF_MN] += (xi - R(1)) * pdis;
    F[RF_E] += (xi - R(1)) * pdis * SM;
  }
  for (int q = 0; q < 7; ++q) f[q] = F[q];
#pragma unroll
  for (int l = 0; l < NS; ++l)
    if (l < nspec) f[RF_X0 + l] = F[RF_RHO] * (left ? xl[l] : xr[l]);
  up = contact_dir(F[RF_RHO], L.rho, R_.rho, SL, SR);
}

}  // namespace phl
