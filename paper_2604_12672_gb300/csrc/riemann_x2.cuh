// riemann_x2.cuh -- the ideal-gas face flux of riemann.cuh for two faces at
// once, on Blackwell's packed FP32x2 arithmetic.
//
// Same method, same formulas and the same deviation form as riemann_dev with
// IDEAL = true and no mass fractions (Sects. 2.6-2.8): Davis wave speeds, the
// HLLD intermediate states of Miyoshi & Kusano, the LHLLD scaling of the
// dissipative part of the interface total pressure by xi = max(M_L, M_R) below
// the Mach threshold, and the HLL flux on shock-flagged faces.  Each value is
// a pair (lane x = first face, lane y = second face); additions,
// subtractions, multiplications and fused multiply-adds of pairs are single
// add/sub/mul/fma.rn.ftz.f32x2 instructions, while reciprocals, square roots,
// comparisons and selections act on each lane.  Products that the scalar
// solver leaves to the compiler's contraction are written here as explicit
// FMAs, so the two agree to FP32 rounding, not bit for bit.
#pragma once
#include <cuda_runtime.h>

#include "riemann.cuh"

namespace phl {
namespace x2 {

struct V {
  float x, y;
};
struct B2 {
  bool x, y;
};

__device__ __forceinline__ V vv(float a) { return V{a, a}; }
__device__ __forceinline__ V vv(float a, float b) { return V{a, b}; }

__device__ __forceinline__ V operator+(V a, V b) {
  V r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ V operator-(V a, V b) {
  V r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ V operator*(V a, V b) {
  V r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "mul.rn.ftz.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ V fma(V a, V b, V c) {
  V r;
  asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "mov.b64 pc, {%6, %7};\n\tfma.rn.ftz.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ V neg(V a) { return V{-a.x, -a.y}; }
__device__ __forceinline__ V rcp(V a) { return V{1.0f / a.x, 1.0f / a.y}; }
__device__ __forceinline__ V sqrt2(V a) { return V{sqrtf(a.x), sqrtf(a.y)}; }
__device__ __forceinline__ V vabs(V a) { return V{fabsf(a.x), fabsf(a.y)}; }
__device__ __forceinline__ V vmin(V a, V b) { return V{fminf(a.x, b.x), fminf(a.y, b.y)}; }
__device__ __forceinline__ V vmax(V a, V b) { return V{fmaxf(a.x, b.x), fmaxf(a.y, b.y)}; }
__device__ __forceinline__ B2 operator>=(V a, V b) { return B2{a.x >= b.x, a.y >= b.y}; }
__device__ __forceinline__ B2 operator>(V a, V b) { return B2{a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ B2 operator<(V a, V b) { return B2{a.x < b.x, a.y < b.y}; }
__device__ __forceinline__ B2 operator&&(B2 a, B2 b) { return B2{a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ B2 operator||(B2 a, B2 b) { return B2{a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ B2 operator!(B2 a) { return B2{!a.x, !a.y}; }
__device__ __forceinline__ V sel(B2 c, V a, V b) { return V{c.x ? a.x : b.x, c.y ? a.y : b.y}; }

// One side of the face: full rho and P, deviations of the total pressure and
// energy, fast speed, Mach number squared, u.B and the physical flux minus
// the background flux (as Side in riemann.cuh).
struct SideV {
  V rho, un, ut1, ut2, bt1, bt2;
  V dpt, enth, de, cf, m2, vb;
  V F[7];
};

__device__ __forceinline__ void side_init_v(SideV &s, const V *w, V bn, V rh, V ph, const GasK<float> &K) {
  const V half = vv(0.5f);
  s.rho = rh + w[RD_RHO];
  s.un = w[RD_UN]; s.ut1 = w[RD_UT1]; s.ut2 = w[RD_UT2];
  s.bt1 = w[RD_BT1]; s.bt2 = w[RD_BT2];
  const V dp = w[RD_P];
  const V p = ph + dp;
  const V irho = rcp(s.rho);
  const V bn2 = bn * bn;
  const V b2 = fma(s.bt2, s.bt2, fma(s.bt1, s.bt1, bn2));
  const V u2 = fma(s.ut2, s.ut2, fma(s.ut1, s.ut1, s.un * s.un));
  s.dpt = fma(half, b2, dp);
  const V kin = (half * s.rho) * u2;
  s.de = fma(half, b2, fma(dp, vv(K.igm1), kin));
  s.enth = fma(vv(K.ggm1), p, kin) + b2;
  const V a2 = (vv(K.g) * p) * irho;
  const V bb = b2 * irho, bnn = bn2 * irho;
  const V ab = a2 + bb;
  V disc = fma(ab, ab, neg(vv(4.0f) * a2 * bnn));
  disc = vmax(disc, vv(0.0f));
  s.cf = sqrt2(half * (ab + sqrt2(disc)));
  s.m2 = u2 * rcp(a2);
  s.vb = fma(s.ut2, s.bt2, fma(s.ut1, s.bt1, s.un * bn));
  s.F[RF_RHO] = s.rho * s.un;
  s.F[RF_MN] = fma(s.F[RF_RHO], s.un, s.dpt - bn2);
  s.F[RF_MT1] = fma(s.F[RF_RHO], s.ut1, neg(bn * s.bt1));
  s.F[RF_MT2] = fma(s.F[RF_RHO], s.ut2, neg(bn * s.bt2));
  s.F[RF_E] = fma(s.enth, s.un, neg(bn * s.vb));
  s.F[RF_BT1] = fma(s.un, s.bt1, neg(s.ut1 * bn));
  s.F[RF_BT2] = fma(s.un, s.bt2, neg(s.ut2 * bn));
}

// U* - U of one side and its intermediate transverse velocity and field (as
// star_diff in riemann.cuh).
__device__ __forceinline__ void star_diff_v(const SideV &s, V S, V SM, V dpts, V bn, V *dU, V &rhos, V &vs1, V &vs2,
                                            V &bs1, V &bs2) {
  const V su = S - s.un;
  const V q = S - SM;
  const V iq = rcp(q);
  const V smu = SM - s.un;
  const V rsu = s.rho * su;
  rhos = rsu * iq;
  const V bn2 = bn * bn;
  const V den = fma(rsu, q, neg(bn2));
  const V scale = fma(rsu, su, bn2);
  const B2 deg = vabs(den) < vv(1e-12f) * scale;
  const V iden = rcp(den);
  const V fv = sel(deg, vv(0.0f), bn * smu * iden);
  const V dbf = sel(deg, vv(0.0f), rsu * smu * iden);
  vs1 = fma(neg(s.bt1), fv, s.ut1);
  vs2 = fma(neg(s.bt2), fv, s.ut2);
  bs1 = fma(s.bt1, dbf, s.bt1);
  bs2 = fma(s.bt2, dbf, s.bt2);
  const V vbs = fma(vs2, bs2, fma(vs1, bs1, SM * bn));
  dU[RF_RHO] = s.rho * smu * iq;
  dU[RF_MN] = fma(rhos, SM, neg(s.rho * s.un));
  dU[RF_MT1] = fma(rhos, vs1, neg(s.rho * s.ut1));
  dU[RF_MT2] = fma(rhos, vs2, neg(s.rho * s.ut2));
  dU[RF_E] = fma(bn, s.vb - vbs, fma(dpts - s.dpt, SM, smu * s.enth)) * iq;
  dU[RF_BT1] = s.bt1 * dbf;
  dU[RF_BT2] = s.bt2 * dbf;
}

// Contact direction per lane (contact_dir in riemann.cuh).
__device__ __forceinline__ void contact_dir_v(V frho, V rl, V rr, V SL, V SR, int &ux, int &uy) {
  const V scale = vv(1e-12f) * vmax(rl, rr) * vmax(vabs(SL), vabs(SR));
  ux = frho.x > scale.x ? 1 : (frho.x < -scale.x ? -1 : 0);
  uy = frho.y > scale.y ? 1 : (frho.y < -scale.y ? -1 : 0);
}

// Two faces' F - F_hat (7 components, RF_* order) and contact directions.
// wl, wr: normal-frame deviation states (RD_RHO .. RD_P); bn: normal field;
// rh, ph: background density and pressure at each face; hll: per face, the
// shock-flagged HLL solver instead of `solver`.
__device__ __forceinline__ void riemann_ideal_x2(const V *wl, const V *wr, V bn, V rh, V ph, B2 hll, int solver,
                                                 float mthr, V *f, int &upx, int &upy, const GasK<float> &K) {
  SideV L, R;
  side_init_v(L, wl, bn, rh, ph, K);
  side_init_v(R, wr, bn, rh, ph, K);
  const V SL = vmin(L.un - L.cf, R.un - R.cf);
  const V SR = vmax(L.un + L.cf, R.un + R.cf);
  const V zero = vv(0.0f), one = vv(1.0f);

  // LHLLD / HLLD for both lanes
  V xi = one;
  if (solver == SOLVER_LHLLD) {
    const V m2 = vmax(L.m2, R.m2);
    xi = sel(m2 < vv(mthr * mthr), sqrt2(m2), one);
  }
  const V sR = SR - R.un, sL = SL - L.un;
  const V rsR = sR * R.rho, rsL = sL * L.rho;
  const V Dn = rsR - rsL;
  const V iD = rcp(Dn);
  const V SM = (fma(rsR, R.un, neg(rsL * L.un)) - R.dpt + L.dpt) * iD;
  const V pdis = L.rho * R.rho * sR * sL * (R.un - L.un) * iD;
  const V dpts = fma(fma(rsR, L.dpt, neg(rsL * R.dpt)), iD, pdis);
  V dUL[7], dUR[7], rhosL, rhosR, vL1, vL2, bL1, bL2, vR1, vR2, bR1, bR2;
  star_diff_v(L, SL, SM, dpts, bn, dUL, rhosL, vL1, vL2, bL1, bL2);
  star_diff_v(R, SR, SM, dpts, bn, dUR, rhosR, vR1, vR2, bR1, bR2);
  const V sqL = sqrt2(rhosL), sqR = sqrt2(rhosR);
  const V abn = vabs(bn);
  const V SsL = SM - abn * rcp(sqL), SsR = SM + abn * rcp(sqR);
  const B2 outL = SL >= zero, outR = !outL && (SR < zero), fan = !outL && !outR;
  const B2 starL = SsL >= zero, starR = !starL && (SsR < zero), dbl = fan && !starL && !starR;
  const B2 left = outL || (fan && (starL || (!starR && (SM >= zero))));
  const V sgn = sel(bn >= zero, one, vv(-1.0f));
  const V isum = rcp(sqL + sqR);
  const V vss1 = fma(bR1 - bL1, sgn, fma(sqR, vR1, sqL * vL1)) * isum;
  const V vss2 = fma(bR2 - bL2, sgn, fma(sqR, vR2, sqL * vL2)) * isum;
  const V sqLR = sqL * sqR;
  const V bss1 = fma(sqLR * (vR1 - vL1), sgn, fma(sqR, bL1, sqL * bR1)) * isum;
  const V bss2 = fma(sqLR * (vR2 - vL2), sgn, fma(sqR, bL2, sqL * bR2)) * isum;
  const V vbss = fma(vss2, bss2, fma(vss1, bss1, SM * bn));
  const V S = sel(left, SL, SR), Ss = sel(left, SsL, SsR), rhos = sel(left, rhosL, rhosR);
  const V sqs = sel(left, neg(sqL), sqR);
  const V v1 = sel(left, vL1, vR1), v2 = sel(left, vL2, vR2), b1 = sel(left, bL1, bR1), b2 = sel(left, bL2, bR2);
  const V vbs = fma(v2, b2, fma(v1, b1, SM * bn));
  V d2[7];
  d2[RF_RHO] = zero; d2[RF_MN] = zero;
  d2[RF_MT1] = rhos * (vss1 - v1); d2[RF_MT2] = rhos * (vss2 - v2);
  d2[RF_E] = sqs * (vbs - vbss) * sgn;
  d2[RF_BT1] = bss1 - b1; d2[RF_BT2] = bss2 - b2;
  // F = F_X + [fan] S_X (U*_X - U_X) + [double star] S*_X (U**_X - U*_X)
  // (outside the fan the flux is F_X itself: selected, not multiplied by
  // zero, so that an unused intermediate state can never leak into it)
  const V Ssd = sel(dbl, Ss, zero);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const V fx = sel(left, L.F[q], R.F[q]);
    const V dux = sel(left, dUL[q], dUR[q]);
    f[q] = sel(fan, fma(Ssd, d2[q], fma(S, dux, fx)), fx);
  }
  // LHLLD: inside the fan the dissipative part of p_T* is scaled by xi
  {
    const B2 lo = fan && B2{xi.x != 1.0f, xi.y != 1.0f} && (SR > zero);
    const V c = (xi - one) * pdis;
    f[RF_MN] = sel(lo, f[RF_MN] + c, f[RF_MN]);
    f[RF_E] = sel(lo, fma(c, SM, f[RF_E]), f[RF_E]);
  }

  if (hll.x || hll.y) {   // shock-flagged faces: the two-wave HLL flux
    V h[7];
    const B2 oL = SL >= zero;
    const B2 rOut = B2{SR.x <= 0.0f, SR.y <= 0.0f};
    V dU[7];
    dU[RF_RHO] = wr[RD_RHO] - wl[RD_RHO];
    dU[RF_MN] = fma(R.rho, R.un, neg(L.rho * L.un));
    dU[RF_MT1] = fma(R.rho, R.ut1, neg(L.rho * L.ut1));
    dU[RF_MT2] = fma(R.rho, R.ut2, neg(L.rho * L.ut2));
    dU[RF_E] = R.de - L.de;
    dU[RF_BT1] = R.bt1 - L.bt1;
    dU[RF_BT2] = R.bt2 - L.bt2;
    const V idn = rcp(SR - SL);
    const V sLR = SL * SR;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const V mid = fma(sLR, dU[q], fma(SR, L.F[q], neg(SL * R.F[q]))) * idn;
      h[q] = sel(oL, L.F[q], sel(rOut, R.F[q], mid));
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) f[q] = sel(hll, h[q], f[q]);
  }
  contact_dir_v(f[RF_RHO], L.rho, R.rho, SL, SR, upx, upy);
}

}  // namespace x2
}  // namespace phl

namespace phl {
namespace x2 {

// ---------------------------------------------------------------------------
// One face, its left and right states as the two lanes (lane x = L, lane y =
// R).  The side quantities, the fast speeds, the physical fluxes and both
// HLLD intermediate states are the same arithmetic on each side, so they run
// as packed pairs without doubling the live state; everything that mixes the
// sides (wave speeds, S_M, p_T*, the double-star states, the region choice)
// stays scalar.  Same method and formulas as riemann_dev with IDEAL = true.

__device__ __forceinline__ void sides_init_lr(SideV &s, const float *wl, const float *wr, float bn, float rh, float ph,
                                              const GasK<float> &K) {
  const float w2[RD_P + 1][2] = {{wl[RD_RHO], wr[RD_RHO]}, {wl[RD_UN], wr[RD_UN]}, {wl[RD_UT1], wr[RD_UT1]},
                                 {wl[RD_UT2], wr[RD_UT2]}, {wl[RD_BT1], wr[RD_BT1]}, {wl[RD_BT2], wr[RD_BT2]},
                                 {wl[RD_P], wr[RD_P]}};
  V w[RD_P + 1];
#pragma unroll
  for (int q = 0; q <= RD_P; ++q) w[q] = vv(w2[q][0], w2[q][1]);
  side_init_v(s, w, vv(bn), vv(rh), vv(ph), K);
}

__device__ __forceinline__ void riemann_ideal_lr(const float *wl, const float *wr, float bn, float rh, float ph,
                                                 int solver, float mthr, float *f, int &up, const GasK<float> &K) {
  SideV s;   // lane x: left side, lane y: right side
  sides_init_lr(s, wl, wr, bn, rh, ph, K);
  const V lo = s.un - s.cf, hi = s.un + s.cf;
  const float SL = fminf(lo.x, lo.y), SR = fmaxf(hi.x, hi.y);
  if (solver == SOLVER_HLL) {
    if (SL >= 0.0f) {
#pragma unroll
      for (int q = 0; q < 7; ++q) f[q] = s.F[q].x;
    } else if (SR <= 0.0f) {
#pragma unroll
      for (int q = 0; q < 7; ++q) f[q] = s.F[q].y;
    } else {
      const V m = s.rho * s.un, m1 = s.rho * s.ut1, m2 = s.rho * s.ut2;
      float dU[7];
      dU[RF_RHO] = wr[RD_RHO] - wl[RD_RHO];
      dU[RF_MN] = m.y - m.x;
      dU[RF_MT1] = m1.y - m1.x;
      dU[RF_MT2] = m2.y - m2.x;
      dU[RF_E] = s.de.y - s.de.x;
      dU[RF_BT1] = s.bt1.y - s.bt1.x;
      dU[RF_BT2] = s.bt2.y - s.bt2.x;
      const float idn = 1.0f / (SR - SL);
#pragma unroll
      for (int q = 0; q < 7; ++q) f[q] = (SR * s.F[q].x - SL * s.F[q].y + SL * SR * dU[q]) * idn;
    }
    const float scale = 1e-12f * fmaxf(s.rho.x, s.rho.y) * fmaxf(fabsf(SL), fabsf(SR));
    up = f[RF_RHO] > scale ? 1 : (f[RF_RHO] < -scale ? -1 : 0);
    return;
  }
  float xi = 1.0f;
  if (solver == SOLVER_LHLLD) {
    const float m2 = fmaxf(s.m2.x, s.m2.y);
    xi = m2 < mthr * mthr ? sqrtf(m2) : 1.0f;
  }
  const V S2 = vv(SL, SR);
  const V sv = S2 - s.un;            // (S_L - u_L, S_R - u_R)
  const V rs = sv * s.rho;
  const float iD = 1.0f / (rs.y - rs.x);
  const V rsu = rs * s.un;
  const float SM = (rsu.y - rsu.x - s.dpt.y + s.dpt.x) * iD;
  const float pdis = s.rho.x * s.rho.y * sv.y * sv.x * (s.un.y - s.un.x) * iD;
  const float dpts = (rs.y * s.dpt.x - rs.x * s.dpt.y) * iD + pdis;   // p_T* - P_hat
  // both sides' HLLD intermediate states (star_diff of riemann.cuh, paired)
  const V SMv = vv(SM), bnv = vv(bn);
  const V qv = S2 - SMv;
  const V iq = rcp(qv);
  const V smu = SMv - s.un;
  const V rhos = rs * iq;
  const float bn2 = bn * bn;
  const V den = fma(rs, qv, vv(-bn2));
  const V scl = fma(rs, sv, vv(bn2));
  const B2 deg = vabs(den) < vv(1e-12f) * scl;
  const V iden = rcp(den);
  const V fv = sel(deg, vv(0.0f), bnv * smu * iden);
  const V dbf = sel(deg, vv(0.0f), rs * smu * iden);
  const V vs1 = fma(neg(s.bt1), fv, s.ut1), vs2 = fma(neg(s.bt2), fv, s.ut2);
  const V bs1 = fma(s.bt1, dbf, s.bt1), bs2 = fma(s.bt2, dbf, s.bt2);
  const V vbs = fma(vs2, bs2, fma(vs1, bs1, SMv * bnv));
  V dU[7];
  dU[RF_RHO] = s.rho * smu * iq;
  dU[RF_MN] = fma(rhos, SMv, neg(s.rho * s.un));
  dU[RF_MT1] = fma(rhos, vs1, neg(s.rho * s.ut1));
  dU[RF_MT2] = fma(rhos, vs2, neg(s.rho * s.ut2));
  dU[RF_E] = fma(bnv, s.vb - vbs, fma(vv(dpts) - s.dpt, SMv, smu * s.enth)) * iq;
  dU[RF_BT1] = s.bt1 * dbf;
  dU[RF_BT2] = s.bt2 * dbf;
  const V sq = sqrt2(rhos);
  const float abn = fabsf(bn);
  const V Ss = fma(vv(-abn, abn), rcp(sq), SMv);   // (S*_L, S*_R)
  const bool outL = SL >= 0.0f, outR = !outL && SR < 0.0f, fan = !outL && !outR;
  const bool starL = Ss.x >= 0.0f, starR = !starL && Ss.y < 0.0f, dbl = fan && !starL && !starR;
  const bool left = outL || (fan && (starL || (!starR && SM >= 0.0f)));
  const float sgn = bn >= 0.0f ? 1.0f : -1.0f;
  const float isum = 1.0f / (sq.x + sq.y);
  const V sqv1 = sq * vs1, sqv2 = sq * vs2;
  const float vss1 = (sqv1.x + sqv1.y + (bs1.y - bs1.x) * sgn) * isum;
  const float vss2 = (sqv2.x + sqv2.y + (bs2.y - bs2.x) * sgn) * isum;
  const float sqLR = sq.x * sq.y;
  const float bss1 = (sq.x * bs1.y + sq.y * bs1.x + sqLR * (vs1.y - vs1.x) * sgn) * isum;
  const float bss2 = (sq.x * bs2.y + sq.y * bs2.x + sqLR * (vs2.y - vs2.x) * sgn) * isum;
  const float vbss = SM * bn + vss1 * bss1 + vss2 * bss2;
  auto pick = [&](const V &v) { return left ? v.x : v.y; };
  const float S = left ? SL : SR, Ssx = pick(Ss), rhosx = pick(rhos);
  const float sqs = left ? -sq.x : sq.y;
  const float v1 = pick(vs1), v2 = pick(vs2), b1 = pick(bs1), b2 = pick(bs2);
  const float vbsx = SM * bn + v1 * b1 + v2 * b2;
  float d2[7];
  d2[RF_RHO] = 0.0f; d2[RF_MN] = 0.0f;
  d2[RF_MT1] = rhosx * (vss1 - v1); d2[RF_MT2] = rhosx * (vss2 - v2);
  d2[RF_E] = sqs * (vbsx - vbss) * sgn;
  d2[RF_BT1] = bss1 - b1; d2[RF_BT2] = bss2 - b2;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const float fx = pick(s.F[q]);
    const float t1 = fan ? S * pick(dU[q]) : 0.0f;
    const float t2 = dbl ? Ssx * d2[q] : 0.0f;
    f[q] = fx + t1 + t2;
  }
  // LHLLD: inside the fan the dissipative part of p_T* is scaled by xi
  if (fan && xi != 1.0f && SR > 0.0f) {
    f[RF_MN] += (xi - 1.0f) * pdis;
    f[RF_E] += (xi - 1.0f) * pdis * SM;
  }
  const float scale = 1e-12f * fmaxf(s.rho.x, s.rho.y) * fmaxf(fabsf(SL), fabsf(SR));
  up = f[RF_RHO] > scale ? 1 : (f[RF_RHO] < -scale ? -1 : 0);
}

}  // namespace x2
}  // namespace phl
