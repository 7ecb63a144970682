// mixed_common.cuh -- device bodies of the mixed-precision stage (FP32
// deviations, FP64 state), shared by the per-kernel path (kernels_mixed.cu)
// and the persistent ensemble path (ensemble.cu).
//
// State during a step: U^n in FP64 (cells and faces) and the stage increment
// dU = U^(s) - U^n in FP32.  SSP-RK stages (Sect. 2.9) with a + b = 1 give
//   U^(s) - U^n = b (U^(s-1) - U^n) - b dt R   =>   dU_out = b (dU_in - dt R),
// so every stage works on FP32 increments and only the last stage adds its
// increment into U^n in FP64.  Primitive deviations (Sect. 2.8) are formed
// from U^n - U_hat in FP64 (one subtraction each for rho and E) plus dU.
#pragma once
#include <math.h>

#include "phl_internal.cuh"
#include "stage_common.cuh"

namespace phl {
namespace stage {
namespace {

// The deviations of one cell from its conserved deviations and face fields
// in scaled FP32 units -- rho, u, B (face mean), P (Eq. energy), the gamma
// deviations -- the same operations in the same order for every caller.
// Returns 1/rho.
__device__ __forceinline__ float prims_mx_finish(const DevGeo &G, const BgT<float> &bf, float drho, float m0,
                                                 float m1, float m2, float dE, float bxl, float bxh, float byl,
                                                 float byh, float bzl, float bzh, float *w, int *dflag) {
  const float rho = bf.rho + drho;
  const float ir = 1.0f / rho;
  const float vx = m0 * ir, vy = m1 * ir, vz = m2 * ir;
  const float bx = 0.5f * (bxl + bxh), by = 0.5f * (byl + byh), bz = 0.5f * (bzl + bzh);
  const float gm1 = G.gm1f;
  const float dP = gm1 * (dE - 0.5f * rho * (vx * vx + vy * vy + vz * vz) - 0.5f * (bx * bx + by * by + bz * bz));
  w[W_RHO] = drho;
  w[W_VX] = vx; w[W_VY] = vy; w[W_VZ] = vz;
  w[W_BX] = bx; w[W_BY] = by; w[W_BZ] = bz;
  w[W_P] = dP;
  w[W_GE] = G.gammaf - bf.ge;
  w[W_GC] = G.gammaf - bf.gc;
  const float P = bf.p + dP;
  if (!(rho > 0.0f) || !(P > 0.0f)) atomicOr(dflag, FLAG_NEG);
  if (!isfinite(P) || !isfinite(rho)) atomicOr(dflag, FLAG_NAN);
  return ir;
}

// Deviations of the stage-input state at interior cell (i, j, k), in FP32.
__device__ __forceinline__ void cell_prims_mx(const DevGeo &G, const double *__restrict__ U,
                                              const double *__restrict__ Bf, const float *__restrict__ dU,
                                              const float *__restrict__ dB, int i, int j, int k, float *w,
                                              int *dflag) {
  const long p = sidx(G, i, j, k);
  const long pl = G.plane;
  const Bg b = bg_cell(G, k);                       // FP64 background for the deviations
  const double ehat = G.has_bg ? G.bg_e_c[k + BG_NG] : 0.0;
  // to scaled units: powers of two folded into the conversion (exact)
  const int kr = -G.e_rho, km = -G.e_m, ke = -G.e_e, kb = -G.e_b;
  float drho = d2f_scaled(U[p] - b.rho, kr);
  float m0 = d2f_scaled(U[pl + p], km), m1 = d2f_scaled(U[2 * pl + p], km), m2 = d2f_scaled(U[3 * pl + p], km);
  float dE = d2f_scaled(U[4 * pl + p] - ehat, ke);
  float bxl = d2f_scaled(Bf[p], kb), bxh = d2f_scaled(Bf[p + 1], kb);
  float byl = d2f_scaled(Bf[pl + p], kb), byh = d2f_scaled(Bf[pl + p + G.sy], kb);
  float bzl = d2f_scaled(Bf[2 * pl + p], kb), bzh = d2f_scaled(Bf[2 * pl + p + G.sz], kb);
  if (dU) {
    drho += dU[p];
    m0 += dU[pl + p]; m1 += dU[2 * pl + p]; m2 += dU[3 * pl + p];
    dE += dU[4 * pl + p];
  }
  if (dB) {
    bxl += dB[p]; bxh += dB[p + 1];
    byl += dB[pl + p]; byh += dB[pl + p + G.sy];
    bzl += dB[2 * pl + p]; bzh += dB[2 * pl + p + G.sz];
  }
  const float ir = prims_mx_finish(G, bg_cell_t<float>(G, k), drho, m0, m1, m2, dE, bxl, bxh, byl, byh, bzl, bzh,
                                   w, dflag);
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l) {
    if (l >= G.nspec) continue;
    float rx = d2f_scaled(U[(U_X0 + l) * pl + p], kr);
    if (dU) rx += dU[(U_X0 + l) * pl + p];
    w[W_X0 + l] = rx * ir;
  }
}

// CFL rate sum_d (|u_d| + c_f,d) / dx_d of a cell from its deviations w at
// height k, in scaled units.
__device__ __forceinline__ float dt_rate_w(const DevGeo &G, const float *w, int k) {
  const BgT<float> b = bg_cell_t<float>(G, k);
  const float rho = b.rho + w[W_RHO], P = b.p + w[W_P], gc = b.gc + w[W_GC];
  const float ir = 1.0f / rho;
  const float a2 = gc * P * ir;
  const float b2 = (w[W_BX] * w[W_BX] + w[W_BY] * w[W_BY] + w[W_BZ] * w[W_BZ]) * ir;
  float s = 0.0f;
  for (int d = 0; d < 3; ++d) {
    if (!G.act[d]) continue;
    const float bd2 = w[W_BX + d] * w[W_BX + d] * ir;
    float disc = (a2 + b2) * (a2 + b2) - 4.0f * a2 * bd2;
    disc = fmaxf(disc, 0.0f);
    const float cf = sqrtf(0.5f * (a2 + b2 + sqrtf(disc)));
    s += (fabsf(w[W_VX + d]) + cf) * G.idxf[d];
  }
  return (s == s) ? s : INFINITY;
}

// Deviations of work cell c (ghosts from their source cells, mirrored where
// a reflecting wall applies) stored into W and its auxiliary planes.  rate
// (optional): the CFL rate of an interior cell from the same deviations (the
// operations of dt_rate_mx), 0 for a ghost.
__device__ __forceinline__ void prim_store_cell(const DevGeo &G, const int *c, const double *__restrict__ U,
                                                const double *__restrict__ Bf, const float *__restrict__ dU,
                                                const float *__restrict__ dB, float *__restrict__ W, int *dflag,
                                                float *rate = nullptr) {
  int s[3];
  bool fl[3];
  bool in = true;
  for (int d = 0; d < 3; ++d) {
    fl[d] = false;
    s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]) : 0;
    in = in && c[d] >= 0 && c[d] < G.n[d];
  }
  float w[NW_MAX];
  cell_prims_mx(G, U, Bf, dU, dB, s[0], s[1], s[2], w, dflag);
  if (rate) *rate = in ? dt_rate_w(G, w, c[2]) : 0.0f;
  for (int d = 0; d < 3; ++d)
    if (fl[d]) { w[W_VX + d] = -w[W_VX + d]; w[W_BX + d] = -w[W_BX + d]; }
  const long q = widx(G, c[0], c[1], c[2]);
  if (G.wstr == 8) {   // ideal gas without species: the two float4 planes, one 16-byte store each
    float4 *W4 = reinterpret_cast<float4 *>(W);
    W4[q] = make_float4(w[W_RHO], w[W_VX], w[W_VY], w[W_VZ]);
    W4[G.wtot + q] = make_float4(w[W_BX], w[W_BY], w[W_BZ], w[W_P]);
  } else {
#pragma unroll
    for (int v = 0; v < NW_MAX; ++v)
      if (v < G.nw && v < G.wstr) W[wix<float>(G, v, q)] = w[v];
  }
  write_aux(G, W, q, w);
}

__device__ __forceinline__ void k_prim_mx_at(long tl, const DevGeo &G, const Box &box, const double *__restrict__ U, const double *__restrict__ Bf,
                          const float *__restrict__ dU, const float *__restrict__ dB, float *__restrict__ W,
                          int *dflag) {
  int c[3];
  if (!cell_at(box, tl, c)) return;
  prim_store_cell(G, c, U, Bf, dU, dB, W, dflag);
}

// Two neighbouring work cells of one row per thread: element (m, j, k) of
// hbox (x extent (n_x + 2 ge_x) / 2) is the pair x0 = 2m - ge_x, x0 + 1.  The
// thread reads the aligned state pair holding both cells' sources (each
// plane one FP64 pair, each increment plane one FP32 pair, the x-faces
// 2a .. 2a + 2), picks each cell's values by its offset in the pair and
// forms it with the operations of the single-cell path (bit-identical W),
// with no branch between interior and ghost pairs.
// CFL: also returns the larger CFL rate of the pair's interior cells (0 if
// none), from the same deviations (the operations of dt_rate_mx).
template <bool CFL>
__device__ __forceinline__ float k_prim_mx2_at(long tl, const DevGeo &G, const Box &hbox, const double *__restrict__ U,
                                               const double *__restrict__ Bf, const float *__restrict__ dU,
                                               const float *__restrict__ dB, float *__restrict__ W, int *dflag) {
  int c[3];
  if (!cell_at(hbox, tl, c)) return 0.0f;
  c[0] = 2 * c[0] - G.ge[0];
  bool flA = false, flB = false, fl[3] = {false, false, false};
  const int sA = cell_src(c[0], G.n[0], G.bc[0][0], G.bc[0][1], flA);
  const int sB = cell_src(c[0] + 1, G.n[0], G.bc[0][0], G.bc[0][1], flB);
  const int a0 = min(sA, sB) & ~1;
  const int oA = sA - a0, oB = sB - a0;   // 0 or 1
  const int j = G.act[1] ? cell_src(c[1], G.n[1], G.bc[1][0], G.bc[1][1], fl[1]) : 0;
  const int k = G.act[2] ? cell_src(c[2], G.n[2], G.bc[2][0], G.bc[2][1], fl[2]) : 0;
  const long p = sidx(G, a0, j, k);   // even
  const long pl = G.plane;
  auto ld2 = [](const double *a) { return *reinterpret_cast<const double2 *>(a); };
  auto lf2 = [](const float *a) { return *reinterpret_cast<const float2 *>(a); };
  auto pk = [](int o, double2 v) { return o ? v.y : v.x; };
  auto pf = [](int o, float2 v) { return o ? v.y : v.x; };
  const Bg b = bg_cell(G, k);
  const double ehat = G.has_bg ? G.bg_e_c[k + BG_NG] : 0.0;
  const int kr = -G.e_rho, km = -G.e_m, ke = -G.e_e, kb = -G.e_b;
  const double2 ur = ld2(U + p), u0 = ld2(U + pl + p), u1 = ld2(U + 2 * pl + p), u2 = ld2(U + 3 * pl + p),
                ue = ld2(U + 4 * pl + p);
  const double2 fx = ld2(Bf + p), fyl = ld2(Bf + pl + p), fyh = ld2(Bf + pl + p + G.sy), fzl = ld2(Bf + 2 * pl + p),
                fzh = ld2(Bf + 2 * pl + p + G.sz);
  const double fx2 = Bf[p + 2];
  // the x-faces of state cell a0 + o are x-faces o and o + 1 of the three
  auto xf = [&](int f) { return f == 0 ? fx.x : (f == 1 ? fx.y : fx2); };
  float drA = d2f_scaled(pk(oA, ur) - b.rho, kr), drB = d2f_scaled(pk(oB, ur) - b.rho, kr);
  float m0A = d2f_scaled(pk(oA, u0), km), m0B = d2f_scaled(pk(oB, u0), km);
  float m1A = d2f_scaled(pk(oA, u1), km), m1B = d2f_scaled(pk(oB, u1), km);
  float m2A = d2f_scaled(pk(oA, u2), km), m2B = d2f_scaled(pk(oB, u2), km);
  float dEA = d2f_scaled(pk(oA, ue) - ehat, ke), dEB = d2f_scaled(pk(oB, ue) - ehat, ke);
  float bxlA = d2f_scaled(xf(oA), kb), bxhA = d2f_scaled(xf(oA + 1), kb);
  float bxlB = d2f_scaled(xf(oB), kb), bxhB = d2f_scaled(xf(oB + 1), kb);
  float bylA = d2f_scaled(pk(oA, fyl), kb), bylB = d2f_scaled(pk(oB, fyl), kb);
  float byhA = d2f_scaled(pk(oA, fyh), kb), byhB = d2f_scaled(pk(oB, fyh), kb);
  float bzlA = d2f_scaled(pk(oA, fzl), kb), bzlB = d2f_scaled(pk(oB, fzl), kb);
  float bzhA = d2f_scaled(pk(oA, fzh), kb), bzhB = d2f_scaled(pk(oB, fzh), kb);
  if (dU) {
    const float2 r = lf2(dU + p), a = lf2(dU + pl + p), bb = lf2(dU + 2 * pl + p), cc = lf2(dU + 3 * pl + p),
                 e = lf2(dU + 4 * pl + p);
    drA += pf(oA, r); drB += pf(oB, r);
    m0A += pf(oA, a); m0B += pf(oB, a);
    m1A += pf(oA, bb); m1B += pf(oB, bb);
    m2A += pf(oA, cc); m2B += pf(oB, cc);
    dEA += pf(oA, e); dEB += pf(oB, e);
  }
  if (dB) {
    const float2 x = lf2(dB + p), yl = lf2(dB + pl + p), yh = lf2(dB + pl + p + G.sy), zl = lf2(dB + 2 * pl + p),
                 zh = lf2(dB + 2 * pl + p + G.sz);
    const float x2 = dB[p + 2];
    auto dxf = [&](int f) { return f == 0 ? x.x : (f == 1 ? x.y : x2); };
    bxlA += dxf(oA); bxhA += dxf(oA + 1); bxlB += dxf(oB); bxhB += dxf(oB + 1);
    bylA += pf(oA, yl); bylB += pf(oB, yl); byhA += pf(oA, yh); byhB += pf(oB, yh);
    bzlA += pf(oA, zl); bzlB += pf(oB, zl); bzhA += pf(oA, zh); bzhB += pf(oB, zh);
  }
  const BgT<float> bf = bg_cell_t<float>(G, k);
  float wA[NW_MAX], wB[NW_MAX];
  prims_mx_finish(G, bf, drA, m0A, m1A, m2A, dEA, bxlA, bxhA, bylA, byhA, bzlA, bzhA, wA, dflag);
  prims_mx_finish(G, bf, drB, m0B, m1B, m2B, dEB, bxlB, bxhB, bylB, byhB, bzlB, bzhB, wB, dflag);
  float rate = 0.0f;
  if (CFL) {
    const bool row = (!G.act[1] || (c[1] >= 0 && c[1] < G.n[1])) && (!G.act[2] || (c[2] >= 0 && c[2] < G.n[2]));
    if (row && c[0] >= 0 && c[0] < G.n[0]) rate = dt_rate_w(G, wA, c[2]);
    if (row && c[0] + 1 >= 0 && c[0] + 1 < G.n[0]) rate = fmaxf(rate, dt_rate_w(G, wB, c[2]));
  }
  if (flA) { wA[W_VX] = -wA[W_VX]; wA[W_BX] = -wA[W_BX]; }
  if (flB) { wB[W_VX] = -wB[W_VX]; wB[W_BX] = -wB[W_BX]; }
  for (int d = 1; d < 3; ++d)
    if (fl[d]) {
      wA[W_VX + d] = -wA[W_VX + d]; wA[W_BX + d] = -wA[W_BX + d];
      wB[W_VX + d] = -wB[W_VX + d]; wB[W_BX + d] = -wB[W_BX + d];
    }
  const long q = widx(G, c[0], c[1], c[2]);
  float4 *W4 = reinterpret_cast<float4 *>(W);
  W4[q] = make_float4(wA[W_RHO], wA[W_VX], wA[W_VY], wA[W_VZ]);
  W4[q + 1] = make_float4(wB[W_RHO], wB[W_VX], wB[W_VY], wB[W_VZ]);
  W4[G.wtot + q] = make_float4(wA[W_BX], wA[W_BY], wA[W_BZ], wA[W_P]);
  W4[G.wtot + q + 1] = make_float4(wB[W_BX], wB[W_BY], wB[W_BZ], wB[W_P]);
  write_aux(G, W, q, wA);
  write_aux(G, W, q + 1, wB);
  return rate;
}

struct StageMx {
  double *U, *B;          // U^n (updated in place by the last stage)
  float *dU, *dB;         // stage increments (in place)
  bool first, last;       // first stage: dU_in = 0; last: fold into U^n
  float b;                // RK coefficient of the stage
  const double *dt;
  const float *W, *F[3], *E;
};

__device__ __forceinline__ void k_update_cells_mx_at(long tl, const DevGeo &G, const Box &box, StageMx S) {
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  {
    int c[3];
    if (!cell_at(box, tl, c)) return;
    const long p = widx(G, c[0], c[1], c[2]);
    const long ps = sidx(G, c[0], c[1], c[2]);
    const long wt = G.wtot, pl = G.plane;
    float r[5 + PHL_NSPEC_MAX];
#pragma unroll
    for (int v = 0; v < 5 + PHL_NSPEC_MAX; ++v) {
      if (v >= G.nv) continue;
      const int fc = v < 5 ? v : F_X0 + (v - U_X0);
      float s = 0.0f;
      for (int d = 0; d < 3; ++d) {
        if (!G.act[d]) continue;
        const float *f = S.F[d] + fc * wt;
        s += (f[p + (d == 0 ? 1L : (d == 1 ? G.wy : G.wz))] - f[p]) * G.idxf[d];
      }
      r[v] = s;
    }
    // sources S - S_hat: (rho - rho_hat) g on momentum, rho u . g (+ heating) on energy
    const float drho = S.W[wix<float>(G, W_RHO, p)];
    const float rho = bg_cell_t<float>(G, c[2]).rho + drho;
    float se = 0.0f;
    for (int d = 0; d < 3; ++d) {
      const float gd = G.gf[d];
      r[U_MX + d] -= drho * gd;
      se += rho * S.W[wix<float>(G, W_VX + d, p)] * gd;
    }
    if (G.heatf) se += G.heatf[c[2]];
    r[U_E] -= se;
#pragma unroll
    for (int v = 0; v < 5 + PHL_NSPEC_MAX; ++v) {
      if (v >= G.nv) continue;
      const long q = v * pl + ps;
      const float din = S.first ? 0.0f : S.dU[q];
      const float dout = S.b * (din - dt * r[v]);
      if (S.last) S.U[q] += f2d_scaled(dout, uexp(G, v));
      else S.dU[q] = dout;
    }
  }
}

template <int D>
__device__ __forceinline__ void k_update_faces_mx_at(long tl, const DevGeo &G, const Box &box, StageMx S) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  {
    int c[3];
    if (!cell_at(box, tl, c)) return;
    int e[3] = {c[0], c[1], c[2]};
    if (!G.act[D]) e[D] = 0;
    const long p = widx(G, e[0], e[1], e[2]);
    const long wt = G.wtot;
    float r = 0.0f;
    if (G.act[A]) r += (S.E[(long)B * wt + p + wstride(G, A)] - S.E[(long)B * wt + p]) * G.idxf[A];
    if (G.act[B]) r -= (S.E[(long)A * wt + p + wstride(G, B)] - S.E[(long)A * wt + p]) * G.idxf[B];
    const long q = (long)D * G.plane + sidx(G, c[0], c[1], c[2]);
    const float din = S.first ? 0.0f : S.dB[q];
    const float dout = S.b * (din - dt * r);
    if (S.last) S.B[q] += f2d_scaled(dout, G.e_b);
    else S.dB[q] = dout;
  }
}


// CFL rate of one interior cell of U^n, in scaled units.
__device__ __forceinline__ float dt_rate_mx(const DevGeo &G, const double *__restrict__ U,
                                            const double *__restrict__ Bf, const int *c, int *dflag) {
  float w[NW_MAX];
  cell_prims_mx(G, U, Bf, nullptr, nullptr, c[0], c[1], c[2], w, dflag);
  return dt_rate_w(G, w, c[2]);
}

}  // namespace
}  // namespace stage
}  // namespace phl
