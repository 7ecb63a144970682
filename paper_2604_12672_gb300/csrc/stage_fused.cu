// stage_fused.cu -- fused face-flux + cell-update kernel of the mixed-precision
// stage (ideal gas, no mass fractions, three active dimensions) and the
// Contact-CT EMF kernel that reads the interior-only face fluxes it leaves.
//
// One CTA owns a tile of FX x FY x FZ cells.  A single 4-D TMA copy
// (cp.async.bulk.tensor, completion on an mbarrier) stages the tile's
// primitive deviations W with NGW = 2 ghost layers on every side, both float4
// planes, in shared memory.  The CTA then evaluates every face of the tile in
// all three directions from shared memory -- van Leer PLM on the deviations
// (Sect. 2.5), LHLLD / HLL flux in deviation form with the background flux
// removed (Sects. 2.6-2.8, Eq. wb1) -- keeps the five fluid flux components
// of each face in shared memory, and finishes with the residual, the gravity
// and heating sources and the SSP-RK increment of its own cells (Sect. 2.9,
// Eq. spatres).  Only the tangential-B fluxes and the contact direction of
// each owned face go to global memory, for the edge EMFs (Sect. 2.4).
//
// Compared with one kernel per direction plus a separate update, the face
// fluxes never round-trip through HBM, each face costs shared-memory loads
// instead of global gathers with ghost remapping, and the only per-face global
// traffic left is the normal field, two flag bytes and three EMF inputs.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "mixed_common.cuh"
#include "riemann_x2.cuh"

namespace phl {
using namespace stage;
namespace {

constexpr int FX = 8, FY = 8, FZ = 8;                                  // cells per tile
constexpr int HX = FX + 2 * NGW, HY = FY + 2 * NGW, HZ = FZ + 2 * NGW;   // staged extent
constexpr int NHC = HX * HY * HZ;                                      // staged cells
constexpr int NXF = (FX + 1) * FY * FZ, NYF = FX * (FY + 1) * FZ, NZF = FX * FY * (FZ + 1);
constexpr int NFACE = NXF + NYF + NZF;
constexpr int FTPB = 256;
constexpr unsigned W_TILE_BYTES = 2u * NHC * 16u;
static_assert(NXF % 32 == 0 && NYF % 32 == 0, "a warp's faces must share one direction");

// Shared memory of a tile: the barrier, the tile's background profiles and
// shock flags, then the staged W (128-byte aligned for the TMA destination),
// then the face buffer, which the phased variant sizes for one direction's
// faces only (its launch requests less).
struct FusedSmem {
  unsigned long long bar;              // TMA completion barrier
  float bgc[2][FZ];                    // background rho, P at the tile's cell centres (scaled units)
  float bgf[2][FZ + 1];                // the same at its z-faces
  uint8_t flg[FZ + 2][FY + 2][FX + 2]; // dilated shock flags of cells -1 .. F (a ghost carries its source's)
  alignas(128) float4 w[2][NHC];       // staged W: (drho, vx, vy, vz) and (Bx, By, Bz, dP) per cell
  float f[5][NFACE];                   // face fluxes, normal frame (rho, m_n, m_t1, m_t2, E); the
                                       // kernel indexes it flat with row stride NXF (phased) or NFACE
};
static_assert(offsetof(FusedSmem, w) % 128 == 0, "TMA destination alignment");
constexpr size_t smem_bytes(bool phased) {
  return offsetof(FusedSmem, f) + sizeof(float) * 5 * (phased ? NXF : NFACE) + 128;   // + alignment slack
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the barrier phase with a wall-clock limit; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > limit_ns) return false;
  return true;
}

// Flux of the D-face at the lower side of staged cell s2 (its right cell),
// tile cell (i, j, k), global cell c.  Returns the five fluid components in
// out[] and stores the EMF inputs when the tile owns the face.
template <int D, bool LR, bool PPH>
__device__ __forceinline__ void fused_face(const DevGeo &G, const StageMx &S, const FusedSmem &sm, int s2, int i,
                                           int j, int k, const int *c, bool own, float *__restrict__ Fd,
                                           const GasK<float> &K, float *out, int *dflag) {
  constexpr int sD = D == 0 ? 1 : (D == 1 ? HX : HX * HY);
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  float ql[8], qr[8];
  {
    float4 a[4], b[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      a[m] = sm.w[0][s2 + (m - 2) * sD];
      b[m] = sm.w[1][s2 + (m - 2) * sD];
    }
    // PPH: unlimited parabola (no mass fractions on this path); a cell flagged
    // by the shock flattener reconstructs with van Leer (Sect. 2.7)
    const uint8_t *fc = &sm.flg[k + 1][j + 1][i + 1];
    constexpr int fsD = D == 0 ? 1 : (D == 1 ? FX + 2 : (FX + 2) * (FY + 2));
    const bool pphL = PPH && !fc[-fsD], pphR = PPH && !fc[0];
    auto plm = [&](int v, float w0, float w1, float w2, float w3) {
      if constexpr (PPH) {   // the per-cell choice only in the PPH instantiation
        ql[v] = pphL ? pph_right(w0, w1, w2) : w1 + 0.5f * vl_slope(w0, w1, w2);
        qr[v] = pphR ? pph_left(w1, w2, w3) : w2 - 0.5f * vl_slope(w1, w2, w3);
      } else {
        // the two van Leer slopes (cell i for the left state, cell i+1 for
        // the right) as one FP32x2 pair: differences, products, sums and the
        // face values packed; the quotient 2 dm dp / (dm + dp) per lane by
        // the fast division (its denominators are O(1) in scaled units)
        const x2::V dm = x2::vv(w1, w2) - x2::vv(w0, w1), dp = x2::vv(w2, w3) - x2::vv(w1, w2);
        const x2::V pr = dm * dp, den = dm + dp;
        const x2::V sl = x2::vv(pr.x > 0.0f ? __fdividef(pr.x + pr.x, den.x) : 0.0f,
                                pr.y > 0.0f ? __fdividef(pr.y + pr.y, den.y) : 0.0f);
        const x2::V q = x2::fma(x2::vv(0.5f, -0.5f), sl, x2::vv(w1, w2));
        ql[v] = q.x;
        qr[v] = q.y;
      }
    };
    plm(W_RHO, a[0].x, a[1].x, a[2].x, a[3].x);
    plm(W_VX, a[0].y, a[1].y, a[2].y, a[3].y);
    plm(W_VY, a[0].z, a[1].z, a[2].z, a[3].z);
    plm(W_VZ, a[0].w, a[1].w, a[2].w, a[3].w);
    if (D != 0) plm(W_BX, b[0].x, b[1].x, b[2].x, b[3].x);   // the normal field is not reconstructed
    if (D != 1) plm(W_BY, b[0].y, b[1].y, b[2].y, b[3].y);
    if (D != 2) plm(W_BZ, b[0].z, b[1].z, b[2].z, b[3].z);
    plm(W_P, b[0].w, b[1].w, b[2].w, b[3].w);
  }
  // normal frame (n, t1, t2) = (D, D+1, D+2 mod 3)
  float wl[W_X0], wr[W_X0];
  auto frame = [&](const float *q, float *w) {
    w[RD_RHO] = q[W_RHO];
    w[RD_UN] = q[W_VX + D];
    w[RD_UT1] = q[W_VX + T1];
    w[RD_UT2] = q[W_VX + T2];
    w[RD_BT1] = q[W_BX + T1];
    w[RD_BT2] = q[W_BX + T2];
    w[RD_P] = q[W_P];
    w[RD_GE] = 0.0f;
    w[RD_GC] = 0.0f;
  };
  frame(ql, wl);
  frame(qr, wr);
  const float brho = D == 2 ? sm.bgf[0][k] : sm.bgc[0][k], bp = D == 2 ? sm.bgf[1][k] : sm.bgc[1][k];
  if (!(brho + wl[RD_RHO] > 0.0f && brho + wr[RD_RHO] > 0.0f && bp + wl[RD_P] > 0.0f && bp + wr[RD_P] > 0.0f))
    atomicOr(dflag, FLAG_NEG);
  // 32-bit offsets (fused_stage_ok bounds the planes)
  const int qb = D * (int)G.plane + c[0] + (int)G.sy * c[1] + (int)G.sz * c[2];
  const float b0 = d2f_scaled(S.B[qb], -G.e_b);
  const float bn = S.first ? b0 : b0 + S.dB[qb];
  // dilated shock flags of the two cells; local cell (i, j, k) sits at flg[k+1][j+1][i+1]
  const uint8_t *fr = &sm.flg[k + 1][j + 1][i + 1];
  constexpr int fs = D == 0 ? 1 : (D == 1 ? FX + 2 : (FX + 2) * (FY + 2));
  const int solver = (fr[0] | fr[-fs]) ? SOLVER_HLL : G.riemann;
  float fl[7];
  int up;
  if constexpr (LR) x2::riemann_ideal_lr(wl, wr, bn, brho, bp, solver, G.machf, fl, up, K);
  else riemann_dev<float, 0, true>(wl, wr, bn, brho, bp, 0.0f, 0.0f, 0, solver, G.machf, fl, up, K);
  // reflecting wall face: a symmetry plane; only the normal-momentum flux survives
  if ((c[D] == 0 && G.bc[D][0] == 1) || (c[D] == G.n[D] && G.bc[D][1] == 1)) {
#pragma unroll
    for (int q = 0; q < 7; ++q)
      if (q != RF_MN) fl[q] = 0.0f;
    up = 0;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q] = fl[q];
  if (own) {
    const int wt = (int)G.wtot;
    const int pR = (c[0] + G.ge[0]) + (int)G.wy * (c[1] + G.ge[1]) + (int)G.wz * (c[2] + G.ge[2]);
    Fd[(F_BX + T1) * wt + pR] = fl[RF_BT1];
    Fd[(F_BX + T2) * wt + pR] = fl[RF_BT2];
    Fd[G.nf * wt + pR] = (float)up;
  }
}

// Evaluates face f of direction D (its index among the tile's D-faces) and
// returns the five fluid flux components (zeros outside the domain).
template <int D, bool LR, bool PPH>
__device__ __forceinline__ void tile_face(const DevGeo &G, const StageMx &S, const FusedSmem &sm, int f, int x0,
                                          int y0, int z0, float *F0, float *F1, float *F2, const GasK<float> &K,
                                          float *out, int *dflag) {
  int i, j, k;
  if (D == 0) { i = f % (FX + 1); const int r = f / (FX + 1); j = r % FY; k = r / FY; }
  else if (D == 1) { i = f % FX; const int r = f / FX; j = r % (FY + 1); k = r / (FY + 1); }
  else { i = f % FX; const int r = f / FX; j = r % FY; k = r / FY; }
  const int c[3] = {x0 + i, y0 + j, z0 + k};
  const bool valid = c[0] <= G.n[0] - (D != 0) && c[1] <= G.n[1] - (D != 1) && c[2] <= G.n[2] - (D != 2);
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q] = 0.0f;
  if (!valid) return;
  const int s2 = ((k + NGW) * HY + (j + NGW)) * HX + (i + NGW);
  constexpr int ext = D == 0 ? FX : (D == 1 ? FY : FZ);
  const int loc = D == 0 ? i : (D == 1 ? j : k);
  const bool own = loc < ext || c[D] == G.n[D];
  float *Fd = D == 0 ? F0 : (D == 1 ? F1 : F2);
  fused_face<D, LR, PPH>(G, S, sm, s2, i, j, k, c, own, Fd, K, out, dflag);
}

// Two D-faces of the tile (fa, fb: indices among its D-faces) evaluated
// together on packed FP32x2 arithmetic: PLM and the ideal-gas LHLLD / HLL flux
// of riemann_x2.cuh, lane x = face fa, lane y = face fb.  With hasb false the
// second lane repeats fa and its results are dropped.  Faces outside the
// domain give zeros, as in tile_face.
template <int D, bool PPH>
__device__ __forceinline__ void tile_face2(const DevGeo &G, const StageMx &S, const FusedSmem &sm, int fa, int fb,
                                           bool hasb, int x0, int y0, int z0, float *F0, float *F1, float *F2,
                                           const GasK<float> &K, float *oa, float *ob, int *dflag) {
  using namespace x2;
  constexpr int sD = D == 0 ? 1 : (D == 1 ? HX : HX * HY);
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  constexpr int ext = D == 0 ? FX : (D == 1 ? FY : FZ);
  constexpr int fs = D == 0 ? 1 : (D == 1 ? FX + 2 : (FX + 2) * (FY + 2));
  int l[2][3];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int f = h == 0 ? fa : fb;
    if (D == 0) { l[h][0] = f % (FX + 1); const int r = f / (FX + 1); l[h][1] = r % FY; l[h][2] = r / FY; }
    else if (D == 1) { l[h][0] = f % FX; const int r = f / FX; l[h][1] = r % (FY + 1); l[h][2] = r / (FY + 1); }
    else { l[h][0] = f % FX; const int r = f / FX; l[h][1] = r % FY; l[h][2] = r / FY; }
  }
  const int ca[3] = {x0 + l[0][0], y0 + l[0][1], z0 + l[0][2]};
  const int cb[3] = {x0 + l[1][0], y0 + l[1][1], z0 + l[1][2]};
  auto inside = [&](const int *c) {
    return c[0] <= G.n[0] - (D != 0) && c[1] <= G.n[1] - (D != 1) && c[2] <= G.n[2] - (D != 2);
  };
  const bool va = inside(ca), vb = hasb && inside(cb);
#pragma unroll
  for (int q = 0; q < 5; ++q) { oa[q] = 0.0f; ob[q] = 0.0f; }
  if (!va && !vb) return;
  const int s2a = ((l[0][2] + NGW) * HY + (l[0][1] + NGW)) * HX + (l[0][0] + NGW);
  const int s2b = ((l[1][2] + NGW) * HY + (l[1][1] + NGW)) * HX + (l[1][0] + NGW);
  // cells flagged by the shock flattener (left / right of each face)
  const uint8_t *fla = &sm.flg[l[0][2] + 1][l[0][1] + 1][l[0][0] + 1];
  const uint8_t *flb = &sm.flg[l[1][2] + 1][l[1][1] + 1][l[1][0] + 1];
  const B2 vlL{fla[-fs] != 0, flb[-fs] != 0}, vlR{fla[0] != 0, flb[0] != 0};
  const bool vlAny = vlL.x || vlL.y || vlR.x || vlR.y;
  V ql[8], qr[8];
  {
    const V half = vv(0.5f), zero = vv(0.0f);
    auto slope = [&](V w0, V w1, V w2) -> V {   // van Leer harmonic slope (Sect. 2.5, item i)
      const V dm = w1 - w0, dp = w2 - w1;
      const V pr = dm * dp;
      return sel(pr > zero, (pr + pr) * rcp(dm + dp), zero);
    };
#pragma unroll
    for (int hw = 0; hw < 2; ++hw) {
      float4 A[4], Bv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        A[m] = sm.w[hw][s2a + (m - 2) * sD];
        Bv[m] = sm.w[hw][s2b + (m - 2) * sD];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int v = 4 * hw + e;
        if (v == W_BX + D) continue;   // the normal field is not reconstructed
        auto comp = [&](const float4 &u) { return e == 0 ? u.x : (e == 1 ? u.y : (e == 2 ? u.z : u.w)); };
        const V w0 = vv(comp(A[0]), comp(Bv[0])), w1 = vv(comp(A[1]), comp(Bv[1]));
        const V w2 = vv(comp(A[2]), comp(Bv[2])), w3 = vv(comp(A[3]), comp(Bv[3]));
        if constexpr (PPH) {   // unlimited parabola: (-w0 + 5 w1 + 2 w2) / 6, (2 w1 + 5 w2 - w3) / 6
          const V s6 = vv(1.0f / 6.0f), five = vv(5.0f), two = vv(2.0f);
          ql[v] = fma(two, w2, fma(five, w1, neg(w0))) * s6;
          qr[v] = (fma(two, w1, five * w2) - w3) * s6;
          if (vlAny) {   // cells flagged by the shock flattener reconstruct with van Leer (Sect. 2.7)
            ql[v] = sel(vlL, fma(half, slope(w0, w1, w2), w1), ql[v]);
            qr[v] = sel(vlR, fma(neg(half), slope(w1, w2, w3), w2), qr[v]);
          }
        } else {
          ql[v] = fma(half, slope(w0, w1, w2), w1);
          qr[v] = fma(neg(half), slope(w1, w2, w3), w2);
        }
      }
    }
  }
  V wl[W_X0], wr[W_X0];
  auto frame = [&](const V *q, V *w) {
    w[RD_RHO] = q[W_RHO];
    w[RD_UN] = q[W_VX + D];
    w[RD_UT1] = q[W_VX + T1];
    w[RD_UT2] = q[W_VX + T2];
    w[RD_BT1] = q[W_BX + T1];
    w[RD_BT2] = q[W_BX + T2];
    w[RD_P] = q[W_P];
  };
  frame(ql, wl);
  frame(qr, wr);
  const int ka = l[0][2], kb = l[1][2];
  const V brho = D == 2 ? vv(sm.bgf[0][ka], sm.bgf[0][kb]) : vv(sm.bgc[0][ka], sm.bgc[0][kb]);
  const V bp = D == 2 ? vv(sm.bgf[1][ka], sm.bgf[1][kb]) : vv(sm.bgc[1][ka], sm.bgc[1][kb]);
  {
    const V rl = brho + wl[RD_RHO], rr = brho + wr[RD_RHO], pl = bp + wl[RD_P], pr = bp + wr[RD_P];
    const bool na = !(rl.x > 0.0f && rr.x > 0.0f && pl.x > 0.0f && pr.x > 0.0f);
    const bool nb = !(rl.y > 0.0f && rr.y > 0.0f && pl.y > 0.0f && pr.y > 0.0f);
    if ((va && na) || (vb && nb)) atomicOr(dflag, FLAG_NEG);
  }
  const long qba = (long)D * G.plane + sidx(G, ca[0], ca[1], ca[2]);
  const long qbb = (long)D * G.plane + sidx(G, cb[0], cb[1], cb[2]);
  float bna = d2f_scaled(S.B[qba], -G.e_b), bnb = d2f_scaled(S.B[qbb], -G.e_b);
  if (!S.first) { bna += S.dB[qba]; bnb += S.dB[qbb]; }
  const uint8_t *fra = &sm.flg[l[0][2] + 1][l[0][1] + 1][l[0][0] + 1];
  const uint8_t *frb = &sm.flg[l[1][2] + 1][l[1][1] + 1][l[1][0] + 1];
  const bool hla = (fra[0] | fra[-fs]) != 0, hlb = (frb[0] | frb[-fs]) != 0;
  V fl[7];
  int upa, upb;
  const bool any_hll_solver = G.riemann == SOLVER_HLL;
  riemann_ideal_x2(wl, wr, vv(bna, bnb), brho, bp, B2{hla || any_hll_solver, hlb || any_hll_solver},
                   any_hll_solver ? SOLVER_LHLLD : G.riemann, G.machf, fl, upa, upb, K);
  const bool wa = (ca[D] == 0 && G.bc[D][0] == 1) || (ca[D] == G.n[D] && G.bc[D][1] == 1);
  const bool wb = (cb[D] == 0 && G.bc[D][0] == 1) || (cb[D] == G.n[D] && G.bc[D][1] == 1);
  float fa7[7], fb7[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {   // reflecting wall face: only the normal-momentum flux survives
    fa7[q] = (wa && q != RF_MN) ? 0.0f : fl[q].x;
    fb7[q] = (wb && q != RF_MN) ? 0.0f : fl[q].y;
  }
  if (wa) upa = 0;
  if (wb) upb = 0;
  float *Fd = D == 0 ? F0 : (D == 1 ? F1 : F2);
  const long wt = G.wtot;
  if (va) {
#pragma unroll
    for (int q = 0; q < 5; ++q) oa[q] = fa7[q];
    if (l[0][D] < ext || ca[D] == G.n[D]) {
      const long pR = widx(G, ca[0], ca[1], ca[2]);
      Fd[(F_BX + T1) * wt + pR] = fa7[RF_BT1];
      Fd[(F_BX + T2) * wt + pR] = fa7[RF_BT2];
      Fd[(long)G.nf * wt + pR] = (float)upa;
    }
  }
  if (vb) {
#pragma unroll
    for (int q = 0; q < 5; ++q) ob[q] = fb7[q];
    if (l[1][D] < ext || cb[D] == G.n[D]) {
      const long pR = widx(G, cb[0], cb[1], cb[2]);
      Fd[(F_BX + T1) * wt + pR] = fb7[RF_BT1];
      Fd[(F_BX + T2) * wt + pR] = fb7[RF_BT2];
      Fd[(long)G.nf * wt + pR] = (float)upb;
    }
  }
}

// One direction's faces of the tile through the face buffer, then each
// thread's running residuals of its cells (phased variant).
template <int D, int NT, int CPT, int FS, bool PAIRED, bool LR, bool PPH>
__device__ __forceinline__ void tile_phase(const DevGeo &G, const StageMx &S, FusedSmem &sm, float *fb, int tid,
                                           int x0, int y0, int z0, float *F0, float *F1, float *F2,
                                           const GasK<float> &K, float (*racc)[5], int *dflag) {
  constexpr int qm[5][3] = {{0, 0, 0}, {1, 3, 2}, {2, 1, 3}, {3, 2, 1}, {4, 4, 4}};
  constexpr int NC = FX * FY * FZ;
  if constexpr (PAIRED) {   // faces f and f + NT together
    for (int f = tid; f < NXF; f += 2 * NT) {
      const int g2 = f + NT;
      const bool hasb = g2 < NXF;
      float oa[5], ob[5];
      tile_face2<D, PPH>(G, S, sm, f, hasb ? g2 : f, hasb, x0, y0, z0, F0, F1, F2, K, oa, ob, dflag);
#pragma unroll
      for (int q = 0; q < 5; ++q) fb[q * FS + f] = oa[q];
      if (hasb) {
#pragma unroll
        for (int q = 0; q < 5; ++q) fb[q * FS + g2] = ob[q];
      }
    }
  } else {
    for (int f = tid; f < NXF; f += NT) {
      float out[5];
      tile_face<D, LR, PPH>(G, S, sm, f, x0, y0, z0, F0, F1, F2, K, out, dflag);
#pragma unroll
      for (int q = 0; q < 5; ++q) fb[q * FS + f] = out[q];
    }
  }
  __syncthreads();
  constexpr int st = D == 0 ? 1 : (D == 1 ? FX : FX * FY);
  const float idd = G.idxf[D];
#pragma unroll
  for (int m = 0; m < CPT; ++m) {
    const int cc = tid + m * NT;
    if (cc < NC) {
      const int i = cc % FX, j = (cc / FX) % FY, k = cc / (FX * FY);
      const int f0 = D == 0 ? (k * FY + j) * (FX + 1) + i : (D == 1 ? (k * (FY + 1) + j) * FX + i : (k * FY + j) * FX + i);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int q = qm[v][D];
        racc[m][v] += (fb[q * FS + f0 + st] - fb[q * FS + f0]) * idd;
      }
    }
  }
  __syncthreads();
}

// The work of one tile with lower corner (x0, y0, z0).  PHASED = false: all
// faces of the tile are evaluated in one loop and kept in shared memory
// (5 x NFACE floats), then every cell sums its six faces.  PHASED = true: one
// direction at a time through a buffer of one direction's faces; each thread
// keeps the running residuals of its cells in registers (same summation order
// x, y, z), so the CTA needs ~1/3 of the shared memory and more CTAs fit on
// an SM.  The TMA copy completes on the CTA's barrier sm.bar, whose phase of
// this use is `parity`.  Returns false when the copy did not land within the
// bounded wait (the error bit set, the copy waited for once more).
template <int NT, bool PHASED, bool PAIRED, bool LR, bool PPH>
__device__ __forceinline__ bool tile_body(const CUtensorMap *tmW, const DevGeo &G, const StageMx &S,
                                          const uint8_t *__restrict__ flag, float *__restrict__ F0,
                                          float *__restrict__ F1, float *__restrict__ F2, int x0, int y0, int z0,
                                          int *dflag, unsigned extra_tx, int raw_flags, FusedSmem &sm,
                                          unsigned parity) {
  const int tid = threadIdx.x;
  const unsigned bar = smem_u32(&sm.bar);
  if (tid == 0) {
    // extra_tx is 0 except in the timeout test (bytes that never arrive)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(W_TILE_BYTES + extra_tx)
                 : "memory");
    // work-layout coordinates of staged cell (-NGW, -NGW, -NGW): (x0 - NGW + ge) = x0
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(&sm.w[0][0])),
        "l"((unsigned long long)tmW), "r"(4 * x0), "r"(y0), "r"(z0), "r"(0), "r"(bar)
        : "memory");
  }
  // while the copy is in flight: the tile's background profiles and the
  // dilated shock flags of cells -1 .. F along each axis (a ghost cell carries
  // the flag of the interior cell its data comes from; cells further out feed
  // no face and stay unflagged)
  if (tid < FZ + 1) {
    const int z = z0 + tid;
    const bool in = G.has_bg && z <= G.n[2];
    sm.bgf[0][tid] = in ? G.bgf_rho_f[z + BG_NG] : 0.0f;
    sm.bgf[1][tid] = in ? G.bgf_p_f[z + BG_NG] : 0.0f;
    if (tid < FZ) {
      const bool inc = G.has_bg && z < G.n[2];
      sm.bgc[0][tid] = inc ? G.bgf_rho_c[z + BG_NG] : 0.0f;
      sm.bgc[1][tid] = inc ? G.bgf_p_c[z + BG_NG] : 0.0f;
    }
  }
  if (raw_flags) {
    // flag holds the raw flags (interior layout): the 5^3 dilation of the
    // tile's cells -1 .. F is done here from the raw flags of cells -3 .. F+2,
    // wrapped on periodic axes and unflagged beyond any other boundary, the
    // ORs nested axis by axis (x, y, z) in the face buffer (unused until the
    // faces).  A ghost cell then carries the dilated flag of the interior cell
    // its data comes from, cells further out none -- as the dilation kernel
    // and the staging below give on the other path.
    constexpr int RB = FX + 6, RY = FY + 6, RZ = FZ + 6;   // raw box: cells -3 .. F+2
    uint8_t *rb = reinterpret_cast<uint8_t *>(&sm.f[0][0]);
    uint8_t *r1 = rb + RB * RY * RZ;             // x-ORed: cells -1 .. F along x
    uint8_t *r2 = r1 + (FX + 2) * RY * RZ;       // then y
    uint8_t *r3 = r2 + (FX + 2) * (FY + 2) * RZ; // then z
    const int o[3] = {x0, y0, z0};
    // one thread per raw-box row of RB bytes: the row's y, z wrap once; along
    // x a step of at most 3 cells past a boundary wraps by one period (the
    // fused path needs n >= 4 along every axis -- fused_stage_ok)
    for (int row = tid; row < RY * RZ; row += NT) {
      int y = o[1] - 3 + row % RY, z = o[2] - 3 + row / RY;
      bool in = true;
      if (y < 0 || y >= G.n[1]) { if (G.bc[1][0] == 0) y += y < 0 ? G.n[1] : -G.n[1]; else in = false; }
      if (z < 0 || z >= G.n[2]) { if (G.bc[2][0] == 0) z += z < 0 ? G.n[2] : -G.n[2]; else in = false; }
      const uint8_t *fr = flag + (long)G.n[0] * (y + (long)G.n[1] * z);
      uint8_t *dst = rb + row * RB;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        int x = o[0] - 3 + i;
        bool ok = in;
        if (x < 0 || x >= G.n[0]) { if (G.bc[0][0] == 0) x += x < 0 ? G.n[0] : -G.n[0]; else ok = false; }
        dst[i] = ok ? fr[x] : (uint8_t)0;
      }
    }
    __syncthreads();
    for (int q = tid; q < (FX + 2) * RY * RZ; q += NT) {
      const int i = q % (FX + 2), r = q / (FX + 2);
      const uint8_t *a = rb + r * RB + i;
      r1[q] = a[0] | a[1] | a[2] | a[3] | a[4];
    }
    __syncthreads();
    for (int q = tid; q < (FX + 2) * (FY + 2) * RZ; q += NT) {
      const int i = q % (FX + 2), j = (q / (FX + 2)) % (FY + 2), k = q / ((FX + 2) * (FY + 2));
      const uint8_t *a = r1 + (k * RY + j) * (FX + 2) + i;
      r2[q] = a[0] | a[FX + 2] | a[2 * (FX + 2)] | a[3 * (FX + 2)] | a[4 * (FX + 2)];
    }
    __syncthreads();
    for (int q = tid; q < (FX + 2) * (FY + 2) * (FZ + 2); q += NT) {
      constexpr int P2 = (FX + 2) * (FY + 2);
      const uint8_t *a = r2 + q;
      r3[q] = a[0] | a[P2] | a[2 * P2] | a[3 * P2] | a[4 * P2];
    }
    __syncthreads();
    for (int q = tid; q < (FX + 2) * (FY + 2) * (FZ + 2); q += NT) {
      int l[3] = {q % (FX + 2), (q / (FX + 2)) % (FY + 2), q / ((FX + 2) * (FY + 2))};
      bool in = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int x = o[d] - 1 + l[d];
        if (x < -1 || x > G.n[d]) in = false;
        else if (G.bc[d][0] != 0 && x == -1) l[d] += 1;        // the source cell 0
        else if (G.bc[d][1] != 0 && x == G.n[d]) l[d] -= 1;    // the source cell n - 1
      }
      (&sm.flg[0][0][0])[q] = in ? r3[(l[2] * (FY + 2) + l[1]) * (FX + 2) + l[0]] : (uint8_t)0;
    }
  } else {
    for (int q = tid; q < (FX + 2) * (FY + 2) * (FZ + 2); q += NT) {
      const int l[3] = {q % (FX + 2), (q / (FX + 2)) % (FY + 2), q / ((FX + 2) * (FY + 2))};
      const int o[3] = {x0, y0, z0};
      uint8_t v = 0;
      if (flag) {
        int g[3];
        bool in = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          int x = o[d] - 1 + l[d];
          if (x < -1 || x > G.n[d]) in = false;
          else if (x == -1 || x == G.n[d]) {
            bool fl;
            x = cell_src(x, G.n[d], G.bc[d][0], G.bc[d][1], fl);
          }
          g[d] = x;
        }
        if (in) v = flag[g[0] + (long)G.n[0] * (g[1] + (long)G.n[1] * g[2])];
      }
      (&sm.flg[0][0][0])[q] = v;
    }
  }
  const bool ok = mbar_wait_bounded(bar, parity, 1000000000ull);
  if (__syncthreads_or(!ok)) {   // the copy did not land in 1 s: report, let it finish, leave
    if (tid == 0) atomicOr(dflag, FLAG_TIMEOUT);
    mbar_wait_bounded(bar, parity, 1000000000ull);
    return false;
  }

  GasK<float> K;
  K.g = G.gammaf;
  K.igm1 = 1.0f / (K.g - 1.0f);
  K.ggm1 = K.g * K.igm1;
  // face buffer: component q of buffered face f at fb[q * FS + f]
  constexpr int FS = PHASED ? NXF : NFACE;
  float *fb = &sm.f[0][0];
  // normal-frame component that carries global component v on d-faces
  constexpr int qm[5][3] = {{0, 0, 0}, {1, 3, 2}, {2, 1, 3}, {3, 2, 1}, {4, 4, 4}};
  constexpr int NC = FX * FY * FZ, CPT = (NC + NT - 1) / NT;   // cells per thread
  float racc[CPT][5];
#pragma unroll
  for (int m = 0; m < CPT; ++m)
#pragma unroll
    for (int v = 0; v < 5; ++v) racc[m][v] = 0.0f;

  if constexpr (PHASED) {
    static_assert(NXF == NYF && NYF == NZF, "phased tiles need equal face counts per direction");
    tile_phase<0, NT, CPT, FS, PAIRED, LR, PPH>(G, S, sm, fb, tid, x0, y0, z0, F0, F1, F2, K, racc, dflag);
    tile_phase<1, NT, CPT, FS, PAIRED, LR, PPH>(G, S, sm, fb, tid, x0, y0, z0, F0, F1, F2, K, racc, dflag);
    tile_phase<2, NT, CPT, FS, PAIRED, LR, PPH>(G, S, sm, fb, tid, x0, y0, z0, F0, F1, F2, K, racc, dflag);
  } else {
    // NXF and NXF + NYF are multiples of 32: the direction is uniform in a warp
    for (int f = tid; f < NFACE; f += NT) {
      float out[5];
      if (f < NXF) tile_face<0, LR, PPH>(G, S, sm, f, x0, y0, z0, F0, F1, F2, K, out, dflag);
      else if (f < NXF + NYF) tile_face<1, LR, PPH>(G, S, sm, f - NXF, x0, y0, z0, F0, F1, F2, K, out, dflag);
      else tile_face<2, LR, PPH>(G, S, sm, f - NXF - NYF, x0, y0, z0, F0, F1, F2, K, out, dflag);
#pragma unroll
      for (int q = 0; q < 5; ++q) fb[q * FS + f] = out[q];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int cc = tid + m * NT;
      if (cc < NC) {
        const int i = cc % FX, j = (cc / FX) % FY, k = cc / (FX * FY);
        const int fx = (k * FY + j) * (FX + 1) + i, fy = NXF + (k * (FY + 1) + j) * FX + i,
                  fz = NXF + NYF + (k * FY + j) * FX + i;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          racc[m][v] += (fb[qm[v][0] * FS + fx + 1] - fb[qm[v][0] * FS + fx]) * G.idxf[0];
          racc[m][v] += (fb[qm[v][1] * FS + fy + FX] - fb[qm[v][1] * FS + fy]) * G.idxf[1];
          racc[m][v] += (fb[qm[v][2] * FS + fz + FX * FY] - fb[qm[v][2] * FS + fz]) * G.idxf[2];
        }
      }
    }
  }

  // R = sum_d (F_d(+) - F_d(-)) / dx_d - (S - S_hat), then the RK increment.
  // The cells' increments (and, in the last stage, their FP64 state) are
  // read before anything is stored: a read of dU or U after a store to the
  // same array cannot move above it, so interleaving them would leave one
  // memory round trip per value at the end of every tile.
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  int psc[CPT];
  float din[CPT][5];
  double uin[CPT][5];
#pragma unroll
  for (int m = 0; m < CPT; ++m) {
    const int cc = tid + m * NT;
    const int i = cc % FX, j = (cc / FX) % FY, k = cc / (FX * FY);
    const int c0 = x0 + i, c1 = y0 + j, c2 = z0 + k;
    const bool ok = cc < NC && c0 < G.n[0] && c1 < G.n[1] && c2 < G.n[2];
    psc[m] = ok ? c0 + (int)G.sy * c1 + (int)G.sz * c2 : -1;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int q = v * (int)G.plane + psc[m];
      din[m][v] = (ok && !S.first) ? S.dU[q] : 0.0f;
      uin[m][v] = (ok && S.last) ? S.U[q] : 0.0;
    }
  }
#pragma unroll
  for (int m = 0; m < CPT; ++m) {
    if (psc[m] < 0) continue;
    const int cc = tid + m * NT;
    const int i = cc % FX, j = (cc / FX) % FY, k = cc / (FX * FY);
    const int c2 = z0 + k;
    float *r = racc[m];
    // sources S - S_hat: (rho - rho_hat) g on momentum, rho u . g (+ heating) on energy
    const float4 wa = sm.w[0][((k + NGW) * HY + (j + NGW)) * HX + (i + NGW)];
    const float drho = wa.x;
    const float rho = sm.bgc[0][k] + drho;
    const float vel[3] = {wa.y, wa.z, wa.w};
    float se = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float gd = G.gf[d];
      r[U_MX + d] -= drho * gd;
      se += rho * vel[d] * gd;
    }
    if (G.heatf) se += G.heatf[c2];
    r[U_E] -= se;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int q = v * (int)G.plane + psc[m];
      const float dout = S.b * (din[m][v] - dt * r[v]);
      if (S.last) S.U[q] = uin[m][v] + f2d_scaled(dout, uexp(G, v));
      else S.dU[q] = dout;
    }
  }
  return true;
}

// Tile kernel: one CTA per tile.
template <int NT, int MINB, bool PHASED, bool PAIRED = false, bool LR = false, bool PPH = false>
__global__ void __launch_bounds__(NT, MINB)
    k_flux_update_mx(const __grid_constant__ CUtensorMap tmW, DevGeo G, StageMx S, const uint8_t *__restrict__ flag,
                     float *__restrict__ F0, float *__restrict__ F1, float *__restrict__ F2, int ntx, int nty,
                     int *dflag, unsigned extra_tx, int raw_flags, const unsigned int *__restrict__ any) {
  extern __shared__ unsigned char smraw[];
  if (any && *any == 0u) flag = nullptr;   // no cell flagged: the tile stages zero flags
  FusedSmem &sm = *reinterpret_cast<FusedSmem *>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty, tz = t / nty;
  if (threadIdx.x == 0) {
    const unsigned bar = smem_u32(&sm.bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  tile_body<NT, PHASED, PAIRED, LR, PPH>(&tmW, G, S, flag, F0, F1, F2, tx * FX, ty * FY, tz * FZ, dflag, extra_tx,
                                         raw_flags, sm, 0u);
}

// 5^3 dilation of the raw shock flags (Sect. 2.7) for one 8^3 tile of
// interior cells in one pass, eight flags (one byte each) per 64-bit word: the
// raw flags of x0-4 .. x0+11 for every row of the tile and its two neighbour
// rows on each side are staged in shared memory as two words, then ORed along
// x (byte shifts of the 16-byte window), y and z (word ORs) in turn -- the OR
// over a box is the nested ORs over its axes.  Beyond a periodic boundary the
// flags wrap; beyond any other boundary they count as unflagged.
// The dilation of the tile at (x0, y0, z0) with the CTA's threads; r0, r1, r2:
// shared scratch of HZ HY 2, HZ HY and HZ FY words.
__device__ __forceinline__ void dilate_tile(const DevGeo &G, const uint8_t *__restrict__ raw, uint8_t *__restrict__ dil,
                                            int x0, int y0, int z0, unsigned long long (*r0)[2],
                                            unsigned long long *r1, unsigned long long *r2) {
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const int xs = x0 - 4;
  const bool wide = (nx % 8) == 0 && xs >= 0 && xs + 16 <= nx;   // aligned window inside the row
  const bool px = G.bc[0][0] == 0, py = G.bc[1][0] == 0, pz = G.bc[2][0] == 0;
  for (int q = threadIdx.x; q < HZ * HY * 4; q += blockDim.x) {
    const int w = q & 3, row = q >> 2;
    int y = y0 - NGW + row % HY, z = z0 - NGW + row / HY;
    bool in = true;
    if (y < 0 || y >= ny) { if (py) y = (y % ny + ny) % ny; else in = false; }
    if (z < 0 || z >= nz) { if (pz) z = (z % nz + nz) % nz; else in = false; }
    unsigned v = 0u;
    if (in) {
      const uint8_t *rr = raw + (long)nx * (y + (long)ny * z);
      if (wide) {
        v = *reinterpret_cast<const unsigned *>(rr + xs + 4 * w);
      } else {
        for (int bb = 0; bb < 4; ++bb) {
          int x = xs + 4 * w + bb;
          bool ok = true;
          if (x < 0 || x >= nx) { if (px) x = (x % nx + nx) % nx; else ok = false; }
          if (ok) v |= (unsigned)rr[x] << (8 * bb);
        }
      }
    }
    reinterpret_cast<unsigned *>(&r0[row][0])[w] = v;
  }
  __syncthreads();
  for (int row = threadIdx.x; row < HZ * HY; row += blockDim.x) {
    // output byte j (x = x0 + j) ORs window bytes j+2 .. j+6
    const unsigned long long lo = r0[row][0], hi = r0[row][1];
    unsigned long long o = 0ull;
#pragma unroll
    for (int sh = 2; sh <= 6; ++sh) o |= (lo >> (8 * sh)) | (hi << (64 - 8 * sh));
    r1[row] = o;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < HZ * FY; q += blockDim.x) {
    const int y = q % FY, z = q / FY;
    const unsigned long long *c = &r1[z * HY + y];
    r2[q] = c[0] | c[1] | c[2] | c[3] | c[4];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < FZ * FY; q += blockDim.x) {
    const int y = q % FY, z = q / FY;
    const int c1 = y0 + y, c2 = z0 + z;
    if (c1 >= ny || c2 >= nz) continue;
    const unsigned long long o = r2[z * FY + y] | r2[(z + 1) * FY + y] | r2[(z + 2) * FY + y] |
                                 r2[(z + 3) * FY + y] | r2[(z + 4) * FY + y];
    uint8_t *d = dil + x0 + (long)nx * (c1 + (long)ny * c2);
    if ((nx % 8) == 0 && x0 + 8 <= nx) {
      *reinterpret_cast<unsigned long long *>(d) = o;
    } else {
      for (int j = 0; j < 8 && x0 + j < nx; ++j) d[j] = (uint8_t)(o >> (8 * j));
    }
  }
}

// any (optional): the raw-flag kernel's vote; zero means no cell is flagged,
// the dilation is all zero and the tile kernel, reading the same vote, loads
// none of it -- nothing is written.
__global__ void __launch_bounds__(256) k_flag_dilate3(DevGeo G, const uint8_t *__restrict__ raw,
                                                     uint8_t *__restrict__ dil, int ntx, int nty,
                                                     const unsigned int *__restrict__ any) {
  __shared__ unsigned long long r0[HZ * HY][2];
  __shared__ unsigned long long r1[HZ * HY], r2[HZ * FY];
  if (any && *any == 0u) return;
  const int nb = ntx * nty * ((G.n[2] + FZ - 1) / FZ);
  for (int t0 = blockIdx.x; t0 < nb; t0 += gridDim.x) {   // the block's tiles; the grid fills the SMs once
    int t = t0;
    const int tx = t % ntx;
    t /= ntx;
    const int ty = t % nty, tz = t / nty;
    dilate_tile(G, raw, dil, tx * FX, ty * FY, tz * FZ, r0, r1, r2);
  }
}

// Contact-CT edge EMF along D at the lower corner (a-1/2, b-1/2) of cell c,
// (D, A, B) cyclic (Sect. 2.4): the mean of the four face EMFs plus the
// upwinded half-derivatives towards the cell-centred E = -u x B.  The face
// fluxes are stored for interior faces only: a face in a ghost row reads the
// interior row its data comes from (periodic wrap, outflow copy).  Ghost rows
// behind a reflecting wall feed only wall edges, whose EMF is zero (u_n = B_n
// = 0 there), so no mirror signs are needed.
template <int D>
__device__ __forceinline__ float emf_edge(const DevGeo &G, const int *c, bool interior, long p,
                                          const float *__restrict__ W, const float *__restrict__ FA,
                                          const float *__restrict__ FB) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const long sa = wstride(G, A), sb = wstride(G, B);
  long pa1 = p, pa0 = p - sb, pb1 = p, pb0 = p - sa;   // faces of an interior site
  if (!interior) {   // rows beyond the boundary read the interior rows their data come from
    bool fl;
    const int bm = cell_src(c[B] - 1, G.n[B], G.bc[B][0], G.bc[B][1], fl);
    const int b0 = cell_src(c[B], G.n[B], G.bc[B][0], G.bc[B][1], fl);
    const int am = cell_src(c[A] - 1, G.n[A], G.bc[A][0], G.bc[A][1], fl);
    const int a0 = cell_src(c[A], G.n[A], G.bc[A][0], G.bc[A][1], fl);
    pa1 = p + (b0 - c[B]) * sb;
    pa0 = p + (bm - c[B]) * sb;
    pb1 = p + (a0 - c[A]) * sa;
    pb0 = p + (am - c[A]) * sa;
  }
  const long wt = G.wtot;
  const float *fab = FA + (F_BX + B) * wt;   // F_a(B_b) on a-faces
  const float *fba = FB + (F_BX + A) * wt;   // F_b(B_a) on b-faces
  const float *ua = FA + (long)G.nf * wt, *ub = FB + (long)G.nf * wt;
  const float Ea1 = -fab[pa1], Ea0 = -fab[pa0];
  const float Eb1 = fba[pb1], Eb0 = fba[pb0];
  const float ma1 = ua[pa1], ma0 = ua[pa0];
  const float mb1 = ub[pb1], mb0 = ub[pb0];
  const float *ecell = W + waux(G, AUX_E + D, 0);
  const float E00 = ecell[p - sa - sb], E10 = ecell[p - sb], E01 = ecell[p - sa], E11 = ecell[p];
  const float lo_l = Eb0 - E00, lo_r = Eb1 - E10;
  const float up_l = E01 - Eb0, up_r = E11 - Eb1;
  const float h = 0.5f, q4 = 0.25f;
  const float dlo = ma0 > 0.0f ? lo_l : (ma0 < 0.0f ? lo_r : h * (lo_l + lo_r));
  const float dup = ma1 > 0.0f ? up_l : (ma1 < 0.0f ? up_r : h * (up_l + up_r));
  const float le_d = Ea0 - E00, le_u = Ea1 - E01;
  const float ri_d = E10 - Ea0, ri_u = E11 - Ea1;
  const float dle = mb0 > 0.0f ? le_d : (mb0 < 0.0f ? le_u : h * (le_d + le_u));
  const float dri = mb1 > 0.0f ? ri_d : (mb1 < 0.0f ? ri_u : h * (ri_d + ri_u));
  float v = q4 * (Ea1 + Ea0 + Eb1 + Eb0) + q4 * (dlo - dup) + q4 * (dle - dri);
  if (!interior && ((c[A] == 0 && G.bc[A][0] == 1) || (c[A] == G.n[A] && G.bc[A][1] == 1) ||
                    (c[B] == 0 && G.bc[B][0] == 1) || (c[B] == G.n[B] && G.bc[B][1] == 1)))
    v = 0.0f;
  return v;
}

// All three edge EMFs at the lower corners of site c in [0, n0] x [0, n1] x
// [0, n2] (an edge along D exists for c_D < n_D).  Sites away from every
// boundary (all faces and cells they touch are interior) skip the ghost
// mapping.
// 3-D blocks of EB_X x EB_Y x EB_Z sites for the EMF kernel: a block's
// neighbouring rows share L1 (0.305 -> 0.279 ms per launch at 256^3).
constexpr int EB_X = 32, EB_Y = 4, EB_Z = 2;
__device__ __forceinline__ bool site3(const DevGeo &G, int *c) {
  c[0] = blockIdx.x * EB_X + threadIdx.x;
  c[1] = blockIdx.y * EB_Y + threadIdx.y;
  c[2] = blockIdx.z * EB_Z + threadIdx.z;
  return c[0] <= G.n[0] && c[1] <= G.n[1] && c[2] <= G.n[2];
}
inline dim3 site_grid(const DevGeo &G) {
  return dim3((unsigned)((G.n[0] + EB_X) / EB_X), (unsigned)((G.n[1] + EB_Y) / EB_Y), (unsigned)((G.n[2] + EB_Z) / EB_Z));
}

// Contact-CT of one edge from its four face EMFs (a1, a0, b1, b0), their
// mass-flux signs and the four cell EMFs (emf_edge's formula).
__device__ __forceinline__ float ct_corner(float Ea1, float Ea0, float Eb1, float Eb0, float ma1, float ma0,
                                           float mb1, float mb0, float E00, float E10, float E01, float E11) {
  const float lo_l = Eb0 - E00, lo_r = Eb1 - E10;
  const float up_l = E01 - Eb0, up_r = E11 - Eb1;
  const float h = 0.5f, q4 = 0.25f;
  const float dlo = ma0 > 0.0f ? lo_l : (ma0 < 0.0f ? lo_r : h * (lo_l + lo_r));
  const float dup = ma1 > 0.0f ? up_l : (ma1 < 0.0f ? up_r : h * (up_l + up_r));
  const float le_d = Ea0 - E00, le_u = Ea1 - E01;
  const float ri_d = E10 - Ea0, ri_u = E11 - Ea1;
  const float dle = mb0 > 0.0f ? le_d : (mb0 < 0.0f ? le_u : h * (le_d + le_u));
  const float dri = mb1 > 0.0f ? ri_d : (mb1 < 0.0f ? ri_u : h * (ri_d + ri_u));
  return q4 * (Ea1 + Ea0 + Eb1 + Eb0) + q4 * (dlo - dup) + q4 * (dle - dri);
}

__global__ void k_emf3(DevGeo G, Box box, const float *__restrict__ W, const float *__restrict__ F0,
                       const float *__restrict__ F1, const float *__restrict__ F2, float *__restrict__ E) {
  int c[3];
  if (!site3(G, c)) return;
  const long wt = G.wtot;
  const bool interior = c[0] >= 1 && c[0] < G.n[0] && c[1] >= 1 && c[1] < G.n[1] && c[2] >= 1 && c[2] < G.n[2];
  if (interior && wt < 0x7fffffffL) {
    // an interior site (nearly all of them): every face and cell it reads is
    // interior; 32-bit offsets within each plane (the same values and
    // formula as emf_edge)
    const int p = (int)(c[0] + G.ge[0]) + (int)G.wy * (c[1] + G.ge[1]) + (int)G.wz * (c[2] + G.ge[2]);
    const int wy = (int)G.wy, wz = (int)G.wz;
    const float *xBy = F0 + (F_BX + 1) * wt, *xBz = F0 + (F_BX + 2) * wt, *ux = F0 + (long)G.nf * wt;
    const float *yBz = F1 + (F_BX + 2) * wt, *yBx = F1 + (F_BX + 0) * wt, *uy = F1 + (long)G.nf * wt;
    const float *zBx = F2 + (F_BX + 0) * wt, *zBy = F2 + (F_BX + 1) * wt, *uz = F2 + (long)G.nf * wt;
    const float *e0 = W + waux(G, AUX_E + 0, 0), *e1 = W + waux(G, AUX_E + 1, 0), *e2 = W + waux(G, AUX_E + 2, 0);
    // x-edges: a = y-faces, b = z-faces
    E[p] = ct_corner(-yBz[p], -yBz[p - wz], zBy[p], zBy[p - wy], uy[p], uy[p - wz], uz[p], uz[p - wy],
                     e0[p - wy - wz], e0[p - wz], e0[p - wy], e0[p]);
    // y-edges: a = z-faces, b = x-faces
    E[wt + p] = ct_corner(-zBx[p], -zBx[p - 1], xBz[p], xBz[p - wz], uz[p], uz[p - 1], ux[p], ux[p - wz],
                          e1[p - wz - 1], e1[p - 1], e1[p - wz], e1[p]);
    // z-edges: a = x-faces, b = y-faces
    E[2 * wt + p] = ct_corner(-xBy[p], -xBy[p - wy], yBx[p], yBx[p - 1], ux[p], ux[p - wy], uy[p], uy[p - 1],
                              e2[p - 1 - wy], e2[p - wy], e2[p - 1], e2[p]);
    return;
  }
  const long p = widx(G, c[0], c[1], c[2]);
  if (c[0] < G.n[0]) E[p] = emf_edge<0>(G, c, interior, p, W, F1, F2);
  if (c[1] < G.n[1]) E[wt + p] = emf_edge<1>(G, c, interior, p, W, F2, F0);
  if (c[2] < G.n[2]) E[2 * wt + p] = emf_edge<2>(G, c, interior, p, W, F0, F1);
}

// Contact-CT and the face update in one kernel (the three-launch stage): an
// 8^3 tile of sites computes, with emf_edge, the edge EMFs its faces need --
// E_D at sites s_D in [o_D, hi_D] (s_D < n_D), s_A in [o_A, hi_A + 1] (<= n_A),
// the same for B, hi the tile's last site (n for the tile at the upper
// boundary, which also owns the boundary faces) -- into shared memory, then
// updates its own faces from the curl of those EMFs.  The EMF inputs come
// straight from the tile kernel's output (L1/L2), as in k_emf3; only the
// tile's ~1.27 edges per site are kept.
constexpr int CTT = 8, CTE = CTT + 2, CTE3 = CTE * CTE * CTE;
__device__ __forceinline__ int ct_hi(int o, int n) { return o + CTT >= n ? n : o + CTT - 1; }

// The edges along D a tile needs, into ed (box of CTE^3 sites from o).
template <int D>
__device__ __forceinline__ void ct_edges(const DevGeo &G, const StageMx &S, const int *o, const int *hi, float *ed,
                                         int tid) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const float *FA = S.F[A], *FB = S.F[B];
  for (int r = tid; r < CTE3; r += 256) {
    const int ex = r % CTE, ey = (r / CTE) % CTE, ez = r / (CTE * CTE);
    const int c[3] = {o[0] + ex, o[1] + ey, o[2] + ez};
    const bool need = c[D] <= hi[D] && c[D] < G.n[D] && c[A] <= hi[A] + 1 && c[A] <= G.n[A] &&
                      c[B] <= hi[B] + 1 && c[B] <= G.n[B];
    float v = 0.0f;
    if (need) {
      const long p = widx(G, c[0], c[1], c[2]);
      const bool interior =
          c[0] >= 1 && c[0] < G.n[0] && c[1] >= 1 && c[1] < G.n[1] && c[2] >= 1 && c[2] < G.n[2];
      v = emf_edge<D>(G, c, interior, p, S.W, FA, FB);
    }
    ed[r] = v;
  }
}

// The tile's own D-faces from the curl of the edge EMFs in shared memory.
template <int D>
__device__ __forceinline__ void ct_faces(const DevGeo &G, const StageMx &S, const int *o, const int *hi,
                                         float (*ed)[CTE3], float dt, int tid) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  constexpr int NFT = (CTT + 1) * CTT * CTT;
  constexpr int eA = A == 0 ? 1 : (A == 1 ? CTE : CTE * CTE), eB = B == 0 ? 1 : (B == 1 ? CTE : CTE * CTE);
  for (int r = tid; r < NFT; r += 256) {
    int e[3];
    e[D] = r % (CTT + 1);
    e[A] = (r / (CTT + 1)) % CTT;
    e[B] = r / ((CTT + 1) * CTT);
    const int c[3] = {o[0] + e[0], o[1] + e[1], o[2] + e[2]};
    if (c[D] > hi[D] || c[A] > hi[A] || c[A] >= G.n[A] || c[B] > hi[B] || c[B] >= G.n[B]) continue;
    const int k0 = (e[2] * CTE + e[1]) * CTE + e[0];
    float rr = 0.0f;
    rr += (ed[B][k0 + eA] - ed[B][k0]) * G.idxf[A];
    rr -= (ed[A][k0 + eB] - ed[A][k0]) * G.idxf[B];
    const long qg = (long)D * G.plane + sidx(G, c[0], c[1], c[2]);
    const float din = S.first ? 0.0f : S.dB[qg];
    const float dout = S.b * (din - dt * rr);
    if (S.last) S.B[qg] += f2d_scaled(dout, G.e_b);
    else S.dB[qg] = dout;
  }
}

__global__ void __launch_bounds__(256) k_ct_faces(DevGeo G, StageMx S, int ntx, int nty) {
  __shared__ float ed[3][CTE3];
  const int tid = threadIdx.x;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty, tz = t / nty;
  const int o[3] = {tx * CTT, ty * CTT, tz * CTT};
  const int hi[3] = {ct_hi(o[0], G.n[0]), ct_hi(o[1], G.n[1]), ct_hi(o[2], G.n[2])};
  ct_edges<0>(G, S, o, hi, ed[0], tid);
  ct_edges<1>(G, S, o, hi, ed[1], tid);
  ct_edges<2>(G, S, o, hi, ed[2], tid);
  __syncthreads();
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  ct_faces<0>(G, S, o, hi, ed, dt, tid);
  ct_faces<1>(G, S, o, hi, ed, dt, tid);
  ct_faces<2>(G, S, o, hi, ed, dt, tid);
}

// Face update of the normal field on the D-face at site c from the curl of
// the edge EMFs (Eq. induction in discrete form), as k_update_faces_mx.
template <int D>
__device__ __forceinline__ void face_update(const DevGeo &G, const int *c, const StageMx &S, float dt) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const long p = widx(G, c[0], c[1], c[2]);
  const long wt = G.wtot;
  float r = 0.0f;
  r += (S.E[(long)B * wt + p + wstride(G, A)] - S.E[(long)B * wt + p]) * G.idxf[A];
  r -= (S.E[(long)A * wt + p + wstride(G, B)] - S.E[(long)A * wt + p]) * G.idxf[B];
  const long q = (long)D * G.plane + sidx(G, c[0], c[1], c[2]);
  const float din = S.first ? 0.0f : S.dB[q];
  const float dout = S.b * (din - dt * r);
  if (S.last) S.B[q] += f2d_scaled(dout, G.e_b);
  else S.dB[q] = dout;
}

// face_update with 32-bit offsets: on the fused path every W-layout array
// (E: three planes) and every state array (B, dB: three planes) is below 2^31
// elements.  p: the site's work index, ps: its state index.
template <int D>
__device__ __forceinline__ void face_update32(const DevGeo &G, unsigned p, unsigned ps, const StageMx &S, float dt) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const unsigned wt = (unsigned)G.wtot;
  const unsigned sA = A == 0 ? 1u : (A == 1 ? (unsigned)G.wy : (unsigned)G.wz);
  const unsigned sB = B == 0 ? 1u : (B == 1 ? (unsigned)G.wy : (unsigned)G.wz);
  const float *EB = S.E + B * wt, *EA = S.E + A * wt;
  float r = 0.0f;
  r += (EB[p + sA] - EB[p]) * G.idxf[A];
  r -= (EA[p + sB] - EA[p]) * G.idxf[B];
  const unsigned q = D * (unsigned)G.plane + ps;
  const float din = S.first ? 0.0f : S.dB[q];
  const float dout = S.b * (din - dt * r);
  if (S.last) S.B[q] += f2d_scaled(dout, G.e_b);
  else S.dB[q] = dout;
}

__global__ void k_update_faces3(DevGeo G, Box box, StageMx S) {
  int c[3];
  if (!cell3(box, c)) return;
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  const unsigned p = (unsigned)(c[0] + G.ge[0]) + (unsigned)G.wy * (unsigned)(c[1] + G.ge[1]) +
                     (unsigned)G.wz * (unsigned)(c[2] + G.ge[2]);
  const unsigned ps = (unsigned)c[0] + (unsigned)G.sy * (unsigned)c[1] + (unsigned)G.sz * (unsigned)c[2];
  if (c[1] < G.n[1] && c[2] < G.n[2]) face_update32<0>(G, p, ps, S, dt);
  if (c[0] < G.n[0] && c[2] < G.n[2]) face_update32<1>(G, p, ps, S, dt);
  if (c[0] < G.n[0] && c[1] < G.n[1]) face_update32<2>(G, p, ps, S, dt);
}

// ---------------------------------------------------------------------------
// An ensemble of boxes in one persistent cooperative launch per RK stage, on
// the tile kernel's body: phases over all boxes' items with a grid-wide
// barrier between them -- (first stage: CFL rate per box, then its dt) ->
// primitives -> raw shock flags -> their 5^3 dilation per tile -> tiles (each
// CTA takes tiles from the concatenated tile list: TMA from the box's own
// tensor map, faces, residual and cell update) -> edge EMFs -> face updates.  Every CTA reaches every barrier: a CTA whose copy timed out sets
// the error bit and skips its remaining tiles, nothing returns early.

struct FusedBox {
  DevGeo G;
  const CUtensorMap *tm;   // the box's W descriptor, in device memory
  double *U, *B;
  float *dU, *dB, *W, *F[3], *E;
  uint8_t *raw;
  double *dt;
  unsigned int *fmax;
  int *dflag;
  Box b_int, b_work, b_site;
  int ntx, nty;
};
enum { FE_DT, FE_PRIM, FE_RAW, FE_TILE, FE_SITE, FE_NPH };
struct FusedEnsArgs {
  const FusedBox *box;
  const long *pref;   // [FE_NPH][nbox + 1] prefix sums of each phase's items
  int nbox;
  int stage, nstages;
  float b;
};
constexpr int ENS_NT = 288, ENS_MINB = 3;

__device__ __forceinline__ int ens_box(const long *p, int nbox, long w) {
  int lo = 0, hi = nbox;   // p[lo] <= w < p[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ StageMx ens_stage_bufs(const FusedBox &R, const FusedEnsArgs &a) {
  StageMx S;
  S.U = R.U; S.B = R.B; S.dU = R.dU; S.dB = R.dB;
  S.first = a.stage == 0; S.last = a.stage == a.nstages - 1; S.b = a.b; S.dt = R.dt;
  S.W = R.W; S.F[0] = R.F[0]; S.F[1] = R.F[1]; S.F[2] = R.F[2]; S.E = R.E;
  return S;
}

// the box's geometry staged in shared memory (block-uniform), so that the
// phases' per-item work reads it without dependent global loads
__device__ __forceinline__ void ens_stage_geo(DevGeo *dst, const DevGeo &src) {
  const unsigned *s = reinterpret_cast<const unsigned *>(&src);
  unsigned *d = reinterpret_cast<unsigned *>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(DevGeo) / 4); i += blockDim.x) d[i] = s[i];
}
constexpr size_t ens_geo_offset() { return offsetof(FusedSmem, f) + sizeof(float) * 5 * NXF; }
constexpr size_t ens_smem_bytes() { return smem_bytes(true) + sizeof(DevGeo) + 16; }

template <bool PPH, int MINB>
__global__ void __launch_bounds__(ENS_NT, MINB) k_ens_fused(FusedEnsArgs a) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ unsigned char smraw[];
  unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
  FusedSmem &sm = *reinterpret_cast<FusedSmem *>(base);
  DevGeo &G = *reinterpret_cast<DevGeo *>(base + ((ens_geo_offset() + 15) & ~(size_t)15));
  const int tid = threadIdx.x;
  const long nth = (long)gridDim.x * ENS_NT, t0 = (long)blockIdx.x * ENS_NT + tid;
  const int nb = a.nbox;
  const bool first = a.stage == 0;
  if (tid == 0) {
    const unsigned bar = smem_u32(&sm.bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto pref = [&](int ph) { return a.pref + (long)ph * (nb + 1); };
  // one box after another (all blocks together), its items grid-strided
  auto per_box = [&](int ph, auto &&item) {
    const long *p = pref(ph);
    for (int bx = 0; bx < nb; ++bx) {
      const long n = p[bx + 1] - p[bx];
      if (n == 0) continue;
      __syncthreads();   // the previous box's readers are done
      ens_stage_geo(&G, a.box[bx].G);
      __syncthreads();
      const FusedBox &R = a.box[bx];
      for (long w = t0; w < n; w += nth) item(R, w);
    }
  };
  if (first) {   // the CFL step of U^n per box (Eq. cfl)
    per_box(FE_DT, [&](const FusedBox &R, long w) {
      int c[3];
      cell_at(R.b_int, w, c);
      const unsigned r = __float_as_uint(dt_rate_mx(G, R.U, R.B, c, R.dflag));   // >= 0: bits order as floats
      const unsigned m = __activemask();
      const unsigned mx = __reduce_max_sync(m, r);   // one atomic per warp: the box is block-uniform
      if ((int)(tid & 31) == __ffs(m) - 1) atomicMax(R.fmax, mx);
    });
    grid.sync();
    if (t0 < nb) {
      const FusedBox &R = a.box[t0];
      *R.dt = R.G.cfl * R.G.sc_t / (double)__uint_as_float(*R.fmax);
      *R.fmax = 0u;
    }
    grid.sync();
  }
  // primitive deviations and auxiliaries of the stage input (work layout)
  per_box(FE_PRIM, [&](const FusedBox &R, long w) {
    k_prim_mx_at(w, G, R.b_work, R.U, R.B, first ? nullptr : R.dU, first ? nullptr : R.dB, R.W, R.dflag);
  });
  grid.sync();
  if (pref(FE_RAW)[nb] > 0) {   // raw shock flags of the boxes that flatten, then their 5^3 dilation per tile
    per_box(FE_RAW, [&](const FusedBox &R, long w) { k_flag_raw_at<float>(w, G, R.b_int, R.W, R.raw); });
    grid.sync();
    const long *p = pref(FE_TILE);
    // scratch in the face buffer, unused outside the tile phase
    unsigned long long *scr = reinterpret_cast<unsigned long long *>(&sm.f[0][0]);
    int bx = -1;
    for (long w = blockIdx.x; w < p[nb]; w += gridDim.x) {
      int nbx = bx < 0 ? 0 : bx;
      while (w >= p[nbx + 1]) ++nbx;
      __syncthreads();
      if (nbx != bx) {
        bx = nbx;
        ens_stage_geo(&G, a.box[bx].G);
        __syncthreads();
      }
      if (!(G.eps_sf > 0.0)) continue;   // block-uniform
      const FusedBox &R = a.box[bx];
      int t = (int)(w - p[bx]);
      const int tx = t % R.ntx;
      t /= R.ntx;
      const int ty = t % R.nty, tz = t / R.nty;
      dilate_tile(G, R.raw, R.raw + R.b_int.n, tx * FX, ty * FY, tz * FZ,
                  reinterpret_cast<unsigned long long (*)[2]>(scr), scr + 2 * HZ * HY, scr + 3 * HZ * HY);
    }
    grid.sync();
  }
  {   // tiles: each CTA takes tiles from the concatenated list
    const long *p = pref(FE_TILE);
    unsigned parity = 0u;
    bool dead = false;
    int bx = -1;
    for (long w = blockIdx.x; w < p[nb] && !dead; w += gridDim.x) {
      int nbx = bx < 0 ? 0 : bx;
      while (w >= p[nbx + 1]) ++nbx;
      // the previous tile's shared-memory reads are done before the next copy lands
      __syncthreads();
      if (nbx != bx) {
        bx = nbx;
        ens_stage_geo(&G, a.box[bx].G);
        __syncthreads();
      }
      const FusedBox &R = a.box[bx];
      int t = (int)(w - p[bx]);
      const int tx = t % R.ntx;
      t /= R.ntx;
      const int ty = t % R.nty, tz = t / R.nty;
      const StageMx S = ens_stage_bufs(R, a);
      const bool flags = G.eps_sf > 0.0;
      if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      dead = !tile_body<ENS_NT, true, false, true, PPH>(R.tm, G, S, flags ? R.raw + R.b_int.n : nullptr, R.F[0],
                                                        R.F[1], R.F[2], tx * FX, ty * FY, tz * FZ, R.dflag, 0u, 0,
                                                        sm, parity);
      parity ^= 1u;
    }
  }
  grid.sync();
  // Contact-CT edge EMFs at every site (Sect. 2.4)
  per_box(FE_SITE, [&](const FusedBox &R, long w) {
    int c[3];
    cell_at(R.b_site, w, c);
    const long q = widx(G, c[0], c[1], c[2]), wt = G.wtot;
    const bool interior = c[0] >= 1 && c[0] < G.n[0] && c[1] >= 1 && c[1] < G.n[1] && c[2] >= 1 && c[2] < G.n[2];
    if (c[0] < G.n[0]) R.E[q] = emf_edge<0>(G, c, interior, q, R.W, R.F[1], R.F[2]);
    if (c[1] < G.n[1]) R.E[wt + q] = emf_edge<1>(G, c, interior, q, R.W, R.F[2], R.F[0]);
    if (c[2] < G.n[2]) R.E[2 * wt + q] = emf_edge<2>(G, c, interior, q, R.W, R.F[0], R.F[1]);
  });
  grid.sync();
  // face updates from the curl of the EMFs
  per_box(FE_SITE, [&](const FusedBox &R, long w) {
    int c[3];
    cell_at(R.b_site, w, c);
    const StageMx S = ens_stage_bufs(R, a);
    const float dt = d2f_scaled(*S.dt, -G.e_t);
    if (c[1] < G.n[1] && c[2] < G.n[2]) face_update<0>(G, c, S, dt);
    if (c[0] < G.n[0] && c[2] < G.n[2]) face_update<1>(G, c, S, dt);
    if (c[0] < G.n[0] && c[1] < G.n[1]) face_update<2>(G, c, S, dt);
  });
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
      cudaGetLastError();
  }
  return enc;
}

}  // namespace

cudaError_t fused_init() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  cudaError_t e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<384, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 3, true, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes(true));
  // the PPH instantiations
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, false, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 3, true, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 3, true, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<384, 2, true, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 2, true, true, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 1, true, true, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<288, 3, true, false, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, false, false, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_flux_update_mx<256, 2, true, true, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true));
  done = e;
  return e;
}

bool fused_stage_ok(const DevGeo &G) {
  return G.eos == PHL_EOS_IDEAL && G.nspec == 0 && G.wstr == 8 && G.act[0] && G.act[1] && G.act[2] &&
         G.n[0] >= 4 && G.n[1] >= 4 && G.n[2] >= 4 &&
         G.recon != PHL_RECON_PQH &&   // the tile stages two ghost layers; PQH needs three
         // the tile kernel indexes the state's and the face fluxes' planes with 32-bit offsets
         5 * G.plane < 0x7fffffffL && (long)(G.nf + 1) * G.wtot < 0x7fffffffL;
}

// TMA descriptor of W's two float4 planes as a 4-D tensor (x * 4 floats, y, z,
// plane); the box is one staged tile.  Strides are multiples of 16 bytes
// (float4 rows) and the allocation is 256-byte aligned.
int make_fused_tmap(const DevGeo &G, const float *W, void *tmap128) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc) return set_error(PHL_ECUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[4] = {(cuuint64_t)(4 * G.wy), (cuuint64_t)(G.wz / G.wy), (cuuint64_t)(G.wtot / G.wz), 2};
  cuuint64_t strides[3] = {(cuuint64_t)(G.wy * 16), (cuuint64_t)(G.wz * 16), (cuuint64_t)(G.wtot * 16)};
  cuuint32_t box[4] = {4 * HX, HY, HZ, 2};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc((CUtensorMap *)tmap128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)W, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(PHL_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PHL_OK;
}

// Faces, EMFs and updates of one mixed stage on the fused path (prim and
// flags already done): k_flux_update_mx, three EMF launches, three face
// updates.
cudaError_t launch_raw_flags_form(const DevGeo &G, const float *W, uint8_t *raw, int form, unsigned int *any,
                                  cudaStream_t s) {
  if (form == 1) {
    Box b4 = make_box(0, G.n[0] / 4, 0, G.n[1], 0, G.n[2]);
    k_flag_raw4<<<grid3(b4), block3(b4), 0, s>>>(G, b4, W, raw, any);
  } else {
    Box bi = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    k_flag_raw<float><<<grid3(bi), block3(bi), 0, s>>>(G, bi, W, raw, any);
  }
  return cudaGetLastError();
}

void launch_fused_tail(const DevGeo &G, const MixedBufs &M, bool first, bool last, double b, cudaStream_t s,
                       int *nl, Prof *prof) {
  StageMx S;
  S.U = M.U; S.B = M.B; S.dU = M.dU; S.dB = M.dB;
  S.first = first; S.last = last; S.b = (float)b; S.dt = M.dt;
  S.W = M.W; S.F[0] = M.F[0]; S.F[1] = M.F[1]; S.F[2] = M.F[2]; S.E = M.E;
  const int ntx = (G.n[0] + FX - 1) / FX, nty = (G.n[1] + FY - 1) / FY, ntz = (G.n[2] + FZ - 1) / FZ;
  const int nb = ntx * nty * ntz;
  const long ncell = (long)G.n[0] * G.n[1] * G.n[2];
  const uint8_t *dil = nullptr;
  const unsigned int *any = nullptr;
  int raw_mode = 0;
  if (G.eps_sf > 0.0 && M.pipeline3) {   // the tile kernel dilates the raw flags itself
    dil = M.raw;
    raw_mode = 1;
  } else if (G.eps_sf > 0.0) {   // raw flags, then their 5^3 dilation, both on the interior layout
    Box bi = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    if (M.anyraw) cudaMemsetAsync(M.anyraw, 0, sizeof(unsigned int), s);
    if (flag_raw4_ok(G)) {   // four cells of a row per thread
      Box b4 = make_box(0, G.n[0] / 4, 0, G.n[1], 0, G.n[2]);
      PHL_LAUNCH(KC_FLAG_RAW, prof, s, k_flag_raw4<<<grid3(b4), block3(b4), 0, s>>>(G, b4, M.W, M.raw, M.anyraw));
    } else {
      PHL_LAUNCH(KC_FLAG_RAW, prof, s,
                 k_flag_raw<float><<<grid3(bi), block3(bi), 0, s>>>(G, bi, M.W, M.raw, M.anyraw));
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nbd = std::min(nb, 8 * std::max(nsm, 1));   // eight 256-thread CTAs per SM
    PHL_LAUNCH(KC_FLAG_DILATE, prof, s,
               k_flag_dilate3<<<nbd, 256, 0, s>>>(G, M.raw, M.raw + ncell, ntx, nty, M.anyraw));
    dil = M.raw + ncell;
    any = M.anyraw;
    *nl += 2;
  }
  const CUtensorMap *tm = (const CUtensorMap *)M.tmapW;
  // launch shapes: (threads, min CTAs per SM, phased)
#define PHL_FUSED1(NT, MB, PH, PA, LRS, PP)                                                                     \
  PHL_LAUNCH(KC_FLUX_UPDATE, prof, s,                                                                          \
             (k_flux_update_mx<NT, MB, PH, PA, LRS, PP><<<nb, NT, smem_bytes(PH), s>>>(*tm, G, S, dil, M.F[0],   \
                                                                                   M.F[1], M.F[2], ntx, nty,     \
                                                                                   M.dflag, M.test_extra_tx, raw_mode, any)))
  // the reconstruction is a template parameter: the van Leer kernels carry no PPH code
#define PHL_FUSED(NT, MB, PH, PA, LRS)                      \
  do {                                                     \
    if (G.recon == PHL_RECON_PPH) PHL_FUSED1(NT, MB, PH, PA, LRS, true); \
    else PHL_FUSED1(NT, MB, PH, PA, LRS, false);           \
  } while (0)
  switch (M.fused_variant) {
    case 2: PHL_FUSED(288, 3, true, false, false); break;
    case 3: PHL_FUSED(256, 3, true, false, false); break;
    case 4: PHL_FUSED(384, 2, true, false, false); break;
    case 5: PHL_FUSED(288, 1, true, true, false); break;
    case 6: PHL_FUSED(256, 2, true, true, false); break;
    case 7: PHL_FUSED(288, 2, true, true, false); break;
    case 8: PHL_FUSED(288, 3, true, false, true); break;
    case 9: PHL_FUSED(256, 2, false, false, true); break;
    default: PHL_FUSED(256, 2, false, false, false); break;
  }
#undef PHL_FUSED
#undef PHL_FUSED1
  ++*nl;
  if (M.pipeline3) {   // Contact-CT with the face update, then the next stage's primitives and raw flags
    const int ctx = (G.n[0] + CTT - 1) / CTT, cty = (G.n[1] + CTT - 1) / CTT, ctz = (G.n[2] + CTT - 1) / CTT;
    PHL_LAUNCH(KC_EMF, prof, s, k_ct_faces<<<ctx * cty * ctz, 256, 0, s>>>(G, S, ctx, cty));
    ++*nl;
    launch_prim_flags(G, M, last, M.fmax, s, nl, prof);
    return;
  }
  Box bs = make_box(0, G.n[0] + 1, 0, G.n[1] + 1, 0, G.n[2] + 1);
  const dim3 sg = site_grid(G), sb(EB_X, EB_Y, EB_Z);
  PHL_LAUNCH(KC_EMF, prof, s, k_emf3<<<sg, sb, 0, s>>>(G, bs, M.W, M.F[0], M.F[1], M.F[2], M.E));
  // the face update reads no neighbouring rows beyond one: the linear mapping measured faster
  PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces3<<<grid3(bs), block3(bs), 0, s>>>(G, bs, S));
  *nl += 2;
}

// The persistent fused ensemble: device records of the boxes, the phases'
// prefix sums and the boxes' tensor maps; the grid is every SM times the
// CTAs of the launch shape that fit on one (cooperative launch).
cudaError_t ens_fused_create(const GridView *views, int nbox, EnsFused *out) {
  *out = EnsFused();
  cudaError_t e = fused_init();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ens_fused<false, ENS_MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ens_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ens_fused<true, ENS_MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ens_smem_bytes());
  if (e != cudaSuccess) return e;
  bool pph = false;
  std::vector<FusedBox> h(nbox);
  std::vector<CUtensorMap> tm(nbox);
  std::vector<long> pref((size_t)FE_NPH * (nbox + 1), 0);
  for (int b = 0; b < nbox; ++b) {
    const GridView &v = views[b];
    if (!v.tmapW || !fused_stage_ok(*v.G)) return cudaErrorInvalidValue;
    const DevGeo &G = *v.G;
    if (b == 0) pph = G.recon == PHL_RECON_PPH;
    else if ((G.recon == PHL_RECON_PPH) != pph) return cudaErrorInvalidValue;   // one reconstruction per launch
    FusedBox &R = h[b];
    memset(&R, 0, sizeof(R));
    R.G = G;
    R.U = v.U; R.B = v.B; R.dU = v.dU; R.dB = v.dB; R.W = v.W;
    for (int k = 0; k < 3; ++k) R.F[k] = v.F[k];
    R.E = v.E; R.raw = v.raw; R.dt = v.dt; R.fmax = v.fmax; R.dflag = v.dflag;
    memcpy(&tm[b], v.tmapW, sizeof(CUtensorMap));
    const int n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    R.b_int = make_box(0, n0, 0, n1, 0, n2);
    R.b_work = make_box(-G.ge[0], n0 + G.ge[0], -G.ge[1], n1 + G.ge[1], -G.ge[2], n2 + G.ge[2]);
    R.b_site = make_box(0, n0 + 1, 0, n1 + 1, 0, n2 + 1);
    R.ntx = (n0 + FX - 1) / FX;
    R.nty = (n1 + FY - 1) / FY;
    const long ntiles = (long)R.ntx * R.nty * ((n2 + FZ - 1) / FZ);
    const long items[FE_NPH] = {R.b_int.n, R.b_work.n, G.eps_sf > 0.0 ? R.b_int.n : 0, ntiles, R.b_site.n};
    for (int ph = 0; ph < FE_NPH; ++ph)
      pref[(size_t)ph * (nbox + 1) + b + 1] = pref[(size_t)ph * (nbox + 1) + b] + items[ph];
  }
  void *db = nullptr, *dtm = nullptr, *dp = nullptr;
  e = cudaMalloc(&db, sizeof(FusedBox) * nbox);
  if (e == cudaSuccess) e = cudaMalloc(&dtm, sizeof(CUtensorMap) * nbox);   // 256-byte aligned: TMA descriptors
  if (e == cudaSuccess) e = cudaMalloc(&dp, sizeof(long) * pref.size());
  if (e == cudaSuccess) e = cudaMemcpy(dtm, tm.data(), sizeof(CUtensorMap) * nbox, cudaMemcpyHostToDevice);
  for (int b = 0; b < nbox; ++b) h[b].tm = (const CUtensorMap *)dtm + b;
  if (e == cudaSuccess) e = cudaMemcpy(db, h.data(), sizeof(FusedBox) * nbox, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dp, pref.data(), sizeof(long) * pref.size(), cudaMemcpyHostToDevice);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pph ? (const void *)k_ens_fused<true, ENS_MINB>
                                                                    : (const void *)k_ens_fused<false, ENS_MINB>,
                                                      ENS_NT, ens_smem_bytes());
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) {
    cudaFree(db); cudaFree(dtm); cudaFree(dp);
    return e;
  }
  out->boxes = db;
  out->tmaps = dtm;
  out->pref = (long *)dp;
  out->nbox = nbox;
  out->pph = pph;
  out->blocks = per_sm * sms;
  out->per_sm = per_sm;
  return cudaSuccess;
}

void ens_fused_destroy(EnsFused *e) {
  if (e->boxes) cudaFree(e->boxes);
  if (e->tmaps) cudaFree(e->tmaps);
  if (e->pref) cudaFree(e->pref);
  *e = EnsFused();
}

cudaError_t launch_ens_fused(const EnsFused &E, int stage, int nstages, float b, cudaStream_t s) {
  FusedEnsArgs a;
  a.box = (const FusedBox *)E.boxes;
  a.pref = E.pref;
  a.nbox = E.nbox;
  a.stage = stage;
  a.nstages = nstages;
  a.b = b;
  void *args[] = {&a};
  const void *fn = E.pph ? (const void *)k_ens_fused<true, ENS_MINB> : (const void *)k_ens_fused<false, ENS_MINB>;
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)E.blocks), dim3(ENS_NT), args, ens_smem_bytes(), s);
}

}  // namespace phl
