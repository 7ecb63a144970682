// stage_common.cuh -- launch helpers and the stage kernels shared by the FP64
// and mixed-precision paths, templated on the arithmetic type R of the work
// arrays (primitive deviations W, face fluxes F, edge EMFs E).
#pragma once
#include <math.h>

#include "phl_internal.cuh"

namespace phl {
namespace stage {
namespace {   // internal linkage: each translation unit gets its own kernels


constexpr int TPB = 256;

// launch with optional event bracketing for the per-kernel timing
#define PHL_LAUNCH(cls, prof, s, ...)        \
  do {                                       \
    if (prof) (prof)->begin((cls), (s));     \
    __VA_ARGS__;                             \
    if (prof) (prof)->end(s);                \
  } while (0)

struct Box {
  int lo[3], hi[3];
  long n;
  FastDiv fx, fy;   // divisions by the x and y extents
};

inline Box make_box(int lx, int hx, int ly, int hy, int lz, int hz) {
  Box b;
  b.lo[0] = lx; b.hi[0] = hx; b.lo[1] = ly; b.hi[1] = hy; b.lo[2] = lz; b.hi[2] = hz;
  b.n = (long)(hx - lx) * (hy - ly) * (hz - lz);
  b.fx = make_fastdiv((unsigned)(hx - lx));
  b.fy = make_fastdiv((unsigned)(hy - ly));
  return b;
}

// One thread per box element, 1D launch; the (i, j, k) decode uses FastDiv.
inline dim3 block3(const Box &) { return dim3(256, 1, 1); }
inline dim3 grid3(const Box &b) { return dim3((unsigned)((b.n + 255) / 256), 1, 1); }
// Cell of linear index tl in the box (x fastest); false beyond the box.
__device__ __forceinline__ bool cell_at(const Box &b, long tl, int *c) {
  if (tl >= b.n) return false;
  const unsigned t = (unsigned)tl;
  const unsigned q1 = fastdiv(t, b.fx);
  const unsigned q2 = fastdiv(q1, b.fy);
  c[0] = b.lo[0] + (int)(t - q1 * b.fx.d);
  c[1] = b.lo[1] + (int)(q1 - q2 * b.fy.d);
  c[2] = b.lo[2] + (int)q2;
  return true;
}
__device__ __forceinline__ bool cell3(const Box &b, int *c) {
  return cell_at(b, blockIdx.x * (long)blockDim.x + threadIdx.x, c);
}

__device__ __forceinline__ void unflat(const Box &b, long t, int *c) {
  const int ex = b.hi[0] - b.lo[0], ey = b.hi[1] - b.lo[1];
  c[0] = b.lo[0] + (int)(t % ex);
  t /= ex;
  c[1] = b.lo[1] + (int)(t % ey);
  t /= ey;
  c[2] = b.lo[2] + (int)t;
}

inline int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// van Leer harmonic limited slope (Sect. 2.5, item i).  In FP32 (the mixed
// form, O(1) deviations in scaled units) the quotient takes the fast
// division, as the tile kernel's paired slopes do, so a cell reconstructs
// the same way on every path.
template <typename R>
__device__ __forceinline__ R vl_slope(R a, R b, R c) {
  const R dm = b - a, dp = c - b;
  if constexpr (sizeof(R) == 4) return (dm * dp > R(0)) ? __fdividef(R(2) * dm * dp, dm + dp) : R(0);
  else return (dm * dp > R(0)) ? R(2) * dm * dp / (dm + dp) : R(0);
}

// PPH (Sect. 2.5, item ii): the parabola whose averages over cells i-1, i,
// i+1 are (a, b, c), at the cell's right and left faces; unlimited.
template <typename R>
__device__ __forceinline__ R pph_right(R a, R b, R c) { return (-a + R(5) * b + R(2) * c) / R(6); }
template <typename R>
__device__ __forceinline__ R pph_left(R a, R b, R c) { return (R(2) * a + R(5) * b - c) / R(6); }
// Limited parabola for mass fractions: face values clipped to the range of the
// two cells sharing the face, a local extremum stays constant, and the far
// face value is pulled back where the parabola would overshoot inside the
// cell (the piecewise parabolic method's monotonicity constraints, Colella &
// Woodward 1984).  Returns the cell's left and right face values.
template <typename R>
__device__ __forceinline__ void pph_limited(R a, R b, R c, R &fl, R &fr) {
  if ((b - a) * (c - b) <= R(0)) { fl = b; fr = b; return; }
  R l = pph_left(a, b, c), r = pph_right(a, b, c);
  l = fmin(fmax(l, fmin(a, b)), fmax(a, b));
  r = fmin(fmax(r, fmin(b, c)), fmax(b, c));
  const R d = r - l, a6 = R(6) * (b - R(0.5) * (l + r));
  if (d * a6 > d * d) l = R(3) * b - R(2) * r;
  else if (d * a6 < -d * d) r = R(3) * b - R(2) * l;
  fl = l;
  fr = r;
}

// Limited fifth-order reconstruction (Sect. 2.5, item iii; the cited PQH
// method is not printed): the face value of the degree-4 polynomial whose
// averages over five cells are the cell values, limited by the
// monotonicity-preserving bounds of Suresh & Huynh (1997).  mp5_face(a..e):
// the value at the face between c and d; the left face of c is
// mp5_face(e, d, c, b, a).
template <typename R>
__device__ __forceinline__ R mm2(R x, R y) {
  return (x > R(0) && y > R(0)) ? fmin(x, y) : ((x < R(0) && y < R(0)) ? fmax(x, y) : R(0));
}
template <typename R>
__device__ __forceinline__ R mp5_face(R a, R b, R c, R d, R e) {
  const R vor = (R(2) * a - R(13) * b + R(47) * c + R(27) * d - R(3) * e) / R(60);
  const R vmp = c + mm2(d - c, R(4) * (c - b));
  if ((vor - c) * (vor - vmp) <= R(0)) return vor;
  const R djm1 = a - R(2) * b + c, dj = b - R(2) * c + d, djp1 = c - R(2) * d + e;
  const R dm4p = mm2(mm2(R(4) * dj - djp1, R(4) * djp1 - dj), mm2(dj, djp1));
  const R dm4m = mm2(mm2(R(4) * dj - djm1, R(4) * djm1 - dj), mm2(dj, djm1));
  const R vul = c + R(4) * (c - b);
  const R vmd = R(0.5) * (c + d) - R(0.5) * dm4p;
  const R vlc = c + R(0.5) * (c - b) + R(4.0 / 3.0) * dm4m;
  const R lo = fmax(fmin(fmin(c, d), vmd), fmin(fmin(c, vul), vlc));
  const R hi = fmin(fmax(fmax(c, d), vmd), fmax(fmax(c, vul), vlc));
  return vor + mm2(lo - vor, hi - vor);
}

__device__ __forceinline__ long wstride(const DevGeo &G, int d) { return d == 0 ? 1L : (d == 1 ? G.wy : G.wz); }

template <typename R>
__device__ __forceinline__ bool k_flag_raw_at(long tl, const DevGeo &G, const Box &box, const R *__restrict__ W, uint8_t *__restrict__ raw) {
  {
    int c[3];
    if (!cell_at(box, tl, c)) return false;
    const long q = widx(G, c[0], c[1], c[2]);
    auto P = [&](long r) {
      if constexpr (sizeof(R) == 4) return W[waux(G, AUX_P, r)];
      else return W[wix<R>(G, W_P, r)];
    };
    const R P0 = P(q) + bg_cell_t<R>(G, c[2]).p;
    R sum = R(0);
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const long sd = wstride(G, d);
      const int kp = c[2] + (d == 2), km = c[2] - (d == 2);
      const R Pp = P(q + sd) + bg_cell_t<R>(G, kp).p;
      const R Pm = P(q - sd) + bg_cell_t<R>(G, km).p;
      sum += fabs(Pp - Pm);
    }
    const bool f = sum / (eps_sf_t<R>(G) * P0) > R(1);
    raw[c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])] = f ? 1 : 0;
    return f;
  }
}
// any (optional, zeroed before the launch): set to 1 when some cell of the
// box is flagged -- one atomic per warp that holds a flagged cell, none in a
// flow without shocks, where the dilation and its loads are then skipped.
// The block size is a multiple of 32 and no thread leaves before the vote.
template <typename R>
__global__ void k_flag_raw(DevGeo G, Box box, const R *__restrict__ W, uint8_t *__restrict__ raw,
                           unsigned int *any = nullptr) {
  const bool f = k_flag_raw_at<R>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, W, raw);
  if (any && __any_sync(0xffffffffu, f) && (threadIdx.x & 31) == 0) atomicOr(any, 1u);
}

// The raw flags of four cells of a row per thread (x0 = 4m .. 4m + 3; the
// mixed form with n_x a multiple of 4): each cell's test with the operations
// of k_flag_raw_at (bit-identical flags), the x-neighbours' pressures shared
// between the four, the background read once, one 4-byte store.  box: the
// interior with its x extent divided by 4.  any: as k_flag_raw.
__global__ void __launch_bounds__(256) k_flag_raw4(DevGeo G, Box box, const float *__restrict__ W,
                                                   uint8_t *__restrict__ raw, unsigned int *any) {
  int c[3];
  unsigned fw = 0u;
  if (cell_at(box, blockIdx.x * (long)blockDim.x + threadIdx.x, c)) {
    c[0] *= 4;
    const float *P = W + waux(G, AUX_P, 0);
    const long q = widx(G, c[0], c[1], c[2]);
    const float b0 = bg_cell_t<float>(G, c[2]).p;
    float px[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) px[i] = P[q - 1 + i] + b0;
    float sy[4], sz[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { sy[i] = 0.0f; sz[i] = 0.0f; }
    if (G.act[1]) {
#pragma unroll
      for (int i = 0; i < 4; ++i) sy[i] = fabsf((P[q + i + G.wy] + b0) - (P[q + i - G.wy] + b0));
    }
    if (G.act[2]) {
      const float bp = bg_cell_t<float>(G, c[2] + 1).p, bm = bg_cell_t<float>(G, c[2] - 1).p;
#pragma unroll
      for (int i = 0; i < 4; ++i) sz[i] = fabsf((P[q + i + G.wz] + bp) - (P[q + i - G.wz] + bm));
    }
    const float e = eps_sf_t<float>(G);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float sum = 0.0f;
      sum += fabsf(px[i + 2] - px[i]);   // x is active on this path
      if (G.act[1]) sum += sy[i];
      if (G.act[2]) sum += sz[i];
      if (sum / (e * px[i + 1]) > 1.0f) fw |= 1u << (8 * i);
    }
    *reinterpret_cast<unsigned *>(raw + c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])) = fw;
  }
  if (any && __any_sync(0xffffffffu, fw != 0u) && (threadIdx.x & 31) == 0) atomicOr(any, 1u);
}
__host__ __device__ inline bool flag_raw4_ok(const DevGeo &G) { return G.act[0] && G.n[0] % 4 == 0; }

// 5^d dilation of the raw shock flags (Sect. 2.7), done as one 5-wide OR per
// active axis: OR over a box equals the nested ORs over its axes.  Neighbours
// beyond a periodic boundary wrap, beyond any other boundary are skipped.
template <int D>
__device__ __forceinline__ void k_dilate_axis_at(long tl, const DevGeo &G, const Box &box, const uint8_t *__restrict__ in, uint8_t *__restrict__ out) {
  {
    int c[3];
    if (!cell_at(box, tl, c)) return;
    const int n = G.n[D];
    const bool per = G.bc[D][0] == 0;
    uint8_t f = 0;
    for (int d = -2; d <= 2; ++d) {
      int cc[3] = {c[0], c[1], c[2]};
      int x = c[D] + d;
      if (x < 0 || x >= n) {
        if (!per) continue;
        x = (x + n) % n;
      }
      cc[D] = x;
      f |= in[cc[0] + (long)G.n[0] * (cc[1] + (long)G.n[1] * cc[2])];
    }
    out[c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])] = f;
  }
}
template <int D>
__global__ void k_dilate_axis(DevGeo G, Box box, const uint8_t *__restrict__ in, uint8_t *__restrict__ out) {
  k_dilate_axis_at<D>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, in, out);
}

// Flags of the cells the face stencils touch ([-1, n] on active axes): a ghost
// cell carries the flag of the interior cell its data comes from.
__device__ __forceinline__ void k_flag_expand_at(long tl, const DevGeo &G, const Box &box, const uint8_t *__restrict__ dil, uint8_t *__restrict__ flag) {
  {
    int c[3], s[3];
    if (!cell_at(box, tl, c)) return;
    for (int d = 0; d < 3; ++d) {
      bool fl;
      s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl) : 0;
    }
    flag[widx(G, c[0], c[1], c[2])] = dil[s[0] + (long)G.n[0] * (s[1] + (long)G.n[1] * s[2])];
  }
}
__global__ void k_flag_expand(DevGeo G, Box box, const uint8_t *__restrict__ dil, uint8_t *__restrict__ flag) {
  k_flag_expand_at(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, dil, flag);
}

// raw -> dilated (interior) -> flags on the work layout; tmp: one interior byte field.
inline int launch_flags(const DevGeo &G, uint8_t *raw, uint8_t *tmp, uint8_t *flag, cudaStream_t s, Prof *prof) {
  Box bi = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  uint8_t *a = raw, *b = tmp;
  int nl = 0;
  for (int D = 0; D < 3; ++D) {
    if (!G.act[D]) continue;
    if (D == 0) PHL_LAUNCH(KC_FLAG_DILATE, prof, s, k_dilate_axis<0><<<grid3(bi), block3(bi), 0, s>>>(G, bi, a, b));
    if (D == 1) PHL_LAUNCH(KC_FLAG_DILATE, prof, s, k_dilate_axis<1><<<grid3(bi), block3(bi), 0, s>>>(G, bi, a, b));
    if (D == 2) PHL_LAUNCH(KC_FLAG_DILATE, prof, s, k_dilate_axis<2><<<grid3(bi), block3(bi), 0, s>>>(G, bi, a, b));
    uint8_t *t = a; a = b; b = t;
    ++nl;
  }
  int l[3], h[3];
  for (int d = 0; d < 3; ++d) {
    if (G.act[d]) { l[d] = -1; h[d] = G.n[d] + 1; } else { l[d] = 0; h[d] = 1; }
  }
  Box be = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
  PHL_LAUNCH(KC_FLAG_DILATE, prof, s, k_flag_expand<<<grid3(be), block3(be), 0, s>>>(G, be, a, flag));
  return nl + 1;
}

// Flux at the D-face of work cell c (index pR, left neighbour pR - sd).
// fetch(v, k) returns component v of W at stencil cell k = 0..3 (pL - sd, pL,
// pR, pR + sd).  Stores F - F_hat and the contact direction.
template <int D, typename R, int NS, typename Fetch>
__device__ __forceinline__ void flux_face(const DevGeo &G, const int *c, long pR, Fetch fetch,
                                          const double *__restrict__ Bf, const R *__restrict__ dB,
                                          const uint8_t *__restrict__ flag, R *__restrict__ F, int *dflag) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const long sd = wstride(G, D);
  const long pL = pR - sd;
  constexpr int NWC = W_X0 + NS;   // components this instantiation can hold
  R wl[NWC], wr[NWC];
  const bool ideal = G.eos == 0;   // ideal gas: gamma_e = gamma_c = gamma (not reconstructed)
  // shock flattening (Sect. 2.7): a flagged cell reconstructs with van Leer
  const bool vlL = G.recon == PHL_RECON_VANLEER || flag[pL], vlR = G.recon == PHL_RECON_VANLEER || flag[pR];
  R ql[NWC], qr[NWC];
#pragma unroll
  for (int v = 0; v < NWC; ++v) {
    if (v >= G.nw || (ideal && (v == W_GE || v == W_GC))) continue;
    const R w0 = fetch(v, 0), w1 = fetch(v, 1), w2 = fetch(v, 2), w3 = fetch(v, 3);
    if (G.recon == PHL_RECON_PQH && (!vlL || !vlR)) {   // cells pL-2..pR+2 (three ghost layers)
      const R wm = fetch(v, -1), w4 = fetch(v, 4);
      ql[v] = vlL ? w1 + R(0.5) * vl_slope(w0, w1, w2) : mp5_face(wm, w0, w1, w2, w3);
      qr[v] = vlR ? w2 - R(0.5) * vl_slope(w1, w2, w3) : mp5_face(w4, w3, w2, w1, w0);
    } else if (!vlL || !vlR) {   // PPH: left state from cell pL's right face, right state from pR's left face
      R pl, pr;
      if (v < W_X0) {
        pl = pph_right(w0, w1, w2);
        pr = pph_left(w1, w2, w3);
      } else {
        R fl, fr;
        pph_limited(w0, w1, w2, fl, fr);
        pl = fr;
        pph_limited(w1, w2, w3, fl, fr);
        pr = fl;
      }
      ql[v] = vlL ? w1 + R(0.5) * vl_slope(w0, w1, w2) : pl;
      qr[v] = vlR ? w2 - R(0.5) * vl_slope(w1, w2, w3) : pr;
    } else {
      ql[v] = w1 + R(0.5) * vl_slope(w0, w1, w2);
      qr[v] = w2 - R(0.5) * vl_slope(w1, w2, w3);
    }
  }
  if (ideal) {   // not used by the ideal-gas solver (constant gamma)
    ql[W_GE] = qr[W_GE] = R(0);
    ql[W_GC] = qr[W_GC] = R(0);
  }
  wl[RD_RHO] = ql[W_RHO];        wr[RD_RHO] = qr[W_RHO];
  wl[RD_UN] = ql[W_VX + D];      wr[RD_UN] = qr[W_VX + D];
  wl[RD_UT1] = ql[W_VX + T1];    wr[RD_UT1] = qr[W_VX + T1];
  wl[RD_UT2] = ql[W_VX + T2];    wr[RD_UT2] = qr[W_VX + T2];
  wl[RD_BT1] = ql[W_BX + T1];    wr[RD_BT1] = qr[W_BX + T1];
  wl[RD_BT2] = ql[W_BX + T2];    wr[RD_BT2] = qr[W_BX + T2];
  wl[RD_P] = ql[W_P];            wr[RD_P] = qr[W_P];
  wl[RD_GE] = ql[W_GE];          wr[RD_GE] = qr[W_GE];
  wl[RD_GC] = ql[W_GC];          wr[RD_GC] = qr[W_GC];
#pragma unroll
  for (int l = 0; l < NS; ++l)
    if (l < G.nspec) { wl[RD_X0 + l] = ql[W_X0 + l]; wr[RD_X0 + l] = qr[W_X0 + l]; }
  const BgT<R> bf = (D == 2) ? bg_zface_t<R>(G, c[2]) : bg_cell_t<R>(G, c[2]);
  if (!(bf.rho + wl[RD_RHO] > R(0) && bf.rho + wr[RD_RHO] > R(0) && bf.p + wl[RD_P] > R(0) &&
        bf.p + wr[RD_P] > R(0)))
    atomicOr(dflag, FLAG_NEG);
  // normal field on this face; transverse ghost rows map to their source rows
  int s[3];
  s[D] = c[D];
  {
    bool fl;
    s[T1] = G.act[T1] ? cell_src(c[T1], G.n[T1], G.bc[T1][0], G.bc[T1][1], fl) : 0;
    s[T2] = G.act[T2] ? cell_src(c[T2], G.n[T2], G.bc[T2][0], G.bc[T2][1], fl) : 0;
  }
  const long qb = (long)D * G.plane + sidx(G, s[0], s[1], s[2]);
  R bn;
  if constexpr (sizeof(R) == 4) {   // B^n + dB in scaled units
    const float b0 = d2f_scaled(Bf[qb], -G.e_b);
    bn = dB ? b0 + dB[qb] : b0;
  }
  else bn = (R)Bf[qb];
  const int solver = (flag[pL] | flag[pR]) ? SOLVER_HLL : G.riemann;
  R f[7 + NS];
  int up;
  if (G.eos == 0) {   // ideal gas: gamma constant
    GasK<R> K;
    K.g = sizeof(R) == 4 ? (R)G.gammaf : (R)G.gamma;
    K.igm1 = R(1) / (K.g - R(1));
    K.ggm1 = K.g * K.igm1;
    riemann_dev<R, NS, true>(wl, wr, bn, bf.rho, bf.p, bf.ge, bf.gc, G.nspec, solver, mach_thr_t<R>(G), f, up, K);
  } else {
    riemann_dev<R, NS, false>(wl, wr, bn, bf.rho, bf.p, bf.ge, bf.gc, G.nspec, solver, mach_thr_t<R>(G), f, up);
  }
  // reflecting wall face: a symmetry plane (Table bcs, u_n = 0, B_n = 0); only
  // the normal-momentum flux survives, the others are exactly zero
  if ((c[D] == 0 && G.bc[D][0] == 1) || (c[D] == G.n[D] && G.bc[D][1] == 1)) {
#pragma unroll
    for (int q = 0; q < 7 + NS; ++q)
      if (q != RF_MN) f[q] = R(0);
    up = 0;
  }
  const long wt = G.wtot;
  F[F_RHO * wt + pR] = f[RF_RHO];
  F[(F_MX + D) * wt + pR] = f[RF_MN];
  F[(F_MX + T1) * wt + pR] = f[RF_MT1];
  F[(F_MX + T2) * wt + pR] = f[RF_MT2];
  F[F_E * wt + pR] = f[RF_E];
  F[(F_BX + T1) * wt + pR] = f[RF_BT1];
  F[(F_BX + T2) * wt + pR] = f[RF_BT2];
#pragma unroll
  for (int l = 0; l < NS; ++l)
    if (l < G.nspec) F[(F_X0 + l) * wt + pR] = f[RF_X0 + l];
  F[(long)G.nf * wt + pR] = (R)up;   // contact direction for Contact-CT
}

template <int D, typename R, int NS>
__device__ __forceinline__ void k_flux_at(long tl, const DevGeo &G, const Box &box, const R *__restrict__ W,
                                          const double *__restrict__ Bf, const R *__restrict__ dB,
                                          const uint8_t *__restrict__ flag, R *__restrict__ F, int *dflag) {
  int c[3];
  if (!cell_at(box, tl, c)) return;
  const long sd = wstride(G, D);
  const long pR = widx(G, c[0], c[1], c[2]);
  const long base = pR - 2 * sd;
  auto fetch = [&](int v, int k) -> R { return W[wix<R>(G, v, base + k * sd)]; };
  flux_face<D, R, NS>(G, c, pR, fetch, Bf, dB, flag, F, dflag);
}

template <int D, typename R, int NS>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 1) k_flux(DevGeo G, Box box, const R *__restrict__ W, const double *__restrict__ Bf,
                       const R *__restrict__ dB, const uint8_t *__restrict__ flag, R *__restrict__ F, int *dflag) {
  k_flux_at<D, R, NS>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, W, Bf, dB, flag, F, dflag);
}

// Edge EMF along D at the lower corner (a-1/2, b-1/2), (D, A, B) cyclic.
template <int D, typename R>
__device__ __forceinline__ void k_emf_at(long tl, const DevGeo &G, const Box &box, const R *__restrict__ W, const R *__restrict__ FA,
                      const R *__restrict__ FB, R *__restrict__ E) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  {
    int c[3];
    if (!cell_at(box, tl, c)) return;
    const long p = widx(G, c[0], c[1], c[2]);
    const long wt = G.wtot;
    R e;
    if (G.act[A] && G.act[B]) {
      const long sa = wstride(G, A), sb = wstride(G, B);
      const R *fab = FA + (F_BX + B) * wt;   // F_a(B_b) on a-faces
      const R *fba = FB + (F_BX + A) * wt;   // F_b(B_a) on b-faces
      const R Ea1 = -fab[p], Ea0 = -fab[p - sb];
      const R Eb1 = fba[p], Eb0 = fba[p - sa];
      // contact directions stored after the nf flux components
      const R *ua = FA + (long)G.nf * wt, *ub = FB + (long)G.nf * wt;
      const R ma1 = ua[p], ma0 = ua[p - sb];
      const R mb1 = ub[p], mb0 = ub[p - sa];
      auto ec = [&](long q) -> R {
        if constexpr (sizeof(R) == 4) return W[waux(G, AUX_E + D, q)];
        else
          return -(W[wix<R>(G, W_VX + A, q)] * W[wix<R>(G, W_BX + B, q)] -
                   W[wix<R>(G, W_VX + B, q)] * W[wix<R>(G, W_BX + A, q)]);
      };
      const R E00 = ec(p - sa - sb), E10 = ec(p - sb), E01 = ec(p - sa), E11 = ec(p);
      const R lo_l = Eb0 - E00, lo_r = Eb1 - E10;
      const R up_l = E01 - Eb0, up_r = E11 - Eb1;
      const R h = R(0.5), q4 = R(0.25);
      const R dlo = ma0 > R(0) ? lo_l : (ma0 < R(0) ? lo_r : h * (lo_l + lo_r));
      const R dup = ma1 > R(0) ? up_l : (ma1 < R(0) ? up_r : h * (up_l + up_r));
      const R le_d = Ea0 - E00, le_u = Ea1 - E01;
      const R ri_d = E10 - Ea0, ri_u = E11 - Ea1;
      const R dle = mb0 > R(0) ? le_d : (mb0 < R(0) ? le_u : h * (le_d + le_u));
      const R dri = mb1 > R(0) ? ri_d : (mb1 < R(0) ? ri_u : h * (ri_d + ri_u));
      e = q4 * (Ea1 + Ea0 + Eb1 + Eb0) + q4 * (dlo - dup) + q4 * (dle - dri);
    } else if (G.act[A]) {
      e = -FA[(F_BX + B) * wt + p];
    } else {
      e = FB[(F_BX + A) * wt + p];
    }
    // edge on a reflecting wall: u_n = B_n = 0 there (Table bcs), so the
    // tangential EMF -(u x B)_t is zero
    if ((G.act[A] && ((c[A] == 0 && G.bc[A][0] == 1) || (c[A] == G.n[A] && G.bc[A][1] == 1))) ||
        (G.act[B] && ((c[B] == 0 && G.bc[B][0] == 1) || (c[B] == G.n[B] && G.bc[B][1] == 1))))
      e = R(0);
    E[(long)D * wt + p] = e;
  }
}
template <int D, typename R>
__global__ void k_emf(DevGeo G, Box box, const R *__restrict__ W, const R *__restrict__ FA,
                      const R *__restrict__ FB, R *__restrict__ E) {
  k_emf_at<D, R>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, W, FA, FB, E);
}


// Launch of k_flux<D, R, NS> with NS = 0 (no mass fractions) or PHL_NSPEC_MAX.
template <typename R>
inline void launch_flux(int D, const DevGeo &G, const Box &b, const R *W, const double *Bf, const R *dB,
                        const uint8_t *flag, R *F, int *dflag, cudaStream_t s, Prof *prof) {
  const int kc = D == 0 ? KC_FLUX_X : (D == 1 ? KC_FLUX_Y : KC_FLUX_Z);
  const dim3 gr = grid3(b), bl = block3(b);
#define PHL_FLUX(DD, NN) PHL_LAUNCH(kc, prof, s, (k_flux<DD, R, NN><<<gr, bl, 0, s>>>(G, b, W, Bf, dB, flag, F, dflag)))
  if (G.nspec == 0) {
    if (D == 0) PHL_FLUX(0, 0);
    if (D == 1) PHL_FLUX(1, 0);
    if (D == 2) PHL_FLUX(2, 0);
  } else {
    if (D == 0) PHL_FLUX(0, PHL_NSPEC_MAX);
    if (D == 1) PHL_FLUX(1, PHL_NSPEC_MAX);
    if (D == 2) PHL_FLUX(2, PHL_NSPEC_MAX);
  }
#undef PHL_FLUX
}

}  // namespace
}  // namespace stage
}  // namespace phl
