// kernels_fp64.cu -- FP64 stage of the explicit MHD scheme, one kernel per
// step of the paper's algorithm, with per-stage scratch in HBM.
//
//   k_prim        primitives + EOS at every cell the stencils touch, as
//                 deviations from the background (Sects. 2.2, 2.8); ghost
//                 cells are produced by mapping to their interior source cell
//                 (Table bcs) -- no ghost storage in the state.
//   k_flag_raw    shock indicator of Sect. 2.7 on interior cells.
//   k_flag_dilate 5^d dilation of the indicator (Sect. 2.7).
//   k_flux<D>     van Leer PLM of the deviations (Sect. 2.5), background added
//                 at the face, LHLLD / HLL flux minus F_hat (Eqs. flux-hlld,
//                 pstar, wb1).
//   k_emf<D>      Contact-CT edge EMFs (Sect. 2.4).
//   k_update_*    residual with sources (Eqs. fv, spatres, wb2) and the SSP-RK
//                 combination for cells and faces (Sect. 2.9).
//   k_dt          CFL condition (Eq. cfl): warp-shuffle / block max, one
//                 atomic per block, finalised on the device.
#include <math.h>

#include "phl_internal.cuh"

namespace phl {

namespace {

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
};

Box make_box(int lx, int hx, int ly, int hy, int lz, int hz) {
  Box b;
  b.lo[0] = lx; b.hi[0] = hx; b.lo[1] = ly; b.hi[1] = hy; b.lo[2] = lz; b.hi[2] = hz;
  b.n = (long)(hx - lx) * (hy - ly) * (hz - lz);
  return b;
}

__device__ __forceinline__ void unflat(const Box &b, long t, int *c) {
  const int ex = b.hi[0] - b.lo[0], ey = b.hi[1] - b.lo[1];
  c[0] = b.lo[0] + (int)(t % ex);
  t /= ex;
  c[1] = b.lo[1] + (int)(t % ey);
  t /= ey;
  c[2] = b.lo[2] + (int)t;
}

int nblocks(long n) {
  long b = (n + TPB - 1) / TPB;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ double vl_slope(double a, double b, double c) {
  const double dm = b - a, dp = c - b;
  return (dm * dp > 0.0) ? 2.0 * dm * dp / (dm + dp) : 0.0;
}

__device__ __forceinline__ long wstride(const DevGeo &G, int d) { return d == 0 ? 1L : (d == 1 ? G.wy : G.wz); }

// Primitive deviations of interior cell (i, j, k) from the conserved state.
// Returns false (and sets the device flag) for rho <= 0, P <= 0 or NaN.
__device__ __forceinline__ bool cell_prims(const DevGeo &G, const double *__restrict__ U,
                                           const double *__restrict__ Bf, int i, int j, int k,
                                           double *w, int *dflag) {
  const long p = sidx(G, i, j, k);
  const long pl = G.plane;
  const double rho = U[p];
  const double vx = U[pl + p] / rho, vy = U[2 * pl + p] / rho, vz = U[3 * pl + p] / rho;
  const double bx = 0.5 * (Bf[p] + Bf[p + 1]);
  const double by = 0.5 * (Bf[pl + p] + Bf[pl + p + G.sy]);
  const double bz = 0.5 * (Bf[2 * pl + p] + Bf[2 * pl + p + G.sz]);
  const double eint = U[4 * pl + p] / rho - 0.5 * (vx * vx + vy * vy + vz * vz) -
                      0.5 * (bx * bx + by * by + bz * bz) / rho;
  const double P = (G.gamma - 1.0) * rho * eint;
  const Bg b = bg_cell(G, k);
  w[W_RHO] = rho - b.rho;
  w[W_VX] = vx; w[W_VY] = vy; w[W_VZ] = vz;
  w[W_BX] = bx; w[W_BY] = by; w[W_BZ] = bz;
  w[W_P] = P - b.p;
  w[W_GE] = G.gamma - b.ge;
  w[W_GC] = G.gamma - b.gc;
  for (int l = 0; l < G.nspec; ++l) w[W_X0 + l] = U[(U_X0 + l) * pl + p] / rho;
  bool ok = true;
  if (!(rho > 0.0) || !(P > 0.0)) { atomicOr(dflag, FLAG_NEG); ok = false; }
  if (!isfinite(P) || !isfinite(rho)) { atomicOr(dflag, FLAG_NAN); ok = false; }
  return ok;
}

__global__ void k_prim(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                       double *__restrict__ W, int *dflag) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3], s[3];
    bool fl[3];
    unflat(box, t, c);
    for (int d = 0; d < 3; ++d) {
      fl[d] = false;
      s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]) : 0;
    }
    double w[NW_MAX];
    cell_prims(G, U, Bf, s[0], s[1], s[2], w, dflag);
    for (int d = 0; d < 3; ++d)
      if (fl[d]) { w[W_VX + d] = -w[W_VX + d]; w[W_BX + d] = -w[W_BX + d]; }
    const long q = widx(G, c[0], c[1], c[2]);
    for (int v = 0; v < G.nw; ++v) W[v * G.wtot + q] = w[v];
  }
}

__global__ void k_flag_raw(DevGeo G, Box box, const double *__restrict__ W, uint8_t *__restrict__ raw) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    const long q = widx(G, c[0], c[1], c[2]);
    const double *P = W + (long)W_P * G.wtot;
    const double P0 = P[q] + bg_cell(G, c[2]).p;
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const long sd = wstride(G, d);
      const int kp = c[2] + (d == 2), km = c[2] - (d == 2);
      const double Pp = P[q + sd] + bg_cell(G, kp).p;
      const double Pm = P[q - sd] + bg_cell(G, km).p;
      sum += fabs(Pp - Pm);
    }
    raw[c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])] = (sum / (G.eps_sf * P0) > 1.0) ? 1 : 0;
  }
}

__global__ void k_flag_dilate(DevGeo G, Box box, const uint8_t *__restrict__ raw, uint8_t *__restrict__ flag) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3], s[3];
    unflat(box, t, c);
    for (int d = 0; d < 3; ++d) {
      bool fl;
      s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl) : 0;
    }
    const int r0 = G.act[0] ? 2 : 0, r1 = G.act[1] ? 2 : 0, r2 = G.act[2] ? 2 : 0;
    uint8_t f = 0;
    for (int dk = -r2; dk <= r2 && !f; ++dk)
      for (int dj = -r1; dj <= r1 && !f; ++dj)
        for (int di = -r0; di <= r0 && !f; ++di) {
          int cc[3] = {s[0] + di, s[1] + dj, s[2] + dk};
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            if (cc[d] < 0 || cc[d] >= G.n[d]) {
              const int bc = cc[d] < 0 ? G.bc[d][0] : G.bc[d][1];
              if (bc != 0) { ok = false; break; }
              cc[d] = ((cc[d] % G.n[d]) + G.n[d]) % G.n[d];
            }
          }
          if (ok && raw[cc[0] + (long)G.n[0] * (cc[1] + (long)G.n[1] * cc[2])]) f = 1;
        }
    flag[widx(G, c[0], c[1], c[2])] = f;
  }
}

template <int D>
__global__ void k_flux(DevGeo G, Box box, const double *__restrict__ W, const double *__restrict__ Bf,
                       const uint8_t *__restrict__ flag, double *__restrict__ F, int *dflag) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    const long sd = wstride(G, D);
    const long pR = widx(G, c[0], c[1], c[2]), pL = pR - sd;
    double wl[NW_MAX], wr[NW_MAX];
    const int nrec = (G.eos == 0) ? W_GE : G.nw;   // ideal gas: gamma_e = gamma_c = gamma
    double ql[NW_MAX], qr[NW_MAX];
    for (int v = 0; v < G.nw; ++v) {
      if (v >= nrec && v < W_X0) continue;
      const double *a = W + v * G.wtot;
      const double w0 = a[pL - sd], w1 = a[pL], w2 = a[pR], w3 = a[pR + sd];
      ql[v] = w1 + 0.5 * vl_slope(w0, w1, w2);
      qr[v] = w2 - 0.5 * vl_slope(w1, w2, w3);
    }
    if (G.eos == 0) {
      ql[W_GE] = qr[W_GE] = W[W_GE * G.wtot + pR];
      ql[W_GC] = qr[W_GC] = W[W_GC * G.wtot + pR];
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
    for (int l = 0; l < G.nspec; ++l) { wl[RD_X0 + l] = ql[W_X0 + l]; wr[RD_X0 + l] = qr[W_X0 + l]; }
    const Bg bf = (D == 2) ? bg_zface(G, c[2]) : bg_cell(G, c[2]);
    if (!(bf.rho + wl[RD_RHO] > 0.0 && bf.rho + wr[RD_RHO] > 0.0 && bf.p + wl[RD_P] > 0.0 &&
          bf.p + wr[RD_P] > 0.0))
      atomicOr(dflag, FLAG_NEG);
    // normal field on this face; transverse ghost rows map to their source rows
    int s[3];
    s[D] = c[D];
    {
      bool fl;
      s[T1] = G.act[T1] ? cell_src(c[T1], G.n[T1], G.bc[T1][0], G.bc[T1][1], fl) : 0;
      s[T2] = G.act[T2] ? cell_src(c[T2], G.n[T2], G.bc[T2][0], G.bc[T2][1], fl) : 0;
    }
    const double bn = Bf[(long)D * G.plane + sidx(G, s[0], s[1], s[2])];
    const int solver = (flag[pL] | flag[pR]) ? SOLVER_HLL : G.riemann;
    double f[7 + PHL_NSPEC_MAX];
    int up;
    riemann_dev<double>(wl, wr, bn, bf.rho, bf.p, bf.ge, bf.gc, G.nspec, solver, G.mach_thr, f, up);
    // reflecting wall face: a symmetry plane (Table bcs, u_n = 0, B_n = 0); only
    // the normal-momentum flux survives, the others are exactly zero
    if ((c[D] == 0 && G.bc[D][0] == 1) || (c[D] == G.n[D] && G.bc[D][1] == 1)) {
      for (int q = 0; q < 7 + G.nspec; ++q)
        if (q != RF_MN) f[q] = 0.0;
      up = 0;
    }
    const long wt = G.wtot;
    F[F_RHO * wt + pR] = f[RF_RHO];
    F[(F_MX + D) * wt + pR] = f[RF_MN];
    F[(F_MX + T1) * wt + pR] = f[RF_MT1];
    F[(F_MX + T2) * wt + pR] = f[RF_MT2];
    F[F_E * wt + pR] = f[RF_E];
    F[(F_BX + D) * wt + pR] = 0.0;
    F[(F_BX + T1) * wt + pR] = f[RF_BT1];
    F[(F_BX + T2) * wt + pR] = f[RF_BT2];
    for (int l = 0; l < G.nspec; ++l) F[(F_X0 + l) * wt + pR] = f[RF_X0 + l];
    F[(long)G.nf * wt + pR] = (double)up;   // contact direction for Contact-CT
  }
}

// Edge EMF along D at the lower corner (a-1/2, b-1/2), (D, A, B) cyclic.
template <int D>
__global__ void k_emf(DevGeo G, Box box, const double *__restrict__ W, const double *__restrict__ FA,
                      const double *__restrict__ FB, double *__restrict__ E) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    const long p = widx(G, c[0], c[1], c[2]);
    const long wt = G.wtot;
    double e;
    if (G.act[A] && G.act[B]) {
      const long sa = wstride(G, A), sb = wstride(G, B);
      const double *fab = FA + (F_BX + B) * wt;   // F_a(B_b) on a-faces
      const double *fba = FB + (F_BX + A) * wt;   // F_b(B_a) on b-faces
      const double Ea1 = -fab[p], Ea0 = -fab[p - sb];
      const double Eb1 = fba[p], Eb0 = fba[p - sa];
      // contact directions stored after the nf flux components
      const double *ua = FA + (long)G.nf * wt, *ub = FB + (long)G.nf * wt;
      const double ma1 = ua[p], ma0 = ua[p - sb];
      const double mb1 = ub[p], mb0 = ub[p - sa];
      const double *va = W + (W_VX + A) * wt, *vb = W + (W_VX + B) * wt;
      const double *ba = W + (W_BX + A) * wt, *bb = W + (W_BX + B) * wt;
      auto ec = [&](long q) { return -(va[q] * bb[q] - vb[q] * ba[q]); };
      const double E00 = ec(p - sa - sb), E10 = ec(p - sb), E01 = ec(p - sa), E11 = ec(p);
      const double lo_l = Eb0 - E00, lo_r = Eb1 - E10;
      const double up_l = E01 - Eb0, up_r = E11 - Eb1;
      const double dlo = ma0 > 0.0 ? lo_l : (ma0 < 0.0 ? lo_r : 0.5 * (lo_l + lo_r));
      const double dup = ma1 > 0.0 ? up_l : (ma1 < 0.0 ? up_r : 0.5 * (up_l + up_r));
      const double le_d = Ea0 - E00, le_u = Ea1 - E01;
      const double ri_d = E10 - Ea0, ri_u = E11 - Ea1;
      const double dle = mb0 > 0.0 ? le_d : (mb0 < 0.0 ? le_u : 0.5 * (le_d + le_u));
      const double dri = mb1 > 0.0 ? ri_d : (mb1 < 0.0 ? ri_u : 0.5 * (ri_d + ri_u));
      e = 0.25 * (Ea1 + Ea0 + Eb1 + Eb0) + 0.25 * (dlo - dup) + 0.25 * (dle - dri);
    } else if (G.act[A]) {
      e = -FA[(F_BX + B) * wt + p];
    } else {
      e = FB[(F_BX + A) * wt + p];
    }
    // edge on a reflecting wall: u_n = B_n = 0 there (Table bcs), so the
    // tangential EMF -(u x B)_t is zero
    if ((G.act[A] && ((c[A] == 0 && G.bc[A][0] == 1) || (c[A] == G.n[A] && G.bc[A][1] == 1))) ||
        (G.act[B] && ((c[B] == 0 && G.bc[B][0] == 1) || (c[B] == G.n[B] && G.bc[B][1] == 1))))
      e = 0.0;
    E[(long)D * wt + p] = e;
  }
}

__global__ void k_update_cells(DevGeo G, Box box, StageBufs S) {
  const double dt = *S.dt;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    const long p = widx(G, c[0], c[1], c[2]);
    const long ps = sidx(G, c[0], c[1], c[2]);
    const long wt = G.wtot, pl = G.plane;
    double r[5 + PHL_NSPEC_MAX];
    for (int v = 0; v < G.nv; ++v) {
      const int fc = v < 5 ? v : F_X0 + (v - U_X0);
      double s = 0.0;
      for (int d = 0; d < 3; ++d) {
        if (!G.act[d]) continue;
        const double *f = S.F[d] + fc * wt;
        s += (f[p + wstride(G, d)] - f[p]) / G.dx[d];
      }
      r[v] = s;
    }
    const double rho = S.Uin[ps];
    const double rhohat = bg_cell(G, c[2]).rho;
    double se = 0.0;
    for (int d = 0; d < 3; ++d) {
      r[U_MX + d] -= (rho - rhohat) * G.g[d];
      se += S.Uin[(U_MX + d) * pl + ps] * G.g[d];
    }
    if (G.heat) se += G.heat[c[2]];
    r[U_E] -= se;
    for (int v = 0; v < G.nv; ++v) {
      const long q = v * pl + ps;
      S.Uout[q] = S.a * S.Ubase[q] + S.b * S.Uin[q] - S.b * dt * r[v];
    }
  }
}

template <int D>
__global__ void k_update_faces(DevGeo G, Box box, StageBufs S) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const double dt = *S.dt;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    int e[3] = {c[0], c[1], c[2]};
    if (!G.act[D]) e[D] = 0;
    const long p = widx(G, e[0], e[1], e[2]);
    const long wt = G.wtot;
    double r = 0.0;
    if (G.act[A]) r += (S.E[(long)B * wt + p + wstride(G, A)] - S.E[(long)B * wt + p]) / G.dx[A];
    if (G.act[B]) r -= (S.E[(long)A * wt + p + wstride(G, B)] - S.E[(long)A * wt + p]) / G.dx[B];
    const long q = (long)D * G.plane + sidx(G, c[0], c[1], c[2]);
    S.Bout[q] = S.a * S.Bbase[q] + S.b * S.Bin[q] - S.b * dt * r;
  }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_dt(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                     unsigned long long *dmax, int *dflag) {
  double m = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    double w[NW_MAX];
    cell_prims(G, U, Bf, c[0], c[1], c[2], w, dflag);
    const Bg b = bg_cell(G, c[2]);
    const double rho = w[W_RHO] + b.rho, P = w[W_P] + b.p, gc = w[W_GC] + b.gc;
    const double a2 = gc * P / rho;
    const double b2 = (w[W_BX] * w[W_BX] + w[W_BY] * w[W_BY] + w[W_BZ] * w[W_BZ]) / rho;
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const double bd2 = w[W_BX + d] * w[W_BX + d] / rho;
      double disc = (a2 + b2) * (a2 + b2) - 4.0 * a2 * bd2;
      if (disc < 0.0) disc = 0.0;
      const double cf = sqrt(0.5 * (a2 + b2 + sqrt(disc)));
      s += (fabs(w[W_VX + d]) + cf) / G.dx[d];
    }
    if (s > m || !(s == s)) m = (s == s) ? s : INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[TPB / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomic_max_pos(dmax, v);
  }
}

__global__ void k_dt_finalize(double cfl, unsigned long long *dmax, double *dt) {
  const double m = __longlong_as_double((long long)*dmax);
  *dt = cfl / m;
  *dmax = 0ull;
}

__global__ void k_set_scalar(double *p, double v) { *p = v; }

}  // namespace

void launch_set_scalar(double *p, double v, cudaStream_t s, Prof *prof) { PHL_LAUNCH(KC_SCALAR, prof, s, k_set_scalar<<<1, 1, 0, s>>>(p, v)); }

void launch_dt_fp64(const DevGeo &G, const double *U, const double *Bf, double *T, unsigned long long *dmax,
                    double *dt, int *dflag, cudaStream_t s, int *nlaunch, Prof *prof) {
  (void)T;
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  PHL_LAUNCH(KC_DT, prof, s, k_dt<<<nblocks(b.n), TPB, 0, s>>>(G, b, U, Bf, dmax, dflag));
  PHL_LAUNCH(KC_DT, prof, s, k_dt_finalize<<<1, 1, 0, s>>>(G.cfl, dmax, dt));
  if (nlaunch) *nlaunch += 2;
}

void launch_stage_fp64(const DevGeo &G, const StageBufs &S, cudaStream_t s, int *nlaunch, Prof *prof) {
  int nl = 0;
  auto rng = [&](int d, int lo_g, int hi_extra, int &lo, int &hi) {
    if (G.act[d]) { lo = -lo_g; hi = G.n[d] + hi_extra; }
    else { lo = 0; hi = 1; }
  };
  // (1) primitives on cells [-2, n+2) of every active dimension
  {
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) rng(d, NGW, NGW, l[d], h[d]);
    Box b = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    PHL_LAUNCH(KC_PRIM, prof, s, k_prim<<<nblocks(b.n), TPB, 0, s>>>(G, b, S.Uin, S.Bin, S.W, S.dflag));
    ++nl;
  }
  // (2) shock flags
  if (G.eps_sf > 0.0) {
    Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_FLAG_RAW, prof, s, k_flag_raw<<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.raw));
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) rng(d, 1, 1, l[d], h[d]);
    Box b2 = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    PHL_LAUNCH(KC_FLAG_DILATE, prof, s, k_flag_dilate<<<nblocks(b2.n), TPB, 0, s>>>(G, b2, S.raw, S.flag));
    nl += 2;
  }
  // (3) fluxes: normal faces [0, n], one transverse ghost row each side
  for (int D = 0; D < 3; ++D) {
    if (!G.act[D]) continue;
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) {
      if (d == D) { l[d] = 0; h[d] = G.n[d] + 1; }
      else rng(d, 1, 1, l[d], h[d]);
    }
    Box b = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    if (D == 0) PHL_LAUNCH(KC_FLUX_X, prof, s, k_flux<0><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.Bin, S.flag, S.F[0], S.dflag));
    if (D == 1) PHL_LAUNCH(KC_FLUX_Y, prof, s, k_flux<1><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.Bin, S.flag, S.F[1], S.dflag));
    if (D == 2) PHL_LAUNCH(KC_FLUX_Z, prof, s, k_flux<2><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.Bin, S.flag, S.F[2], S.dflag));
    ++nl;
  }
  // (4) edge EMFs
  for (int D = 0; D < 3; ++D) {
    const int A = (D + 1) % 3, B = (D + 2) % 3;
    if (!G.act[A] && !G.act[B]) continue;
    int l[3] = {0, 0, 0}, h[3];
    h[D] = G.n[D];
    h[A] = G.act[A] ? G.n[A] + 1 : 1;
    h[B] = G.act[B] ? G.n[B] + 1 : 1;
    Box b = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    if (D == 0) PHL_LAUNCH(KC_EMF, prof, s, k_emf<0><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.F[1], S.F[2], S.E));
    if (D == 1) PHL_LAUNCH(KC_EMF, prof, s, k_emf<1><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.F[2], S.F[0], S.E));
    if (D == 2) PHL_LAUNCH(KC_EMF, prof, s, k_emf<2><<<nblocks(b.n), TPB, 0, s>>>(G, b, S.W, S.F[0], S.F[1], S.E));
    ++nl;
  }
  // (5) updates
  {
    Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_UPDATE_CELLS, prof, s, k_update_cells<<<nblocks(b.n), TPB, 0, s>>>(G, b, S));
    ++nl;
  }
  for (int D = 0; D < 3; ++D) {
    // every face array is written: a field with no active curl direction still
    // takes the RK combination a * base + b * in
    int h[3] = {G.n[0], G.n[1], G.n[2]};
    h[D] += 1;
    Box b = make_box(0, h[0], 0, h[1], 0, h[2]);
    if (D == 0) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<0><<<nblocks(b.n), TPB, 0, s>>>(G, b, S));
    if (D == 1) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<1><<<nblocks(b.n), TPB, 0, s>>>(G, b, S));
    if (D == 2) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<2><<<nblocks(b.n), TPB, 0, s>>>(G, b, S));
    ++nl;
  }
  if (nlaunch) *nlaunch += nl;
}

}  // namespace phl
