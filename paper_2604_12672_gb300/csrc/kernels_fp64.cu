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
#include "stage_common.cuh"

namespace phl {
using namespace stage;
namespace {

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
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) w[W_X0 + l] = U[(U_X0 + l) * pl + p] / rho;
  bool ok = true;
  if (!(rho > 0.0) || !(P > 0.0)) { atomicOr(dflag, FLAG_NEG); ok = false; }
  if (!isfinite(P) || !isfinite(rho)) { atomicOr(dflag, FLAG_NAN); ok = false; }
  return ok;
}

__global__ void k_prim(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                       double *__restrict__ W, int *dflag) {
  {
    int c[3], s[3];
    bool fl[3];
    if (!cell3(box, c)) return;
    for (int d = 0; d < 3; ++d) {
      fl[d] = false;
      s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]) : 0;
    }
    double w[NW_MAX];
    cell_prims(G, U, Bf, s[0], s[1], s[2], w, dflag);
    for (int d = 0; d < 3; ++d)
      if (fl[d]) { w[W_VX + d] = -w[W_VX + d]; w[W_BX + d] = -w[W_BX + d]; }
    const long q = widx(G, c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < NW_MAX; ++v)
      if (v < G.nw) W[v * G.wtot + q] = w[v];
  }
}

__global__ void k_update_cells(DevGeo G, Box box, StageBufs S) {
  const double dt = *S.dt;
  {
    int c[3];
    if (!cell3(box, c)) return;
    const long p = widx(G, c[0], c[1], c[2]);
    const long ps = sidx(G, c[0], c[1], c[2]);
    const long wt = G.wtot, pl = G.plane;
    double r[5 + PHL_NSPEC_MAX];
#pragma unroll
    for (int v = 0; v < 5 + PHL_NSPEC_MAX; ++v) {
      if (v >= G.nv) continue;
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
#pragma unroll
    for (int v = 0; v < 5 + PHL_NSPEC_MAX; ++v) {
      if (v >= G.nv) continue;
      const long q = v * pl + ps;
      S.Uout[q] = S.a * S.Ubase[q] + S.b * S.Uin[q] - S.b * dt * r[v];
    }
  }
}

template <int D>
__global__ void k_update_faces(DevGeo G, Box box, StageBufs S) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const double dt = *S.dt;
  {
    int c[3];
    if (!cell3(box, c)) return;
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
  // (1) primitives on cells [-ge, n+ge) of every active dimension (ge: the work layout's ghost layers)
  {
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) rng(d, G.ge[d], G.ge[d], l[d], h[d]);
    Box b = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    if (G.eos == 1) {
      launch_eos_cells<double>(G, S.Uin, S.Bin, nullptr, nullptr, S.Tin, S.Tout, S.W, S.dflag, s, &nl, prof,
                               S.cfl_dmax, const_cast<double *>(S.dt));
    } else {
      PHL_LAUNCH(KC_PRIM, prof, s, k_prim<<<grid3(b), block3(b), 0, s>>>(G, b, S.Uin, S.Bin, S.W, S.dflag));
      ++nl;
    }
  }
  // (2) shock flags
  if (G.eps_sf > 0.0) {
    Box bx = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_FLAG_RAW, prof, s, k_flag_raw<double><<<grid3(bx), block3(bx), 0, s>>>(G, bx, S.W, S.raw));
    nl += 1 + launch_flags(G, S.raw, S.raw + (long)G.n[0] * G.n[1] * G.n[2], S.flag, s, prof);
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
    launch_flux<double>(D, G, b, S.W, S.Bin, (const double *)nullptr, S.flag, S.F[D], S.dflag, s, prof);
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
    if (D == 0) PHL_LAUNCH(KC_EMF, prof, s, k_emf<0, double><<<grid3(b), block3(b), 0, s>>>(G, b, S.W, S.F[1], S.F[2], S.E));
    if (D == 1) PHL_LAUNCH(KC_EMF, prof, s, k_emf<1, double><<<grid3(b), block3(b), 0, s>>>(G, b, S.W, S.F[2], S.F[0], S.E));
    if (D == 2) PHL_LAUNCH(KC_EMF, prof, s, k_emf<2, double><<<grid3(b), block3(b), 0, s>>>(G, b, S.W, S.F[0], S.F[1], S.E));
    ++nl;
  }
  // (5) updates
  {
    Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_UPDATE_CELLS, prof, s, k_update_cells<<<grid3(b), block3(b), 0, s>>>(G, b, S));
    ++nl;
  }
  for (int D = 0; D < 3; ++D) {
    // every face array is written: a field with no active curl direction still
    // takes the RK combination a * base + b * in
    int h[3] = {G.n[0], G.n[1], G.n[2]};
    h[D] += 1;
    Box b = make_box(0, h[0], 0, h[1], 0, h[2]);
    if (D == 0) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<0><<<grid3(b), block3(b), 0, s>>>(G, b, S));
    if (D == 1) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<1><<<grid3(b), block3(b), 0, s>>>(G, b, S));
    if (D == 2) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces<2><<<grid3(b), block3(b), 0, s>>>(G, b, S));
    ++nl;
  }
  if (nlaunch) *nlaunch += nl;
}

}  // namespace phl
