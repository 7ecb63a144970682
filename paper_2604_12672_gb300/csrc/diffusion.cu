// diffusion.cu -- thermal diffusion by RKL2 super-time-stepping (Sect. 2.10)
// on the device, behind phl_diffuse.
//
// With the density, velocity, magnetic field and mass fractions held fixed,
// rho d(e_int)/dt = div(K grad T) is advanced over a whole step dt by the
// RKL2 stages of Meyer, Balsara & Aslam (2012) in the paper's form (Sect.
// 2.10, items i-iv), with the paper's stage count from the parabolic limit at
// the start of the step.  Ideal gas: T = e_int / c_v; conductivity
// K = k0 T^nT / rho^nR.  Space: conservative seven-point operator, face flux
// -K_f (T_R - T_L) / dx with K_f the harmonic mean 2 K_L K_R / (K_L + K_R) of
// the two cells' K (Sect. 2.10); a side that is not periodic carries no flux.
//
// Two forms.  FP64: the stages evolve e_int itself in double.  Mixed: the
// stages evolve the change d = (e_int - e_int^(0)) / 2^eY in float, where
// e_int^(0) enters only through its face differences (taken in FP64, then
// rounded) and, for K, as a float; since e_int^(m) = e_int^(0) + d^(m) 2^eY
// the paper's stage formula becomes
//   d^(m) = mu_m d^(m-1) + nu_m d^(m-2) + mu~_m dt M[.] + gamma~_m dt M[0]
// (the (1 - mu - nu) e_int^(0) term cancels).  With delta_T the operator acts
// on T - T_hat (Sect. 2.10's option): the FP64 form subtracts T_hat's step on
// z faces, the mixed form folds it into the face differences of e_int^(0).
// Power-of-two scales (eY for
// e_int, eK for K, ea for 1/(rho c_v), ew for 1/dx^2, from maxima reduced at
// the start) keep every float O(1); the stage factors absorb them.  The
// stage kernel then moves 40 bytes per cell and does no FP64 arithmetic.
//
// Layout: the grid's own diffusion arrays, dense over the interior cells (x
// fastest), 7 doubles per cell, then 8 words for the reductions, one double
// per z layer (the background temperature of the delta_T option), and 4
// doubles per cell for the FP64 form's K and face fluxes.  FP64:
// 1/rho, k0/rho^nR, e_int^(0), the operator at e_int^(0), three stage
// buffers.  Mixed: e_int^(0) in double (set-up only), then as floats
// y0 = e_int^(0)/2^eY, the scaled conductivity factor, 1/(rho c_v), the
// operator at d = 0, the three upper-face differences of y0 and three stage
// buffers.
#include <math.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "phl_internal.cuh"
#include "stage_common.cuh"

namespace phl {
using namespace stage;
namespace {

constexpr int NRED = 4;   // reductions: parabolic rate, max e_int, max k0/rho^nR, max 1/rho

struct DiffArrays {       // FP64 form
  double *irho, *krho, *Y0, *L0, *Y[3];
  const double *That;     // background temperature per z layer (null: the full temperature)
};

struct DiffMx {           // mixed form
  double *Y0d;            // e_int^(0) (set-up only)
  float *y0, *kp, *a, *l0, *g[3], *d[3];
  const double *That;
};

// the background temperature P_hat / ((gamma - 1) rho_hat c_v) of each z layer
__global__ void k_diff_that(DevGeo G, double cv, double *That) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G.n[2]; k += gridDim.x * blockDim.x)
    That[k] = G.bg_p_c[k + BG_NG] / ((G.gamma - 1.0) * G.bg_rho_c[k + BG_NG] * cv);
}

struct Stencil {          // interior cells, dense, x fastest
  int n[3], act[3], per[3];
  long st[3];
  float w[3];             // 2 / dx^2 * 2^-ew
};

template <class T>
__device__ __forceinline__ T powi_dev(T x, int n) {
  T r = T(1);
  for (int q = 0; q < n; ++q) r *= x;
  return r;
}

__device__ __forceinline__ long dense(const DevGeo &G, const int *c) {
  return c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);
}

// Block maximum of a non-negative double into *dst.  Non-negative doubles
// order as their bit patterns, so the reduction runs on the integer pipe
// (GB300's FP64 pipe is 1/64 of the FP32 rate); a negative input counts as
// zero (a NaN wins, and the host then treats the maximum as absent).
__device__ __forceinline__ unsigned long long dbits(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0 ? (unsigned long long)b : 0ull;
}
__device__ __forceinline__ void block_max(unsigned long long v, unsigned long long *dst, unsigned long long *red) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, w, o);
      w = u > w ? u : w;
    }
    if (threadIdx.x == 0) atomicMax(dst, w);
  }
  __syncthreads();
}

// e_int^(0), 1/rho and k0/rho^nR of every interior cell; block maxima of
// the parabolic rate sum_s D / dx_s^2 (D = K / (rho c_v)), of e_int, of
// k0/rho^nR and of 1/rho into red[0..3].  FP64.
template <bool MX>
__global__ void k_diff_init(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                            phl_diffusion p, double icv, DiffArrays A, DiffMx M, unsigned long long *red,
                            int *dflag) {
  unsigned long long rate = 0, emax = 0, kmax = 0, imax = 0;
  int c[3];
  if (cell3(box, c)) {
    const long ps = sidx(G, c[0], c[1], c[2]);
    const long q = dense(G, c);
    const long pl = G.plane;
    const double r = U[ps];
    const double ir = 1.0 / r;
    const double mx = U[pl + ps], my = U[2 * pl + ps], mz = U[3 * pl + ps];
    const double bx = 0.5 * (Bf[ps] + Bf[ps + 1]);
    const double by = 0.5 * (Bf[pl + ps] + Bf[pl + ps + G.sy]);
    const double bz = 0.5 * (Bf[2 * pl + ps] + Bf[2 * pl + ps + G.sz]);
    const double e = (U[4 * pl + ps] - 0.5 * ((mx * mx + my * my + mz * mz) * ir + (bx * bx + by * by + bz * bz))) * ir;
    if (!(r > 0.0) || !(e > 0.0)) atomicOr(dflag, FLAG_NEG);
    const double kr = p.k0 * powi_dev(ir, p.nR);
    if (MX) {   // kp and a as raw floats, rescaled once the maxima are known
      M.Y0d[q] = e;
      M.kp[q] = d2f_scaled(kr, 0);
      M.a[q] = d2f_scaled(ir * icv, 0);
    } else {
      A.irho[q] = ir;
      A.krho[q] = kr;
      A.Y0[q] = e;
    }
    const double D = kr * powi_dev(e * icv, p.nT) * ir * icv;
    double s2 = 0.0;
    for (int d = 0; d < 3; ++d)
      if (G.act[d]) s2 += G.idx[d] * G.idx[d];
    rate = dbits(D * s2);
    emax = dbits(e);
    kmax = dbits(kr);
    imax = dbits(ir);
  }
  __shared__ unsigned long long red_s[TPB / 32];
  block_max(rate, red + 0, red_s);
  if (MX) {
    block_max(emax, red + 1, red_s);
    block_max(kmax, red + 2, red_s);
    block_max(imax, red + 3, red_s);
  }
}

// ---------------------------------------------------------------- FP64 form

__device__ __forceinline__ double hmean(double a, double b) {
  const double s = a + b;
  return s > 0.0 ? 2.0 * a * b / s : 0.0;
}

// The FP64 operator in three passes per stage, so that each cell's K and
// each face's harmonic mean (an FP64 division) are evaluated once: the FP64
// pipe (1/64 of the FP32 rate on GB300) bounds this form.
//   k_diff_k:     K = k0/rho^nR (Y / c_v)^nT of every cell
//   k_diff_faces: F_d = hm(K_c, K_up) (T_up - T_c [- the background step]) / dx_d
//                 at the upper d-face of every cell (zero on a non-periodic side)
//   k_diff_comb:  L = sum_d (F_d(upper) - F_d(lower)) / dx_d / rho, then the
//                 RKL2 stage combination
__global__ void k_diff_k(DevGeo G, Box box, phl_diffusion p, double icv, DiffArrays A, const double *__restrict__ Y,
                         double *__restrict__ K) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  K[q] = A.krho[q] * powi_dev(Y[q] * icv, p.nT);
}

__global__ void k_diff_faces(DevGeo G, Box box, double icv, DiffArrays A, const double *__restrict__ Y,
                             const double *__restrict__ K, double *__restrict__ F0, double *__restrict__ F1,
                             double *__restrict__ F2) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  const long st[3] = {1L, (long)G.n[0], (long)G.n[0] * G.n[1]};
  double *F[3] = {F0, F1, F2};
  const double Tc = Y[q] * icv, Kc = K[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!G.act[d]) continue;
    int x = c[d] + 1;
    double f = 0.0;   // no flux through a wall or an outflow side
    if (x < G.n[d] || G.bc[d][0] == PHL_PERIODIC) {
      if (x == G.n[d]) x = 0;
      const long qn = q + (long)(x - c[d]) * st[d];
      double dT = Y[qn] * icv - Tc;
      if (d == 2 && A.That) dT -= A.That[x] - A.That[c[2]];   // the deviation from the background
      f = hmean(Kc, K[qn]) * (dT * G.idx[d]);
    }
    F[d][q] = f;
  }
}

// FIRST: L0 = the operator at e_int^(0) (stored), Y1 = Y0 + mu~_1 dt L0;
// else Y_j = mu Y_{j-1} + nu Y_{j-2} + (1 - mu - nu) Y0 + mu~ dt L(Y_{j-1}) + gamma~ dt L0
template <bool FIRST>
__global__ void k_diff_comb(DevGeo G, Box box, DiffArrays A, const double *__restrict__ F0,
                            const double *__restrict__ F1, const double *__restrict__ F2, double mu, double nu,
                            double mdt, double gdt, const double *__restrict__ Ym1, const double *__restrict__ Ym2,
                            double *__restrict__ Yj) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  const long st[3] = {1L, (long)G.n[0], (long)G.n[0] * G.n[1]};
  const double *F[3] = {F0, F1, F2};
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!G.act[d]) continue;
    double low = 0.0;   // the lower face's flux (zero on a non-periodic side)
    if (c[d] > 0) low = F[d][q - st[d]];
    else if (G.bc[d][0] == PHL_PERIODIC) low = F[d][q + (long)(G.n[d] - 1) * st[d]];
    s += (-low + F[d][q]) * G.idx[d];
  }
  const double L = s * A.irho[q];
  if (FIRST) {
    A.L0[q] = L;
    Yj[q] = A.Y0[q] + mdt * L;
  } else {
    Yj[q] = mu * Ym1[q] + nu * Ym2[q] + (1.0 - mu - nu) * A.Y0[q] + mdt * L + gdt * A.L0[q];
  }
}

// E += rho (e_int^(N) - e_int^(0))
__global__ void k_diff_finish(DevGeo G, Box box, DiffArrays A, const double *__restrict__ YN, double *__restrict__ U) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  const long ps = sidx(G, c[0], c[1], c[2]);
  U[4 * G.plane + ps] += U[ps] * (YN[q] - A.Y0[q]);
}

// --------------------------------------------------------------- mixed form

// The per-cell floats of the mixed form: y0 = e_int^(0) 2^-eY,
// kp = k0/rho^nR (2^eY / c_v)^nT 2^-eK (so K = 2^eK kp y^nT), a = 1/(rho c_v)
// 2^-ea, and the upper-face differences of y0 (FP64 difference, then
// rounded; zero on a non-periodic upper side, where no flux passes).
__global__ void k_dmx_prep(DevGeo G, Box box, Stencil S, DiffMx M, double kt, int eK, int eY, float asc,
                           double cv) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  const double Y = M.Y0d[q];
  float gd[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!S.act[d]) continue;
    int up = -1;
    if (c[d] + 1 < S.n[d]) up = c[d] + 1;
    else if (S.per[d]) up = 0;
    if (up < 0) continue;
    double dY = M.Y0d[q + (long)(up - c[d]) * S.st[d]] - Y;
    // diffusing the deviation from the background: its (fixed) step moves into g
    if (d == 2 && M.That) dY -= cv * (M.That[up] - M.That[c[2]]);
    gd[d] = d2f_scaled(dY, -eY);
  }
  M.y0[q] = d2f_scaled(Y, -eY);
  M.kp[q] = d2f_scaled((double)M.kp[q] * kt, -eK);
  M.a[q] *= asc;
  for (int d = 0; d < 3; ++d)
    if (S.act[d]) M.g[d][q] = gd[d];
}

// Half the harmonic mean of the two cells' conductivity factors.
__device__ __forceinline__ float hmean_f(float a, float b) {
  const float s = a + b;
  return s > 0.0f ? __fdividef(a * b, s) : 0.0f;
}

template <int NT>
__device__ __forceinline__ float pw(float y) {
  float r = 1.0f;
#pragma unroll
  for (int q = 0; q < NT; ++q) r *= y;
  return r;
}

constexpr int DTX = 32, DTY = 8;                  // xy tile of the stage kernel
constexpr int DHALO = 2 * DTX + 2 * DTY;          // its x and y halo cells
constexpr int DTZ_DEFAULT = 16;                   // planes per CTA

// Raw slot data of one cell as loaded: d^(m-1), y0, kp (src = NOSRC: a
// cell outside the domain on a non-periodic side, all zero).
struct Raw {
  float d, y, k;
};
constexpr unsigned NOSRC = 0xffffffffu;

template <bool FIRST>
__device__ __forceinline__ Raw raw_load(const DiffMx &M, const float *__restrict__ dm1, unsigned i) {
  Raw r{0.0f, 0.0f, 0.0f};
  if (i == NOSRC) return r;
  if (!FIRST) r.d = __ldg(dm1 + i);
  r.y = __ldg(M.y0 + i);
  r.k = __ldg(M.kp + i);
  return r;
}

template <int NT>
__device__ __forceinline__ float kval(const Raw &r) { return r.k * pw<NT>(r.y + r.d); }

// Per-plane inputs besides the own slot: the halo slot, the own upper-face
// differences, g of the cells below the tile's lower boundary faces, and
// 1/(rho c_v), the operator at d = 0 and d^(m-2) of the own cell.
struct Aux {
  Raw h;
  float gx, gy, gz, glx, gly, a, l0, d2;
};

__device__ __forceinline__ int wrap_or_out(int x, int n, int per) {
  if (x >= 0 && x < n) return x;
  if (!per) return -1;
  return ((x % n) + n) % n;
}

// One stage of the mixed form.  A CTA owns a 32 x 8 column of cells and
// marches up tz planes of it.  Per plane, (d, k) of the tile and its x/y
// halo go to shared memory (two buffers by plane parity, so one barrier per
// plane suffices); each cell forms its faces' quantities
//   G = hm(k_L, k_R) (g_L + d_R - d_L)     (hm: half the harmonic mean)
// -- a lower face with the same operands in the same order as the
// neighbour's upper face, so both see the same value (z faces in registers,
// the lower one carried from the plane below), and takes
//   lambda = a sum_d w_d (G_upper - G_lower).
// A face on a non-periodic side is zero.  The loads are software-pipelined:
// the own slot two planes ahead, everything else one plane ahead, so the
// plane's barrier does not wait on memory.  Indices are 32-bit (the
// caller checks the cell count).  FIRST: d^(m-1) = 0, lambda is the operator
// at e_int^(0) (stored in l0) and d^(1) = mt lambda; else
// d^(m) = mu d^(m-1) + nu d^(m-2) + mt lambda + gt l0.
template <int NT, bool FIRST>
__global__ void __launch_bounds__(DTX * DTY) k_dmx_stage(Stencil S, DiffMx M, float mu, float nu, float mt, float gt,
                                                        const float *__restrict__ dm1, const float *__restrict__ dm2,
                                                        float *__restrict__ dj, int tz) {
  __shared__ float sdb[2][DTY + 2][DTX + 2], skb[2][DTY + 2][DTX + 2];   // double-buffered by plane parity
  const int tx = threadIdx.x % DTX, ty = threadIdx.x / DTX;
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int x0 = blockIdx.x * DTX, y0 = blockIdx.y * DTY, z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, nz);
  const unsigned pl = (unsigned)S.st[2];
  const int gx = x0 + tx, gy = y0 + ty;
  const bool own = gx < nx && gy < ny;
  // own slot's source cell within a plane (wrapped), or NOSRC
  unsigned osrc = NOSRC;
  {
    const int sx = wrap_or_out(gx, nx, S.per[0]), sy = wrap_or_out(gy, ny, S.per[1]);
    if (sx >= 0 && sy >= 0) osrc = (unsigned)(sx + nx * sy);
  }
  // this thread's halo slot (threadIdx.x < DHALO): position and source
  int hr = 0, hc = 0;
  unsigned hsrc = NOSRC;
  if (threadIdx.x < DHALO) {
    const int h = threadIdx.x;
    if (h < DTY) { hc = 0; hr = h + 1; }
    else if (h < 2 * DTY) { hc = DTX + 1; hr = h - DTY + 1; }
    else if (h < 2 * DTY + DTX) { hr = 0; hc = h - 2 * DTY + 1; }
    else { hr = DTY + 1; hc = h - 2 * DTY - DTX + 1; }
    const int sx = wrap_or_out(x0 + hc - 1, nx, S.per[0]), sy = wrap_or_out(y0 + hr - 1, ny, S.per[1]);
    if (sx >= 0 && sy >= 0 && S.act[(hr == 0 || hr == DTY + 1) ? 1 : 0]) hsrc = (unsigned)(sx + nx * sy);
  }
  // in-plane cells below the tile's lower boundary faces (their g), or NOSRC
  unsigned lxsrc = NOSRC, lysrc = NOSRC;
  if (own && S.act[0]) {
    const int lx = wrap_or_out(gx - 1, nx, S.per[0]);
    if (lx >= 0) lxsrc = (unsigned)(lx + nx * gy);
  }
  if (own && S.act[1]) {
    const int ly = wrap_or_out(gy - 1, ny, S.per[1]);
    if (ly >= 0) lysrc = (unsigned)(gx + nx * ly);
  }
  const bool hasz = S.act[2] != 0;

  auto aux_load = [&](int z) {
    Aux X{};
    const unsigned base = (unsigned)z * pl;
    if (threadIdx.x < DHALO && hsrc != NOSRC) X.h = raw_load<FIRST>(M, dm1, base + hsrc);
    if (own) {
      const unsigned q = base + osrc;
      if (S.act[0]) X.gx = __ldg(M.g[0] + q);
      if (S.act[1]) X.gy = __ldg(M.g[1] + q);
      if (hasz) X.gz = __ldg(M.g[2] + q);
      X.a = __ldg(M.a + q);
      if (!FIRST) {
        X.l0 = __ldg(M.l0 + q);
        X.d2 = __ldg(dm2 + q);
      }
    }
    if (lxsrc != NOSRC) X.glx = __ldg(M.g[0] + base + lxsrc);
    if (lysrc != NOSRC) X.gly = __ldg(M.g[1] + base + lysrc);
    return X;
  };
  auto own_load = [&](int z) {   // own slot of plane z (wrapped), zeros outside
    const int zz = hasz ? wrap_or_out(z, nz, S.per[2]) : (z == 0 ? 0 : -1);
    return (zz >= 0 && osrc != NOSRC) ? raw_load<FIRST>(M, dm1, (unsigned)zz * pl + osrc) : Raw{0.0f, 0.0f, 0.0f};
  };

  Raw oc = own_load(z0), on = own_load(z0 + 1);
  Aux ac = aux_load(z0);
  float gzl = 0.0f;   // G of the z face below the current plane
  if (hasz && own) {
    const int pz = wrap_or_out(z0 - 1, nz, S.per[2]);
    if (pz >= 0) {
      const Raw pr = raw_load<FIRST>(M, dm1, (unsigned)pz * pl + osrc);
      gzl = hmean_f(kval<NT>(pr), kval<NT>(oc)) * (__ldg(M.g[2] + (unsigned)pz * pl + osrc) + (oc.d - pr.d));
    }
  }
  for (int z = z0; z < z1; ++z) {
    Raw onn = on;
    Aux an = ac;
    if (z + 1 < z1) {
      onn = own_load(z + 2);
      an = aux_load(z + 1);
    }
    const float cd = oc.d, ck = kval<NT>(oc);
    float(*sd)[DTX + 2] = sdb[z & 1];
    float(*sk)[DTX + 2] = skb[z & 1];
    sd[ty + 1][tx + 1] = cd;
    sk[ty + 1][tx + 1] = ck;
    if (threadIdx.x < DHALO) {
      sd[hr][hc] = ac.h.d;
      sk[hr][hc] = kval<NT>(ac.h);
    }
    // one barrier per plane: the slots alternate between two buffers, and a
    // thread two planes ahead has passed the barrier every reader reached
    __syncthreads();
    if (own) {
      float s = 0.0f;
      if (S.act[0]) {   // each cell forms both its faces (the lower one as its neighbour does)
        const float up = (gx + 1 < nx || S.per[0])
                             ? hmean_f(ck, sk[ty + 1][tx + 2]) * (ac.gx + (sd[ty + 1][tx + 2] - cd)) : 0.0f;
        const float lo = lxsrc != NOSRC ? hmean_f(sk[ty + 1][tx], ck) * (ac.glx + (cd - sd[ty + 1][tx])) : 0.0f;
        s += S.w[0] * (up - lo);
      }
      if (S.act[1]) {
        const float up = (gy + 1 < ny || S.per[1])
                             ? hmean_f(ck, sk[ty + 2][tx + 1]) * (ac.gy + (sd[ty + 2][tx + 1] - cd)) : 0.0f;
        const float lo = lysrc != NOSRC ? hmean_f(sk[ty][tx + 1], ck) * (ac.gly + (cd - sd[ty][tx + 1])) : 0.0f;
        s += S.w[1] * (up - lo);
      }
      if (hasz) {
        const bool up = z + 1 < nz || S.per[2];
        const float gzu = up ? hmean_f(ck, kval<NT>(on)) * (ac.gz + (on.d - cd)) : 0.0f;
        s += S.w[2] * (gzu - gzl);
        gzl = gzu;
      }
      const float lam = ac.a * s;
      const unsigned q = (unsigned)z * pl + osrc;
      if (FIRST) {
        M.l0[q] = lam;
        dj[q] = mt * lam;
      } else {
        dj[q] = mu * cd + nu * ac.d2 + mt * lam + gt * ac.l0;
      }
    }
    oc = on;
    on = onn;
    ac = an;
  }
}

template <bool FIRST>
void launch_dmx_stage(int nT, dim3 grd, int tz, cudaStream_t s, const Stencil &S, const DiffMx &M, float mu,
                      float nu, float mt, float gt, const float *dm1, const float *dm2, float *dj) {
  const dim3 blk(DTX * DTY);
  switch (nT) {
    case 0: k_dmx_stage<0, FIRST><<<grd, blk, 0, s>>>(S, M, mu, nu, mt, gt, dm1, dm2, dj, tz); break;
    case 1: k_dmx_stage<1, FIRST><<<grd, blk, 0, s>>>(S, M, mu, nu, mt, gt, dm1, dm2, dj, tz); break;
    case 2: k_dmx_stage<2, FIRST><<<grd, blk, 0, s>>>(S, M, mu, nu, mt, gt, dm1, dm2, dj, tz); break;
    case 3: k_dmx_stage<3, FIRST><<<grd, blk, 0, s>>>(S, M, mu, nu, mt, gt, dm1, dm2, dj, tz); break;
    default: k_dmx_stage<4, FIRST><<<grd, blk, 0, s>>>(S, M, mu, nu, mt, gt, dm1, dm2, dj, tz); break;
  }
}

// E += rho 2^eY d^(N)
__global__ void k_dmx_finish(DevGeo G, Box box, const float *__restrict__ dN, int eY, double *__restrict__ U) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = dense(G, c);
  const long ps = sidx(G, c[0], c[1], c[2]);
  U[4 * G.plane + ps] += U[ps] * f2d_scaled(dN[q], eY);
}

int exp_above(double v) {   // e with v < 2^e (v > 0), 0 otherwise
  if (!(v > 0.0) || !std::isfinite(v)) return 0;
  int e = 0;
  std::frexp(v, &e);
  return e;
}

}  // namespace

// RKL2 coefficients (Meyer, Balsara & Aslam 2012) for s stages, j = 1..s.
void rkl2_coeffs(int s, double *mu, double *nu, double *mut, double *gat) {
  std::vector<double> b((size_t)s + 1);
  for (int j = 0; j <= s; ++j) b[j] = j <= 2 ? 1.0 / 3.0 : (double)(j * j + j - 2) / (2.0 * j * (j + 1));
  const double w1 = 4.0 / (double)(s * s + s - 2);
  for (int j = 0; j <= s; ++j) { mu[j] = nu[j] = mut[j] = gat[j] = 0.0; }
  mut[1] = b[1] * w1;
  for (int j = 2; j <= s; ++j) {
    mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1];
    nu[j] = -(j - 1.0) / j * b[j] / b[j - 2];
    mut[j] = mu[j] * w1;
    gat[j] = -(1.0 - b[j - 1]) * mut[j];
  }
}

int sts_stage_count(double dt, double dt_p) {
  const double f = 1.0 + std::floor(0.5 * (std::sqrt(9.0 + 16.0 * dt / dt_p) - 1.0));
  if (!(f < 1e9)) return 1000000000;   // beyond any stage limit
  const int n = (int)f;
  return n < 3 ? 3 : n;
}

cudaError_t launch_diffuse(const DevGeo &G, double *U, const double *Bf, const phl_diffusion &p, double dt,
                           int max_stages, bool mixed, double *scratch, int *dflag, cudaStream_t s, int *nsts,
                           int *nlaunch) {
  const long nc = (long)G.n[0] * G.n[1] * G.n[2];
  unsigned long long *red = (unsigned long long *)(scratch + 7 * nc);
  DiffArrays A{};
  DiffMx M{};
  A.That = nullptr;
  M.That = nullptr;
  if (mixed) {   // e_int^(0) in double, then ten float arrays: 6 doubles per cell
    M.Y0d = scratch;
    float *f = (float *)(scratch + nc);
    M.y0 = f;
    M.kp = f + nc;
    M.a = f + 2 * nc;
    M.l0 = f + 3 * nc;
    for (int k = 0; k < 3; ++k) M.g[k] = f + (4 + k) * nc;
    for (int k = 0; k < 3; ++k) M.d[k] = f + (7 + k) * nc;
  } else {
    A.irho = scratch;
    A.krho = scratch + nc;
    A.Y0 = scratch + 2 * nc;
    A.L0 = scratch + 3 * nc;
    for (int k = 0; k < 3; ++k) A.Y[k] = scratch + (4 + k) * nc;
  }
  const double icv = 1.0 / p.cv;
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  cudaError_t e = cudaMemsetAsync(red, 0, NRED * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (p.delta_T) {   // the background temperature per layer, after the reduction words
    double *That = scratch + 7 * nc + 8;
    k_diff_that<<<(G.n[2] + 255) / 256, 256, 0, s>>>(G, p.cv, That);
    A.That = That;
    M.That = That;
  }
  if (mixed)
    k_diff_init<true><<<grid3(b), block3(b), 0, s>>>(G, b, U, Bf, p, icv, A, M, red, dflag);
  else
    k_diff_init<false><<<grid3(b), block3(b), 0, s>>>(G, b, U, Bf, p, icv, A, M, red, dflag);
  unsigned long long bits[NRED] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(bits, red, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  double mx[NRED];
  memcpy(mx, bits, sizeof(mx));
  const double rate = mx[0];
  // a NaN maximum comes with a flagged cell (reported at the next check); an
  // infinite parabolic rate needs more stages than any limit
  const int ns = !(rate > 0.0) ? 3 : std::isfinite(rate * dt) ? sts_stage_count(dt, 0.5 / rate) : max_stages + 1;
  *nsts = ns;
  if (ns > max_stages) return cudaErrorInvalidValue;
  std::vector<double> mu((size_t)ns + 1), nu((size_t)ns + 1), mut((size_t)ns + 1), gat((size_t)ns + 1);
  rkl2_coeffs(ns, mu.data(), nu.data(), mut.data(), gat.data());

  if (!mixed) {
    // K and the three face-flux arrays after the background temperatures
    double *K = scratch + 7 * nc + 8 + G.n[2];
    double *F0 = K + nc, *F1 = K + 2 * nc, *F2 = K + 3 * nc;
    auto op = [&](const double *Y) {
      k_diff_k<<<grid3(b), block3(b), 0, s>>>(G, b, p, icv, A, Y, K);
      k_diff_faces<<<grid3(b), block3(b), 0, s>>>(G, b, icv, A, Y, K, F0, F1, F2);
    };
    op(A.Y0);
    k_diff_comb<true><<<grid3(b), block3(b), 0, s>>>(G, b, A, F0, F1, F2, 0.0, 0.0, mut[1] * dt, 0.0, nullptr, nullptr,
                                                      A.Y[1]);
    const double *ym2 = A.Y0, *ym1 = A.Y[1];
    int slot = 2;
    for (int j = 2; j <= ns; ++j) {
      double *yj = A.Y[slot];
      op(ym1);
      k_diff_comb<false><<<grid3(b), block3(b), 0, s>>>(G, b, A, F0, F1, F2, mu[j], nu[j], mut[j] * dt, gat[j] * dt,
                                                         ym1, ym2, yj);
      ym2 = ym1;
      ym1 = yj;
      slot = (slot + 1) % 3;
      if (A.Y[slot] == ym1 || A.Y[slot] == ym2) slot = (slot + 1) % 3;
    }
    k_diff_finish<<<grid3(b), block3(b), 0, s>>>(G, b, A, ym1, U);
    if (nlaunch) *nlaunch = 3 * ns + 2;
    return cudaGetLastError();
  }

  // mixed form: power-of-two scales from the maxima
  const int eY = exp_above(mx[1]);
  const double kt = std::pow(std::ldexp(1.0, eY) * icv, p.nT);   // (2^eY / c_v)^nT
  const int eK = exp_above(mx[2] * kt);
  const int ea = exp_above(mx[3] * icv);
  double wmax = 0.0;
  for (int d = 0; d < 3; ++d)
    if (G.act[d]) wmax = std::fmax(wmax, 2.0 * G.idx[d] * G.idx[d]);
  const int ew = exp_above(wmax);
  Stencil S;
  for (int d = 0; d < 3; ++d) {
    S.n[d] = G.n[d];
    S.act[d] = G.act[d];
    S.per[d] = G.bc[d][0] == PHL_PERIODIC;
    S.w[d] = (float)std::ldexp(2.0 * G.idx[d] * G.idx[d], -ew);
  }
  S.st[0] = 1;
  S.st[1] = G.n[0];
  S.st[2] = (long)G.n[0] * G.n[1];
  k_dmx_prep<<<grid3(b), block3(b), 0, s>>>(G, b, S, M, kt, eK, eY, (float)std::ldexp(1.0, -ea), p.cv);
  // dt M = 2^(eY + eK + ea + ew) dt lambda: the stage factors carry the scales
  const double sc = std::ldexp(dt, eK + ea + ew);
  const int tz = p.tile_z > 0 ? p.tile_z : DTZ_DEFAULT;
  const dim3 grd((unsigned)((G.n[0] + DTX - 1) / DTX), (unsigned)((G.n[1] + DTY - 1) / DTY),
                 (unsigned)((G.n[2] + tz - 1) / tz));
  launch_dmx_stage<true>(p.nT, grd, tz, s, S, M, 0.f, 0.f, (float)(mut[1] * sc), 0.f, nullptr, nullptr, M.d[1]);
  const float *dm2 = nullptr, *dm1 = M.d[1];
  int slot = 2;
  for (int j = 2; j <= ns; ++j) {
    float *dj = M.d[slot];
    // d^(0) = 0: the second stage's nu_2 d^(0) term vanishes
    const float nuj = dm2 ? (float)nu[j] : 0.0f;
    launch_dmx_stage<false>(p.nT, grd, tz, s, S, M, (float)mu[j], nuj, (float)(mut[j] * sc), (float)(gat[j] * sc), dm1,
                            dm2 ? dm2 : dm1, dj);
    dm2 = dm1;
    dm1 = dj;
    slot = (slot + 1) % 3;
    if (M.d[slot] == dm1 || M.d[slot] == dm2) slot = (slot + 1) % 3;
  }
  k_dmx_finish<<<grid3(b), block3(b), 0, s>>>(G, b, dm1, eY, U);
  if (nlaunch) *nlaunch = ns + 3;
  return cudaGetLastError();
}

}  // namespace phl
