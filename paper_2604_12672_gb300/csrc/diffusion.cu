// diffusion.cu -- thermal diffusion by RKL2 super-time-stepping (Sect. 2.10)
// on the device, FP64, behind phl_diffuse.
//
// With the density, velocity, magnetic field and mass fractions held fixed,
// rho d(e_int)/dt = div(K grad T) is advanced over a whole step dt by the
// RKL2 stages of Meyer, Balsara & Aslam (2012) in the paper's form (Sect.
// 2.10, items i-iv), with the paper's stage count from the parabolic limit at
// the start of the step.  Ideal gas: T = e_int / c_v; conductivity
// K = k0 T^nT / rho^nR.  Space: conservative seven-point operator, face flux
// -K_f (T_R - T_L) / dx with K_f the mean of the two cells' K; a side that is
// not periodic carries no flux.
//
// Layout: the grid's own diffusion arrays, dense over the interior cells
// (x fastest): 1/rho and k0/rho^nR (fixed during the step), e_int^(0), the
// operator at e_int^(0), and three stage buffers that rotate.  One kernel
// evaluates the operator at stage j-1 from its seven-point stencil and forms
// stage j; the last stage's change, times rho, goes into the total energy.
#include <math.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "phl_internal.cuh"
#include "stage_common.cuh"

namespace phl {
using namespace stage;
namespace {

struct DiffArrays {
  double *irho, *krho, *Y0, *L0, *Y[3];
};

__device__ __forceinline__ double powi_dev(double x, int n) {
  double r = 1.0;
  for (int q = 0; q < n; ++q) r *= x;
  return r;
}

// e_int, 1/rho, k0/rho^nR of interior cell c, and its parabolic rate
// sum_s D / dx_s^2 with D = K / (rho c_v); block maxima into *dmax (bit
// pattern of a non-negative double, so unsigned order is numeric order).
__global__ void k_diff_init(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                            phl_diffusion p, DiffArrays A, unsigned long long *dmax, int *dflag) {
  double rate = 0.0;
  int c[3];
  if (cell3(box, c)) {
    const long ps = sidx(G, c[0], c[1], c[2]);
    const long q = c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);
    const long pl = G.plane;
    const double r = U[ps];
    const double ux = U[pl + ps] / r, uy = U[2 * pl + ps] / r, uz = U[3 * pl + ps] / r;
    const double bx = 0.5 * (Bf[ps] + Bf[ps + 1]);
    const double by = 0.5 * (Bf[pl + ps] + Bf[pl + ps + G.sy]);
    const double bz = 0.5 * (Bf[2 * pl + ps] + Bf[2 * pl + ps + G.sz]);
    const double e = U[4 * pl + ps] / r - 0.5 * (ux * ux + uy * uy + uz * uz) - 0.5 * (bx * bx + by * by + bz * bz) / r;
    if (!(r > 0.0) || !(e > 0.0)) atomicOr(dflag, FLAG_NEG);
    const double kr = p.k0 / powi_dev(r, p.nR);
    A.irho[q] = 1.0 / r;
    A.krho[q] = kr;
    A.Y0[q] = e;
    const double D = kr * powi_dev(e / p.cv, p.nT) / (r * p.cv);
    for (int d = 0; d < 3; ++d)
      if (G.act[d]) rate += D * G.idx[d] * G.idx[d];
  }
  for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
  __shared__ double red[TPB / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(v));
  }
}

// div(K grad T(Y)) / rho at interior cell c from the seven-point stencil.
__device__ __forceinline__ double diff_op(const DevGeo &G, const phl_diffusion &p, double icv,
                                          const DiffArrays &A, const double *__restrict__ Y, const int *c,
                                          long q) {
  const double Tc = Y[q] * icv;
  const double Kc = A.krho[q] * powi_dev(Tc, p.nT);
  const long st[3] = {1L, (long)G.n[0], (long)G.n[0] * G.n[1]};
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!G.act[d]) continue;
    const bool per = G.bc[d][0] == PHL_PERIODIC;
    double fsum = 0.0;   // (K grad T) at the upper face minus at the lower face
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
      int x = c[d] + side;
      if (x < 0 || x >= G.n[d]) {
        if (!per) continue;   // no flux through a wall or an outflow side
        x = x < 0 ? x + G.n[d] : x - G.n[d];
      }
      const long qn = q + (long)(x - c[d]) * st[d];
      const double Tn = Y[qn] * icv;
      const double Kn = A.krho[qn] * powi_dev(Tn, p.nT);
      fsum += 0.5 * (Kc + Kn) * ((Tn - Tc) * G.idx[d]);
    }
    s += fsum * G.idx[d];
  }
  return s * A.irho[q];
}

// L0 = operator at e_int^(0); stage 1: Y1 = Y0 + mu~_1 dt L0
__global__ void k_diff_first(DevGeo G, Box box, phl_diffusion p, DiffArrays A, double mdt, double *__restrict__ Y1) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);
  const double L0 = diff_op(G, p, 1.0 / p.cv, A, A.Y0, c, q);
  A.L0[q] = L0;
  Y1[q] = A.Y0[q] + mdt * L0;
}

// stage j: Y_j = mu Y_{j-1} + nu Y_{j-2} + (1 - mu - nu) Y0 + mu~ dt L(Y_{j-1}) + gamma~ dt L0
__global__ void k_diff_stage(DevGeo G, Box box, phl_diffusion p, DiffArrays A, double mu, double nu, double mdt,
                             double gdt, const double *__restrict__ Ym1, const double *__restrict__ Ym2,
                             double *__restrict__ Yj) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);
  const double L = diff_op(G, p, 1.0 / p.cv, A, Ym1, c, q);
  Yj[q] = mu * Ym1[q] + nu * Ym2[q] + (1.0 - mu - nu) * A.Y0[q] + mdt * L + gdt * A.L0[q];
}

// E += rho (e_int^(N) - e_int^(0))
__global__ void k_diff_finish(DevGeo G, Box box, DiffArrays A, const double *__restrict__ YN, double *__restrict__ U) {
  int c[3];
  if (!cell3(box, c)) return;
  const long q = c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);
  const long ps = sidx(G, c[0], c[1], c[2]);
  U[4 * G.plane + ps] += (YN[q] - A.Y0[q]) / A.irho[q];
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
  const int n = 1 + (int)std::floor(0.5 * (std::sqrt(9.0 + 16.0 * dt / dt_p) - 1.0));
  return n < 3 ? 3 : n;
}

cudaError_t launch_diffuse(const DevGeo &G, double *U, const double *Bf, const phl_diffusion &p, double dt,
                           int max_stages, double *scratch, unsigned long long *dmax, int *dflag, cudaStream_t s,
                           int *nsts, int *nlaunch) {
  const long nc = (long)G.n[0] * G.n[1] * G.n[2];
  DiffArrays A;
  A.irho = scratch;
  A.krho = scratch + nc;
  A.Y0 = scratch + 2 * nc;
  A.L0 = scratch + 3 * nc;
  for (int k = 0; k < 3; ++k) A.Y[k] = scratch + (4 + k) * nc;
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_diff_init<<<grid3(b), block3(b), 0, s>>>(G, b, U, Bf, p, A, dmax, dflag);
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  double rate;
  memcpy(&rate, &bits, sizeof(rate));
  const int ns = rate > 0.0 ? sts_stage_count(dt, 0.5 / rate) : 3;
  *nsts = ns;
  if (ns > max_stages) return cudaErrorInvalidValue;
  std::vector<double> mu((size_t)ns + 1), nu((size_t)ns + 1), mut((size_t)ns + 1), gat((size_t)ns + 1);
  rkl2_coeffs(ns, mu.data(), nu.data(), mut.data(), gat.data());
  k_diff_first<<<grid3(b), block3(b), 0, s>>>(G, b, p, A, mut[1] * dt, A.Y[1]);
  const double *ym2 = A.Y0, *ym1 = A.Y[1];
  int slot = 2;
  for (int j = 2; j <= ns; ++j) {
    double *yj = A.Y[slot];
    k_diff_stage<<<grid3(b), block3(b), 0, s>>>(G, b, p, A, mu[j], nu[j], mut[j] * dt, gat[j] * dt, ym1, ym2, yj);
    ym2 = ym1;
    ym1 = yj;
    slot = (slot + 1) % 3;
    if (A.Y[slot] == ym1 || A.Y[slot] == ym2) slot = (slot + 1) % 3;
  }
  k_diff_finish<<<grid3(b), block3(b), 0, s>>>(G, b, A, ym1, U);
  if (nlaunch) *nlaunch = ns + 2;
  return cudaGetLastError();
}

}  // namespace phl
