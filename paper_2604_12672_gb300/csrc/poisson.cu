// poisson.cu -- the Poisson solver for the gravitational potential (Sect.
// 2.12) on the device, behind phl_poisson_*.
//
// Grid: Cartesian, every axis stretched independently (the caller gives the
// face coordinates); cell centres are face midpoints, the ghost centre beyond
// a boundary face the mirror image of the first (last) centre.  Operator:
// the paper's three-point formula per axis (Eq. poisson-FD) with
//   L1 = 2/(dm (dm + dp)), L2 = -2/(dm dp), L3 = 2/(dp (dm + dp)),
// dm, dp the centre spacings below and above.  Boundary values: the exterior
// multipole expansion of the cell masses about their centre of mass
// (monopole; quadrupole for lmax >= 2; octupole for lmax >= 3), moved to the
// right-hand side.  Solver: BiCGSTAB (van der Vorst 1992) with the Jacobi
// preconditioner on the right, in the order of the preconditioned algorithm
// of Barrett et al. (1994); stop when the RMS of the weighted residual
// (weights 1/(4 pi G rho), Eq. poisson-eps, or 1) is below tol, checked after
// the half step and after the full step.  Gravity: g = -grad phi by the
// non-uniform central difference (Eqs. grav_x..grav_z).  FP64 throughout.
//
// Device layout: dense cell vectors (x fastest, 32-bit indices), per-axis
// coefficient arrays.  One BiCGSTAB iteration is five grid-stride kernels:
//   K1  p = r + beta (p - omega v), ph = D^-1 p
//   K2  v = A ph (= p + off-diagonal part of A applied to ph); partials of (rh, v)
//   K3  s = r - alpha v, sh = D^-1 s;  partial sums of |w s|^2
//   K4  t = A sh (= s + off-diagonal part on sh); partials of (t, s), (t, t)
//   K5  x += alpha ph + omega sh, r = s - omega t;  partials of (rh, r), |w r|^2
// Each reduction leaves one partial per block; a consumer kernel's first warp
// sums the partials in a fixed order, so every block derives the same
// scalars (alpha, omega, the norms) and takes the same decision without a
// grid-wide barrier.  Convergence and breakdown are decided on the device and
// recorded in a small status block, so the host enqueues iterations in
// batches and reads the status once per batch; the kernels of an iteration
// after the decision return at once.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "phl.h"
#include "phl_internal.cuh"

namespace phl {
namespace {

constexpr int PT = 256;   // threads per block

enum { Q_RR = 0, Q_NR, Q_RV, Q_NS, Q_TS, Q_TT, Q_COUNT };
enum { ST_RUN = 0, ST_HALF = 2, ST_DONE = 3, ST_BREAK = -2, ST_BADRHO = -3 };

struct Status {
  double rho_old, alpha, omega, rho, resid;
  int status, iters;
};

struct PGeo {
  int n[3];
  unsigned nc, sy, sz;
  const double *L1[3], *L2[3], *L3[3];
  const double *gm[3], *g0[3], *gp[3];   // gravity coefficients of phi_{i-1}, phi_i, phi_{i+1}
  const double *xc[3];                   // centres, index i + 1 for i = -1..n
  const double *wd[3];                   // cell widths
  double G;
  int lmax, relative, nb;
  double tol;
  unsigned gofs[3];                      // offsets of the x, y, z ghost blocks
};

struct Vecs {
  double *x, *r, *rh, *p, *v, *s, *t, *ph, *sh, *dinv, *w, *rho, *ghost;
  double *part;    // [Q_COUNT][nb]
  double *mpart;   // multipole partials [20][nb]
  Status *st;
};

__device__ __forceinline__ void decode(const PGeo &g, unsigned q, int &i, int &j, int &k) {
  const unsigned a = q / (unsigned)g.n[0];
  const unsigned b = a / (unsigned)g.n[1];
  i = (int)(q - a * (unsigned)g.n[0]);
  j = (int)(a - b * (unsigned)g.n[1]);
  k = (int)b;
}

// Block sum of v (all threads), result valid in every thread after the call.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Sum of nb partials by warp 0 in a fixed order (the same in every block).
__device__ __forceinline__ double sum_parts(const double *part, int nb) {
  double s = 0.0;
  for (int b = (int)threadIdx.x; b < nb; b += 32) s += part[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// neighbour of cell (i, j, k) along axis d: the cell's value or the ghost
// potential (ghost null: zero, the homogeneous operator)
__device__ __forceinline__ double nbv(const PGeo &g, const double *__restrict__ f, const double *__restrict__ ghost,
                                      unsigned q, int i, int j, int k, int d, int side) {
  const int c = d == 0 ? i : (d == 1 ? j : k);
  const unsigned st = d == 0 ? 1u : (d == 1 ? g.sy : g.sz);
  if (side < 0 && c > 0) return f[q - st];
  if (side > 0 && c + 1 < g.n[d]) return f[q + st];
  if (!ghost) return 0.0;
  const unsigned hi = side > 0;
  if (d == 0) return ghost[g.gofs[0] + hi * (unsigned)g.n[1] * g.n[2] + j + (unsigned)g.n[1] * k];
  if (d == 1) return ghost[g.gofs[1] + hi * (unsigned)g.n[0] * g.n[2] + i + (unsigned)g.n[0] * k];
  return ghost[g.gofs[2] + hi * (unsigned)g.n[0] * g.n[1] + i + (unsigned)g.n[0] * j];
}

__device__ __forceinline__ double apply_at(const PGeo &g, const double *__restrict__ f,
                                           const double *__restrict__ ghost, unsigned q, int i, int j, int k) {
  const int c[3] = {i, j, k};
  const double fc = f[q];
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    s += g.L1[d][c[d]] * nbv(g, f, ghost, q, i, j, k, d, -1) + g.L2[d][c[d]] * fc +
         g.L3[d][c[d]] * nbv(g, f, ghost, q, i, j, k, d, +1);
  return s;
}

// the ghost terms of the operator at cell (i, j, k): A applied to zero
// interior values with the ghost potentials (zero away from the sides)
__device__ __forceinline__ double ghost_terms(const PGeo &g, const double *__restrict__ ghost, int i, int j, int k) {
  const int c[3] = {i, j, k};
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double lo = 0.0, hi = 0.0;
    if (c[d] == 0) lo = nbv(g, ghost, ghost, 0u, i, j, k, d, -1);
    if (c[d] + 1 == g.n[d]) hi = nbv(g, ghost, ghost, 0u, i, j, k, d, +1);
    s += g.L1[d][c[d]] * lo + g.L2[d][c[d]] * 0.0 + g.L3[d][c[d]] * hi;
  }
  return s;
}

// A D^-1 u at cell q for the Jacobi-preconditioned iteration, given
// uh = D^-1 u: the diagonal part D uh is u itself, so only the off-diagonal
// neighbours are multiplied (six FMAs instead of nine multiplies and adds).
__device__ __forceinline__ double apply_pre(const PGeo &g, const double *__restrict__ u,
                                            const double *__restrict__ uh, unsigned q, int i, int j, int k) {
  const int c[3] = {i, j, k};
  const unsigned st[3] = {1u, g.sy, g.sz};
  double s = u[q];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (c[d] > 0) s += g.L1[d][c[d]] * uh[q - st[d]];
    if (c[d] + 1 < g.n[d]) s += g.L3[d][c[d]] * uh[q + st[d]];
  }
  return s;
}

__device__ __forceinline__ bool block0_lead() { return blockIdx.x == 0 && threadIdx.x == 0; }

// ---------------------------------------------------------------- multipoles

__device__ __forceinline__ double cell_mass(const PGeo &g, const double *rho, unsigned q, int i, int j, int k) {
  return rho[q] * (g.wd[0][i] * g.wd[1][j] * g.wd[2][k]);
}

// partials of m, m x, m y, m z
__global__ void k_mom1(PGeo g, Vecs V) {
  __shared__ double sh[PT / 32];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    const double m = cell_mass(g, V.rho, q, i, j, k);
    a[0] += m;
    a[1] += m * g.xc[0][i + 1];
    a[2] += m * g.xc[1][j + 1];
    a[3] += m * g.xc[2][k + 1];
  }
  for (int c = 0; c < 4; ++c) {
    const double t = block_sum(a[c], sh);
    if (threadIdx.x == 0) V.mpart[c * g.nb + blockIdx.x] = t;
  }
}

// M and the centre of mass from the first partials (every thread)
__device__ __forceinline__ void mass_centre(const PGeo &g, const Vecs &V, double &M, double *X) {
  __shared__ double s4[4];
  if (threadIdx.x < 32)
    for (int c = 0; c < 4; ++c) {
      const double t = sum_parts(V.mpart + c * g.nb, g.nb);
      if (threadIdx.x == 0) s4[c] = t;
    }
  __syncthreads();
  M = s4[0];
  for (int a = 0; a < 3; ++a) X[a] = M != 0.0 ? s4[a + 1] / M : 0.0;
  __syncthreads();
}

// the 6 + 10 independent components of Q_ij, O_ijk of one mass at x (about X)
__device__ __forceinline__ void qo_terms(double m, const double *x, double *o16) {
  const double x2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  // Q: xx, yy, zz, xy, xz, yz
  o16[0] = m * (3.0 * x[0] * x[0] - x2);
  o16[1] = m * (3.0 * x[1] * x[1] - x2);
  o16[2] = m * (3.0 * x[2] * x[2] - x2);
  o16[3] = m * 3.0 * x[0] * x[1];
  o16[4] = m * 3.0 * x[0] * x[2];
  o16[5] = m * 3.0 * x[1] * x[2];
  // O: xxx yyy zzz xxy xxz yyx yyz zzx zzy xyz
  // O_aaa = 15 x_a^3 - 9 |x|^2 x_a; O_aab = 15 x_a^2 x_b - 3 |x|^2 x_b; O_xyz = 15 x y z
  o16[6] = m * (15.0 * x[0] * x[0] * x[0] - 9.0 * x2 * x[0]);
  o16[7] = m * (15.0 * x[1] * x[1] * x[1] - 9.0 * x2 * x[1]);
  o16[8] = m * (15.0 * x[2] * x[2] * x[2] - 9.0 * x2 * x[2]);
  o16[9] = m * (15.0 * x[0] * x[0] * x[1] - 3.0 * x2 * x[1]);
  o16[10] = m * (15.0 * x[0] * x[0] * x[2] - 3.0 * x2 * x[2]);
  o16[11] = m * (15.0 * x[1] * x[1] * x[0] - 3.0 * x2 * x[0]);
  o16[12] = m * (15.0 * x[1] * x[1] * x[2] - 3.0 * x2 * x[2]);
  o16[13] = m * (15.0 * x[2] * x[2] * x[0] - 3.0 * x2 * x[0]);
  o16[14] = m * (15.0 * x[2] * x[2] * x[1] - 3.0 * x2 * x[1]);
  o16[15] = m * 15.0 * x[0] * x[1] * x[2];
}

__global__ void k_mom2(PGeo g, Vecs V) {
  __shared__ double sh[PT / 32];
  double M, X[3];
  mass_centre(g, V, M, X);
  double a[16];
  for (int c = 0; c < 16; ++c) a[c] = 0.0;
  if (g.lmax >= 2)
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
      int i, j, k;
      decode(g, q, i, j, k);
      const double m = cell_mass(g, V.rho, q, i, j, k);
      const double x[3] = {g.xc[0][i + 1] - X[0], g.xc[1][j + 1] - X[1], g.xc[2][k + 1] - X[2]};
      double t[16];
      qo_terms(m, x, t);
      for (int c = 0; c < 16; ++c) a[c] += t[c];
    }
  for (int c = 0; c < 16; ++c) {
    const double t = block_sum(a[c], sh);
    if (threadIdx.x == 0) V.mpart[(4 + c) * g.nb + blockIdx.x] = t;
  }
}

// ghost potentials at the ghost centres from the expansion
__global__ void k_ghost(PGeo g, Vecs V, unsigned nghost) {
  double M, X[3];
  mass_centre(g, V, M, X);
  __shared__ double s16[16];
  if (threadIdx.x < 32)
    for (int c = 0; c < 16; ++c) {
      const double t = sum_parts(V.mpart + (4 + c) * g.nb, g.nb);
      if (threadIdx.x == 0) s16[c] = t;
    }
  __syncthreads();
  const double Q[6] = {s16[0], s16[1], s16[2], s16[3], s16[4], s16[5]};
  const double *Oc = s16 + 6;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  for (unsigned h = blockIdx.x * blockDim.x + threadIdx.x; h < nghost; h += gridDim.x * blockDim.x) {
    double r[3];
    unsigned u;
    if (h < g.gofs[1]) {   // x faces [2][nz][ny]
      u = h;
      const unsigned side = u / ((unsigned)ny * nz), rem = u % ((unsigned)ny * nz);
      r[0] = g.xc[0][side ? nx + 1 : 0];
      r[1] = g.xc[1][rem % ny + 1];
      r[2] = g.xc[2][rem / ny + 1];
    } else if (h < g.gofs[2]) {   // y faces [2][nz][nx]
      u = h - g.gofs[1];
      const unsigned side = u / ((unsigned)nx * nz), rem = u % ((unsigned)nx * nz);
      r[0] = g.xc[0][rem % nx + 1];
      r[1] = g.xc[1][side ? ny + 1 : 0];
      r[2] = g.xc[2][rem / nx + 1];
    } else {   // z faces [2][ny][nx]
      u = h - g.gofs[2];
      const unsigned side = u / ((unsigned)nx * ny), rem = u % ((unsigned)nx * ny);
      r[0] = g.xc[0][rem % nx + 1];
      r[1] = g.xc[1][rem / nx + 1];
      r[2] = g.xc[2][side ? nz + 1 : 0];
    }
    double phi = 0.0;
    if (M != 0.0) {
      const double R[3] = {r[0] - X[0], r[1] - X[1], r[2] - X[2]};
      const double R2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      const double ir = 1.0 / sqrt(R2);
      double sum = M * ir;
      if (g.lmax >= 2) {
        const double qq = Q[0] * R[0] * R[0] + Q[1] * R[1] * R[1] + Q[2] * R[2] * R[2] +
                          2.0 * (Q[3] * R[0] * R[1] + Q[4] * R[0] * R[2] + Q[5] * R[1] * R[2]);
        const double ir2 = ir * ir;
        sum += 0.5 * qq * ir2 * ir2 * ir;
        if (g.lmax >= 3) {
          // sum over all (a, b, c) of O_abc R_a R_b R_c with the multiplicities of
          // the independent components (3 for aab, 6 for xyz)
          const double oo = Oc[0] * R[0] * R[0] * R[0] + Oc[1] * R[1] * R[1] * R[1] + Oc[2] * R[2] * R[2] * R[2] +
                            3.0 * (Oc[3] * R[0] * R[0] * R[1] + Oc[4] * R[0] * R[0] * R[2] +
                                   Oc[5] * R[1] * R[1] * R[0] + Oc[6] * R[1] * R[1] * R[2] +
                                   Oc[7] * R[2] * R[2] * R[0] + Oc[8] * R[2] * R[2] * R[1]) +
                            6.0 * Oc[9] * R[0] * R[1] * R[2];
          sum += oo / 6.0 * ir2 * ir2 * ir2 * ir;
        }
      }
      phi = -g.G * sum;
    }
    V.ghost[h] = phi;
  }
}

// ------------------------------------------------------------ BiCGSTAB set-up

// r = b - A x0 with b = 4 pi G rho - (ghost terms); rh = r; p = v = 0;
// D^-1, the residual weights; partials of (rh, r) and |w r|^2.
__global__ void k_init(PGeo g, Vecs V) {
  __shared__ double sh[PT / 32];
  const double fpg = 4.0 * 3.14159265358979323846 * g.G;
  double rr = 0.0, nr = 0.0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    const double b = fpg * V.rho[q] - ghost_terms(g, V.ghost, i, j, k);
    const double r = b - apply_at(g, V.x, nullptr, q, i, j, k);
    if (g.relative && !(V.rho[q] > 0.0)) V.st->status = ST_BADRHO;   // every writer writes the same value
    const double w = g.relative ? 1.0 / (fpg * V.rho[q]) : 1.0;
    V.r[q] = r;
    V.rh[q] = r;
    V.p[q] = 0.0;
    V.v[q] = 0.0;
    V.dinv[q] = 1.0 / (g.L2[0][i] + g.L2[1][j] + g.L2[2][k]);
    V.w[q] = w;
    rr += r * r;
    nr += (w * r) * (w * r);
  }
  rr = block_sum(rr, sh);
  nr = block_sum(nr, sh);
  if (threadIdx.x == 0) {
    V.part[Q_RR * g.nb + blockIdx.x] = rr;
    V.part[Q_NR * g.nb + blockIdx.x] = nr;
  }
}

// ------------------------------------------------------------ one iteration

// K1: residual check of the previous full step; p and ph.
__global__ void k_bi_p(PGeo g, Vecs V, int it) {
  if (V.st->status != ST_RUN) return;
  __shared__ double s2[2];
  if (threadIdx.x < 32) {
    const double rr = sum_parts(V.part + Q_RR * g.nb, g.nb), nr = sum_parts(V.part + Q_NR * g.nb, g.nb);
    if (threadIdx.x == 0) { s2[0] = rr; s2[1] = nr; }
  }
  __syncthreads();
  const double rr = s2[0], res = sqrt(s2[1] / (double)g.nc);
  if (res < g.tol) {
    if (block0_lead()) { V.st->status = ST_DONE; V.st->iters = it - 1; V.st->resid = res; }
    return;
  }
  if ((it > 1 && V.st->omega == 0.0) || rr == 0.0) {
    if (block0_lead()) { V.st->status = ST_BREAK; V.st->iters = it - 1; V.st->resid = res; }
    return;
  }
  const double beta = it == 1 ? 0.0 : (rr / V.st->rho_old) * (V.st->alpha / V.st->omega);
  const double om = V.st->omega;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    const double p = it == 1 ? V.r[q] : V.r[q] + beta * (V.p[q] - om * V.v[q]);
    V.p[q] = p;
    V.ph[q] = V.dinv[q] * p;
  }
  if (block0_lead()) { V.st->rho = rr; V.st->resid = res; }
}

// K2: v = A ph, partials of (rh, v)
__global__ void k_bi_av(PGeo g, Vecs V) {
  if (V.st->status != ST_RUN) return;
  __shared__ double sh[PT / 32];
  double rv = 0.0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    const double v = apply_pre(g, V.p, V.ph, q, i, j, k);
    V.v[q] = v;
    rv += V.rh[q] * v;
  }
  rv = block_sum(rv, sh);
  if (threadIdx.x == 0) V.part[Q_RV * g.nb + blockIdx.x] = rv;
}

// K3: alpha, s, sh; partials of |w s|^2
__global__ void k_bi_s(PGeo g, Vecs V, int it) {
  if (V.st->status != ST_RUN) return;
  __shared__ double sh[PT / 32];
  __shared__ double s1;
  if (threadIdx.x < 32) {
    const double rv = sum_parts(V.part + Q_RV * g.nb, g.nb);
    if (threadIdx.x == 0) s1 = rv;
  }
  __syncthreads();
  const double rv = s1;
  if (rv == 0.0) {
    if (block0_lead()) { V.st->status = ST_BREAK; V.st->iters = it; }
    return;
  }
  const double alpha = V.st->rho / rv;
  double ns = 0.0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    const double s = V.r[q] - alpha * V.v[q];
    V.s[q] = s;
    V.sh[q] = V.dinv[q] * s;
    const double ws = g.relative ? V.w[q] * s : s;   // the absolute criterion has unit weights
    ns += ws * ws;
  }
  ns = block_sum(ns, sh);
  if (threadIdx.x == 0) V.part[Q_NS * g.nb + blockIdx.x] = ns;
  if (block0_lead()) V.st->alpha = alpha;
}

// K4: half-step check; t = A sh, partials of (t, s), (t, t)
__global__ void k_bi_at(PGeo g, Vecs V, int it) {
  if (V.st->status != ST_RUN) return;
  __shared__ double sh[PT / 32];
  __shared__ double s1;
  if (threadIdx.x < 32) {
    const double ns = sum_parts(V.part + Q_NS * g.nb, g.nb);
    if (threadIdx.x == 0) s1 = ns;
  }
  __syncthreads();
  const double res = sqrt(s1 / (double)g.nc);
  if (res < g.tol) {
    if (block0_lead()) { V.st->status = ST_HALF; V.st->iters = it; V.st->resid = res; }
    return;
  }
  double ts = 0.0, tt = 0.0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    const double t = apply_pre(g, V.s, V.sh, q, i, j, k);
    V.t[q] = t;
    ts += t * V.s[q];
    tt += t * t;
  }
  ts = block_sum(ts, sh);
  tt = block_sum(tt, sh);
  if (threadIdx.x == 0) {
    V.part[Q_TS * g.nb + blockIdx.x] = ts;
    V.part[Q_TT * g.nb + blockIdx.x] = tt;
  }
}

// K5: the solution and residual updates (or the half-step update decided by
// K4 of this iteration); partials of (rh, r) and |w r|^2 for the next K1.
__global__ void k_bi_x(PGeo g, Vecs V, int it) {
  const int st = V.st->status;
  const double alpha = V.st->alpha;
  if (st == ST_HALF) {
    if (V.st->iters != it) return;
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
      V.x[q] += alpha * V.ph[q];
      V.r[q] = V.s[q];
    }
    return;
  }
  if (st != ST_RUN) return;
  __shared__ double sh[PT / 32];
  __shared__ double s2[2];
  if (threadIdx.x < 32) {
    const double ts = sum_parts(V.part + Q_TS * g.nb, g.nb), tt = sum_parts(V.part + Q_TT * g.nb, g.nb);
    if (threadIdx.x == 0) { s2[0] = ts; s2[1] = tt; }
  }
  __syncthreads();
  if (s2[1] == 0.0) {
    if (block0_lead()) { V.st->status = ST_BREAK; V.st->iters = it; }
    return;
  }
  const double omega = s2[0] / s2[1];
  double rr = 0.0, nr = 0.0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    V.x[q] += alpha * V.ph[q] + omega * V.sh[q];
    const double r = V.s[q] - omega * V.t[q];
    V.r[q] = r;
    rr += V.rh[q] * r;
    const double wr = g.relative ? V.w[q] * r : r;
    nr += wr * wr;
  }
  rr = block_sum(rr, sh);
  nr = block_sum(nr, sh);
  if (threadIdx.x == 0) {
    V.part[Q_RR * g.nb + blockIdx.x] = rr;
    V.part[Q_NR * g.nb + blockIdx.x] = nr;
  }
  if (block0_lead()) {
    V.st->omega = omega;
    V.st->rho_old = V.st->rho;
  }
}

// g = -grad phi (non-uniform central difference), ghost potentials at the sides
__global__ void k_gravity(PGeo g, const double *__restrict__ phi, const double *__restrict__ ghost,
                          double *__restrict__ gx, double *__restrict__ gy, double *__restrict__ gz) {
  double *out[3] = {gx, gy, gz};
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < g.nc; q += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    const int c[3] = {i, j, k};
    for (int d = 0; d < 3; ++d)
      out[d][q] = g.gp[d][c[d]] * nbv(g, phi, ghost, q, i, j, k, d, +1) + g.g0[d][c[d]] * phi[q] +
                  g.gm[d][c[d]] * nbv(g, phi, ghost, q, i, j, k, d, -1);
  }
}

}  // namespace
}  // namespace phl

using namespace phl;

struct phl_poisson {
  PGeo g;
  Vecs V;
  cudaStream_t stream = nullptr;
  int max_iter = 0;
  int batch = 16;
  unsigned nghost = 0;
  double *coef = nullptr;   // device: per-axis arrays
  double *vec = nullptr;    // device: cell vectors and partials
  Status *st = nullptr;
  bool solved = false;
};

namespace {

phl_status pfail(phl_status s, const char *msg) {
  set_error((int)s, "%s", msg);
  return s;
}

phl_status pcuda(cudaError_t e, const char *what) {
  set_error((int)PHL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return PHL_ECUDA;
}

}  // namespace

extern "C" {

phl_status phl_poisson_create(const phl_poisson_desc *d, phl_poisson **out) {
  if (!d || !out) return pfail(PHL_EINVAL, "null argument");
  *out = nullptr;
  double cells = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 2 || !d->xf[a]) return pfail(PHL_EINVAL, "each axis needs at least 2 cells and its faces");
    for (int i = 0; i < d->n[a]; ++i)
      if (!(d->xf[a][i + 1] > d->xf[a][i])) return pfail(PHL_EINVAL, "face coordinates must increase");
    cells *= d->n[a];
  }
  // 32-bit cell indices; the margin keeps q + (grid stride) of the grid-stride
  // loops from wrapping past 2^32
  if (cells > 4294967296.0 - 16777216.0)
    return pfail(PHL_EUNSUPPORTED, "the Poisson solver indexes cells with 32 bits (at most 2^32 - 2^24 cells)");
  if (!(d->lmax == 0 || d->lmax == 2 || d->lmax == 3)) return pfail(PHL_EINVAL, "lmax must be 0, 2 or 3");
  if (d->criterion != PHL_POISSON_RELATIVE && d->criterion != PHL_POISSON_ABSOLUTE)
    return pfail(PHL_EINVAL, "bad convergence criterion");
  if (!(d->tol > 0.0) || d->max_iter < 1 || !(d->G > 0.0)) return pfail(PHL_EINVAL, "bad tol, max_iter or G");
  phl_poisson *P = new phl_poisson();
  PGeo &g = P->g;
  for (int a = 0; a < 3; ++a) g.n[a] = d->n[a];
  g.nc = (unsigned)cells;
  g.sy = (unsigned)g.n[0];
  g.sz = (unsigned)g.n[0] * g.n[1];
  g.G = d->G;
  g.lmax = d->lmax;
  g.relative = d->criterion == PHL_POISSON_RELATIVE;
  g.tol = d->tol;
  P->max_iter = d->max_iter;
  P->stream = (cudaStream_t)d->stream;
  g.gofs[0] = 0;
  g.gofs[1] = 2u * g.n[1] * g.n[2];
  g.gofs[2] = g.gofs[1] + 2u * g.n[0] * g.n[2];
  P->nghost = g.gofs[2] + 2u * g.n[0] * g.n[1];
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned want = (unsigned)(sms > 0 ? sms : 1) * 4u, most = (g.nc + PT - 1) / PT;
  g.nb = (int)(want < most ? want : most);

  // per-axis coefficients on the host (FP64)
  std::vector<double> hc;
  size_t ofs[3][8];
  for (int a = 0; a < 3; ++a) {
    const int n = g.n[a];
    const double *xf = d->xf[a];
    std::vector<double> xc((size_t)n + 2);
    for (int i = 0; i < n; ++i) xc[(size_t)i + 1] = 0.5 * (xf[i] + xf[i + 1]);
    xc[0] = 2.0 * xf[0] - xc[1];
    xc[(size_t)n + 1] = 2.0 * xf[n] - xc[(size_t)n];
    std::vector<double> L1(n), L2(n), L3(n), gm(n), g0(n), gp(n), wd(n);
    for (int i = 0; i < n; ++i) {
      const double dm = xc[(size_t)i + 1] - xc[(size_t)i], dp = xc[(size_t)i + 2] - xc[(size_t)i + 1];
      L1[i] = 2.0 / (dm * (dm + dp));
      L2[i] = -2.0 / (dm * dp);
      L3[i] = 2.0 / (dp * (dm + dp));
      gp[i] = -dm / (dp * (dp + dm));
      g0[i] = -(dp - dm) / (dp * dm);
      gm[i] = dp / (dm * (dp + dm));
      wd[i] = xf[i + 1] - xf[i];
    }
    const std::vector<double> *arrs[8] = {&L1, &L2, &L3, &gm, &g0, &gp, &xc, &wd};
    for (int k = 0; k < 8; ++k) {
      ofs[a][k] = hc.size();
      hc.insert(hc.end(), arrs[k]->begin(), arrs[k]->end());
    }
  }
  cudaError_t e = cudaMalloc(&P->coef, hc.size() * sizeof(double));
  if (e != cudaSuccess) { delete P; return pfail(PHL_ENOMEM, "Poisson coefficients"); }
  e = cudaMemcpy(P->coef, hc.data(), hc.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(P->coef); delete P; return pcuda(e, "Poisson coefficients"); }
  for (int a = 0; a < 3; ++a) {
    g.L1[a] = P->coef + ofs[a][0];
    g.L2[a] = P->coef + ofs[a][1];
    g.L3[a] = P->coef + ofs[a][2];
    g.gm[a] = P->coef + ofs[a][3];
    g.g0[a] = P->coef + ofs[a][4];
    g.gp[a] = P->coef + ofs[a][5];
    g.xc[a] = P->coef + ofs[a][6];
    g.wd[a] = P->coef + ofs[a][7];
  }
  // 12 cell vectors, the ghost potentials, partials, status
  const size_t nc = g.nc, nb = (size_t)g.nb;
  const size_t total = 12 * nc + P->nghost + (Q_COUNT + 20) * nb + 8;
  e = cudaMalloc(&P->vec, total * sizeof(double));
  if (e != cudaSuccess) { cudaFree(P->coef); delete P; return pfail(PHL_ENOMEM, "Poisson vectors"); }
  double *v = P->vec;
  Vecs &V = P->V;
  double **seq[12] = {&V.x, &V.r, &V.rh, &V.p, &V.v, &V.s, &V.t, &V.ph, &V.sh, &V.dinv, &V.w, &V.rho};
  for (int k = 0; k < 12; ++k) *seq[k] = v + k * nc;
  V.ghost = v + 12 * nc;
  V.part = V.ghost + P->nghost;
  V.mpart = V.part + Q_COUNT * nb;
  V.st = (Status *)(V.mpart + 20 * nb);
  P->st = V.st;
  *out = P;
  return PHL_OK;
}

phl_status phl_poisson_destroy(phl_poisson *P) {
  if (!P) return PHL_OK;
  cudaFree(P->vec);
  cudaFree(P->coef);
  delete P;
  return PHL_OK;
}

phl_status phl_poisson_solve(phl_poisson *P, const double *rho, double *phi, int where, int *iters, double *resid) {
  if (!P || !rho || !phi) return pfail(PHL_EINVAL, "null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return pfail(PHL_EINVAL, "bad memory kind");
  const PGeo &g = P->g;
  Vecs &V = P->V;
  cudaStream_t s = P->stream;
  const size_t bytes = (size_t)g.nc * sizeof(double);
  const cudaMemcpyKind kin = where == PHL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaMemcpyAsync(V.rho, rho, bytes, kin, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(V.x, phi, bytes, kin, s);
  Status h0{1.0, 1.0, 1.0, 0.0, 0.0, ST_RUN, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->st, &h0, sizeof(Status), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return pcuda(e, "Poisson inputs");
  const dim3 grid((unsigned)g.nb), block(PT);
  k_mom1<<<grid, block, 0, s>>>(g, V);
  k_mom2<<<grid, block, 0, s>>>(g, V);
  k_ghost<<<grid, block, 0, s>>>(g, V, P->nghost);
  k_init<<<grid, block, 0, s>>>(g, V);
  if ((e = cudaGetLastError()) != cudaSuccess) return pcuda(e, "Poisson set-up");
  Status h{};
  int it = 1;
  for (;;) {
    const int last = it + P->batch - 1 < P->max_iter ? it + P->batch - 1 : P->max_iter;
    for (; it <= last; ++it) {
      k_bi_p<<<grid, block, 0, s>>>(g, V, it);
      k_bi_av<<<grid, block, 0, s>>>(g, V);
      k_bi_s<<<grid, block, 0, s>>>(g, V, it);
      k_bi_at<<<grid, block, 0, s>>>(g, V, it);
      k_bi_x<<<grid, block, 0, s>>>(g, V, it);
    }
    // the residual check of the last full step happens in the next K1
    if (it > P->max_iter) k_bi_p<<<grid, block, 0, s>>>(g, V, it);
    e = cudaMemcpyAsync(&h, P->st, sizeof(Status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pcuda(e, "Poisson iterations");
    if (h.status != ST_RUN || it > P->max_iter) break;
  }
  e = cudaMemcpyAsync(phi, V.x, bytes, where == PHL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return pcuda(e, "Poisson result");
  P->solved = true;
  if (iters) *iters = h.status == ST_RUN ? P->max_iter : h.iters;
  if (resid) *resid = h.resid;
  if (h.status == ST_BADRHO) return pfail(PHL_EINVAL, "the relative criterion needs rho > 0 in every cell");
  if (h.status == ST_BREAK) return pfail(PHL_ENOCONV, "BiCGSTAB broke down (a vanishing inner product)");
  if (h.status == ST_RUN) return pfail(PHL_ENOCONV, "BiCGSTAB did not reach the tolerance within max_iter");
  return PHL_OK;
}

phl_status phl_poisson_ghost(phl_poisson *P, double *ghost, int where) {
  if (!P || !ghost) return pfail(PHL_EINVAL, "null argument");
  if (!P->solved) return pfail(PHL_EINVAL, "no solve yet");
  const cudaError_t e = cudaMemcpy(ghost, P->V.ghost, (size_t)P->nghost * sizeof(double),
                                   where == PHL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  return e == cudaSuccess ? PHL_OK : pcuda(e, "Poisson ghost potentials");
}

phl_status phl_poisson_gravity(phl_poisson *P, const double *phi, double *gx, double *gy, double *gz, int where) {
  if (!P || !phi || !gx || !gy || !gz) return pfail(PHL_EINVAL, "null argument");
  if (!P->solved) return pfail(PHL_EINVAL, "no solve yet (the boundary potentials come from it)");
  const PGeo &g = P->g;
  cudaStream_t s = P->stream;
  const size_t bytes = (size_t)g.nc * sizeof(double);
  const dim3 grid((unsigned)g.nb), block(PT);
  cudaError_t e;
  if (where == PHL_DEVICE) {
    k_gravity<<<grid, block, 0, s>>>(g, phi, P->V.ghost, gx, gy, gz);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PHL_OK : pcuda(e, "gravity");
  }
  // host arrays: stage through the solver's work vectors (p, v, s, t)
  Vecs &V = P->V;
  e = cudaMemcpyAsync(V.p, phi, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_gravity<<<grid, block, 0, s>>>(g, V.p, V.ghost, V.v, V.s, V.t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(gx, V.v, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gy, V.s, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gz, V.t, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? PHL_OK : pcuda(e, "gravity");
}

}  // extern "C"
