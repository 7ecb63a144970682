// eos.cu -- the stellar EOS table, built on the device from Fermi-Dirac
// integrals, and the batch EOS entry point phl_eos.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "eos_nodes.cuh"
#include "eos_stellar.cuh"
#include "phl.h"
#include "phl_internal.cuh"

using namespace phl;
using namespace phl::eos;

struct phl_eos_table {
  Table t;
  double *dv = nullptr;
  float *dvf = nullptr;
  double *dd = nullptr;   // per table cell: the corner values in difference form (Table::d)
};

namespace {

using eosn::GLN;

// Gauss-Legendre nodes/weights on [-1, 1]: Newton on the Legendre recurrence.
void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(PI_D * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// One table node per thread: the free energy and its eight derivatives
// (eos_nodes.cuh); gl holds the quadrature nodes then weights.
__global__ void k_table_nodes(int nx, int ny, double x0, double dx, double y0, double dy, double lam3,
                              const double *gl, double *v, int *fail) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nx * ny) return;
  const int i = idx % nx, j = idx / nx;
  if (!eosn::node_values(exp(x0 + i * dx), exp(y0 + j * dy), lam3, gl, gl + GLN, v + (long)NQ * idx))
    atomicOr(fail, 1);
}

// Per table cell (i, j) and node slot s: q00 and the differences q10 - q00,
// q01 - q00, (q11 - q01) - (q10 - q00) of its corners (x first, then y),
// the same FP64 operations the contraction would do at every evaluation.
__global__ void k_table_diffs(int nx, int ny, double dx, double dy, const double *__restrict__ v,
                              double *__restrict__ d) {
  const long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (q >= (long)(nx - 1) * (ny - 1) * NQ) return;
  const int s = (int)(q % NQ);
  const long cell = q / NQ;
  const int i = (int)(cell % (nx - 1)), j = (int)(cell / (nx - 1));
  const long k0 = ((long)j * nx + i) * NQ + s, k1 = k0 + (long)nx * NQ;
  const double q00 = v[k0], q10 = v[k0 + NQ], q01 = v[k1], q11 = v[k1 + NQ];
  // the slot's derivative orders (p in x, r in y; slot = qslot(p, r)): in
  // units of the cell, times dx^p dy^r
  const int p = (s == 1 || s == 5 || s == 7) ? 1 : ((s == 3 || s == 6 || s == 8) ? 2 : 0);
  const int r = (s == 2 || s == 5 || s == 6) ? 1 : ((s == 4 || s == 7 || s == 8) ? 2 : 0);
  const double sc = (p == 0 ? 1.0 : (p == 1 ? dx : dx * dx)) * (r == 0 ? 1.0 : (r == 1 ? dy : dy * dy));
  double *o = d + cell * 4 * NQ + 4 * s;
  o[0] = q00 * sc;
  o[1] = (q10 - q00) * sc;
  o[2] = (q01 - q00) * sc;
  o[3] = ((q11 - q01) - (q10 - q00)) * sc;
}

template <typename R>
__global__ void k_eos_batch(Table t, long n, const double *rho, const double *eint, const double *abar,
                            const double *ye, double *T, double *P, double *ge, double *gc, double *cs, int *iters,
                            double tol, int maxit) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  EosOut<double> o;
  double Td = T[i];
  int it;
  if (sizeof(R) == 8) it = eos_invert<double>(t, rho[i], eint[i], abar[i], ye[i], Td, tol, maxit, o);
  else it = eos_invert_mixed(t, rho[i], eint[i], abar[i], ye[i], Td, tol, maxit, o);
  const bool ok = it > 0;
  T[i] = Td;
  if (P) P[i] = ok ? o.P : NAN;
  if (ge) ge[i] = o.ge;
  if (gc) gc[i] = o.gc;
  if (cs) cs[i] = sqrt(o.gc * o.P / rho[i]);
  if (iters) iters[i] = ok ? it : -1;
}

}  // namespace

namespace phl {
// Table view for the stage kernels (phl_api.cu)
const Table *eos_table_view(const phl_eos_table *t) { return t ? &t->t : nullptr; }
}  // namespace phl

extern "C" {

phl_status phl_eos_table_create(double lrhoye_lo, double lrhoye_hi, int nrho, double lT_lo, double lT_hi, int nT,
                                phl_eos_table **out) {
  if (!out || nrho < 4 || nT < 4 || !(lrhoye_hi > lrhoye_lo) || !(lT_hi > lT_lo))
    return (phl_status)set_error(PHL_EINVAL, "phl_eos_table_create: bad arguments");
  *out = nullptr;
  double gxw[2 * GLN];
  gauss_legendre(GLN, gxw, gxw + GLN);
  cudaError_t e = cudaSuccess;
  phl_eos_table *t = new phl_eos_table();
  t->t.nx = nrho;
  t->t.ny = nT;
  t->t.x0 = log(pow(10.0, lrhoye_lo) * NAV);
  t->t.dx = (lrhoye_hi - lrhoye_lo) * log(10.0) / (nrho - 1);
  t->t.y0 = lT_lo * log(10.0);
  t->t.dy = (lT_hi - lT_lo) * log(10.0) / (nT - 1);
  t->t.x0f = (float)t->t.x0; t->t.dxf = (float)t->t.dx; t->t.y0f = (float)t->t.y0; t->t.dyf = (float)t->t.dy;
  t->t.idx = 1.0 / t->t.dx; t->t.idy = 1.0 / t->t.dy;
  t->t.idx2 = t->t.idx * t->t.idx; t->t.idy2 = t->t.idy * t->t.idy; t->t.idxdy = t->t.idx * t->t.idy;
  t->t.idxf = (float)t->t.idx; t->t.idyf = (float)t->t.idy;
  t->t.Tlo = exp(t->t.y0); t->t.Thi = exp(t->t.y0 + (nT - 1) * t->t.dy);
  t->t.Tlof = (float)t->t.Tlo; t->t.Thif = (float)t->t.Thi;
  const long nv = (long)NQ * nrho * nT;
  int *fail = nullptr;
  double *dgl = nullptr;
  e = cudaMalloc(&t->dv, nv * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&t->dvf, nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&fail, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&dgl, sizeof(gxw));
  if (e == cudaSuccess) e = cudaMemset(fail, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dgl, gxw, sizeof(gxw), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(t->dv); cudaFree(t->dvf); cudaFree(fail); cudaFree(dgl); delete t;
    return (phl_status)set_error(PHL_ENOMEM, "eos table: %s", cudaGetErrorString(e));
  }
  const double me = MEC2 / (CL * CL), l = me * CL / HPL;
  const int nn = nrho * nT;
  k_table_nodes<<<(nn + 63) / 64, 64>>>(nrho, nT, t->t.x0, t->t.dx, t->t.y0, t->t.dy, l * l * l, dgl, t->dv, fail);
  std::vector<double> h(nv);
  int f = 0;
  e = cudaMemcpy(h.data(), t->dv, nv * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(fail);
  cudaFree(dgl);
  if (e != cudaSuccess || f) {
    cudaFree(t->dv); cudaFree(t->dvf); delete t;
    return (phl_status)set_error(e != cudaSuccess ? PHL_ECUDA : PHL_ENEWTON, "eos table: node solve failed");
  }
  std::vector<float> hf(nv);
  for (long q = 0; q < nv; ++q) hf[q] = (float)h[q];
  cudaMemcpy(t->dvf, hf.data(), nv * sizeof(float), cudaMemcpyHostToDevice);
  const long nd = 4L * NQ * (nrho - 1) * (nT - 1);
  e = cudaMalloc(&t->dd, nd * sizeof(double));
  if (e == cudaSuccess) {
    k_table_diffs<<<(unsigned)((nd / 4 + 255) / 256), 256>>>(nrho, nT, t->t.dx, t->t.dy, t->dv, t->dd);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    cudaFree(t->dv); cudaFree(t->dvf); cudaFree(t->dd); delete t;
    return (phl_status)set_error(PHL_ECUDA, "eos table: %s", cudaGetErrorString(e));
  }
  t->t.v = t->dv;
  t->t.vf = t->dvf;
  t->t.d = t->dd;
  *out = t;
  return PHL_OK;
}

void phl_eos_table_destroy(phl_eos_table *t) {
  if (!t) return;
  cudaFree(t->dv);
  cudaFree(t->dvf);
  cudaFree(t->dd);
  delete t;
}

phl_status phl_eos_table_export(const phl_eos_table *t, double *out, long nout) {
  if (!t || !out) return (phl_status)set_error(PHL_EINVAL, "null argument");
  const long nv = (long)NQ * t->t.nx * t->t.ny;
  if (nout < 6 + nv) return (phl_status)set_error(PHL_EINVAL, "phl_eos_table_export: buffer too small");
  out[0] = t->t.nx; out[1] = t->t.ny; out[2] = t->t.x0; out[3] = t->t.dx; out[4] = t->t.y0; out[5] = t->t.dy;
  if (cudaMemcpy(out + 6, t->dv, nv * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return (phl_status)set_error(PHL_ECUDA, "phl_eos_table_export: copy failed");
  return PHL_OK;
}

phl_status phl_eos(const phl_eos_table *t, long n, const double *rho, const double *eint, const double *abar,
                   const double *ye, double *T_inout, double *P, double *gamma_e, double *gamma_c, double *cs,
                   int *iters, int precision, double tol, int maxit, int where, void *stream) {
  if (!t || n < 0 || !rho || !eint || !abar || !ye || !T_inout)
    return (phl_status)set_error(PHL_EINVAL, "phl_eos: null argument");
  if (n == 0) return PHL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double *drho = rho, *dein = eint, *dab = abar, *dye = ye;
  double *dT = T_inout, *dP = P, *dge = gamma_e, *dgc = gamma_c, *dcs = cs;
  int *dit = iters;
  void *buf = nullptr;
  if (where == PHL_HOST) {   // stage through one device buffer
    const size_t nb = (size_t)n * (9 * sizeof(double) + sizeof(int));
    if (cudaMalloc(&buf, nb) != cudaSuccess) { cudaGetLastError(); return (phl_status)set_error(PHL_ENOMEM, "phl_eos: alloc"); }
    double *b = (double *)buf;
    double *a[9];
    for (int k = 0; k < 9; ++k) a[k] = b + (size_t)k * n;
    cudaMemcpyAsync(a[0], rho, n * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a[1], eint, n * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a[2], abar, n * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a[3], ye, n * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(a[4], T_inout, n * 8, cudaMemcpyHostToDevice, s);
    drho = a[0]; dein = a[1]; dab = a[2]; dye = a[3]; dT = a[4];
    dP = a[5]; dge = a[6]; dgc = a[7]; dcs = a[8];
    dit = (int *)(b + (size_t)9 * n);
  }
  const int blocks = (int)((n + 127) / 128);
  if (precision == PHL_FP64)
    k_eos_batch<double><<<blocks, 128, 0, s>>>(t->t, n, drho, dein, dab, dye, dT, dP, dge, dgc, dcs, dit, tol, maxit);
  else
    k_eos_batch<float><<<blocks, 128, 0, s>>>(t->t, n, drho, dein, dab, dye, dT, dP, dge, dgc, dcs, dit, tol, maxit);
  cudaError_t e = cudaGetLastError();
  if (where == PHL_HOST) {
    if (e == cudaSuccess) {
      cudaMemcpyAsync(T_inout, dT, n * 8, cudaMemcpyDeviceToHost, s);
      if (P) cudaMemcpyAsync(P, dP, n * 8, cudaMemcpyDeviceToHost, s);
      if (gamma_e) cudaMemcpyAsync(gamma_e, dge, n * 8, cudaMemcpyDeviceToHost, s);
      if (gamma_c) cudaMemcpyAsync(gamma_c, dgc, n * 8, cudaMemcpyDeviceToHost, s);
      if (cs) cudaMemcpyAsync(cs, dcs, n * 8, cudaMemcpyDeviceToHost, s);
      if (iters) cudaMemcpyAsync(iters, dit, n * sizeof(int), cudaMemcpyDeviceToHost, s);
      e = cudaStreamSynchronize(s);
    }
    cudaFree(buf);
  }
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_eos: %s", cudaGetErrorString(e));
  return PHL_OK;
}

}  // extern "C"
