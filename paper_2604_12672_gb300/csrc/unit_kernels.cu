// unit_kernels.cu -- the stage's device functions exposed for unit testing.
#include <cuda_runtime.h>
#include <string.h>

#include "phl.h"
#include "phl_internal.cuh"
#include "riemann_x2.cuh"

using namespace phl;

namespace {

template <typename R>
__global__ void k_riemann_batch(long n, const double *wl, const double *wr, const double *bn, const double *bg,
                                int nspec, int solver, double mthr, double *f) {
  const int nw = 9 + nspec, nf = 7 + nspec;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    R a[9 + PHL_NSPEC_MAX], b[9 + PHL_NSPEC_MAX], out[7 + PHL_NSPEC_MAX];
    for (int q = 0; q < nw; ++q) { a[q] = (R)wl[t * nw + q]; b[q] = (R)wr[t * nw + q]; }
    int up;
    riemann_dev<R, PHL_NSPEC_MAX>(a, b, (R)bn[t], (R)bg[4 * t], (R)bg[4 * t + 1], (R)bg[4 * t + 2], (R)bg[4 * t + 3], nspec,
                   solver, (R)mthr, out, up);
    for (int q = 0; q < nf; ++q) f[t * nf + q] = (double)out[q];
  }
}

// Pairs of faces through the packed FP32x2 ideal-gas solver; gamma from the
// background's gamma_e column (bg[4t + 2]) of the pair's first face.
__global__ void k_riemann_batch_x2(long n, const double *wl, const double *wr, const double *bn, const double *bg,
                                   int solver, double mthr, double *f) {
  const long np = (n + 1) / 2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < np; t += (long)gridDim.x * blockDim.x) {
    const long a = 2 * t, b = (2 * t + 1 < n) ? 2 * t + 1 : 2 * t;
    x2::V l[9], r[9];
    for (int q = 0; q < 9; ++q) {
      l[q] = x2::vv((float)wl[a * 9 + q], (float)wl[b * 9 + q]);
      r[q] = x2::vv((float)wr[a * 9 + q], (float)wr[b * 9 + q]);
    }
    GasK<float> K;
    K.g = (float)bg[4 * a + 2];
    K.igm1 = 1.0f / (K.g - 1.0f);
    K.ggm1 = K.g * K.igm1;
    const x2::B2 hll{solver == SOLVER_HLL, solver == SOLVER_HLL};
    x2::V out[7];
    int ua, ub;
    x2::riemann_ideal_x2(l, r, x2::vv((float)bn[a], (float)bn[b]), x2::vv((float)bg[4 * a], (float)bg[4 * b]),
                         x2::vv((float)bg[4 * a + 1], (float)bg[4 * b + 1]), hll,
                         solver == SOLVER_HLL ? SOLVER_LHLLD : solver, (float)mthr, out, ua, ub, K);
    for (int q = 0; q < 7; ++q) {
      f[a * 7 + q] = (double)out[q].x;
      if (b != a) f[b * 7 + q] = (double)out[q].y;
    }
  }
}

// One face per thread through the left/right-paired ideal-gas solver.
__global__ void k_riemann_batch_lr(long n, const double *wl, const double *wr, const double *bn, const double *bg,
                                   int solver, double mthr, double *f) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    float l[9], r[9], out[7];
    for (int q = 0; q < 9; ++q) { l[q] = (float)wl[t * 9 + q]; r[q] = (float)wr[t * 9 + q]; }
    GasK<float> K;
    K.g = (float)bg[4 * t + 2];
    K.igm1 = 1.0f / (K.g - 1.0f);
    K.ggm1 = K.g * K.igm1;
    int up;
    x2::riemann_ideal_lr(l, r, (float)bn[t], (float)bg[4 * t], (float)bg[4 * t + 1], solver, (float)mthr, out, up, K);
    for (int q = 0; q < 7; ++q) f[t * 7 + q] = (double)out[q];
  }
}

__global__ void k_convert_batch(long n, const double *x, int k, float *f, double *back) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const float v = d2f_scaled(x[t], k);
    f[t] = v;
    back[t] = f2d_scaled(v, -k);
  }
}

}  // namespace

extern "C" phl_status phl_convert_batch(long n, const double *x, int k, float *f, double *back) {
  if (n < 0 || k <= -800 || k >= 800)
    return (phl_status)set_error(PHL_EINVAL, "phl_convert_batch: n < 0 or scale exponent out of range");
  if (n == 0) return PHL_OK;
  if (!x || !f || !back) return (phl_status)set_error(PHL_EINVAL, "phl_convert_batch: null argument");
  char *d = nullptr;
  if (cudaMalloc(&d, n * (2 * sizeof(double) + sizeof(float))) != cudaSuccess) { cudaGetLastError(); return PHL_ENOMEM; }
  double *dx = (double *)d, *db = dx + n;
  float *df = (float *)(db + n);
  cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice);
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_convert_batch<<<blocks, 256>>>(n, dx, k, df, db);
  cudaError_t e = cudaMemcpy(f, df, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(back, db, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) { cudaGetLastError(); return PHL_ECUDA; }
  return PHL_OK;
}

extern "C" phl_status phl_riemann_batch(long n, const double *wl, const double *wr, const double *bn,
                                        const double *bg, int nspec, int solver, double mach_thr,
                                        int precision, double *f) {
  if (n < 0 || nspec < 0 || nspec > PHL_MAXSPEC || solver < 0 || solver > 2)
    return (phl_status)set_error(PHL_EINVAL, "phl_riemann_batch: bad n, nspec or solver");
  if ((precision == 2 || precision == 3) && nspec != 0)
    return (phl_status)set_error(PHL_EINVAL, "phl_riemann_batch: the FP32 solvers take no species");
  if (n == 0) return PHL_OK;
  if (!wl || !wr || !bn || !bg || !f) return (phl_status)set_error(PHL_EINVAL, "phl_riemann_batch: null argument");
  const size_t nw = 9 + nspec, nf = 7 + nspec;
  double *d = nullptr;
  const size_t tot = n * (2 * nw + 1 + 4 + nf);
  if (cudaMalloc(&d, tot * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return PHL_ENOMEM; }
  double *dwl = d, *dwr = dwl + n * nw, *dbn = dwr + n * nw, *dbg = dbn + n, *df = dbg + 4 * n;
  cudaMemcpy(dwl, wl, n * nw * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dwr, wr, n * nw * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dbn, bn, n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dbg, bg, 4 * n * sizeof(double), cudaMemcpyHostToDevice);
  const int blocks = (int)((n + 127) / 128 < 4096 ? (n + 127) / 128 : 4096);
  if (precision == PHL_FP64)
    k_riemann_batch<double><<<blocks, 128>>>(n, dwl, dwr, dbn, dbg, nspec, solver, mach_thr, df);
  else if (precision == 2)
    k_riemann_batch_x2<<<blocks, 128>>>(n, dwl, dwr, dbn, dbg, solver, mach_thr, df);
  else if (precision == 3)
    k_riemann_batch_lr<<<blocks, 128>>>(n, dwl, dwr, dbn, dbg, solver, mach_thr, df);
  else
    k_riemann_batch<float><<<blocks, 128>>>(n, dwl, dwr, dbn, dbg, nspec, solver, mach_thr, df);
  cudaError_t e = cudaMemcpy(f, df, n * nf * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) { cudaGetLastError(); return PHL_ECUDA; }
  return PHL_OK;
}
