// dt_noalloc.cu -- CFL time step without any device allocation.
//
// Some callers cannot let a library call cudaMalloc/cudaFree: a host program
// whose own memory pool owns every byte of device memory, or a driver loop that
// must not pay the device-wide synchronisation those calls may imply.  For them
// this file provides a variant of the CFL reduction whose scratch (one partial
// maximum per thread block) lives in a file-scope __device__ array that exists
// on every GPU that loads the library, for as long as the process runs.
//
// The array is shared by every call: a call overwrites exactly the slots it
// later reads, so nothing has to start at zero, but two calls whose kernels
// overlap on the GPU (e.g. on two streams) race on it.
//
// A cell whose state has no sound speed (rho <= 0, P <= 0, or anything
// non-finite) contributes an infinite signal speed, so dt_out = 0 marks a bad
// state; the kernels keep no error word of their own.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <string.h>

#include "phl.h"
#include "phl_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr long NA_CELLS_PER_BLOCK = (long)NA_THREADS * NA_CELLS_PER_THREAD;   // 4096
constexpr int NA_MAX_BLOCKS = PHL_DT_NOALLOC_MAX_CELLS / NA_CELLS_PER_BLOCK;  // 16384

// One partial maximum of the CFL sum per block: 16384 doubles = 128 KiB.
static __device__ __align__(256) double g_dt_partial[NA_MAX_BLOCKS];

struct NaGeo {
  int n[3], act[3];
  double dx[3];
  double gamma, cfl;
};

__global__ void k_dt_partial(NaGeo G, long ncells, const double *__restrict__ cons,
                             const double *__restrict__ bx, const double *__restrict__ by,
                             const double *__restrict__ bz, double *__restrict__ partial) {
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  double m = 0.0;
  const long base = (long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int r = 0; r < NA_CELLS_PER_THREAD; ++r) {
    const long c = base + (long)r * NA_THREADS + threadIdx.x;
    if (c >= ncells) break;
    const int i = (int)(c % nx);
    const int j = (int)((c / nx) % ny);
    const int k = (int)(c / ((long)nx * ny));
    const double rho = cons[c];
    const double vx = cons[ncells + c] / rho, vy = cons[2 * ncells + c] / rho, vz = cons[3 * ncells + c] / rho;
    const double bcx = 0.5 * (bx[i + (long)(nx + 1) * (j + (long)ny * k)] + bx[i + 1 + (long)(nx + 1) * (j + (long)ny * k)]);
    const double bcy = 0.5 * (by[i + (long)nx * (j + (long)(ny + 1) * k)] + by[i + (long)nx * (j + 1 + (long)(ny + 1) * k)]);
    const double bcz = 0.5 * (bz[c] + bz[c + (long)nx * ny]);
    const double b2 = bcx * bcx + bcy * bcy + bcz * bcz;
    const double P = (G.gamma - 1.0) * (cons[4 * ncells + c] - 0.5 * rho * (vx * vx + vy * vy + vz * vz) - 0.5 * b2);
    if (!(rho > 0.0) || !(P > 0.0)) {   // no sound speed: the sentinel dt_out = 0
      m = INFINITY;
      continue;
    }
    const double a2 = G.gamma * P / rho;
    const double bb = b2 / rho;
    const double v[3] = {vx, vy, vz}, bc[3] = {bcx, bcy, bcz};
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const double bd2 = bc[d] * bc[d] / rho;
      double disc = (a2 + bb) * (a2 + bb) - 4.0 * a2 * bd2;
      if (disc < 0.0) disc = 0.0;
      s += (fabs(v[d]) + sqrt(0.5 * (a2 + bb + sqrt(disc)))) / G.dx[d];
    }
    m = (s == s) ? fmax(m, s) : INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < NA_THREADS / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

__global__ void k_dt_final(const double *__restrict__ partial, int nblocks, double cfl, double *dt_out) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) m = fmax(m, partial[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) v = fmax(v, red[w]);
    dt_out[0] = cfl / v;
  }
}

// Device address of g_dt_partial, looked up once per device and context: the
// module holding the array is loaded into each context, so after a device
// reset, or under another (non-primary) context, the array lives at another
// address and the lookup is redone.  The current context comes from the
// driver's cuCtxGetCurrent, fetched through the runtime's entry-point query.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};
void *g_na_ctx[NA_MAX_DEVICES] = {nullptr};
typedef int (*ctx_get_fn)(void **);
ctx_get_fn g_ctx_get = nullptr;

cudaError_t partial_ptr(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_ctx_get) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_ctx_get = (ctx_get_fn)fn;
  }
  void *ctx = nullptr;
  if (g_ctx_get(&ctx) != 0) return cudaErrorDeviceUninitialized;
  if (!g_na_ptr[dev] || ctx != g_na_ctx[dev] || !ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dt_partial);   // also makes the primary context current if none was
    if (e != cudaSuccess) return e;
    if (!ctx && g_ctx_get(&ctx) != 0) return cudaErrorDeviceUninitialized;
    g_na_ptr[dev] = (double *)p;
    g_na_ctx[dev] = ctx;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// True when p is memory the current device's kernels may read as device
// memory (a device or managed allocation).
bool device_accessible(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" phl_status phl_cfl_dt_noalloc(const phl_grid_desc *desc, const double *cons, const double *bx,
                                         const double *by, const double *bz, double *dt_out, void *stream) {
  using phl::set_error;
  if (!desc || !cons || !bx || !by || !bz || !dt_out)
    return (phl_status)set_error(PHL_EINVAL, "phl_cfl_dt_noalloc: null argument");
  if (desc->eos != PHL_EOS_IDEAL)
    return (phl_status)set_error(PHL_EUNSUPPORTED, "phl_cfl_dt_noalloc: ideal-gas EOS only");
  if (!(desc->gamma > 1.0) || !(desc->cfl > 0.0))
    return (phl_status)set_error(PHL_EINVAL, "phl_cfl_dt_noalloc: gamma must exceed 1 and cfl be positive");
  NaGeo G;
  long ncells = 1;
  for (int d = 0; d < 3; ++d) {
    if (desc->n[d] < 1 || !(desc->hi[d] > desc->lo[d]))
      return (phl_status)set_error(PHL_EINVAL, "phl_cfl_dt_noalloc: bad extent in dimension %d", d);
    G.n[d] = desc->n[d];
    G.act[d] = desc->n[d] > 1;
    G.dx[d] = (desc->hi[d] - desc->lo[d]) / desc->n[d];
    // checked after each factor: every factor and partial product stays at
    // or below the maximum, so the product cannot overflow
    if (desc->n[d] > PHL_DT_NOALLOC_MAX_CELLS || ncells * desc->n[d] > PHL_DT_NOALLOC_MAX_CELLS)
      return (phl_status)set_error(PHL_EINVAL, "phl_cfl_dt_noalloc: too many cells (more than the maximum %ld)",
                                   (long)PHL_DT_NOALLOC_MAX_CELLS);
    ncells *= desc->n[d];
  }
  const void *ptrs[5] = {cons, bx, by, bz, dt_out};
  static const char *names[5] = {"cons", "bx", "by", "bz", "dt_out"};
  for (int q = 0; q < 5; ++q)
    if (!device_accessible(ptrs[q]))
      return (phl_status)set_error(PHL_EINVAL, "phl_cfl_dt_noalloc: %s is not device memory", names[q]);
  G.gamma = desc->gamma;
  G.cfl = desc->cfl;
  double *partial = nullptr;
  cudaError_t e = partial_ptr(&partial);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return (phl_status)set_error(PHL_ECUDA, "phl_cfl_dt_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  }
  const int nblocks = (int)((ncells + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  cudaStream_t s = (cudaStream_t)stream;
  k_dt_partial<<<nblocks, NA_THREADS, 0, s>>>(G, ncells, cons, bx, by, bz, partial);
  k_dt_final<<<1, NA_THREADS, 0, s>>>(partial, nblocks, desc->cfl, dt_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_cfl_dt_noalloc: launch: %s", cudaGetErrorString(e));
  return PHL_OK;
}
