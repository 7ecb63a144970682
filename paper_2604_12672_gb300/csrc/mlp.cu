// mlp.cu -- the temperature-guess network: FP32 training kernels (forward,
// backward, weight-gradient reduction, Adam) on EOS samples generated on the
// device, and BF16 tensor-core inference (mlp_dev.cuh).
//
// Training data: (log10 rho, log10 T, X_0) drawn uniformly in the stated
// ranges by a counter-based generator (SplitMix64, Steele, Lea & Flood 2014),
// e_int from the device EOS (eos_rt), inputs (log10 rho, log10 e_int, X_0),
// target log10 T, all mapped affinely onto [-1, 1].  Loss: mean squared error
// of the mapped target.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "eos_stellar.cuh"
#include "mlp_dev.cuh"
#include "phl.h"
#include "phl_internal.cuh"

using namespace phl::mlp;

struct phl_mlp {
  float *w = nullptr;       // FP32 master weights (NPARAM), device
  float *m = nullptr, *v = nullptr;   // Adam moments
  float *grad = nullptr;    // NPARAM
  uint2 *frag = nullptr;    // BF16 fragments (F_TOTAL)
  float *bias = nullptr;    // b1, b2 copies for inference (2 NH)
  float b3 = 0.0f;
  float c[4] = {6.0f, 18.0f, 0.5f, 8.75f}, s[4] = {1.0f, 1.0f, 2.0f, 1.0f};
  long adam_t = 0;
};

namespace phl {
namespace {

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t i, int comp) {
  const uint64_t z = splitmix64(seed ^ splitmix64(3 * i + comp));
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// EOS samples: x[3 n] (raw log10 rho, log10 e, X_0), t[n] raw log10 T.
__global__ void k_samples(eos::Table tab, long n, uint64_t seed, double lr0, double lr1, double lt0, double lt1,
                          double A0, double Z0, double A1, double Z1, float *x, float *t, int *fail) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lr = lr0 + (lr1 - lr0) * uniform01(seed, i, 0);
  const double lt = lt0 + (lt1 - lt0) * uniform01(seed, i, 1);
  const double X0 = uniform01(seed, i, 2);
  const double rho = pow(10.0, lr), T = pow(10.0, lt);
  const double sa = X0 / A0 + (1.0 - X0) / A1;
  const double abar = 1.0 / sa, ye = X0 * Z0 / A0 + (1.0 - X0) * Z1 / A1;
  eos::EosOut<double> o;
  if (!eos::eos_rt<double>(tab, rho, T, abar, ye, o) || !(o.e > 0.0)) {
    atomicOr(fail, 1);
    x[3 * i] = x[3 * i + 1] = x[3 * i + 2] = 0.0f;
    t[i] = 0.0f;
    return;
  }
  x[3 * i] = (float)lr;
  x[3 * i + 1] = (float)log10(o.e);
  x[3 * i + 2] = (float)X0;
  t[i] = (float)lt;
}

// Apply the affine maps in place: x <- (x - c) s, t <- (t - c3) s3.
__global__ void k_normalise(long n, float *x, float *t, float4 c, float4 s) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[3 * i] = (x[3 * i] - c.x) * s.x;
  x[3 * i + 1] = (x[3 * i + 1] - c.y) * s.y;
  x[3 * i + 2] = (x[3 * i + 2] - c.z) * s.z;
  t[i] = (t[i] - c.w) * s.w;
}

// min / max of column 1 (log10 e) over the samples (positive floats order like
// their bit patterns)
__global__ void k_minmax_e(long n, const float *x, unsigned int *mn, unsigned int *mx) {
  unsigned int lo = 0x7f7fffffu, hi = 0u;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned int b = __float_as_uint(x[3 * i + 1]);
    lo = min(lo, b);
    hi = max(hi, b);
  }
  atomicMin(mn, lo);
  atomicMax(mx, hi);
}

// Forward + backward of one sample per thread in FP32 (weights in shared
// memory, rounded to BF16 as in inference: straight-through gradient).  Writes per-sample activations and back-propagated errors in
// feature-major layout [NH][nb] for the weight-gradient reduction.
constexpr int FB_THREADS = 128;
__global__ void __launch_bounds__(FB_THREADS) k_fwd_bwd(const float *__restrict__ w, long nb,
                                                        const float *__restrict__ x, const float *__restrict__ t,
                                                        float inv_n, float *H1, float *H2, float *D1, float *D2,
                                                        float *dy_out, double *loss) {
  // the weight matrices as the inference sees them (rounded to BF16), the
  // biases in FP32; the gradient updates the FP32 master weights
  __shared__ float sw[NPARAM];
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) {
    const bool is_w = k < O_B1 || (k >= O_W2 && k < O_B2) || (k >= O_W3 && k < O_B3);
    sw[k] = is_w ? __bfloat162float(__float2bfloat16_rn(w[k])) : w[k];
  }
  __syncthreads();
  const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float r2 = 0.0f;
  if (s < nb) {
    const float x0 = x[3 * s], x1 = x[3 * s + 1], x2 = x[3 * s + 2];
    float h1[NH];
#pragma unroll
    for (int a = 0; a < NH; ++a) {
      const float z = sw[O_B1 + a] + sw[O_W1 + 3 * a] * x0 + sw[O_W1 + 3 * a + 1] * x1 + sw[O_W1 + 3 * a + 2] * x2;
      h1[a] = tanhf(z);
      H1[(long)a * nb + s] = h1[a];
    }
    float y = sw[O_B3];
    for (int a = 0; a < NH; ++a) {
      float z = sw[O_B2 + a];
#pragma unroll
      for (int b = 0; b < NH; ++b) z += sw[O_W2 + a * NH + b] * h1[b];
      const float h2 = tanhf(z);
      H2[(long)a * nb + s] = h2;
      y += sw[O_W3 + a] * h2;
    }
    const float r = y - t[s];
    r2 = r * r;
    const float dy = 2.0f * r * inv_n;
    dy_out[s] = dy;
    float d1[NH];
#pragma unroll
    for (int b = 0; b < NH; ++b) d1[b] = 0.0f;
    for (int a = 0; a < NH; ++a) {
      const float h2 = H2[(long)a * nb + s];
      const float d2 = dy * sw[O_W3 + a] * (1.0f - h2 * h2);
      D2[(long)a * nb + s] = d2;
#pragma unroll
      for (int b = 0; b < NH; ++b) d1[b] += sw[O_W2 + a * NH + b] * d2;
    }
#pragma unroll
    for (int b = 0; b < NH; ++b) D1[(long)b * nb + s] = d1[b] * (1.0f - h1[b] * h1[b]);
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)r2);
}

// Weight gradients: sums over the samples of a chunk, one 4x4 block of dW2 per
// thread (256 threads = 64 x 64), plus the bias, W1 and W3 sums; partial sums
// are added to grad with atomics.
constexpr int RED_CHUNK = 32;
__global__ void __launch_bounds__(256) k_grad_reduce(long nb, const float *__restrict__ x, const float *H1,
                                                     const float *H2, const float *D1, const float *D2,
                                                     const float *dy, float *grad) {
  __shared__ float sH1[RED_CHUNK][NH + 4], sD2[RED_CHUNK][NH + 4];
  __shared__ float sH2[RED_CHUNK][NH + 1], sD1[RED_CHUNK][NH + 1];
  __shared__ float sx[RED_CHUNK][3], sdy[RED_CHUNK];
  const int tid = threadIdx.x;
  const int tj = tid >> 4, tk = tid & 15;   // dW2 rows 4 tj.., cols 4 tk..
  float acc[4][4] = {};
  float accb1 = 0.f, accb2 = 0.f, accw3 = 0.f, accw1[3] = {0.f, 0.f, 0.f}, accb3 = 0.f;
  for (long s0 = (long)blockIdx.x * RED_CHUNK; s0 < nb; s0 += (long)gridDim.x * RED_CHUNK) {
    const int cnt = (int)min((long)RED_CHUNK, nb - s0);
    __syncthreads();
    for (int e = tid; e < RED_CHUNK * NH; e += blockDim.x) {
      const int a = e / RED_CHUNK, ss = e % RED_CHUNK;
      const bool in = ss < cnt;
      const long gi = (long)a * nb + s0 + ss;
      sH1[ss][a] = in ? H1[gi] : 0.f;
      sD2[ss][a] = in ? D2[gi] : 0.f;
      sH2[ss][a] = in ? H2[gi] : 0.f;
      sD1[ss][a] = in ? D1[gi] : 0.f;
    }
    for (int e = tid; e < RED_CHUNK; e += blockDim.x) {
      const bool in = e < cnt;
      sdy[e] = in ? dy[s0 + e] : 0.f;
      for (int c = 0; c < 3; ++c) sx[e][c] = in ? x[3 * (s0 + e) + c] : 0.f;
    }
    __syncthreads();
    for (int ss = 0; ss < RED_CHUNK; ++ss) {
      float dv[4], hv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { dv[i] = sD2[ss][4 * tj + i]; hv[i] = sH1[ss][4 * tk + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += dv[i] * hv[j];
    }
    if (tid < NH) {
      for (int ss = 0; ss < RED_CHUNK; ++ss) {
        const float d1 = sD1[ss][tid];
        accb1 += d1;
        for (int c = 0; c < 3; ++c) accw1[c] += d1 * sx[ss][c];
        accb2 += sD2[ss][tid];
        accw3 += sdy[ss] * sH2[ss][tid];
      }
    } else if (tid == NH) {
      for (int ss = 0; ss < RED_CHUNK; ++ss) accb3 += sdy[ss];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(&grad[O_W2 + (4 * tj + i) * NH + 4 * tk + j], acc[i][j]);
  if (tid < NH) {
    atomicAdd(&grad[O_B1 + tid], accb1);
    for (int c = 0; c < 3; ++c) atomicAdd(&grad[O_W1 + 3 * tid + c], accw1[c]);
    atomicAdd(&grad[O_B2 + tid], accb2);
    atomicAdd(&grad[O_W3 + tid], accw3);
  } else if (tid == NH) {
    atomicAdd(&grad[O_B3], accb3);
  }
}

__global__ void k_adam(int n, float *w, float *m, float *v, const float *g, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 tensor-core inference over n samples of normalised inputs (x[3 n]).
__global__ void k_infer(phl::mlp::Dev M, long n, const float *__restrict__ x, float *__restrict__ y) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const bool in = i < n;
  const float xin[3] = {in ? x[3 * i] : 0.f, in ? x[3 * i + 1] : 0.f, in ? x[3 * i + 2] : 0.f};
  const int lane = threadIdx.x & 31;
  const float ylo = tile_forward(M, xin, 0);
  const float yhi = tile_forward(M, xin, 16);
  if (in) y[i] = lane < 16 ? ylo : yhi;
}

// Temperature guesses for the batch EOS: T = 10^(network output).
__global__ void k_guess(phl::mlp::Dev M, long n, const double *rho, const double *eint, const double *X0,
                        double Tlo, double Thi, double *T) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const bool in = i < n;
  const float lr = in ? (float)log10(rho[i]) : M.c[0];
  const float le = in ? (float)log10(fmax(eint[i], 1e-300)) : M.c[1];
  const float xx = in ? (float)X0[i] : M.c[2];
  const float lt = guess_log10T(M, lr, le, xx);
  if (in) T[i] = fmin(fmax(exp10((double)lt), Tlo), Thi);
}

phl_status cuda_status(cudaError_t e, const char *what) {
  return (phl_status)set_error(PHL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// BF16 fragments and bias copies from the FP32 master weights.
cudaError_t build_fragments(phl_mlp *M) {
  std::vector<float> w(NPARAM);
  cudaError_t e = cudaMemcpy(w.data(), M->w, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  auto bf = [](float f) -> uint32_t {   // round to nearest even
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u >> 16;
    u += 0x7fffu + ((u >> 16) & 1u);
    return u >> 16;
  };
  auto B = [&](int layer, int k, int n) -> float {   // B[k][n] = W[n][k]
    if (layer == 1) return (k < NIN) ? w[O_W1 + n * NIN + k] : 0.0f;
    if (layer == 2) return w[O_W2 + n * NH + k];
    return n == 0 ? w[O_W3 + k] : 0.0f;
  };
  std::vector<uint2> f(F_TOTAL);
  auto fill = [&](int layer, int off, int KT, int NT) {
    for (int kt = 0; kt < KT; ++kt)
      for (int nt = 0; nt < NT; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane >> 2, q = lane & 3, n = 8 * nt + g, k = 16 * kt + 2 * q;
          uint2 u;
          u.x = bf(B(layer, k, n)) | (bf(B(layer, k + 1, n)) << 16);
          u.y = bf(B(layer, k + 8, n)) | (bf(B(layer, k + 9, n)) << 16);
          f[off + (kt * NT + nt) * 32 + lane] = u;
        }
  };
  fill(1, F_L1, 1, 8);
  fill(2, F_L2, 4, 8);
  fill(3, F_L3, 4, 1);
  e = cudaMemcpy(M->frag, f.data(), F_TOTAL * sizeof(uint2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  std::vector<float> b(2 * NH);
  for (int a = 0; a < NH; ++a) { b[a] = w[O_B1 + a]; b[NH + a] = w[O_B2 + a]; }
  e = cudaMemcpy(M->bias, b.data(), 2 * NH * sizeof(float), cudaMemcpyHostToDevice);
  M->b3 = w[O_B3];
  return e;
}

// Scratch of one training batch (feature-major activations and errors).
struct Scratch {
  float *H1 = nullptr, *H2 = nullptr, *D1 = nullptr, *D2 = nullptr, *dy = nullptr;
  double *loss = nullptr;
  long cap = 0;
  cudaError_t alloc(long nb) {
    cap = nb;
    float *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (4 * NH + 1) * nb * sizeof(float));
    if (e != cudaSuccess) return e;
    H1 = p; H2 = p + NH * nb; D1 = p + 2 * NH * nb; D2 = p + 3 * NH * nb; dy = p + 4 * NH * nb;
    return cudaMalloc(&loss, sizeof(double));
  }
  ~Scratch() { cudaFree(H1); cudaFree(loss); }
};

// grad <- d loss / d w over nb samples (normalised x, t on the device); loss
// (device double) receives the sum of squared residuals.
void launch_loss_grad(phl_mlp *M, long nb, const float *x, const float *t, Scratch &S, cudaStream_t s) {
  cudaMemsetAsync(M->grad, 0, NPARAM * sizeof(float), s);
  cudaMemsetAsync(S.loss, 0, sizeof(double), s);
  k_fwd_bwd<<<(unsigned)((nb + FB_THREADS - 1) / FB_THREADS), FB_THREADS, 0, s>>>(
      M->w, nb, x, t, 1.0f / (float)nb, S.H1, S.H2, S.D1, S.D2, S.dy, S.loss);
  const long chunks = (nb + RED_CHUNK - 1) / RED_CHUNK;
  const unsigned grid = (unsigned)std::min<long>(chunks, 4 * 152);
  k_grad_reduce<<<grid, 256, 0, s>>>(nb, x, S.H1, S.H2, S.D1, S.D2, S.dy, M->grad);
}

}  // namespace

mlp::Dev mlp_view(const phl_mlp *M) {
  mlp::Dev d;
  d.frag = M->frag;
  d.b1 = M->bias;
  d.b2 = M->bias + NH;
  d.b3 = M->b3;
  for (int k = 0; k < 4; ++k) { d.c[k] = M->c[k]; d.s[k] = M->s[k]; }
  return d;
}

}  // namespace phl

using namespace phl;

extern "C" {

phl_status phl_mlp_create(unsigned long long seed, phl_mlp **out) {
  if (!out) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_create: null out");
  *out = nullptr;
  phl_mlp *M = new phl_mlp();
  cudaError_t e = cudaMalloc(&M->w, 4 * NPARAM * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&M->frag, F_TOTAL * sizeof(uint2));
  if (e == cudaSuccess) e = cudaMalloc(&M->bias, 2 * NH * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(M->w); cudaFree(M->frag); cudaFree(M->bias); delete M;
    return (phl_status)set_error(PHL_ENOMEM, "phl_mlp_create: %s", cudaGetErrorString(e));
  }
  M->m = M->w + NPARAM;
  M->v = M->w + 2 * NPARAM;
  M->grad = M->w + 3 * NPARAM;
  // Glorot-uniform initial weights from SplitMix64, zero biases
  std::vector<float> w(NPARAM, 0.0f);
  auto u = [&](long i) { return (double)(splitmix64(seed ^ splitmix64((uint64_t)i)) >> 11) / 9007199254740992.0; };
  const double l1 = sqrt(6.0 / (NIN + NH)), l2 = sqrt(6.0 / (2 * NH)), l3 = sqrt(6.0 / (NH + 1));
  for (int i = 0; i < NH * NIN; ++i) w[O_W1 + i] = (float)(l1 * (2 * u(i) - 1));
  for (int i = 0; i < NH * NH; ++i) w[O_W2 + i] = (float)(l2 * (2 * u(10000 + i) - 1));
  for (int i = 0; i < NH; ++i) w[O_W3 + i] = (float)(l3 * (2 * u(20000 + i) - 1));
  e = cudaMemcpy(M->w, w.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, 2 * NPARAM * sizeof(float));
  if (e == cudaSuccess) e = build_fragments(M);
  if (e != cudaSuccess) {
    phl_mlp_destroy(M);
    return cuda_status(e, "phl_mlp_create");
  }
  *out = M;
  return PHL_OK;
}

void phl_mlp_destroy(phl_mlp *M) {
  if (!M) return;
  cudaFree(M->w);
  cudaFree(M->frag);
  cudaFree(M->bias);
  delete M;
}

phl_status phl_mlp_set_weights(phl_mlp *M, const float *w) {
  if (!M || !w) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_set_weights: null argument");
  cudaError_t e = cudaMemcpy(M->w, w, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, 2 * NPARAM * sizeof(float));
  M->adam_t = 0;
  if (e == cudaSuccess) e = build_fragments(M);
  return e == cudaSuccess ? PHL_OK : cuda_status(e, "phl_mlp_set_weights");
}

phl_status phl_mlp_get_weights(const phl_mlp *M, float *w) {
  if (!M || !w) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_get_weights: null argument");
  cudaError_t e = cudaMemcpy(w, M->w, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? PHL_OK : cuda_status(e, "phl_mlp_get_weights");
}

phl_status phl_mlp_set_norm(phl_mlp *M, const double *c, const double *s) {
  if (!M || !c || !s) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_set_norm: null argument");
  for (int k = 0; k < 4; ++k) {
    if (!(s[k] != 0.0) || !isfinite(c[k]) || !isfinite(s[k]))
      return (phl_status)set_error(PHL_EINVAL, "phl_mlp_set_norm: bad map");
    M->c[k] = (float)c[k];
    M->s[k] = (float)s[k];
  }
  return PHL_OK;
}

phl_status phl_mlp_get_norm(const phl_mlp *M, double *c, double *s) {
  if (!M || !c || !s) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_get_norm: null argument");
  for (int k = 0; k < 4; ++k) { c[k] = M->c[k]; s[k] = M->s[k]; }
  return PHL_OK;
}

phl_status phl_mlp_loss_grad(phl_mlp *M, long n, const float *x, const float *t, double *loss, float *grad,
                             int where) {
  if (!M || n <= 0 || !x || !t || !loss || !grad)
    return (phl_status)set_error(PHL_EINVAL, "phl_mlp_loss_grad: bad arguments");
  const float *dx = x, *dt = t;
  float *tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (where == PHL_HOST) {
    e = cudaMalloc(&tmp, 4 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(tmp, x, 3 * n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tmp + 3 * n, t, n * sizeof(float), cudaMemcpyHostToDevice);
    dx = tmp;
    dt = tmp + 3 * n;
  }
  Scratch S;
  if (e == cudaSuccess) e = S.alloc(n);
  if (e == cudaSuccess) {
    launch_loss_grad(M, n, dx, dt, S, 0);
    e = cudaGetLastError();
  }
  double l = 0.0;
  if (e == cudaSuccess) e = cudaMemcpy(&l, S.loss, sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(grad, M->grad, NPARAM * sizeof(float),
                   where == PHL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_status(e, "phl_mlp_loss_grad");
  *loss = l / (double)n;
  return PHL_OK;
}

phl_status phl_mlp_forward(const phl_mlp *M, long n, const float *x, float *y, int where) {
  if (!M || n <= 0 || !x || !y) return (phl_status)set_error(PHL_EINVAL, "phl_mlp_forward: bad arguments");
  const float *dx = x;
  float *dy = y, *tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (where == PHL_HOST) {
    e = cudaMalloc(&tmp, 4 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(tmp, x, 3 * n * sizeof(float), cudaMemcpyHostToDevice);
    dx = tmp;
    dy = tmp + 3 * n;
  }
  if (e == cudaSuccess) {
    k_infer<<<(unsigned)((n + 127) / 128), 128>>>(mlp_view(M), n, dx, dy);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && where == PHL_HOST) e = cudaMemcpy(y, dy, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  return e == cudaSuccess ? PHL_OK : cuda_status(e, "phl_mlp_forward");
}

phl_status phl_mlp_guess_temperature(const phl_mlp *M, const phl_eos_table *tab, long n, const double *rho,
                           const double *eint, const double *X0, double *T, int where) {
  if (!M || !tab || n <= 0 || !rho || !eint || !X0 || !T)
    return (phl_status)set_error(PHL_EINVAL, "phl_mlp_guess_temperature: bad arguments");
  const eos::Table &t = *eos_table_view(tab);
  const double Tlo = exp(t.y0), Thi = exp(t.y0 + (t.ny - 1) * t.dy);
  const double *dr = rho, *de = eint, *dx = X0;
  double *dT = T, *tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (where == PHL_HOST) {
    e = cudaMalloc(&tmp, 4 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(tmp, rho, n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tmp + n, eint, n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(tmp + 2 * n, X0, n * 8, cudaMemcpyHostToDevice);
    dr = tmp; de = tmp + n; dx = tmp + 2 * n; dT = tmp + 3 * n;
  }
  if (e == cudaSuccess) {
    k_guess<<<(unsigned)((n + 127) / 128), 128>>>(mlp_view(M), n, dr, de, dx, Tlo, Thi, dT);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && where == PHL_HOST) e = cudaMemcpy(T, dT, n * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tmp);
  return e == cudaSuccess ? PHL_OK : cuda_status(e, "phl_mlp_guess_temperature");
}

phl_status phl_mlp_train(phl_mlp *M, const phl_eos_table *tab, const phl_mlp_train_cfg *cfg,
                         phl_mlp_train_stats *st) {
  if (!M || !tab || !cfg || cfg->nsamples < 1000 || cfg->batch < 32 || cfg->epochs < 1 || !(cfg->lr > 0.0))
    return (phl_status)set_error(PHL_EINVAL, "phl_mlp_train: bad arguments");
  const auto t0 = std::chrono::steady_clock::now();
  const eos::Table &t = *eos_table_view(tab);
  const long n = cfg->nsamples;
  const long nval = std::max(1000L, n / 20), ntr = n - nval;
  float *x = nullptr, *tt = nullptr, *pred = nullptr;
  int *fail = nullptr;
  unsigned int *mm = nullptr;
  cudaError_t e = cudaMalloc(&x, 3 * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tt, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&pred, nval * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&fail, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&mm, 2 * sizeof(unsigned int));
  Scratch S;
  if (e == cudaSuccess) e = S.alloc(cfg->batch);
  phl_status ret = PHL_OK;
  auto done = [&](phl_status r) {
    cudaFree(x); cudaFree(tt); cudaFree(pred); cudaFree(fail); cudaFree(mm);
    return r;
  };
  if (e != cudaSuccess) return done((phl_status)set_error(PHL_ENOMEM, "phl_mlp_train: %s", cudaGetErrorString(e)));
  cudaMemset(fail, 0, sizeof(int));
  const unsigned nbk = (unsigned)((n + 255) / 256);
  k_samples<<<nbk, 256>>>(t, n, cfg->seed, cfg->lrho[0], cfg->lrho[1], cfg->lT[0], cfg->lT[1], cfg->A[0], cfg->Z[0],
                          cfg->A[1], cfg->Z[1], x, tt, fail);
  const unsigned int init[2] = {0x7f7fffffu, 0u};
  cudaMemcpy(mm, init, sizeof(init), cudaMemcpyHostToDevice);
  k_minmax_e<<<4 * 152, 256>>>(n, x, mm, mm + 1);
  int f = 0;
  unsigned int hm[2];
  e = cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return done(cuda_status(e, "phl_mlp_train samples"));
  if (f) return done((phl_status)set_error(PHL_EINVAL, "phl_mlp_train: sample range leaves the EOS table"));
  float emin, emax;
  memcpy(&emin, &hm[0], 4);
  memcpy(&emax, &hm[1], 4);
  // affine maps onto [-1, 1]
  M->c[0] = (float)(0.5 * (cfg->lrho[0] + cfg->lrho[1]));
  M->s[0] = (float)(2.0 / (cfg->lrho[1] - cfg->lrho[0]));
  M->c[1] = 0.5f * (emin + emax);
  M->s[1] = 2.0f / (emax - emin);
  M->c[2] = 0.5f;
  M->s[2] = 2.0f;
  M->c[3] = (float)(0.5 * (cfg->lT[0] + cfg->lT[1]));
  M->s[3] = (float)(2.0 / (cfg->lT[1] - cfg->lT[0]));
  k_normalise<<<nbk, 256>>>(n, x, tt, make_float4(M->c[0], M->c[1], M->c[2], M->c[3]),
                            make_float4(M->s[0], M->s[1], M->s[2], M->s[3]));
  // Adam on minibatches in sample order (the samples are i.i.d.); cosine-decayed rate
  const long nbat = std::max(1L, ntr / cfg->batch);
  const long total = nbat * cfg->epochs;
  double last = 0.0;
  long step = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    double ep_loss = 0.0;
    std::vector<double> losses;
    for (long b = 0; b < nbat; ++b, ++step) {
      const long off = b * cfg->batch;
      launch_loss_grad(M, cfg->batch, x + 3 * off, tt + off, S, 0);
      ++M->adam_t;
      const float lr = (float)(cfg->lr * 0.5 * (1.0 + cos(3.141592653589793 * (double)step / (double)total)));
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.0f - powf(b1, (float)M->adam_t), c2 = 1.0f - powf(b2, (float)M->adam_t);
      k_adam<<<(NPARAM + 255) / 256, 256>>>(NPARAM, M->w, M->m, M->v, M->grad, lr, b1, b2, 1e-8f, c1, c2);
      if (b + 1 == nbat) {
        double l = 0.0;
        cudaMemcpy(&l, S.loss, sizeof(double), cudaMemcpyDeviceToHost);
        ep_loss = l / (double)cfg->batch;
      }
    }
    last = ep_loss;
  }
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = build_fragments(M);
  if (e != cudaSuccess) return done(cuda_status(e, "phl_mlp_train"));
  // validation on the held-out samples with the BF16 inference kernel
  k_infer<<<(unsigned)((nval + 127) / 128), 128>>>(mlp_view(M), nval, x + 3 * ntr, pred);
  std::vector<float> hp(nval), ht(nval);
  e = cudaMemcpy(hp.data(), pred, nval * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ht.data(), tt + ntr, nval * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return done(cuda_status(e, "phl_mlp_train validation"));
  double se = 0.0, mx = 0.0;
  for (long i = 0; i < nval; ++i) {
    const double d = fabs((double)hp[i] - (double)ht[i]) / M->s[3];   // in log10 T
    se += d * d;
    mx = std::max(mx, d);
  }
  if (st) {
    st->final_loss = last;
    st->val_rms_log10T = sqrt(se / (double)nval);
    st->val_max_log10T = mx;
    st->steps = step;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return done(ret);
}

}  // extern "C"
