// mlp_dev.cuh -- temperature-guess network on the device: inference with BF16
// weights on the tensor cores (mma.sync m16n8k16, FP32 accumulation; the
// activations enter as a hi + lo pair of BF16 values).
//
// Network: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, 3 inputs, two hidden
// layers of 64, one output.  Inputs (affine maps held with the weights):
//   x0 = (log10 rho - c0) s0,  x1 = (log10 e_int - c1) s1,  x2 = (X_0 - c2) s2,
// output log10 T = c3 + y / s3.  The guess only starts the Newton inversion
// e_int -> T; the converged T does not depend on it.
//
// One warp evaluates 32 cells (one per lane) as two 16-row tiles.  Weights are
// stored per lane in the B-fragment order of mma.m16n8k16 (row.col, bf16):
// lane (g = lane / 4, q = lane % 4) of k-tile kt, n-tile nt holds
//   { B[16 kt + 2q][8 nt + g], B[16 kt + 2q + 1][...] },
//   { B[16 kt + 2q + 8][...],  B[16 kt + 2q + 9][...] }   with B[k][n] = W[n][k],
// two bf16 per 32-bit word, the lower k in the low half.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace phl {
namespace mlp {

constexpr int NIN = 3, NH = 64;
constexpr int NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1;   // oracle layout
// offsets of the flat FP32 parameter vector: W1[NH][NIN], b1, W2[NH][NH], b2, W3[NH], b3
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH, O_W3 = O_B2 + NH,
              O_B3 = O_W3 + NH;
// fragment words (uint2 per lane per tile): layer 1: 1 x 8 tiles, layer 2: 4 x 8, layer 3: 4 x 1
constexpr int F_L1 = 0, F_L2 = F_L1 + 8 * 32, F_L3 = F_L2 + 32 * 32, F_TOTAL = F_L3 + 4 * 32;

struct Dev {
  const uint2 *frag;      // F_TOTAL words
  const float *b1, *b2;   // NH each (FP32 biases)
  float b3;
  float c[4], s[4];       // input / output affine maps
};

__device__ __forceinline__ void mma_bf16(float &d0, float &d1, float &d2, float &d3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Activations enter the tensor cores as a BF16 pair a = a_hi + a_lo (the
// residual of the first rounding), so only the weights are rounded to BF16.
struct Split { uint32_t hi, lo; };
__device__ __forceinline__ Split split_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  Split s;
  s.hi = *reinterpret_cast<const uint32_t *>(&h);
  s.lo = pack_bf16(a - hf.x, b - hf.y);
  return s;
}

// D += (A_hi + A_lo) B for one 16x8 output tile.
__device__ __forceinline__ void mma_split(float &d0, float &d1, float &d2, float &d3, const Split *a, uint2 b) {
  mma_bf16(d0, d1, d2, d3, a[0].hi, a[1].hi, a[2].hi, a[3].hi, b.x, b.y);
  mma_bf16(d0, d1, d2, d3, a[0].lo, a[1].lo, a[2].lo, a[3].lo, b.x, b.y);
}

// Network output for the 16 cells of one tile whose inputs sit in lanes
// base..base+15 (xin[3] of every lane; lanes outside pass zeros).  Returns,
// in lane r of the warp, the output of row (r - base) when base <= r < base+16.
__device__ __forceinline__ float tile_forward(const Dev &M, const float xin[3], int base) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  // A fragment of the inputs: k = 2q, 2q + 1 (features 0..2, zero beyond), rows g, g + 8
  float xa[2][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int src = base + g + 8 * h;
    const float v0 = __shfl_sync(0xffffffffu, xin[0], src);
    const float v1 = __shfl_sync(0xffffffffu, xin[1], src);
    const float v2 = __shfl_sync(0xffffffffu, xin[2], src);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int f = 2 * q + e;
      xa[h][e] = f == 0 ? v0 : (f == 1 ? v1 : (f == 2 ? v2 : 0.0f));
    }
  }
  const Split zero = {0u, 0u};
  const Split A1[4] = {split_bf16(xa[0][0], xa[0][1]), split_bf16(xa[1][0], xa[1][1]), zero, zero};
  // layer 1 -> tanh -> A fragments of layer 2 (4 k-tiles)
  Split A2[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = 8 * nt + 2 * q;
    float d0 = M.b1[col], d1 = M.b1[col + 1], d2 = d0, d3 = d1;
    mma_split(d0, d1, d2, d3, A1, M.frag[F_L1 + nt * 32 + lane]);
    const Split lo = split_bf16(tanh_fast(d0), tanh_fast(d1)), hi = split_bf16(tanh_fast(d2), tanh_fast(d3));
    if (nt & 1) { A2[nt >> 1][2] = lo; A2[nt >> 1][3] = hi; }
    else { A2[nt >> 1][0] = lo; A2[nt >> 1][1] = hi; }
  }
  // layer 2 -> tanh -> A fragments of layer 3
  Split A3[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = 8 * nt + 2 * q;
    float d0 = M.b2[col], d1 = M.b2[col + 1], d2 = d0, d3 = d1;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma_split(d0, d1, d2, d3, A2[kt], M.frag[F_L2 + (kt * 8 + nt) * 32 + lane]);
    const Split lo = split_bf16(tanh_fast(d0), tanh_fast(d1)), hi = split_bf16(tanh_fast(d2), tanh_fast(d3));
    if (nt & 1) { A3[nt >> 1][2] = lo; A3[nt >> 1][3] = hi; }
    else { A3[nt >> 1][0] = lo; A3[nt >> 1][1] = hi; }
  }
  // layer 3: one n-tile, output in column 0 (lanes with q == 0)
  float d0 = (q == 0) ? M.b3 : 0.0f, d1 = 0.0f, d2 = d0, d3 = 0.0f;
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) mma_split(d0, d1, d2, d3, A3[kt], M.frag[F_L3 + kt * 32 + lane]);
  // row r of the tile sits in lane 4 (r mod 8): d0 for r < 8, d2 for r >= 8
  const int r = lane - base;
  const int src = 4 * (r & 7);
  const float y0 = __shfl_sync(0xffffffffu, d0, src & 31);
  const float y2 = __shfl_sync(0xffffffffu, d2, src & 31);
  return (r & 8) ? y2 : y0;
}

// Warp-collective: every lane passes its cell's (log10 rho, log10 e_int, X_0)
// (any finite values for lanes without a cell) and receives log10 T_guess.
__device__ __forceinline__ float guess_log10T(const Dev &M, float lrho, float le, float x0) {
  const float xin[3] = {(lrho - M.c[0]) * M.s[0], (le - M.c[1]) * M.s[1], (x0 - M.c[2]) * M.s[2]};
  const int lane = threadIdx.x & 31;
  const float ylo = tile_forward(M, xin, 0);
  const float yhi = tile_forward(M, xin, 16);
  const float y = lane < 16 ? ylo : yhi;
  return M.c[3] + y / M.s[3];
}

}  // namespace mlp
}  // namespace phl
