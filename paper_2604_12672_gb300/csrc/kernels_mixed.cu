// kernels_mixed.cu -- mixed-precision stage, one kernel per step of the
// stage (device bodies in mixed_common.cuh).
#include <math.h>

#include "mixed_common.cuh"

namespace phl {
using namespace stage;
namespace {

__global__ void k_prim_mx(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                          const float *__restrict__ dU, const float *__restrict__ dB, float *__restrict__ W,
                          int *dflag) {
  k_prim_mx_at(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, U, Bf, dU, dB, W, dflag);
}

// Five CTAs per SM (48 registers, a few spilled to L1): the pass is bound by
// the loads in flight, and this cap measured fastest (3 .. 8 tried).
__global__ void __launch_bounds__(256, 5) k_prim_mx2(DevGeo G, Box hbox, const double *__restrict__ U,
                                                  const double *__restrict__ Bf, const float *__restrict__ dU,
                                                  const float *__restrict__ dB, float *__restrict__ W, int *dflag) {
  k_prim_mx2_at<false>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, hbox, U, Bf, dU, dB, W, dflag);
}

// Block maximum of the CFL rates, one atomicMax per block (non-negative
// floats order like their bit patterns).
__device__ __forceinline__ void block_rate_max(float m, unsigned int *fmax_bits) {
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMax(fmax_bits, __float_as_uint(v));
  }
}

// The first stage's primitives of U^n, two cells per thread, with the CFL
// rate of the interior cells taken from the same deviations.
__global__ void __launch_bounds__(256, 5) k_prim_mx2_cfl(DevGeo G, Box hbox, const double *__restrict__ U,
                                                       const double *__restrict__ Bf, float *__restrict__ W,
                                                       int *dflag, unsigned int *fmax_bits) {
  const float m = k_prim_mx2_at<true>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, hbox, U, Bf, nullptr, nullptr,
                                      W, dflag);
  block_rate_max(m, fmax_bits);
}

// The first stage's primitives of U^n with the CFL rate of the interior
// cells folded in (the rate as k_dt_mx, from the deviations the thread has
// just formed): block maximum, one atomicMax per block.
__global__ void __launch_bounds__(256) k_prim_mx_cfl(DevGeo G, Box box, const double *__restrict__ U,
                                                     const double *__restrict__ Bf, float *__restrict__ W, int *dflag,
                                                     unsigned int *fmax_bits) {
  float m = 0.0f;
  int c[3];
  if (cell_at(box, blockIdx.x * (long)blockDim.x + threadIdx.x, c))
    prim_store_cell(G, c, U, Bf, nullptr, nullptr, W, dflag, &m);
  block_rate_max(m, fmax_bits);
}

__global__ void k_update_cells_mx(DevGeo G, Box box, StageMx S) {
  k_update_cells_mx_at(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, S);
}

template <int D>
__global__ void k_update_faces_mx(DevGeo G, Box box, StageMx S) {
  k_update_faces_mx_at<D>(blockIdx.x * (long)blockDim.x + threadIdx.x, G, box, S);
}

// CFL condition in FP32 from U^n (Eq. cfl); non-negative floats order like
// their bit patterns, so the block maxima combine with an integer atomicMax.
__global__ void k_dt_mx(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                        unsigned int *fmax_bits, int *dflag) {
  float m = 0.0f;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < box.n; t += (long)gridDim.x * blockDim.x) {
    int c[3];
    unflat(box, t, c);
    m = fmaxf(m, dt_rate_mx(G, U, Bf, c, dflag));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[TPB / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMax(fmax_bits, __float_as_uint(v));
  }
}

__global__ void k_dt_mx_finalize(double cfl, double t_s, unsigned int *fmax_bits, double *dt) {
  *dt = cfl * t_s / (double)__uint_as_float(*fmax_bits);
  *fmax_bits = 0u;
}

// A step of given length: sets dt and clears the CFL maximum the step's last
// stage folds into.
__global__ void k_dt_fixed(double v, unsigned int *fmax_bits, double *dt) {
  *dt = v;
  *fmax_bits = 0u;
}

}  // namespace

void launch_dt_mixed(const DevGeo &G, const double *U, const double *Bf, unsigned int *fmax_bits, double *dt,
                     int *dflag, cudaStream_t s, int *nlaunch, Prof *prof) {
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  PHL_LAUNCH(KC_DT, prof, s, k_dt_mx<<<nblocks(b.n), TPB, 0, s>>>(G, b, U, Bf, fmax_bits, dflag));
  PHL_LAUNCH(KC_DT, prof, s, k_dt_mx_finalize<<<1, 1, 0, s>>>(G.cfl, G.sc_t, fmax_bits, dt));
  if (nlaunch) *nlaunch += 2;
}

void launch_dt_mixed_from_max(const DevGeo &G, double fixed_dt, unsigned int *fmax_bits, double *dt, cudaStream_t s,
                              int *nlaunch, Prof *prof) {
  if (fixed_dt > 0.0) PHL_LAUNCH(KC_DT, prof, s, k_dt_fixed<<<1, 1, 0, s>>>(fixed_dt, fmax_bits, dt));
  else PHL_LAUNCH(KC_DT, prof, s, k_dt_mx_finalize<<<1, 1, 0, s>>>(G.cfl, G.sc_t, fmax_bits, dt));
  if (nlaunch) *nlaunch += 1;
}

cudaError_t launch_prims_form(const DevGeo &G, const double *U, const double *Bf, const float *dU, const float *dB,
                              float *W, int *dflag, int form, unsigned int *fmax_bits, cudaStream_t s) {
  int l[3], h[3];
  for (int d = 0; d < 3; ++d) {
    if (G.act[d]) { l[d] = -G.ge[d]; h[d] = G.n[d] + G.ge[d]; }
    else { l[d] = 0; h[d] = 1; }
  }
  const Box bx = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
  const Box hb = make_box(0, (G.n[0] + 2 * G.ge[0]) / 2, l[1], h[1], l[2], h[2]);
  switch (form) {
    case 0: k_prim_mx<<<grid3(bx), block3(bx), 0, s>>>(G, bx, U, Bf, dU, dB, W, dflag); break;
    case 1: k_prim_mx2<<<grid3(hb), block3(hb), 0, s>>>(G, hb, U, Bf, dU, dB, W, dflag); break;
    case 2: k_prim_mx_cfl<<<grid3(bx), block3(bx), 0, s>>>(G, bx, U, Bf, W, dflag, fmax_bits); break;
    default: k_prim_mx2_cfl<<<grid3(hb), block3(hb), 0, s>>>(G, hb, U, Bf, W, dflag, fmax_bits); break;
  }
  return cudaGetLastError();
}

void launch_stage_mixed(const DevGeo &G, const MixedBufs &M, int stage, int nstages, double b, cudaStream_t s,
                        int *nlaunch, Prof *prof) {
  int nl = 0;
  const bool first = stage == 0, last = stage == nstages - 1;
  const float *dU = first ? nullptr : M.dU;
  const float *dB = first ? nullptr : M.dB;
  auto rng = [&](int d, int lo_g, int hi_extra, int &lo, int &hi) {
    if (G.act[d]) { lo = -lo_g; hi = G.n[d] + hi_extra; }
    else { lo = 0; hi = 1; }
  };
  const bool fused = M.tmapW && fused_stage_ok(G);
  const bool three = fused && M.pipeline3;
  // on the three-launch path the previous stage formed this stage's W and raw
  // flags; only a stage whose input was set from outside starts with them
  if (!three || (first && !M.primed)) {
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) rng(d, G.ge[d], G.ge[d], l[d], h[d]);
    Box bx = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    if (G.eos == 1) {
      // each cell starts from its previous inversion's record (a cleared
      // record falls back to the plain start); network-first mode: the
      // network's guess instead
      launch_eos_cells<float>(G, M.U, M.B, dU, dB, M.Tin, M.Tout, M.W, M.dflag, s, &nl, prof,
                              first ? M.cfl_dmax : nullptr, const_cast<double *>(M.dt), G.use_mlp == 1 ? 0 : 2);
    } else {
      if (first && M.cfl_fmax) {   // the step's CFL step from the same pass over U^n
        if (prim_pairs_ok(G)) {
          Box hb = make_box(0, (G.n[0] + 2 * G.ge[0]) / 2, l[1], h[1], l[2], h[2]);
          PHL_LAUNCH(KC_PRIM, prof, s,
                     k_prim_mx2_cfl<<<grid3(hb), block3(hb), 0, s>>>(G, hb, M.U, M.B, M.W, M.dflag, M.cfl_fmax));
        } else {
          PHL_LAUNCH(KC_PRIM, prof, s,
                     k_prim_mx_cfl<<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.U, M.B, M.W, M.dflag, M.cfl_fmax));
        }
        PHL_LAUNCH(KC_DT, prof, s, k_dt_mx_finalize<<<1, 1, 0, s>>>(G.cfl, G.sc_t, M.cfl_fmax, const_cast<double *>(M.dt)));
        nl += 2;
      } else if (prim_pairs_ok(G)) {   // two cells of a row per thread
        Box hb = make_box(0, (G.n[0] + 2 * G.ge[0]) / 2, l[1], h[1], l[2], h[2]);
        PHL_LAUNCH(KC_PRIM, prof, s,
                   k_prim_mx2<<<grid3(hb), block3(hb), 0, s>>>(G, hb, M.U, M.B, dU, dB, M.W, M.dflag));
        ++nl;
      } else {
        PHL_LAUNCH(KC_PRIM, prof, s, k_prim_mx<<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.U, M.B, dU, dB, M.W, M.dflag));
        ++nl;
      }
    }
    if (three && G.eps_sf > 0.0) {
      Box bi = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
      PHL_LAUNCH(KC_FLAG_RAW, prof, s, k_flag_raw<float><<<grid3(bi), block3(bi), 0, s>>>(G, bi, M.W, M.raw));
      ++nl;
    }
  }
  if (G.eps_sf > 0.0 && !fused) {
    Box bx = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_FLAG_RAW, prof, s, k_flag_raw<float><<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.W, M.raw));
    nl += 1 + launch_flags(G, M.raw, M.raw + (long)G.n[0] * G.n[1] * G.n[2], M.flag, s, prof);
  }
  if (fused) launch_fused_tail(G, M, first, last, b, s, &nl, prof);   // flags, faces, cells, EMFs, faces B
  for (int D = 0; D < 3 && !fused; ++D) {
    if (!G.act[D]) continue;
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) {
      if (d == D) { l[d] = 0; h[d] = G.n[d] + 1; }
      else rng(d, 1, 1, l[d], h[d]);
    }
    Box bx = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    launch_flux<float>(D, G, bx, M.W, M.B, dB, M.flag, M.F[D], M.dflag, s, prof);
    ++nl;
  }
  for (int D = 0; D < 3 && !fused; ++D) {
    const int A = (D + 1) % 3, B = (D + 2) % 3;
    if (!G.act[A] && !G.act[B]) continue;
    int l[3] = {0, 0, 0}, h[3];
    h[D] = G.n[D];
    h[A] = G.act[A] ? G.n[A] + 1 : 1;
    h[B] = G.act[B] ? G.n[B] + 1 : 1;
    Box bx = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    if (D == 0) PHL_LAUNCH(KC_EMF, prof, s, k_emf<0, float><<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.W, M.F[1], M.F[2], M.E));
    if (D == 1) PHL_LAUNCH(KC_EMF, prof, s, k_emf<1, float><<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.W, M.F[2], M.F[0], M.E));
    if (D == 2) PHL_LAUNCH(KC_EMF, prof, s, k_emf<2, float><<<grid3(bx), block3(bx), 0, s>>>(G, bx, M.W, M.F[0], M.F[1], M.E));
    ++nl;
  }
  StageMx S;
  S.U = M.U; S.B = M.B; S.dU = M.dU; S.dB = M.dB;
  S.first = first; S.last = last; S.b = (float)b; S.dt = M.dt;
  S.W = M.W; S.F[0] = M.F[0]; S.F[1] = M.F[1]; S.F[2] = M.F[2]; S.E = M.E;
  if (!fused) {
    Box bx = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
    PHL_LAUNCH(KC_UPDATE_CELLS, prof, s, k_update_cells_mx<<<grid3(bx), block3(bx), 0, s>>>(G, bx, S));
    ++nl;
  }
  for (int D = 0; D < 3 && !fused; ++D) {
    int h[3] = {G.n[0], G.n[1], G.n[2]};
    h[D] += 1;
    Box bx = make_box(0, h[0], 0, h[1], 0, h[2]);
    if (D == 0) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces_mx<0><<<grid3(bx), block3(bx), 0, s>>>(G, bx, S));
    if (D == 1) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces_mx<1><<<grid3(bx), block3(bx), 0, s>>>(G, bx, S));
    if (D == 2) PHL_LAUNCH(KC_UPDATE_FACES, prof, s, k_update_faces_mx<2><<<grid3(bx), block3(bx), 0, s>>>(G, bx, S));
    ++nl;
  }
  if (nlaunch) *nlaunch += nl;
}

}  // namespace phl
