// stage_prim.cu -- the last kernel of a mixed stage on the three-launch fused
// path: the primitive deviations of the next stage (Sect. 2.8), written to
// the work array with every ghost image of each cell (periodic wrap, mirror
// with the normal components flipped, outflow copy: Table bcs), the raw
// shock flags (Sect. 2.7), and in the last stage of a step the CFL rate of
// the new state (Eq. cfl) folded into the next step's maximum.
//
// One CTA takes a tile of PX x PY x PZ cells and its one-cell halo.  Every
// position of the box forms its primitives from the state (a halo position
// beyond a boundary from its source cell) and leaves its full pressure in
// shared memory; a position that is one of the tile's cells also writes its
// deviations and auxiliaries at once.  The raw flag of each tile cell then
// compares the pressures of its six neighbours.  Halo positions are the
// price of not storing the pressure in HBM: (PX+2)(PY+2)(PZ+2) / (PX PY PZ)
// = 1.58 evaluations per cell at 16 x 16 x 8.
#include <math.h>

#include "mixed_common.cuh"

namespace phl {
using namespace stage;
namespace {

constexpr int PX = 16, PY = 16, PZ = 8;
constexpr int BX = PX + 2, BY = PY + 2, BZ = PZ + 2, BN = BX * BY * BZ;
constexpr int PT = 256;

struct PrimArgs {
  const double *U, *B;   // U^n (or U^(n+1) after the last stage)
  const float *dU, *dB;  // increments of the stage output (null: none)
  float *W;              // work array of the next stage
  uint8_t *raw;          // raw shock flags, interior layout
  unsigned int *fmax;    // CFL rate maximum (bits), when cfl
  int *dflag;
  int cfl;
};

// Every work-layout position along one axis whose data is interior cell i
// (i itself and the ghost positions that map to it), with its mirror flag;
// at most 1 + 2 ge entries.
__device__ __forceinline__ int images(const DevGeo &G, int d, int i, int *pos, bool *flip) {
  int m = 0;
  pos[m] = i;
  flip[m++] = false;
  if (i >= G.ge[d] && i < G.n[d] - G.ge[d]) return m;   // far from both sides: no ghost maps here
  for (int g = -G.ge[d]; g < 0; ++g) {
    bool fl;
    if (cell_src(g, G.n[d], G.bc[d][0], G.bc[d][1], fl) == i) { pos[m] = g; flip[m++] = fl; }
  }
  for (int g = G.n[d]; g < G.n[d] + G.ge[d]; ++g) {
    bool fl;
    if (cell_src(g, G.n[d], G.bc[d][0], G.bc[d][1], fl) == i) { pos[m] = g; flip[m++] = fl; }
  }
  return m;
}

__global__ void __launch_bounds__(PT) k_prim_flags(DevGeo G, PrimArgs A, int ntx, int nty) {
  __shared__ float sp[BN];   // full pressure of the box cells, background at the position's own height
  __shared__ float red[PT / 32];
  const int tid = threadIdx.x;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty, tz = t / nty;
  const int o[3] = {tx * PX, ty * PY, tz * PZ};
  float m = 0.0f;
  float4 *W4 = reinterpret_cast<float4 *>(A.W);
  for (int q = tid; q < BN; q += PT) {
    const int l0 = q % BX, l1 = (q / BX) % BY, l2 = q / (BX * BY);
    const int x[3] = {o[0] - 1 + l0, o[1] - 1 + l1, o[2] - 1 + l2};
    if (x[0] < -1 || x[0] > G.n[0] || x[1] < -1 || x[1] > G.n[1] || x[2] < -1 || x[2] > G.n[2]) continue;
    int s[3];
    bool fl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = cell_src(x[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]);
    float w[NW_MAX];
    cell_prims_mx(G, A.U, A.B, A.dU, A.dB, s[0], s[1], s[2], w, A.dflag);
    sp[q] = w[W_P] + bg_cell_t<float>(G, x[2]).p;   // the pressure deviation is not flipped
    const bool own = l0 >= 1 && l0 <= PX && l1 >= 1 && l1 <= PY && l2 >= 1 && l2 <= PZ && x[0] < G.n[0] &&
                     x[1] < G.n[1] && x[2] < G.n[2];
    if (!own) continue;
    // the cell at every position that holds its data
    int px[1 + 2 * NGW], py[1 + 2 * NGW], pz[1 + 2 * NGW];
    bool fx[1 + 2 * NGW], fy[1 + 2 * NGW], fz[1 + 2 * NGW];
    const int nx = images(G, 0, x[0], px, fx), ny = images(G, 1, x[1], py, fy), nz = images(G, 2, x[2], pz, fz);
    for (int kz = 0; kz < nz; ++kz)
      for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < nx; ++kx) {
          float u[NW_MAX];
#pragma unroll
          for (int v = 0; v <= W_P; ++v) u[v] = w[v];
          const bool f3[3] = {fx[kx], fy[ky], fz[kz]};
#pragma unroll
          for (int d = 0; d < 3; ++d)
            if (f3[d]) { u[W_VX + d] = -u[W_VX + d]; u[W_BX + d] = -u[W_BX + d]; }
          const long p = widx(G, px[kx], py[ky], pz[kz]);
          W4[p] = make_float4(u[W_RHO], u[W_VX], u[W_VY], u[W_VZ]);
          W4[G.wtot + p] = make_float4(u[W_BX], u[W_BY], u[W_BZ], u[W_P]);
          write_aux(G, A.W, p, u);
        }
    if (A.cfl) m = fmaxf(m, dt_rate_w(G, w, x[2]));
  }
  __syncthreads();
  if (G.eps_sf > 0.0) {   // raw flags: sum_d |P(+1) - P(-1)| / (eps P) > 1
    for (int q = tid; q < PX * PY * PZ; q += PT) {
      const int c[3] = {o[0] + q % PX, o[1] + (q / PX) % PY, o[2] + q / (PX * PY)};
      if (c[0] >= G.n[0] || c[1] >= G.n[1] || c[2] >= G.n[2]) continue;
      const int b = ((c[2] - o[2] + 1) * BY + (c[1] - o[1] + 1)) * BX + (c[0] - o[0] + 1);
      const float P0 = sp[b];
      float sum = 0.0f;
      sum += fabsf(sp[b + 1] - sp[b - 1]);
      sum += fabsf(sp[b + BX] - sp[b - BX]);
      sum += fabsf(sp[b + BX * BY] - sp[b - BX * BY]);
      A.raw[c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])] = (sum / (G.epsf * P0) > 1.0f) ? 1 : 0;
    }
  }
  if (A.cfl) {   // block maximum; non-negative floats order like their bits
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      float v = tid < PT / 32 ? red[tid] : 0.0f;
      for (int s = 16; s > 0; s >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, s));
      if (tid == 0) atomicMax(A.fmax, __float_as_uint(v));
    }
  }
}

}  // namespace

// The next stage's primitives (last stage: of U^(n+1), no increments, and
// unless fmax is null the CFL rate of each cell folded into fmax).
void launch_prim_flags(const DevGeo &G, const MixedBufs &M, bool last, unsigned int *fmax, cudaStream_t s, int *nl,
                       Prof *prof) {
  const int ntx = (G.n[0] + PX - 1) / PX, nty = (G.n[1] + PY - 1) / PY, ntz = (G.n[2] + PZ - 1) / PZ;
  PrimArgs A;
  A.U = M.U; A.B = M.B;
  A.dU = last ? nullptr : M.dU;
  A.dB = last ? nullptr : M.dB;
  A.W = M.W; A.raw = M.raw; A.fmax = fmax; A.dflag = M.dflag; A.cfl = (last && fmax) ? 1 : 0;
  PHL_LAUNCH(KC_PRIM, prof, s, k_prim_flags<<<ntx * nty * ntz, PT, 0, s>>>(G, A, ntx, nty));
  *nl += 1;
}

}  // namespace phl
