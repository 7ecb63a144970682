// stage_ct.cu -- the two kernels that close a mixed stage on the fused path
// after the tile kernel (stage_fused.cu) has evaluated the faces and updated
// the cells:
//
//   k_ct_faces    Contact-CT edge EMFs (Sect. 2.4) of an 8^3 tile of sites
//                 from the tangential-B fluxes and contact directions the tile
//                 kernel left for its owned faces, then the update of the
//                 normal field on the tile's own faces from the curl of those
//                 EMFs (Eq. induction in discrete form, Sect. 2.9).
//   k_prim_flags  the primitive deviations of the next stage (Sect. 2.8) for
//                 an 8^3 tile of cells, written to the work array with every
//                 ghost image of each cell (periodic wrap, mirror with flipped
//                 normal components, outflow copy: Table bcs), the raw shock
//                 flags of the tile's cells (Sect. 2.7) from the pressure of
//                 the tile and a one-cell halo, and in the last stage of a
//                 step the CFL rate of the new state (Eq. cfl) folded into a
//                 block maximum.
//
// With the tile kernel this makes a stage three launches.  Each kernel keeps
// what its neighbours in the stage need in shared memory: the EMFs of the
// edges its faces touch, and the halo pressures its flags compare.  The face
// fields are updated in place: a face is written by exactly one tile, and the
// primitives are formed only after every face has been updated (next kernel).
#include <math.h>

#include "mixed_common.cuh"

namespace phl {
using namespace stage;
namespace {

constexpr int CT = 8;              // tile edge, sites or cells
constexpr int CB = CT + 3;         // staged box edge of the CT kernel: sites o-1 .. o+9
constexpr int CB3 = CB * CB * CB;
constexpr int EB = CT + 2;         // edge box edge: sites o .. o+9
constexpr int EB3 = EB * EB * EB;
constexpr int CT_THREADS = 256;

struct CtSmem {
  float f[3][3][CB3];   // D-faces: tangential-B fluxes F_D(B_T1), F_D(B_T2), contact direction
  float ec[3][CB3];     // cell reference EMFs -(u x B)_D
  float ed[3][EB3];     // edge EMFs E_D
};
constexpr size_t ct_smem_bytes() { return sizeof(CtSmem); }

__device__ __forceinline__ int cbox(int x, int y, int z) { return (z * CB + y) * CB + x; }
__device__ __forceinline__ int ebox(int x, int y, int z) { return (z * EB + y) * EB + x; }

// Last site of the tile along d: o + 7, or n when the tile reaches the upper
// boundary (that tile also owns the boundary face n).
__device__ __forceinline__ int tile_hi(int o, int n) { return o + CT >= n ? n : o + CT - 1; }

__global__ void __launch_bounds__(CT_THREADS) k_ct_faces(DevGeo G, StageMx S, int ntx, int nty) {
  extern __shared__ unsigned char ctraw[];
  CtSmem &sm = *reinterpret_cast<CtSmem *>(ctraw);
  const int tid = threadIdx.x;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty, tz = t / nty;
  const int o[3] = {tx * CT, ty * CT, tz * CT};
  int hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) hi[d] = tile_hi(o[d], G.n[d]);
  const long wt = G.wtot;

  // (1) stage the D-face fluxes on sites o-1 .. o+9 (rows beyond a boundary
  // read the interior row their data come from) and the cell EMFs of the same
  // box (ghost cells are stored in the work layout)
  for (int q = tid; q < CB3; q += CT_THREADS) {
    const int l[3] = {q % CB, (q / CB) % CB, q / (CB * CB)};
    int x[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) x[d] = o[d] - 1 + l[d];
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
      float v1 = 0.0f, v2 = 0.0f, vd = 0.0f;
      if (x[D] >= 0 && x[D] <= G.n[D] && x[T1] >= -1 && x[T1] <= G.n[T1] && x[T2] >= -1 && x[T2] <= G.n[T2]) {
        int r[3] = {x[0], x[1], x[2]};
        bool fl;
        r[T1] = cell_src(x[T1], G.n[T1], G.bc[T1][0], G.bc[T1][1], fl);
        r[T2] = cell_src(x[T2], G.n[T2], G.bc[T2][0], G.bc[T2][1], fl);
        const long p = widx(G, r[0], r[1], r[2]);
        const float *F = S.F[D];
        v1 = F[(F_BX + T1) * wt + p];
        v2 = F[(F_BX + T2) * wt + p];
        vd = F[(long)G.nf * wt + p];
      }
      sm.f[D][0][q] = v1;
      sm.f[D][1][q] = v2;
      sm.f[D][2][q] = vd;
    }
    const bool inw = x[0] >= -G.ge[0] && x[0] < G.n[0] + G.ge[0] && x[1] >= -G.ge[1] && x[1] < G.n[1] + G.ge[1] &&
                     x[2] >= -G.ge[2] && x[2] < G.n[2] + G.ge[2];
    const long p = inw ? widx(G, x[0], x[1], x[2]) : 0;
#pragma unroll
    for (int D = 0; D < 3; ++D) sm.ec[D][q] = inw ? S.W[waux(G, AUX_E + D, p)] : 0.0f;
  }
  __syncthreads();

  // (2) edge EMFs along D at the lower corner of site s, for the sites the
  // tile's faces need: s_D in [o_D, hi_D] (s_D < n_D), s_A in [o_A, hi_A + 1]
  // (<= n_A), the same for B.  (D, A, B) cyclic; E_D = -F_A(B_B) on A-faces,
  // +F_B(B_A) on B-faces, each half-derivative towards the cell EMF upwinded
  // by the face's contact direction (the mean of both sides with none).
  for (int q = tid; q < 3 * EB3; q += CT_THREADS) {
    const int D = q / EB3, r = q % EB3;
    const int e[3] = {r % EB, (r / EB) % EB, r / (EB * EB)};
    const int A = (D + 1) % 3, B = (D + 2) % 3;
    int s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = o[d] + e[d];
    const bool need = s[D] <= hi[D] && s[D] < G.n[D] && s[A] <= hi[A] + 1 && s[A] <= G.n[A] &&
                      s[B] <= hi[B] + 1 && s[B] <= G.n[B];
    float v = 0.0f;
    if (need) {
      // box index of site s is s - o + 1; a step towards -A or -B is -1 there
      const int l0 = e[0] + 1, l1 = e[1] + 1, l2 = e[2] + 1;
      const int c11 = cbox(l0, l1, l2);
      const int sa = A == 0 ? 1 : (A == 1 ? CB : CB * CB), sb = B == 0 ? 1 : (B == 1 ? CB : CB * CB);
      const float *fab = sm.f[A][0];   // F_A(B_B): T1 of A-faces is B
      const float *fba = sm.f[B][1];   // F_B(B_A): T2 of B-faces is A
      const float *ua = sm.f[A][2], *ub = sm.f[B][2];
      const float Ea1 = -fab[c11], Ea0 = -fab[c11 - sb];
      const float Eb1 = fba[c11], Eb0 = fba[c11 - sa];
      const float ma1 = ua[c11], ma0 = ua[c11 - sb];
      const float mb1 = ub[c11], mb0 = ub[c11 - sa];
      const float *ecell = sm.ec[D];
      const float E00 = ecell[c11 - sa - sb], E10 = ecell[c11 - sb], E01 = ecell[c11 - sa], E11 = ecell[c11];
      const float lo_l = Eb0 - E00, lo_r = Eb1 - E10;
      const float up_l = E01 - Eb0, up_r = E11 - Eb1;
      const float h = 0.5f, q4 = 0.25f;
      const float dlo = ma0 > 0.0f ? lo_l : (ma0 < 0.0f ? lo_r : h * (lo_l + lo_r));
      const float dup = ma1 > 0.0f ? up_l : (ma1 < 0.0f ? up_r : h * (up_l + up_r));
      const float le_d = Ea0 - E00, le_u = Ea1 - E01;
      const float ri_d = E10 - Ea0, ri_u = E11 - Ea1;
      const float dle = mb0 > 0.0f ? le_d : (mb0 < 0.0f ? le_u : h * (le_d + le_u));
      const float dri = mb1 > 0.0f ? ri_d : (mb1 < 0.0f ? ri_u : h * (ri_d + ri_u));
      v = q4 * (Ea1 + Ea0 + Eb1 + Eb0) + q4 * (dlo - dup) + q4 * (dle - dri);
      // an edge on a reflecting wall: u_n = B_n = 0 there (Table bcs)
      if ((s[A] == 0 && G.bc[A][0] == 1) || (s[A] == G.n[A] && G.bc[A][1] == 1) ||
          (s[B] == 0 && G.bc[B][0] == 1) || (s[B] == G.n[B] && G.bc[B][1] == 1))
        v = 0.0f;
    }
    sm.ed[D][r] = v;
  }
  __syncthreads();

  // (3) the tile's own faces: D-face at site s, s_D in [o_D, hi_D],
  // s_T in [o_T, min(hi_T, n_T - 1)]; dB/dt = -(d_A E_B - d_B E_A)
  const float dt = d2f_scaled(*S.dt, -G.e_t);
  for (int q = tid; q < 3 * (CT + 1) * CT * CT; q += CT_THREADS) {
    const int D = q / ((CT + 1) * CT * CT), r = q % ((CT + 1) * CT * CT);
    const int A = (D + 1) % 3, B = (D + 2) % 3;
    int e[3];
    e[D] = r % (CT + 1);
    e[A] = (r / (CT + 1)) % CT;
    e[B] = r / ((CT + 1) * CT);
    int s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = o[d] + e[d];
    if (s[D] > hi[D] || s[A] > hi[A] || s[A] >= G.n[A] || s[B] > hi[B] || s[B] >= G.n[B]) continue;
    const int eA = A == 0 ? 1 : (A == 1 ? EB : EB * EB), eB = B == 0 ? 1 : (B == 1 ? EB : EB * EB);
    const int k0 = ebox(e[0], e[1], e[2]);
    float rr = 0.0f;
    rr += (sm.ed[B][k0 + eA] - sm.ed[B][k0]) * G.idxf[A];
    rr -= (sm.ed[A][k0 + eB] - sm.ed[A][k0]) * G.idxf[B];
    const long qg = (long)D * G.plane + sidx(G, s[0], s[1], s[2]);
    const float din = S.first ? 0.0f : S.dB[qg];
    const float dout = S.b * (din - dt * rr);
    if (S.last) S.B[qg] += f2d_scaled(dout, G.e_b);
    else S.dB[qg] = dout;
  }
}

// ---------------------------------------------------------------------------
constexpr int PB = CT + 2;           // primitive box: cells o-1 .. o+8
constexpr int PB3 = PB * PB * PB;
constexpr int PF_THREADS = 256;

struct PrimArgs {
  const double *U, *B;   // U^n (or U^(n+1) after the last stage)
  const float *dU, *dB;  // increments of the stage output (null: none)
  float *W;              // work array of the next stage
  uint8_t *raw;          // raw shock flags, interior layout
  unsigned int *fmax;    // CFL rate maximum (bits), last stage only
  int *dflag;
  int cfl;
};

// Every work-layout position along one axis whose data is interior cell i
// (i itself and the ghost positions that map to it), with its mirror flag;
// at most 1 + 2 ge entries (ge <= NGW).
__device__ __forceinline__ int images(const DevGeo &G, int d, int i, int *pos, bool *flip) {
  int m = 0;
  pos[m] = i;
  flip[m++] = false;
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

__global__ void __launch_bounds__(PF_THREADS) k_prim_flags(DevGeo G, PrimArgs A, int ntx, int nty) {
  __shared__ float sw[PB3][8];   // deviations of the box cells (interior values at their positions)
  __shared__ float sp[PB3];      // their full pressure, background at the position's own height
  __shared__ float red[PF_THREADS / 32];
  const int tid = threadIdx.x;
  int t = blockIdx.x;
  const int tx = t % ntx;
  t /= ntx;
  const int ty = t % nty, tz = t / nty;
  const int o[3] = {tx * CT, ty * CT, tz * CT};

  // (1) primitives of the tile and its one-cell halo; a halo position beyond
  // a boundary takes its source cell's deviations, mirrored at walls
  for (int q = tid; q < PB3; q += PF_THREADS) {
    const int l[3] = {q % PB, (q / PB) % PB, q / (PB * PB)};
    int x[3], s[3];
    bool fl[3], in = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x[d] = o[d] - 1 + l[d];
      in = in && x[d] >= -1 && x[d] <= G.n[d];
      fl[d] = false;
    }
    if (!in) continue;
#pragma unroll
    for (int d = 0; d < 3; ++d) s[d] = cell_src(x[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]);
    float w[NW_MAX];
    cell_prims_mx(G, A.U, A.B, A.dU, A.dB, s[0], s[1], s[2], w, A.dflag);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (fl[d]) { w[W_VX + d] = -w[W_VX + d]; w[W_BX + d] = -w[W_BX + d]; }
#pragma unroll
    for (int v = 0; v < 8; ++v) sw[q][v] = w[v];
    sp[q] = w[W_P] + bg_cell_t<float>(G, x[2]).p;
  }
  __syncthreads();

  // (2) the tile's cells: W and auxiliaries at the cell and at every ghost
  // position that maps to it; raw flag; CFL rate
  float m = 0.0f;
  for (int q = tid; q < CT * CT * CT; q += PF_THREADS) {
    const int c[3] = {o[0] + q % CT, o[1] + (q / CT) % CT, o[2] + q / (CT * CT)};
    if (c[0] >= G.n[0] || c[1] >= G.n[1] || c[2] >= G.n[2]) continue;
    const int l0 = c[0] - o[0] + 1, l1 = c[1] - o[1] + 1, l2 = c[2] - o[2] + 1;
    const int b = (l2 * PB + l1) * PB + l0;
    float w[NW_MAX];
#pragma unroll
    for (int v = 0; v < 8; ++v) w[v] = sw[b][v];
    const BgT<float> bf = bg_cell_t<float>(G, c[2]);
    w[W_GE] = G.gammaf - bf.ge;
    w[W_GC] = G.gammaf - bf.gc;
    int px[1 + 2 * NGW], py[1 + 2 * NGW], pz[1 + 2 * NGW];   // a cell and at most 2 NGW ghost images per axis
    bool fx[1 + 2 * NGW], fy[1 + 2 * NGW], fz[1 + 2 * NGW];
    const int nx = images(G, 0, c[0], px, fx), ny = images(G, 1, c[1], py, fy), nz = images(G, 2, c[2], pz, fz);
    float4 *W4 = reinterpret_cast<float4 *>(A.W);
    for (int kz = 0; kz < nz; ++kz)
      for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < nx; ++kx) {
          float u[NW_MAX];
#pragma unroll
          for (int v = 0; v < 8; ++v) u[v] = w[v];
          const bool f3[3] = {fx[kx], fy[ky], fz[kz]};
#pragma unroll
          for (int d = 0; d < 3; ++d)
            if (f3[d]) { u[W_VX + d] = -u[W_VX + d]; u[W_BX + d] = -u[W_BX + d]; }
          const long p = widx(G, px[kx], py[ky], pz[kz]);
          W4[p] = make_float4(u[W_RHO], u[W_VX], u[W_VY], u[W_VZ]);
          W4[G.wtot + p] = make_float4(u[W_BX], u[W_BY], u[W_BZ], u[W_P]);
          write_aux(G, A.W, p, u);
        }
    if (G.eps_sf > 0.0) {   // raw flag: sum_d |P(+1) - P(-1)| / (eps P) > 1
      const float P0 = sp[b];
      float sum = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int sd = d == 0 ? 1 : (d == 1 ? PB : PB * PB);
        sum += fabsf(sp[b + sd] - sp[b - sd]);
      }
      A.raw[c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2])] = (sum / (G.epsf * P0) > 1.0f) ? 1 : 0;
    }
    if (A.cfl) m = fmaxf(m, dt_rate_w(G, w, c[2]));
  }
  if (A.cfl) {   // block maximum; non-negative floats order like their bits
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      float v = tid < PF_THREADS / 32 ? red[tid] : 0.0f;
      for (int s = 16; s > 0; s >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, s));
      if (tid == 0) atomicMax(A.fmax, __float_as_uint(v));
    }
  }
}

}  // namespace

cudaError_t ct_init() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaSuccess) return done;
  done = cudaFuncSetAttribute(k_ct_faces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ct_smem_bytes());
  return done;
}

// The Contact-CT / face-update kernel and the primitive / flag kernel of one
// mixed stage on the fused path (after the tile kernel).  In the last stage
// the primitives are those of U^(n+1) (no increments) and, unless fmax is
// null, the CFL rate of each cell is folded into fmax.
void launch_ct_prim(const DevGeo &G, const MixedBufs &M, bool first, bool last, double b, unsigned int *fmax,
                    cudaStream_t s, int *nl, Prof *prof) {
  StageMx S;
  S.U = M.U; S.B = M.B; S.dU = M.dU; S.dB = M.dB;
  S.first = first; S.last = last; S.b = (float)b; S.dt = M.dt;
  S.W = M.W; S.F[0] = M.F[0]; S.F[1] = M.F[1]; S.F[2] = M.F[2]; S.E = M.E;
  const int ntx = (G.n[0] + CT - 1) / CT, nty = (G.n[1] + CT - 1) / CT, ntz = (G.n[2] + CT - 1) / CT;
  const int nb = ntx * nty * ntz;
  PHL_LAUNCH(KC_EMF, prof, s, k_ct_faces<<<nb, CT_THREADS, ct_smem_bytes(), s>>>(G, S, ntx, nty));
  PrimArgs A;
  A.U = M.U; A.B = M.B;
  A.dU = last ? nullptr : M.dU;
  A.dB = last ? nullptr : M.dB;
  A.W = M.W; A.raw = M.raw; A.fmax = fmax; A.dflag = M.dflag; A.cfl = (last && fmax) ? 1 : 0;
  PHL_LAUNCH(KC_PRIM, prof, s, k_prim_flags<<<nb, PF_THREADS, 0, s>>>(G, A, ntx, nty));
  *nl += 2;
}

}  // namespace phl
