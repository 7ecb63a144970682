// phl_api.cu -- host implementation of the C ABI declared in include/phl.h.
//
// A phl_grid owns: the state (U^n and one stage buffer, cell and face
// fields), the device copies of the background profiles, the per-stage work
// arrays of the FP64 path, and three device scalars (dt, the running max of
// the CFL sum, an error word).  Every launch goes to the grid's stream; the
// time step can stay on the device so that a whole step needs no host sync.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include <utility>
#include <vector>

#include "phl.h"
#include "phl_internal.cuh"

using namespace phl;

namespace {

thread_local char g_err[512] = "";

phl_status fail(phl_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

phl_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? PHL_ENOMEM : PHL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace

namespace phl {
int set_error(int st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}
}  // namespace phl

struct phl_grid {
  phl_grid_desc desc;
  DevGeo G;
  cudaStream_t stream;
  // state
  double *U = nullptr, *U1 = nullptr, *B = nullptr, *B1 = nullptr, *T = nullptr, *T2 = nullptr;
  unsigned long long *niter = nullptr;   // Newton iteration counter (stellar EOS)
  // background and heating profiles
  double *bg = nullptr, *heat = nullptr;
  float *bgf = nullptr, *heatf = nullptr;
  // work
  double *W = nullptr, *F[3] = {nullptr, nullptr, nullptr}, *E = nullptr;
  uint8_t *raw = nullptr, *flag = nullptr;
  // mixed precision: FP32 increments and work arrays
  float *dUf = nullptr, *dBf = nullptr, *Wf = nullptr, *Ff[3] = {nullptr, nullptr, nullptr}, *Ef = nullptr;
  unsigned int *fmax = nullptr;         // [0]: the step's CFL maximum (three-launch path), [1]: phl_compute_dt
  unsigned int *anyraw = nullptr;       // fused path: some cell carries a raw shock flag (this stage)
  bool mixed = false;
  bool pipeline3 = false;               // fused mixed stage in three launches (phl_set_fused 201..209)
  bool w_valid = false;                 // W, raw flags and fmax[0] hold the current state's (three-launch path)
  // scalars
  double *dt = nullptr;
  unsigned long long *dmax = nullptr;
  int *dflag = nullptr;
  std::vector<void *> allocs;
  size_t bytes = 0;
  long steps = 0;
  double last_dt = 0.0;
  int launches_per_step = 0;
  Prof prof;
  int fused = 0;                        // mixed stage on the fused tile kernel: launch shape, 0 = off
  unsigned test_extra_tx = 0;           // phl_test_tile_wait_timeout
  double *stage_a = nullptr, *stage_b = nullptr;   // work arrays reused as host-transfer staging
  double *diff = nullptr;               // thermal-diffusion arrays (7 per cell), allocated on first use
  size_t stage_a_bytes = 0, stage_b_bytes = 0;
  alignas(64) unsigned char tmapW[128]; // its TMA descriptor of W
};

namespace {

template <typename T>
phl_status dalloc(phl_grid *g, T **p, size_t n) {
  void *q = nullptr;
  size_t bytes = n * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemset(q, 0, bytes);
  if (e != cudaSuccess) { cudaFree(q); return cuda_fail(e, "cudaMemset"); }
  g->allocs.push_back(q);
  g->bytes += bytes;
  *p = (T *)q;
  return PHL_OK;
}

// Copy between the ABI layout (dense) and the padded device layout.
// ext = (nx', ny', nz') extents of the field; to_dev selects the direction.
phl_status copy_field(phl_grid *g, double *dev, const double *abi_src, double *abi_dst, int ex, int ey, int ez,
                      bool to_dev) {
  const DevGeo &G = g->G;
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof(p));
  cudaPitchedPtr dptr = make_cudaPitchedPtr(dev, (size_t)G.sy * sizeof(double), (size_t)G.sy, (size_t)(G.sz / G.sy));
  if (to_dev) {
    p.srcPtr = make_cudaPitchedPtr((void *)abi_src, (size_t)ex * sizeof(double), (size_t)ex, (size_t)ey);
    p.dstPtr = dptr;
  } else {
    p.srcPtr = dptr;
    p.dstPtr = make_cudaPitchedPtr((void *)abi_dst, (size_t)ex * sizeof(double), (size_t)ex, (size_t)ey);
  }
  p.extent = make_cudaExtent((size_t)ex * sizeof(double), (size_t)ey, (size_t)ez);
  p.kind = cudaMemcpyDefault;
  CK(cudaMemcpy3DAsync(&p, g->stream), "cudaMemcpy3DAsync");
  return PHL_OK;
}

// Dense (ABI) <-> padded device layout of one field with extents (ex, ey, ez):
// one CTA per x-row, consecutive threads on consecutive elements.
__global__ void k_repitch(const double *__restrict__ src, double *__restrict__ dst, int ex, int ey, long sy, long sz,
                          int to_dev) {
  const long row = blockIdx.x;   // j + ey * k
  const long j = row % ey, k = row / ey;
  const long dense = row * ex, padded = j * sy + k * sz;
  for (int i = threadIdx.x; i < ex; i += blockDim.x) {
    if (to_dev) dst[padded + i] = src[dense + i];
    else dst[dense + i] = src[padded + i];
  }
}

// The state (nv cell fields and three face fields) between ABI arrays and the
// device layout.  Device arrays: one repitch kernel per field, straight from
// or into the caller's buffers.  Host arrays: one linear copy per array
// through the grid's work arrays (dead between steps), at full link bandwidth,
// plus the repitch kernels; pitched 3-D copies only when the work arrays are
// too small to hold the dense state.
phl_status state_io(phl_grid *g, double *cons, double *bx, double *by, double *bz, bool to_dev, bool host) {
  const DevGeo &G = g->G;
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const long nc = (long)nx * ny * nz;
  const long nf[3] = {(long)(nx + 1) * ny * nz, (long)nx * (ny + 1) * nz, (long)nx * ny * (nz + 1)};
  const int ext[3][3] = {{nx + 1, ny, nz}, {nx, ny + 1, nz}, {nx, ny, nz + 1}};
  double *face_abi[3] = {bx, by, bz};
  const size_t cons_bytes = (size_t)G.nv * nc * sizeof(double);
  const size_t face_bytes = (size_t)(nf[0] + nf[1] + nf[2]) * sizeof(double);
  const bool staged = host && g->stage_a && g->stage_b && cons_bytes <= g->stage_a_bytes && face_bytes <= g->stage_b_bytes;
  if (host && !staged) {   // pitched copies
    phl_status st;
    for (int v = 0; v < G.nv; ++v)
      if ((st = copy_field(g, g->U + v * G.plane, to_dev ? cons + v * nc : nullptr, to_dev ? nullptr : cons + v * nc,
                           nx, ny, nz, to_dev)) != PHL_OK)
        return st;
    for (int d = 0; d < 3; ++d)
      if ((st = copy_field(g, g->B + d * G.plane, to_dev ? face_abi[d] : nullptr, to_dev ? nullptr : face_abi[d],
                           ext[d][0], ext[d][1], ext[d][2], to_dev)) != PHL_OK)
        return st;
    return PHL_OK;
  }
  // the staging work arrays hold the next stage's primitives on the
  // three-launch path: reading the state through them retires those
  if (staged) g->w_valid = false;
  double *ca = staged ? g->stage_a : cons;
  double *fa[3];
  fa[0] = staged ? g->stage_b : bx;
  fa[1] = staged ? g->stage_b + nf[0] : by;
  fa[2] = staged ? g->stage_b + nf[0] + nf[1] : bz;
  if (staged && to_dev) {
    CK(cudaMemcpyAsync(ca, cons, cons_bytes, cudaMemcpyHostToDevice, g->stream), "copy state");
    for (int d = 0; d < 3; ++d)
      CK(cudaMemcpyAsync(fa[d], face_abi[d], nf[d] * sizeof(double), cudaMemcpyHostToDevice, g->stream), "copy B");
  }
  for (int v = 0; v < G.nv; ++v) {
    double *dev = g->U + v * G.plane;
    if (to_dev) k_repitch<<<(unsigned)((long)ny * nz), 256, 0, g->stream>>>(ca + v * nc, dev, nx, ny, G.sy, G.sz, 1);
    else k_repitch<<<(unsigned)((long)ny * nz), 256, 0, g->stream>>>(dev, ca + v * nc, nx, ny, G.sy, G.sz, 0);
  }
  for (int d = 0; d < 3; ++d) {
    double *dev = g->B + d * G.plane;
    const unsigned rows = (unsigned)((long)ext[d][1] * ext[d][2]);
    if (to_dev) k_repitch<<<rows, 256, 0, g->stream>>>(fa[d], dev, ext[d][0], ext[d][1], G.sy, G.sz, 1);
    else k_repitch<<<rows, 256, 0, g->stream>>>(dev, fa[d], ext[d][0], ext[d][1], G.sy, G.sz, 0);
  }
  CK(cudaGetLastError(), "repitch");
  if (staged && !to_dev) {
    CK(cudaMemcpyAsync(cons, ca, cons_bytes, cudaMemcpyDeviceToHost, g->stream), "copy state");
    for (int d = 0; d < 3; ++d)
      CK(cudaMemcpyAsync(face_abi[d], fa[d], nf[d] * sizeof(double), cudaMemcpyDeviceToHost, g->stream), "copy B");
  }
  return PHL_OK;
}

phl_status check_flags(phl_grid *g) {
  int f = 0;
  CK(cudaMemcpyAsync(&f, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream), "read flags");
  CK(cudaStreamSynchronize(g->stream), "sync");
  // a timeout is reported first: the tiles that gave up left their cells unwritten
  if (f & FLAG_TIMEOUT) return fail(PHL_ETIMEOUT, "a bounded device wait (tile copy) gave up");
  if (f & FLAG_NAN) return fail(PHL_ENAN, "non-finite value in the state");
  if (f & FLAG_NEG) return fail(PHL_ENEGATIVE, "non-positive density or pressure");
  if (f & FLAG_NEWTON) return fail(PHL_ENEWTON, "EOS Newton iteration did not converge");
  return PHL_OK;
}

void launch_dt(phl_grid *g, int *nl) {
  Prof *pf = g->prof.on ? &g->prof : nullptr;
  if (g->G.eos == PHL_EOS_STELLAR)
    launch_dt_stellar(g->G, g->mixed, g->U, g->B, g->T, g->dmax, g->dt, g->dflag, g->stream, nl, pf);
  else if (g->mixed)
    launch_dt_mixed(g->G, g->U, g->B, g->fmax + 1, g->dt, g->dflag, g->stream, nl, pf);
  else
    launch_dt_fp64(g->G, g->U, g->B, g->T, g->dmax, g->dt, g->dflag, g->stream, nl, pf);
}

void do_stage(phl_grid *g, const double *Uin, const double *Bin, double *Uout, double *Bout, double a,
              double b, int *nl, unsigned long long *cfl_dmax = nullptr) {
  StageBufs S;
  S.cfl_dmax = cfl_dmax;
  S.Uin = Uin; S.Bin = Bin; S.Ubase = g->U; S.Bbase = g->B;
  S.Uout = Uout; S.Bout = Bout; S.a = a; S.b = b; S.dt = g->dt;
  S.W = g->W; S.F[0] = g->F[0]; S.F[1] = g->F[1]; S.F[2] = g->F[2]; S.E = g->E;
  S.raw = g->raw; S.flag = g->flag; S.Tin = g->T; S.Tout = g->T2; S.dflag = g->dflag;
  launch_stage_fp64(g->G, S, g->stream, nl, g->prof.on ? &g->prof : nullptr);
  if (g->T) std::swap(g->T, g->T2);   // this stage's temperatures are the next guesses
}

}  // namespace

namespace phl {
GridView grid_view(phl_grid *g) {
  GridView v;
  v.G = &g->G;
  v.U = g->U; v.B = g->B;
  v.dU = g->dUf; v.dB = g->dBf; v.W = g->Wf;
  for (int k = 0; k < 3; ++k) v.F[k] = g->Ff[k];
  v.E = g->Ef;
  v.raw = g->raw; v.flag = g->flag; v.anyraw = g->anyraw;
  v.dt = g->dt; v.fmax = g->fmax + 1; v.dflag = g->dflag;
  v.w_valid = &g->w_valid;
  v.pipeline3 = g->pipeline3;
  v.stream = g->stream;
  v.steps = &g->steps;
  v.mixed = g->mixed;
  v.tmapW = g->fused ? g->tmapW : nullptr;
  v.fused = g->fused;
  return v;
}
}  // namespace phl

extern "C" {

const char *phl_last_error(void) { return g_err; }

phl_status phl_create_grid(const phl_grid_desc *d, phl_grid **out) {
  g_err[0] = 0;
  if (!d || !out) return fail(PHL_EINVAL, "null argument");
  *out = nullptr;
  for (int k = 0; k < 3; ++k) {
    if (d->n[k] < 1) return fail(PHL_EINVAL, "n[%d] = %d < 1", k, d->n[k]);
    if (d->n[k] > 1 && d->n[k] < 4) return fail(PHL_EINVAL, "active dimension %d needs n >= 4", k);
    if (!(d->hi[k] > d->lo[k])) return fail(PHL_EINVAL, "hi[%d] <= lo[%d]", k, k);
    for (int s = 0; s < 2; ++s)
      if (d->bc[k][s] < 0 || d->bc[k][s] > 2) return fail(PHL_EINVAL, "bad boundary condition");
    if ((d->bc[k][0] == PHL_PERIODIC) != (d->bc[k][1] == PHL_PERIODIC))
      return fail(PHL_EINVAL, "periodic boundaries must be periodic on both sides");
  }
  if (d->nspec < 0 || d->nspec > PHL_MAXSPEC) return fail(PHL_EINVAL, "nspec out of range");
  if (d->eos != PHL_EOS_IDEAL && d->eos != PHL_EOS_STELLAR) return fail(PHL_EINVAL, "bad eos");
  if (d->eos == PHL_EOS_STELLAR) {
    if (!d->eos_table) return fail(PHL_EINVAL, "stellar EOS needs an eos_table");
    if (d->nspec < 1) return fail(PHL_EINVAL, "stellar EOS needs mass fractions (nspec >= 1)");
    for (int l = 0; l < d->nspec; ++l)
      if (!(d->A[l] > 0.0) || !(d->Z[l] > 0.0)) return fail(PHL_EINVAL, "species A, Z must be positive");
  }
  if (d->use_mlp < 0 || d->use_mlp > 2) return fail(PHL_EINVAL, "use_mlp must be 0, 1 or 2");
  if (d->use_mlp && (d->eos != PHL_EOS_STELLAR || !d->mlp))
    return fail(PHL_EINVAL, "use_mlp needs the stellar EOS and desc.mlp");
  if (!(d->gamma > 1.0)) return fail(PHL_EINVAL, "gamma must exceed 1");
  if (!(d->cfl > 0.0)) return fail(PHL_EINVAL, "cfl must be positive");
  if (d->rk != 2 && d->rk != 3) return fail(PHL_EINVAL, "rk must be 2 or 3");
  if (d->riemann < 0 || d->riemann > 2) return fail(PHL_EINVAL, "bad riemann solver");
  if (d->recon != PHL_RECON_VANLEER && d->recon != PHL_RECON_PPH && d->recon != PHL_RECON_PQH)
    return fail(PHL_EINVAL, "bad reconstruction");
  if (d->precision != PHL_FP64 && d->precision != PHL_MIXED) return fail(PHL_EINVAL, "bad precision mode");
  if (d->bg_rho_c && (!d->bg_p_c || !d->bg_rho_f || !d->bg_p_f))
    return fail(PHL_EINVAL, "incomplete background profiles");
  const long ncell = (long)d->n[0] * d->n[1] * d->n[2];
  if (ncell > (1L << 31)) return fail(PHL_EINVAL, "grid too large");

  phl_grid *g = new phl_grid();
  g->desc = *d;
  g->stream = (cudaStream_t)d->stream;
  DevGeo &G = g->G;
  memset(&G, 0, sizeof(G));
  for (int k = 0; k < 3; ++k) {
    G.n[k] = d->n[k];
    G.act[k] = d->n[k] > 1;
    G.bc[k][0] = d->bc[k][0];
    G.bc[k][1] = d->bc[k][1];
    G.dx[k] = (d->hi[k] - d->lo[k]) / d->n[k];
    G.idx[k] = 1.0 / G.dx[k];
    G.ge[k] = G.act[k] ? (d->recon == PHL_RECON_PQH ? NGW + 1 : NGW) : 0;   // PQH: five-cell stencil
    G.g[k] = d->g[k];
  }
  const long pitch = ((long)d->n[0] + 1 + 3) / 4 * 4;
  G.sy = pitch;
  G.sz = pitch * (d->n[1] + 1);
  G.plane = G.sz * (d->n[2] + 1);
  G.wy = d->n[0] + 2L * G.ge[0] + 1;
  G.wz = G.wy * (d->n[1] + 2L * G.ge[1] + 1);
  G.wtot = G.wz * (d->n[2] + 2L * G.ge[2] + 1);
  // FP32 W interleaving: 8 values per cell for an ideal gas without species
  // (rho, u, B, P deviations), else the padded component count (gamma_e,
  // gamma_c, mass fractions)
  G.wstr = (d->eos == PHL_EOS_IDEAL && d->nspec == 0) ? 8 : (d->nspec == 0 ? 12 : 16);
  G.nspec = d->nspec;
  G.nv = 5 + d->nspec;
  G.nw = 10 + d->nspec;
  G.nf = 8 + d->nspec;
  G.eos = d->eos;
  G.gamma = d->gamma;
  G.riemann = d->riemann;
  G.recon = d->recon;
  G.eps_sf = d->eps_sf;
  G.mach_thr = d->mach_thr;
  G.cfl = d->cfl;
  {   // power-of-two unit scales of the mixed form's FP32 quantities
    double rho_ref = 1.0, p_ref = 1.0, dx_min = 0.0;
    if (d->bg_rho_c && d->bg_p_c) {
      rho_ref = p_ref = 0.0;
      for (int k = 0; k < d->n[2] + 2 * BG_NG; ++k) {
        rho_ref = std::max(rho_ref, std::fabs(d->bg_rho_c[k]));
        p_ref = std::max(p_ref, std::fabs(d->bg_p_c[k]));
      }
      if (!(rho_ref > 0.0) || !(p_ref > 0.0)) rho_ref = p_ref = 1.0;
    }
    for (int k = 0; k < 3; ++k)
      if (G.act[k]) dx_min = dx_min > 0.0 ? std::min(dx_min, G.dx[k]) : G.dx[k];
    if (!(dx_min > 0.0)) dx_min = 1.0;
    const int ea = (int)std::lround(0.5 * std::log2(p_ref)), eb = (int)std::lround(0.5 * std::log2(rho_ref));
    const double P_s = std::ldexp(1.0, 2 * ea), rho_s = std::ldexp(1.0, 2 * eb);
    const double v_s = std::ldexp(1.0, ea - eb), B_s = std::ldexp(1.0, ea);
    const double L_s = std::ldexp(1.0, (int)std::lround(std::log2(dx_min)));
    const double t_s = L_s / v_s;
    G.sc_rho = rho_s; G.sc_m = rho_s * v_s; G.sc_e = P_s; G.sc_b = B_s; G.sc_t = t_s;
    G.e_rho = 2 * eb; G.e_m = ea + eb; G.e_e = 2 * ea; G.e_b = ea;
    G.e_t = (int)std::lround(std::log2(dx_min)) - (ea - eb);
    G.isc_rho = 1.0 / rho_s; G.isc_m = 1.0 / (rho_s * v_s); G.isc_e = 1.0 / P_s; G.isc_b = 1.0 / B_s;
    G.isc_t = 1.0 / t_s; G.isc_v = 1.0 / v_s;
    for (int k = 0; k < 3; ++k) {
      G.idxf[k] = (float)(G.idx[k] * L_s);
      G.gf[k] = (float)(d->g[k] * t_s * t_s / L_s);
    }
  }
  G.gammaf = (float)d->gamma;
  G.gm1f = (float)(d->gamma - 1.0);
  G.machf = (float)d->mach_thr;
  G.epsf = (float)d->eps_sf;
  G.newton_tol = d->newton_tol > 0.0 ? d->newton_tol : 1e-11;
  G.newton_maxit = d->newton_maxit > 0 ? d->newton_maxit : 50;
  for (int l = 0; l < PHL_NSPEC_MAX; ++l) {
    G.Acomp[l] = d->A[l];
    G.Zcomp[l] = d->Z[l];
    G.iAcomp[l] = d->A[l] > 0.0 ? 1.0 / d->A[l] : 0.0;
    G.ZoAcomp[l] = d->A[l] > 0.0 ? d->Z[l] / d->A[l] : 0.0;
  }
  if (d->eos == PHL_EOS_STELLAR) G.tab = *eos_table_view(d->eos_table);
  if (d->use_mlp) {
    G.use_mlp = d->use_mlp;
    G.mlp = mlp_view(d->mlp);
  }

  phl_status st = PHL_OK;
#define AL(p, n)                                  \
  do {                                            \
    st = dalloc(g, p, (size_t)(n));               \
    if (st != PHL_OK) { phl_destroy(g); return st; } \
  } while (0)
  g->mixed = d->precision == PHL_MIXED;
  AL(&g->U, G.nv * G.plane);
  AL(&g->B, 3 * G.plane);
  if (!g->mixed) {
    AL(&g->U1, G.nv * G.plane);
    AL(&g->B1, 3 * G.plane);
    AL(&g->W, (long)G.nw * G.wtot);
    for (int k = 0; k < 3; ++k)
      if (G.act[k]) AL(&g->F[k], (long)(G.nf + 1) * G.wtot);   // + contact direction
    AL(&g->E, 3 * G.wtot);
    g->stage_a = g->W;
    g->stage_a_bytes = (size_t)G.nw * G.wtot * sizeof(double);
    g->stage_b = g->F[0];
    g->stage_b_bytes = g->F[0] ? (size_t)(G.nf + 1) * G.wtot * sizeof(double) : 0;
  } else {
    AL(&g->dUf, G.nv * G.plane);
    AL(&g->dBf, 3 * G.plane);
    AL(&g->Wf, (long)(G.wstr + NAUX) * G.wtot);   // interleaved W + auxiliary planes
    for (int k = 0; k < 3; ++k)
      if (G.act[k]) AL(&g->Ff[k], (long)(G.nf + 1) * G.wtot);
    AL(&g->Ef, 3 * G.wtot);
    AL(&g->fmax, 2);
    g->stage_a = (double *)g->Wf;
    g->stage_a_bytes = (size_t)(G.wstr + NAUX) * G.wtot * sizeof(float);
    g->stage_b = (double *)g->Ff[0];
    g->stage_b_bytes = g->Ff[0] ? (size_t)(G.nf + 1) * G.wtot * sizeof(float) : 0;
    if (fused_stage_ok(G)) {
      if (make_fused_tmap(G, g->Wf, g->tmapW) != PHL_OK) { phl_destroy(g); return PHL_ECUDA; }
      const cudaError_t e = fused_init();
      if (e != cudaSuccess) { phl_destroy(g); return cuda_fail(e, "fused stage set-up"); }
      g->fused = PHL_FUSED_DEFAULT;
    }
  }
  AL(&g->raw, 2 * ncell);   // raw flags + one dilation pass buffer
  AL(&g->anyraw, 1);
  if (d->eos == PHL_EOS_STELLAR) {
    AL(&g->T, G.plane);
    AL(&g->T2, G.plane);
    AL(&g->niter, 1);
    G.niter = g->niter;
    if (g->mixed) {   // each cell's last inversion (eos::Pred): the next stage's first guess
      AL(&G.pred, 8 * G.plane);
    }
  }
  AL(&g->flag, G.wtot);
  AL(&g->dt, 1);
  AL(&g->dmax, 1);
  AL(&g->dflag, 1);
  const int nz = d->n[2];
  const long nbg = 9L * (nz + 2 * BG_NG + 1);   // 8 profiles + E_hat at centres
  AL(&g->bg, nbg);
  AL(&g->bgf, nbg);
  if (d->bg_rho_c) {
    std::vector<double> h(nbg, 0.0);
    const long L = nz + 2 * BG_NG + 1;
    const double *src[8] = {d->bg_rho_c, d->bg_p_c, d->bg_rho_f, d->bg_p_f,
                            d->bg_ge_c, d->bg_gc_c, d->bg_ge_f, d->bg_gc_f};
    for (int q = 0; q < 8; ++q) {
      if (!src[q]) continue;
      const long cnt = (q == 2 || q == 3 || q == 6 || q == 7) ? L : L - 1;
      memcpy(&h[q * L], src[q], cnt * sizeof(double));
    }
    for (long q = 0; q < L - 1; ++q) h[8 * L + q] = d->bg_p_c[q] / (d->gamma - 1.0);   // E_hat
    const bool stellar_bg = d->eos == PHL_EOS_STELLAR && !d->bg_ge_c;
    const bool gam = d->bg_ge_c || stellar_bg;
    if (stellar_bg) {   // gamma_e, gamma_c, E_hat of the background from the device EOS
      cudaError_t e0 = cudaMemcpy(g->bg, h.data(), nbg * sizeof(double), cudaMemcpyHostToDevice);
      if (e0 == cudaSuccess) e0 = stellar_background(G, (int)L, g->bg, d->bg_X);
      if (e0 == cudaSuccess) e0 = cudaMemcpy(h.data(), g->bg, nbg * sizeof(double), cudaMemcpyDeviceToHost);
      if (e0 != cudaSuccess) { phl_destroy(g); return cuda_fail(e0, "stellar background"); }
    }
    std::vector<float> hf(nbg);
    for (long q = 0; q < nbg; ++q) {   // rho rows 0, 2; pressure rows 1, 3, 8 scaled
      const long row = q / L;
      const double sc = (row == 0 || row == 2) ? G.isc_rho : ((row == 1 || row == 3 || row == 8) ? G.isc_e : 1.0);
      hf[q] = (float)(h[q] * sc);
    }
    cudaError_t e = cudaMemcpy(g->bg, h.data(), nbg * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { phl_destroy(g); return cuda_fail(e, "copy background"); }
    e = cudaMemcpy(g->bgf, hf.data(), nbg * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { phl_destroy(g); return cuda_fail(e, "copy background"); }
    G.bgf_rho_c = g->bgf; G.bgf_p_c = g->bgf + L; G.bgf_rho_f = g->bgf + 2 * L; G.bgf_p_f = g->bgf + 3 * L;
    G.bgf_ge_c = gam ? g->bgf + 4 * L : nullptr;
    G.bgf_gc_c = gam ? g->bgf + 5 * L : nullptr;
    G.bgf_ge_f = gam ? g->bgf + 6 * L : nullptr;
    G.bgf_gc_f = gam ? g->bgf + 7 * L : nullptr;
    G.bg_e_c = g->bg + 8 * L;
    G.has_bg = 1;
    G.bg_rho_c = g->bg; G.bg_p_c = g->bg + L; G.bg_rho_f = g->bg + 2 * L; G.bg_p_f = g->bg + 3 * L;
    G.bg_ge_c = gam ? g->bg + 4 * L : nullptr;
    G.bg_gc_c = gam ? g->bg + 5 * L : nullptr;
    G.bg_ge_f = gam ? g->bg + 6 * L : nullptr;
    G.bg_gc_f = gam ? g->bg + 7 * L : nullptr;
  }
  if (d->heat) {
    AL(&g->heat, nz);
    AL(&g->heatf, nz);
    std::vector<float> hf(nz);
    for (int q = 0; q < nz; ++q) hf[q] = (float)(d->heat[q] * G.sc_t * G.isc_e);   // scaled units
    cudaError_t e = cudaMemcpy(g->heat, d->heat, nz * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->heatf, hf.data(), nz * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { phl_destroy(g); return cuda_fail(e, "copy heating"); }
    G.heat = g->heat;
    G.heatf = g->heatf;
  }
#undef AL
  *out = g;
  return PHL_OK;
}

void phl_destroy(phl_grid *g) {
  if (!g) return;
  g->prof.release();
  for (void *p : g->allocs) cudaFree(p);
  delete g;
}

phl_status phl_set_stream(phl_grid *g, void *stream) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  g->stream = (cudaStream_t)stream;
  return PHL_OK;
}

phl_status phl_set_state(phl_grid *g, const double *cons, const double *bx, const double *by,
                         const double *bz, const double *T, int where) {
  if (g) g->w_valid = false;   // the state changes from outside: the next step forms W again
  if (!g || !cons || !bx || !by || !bz) return fail(PHL_EINVAL, "null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return fail(PHL_EINVAL, "bad 'where'");
  const DevGeo &G = g->G;
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const long nc = (long)nx * ny * nz;
  phl_status st;
  (void)nc;
  if ((st = state_io(g, const_cast<double *>(cons), const_cast<double *>(bx), const_cast<double *>(by),
                     const_cast<double *>(bz), true, where == PHL_HOST)) != PHL_OK)
    return st;
  if (g->T) {
    if (T) {
      if ((st = copy_field(g, g->T, T, nullptr, nx, ny, nz, true)) != PHL_OK) return st;
    } else {   // no guesses: the network's (use_mlp) or the table's mid-range temperature
      CK(cudaMemsetAsync(g->T, 0, G.plane * sizeof(double), g->stream), "clear T");
    }
  }
  if (G.pred)   // no inversion record (phl_set_eos_record restores one)
    CK(cudaMemsetAsync(G.pred, 0, 8 * G.plane * sizeof(double), g->stream), "clear the inversion record");
  CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream), "reset flags");
  if (where == PHL_HOST) CK(cudaStreamSynchronize(g->stream), "sync");
  return PHL_OK;
}

phl_status phl_get_state(phl_grid *g, double *cons, double *bx, double *by, double *bz, double *T, int where) {
  if (!g || !cons || !bx || !by || !bz) return fail(PHL_EINVAL, "null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return fail(PHL_EINVAL, "bad 'where'");
  const DevGeo &G = g->G;
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const long nc = (long)nx * ny * nz;
  phl_status st;
  (void)nc;
  if ((st = state_io(g, cons, bx, by, bz, false, where == PHL_HOST)) != PHL_OK) return st;
  if (g->T && T)
    if ((st = copy_field(g, g->T, nullptr, T, nx, ny, nz, false)) != PHL_OK) return st;
  return check_flags(g);
}

phl_status phl_get_eos_record(phl_grid *g, double *rec, int where) {
  if (!g || !rec) return fail(PHL_EINVAL, "phl_get_eos_record: null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return fail(PHL_EINVAL, "bad 'where'");
  const DevGeo &G = g->G;
  if (!G.pred) return fail(PHL_EINVAL, "phl_get_eos_record: no record (mixed stellar grids only)");
  const long nc = (long)G.n[0] * G.n[1] * G.n[2];
  phl_status st;
  for (int q = 0; q < 8; ++q)
    if ((st = copy_field(g, G.pred + q * G.plane, nullptr, rec + q * nc, G.n[0], G.n[1], G.n[2], false)) != PHL_OK)
      return st;
  if (where == PHL_HOST) CK(cudaStreamSynchronize(g->stream), "sync");
  return PHL_OK;
}

phl_status phl_set_eos_record(phl_grid *g, const double *rec, int where) {
  if (!g || !rec) return fail(PHL_EINVAL, "phl_set_eos_record: null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return fail(PHL_EINVAL, "bad 'where'");
  const DevGeo &G = g->G;
  if (!G.pred) return fail(PHL_EINVAL, "phl_set_eos_record: no record (mixed stellar grids only)");
  const long nc = (long)G.n[0] * G.n[1] * G.n[2];
  phl_status st;
  for (int q = 0; q < 8; ++q)
    if ((st = copy_field(g, G.pred + q * G.plane, rec + q * nc, nullptr, G.n[0], G.n[1], G.n[2], true)) != PHL_OK)
      return st;
  if (where == PHL_HOST) CK(cudaStreamSynchronize(g->stream), "sync");
  return PHL_OK;
}

phl_status phl_set_state_prim(phl_grid *g, const double *prim, const double *bx, const double *by,
                              const double *bz, int where) {
  if (g) g->w_valid = false;   // the state changes from outside: the next step forms W again
  if (!g || !prim || !bx || !by || !bz) return fail(PHL_EINVAL, "null argument");
  if (where != PHL_HOST && where != PHL_DEVICE) return fail(PHL_EINVAL, "bad 'where'");
  const DevGeo &G = g->G;
  const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
  const long nc = (long)nx * ny * nz;
  phl_status st;
  if ((st = copy_field(g, g->B, bx, nullptr, nx + 1, ny, nz, true)) != PHL_OK) return st;
  if ((st = copy_field(g, g->B + G.plane, by, nullptr, nx, ny + 1, nz, true)) != PHL_OK) return st;
  if ((st = copy_field(g, g->B + 2 * G.plane, bz, nullptr, nx, ny, nz + 1, true)) != PHL_OK) return st;
  const double *dprim = prim;
  double *tmp = nullptr;
  if (where == PHL_HOST) {
    CK(cudaMalloc(&tmp, (size_t)(5 + G.nspec) * nc * sizeof(double)), "alloc primitive staging");
    cudaError_t e = cudaMemcpyAsync(tmp, prim, (size_t)(5 + G.nspec) * nc * sizeof(double), cudaMemcpyHostToDevice,
                                    g->stream);
    if (e != cudaSuccess) { cudaFree(tmp); return cuda_fail(e, "copy primitives"); }
    dprim = tmp;
  }
  CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream), "reset flags");
  launch_prim_to_cons(G, dprim, g->U, g->B, g->T, g->dflag, g->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && G.pred)   // no inversion record
    e = cudaMemsetAsync(G.pred, 0, 8 * G.plane * sizeof(double), g->stream);
  if (tmp) {
    cudaStreamSynchronize(g->stream);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return cuda_fail(e, "primitive -> conserved");
  return check_flags(g);
}

phl_status phl_compute_dt(phl_grid *g, double *dt_out) {
  if (!g || !dt_out) return fail(PHL_EINVAL, "null argument");
  int nl = 0;
  launch_dt(g, &nl);
  CK(cudaGetLastError(), "launch dt");
  CK(cudaMemcpyAsync(dt_out, g->dt, sizeof(double), cudaMemcpyDeviceToHost, g->stream), "read dt");
  phl_status st = check_flags(g);
  if (st != PHL_OK) return st;
  g->last_dt = *dt_out;
  return PHL_OK;
}

phl_status phl_step(phl_grid *g, double dt, int nsteps) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  if (nsteps < 0) return fail(PHL_EINVAL, "nsteps < 0");
  for (int s = 0; s < nsteps; ++s) {
    int nl = 0;
    const bool three = g->mixed && g->fused && g->pipeline3;
    const bool primed = three && g->w_valid;
    if (primed) {   // the previous step's last stage left the CFL maximum of this state
      launch_dt_mixed_from_max(g->G, dt, g->fmax, g->dt, g->stream, &nl, g->prof.on ? &g->prof : nullptr);
    } else if (dt > 0.0) {
      if (three) launch_dt_mixed_from_max(g->G, dt, g->fmax, g->dt, g->stream, &nl, g->prof.on ? &g->prof : nullptr);
      else {
        launch_set_scalar(g->dt, dt, g->stream, g->prof.on ? &g->prof : nullptr);
        ++nl;
      }
    } else if (g->G.eos != PHL_EOS_STELLAR && !(g->mixed && !three)) {
      launch_dt(g, &nl);
      if (three) CK(cudaMemsetAsync(g->fmax, 0, sizeof(unsigned int), g->stream), "clear CFL maximum");
    }
    // ideal-gas mixed form (six launches per stage) with the device CFL step:
    // the first stage's primitives of U^n give it
    unsigned int *cfl_fmax = (g->mixed && !three && g->G.eos != PHL_EOS_STELLAR && !(dt > 0.0)) ? g->fmax + 1
                                                                                                 : nullptr;
    // stellar EOS with the device CFL step: the first stage's inversion gives it
    unsigned long long *cfl_dmax = (g->G.eos == PHL_EOS_STELLAR && !(dt > 0.0)) ? g->dmax : nullptr;
    if (g->mixed) {
      const double bs3[3] = {1.0, 0.25, 2.0 / 3.0}, bs2[2] = {1.0, 0.5};
      const int ns = g->desc.rk == 2 ? 2 : 3;
      MixedBufs M;
      M.U = g->U; M.B = g->B; M.dU = g->dUf; M.dB = g->dBf; M.W = g->Wf;
      M.F[0] = g->Ff[0]; M.F[1] = g->Ff[1]; M.F[2] = g->Ff[2]; M.E = g->Ef;
      M.raw = g->raw; M.flag = g->flag; M.dt = g->dt; M.dflag = g->dflag;
      M.tmapW = g->fused ? g->tmapW : nullptr;
      M.fused_variant = g->fused;
      M.test_extra_tx = g->test_extra_tx;
      M.pipeline3 = three;
      M.primed = primed;
      M.fmax = g->fmax;
      M.cfl_dmax = cfl_dmax;
      M.cfl_fmax = cfl_fmax;
      M.anyraw = g->anyraw;
      for (int st = 0; st < ns; ++st) {
        M.Tin = g->T;
        M.Tout = g->T2;
        launch_stage_mixed(g->G, M, st, ns, ns == 2 ? bs2[st] : bs3[st], g->stream, &nl,
                           g->prof.on ? &g->prof : nullptr);
        if (g->T) std::swap(g->T, g->T2);
      }
    } else if (g->desc.rk == 2) {
      do_stage(g, g->U, g->B, g->U1, g->B1, 0.0, 1.0, &nl, cfl_dmax);
      do_stage(g, g->U1, g->B1, g->U, g->B, 0.5, 0.5, &nl);
    } else {
      do_stage(g, g->U, g->B, g->U1, g->B1, 0.0, 1.0, &nl, cfl_dmax);
      do_stage(g, g->U1, g->B1, g->U1, g->B1, 0.75, 0.25, &nl);
      do_stage(g, g->U1, g->B1, g->U, g->B, 1.0 / 3.0, 2.0 / 3.0, &nl);
    }
    CK(cudaGetLastError(), "launch stage");
    g->launches_per_step = nl;
    ++g->steps;
    if (three) g->w_valid = true;
  }
  return PHL_OK;
}

phl_status phl_check(phl_grid *g) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  return check_flags(g);
}


phl_status phl_get_stats(phl_grid *g, phl_stats *st) {
  if (!g || !st) return fail(PHL_EINVAL, "null argument");
  memset(st, 0, sizeof(*st));
  st->steps = g->steps;
  st->last_dt = g->last_dt;
  int f = 0;
  CK(cudaMemcpyAsync(&f, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream), "read flags");
  CK(cudaStreamSynchronize(g->stream), "sync");
  st->device_flags = f;
  st->kernels_per_step = g->launches_per_step;
  st->device_bytes = g->bytes;
  if (g->niter) {
    unsigned long long it = 0;
    CK(cudaMemcpy(&it, g->niter, sizeof(it), cudaMemcpyDeviceToHost), "read Newton iterations");
    st->newton_iters = (long)it;
  }
  return PHL_OK;
}

phl_status phl_set_timing(phl_grid *g, int on) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  g->prof.on = on != 0;
  return PHL_OK;
}

phl_status phl_kernel_times(phl_grid *g, phl_kernel_time *out, int max, int *n, int reset) {
  if (!g || !n || (max > 0 && !out)) return fail(PHL_EINVAL, "null argument");
  CK(g->prof.fold(), "fold kernel timings");
  int k = 0;
  for (int c = 0; c < KC_COUNT; ++c) {
    if (g->prof.cnt[c] == 0) continue;
    if (k < max) {
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, kclass_name(c), sizeof(out[k].name) - 1);
      out[k].launches = g->prof.cnt[c];
      out[k].ms = g->prof.ms[c];
    }
    ++k;
  }
  *n = k;
  if (reset)
    for (int c = 0; c < KC_COUNT; ++c) { g->prof.cnt[c] = 0; g->prof.ms[c] = 0.0; }
  return PHL_OK;
}

phl_status phl_set_fused(phl_grid *g, int on) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  g->w_valid = false;
  // 201..209: the same launch shapes with the stage in three launches
  const bool three = on > 200;
  if (three) on -= 200;
  if (on < 0 || on > PHL_FUSED_SHAPES) return fail(PHL_EINVAL, "fused launch shape must be 0..%d (or 201..%d)",
                                                   PHL_FUSED_SHAPES, 200 + PHL_FUSED_SHAPES);
  if (!on) { g->fused = 0; return PHL_OK; }
  if (!g->mixed || !fused_stage_ok(g->G))
    return fail(PHL_EUNSUPPORTED, "the fused stage needs the mixed form, an ideal gas without species and 3 active dimensions");
  if (make_fused_tmap(g->G, g->Wf, g->tmapW) != PHL_OK) return PHL_ECUDA;
  g->fused = on == 1 ? PHL_FUSED_DEFAULT : on;
  g->pipeline3 = three;
  return PHL_OK;
}

phl_status phl_diffuse(phl_grid *g, const phl_diffusion *p, double dt, int max_stages, int *nsts_out) {
  if (g) g->w_valid = false;   // the state changes from outside: the next step forms W again
  if (!g || !p) return fail(PHL_EINVAL, "null argument");
  if (g->G.eos != PHL_EOS_IDEAL) return fail(PHL_EUNSUPPORTED, "thermal diffusion is built for the ideal gas");
  if (!(p->k0 >= 0.0) || !(p->cv > 0.0) || p->nT < 0 || p->nT > 4 || p->nR < 0 || p->nR > 2 || !(dt > 0.0) ||
      max_stages < 3 || p->precision < PHL_DIFF_GRID || p->precision > PHL_DIFF_MIXED || p->tile_z < 0 ||
      p->tile_z > 4096 || (p->delta_T != 0 && p->delta_T != 1))
    return fail(PHL_EINVAL, "bad diffusion parameters");
  if (p->delta_T && !g->G.bg_rho_c)
    return fail(PHL_EINVAL, "diffusing the deviation from the background temperature needs a background");
  if (!g->diff) {
    const long nc = (long)g->G.n[0] * g->G.n[1] * g->G.n[2];
    phl_status st = dalloc(g, &g->diff, (size_t)11 * nc + 8 + (size_t)g->G.n[2]);
    if (st != PHL_OK) return st;
  }
  const bool mixed = p->precision == PHL_DIFF_MIXED || (p->precision == PHL_DIFF_GRID && g->mixed);
  if (mixed && (double)g->G.n[0] * g->G.n[1] * g->G.n[2] >= 4294967295.0)
    return fail(PHL_EUNSUPPORTED, "mixed thermal diffusion indexes cells with 32 bits (fewer than 2^32 - 1 cells)");
  int ns = 0, nl = 0;
  const cudaError_t e = launch_diffuse(g->G, g->U, g->B, *p, dt, max_stages, mixed, g->diff, g->dflag, g->stream,
                                       &ns, &nl);
  if (nsts_out) *nsts_out = ns;
  if (e == cudaErrorInvalidValue && ns > max_stages) {
    cudaGetLastError();
    return fail(PHL_EINVAL, "thermal diffusion needs %d stages, more than max_stages = %d", ns, max_stages);
  }
  if (e != cudaSuccess) return cuda_fail(e, "thermal diffusion");
  return PHL_OK;
}

phl_status phl_test_tile_wait_timeout(phl_grid *g, int on) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  g->w_valid = false;
  if (on && !g->fused) return fail(PHL_EUNSUPPORTED, "the grid does not run the fused tile kernel");
  g->test_extra_tx = on ? 16u : 0u;
  return PHL_OK;
}

phl_status phl_test_prims(phl_grid *g, int form, int increments, float *w_out, long cap, float *rate_out) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  if (!w_out) return fail(PHL_EINVAL, "null output");
  if (form < 0 || form > 3) return fail(PHL_EINVAL, "form must be 0..3");
  if (!g->mixed || g->G.eos != PHL_EOS_IDEAL)
    return fail(PHL_EUNSUPPORTED, "primitive forms exist for mixed ideal-gas grids only");
  if ((form & 1) && !prim_pairs_ok(g->G)) return fail(PHL_EUNSUPPORTED, "the grid does not admit the pair form");
  const long nw = (long)(g->G.wstr + NAUX) * g->G.wtot;
  if (cap < nw) return fail(PHL_EINVAL, "output holds fewer floats than W and its auxiliary planes");
  g->w_valid = false;
  const bool inc = increments && form < 2;
  CK(cudaMemsetAsync(g->Wf, 0, nw * sizeof(float), g->stream), "clear W");
  CK(cudaMemsetAsync(g->fmax + 1, 0, sizeof(unsigned int), g->stream), "clear rate");
  CK(launch_prims_form(g->G, g->U, g->B, inc ? g->dUf : nullptr, inc ? g->dBf : nullptr, g->Wf, g->dflag, form,
                       g->fmax + 1, g->stream),
     "primitives");
  CK(cudaMemcpyAsync(w_out, g->Wf, nw * sizeof(float), cudaMemcpyDeviceToHost, g->stream), "read W");
  unsigned int bits = 0;
  CK(cudaMemcpyAsync(&bits, g->fmax + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, g->stream), "read rate");
  CK(cudaStreamSynchronize(g->stream), "sync");
  if (rate_out) memcpy(rate_out, &bits, sizeof(float));
  return PHL_OK;
}

phl_status phl_test_raw_flags(phl_grid *g, int form, unsigned char *out, long cap, int *any_out) {
  if (!g) return fail(PHL_EINVAL, "null grid");
  if (!out) return fail(PHL_EINVAL, "null output");
  if (form < 0 || form > 1) return fail(PHL_EINVAL, "form must be 0 or 1");
  if (!g->mixed) return fail(PHL_EUNSUPPORTED, "raw-flag forms exist for mixed grids only");
  if (form == 1 && !(g->G.act[0] && g->G.n[0] % 4 == 0))
    return fail(PHL_EUNSUPPORTED, "the four-cell form needs n_x a multiple of 4");
  const long nc = (long)g->G.n[0] * g->G.n[1] * g->G.n[2];
  if (cap < nc) return fail(PHL_EINVAL, "output holds fewer bytes than cells");
  g->w_valid = false;
  CK(cudaMemsetAsync(g->raw, 0, nc, g->stream), "clear flags");
  CK(cudaMemsetAsync(g->anyraw, 0, sizeof(unsigned int), g->stream), "clear vote");
  CK(launch_raw_flags_form(g->G, g->Wf, g->raw, form, g->anyraw, g->stream), "raw flags");
  CK(cudaMemcpyAsync(out, g->raw, nc, cudaMemcpyDeviceToHost, g->stream), "read flags");
  unsigned int any = 0;
  CK(cudaMemcpyAsync(&any, g->anyraw, sizeof(unsigned int), cudaMemcpyDeviceToHost, g->stream), "read vote");
  CK(cudaStreamSynchronize(g->stream), "sync");
  if (any_out) *any_out = (int)any;
  return PHL_OK;
}

phl_status phl_test_prims_size(phl_grid *g, long *nfloat) {
  if (!g || !nfloat) return fail(PHL_EINVAL, "null argument");
  *nfloat = g->mixed ? (long)(g->G.wstr + NAUX) * g->G.wtot : 0;
  return PHL_OK;
}

phl_status phl_dt_device_ptr(phl_grid *g, const double **ptr) {
  if (!g || !ptr) return fail(PHL_EINVAL, "null argument");
  *ptr = g->dt;
  return PHL_OK;
}

}  // extern "C"
