// ensemble.cu -- batched ensemble of independent boxes (uneven sizes) in the
// mixed form: one persistent cooperative launch per RK stage runs every step
// of the stage for every box, phase after phase, with a grid-wide barrier
// between phases:
//   [stage 0: CFL rate per box -> per-box dt]  primitives -> raw shock flags
//   -> dilation x, y, z -> flag expansion -> fluxes (3 directions) ->
//   Contact-CT EMFs -> cell and face updates.
// Work items of a phase are the concatenation of all boxes' items; a block
// strides through them and finds an item's box by binary search over the
// phase's prefix sums.  The step (3 launches) is captured once as a CUDA graph
// and replayed; the launch shape (block size, blocks per SM) is picked by
// timing the candidates (phl_ensemble_autotune).  A second mode launches each
// phase on its own (all boxes per launch, each phase with its own register
// allocation); a third gives every box its own chain of per-kernel launches
// on concurrent streams (fork/join).  The step is one graph in every mode;
// the autotuner times all of them.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mixed_common.cuh"
#include "phl.h"

namespace cg = cooperative_groups;

namespace phl {
using namespace stage;
namespace {

enum { PH_DT, PH_DTFIN, PH_PRIM, PH_RAW, PH_DIL0, PH_DIL1, PH_DIL2, PH_EXP, PH_FLUX, PH_EMF, PH_UPD, NPH };

struct EnsRec {
  DevGeo G;
  double *U, *B;
  float *dU, *dB, *W, *F[3], *E;
  uint8_t *raw, *flag;
  uint8_t *dil_in[3], *dil_out[3], *dil_final;
  double *dt;
  unsigned int *fmax;
  int *dflag;
  Box b_int, b_work, b_exp, b_flux[3], b_emf[3], b_face[3];
};

struct EnsArgs {
  const EnsRec *rec;
  const long *pref;   // [NPH][nbox + 1]
  int nbox;
  int stage, nstages;
  float b;
};

__device__ __forceinline__ int find_box(const long *p, int nbox, long w) {
  int lo = 0, hi = nbox;   // p[lo] <= w < p[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ StageMx stage_bufs(const EnsRec &R, const EnsArgs &a) {
  StageMx S;
  S.U = R.U; S.B = R.B; S.dU = R.dU; S.dB = R.dB;
  S.first = a.stage == 0; S.last = a.stage == a.nstages - 1; S.b = a.b; S.dt = R.dt;
  S.W = R.W; S.F[0] = R.F[0]; S.F[1] = R.F[1]; S.F[2] = R.F[2]; S.E = R.E;
  return S;
}

__device__ __forceinline__ void run_phase(const EnsArgs &a, int ph, long t0, long nth) {
  const long *p = a.pref + (long)ph * (a.nbox + 1);
  const long total = p[a.nbox];
  for (long w = t0; w < total; w += nth) {
    const int bx = find_box(p, a.nbox, w);
    const long t = w - p[bx];
    const EnsRec &R = a.rec[bx];
    const DevGeo &G = R.G;
    const bool first = a.stage == 0;
    switch (ph) {
      case PH_DT: {
        int c[3];
        cell_at(R.b_int, t, c);
        const unsigned s = __float_as_uint(dt_rate_mx(G, R.U, R.B, c, R.dflag));   // >= 0: bits order as floats
        // warp-aggregated maximum when the warp's items share a box
        const unsigned m = __activemask();
        const int lead = __ffs(m) - 1;
        const int b0 = __shfl_sync(m, bx, lead);
        if (__all_sync(m, bx == b0)) {
          const unsigned mx = __reduce_max_sync(m, s);
          if ((int)(threadIdx.x & 31) == lead) atomicMax(R.fmax, mx);
        } else {
          atomicMax(R.fmax, s);
        }
        break;
      }
      case PH_DTFIN:
        *R.dt = G.cfl * G.sc_t / (double)__uint_as_float(*R.fmax);
        *R.fmax = 0u;
        break;
      case PH_PRIM:
        k_prim_mx_at(t, G, R.b_work, R.U, R.B, first ? nullptr : R.dU, first ? nullptr : R.dB, R.W, R.dflag);
        break;
      case PH_RAW:
        k_flag_raw_at<float>(t, G, R.b_int, R.W, R.raw);
        break;
      case PH_DIL0: k_dilate_axis_at<0>(t, G, R.b_int, R.dil_in[0], R.dil_out[0]); break;
      case PH_DIL1: k_dilate_axis_at<1>(t, G, R.b_int, R.dil_in[1], R.dil_out[1]); break;
      case PH_DIL2: k_dilate_axis_at<2>(t, G, R.b_int, R.dil_in[2], R.dil_out[2]); break;
      case PH_EXP:
        k_flag_expand_at(t, G, R.b_exp, R.dil_final, R.flag);
        break;
      case PH_FLUX: {
        const float *dB = first ? nullptr : R.dB;
        const long n0 = G.act[0] ? R.b_flux[0].n : 0, n1 = G.act[1] ? R.b_flux[1].n : 0;
        if (t < n0) k_flux_at<0, float, 0>(t, G, R.b_flux[0], R.W, R.B, dB, R.flag, R.F[0], R.dflag);
        else if (t < n0 + n1) k_flux_at<1, float, 0>(t - n0, G, R.b_flux[1], R.W, R.B, dB, R.flag, R.F[1], R.dflag);
        else k_flux_at<2, float, 0>(t - n0 - n1, G, R.b_flux[2], R.W, R.B, dB, R.flag, R.F[2], R.dflag);
        break;
      }
      case PH_EMF: {
        const long n0 = (G.act[1] || G.act[2]) ? R.b_emf[0].n : 0;
        const long n1 = (G.act[2] || G.act[0]) ? R.b_emf[1].n : 0;
        if (t < n0) k_emf_at<0, float>(t, G, R.b_emf[0], R.W, R.F[1], R.F[2], R.E);
        else if (t < n0 + n1) k_emf_at<1, float>(t - n0, G, R.b_emf[1], R.W, R.F[2], R.F[0], R.E);
        else k_emf_at<2, float>(t - n0 - n1, G, R.b_emf[2], R.W, R.F[0], R.F[1], R.E);
        break;
      }
      case PH_UPD: {
        const StageMx S = stage_bufs(R, a);
        const long nc = R.b_int.n, f0 = R.b_face[0].n, f1 = R.b_face[1].n;
        if (t < nc) k_update_cells_mx_at(t, G, R.b_int, S);
        else if (t < nc + f0) k_update_faces_mx_at<0>(t - nc, G, R.b_face[0], S);
        else if (t < nc + f0 + f1) k_update_faces_mx_at<1>(t - nc - f0, G, R.b_face[1], S);
        else k_update_faces_mx_at<2>(t - nc - f0 - f1, G, R.b_face[2], S);
        break;
      }
    }
  }
}

template <int BS>
__global__ void __launch_bounds__(BS) k_ens_stage(EnsArgs a) {
  cg::grid_group grid = cg::this_grid();
  const long nth = (long)gridDim.x * BS, t0 = (long)blockIdx.x * BS + threadIdx.x;
  if (a.stage == 0) {
    run_phase(a, PH_DT, t0, nth);
    grid.sync();
    run_phase(a, PH_DTFIN, t0, nth);
    grid.sync();
  }
  run_phase(a, PH_PRIM, t0, nth);
  grid.sync();
  const long *p = a.pref;
  if (p[(long)PH_RAW * (a.nbox + 1) + a.nbox] > 0) {   // shock flags (some box has eps_sf > 0)
    run_phase(a, PH_RAW, t0, nth);
    grid.sync();
    for (int ph = PH_DIL0; ph <= PH_DIL2; ++ph) {
      if (p[(long)ph * (a.nbox + 1) + a.nbox] == 0) continue;
      run_phase(a, ph, t0, nth);
      grid.sync();
    }
    run_phase(a, PH_EXP, t0, nth);
    grid.sync();
  }
  run_phase(a, PH_FLUX, t0, nth);
  grid.sync();
  run_phase(a, PH_EMF, t0, nth);
  grid.sync();
  run_phase(a, PH_UPD, t0, nth);
}

// One phase over all boxes (the phase-batched mode: each phase its own
// launch, with its own register allocation, all launches in the step's graph).
template <int PH, int BS>
__global__ void __launch_bounds__(BS) k_ens_phase(EnsArgs a) {
  run_phase(a, PH, (long)blockIdx.x * BS + threadIdx.x, (long)gridDim.x * BS);
}

}  // namespace
}  // namespace phl

using namespace phl;
using namespace phl::stage;

struct phl_ensemble {
  std::vector<phl_grid *> grids;
  EnsRec *drec = nullptr;
  long *dpref = nullptr;
  std::vector<long> hpref;
  int nbox = 0;
  long cells = 0;
  cudaStream_t stream = nullptr;
  int mode = 0;                      // 0: persistent cooperative stage kernel, 1: one launch per phase,
                                     // 2: each box's own kernel chain, boxes on concurrent streams,
                                     // 3: persistent cooperative stage kernel on the fused tile body
  EnsFused fz;                       // mode 3's records (fz_ok: every box fused-eligible)
  bool fz_ok = false;
  int nstreams = 0;                  // mode 2
  int chain_launches = 0;            // mode 2: kernel launches per step
  std::vector<cudaStream_t> aux;     // mode 2 streams
  std::vector<cudaEvent_t> ev;       // fork / join events (aux.size() + 1)
  int block = 256, bps = 0;          // launch shape
  int max_bps[2] = {0, 0};           // occupancy limits for 128 / 256 threads
  cudaStream_t own_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  int graph_ok = 0;
};

namespace {

phl_status ens_fail(phl_status st, const char *msg) { return (phl_status)set_error(st, "%s", msg); }

cudaError_t launch_stage(phl_ensemble *E, int stage, int nstages, float b) {
  EnsArgs a;
  a.rec = E->drec;
  a.pref = E->dpref;
  a.nbox = E->nbox;
  a.stage = stage;
  a.nstages = nstages;
  a.b = b;
  void *args[] = {&a};
  const int sms = 152;
  int dev = 0, nsm = sms;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const dim3 grid((unsigned)(nsm * E->bps)), block((unsigned)E->block);
  if (E->block == 128)
    return cudaLaunchCooperativeKernel((void *)k_ens_stage<128>, grid, block, args, 0, E->stream);
  return cudaLaunchCooperativeKernel((void *)k_ens_stage<256>, grid, block, args, 0, E->stream);
}

template <int BS>
cudaError_t launch_phase(phl_ensemble *E, int ph, const EnsArgs &a) {
  const long total = E->hpref[(size_t)ph * (E->nbox + 1) + E->nbox];
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<long>((total + BS - 1) / BS, 152L * 16);
  switch (ph) {
#define PHL_PH(P) case P: k_ens_phase<P, BS><<<blocks, BS, 0, E->stream>>>(a); break;
    PHL_PH(PH_DT) PHL_PH(PH_DTFIN) PHL_PH(PH_PRIM) PHL_PH(PH_RAW) PHL_PH(PH_DIL0) PHL_PH(PH_DIL1)
    PHL_PH(PH_DIL2) PHL_PH(PH_EXP) PHL_PH(PH_FLUX) PHL_PH(PH_EMF) PHL_PH(PH_UPD)
#undef PHL_PH
  }
  return cudaGetLastError();
}

cudaError_t launch_stage_phases(phl_ensemble *E, int stage, int nstages, float b) {
  EnsArgs a;
  a.rec = E->drec;
  a.pref = E->dpref;
  a.nbox = E->nbox;
  a.stage = stage;
  a.nstages = nstages;
  a.b = b;
  const int order[] = {PH_DT, PH_DTFIN, PH_PRIM, PH_RAW, PH_DIL0, PH_DIL1, PH_DIL2, PH_EXP, PH_FLUX, PH_EMF, PH_UPD};
  for (int ph : order) {
    if ((ph == PH_DT || ph == PH_DTFIN) && stage != 0) continue;
    const cudaError_t e = E->block == 128 ? launch_phase<128>(E, ph, a) : launch_phase<256>(E, ph, a);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Mode 2: every box runs its own per-kernel step (CFL reduction + 3 stages)
// on one of nstreams streams forked from the ensemble's stream and joined back.
cudaError_t launch_step_chains(phl_ensemble *E) {
  const int ns = E->nstreams;
  while ((int)E->aux.size() < ns) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    E->aux.push_back(st);
    E->ev.push_back(ev);
  }
  if (E->ev.size() < E->aux.size() + 1) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    E->ev.push_back(ev);
  }
  cudaEvent_t fork = E->ev.back();
  cudaError_t e = cudaEventRecord(fork, E->stream);
  for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(E->aux[k], fork, 0);
  static const double b3[3] = {1.0, 0.25, 2.0 / 3.0};
  int launches = 0;
  for (int b = 0; b < E->nbox && e == cudaSuccess; ++b) {
    const GridView v = grid_view(E->grids[b]);
    cudaStream_t st = E->aux[b % ns];
    MixedBufs M;
    M.U = v.U; M.B = v.B; M.dU = v.dU; M.dB = v.dB; M.W = v.W;
    for (int k = 0; k < 3; ++k) M.F[k] = v.F[k];
    M.E = v.E; M.raw = v.raw; M.flag = v.flag; M.anyraw = v.anyraw; M.dt = v.dt; M.dflag = v.dflag;
    M.Tin = nullptr; M.Tout = nullptr;
    M.tmapW = v.tmapW; M.fused_variant = v.fused;   // the box's own stage decomposition
    M.pipeline3 = v.pipeline3;
    M.primed = false;   // each replay forms W from the state it finds
    M.fmax = nullptr;   // the step's own CFL launch comes first: no maximum to carry
    *v.w_valid = false;
    int nl = 0;
    launch_dt_mixed(*v.G, v.U, v.B, v.fmax, v.dt, v.dflag, st, &nl, nullptr);
    for (int stg = 0; stg < 3; ++stg) launch_stage_mixed(*v.G, M, stg, 3, b3[stg], st, &nl, nullptr);
    launches += nl;
    e = cudaGetLastError();
  }
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    e = cudaEventRecord(E->ev[k], E->aux[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(E->stream, E->ev[k], 0);
  }
  E->chain_launches = launches;
  return e;
}

cudaError_t launch_step(phl_ensemble *E) {
  static const float b3[3] = {1.0f, 0.25f, 2.0f / 3.0f};
  if (E->mode == 2) return launch_step_chains(E);
  if (E->mode == 3) {
    for (int st = 0; st < 3; ++st) {
      const cudaError_t e = launch_ens_fused(E->fz, st, 3, b3[st], E->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int st = 0; st < 3; ++st) {
    cudaError_t e = E->mode == 0 ? launch_stage(E, st, 3, b3[st]) : launch_stage_phases(E, st, 3, b3[st]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void drop_graph(phl_ensemble *E) {
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  E->exec = nullptr;
  E->graph = nullptr;
  E->graph_ok = 0;
}

// Capture one step; on any failure run without the graph.
void build_graph(phl_ensemble *E) {
  drop_graph(E);
  if (!E->use_graph) return;
  cudaError_t e0 = cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    cudaGetLastError();
    set_error(PHL_ECUDA, "ensemble graph capture not started: %s", cudaGetErrorString(e0));
    return;
  }
  cudaError_t e1 = launch_step(E);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(E->stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    set_error(PHL_ECUDA, "ensemble graph capture failed: launch %s, end %s", cudaGetErrorString(e1),
              cudaGetErrorString(e2));
    return;
  }
  cudaError_t e3 = cudaGraphInstantiate(&E->exec, g, 0);
  if (e3 != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    E->exec = nullptr;
    set_error(PHL_ECUDA, "ensemble graph instantiation failed: %s", cudaGetErrorString(e3));
    return;
  }
  E->graph = g;
  E->graph_ok = 1;
}

}  // namespace

extern "C" {

phl_status phl_ensemble_create(const phl_grid_desc *descs, int nbox, int use_graph, phl_ensemble **out) {
  if (!descs || nbox < 1 || !out) return ens_fail(PHL_EINVAL, "phl_ensemble_create: bad arguments");
  *out = nullptr;
  for (int b = 0; b < nbox; ++b) {
    const phl_grid_desc &d = descs[b];
    if (d.precision != PHL_MIXED || d.eos != PHL_EOS_IDEAL || d.nspec != 0 || d.rk != 3)
      return ens_fail(PHL_EUNSUPPORTED, "ensemble boxes: mixed form, ideal gas, no species, SSP-RK3");
    if (d.stream != descs[0].stream) return ens_fail(PHL_EINVAL, "ensemble boxes must share one stream");
  }
  phl_ensemble *E = new phl_ensemble();
  E->stream = (cudaStream_t)descs[0].stream;
  if (!E->stream) {
    // the legacy default stream cannot be captured: use a blocking stream of
    // our own (ordered with the default stream's work) for the boxes and launches
    if (cudaStreamCreate(&E->own_stream) != cudaSuccess) {
      delete E;
      return ens_fail(PHL_ECUDA, "phl_ensemble_create: stream creation failed");
    }
    E->stream = E->own_stream;
  }
  E->use_graph = use_graph != 0;
  E->nbox = nbox;
  std::vector<EnsRec> rec(nbox);
  E->hpref.assign((size_t)NPH * (nbox + 1), 0);
  for (int b = 0; b < nbox; ++b) {
    phl_grid *g = nullptr;
    phl_grid_desc db = descs[b];
    db.stream = E->stream;
    phl_status st = phl_create_grid(&db, &g);
    if (st != PHL_OK) {
      phl_ensemble_destroy(E);
      return st;
    }
    E->grids.push_back(g);
    const GridView v = grid_view(g);
    const DevGeo &G = *v.G;
    EnsRec &R = rec[b];
    memset(&R, 0, sizeof(R));
    R.G = G;
    R.U = v.U; R.B = v.B; R.dU = v.dU; R.dB = v.dB; R.W = v.W;
    for (int k = 0; k < 3; ++k) R.F[k] = v.F[k];
    R.E = v.E; R.raw = v.raw; R.flag = v.flag; R.dt = v.dt; R.fmax = v.fmax; R.dflag = v.dflag;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const long nc = (long)nx * ny * nz;
    E->cells += nc;
    R.b_int = make_box(0, nx, 0, ny, 0, nz);
    int l[3], h[3];
    for (int d = 0; d < 3; ++d) {
      if (G.act[d]) { l[d] = -G.ge[d]; h[d] = G.n[d] + G.ge[d]; } else { l[d] = 0; h[d] = 1; }
    }
    R.b_work = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    for (int d = 0; d < 3; ++d) {
      if (G.act[d]) { l[d] = -1; h[d] = G.n[d] + 1; } else { l[d] = 0; h[d] = 1; }
    }
    R.b_exp = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
    long nflux = 0, nemf = 0, nface = 0;
    for (int D = 0; D < 3; ++D) {
      for (int d = 0; d < 3; ++d) {
        if (d == D) { l[d] = 0; h[d] = G.n[d] + 1; }
        else if (G.act[d]) { l[d] = -1; h[d] = G.n[d] + 1; }
        else { l[d] = 0; h[d] = 1; }
      }
      R.b_flux[D] = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
      if (G.act[D]) nflux += R.b_flux[D].n;
      const int A = (D + 1) % 3, B = (D + 2) % 3;
      int el[3] = {0, 0, 0}, eh[3];
      eh[D] = G.n[D];
      eh[A] = G.act[A] ? G.n[A] + 1 : 1;
      eh[B] = G.act[B] ? G.n[B] + 1 : 1;
      R.b_emf[D] = make_box(el[0], eh[0], el[1], eh[1], el[2], eh[2]);
      if (G.act[A] || G.act[B]) nemf += R.b_emf[D].n;
      int fh[3] = {G.n[0], G.n[1], G.n[2]};
      fh[D] += 1;
      R.b_face[D] = make_box(0, fh[0], 0, fh[1], 0, fh[2]);
      nface += R.b_face[D].n;
    }
    // flag dilation ping-pong over the active axes (as the per-kernel path)
    uint8_t *cur = R.raw, *other = R.raw + nc;
    long ndil[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      R.dil_in[d] = cur;
      R.dil_out[d] = other;
      if (G.act[d] && G.eps_sf > 0.0) {
        ndil[d] = nc;
        std::swap(cur, other);
      }
    }
    R.dil_final = cur;
    const bool flags = G.eps_sf > 0.0;
    const long cnt[NPH] = {nc, 1, R.b_work.n, flags ? nc : 0, ndil[0], ndil[1], ndil[2],
                           flags ? R.b_exp.n : 0, nflux, nemf, nc + nface};
    for (int ph = 0; ph < NPH; ++ph)
      E->hpref[(size_t)ph * (nbox + 1) + b + 1] = E->hpref[(size_t)ph * (nbox + 1) + b] + cnt[ph];
  }
  cudaError_t e = cudaMalloc(&E->drec, nbox * sizeof(EnsRec));
  if (e == cudaSuccess) e = cudaMalloc(&E->dpref, E->hpref.size() * sizeof(long));
  if (e == cudaSuccess) e = cudaMemcpy(E->drec, rec.data(), nbox * sizeof(EnsRec), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(E->dpref, E->hpref.data(), E->hpref.size() * sizeof(long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&E->max_bps[0], (const void *)k_ens_stage<128>, 128, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&E->max_bps[1], (const void *)k_ens_stage<256>, 256, 0);
  if (e != cudaSuccess || E->max_bps[1] < 1) {
    phl_ensemble_destroy(E);
    return (phl_status)set_error(PHL_ECUDA, "phl_ensemble_create: %s", cudaGetErrorString(e));
  }
  E->block = 256;
  E->bps = E->max_bps[1];
  {   // mode 3 when every box runs the fused stage
    std::vector<GridView> views;
    bool ok = true;
    for (phl_grid *g : E->grids) {
      views.push_back(grid_view(g));
      ok = ok && views.back().tmapW != nullptr;
    }
    if (ok) {
      const cudaError_t ef = ens_fused_create(views.data(), nbox, &E->fz);
      E->fz_ok = ef == cudaSuccess;
      if (!E->fz_ok) cudaGetLastError();
    }
  }
  *out = E;
  return PHL_OK;
}

phl_status phl_ensemble_grid(phl_ensemble *E, int box, phl_grid **g) {
  if (!E || !g || box < 0 || box >= E->nbox) return ens_fail(PHL_EINVAL, "phl_ensemble_grid: bad arguments");
  *g = E->grids[box];
  return PHL_OK;
}

phl_status phl_ensemble_step(phl_ensemble *E, int nsteps) {
  if (!E || nsteps < 0) return ens_fail(PHL_EINVAL, "phl_ensemble_step: bad arguments");
  if (E->use_graph && !E->exec) build_graph(E);
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = E->exec ? cudaGraphLaunch(E->exec, E->stream) : launch_step(E);
    if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_ensemble_step: %s", cudaGetErrorString(e));
  }
  for (phl_grid *g : E->grids) {
    const GridView v = grid_view(g);
    *v.steps += nsteps;
    *v.w_valid = false;   // the ensemble moved the state: a later phl_step forms W again
  }
  return PHL_OK;
}

phl_status phl_ensemble_check(phl_ensemble *E) {
  if (!E) return ens_fail(PHL_EINVAL, "null ensemble");
  for (phl_grid *g : E->grids) {
    const phl_status st = phl_check(g);
    if (st != PHL_OK) return st;
  }
  return PHL_OK;
}

phl_status phl_ensemble_set_shape(phl_ensemble *E, int mode, int block, int blocks_per_sm, int streams) {
  if (!E) return ens_fail(PHL_EINVAL, "null ensemble");
  if (mode < 0 || mode > 3)
    return ens_fail(PHL_EINVAL, "mode must be 0 (persistent), 1 (phases), 2 (chains) or 3 (persistent fused)");
  if (mode == 3 && !E->fz_ok) return ens_fail(PHL_EUNSUPPORTED, "mode 3 needs every box on the fused stage");
  if (mode < 2 && block != 128 && block != 256) return ens_fail(PHL_EINVAL, "block must be 128 or 256");
  if (mode == 0 && (blocks_per_sm < 1 || blocks_per_sm > E->max_bps[block == 128 ? 0 : 1]))
    return ens_fail(PHL_EINVAL, "blocks per SM out of the co-resident range");
  if (mode == 2 && (streams < 1 || streams > 64)) return ens_fail(PHL_EINVAL, "streams must be 1..64");
  E->mode = mode;
  E->block = mode == 2 ? 256 : (mode == 3 ? 288 : block);
  E->bps = mode == 0 ? blocks_per_sm : (mode == 3 ? E->fz.per_sm : 0);
  E->nstreams = mode == 2 ? streams : 0;
  drop_graph(E);
  return PHL_OK;
}

phl_status phl_ensemble_autotune(phl_ensemble *E, int trial_steps, phl_tune_entry *out, int max, int *n) {
  if (!E || trial_steps < 1) return ens_fail(PHL_EINVAL, "phl_ensemble_autotune: bad arguments");
  // save the state of every box, time each candidate, restore
  std::vector<std::pair<double *, size_t>> save;
  std::vector<void *> copies;
  cudaError_t e = cudaSuccess;
  for (phl_grid *g : E->grids) {
    const GridView v = grid_view(g);
    const size_t bu = (size_t)v.G->nv * v.G->plane * sizeof(double), bb = (size_t)3 * v.G->plane * sizeof(double);
    for (auto pr : {std::make_pair(v.U, bu), std::make_pair(v.B, bb)}) {
      void *c = nullptr;
      if (e == cudaSuccess) e = cudaMalloc(&c, pr.second);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c, pr.first, pr.second, cudaMemcpyDeviceToDevice, E->stream);
      copies.push_back(c);
      save.push_back(pr);
    }
  }
  auto restore = [&]() {
    for (size_t i = 0; i < save.size(); ++i)
      if (copies[i]) cudaMemcpyAsync(save[i].first, copies[i], save[i].second, cudaMemcpyDeviceToDevice, E->stream);
  };
  std::vector<phl_tune_entry> res;
  int best_m = E->mode, best_b = E->block, best_p = E->bps, best_s = E->nstreams;
  double best_ms = 1e300;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<phl_tune_entry> cand;
  for (int bsz : {128, 256}) {
    phl_tune_entry c;
    c.mode = 1; c.block = bsz; c.blocks_per_sm = 0; c.streams = 0; c.ms_per_step = 0.0;
    cand.push_back(c);
    for (int p = 1; p <= E->max_bps[bsz == 128 ? 0 : 1]; ++p) {
      c.mode = 0; c.blocks_per_sm = p;
      cand.push_back(c);
    }
  }
  if (E->fz_ok) {
    phl_tune_entry c;
    c.mode = 3; c.block = 288; c.blocks_per_sm = E->fz.per_sm; c.streams = 0; c.ms_per_step = 0.0;
    cand.push_back(c);
  }
  for (int ns : {1, 4, 8, E->nbox}) {
    phl_tune_entry c;
    c.mode = 2; c.block = 256; c.blocks_per_sm = 0; c.streams = std::min(ns, E->nbox); c.ms_per_step = 0.0;
    bool dup = false;
    for (const auto &q : cand) dup |= q.mode == 2 && q.streams == c.streams;
    if (!dup) cand.push_back(c);
  }
  for (const phl_tune_entry &c : cand) {
    if (e != cudaSuccess) break;
    {
      const int bsz = c.block, p = c.blocks_per_sm;
      E->mode = c.mode;
      E->block = bsz;
      E->bps = p;
      E->nstreams = c.streams;
      drop_graph(E);
      build_graph(E);
      restore();
      // one untimed step, then trial_steps timed
      e = E->exec ? cudaGraphLaunch(E->exec, E->stream) : launch_step(E);
      if (e != cudaSuccess) break;
      cudaEventRecord(e0, E->stream);
      for (int s = 0; s < trial_steps && e == cudaSuccess; ++s)
        e = E->exec ? cudaGraphLaunch(E->exec, E->stream) : launch_step(E);
      cudaEventRecord(e1, E->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      phl_tune_entry t = c;
      t.ms_per_step = ms / trial_steps;
      res.push_back(t);
      if (t.ms_per_step < best_ms) {
        best_ms = t.ms_per_step; best_m = c.mode; best_b = bsz; best_p = p; best_s = c.streams;
      }
    }
  }
  restore();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaError_t es = cudaStreamSynchronize(E->stream);
  for (void *c : copies) cudaFree(c);
  if (e == cudaSuccess) e = es;
  E->mode = best_m;
  E->block = best_b;
  E->bps = best_p;
  E->nstreams = best_s;
  drop_graph(E);
  if (e != cudaSuccess) return (phl_status)set_error(PHL_ECUDA, "phl_ensemble_autotune: %s", cudaGetErrorString(e));
  if (n) *n = (int)res.size();
  if (out)
    for (int i = 0; i < (int)res.size() && i < max; ++i) out[i] = res[i];
  return PHL_OK;
}

phl_status phl_ensemble_get_info(const phl_ensemble *E, phl_ensemble_info *info) {
  if (!E || !info) return ens_fail(PHL_EINVAL, "null argument");
  info->nbox = E->nbox;
  info->cells = E->cells;
  info->mode = E->mode;
  info->block = E->block;
  info->blocks_per_sm = E->bps;
  info->streams = E->nstreams;
  info->graph = E->graph_ok;
  int nl = 3;   // modes 0 and 3: one launch per stage
  if (E->mode == 2) {
    nl = E->chain_launches;
  } else if (E->mode == 1) {
    nl = 0;
    for (int st = 0; st < 3; ++st)
      for (int ph = 0; ph < NPH; ++ph) {
        if ((ph == PH_DT || ph == PH_DTFIN) && st != 0) continue;
        if (E->hpref[(size_t)ph * (E->nbox + 1) + E->nbox] > 0) ++nl;
      }
  }
  info->launches_per_step = nl;
  return PHL_OK;
}

void phl_ensemble_destroy(phl_ensemble *E) {
  if (!E) return;
  drop_graph(E);
  for (cudaStream_t st : E->aux) cudaStreamDestroy(st);
  for (cudaEvent_t ev : E->ev) cudaEventDestroy(ev);
  for (phl_grid *g : E->grids) phl_destroy(g);
  cudaFree(E->drec);
  cudaFree(E->dpref);
  ens_fused_destroy(&E->fz);
  if (E->own_stream) cudaStreamDestroy(E->own_stream);
  delete E;
}

}  // extern "C"
