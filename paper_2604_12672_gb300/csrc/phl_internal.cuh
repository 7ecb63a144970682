// phl_internal.cuh -- device-side geometry, layouts and kernel entry points
// shared by the library's translation units.
//
// Device state layout (one allocation per field group, FP64, no ghosts):
//   index(i, j, k) = i + sy * j + sz * k,  sy = pitch >= nx + 1 (multiple of 4),
//   sz = sy * (ny + 1); every array spans (nz + 1) planes so cells (i < nx)
//   and faces (i <= nx) share one geometry.  Conserved variable v lives at
//   U + v * plane; face component d (normal B on d-faces) at Bf + d * plane.
// Ghost cells are never stored for the state: a ghost index is mapped to the
// interior cell its data comes from (periodic wrap, mirror, or copy) and the
// reflecting sign flips are applied on the fly.
//
// Work layout (per-stage scratch, FP64 path): the same index formula with
// "ge" ghost layers (2 on active dimensions) and one extra face layer:
//   windex(i, j, k) = (i + ge0) + wy * (j + ge1) + wz * (k + ge2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eos_stellar.cuh"
#include "phl.h"
#include "mlp_dev.cuh"
#include "riemann.cuh"

namespace phl {

constexpr int NGW = 2;               // work-array ghost layers
constexpr int NW_MAX = 10 + PHL_NSPEC_MAX;
constexpr int NF_MAX = 8 + PHL_NSPEC_MAX;
constexpr int BG_NG = 3;             // background-profile ghost layers

// primitive deviation components (cell-centred work arrays)
enum { W_RHO = 0, W_VX, W_VY, W_VZ, W_BX, W_BY, W_BZ, W_P, W_GE, W_GC, W_X0 };
// conserved components
enum { U_RHO = 0, U_MX, U_MY, U_MZ, U_E, U_X0 };
// global-frame flux components
enum { F_RHO = 0, F_MX, F_MY, F_MZ, F_E, F_BX, F_BY, F_BZ, F_X0 };

enum { FLAG_NEG = 1, FLAG_NAN = 2, FLAG_NEWTON = 4, FLAG_TIMEOUT = 8 };

struct DevGeo {
  int n[3];
  int act[3];
  int bc[3][2];
  long sy, sz, plane;          // state strides / size per field
  int ge[3];
  long wy, wz, wtot;           // work strides / size per field
  int wstr;                    // FP32 W: values per cell (wstr / 4 planes of float4)
  double dx[3], idx[3];
  int nspec, nv, nw, nf;
  int eos;
  double gamma;
  int has_bg;
  const double *bg_rho_c, *bg_p_c, *bg_rho_f, *bg_p_f;   // device profiles
  const double *bg_ge_c, *bg_gc_c, *bg_ge_f, *bg_gc_f;   // may be null
  const double *heat;          // per z-cell, may be null
  double g[3];
  int riemann;
  int recon;                   // PHL_RECON_VANLEER / PHL_RECON_PPH
  double eps_sf, mach_thr, cfl;
  // FP32 copies for the mixed-precision kernels (no per-thread conversions)
  // Mixed form: the FP32 quantities are held in units of powers of two
  // (rho_s, P_s, v_s = sqrt(P_s / rho_s), B_s = sqrt(P_s), L_s, t_s = L_s / v_s)
  // near the background's scales, so stellar CGS magnitudes (P ~ 1e24) stay
  // far inside the FP32 range.  Multiplying by a power of two is exact, so the
  // scaling changes no rounding.  sc_* turn scaled values into physical ones.
  double sc_rho, sc_m, sc_e, sc_b, sc_t;
  int e_rho, e_m, e_e, e_b, e_t;   // sc_x = 2^e_x (applied to the exponent field by d2f_scaled / f2d_scaled)
  double isc_rho, isc_m, isc_e, isc_b, isc_t, isc_v;
  float idxf[3], gf[3], gammaf, gm1f, machf, epsf;   // idxf, gf in scaled units
  const float *bgf_rho_c, *bgf_p_c, *bgf_rho_f, *bgf_p_f;   // null without background
  const float *bgf_ge_c, *bgf_gc_c, *bgf_ge_f, *bgf_gc_f;
  const float *heatf;
  const double *bg_e_c;        // E_hat = P_hat / (gamma - 1) at cell centres (FP64)
  // stellar EOS
  eos::Table tab;
  double Acomp[PHL_NSPEC_MAX], Zcomp[PHL_NSPEC_MAX];
  double iAcomp[PHL_NSPEC_MAX], ZoAcomp[PHL_NSPEC_MAX];   // 1/A and Z/A per species
  double newton_tol;
  int newton_maxit;
  int use_mlp;                 // first Newton guess from the network
  mlp::Dev mlp;
  unsigned long long *niter;   // Newton iterations summed over cells (device)
  double *pred;                // mixed stellar form: 8 planes, each cell's last inversion (eos::Pred)
};

__host__ __device__ __forceinline__ long sidx(const DevGeo &G, int i, int j, int k) {
  return (long)i + G.sy * j + G.sz * k;
}
__host__ __device__ __forceinline__ long widx(const DevGeo &G, int i, int j, int k) {
  return (long)(i + G.ge[0]) + G.wy * (j + G.ge[1]) + G.wz * (k + G.ge[2]);
}

// Ghost mapping of a cell index along one dimension (Table bcs): returns the
// interior source index; *flip = true where the reflecting mirror applies.
__host__ __device__ __forceinline__ int cell_src(int i, int n, int bclo, int bchi, bool &flip) {
  flip = false;
  if (i < 0) {
    if (bclo == 0) { int r = i % n; return r < 0 ? r + n : r; }
    if (bclo == 1) { flip = true; return -1 - i; }
    return 0;
  }
  if (i >= n) {
    if (bchi == 0) return i % n;
    if (bchi == 1) { flip = true; return 2 * n - 1 - i; }
    return n - 1;
  }
  return i;
}

// Background at cell centre k and at z-face k-1/2 (zero without background).
struct Bg { double rho, p, ge, gc; };
__device__ __forceinline__ Bg bg_cell(const DevGeo &G, int k) {
  Bg b{0.0, 0.0, 0.0, 0.0};
  if (G.has_bg) {
    b.rho = G.bg_rho_c[k + BG_NG];
    b.p = G.bg_p_c[k + BG_NG];
    b.ge = G.bg_ge_c ? G.bg_ge_c[k + BG_NG] : G.gamma;
    b.gc = G.bg_gc_c ? G.bg_gc_c[k + BG_NG] : G.gamma;
  }
  return b;
}
__device__ __forceinline__ Bg bg_zface(const DevGeo &G, int k) {
  Bg b{0.0, 0.0, 0.0, 0.0};
  if (G.has_bg) {
    b.rho = G.bg_rho_f[k + BG_NG];
    b.p = G.bg_p_f[k + BG_NG];
    b.ge = G.bg_ge_f ? G.bg_ge_f[k + BG_NG] : G.gamma;
    b.gc = G.bg_gc_f ? G.bg_gc_f[k + BG_NG] : G.gamma;
  }
  return b;
}

// The background in the arithmetic type of a kernel: FP64 profiles for double,
// their FP32 copies for float.
template <typename R>
struct BgT { R rho, p, ge, gc; };
template <typename R>
__device__ __forceinline__ BgT<R> bg_cell_t(const DevGeo &G, int k);
template <typename R>
__device__ __forceinline__ BgT<R> bg_zface_t(const DevGeo &G, int k);
template <>
__device__ __forceinline__ BgT<double> bg_cell_t<double>(const DevGeo &G, int k) {
  const Bg b = bg_cell(G, k);
  return BgT<double>{b.rho, b.p, b.ge, b.gc};
}
template <>
__device__ __forceinline__ BgT<double> bg_zface_t<double>(const DevGeo &G, int k) {
  const Bg b = bg_zface(G, k);
  return BgT<double>{b.rho, b.p, b.ge, b.gc};
}
template <>
__device__ __forceinline__ BgT<float> bg_cell_t<float>(const DevGeo &G, int k) {
  BgT<float> b{0.0f, 0.0f, 0.0f, 0.0f};
  if (G.has_bg) {
    b.rho = G.bgf_rho_c[k + BG_NG];
    b.p = G.bgf_p_c[k + BG_NG];
    b.ge = G.bgf_ge_c ? G.bgf_ge_c[k + BG_NG] : G.gammaf;
    b.gc = G.bgf_gc_c ? G.bgf_gc_c[k + BG_NG] : G.gammaf;
  }
  return b;
}
template <>
__device__ __forceinline__ BgT<float> bg_zface_t<float>(const DevGeo &G, int k) {
  BgT<float> b{0.0f, 0.0f, 0.0f, 0.0f};
  if (G.has_bg) {
    b.rho = G.bgf_rho_f[k + BG_NG];
    b.p = G.bgf_p_f[k + BG_NG];
    b.ge = G.bgf_ge_f ? G.bgf_ge_f[k + BG_NG] : G.gammaf;
    b.gc = G.bgf_gc_f ? G.bgf_gc_f[k + BG_NG] : G.gammaf;
  }
  return b;
}
template <typename R> __device__ __forceinline__ R mach_thr_t(const DevGeo &G);
template <> __device__ __forceinline__ double mach_thr_t<double>(const DevGeo &G) { return G.mach_thr; }
template <> __device__ __forceinline__ float mach_thr_t<float>(const DevGeo &G) { return G.machf; }
template <typename R> __device__ __forceinline__ R eps_sf_t(const DevGeo &G);
template <> __device__ __forceinline__ double eps_sf_t<double>(const DevGeo &G) { return G.eps_sf; }
template <> __device__ __forceinline__ float eps_sf_t<float>(const DevGeo &G) { return G.epsf; }

// IEEE binary64 <-> binary32 conversions done on the integer pipe (the FP64
// pipe, which also executes the conversion instructions, runs at 1/64 of the
// FP32 rate on this GPU).  d2f_bits rounds to nearest (ties away from zero,
// vs. ties-to-even of a hardware conversion), flushes |x| < 2^-126 to zero and
// maps overflow to infinity; f2d_bits is exact for normal floats and zero.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu;
  // exponent rebias 1023 -> 127 inside the high word, then 20 + 3 mantissa bits
  unsigned t = __funnelshift_l(lo, a - (896u << 20), 3);
  t += (lo >> 28) & 1u;
  t = (a < (897u << 20)) ? 0u : t;
  t = (a >= (1151u << 20)) ? (0x7f800000u | ((a > 0x7ff00000u || (a == 0x7ff00000u && lo)) ? 0x400000u : 0u)) : t;
  return __uint_as_float(t | sign);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) hi = sign | 0x7ff00000u | (m >> 3);
  return __hiloint2double((int)hi, (int)lo);
}

// The same conversions with an exact power-of-two scale folded into the
// exponent rebias: d2f_scaled(x, k) == d2f_bits(x * 2^k) and f2d_scaled(f, k)
// == f2d_bits(f) * 2^k bit for bit (for |k| < 800 and results inside the
// FP64 range), without the FP64 multiply.  The mixed form's unit scales are
// powers of two, so its FP64 <-> FP32 boundary costs no FP64 arithmetic.
__device__ __forceinline__ float d2f_scaled(double x, int k) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu;
  const unsigned rb = (unsigned)(896 - k) << 20;
  unsigned t = __funnelshift_l(lo, a - rb, 3);
  t += (lo >> 28) & 1u;
  t = (a < rb + (1u << 20)) ? 0u : t;
  t = (a >= rb + (255u << 20))
          ? (0x7f800000u | ((a > 0x7ff00000u || (a == 0x7ff00000u && lo)) ? 0x400000u : 0u))
          : t;
  return __uint_as_float(t | sign);
}
__device__ __forceinline__ double f2d_scaled(float f, int k) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi = sign | ((e + (unsigned)(896 + k)) << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) hi = sign | 0x7ff00000u | (m >> 3);
  return __hiloint2double((int)hi, (int)lo);
}

// Exact division by a runtime divisor d for numerators below 2^31: with
// s = ceil(log2 d) and m = floor(2^(32+s) / d) + 1 (< 2^33), t / d equals
// (t * m) >> (32 + s) -- one wide multiply instead of an integer division.
struct FastDiv {
  unsigned long long m;
  unsigned s, d;
};
inline FastDiv make_fastdiv(unsigned d) {
  unsigned s = 0;
  while ((1ull << s) < d) ++s;
  return FastDiv{((1ull << (32 + s)) / d) + 1ull, s, d};
}
__device__ __forceinline__ unsigned fastdiv(unsigned t, const FastDiv &f) {
  return (unsigned)(((unsigned long long)t * f.m) >> (32 + f.s));
}

// Kernel classes for the optional per-kernel event timing.
enum KClass {
  KC_PRIM = 0, KC_FLAG_RAW, KC_FLAG_DILATE, KC_FLUX_X, KC_FLUX_Y, KC_FLUX_Z, KC_EMF, KC_UPDATE_CELLS,
  KC_UPDATE_FACES, KC_DT, KC_SCALAR, KC_STAGE_MIXED, KC_FLUX_UPDATE,
  KC_SPH_PRIM, KC_SPH_FLUX, KC_SPH_EMF, KC_SPH_UPDATE_FACES, KC_SPH_UPDATE_CELLS, KC_SPH_DT, KC_COUNT
};
const char *kclass_name(int c);

// Records (start, end) event pairs around launches when enabled.
struct Prof {
  bool on = false;
  cudaEvent_t *ev = nullptr;   // pool of 2 * cap events
  int *cls = nullptr;
  int cap = 0, used = 0;
  double ms[KC_COUNT] = {0};
  long cnt[KC_COUNT] = {0};
  int cur = -1;
  cudaError_t begin(int c, cudaStream_t s);
  cudaError_t end(cudaStream_t s);
  cudaError_t fold();          // synchronises on the recorded events
  void release();
};

// Pointers of one FP64 stage evaluation.
struct StageBufs {
  const double *Uin, *Bin;     // stage input state
  const double *Ubase, *Bbase; // U^n
  double *Uout, *Bout;
  double a, b;                 // out = a * base + b * (in - dt * R)
  const double *dt;            // device scalar
  double *W;                   // nw work fields
  double *F[3];                // nf flux fields per direction
  double *E;                   // 3 edge-EMF fields
  uint8_t *raw, *flag;         // raw flags (interior), dilated flags (work layout)
  const double *Tin;           // temperature guesses (stellar), state layout
  double *Tout;                // temperatures found by this stage
  int *dflag;                  // device error word
  unsigned long long *cfl_dmax = nullptr;   // stellar: the CFL step from this stage's inversion into dt
};

// Buffers of the mixed-precision stage (kernels_mixed.cu): FP64 U^n, FP32
// stage increments and FP32 work arrays.
struct MixedBufs {
  double *U, *B;               // U^n cells / faces (padded state layout)
  float *dU, *dB;              // stage increments, same layout
  float *W, *F[3], *E;         // work arrays (work layout)
  uint8_t *raw, *flag;
  const double *dt;
  int *dflag;
  const double *Tin;           // stellar EOS: guesses in, temperatures out
  double *Tout;
  unsigned long long *cfl_dmax = nullptr;   // stellar: the CFL step from this stage's inversion into dt
  const void *tmapW = nullptr; // TMA descriptor of W (fused path), or null
  int fused_variant = 1;       // launch shape of the fused tile kernel (phl_set_fused)
  unsigned test_extra_tx = 0;  // timeout test: bytes announced to the tile barrier that never arrive
  // Fused path in three launches per stage (tile kernel, Contact-CT + face
  // update, next primitives + raw flags); otherwise six (primitives, raw
  // flags, dilation, tile kernel, EMFs, face update).
  bool pipeline3 = false;
  // pipeline3: W, the auxiliaries and the raw flags already hold the stage
  // input (the previous stage's last kernel formed them); false at the first
  // stage after the state was set from outside
  bool primed = false;
  unsigned int *fmax = nullptr; // CFL rate maximum the last stage folds into (pipeline3)
  // ideal gas, device CFL step: the first stage's primitives of U^n also
  // fold the CFL rate into this maximum and set dt (no separate CFL pass)
  unsigned int *cfl_fmax = nullptr;
  // fused six-launch path: the raw-flag kernel's "some cell is flagged" vote
  // (zeroed before it); null = always dilate and load the flags
  unsigned int *anyraw = nullptr;
};
void launch_stage_mixed(const DevGeo &G, const MixedBufs &M, int stage, int nstages, double b, cudaStream_t s,
                        int *nlaunch, Prof *prof);
// The mixed-form primitives of the whole work box in one form (phl_test_prims):
// 0 cell by cell, 1 in pairs of cells, 2 / 3 the same with the CFL rate of
// U^n into fmax_bits (dU, dB ignored).
cudaError_t launch_prims_form(const DevGeo &G, const double *U, const double *Bf, const float *dU, const float *dB,
                              float *W, int *dflag, int form, unsigned int *fmax_bits, cudaStream_t s);
// Raw shock flags of the interior from W (phl_test_raw_flags): form 0 one
// cell per thread, 1 four cells of a row per thread; any: the flag vote.
cudaError_t launch_raw_flags_form(const DevGeo &G, const float *W, uint8_t *raw, int form, unsigned int *any,
                                  cudaStream_t s);

// The pair form of the primitives needs: an ideal gas without species (W in
// two float4 planes), an active x axis of even length and an even number of
// ghost layers along x, so that the source cells of every pair of work cells
// (2m - ge, 2m - ge + 1) lie in one aligned pair of state cells (2a, 2a + 1)
// -- interior pairs are their own sources; periodic ghost pairs map to the
// pair at the other end, reflecting ones to the mirrored boundary pair,
// outflow ones to the boundary cell twice -- and rows and planes of the
// state have even pitches, so every such pair is a 16-byte FP64 load.
__host__ __device__ inline bool prim_pairs_ok(const DevGeo &G) {
  return G.wstr == 8 && G.nspec == 0 && G.eos == 0 && G.act[0] && G.n[0] % 2 == 0 && G.ge[0] % 2 == 0 &&
         G.sy % 2 == 0 && G.sz % 2 == 0 && G.plane % 2 == 0;
}

void launch_dt_mixed(const DevGeo &G, const double *U, const double *Bf, unsigned int *fmax_bits, double *dt,
                     int *dflag, cudaStream_t s, int *nlaunch, Prof *prof);
// The step length from the CFL maximum the previous step's last stage folded
// into fmax_bits (three-launch path), or fixed_dt > 0; clears fmax_bits.
void launch_dt_mixed_from_max(const DevGeo &G, double fixed_dt, unsigned int *fmax_bits, double *dt, cudaStream_t s,
                              int *nlaunch, Prof *prof);

// Thermal diffusion by RKL2 super-time-stepping (diffusion.cu).
cudaError_t launch_diffuse(const DevGeo &G, double *U, const double *Bf, const phl_diffusion &p, double dt,
                           int max_stages, bool mixed, double *scratch, int *dflag, cudaStream_t s, int *nsts,
                           int *nlaunch);

// Fused mixed stage (stage_fused.cu): faces of all three directions and the
// cell update in one tiled kernel; ideal gas, no species, 3-D grids.
bool fused_stage_ok(const DevGeo &G);
constexpr int PHL_FUSED_SHAPES = 9;    // launch shapes of the tile kernel
constexpr int PHL_FUSED_DEFAULT = 8;   // the shape used unless phl_set_fused picks another (288 threads, 3 CTAs/SM, phased, left/right-paired solver)
int make_fused_tmap(const DevGeo &G, const float *W, void *tmap128);
cudaError_t fused_init();   // shared-memory limits of the tile kernels (once per process)
void launch_fused_tail(const DevGeo &G, const MixedBufs &M, bool first, bool last, double b, cudaStream_t s,
                       int *nl, Prof *prof);
// The next stage's primitives with their ghost images, the raw flags and,
// in the last stage, the CFL maximum (stage_prim.cu).
void launch_prim_flags(const DevGeo &G, const MixedBufs &M, bool last, unsigned int *fmax, cudaStream_t s, int *nl,
                       Prof *prof);

// Buffers of a grid for the ensemble path (ensemble.cu); mixed grids only.
struct GridView {
  const DevGeo *G;
  double *U, *B;
  float *dU, *dB, *W, *F[3], *E;
  uint8_t *raw, *flag;
  unsigned int *anyraw;        // the raw-flag kernel's vote (fused six-launch stage)
  double *dt;
  unsigned int *fmax;
  int *dflag;
  cudaStream_t stream;
  long *steps;
  bool mixed;
  const void *tmapW;           // TMA descriptor of W when the grid runs the fused stage
  int fused;                   // its launch shape (0: per-direction kernels)
  bool *w_valid;               // the grid's record that W holds its state (cleared by ensemble steps)
  bool pipeline3;              // its fused stage runs in three launches
};
GridView grid_view(::phl_grid *g);

// Boxes of an ensemble stepped by one persistent cooperative launch per RK
// stage on the fused tile body (stage_fused.cu); every box fused-eligible and
// with the same reconstruction.
struct EnsFused {
  void *boxes = nullptr;   // device records, one per box
  void *tmaps = nullptr;   // the boxes' W tensor maps (device memory)
  long *pref = nullptr;    // the phases' prefix sums of work items
  int nbox = 0, blocks = 0, per_sm = 0;
  bool pph = false;
};
cudaError_t ens_fused_create(const GridView *views, int nbox, EnsFused *out);
void ens_fused_destroy(EnsFused *e);
cudaError_t launch_ens_fused(const EnsFused &E, int stage, int nstages, float b, cudaStream_t s);

// Stellar EOS path (kernels_stellar.cu)
// cfl_dmax non-null: also the CFL step of this state into *dt (the step's
// first stage; cfl_dmax is the grid's double-bits maximum, left at zero).
template <typename R>
void launch_eos_cells(const DevGeo &G, const double *U, const double *Bf, const float *dU, const float *dB,
                      const double *Tin, double *Tout, R *W, int *dflag, cudaStream_t s, int *nl, Prof *prof,
                      unsigned long long *cfl_dmax = nullptr, double *dt = nullptr, int pm = 0);
void launch_dt_stellar(const DevGeo &G, bool fp32, const double *U, const double *Bf, const double *T,
                       unsigned long long *dmax, double *dt, int *dflag, cudaStream_t s, int *nl, Prof *prof);
cudaError_t stellar_background(const DevGeo &G, int L, double *bg, const double *bgX_host);
void launch_prim_to_cons(const DevGeo &G, const double *prim, double *U, const double *Bf, double *T, int *dflag,
                         cudaStream_t s);
const eos::Table *eos_table_view(const struct phl_eos_table *t);
mlp::Dev mlp_view(const struct phl_mlp *m);

// Index of component v of work cell q in W.  FP64 path: one plane of wtot
// values per component.  FP32 path: planes of float4, components 4h..4h+3 of
// every cell in plane h (wstr / 4 planes), so one cell's deviations are two to
// four 16-byte loads, a face's stencil touches 4 cells instead of 4 x nw
// lines, and a tile staged in shared memory keeps the float4 rows of
// consecutive cells contiguous (no bank conflicts between neighbouring lanes).
template <typename R>
__host__ __device__ __forceinline__ long wix(const DevGeo &G, int v, long q) {
  if constexpr (sizeof(R) == 4) return (((long)(v >> 2) * G.wtot + q) << 2) + (v & 3);
  else return (long)v * G.wtot + q;
}

// FP32 path: after the interleaved W, four planes of per-cell auxiliaries for
// the kernels that need one value per cell: the pressure deviation (shock
// flags) and the cell-centred EMF E = -u x B (Contact-CT), written with W.
enum { AUX_P = 0, AUX_E = 1, NAUX = 4 };
__host__ __device__ __forceinline__ long waux(const DevGeo &G, int a, long q) {
  return (long)G.wstr * G.wtot + (long)a * G.wtot + q;
}
__device__ __forceinline__ void write_aux(const DevGeo &G, float *W, long q, const float *w) {
  W[waux(G, AUX_P, q)] = w[W_P];
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    const int A = (D + 1) % 3, B = (D + 2) % 3;
    W[waux(G, AUX_E + D, q)] = -(w[W_VX + A] * w[W_BX + B] - w[W_VX + B] * w[W_BX + A]);
  }
}

// Scale of conserved variable v of the mixed form (rho, m, E, rho X).
__host__ __device__ __forceinline__ double usc(const DevGeo &G, int v) {
  return (v >= 1 && v <= 3) ? G.sc_m : (v == 4 ? G.sc_e : G.sc_rho);
}
__host__ __device__ __forceinline__ int uexp(const DevGeo &G, int v) {
  return (v >= 1 && v <= 3) ? G.e_m : (v == 4 ? G.e_e : G.e_rho);
}
__host__ __device__ __forceinline__ double iusc(const DevGeo &G, int v) {
  return (v >= 1 && v <= 3) ? G.isc_m : (v == 4 ? G.isc_e : G.isc_rho);
}

// Records the calling thread's last-error message (phl_last_error) and
// returns st (phl_api.cu).
int set_error(int st, const char *fmt, ...);

// FP64 multi-kernel stage (kernels_fp64.cu)
void launch_stage_fp64(const DevGeo &G, const StageBufs &B, cudaStream_t s, int *nlaunch, Prof *prof);
void launch_dt_fp64(const DevGeo &G, const double *U, const double *Bf, double *T, unsigned long long *dmax,
                    double *dt, int *dflag, cudaStream_t s, int *nlaunch, Prof *prof);
void launch_set_scalar(double *p, double v, cudaStream_t s, Prof *prof);

}  // namespace phl
