// kernels_stellar.cu -- stage steps of the stellar EOS path (Sect. 2.2):
// the Newton inversion e_int -> T once per interior cell, ghost cells filled
// from their source cells, the background's auxiliary indices, the CFL step,
// and the primitive -> conserved conversion used to load a state.
#include <math.h>

#include "eos_stellar.cuh"
#include "phl_internal.cuh"
#include "stage_common.cuh"

namespace phl {
using namespace stage;
namespace {

// Mean mass number and electron fraction of normalised mass fractions.
template <typename R>
__device__ __forceinline__ void mixture(const DevGeo &G, const R *X, R &abar, R &ye, R *iabar = nullptr) {
  R sx = R(0), sa = R(0), sz = R(0);
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) sx += X[l];
  // 1/A and Z/A of each species are constants of the grid: two reciprocals
  // per cell (GB300's FP64 divisions are a dozen FP64-pipe instructions)
  const R isx = R(1) / sx;
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) {
      const R x = X[l] * isx;
      sa += x * (R)G.iAcomp[l];
      sz += x * (R)G.ZoAcomp[l];
    }
  abar = R(1) / sa;
  ye = sz;
  if (iabar) *iabar = sa;
}

// Stage-input state of interior cell p: density, velocity, cell-centred B,
// specific internal energy, mass fractions.
struct CellState {
  double rho, irho, v[3], b[3], eint, X[PHL_NSPEC_MAX];
};
__device__ __forceinline__ CellState cell_state(const DevGeo &G, long p, const double *__restrict__ U,
                                                const double *__restrict__ Bf, const float *__restrict__ dU,
                                                const float *__restrict__ dB) {
  CellState c;
  const long pl = G.plane;
  double u[5 + PHL_NSPEC_MAX];
  // the FP32 increments enter through the integer pipe (f2d_scaled: the
  // conversion and the power-of-two unit scale in one; GB300 converts
  // FP32 -> FP64 at the FP64 rate)
#pragma unroll
  for (int v = 0; v < 5 + PHL_NSPEC_MAX; ++v) {
    if (v >= G.nv) continue;
    u[v] = U[v * pl + p];
    if (dU) u[v] += f2d_scaled(dU[v * pl + p], uexp(G, v));
  }
  double bl[3] = {Bf[p], Bf[pl + p], Bf[2 * pl + p]};
  double bh[3] = {Bf[p + 1], Bf[pl + p + G.sy], Bf[2 * pl + p + G.sz]};
  if (dB) {
    const int k = G.e_b;
    bl[0] += f2d_scaled(dB[p], k); bl[1] += f2d_scaled(dB[pl + p], k); bl[2] += f2d_scaled(dB[2 * pl + p], k);
    bh[0] += f2d_scaled(dB[p + 1], k); bh[1] += f2d_scaled(dB[pl + p + G.sy], k);
    bh[2] += f2d_scaled(dB[2 * pl + p + G.sz], k);
  }
  c.rho = u[0];
  const double ir = 1.0 / c.rho;   // one reciprocal for the cell
  c.irho = ir;
  c.v[0] = u[1] * ir; c.v[1] = u[2] * ir; c.v[2] = u[3] * ir;
  c.b[0] = 0.5 * (bl[0] + bh[0]); c.b[1] = 0.5 * (bl[1] + bh[1]); c.b[2] = 0.5 * (bl[2] + bh[2]);
  c.eint = u[4] * ir - 0.5 * (c.v[0] * c.v[0] + c.v[1] * c.v[1] + c.v[2] * c.v[2]) -
           0.5 * (c.b[0] * c.b[0] + c.b[1] * c.b[1] + c.b[2] * c.b[2]) * ir;
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) c.X[l] = u[5 + l] * ir;
  return c;
}

// First guesses from the temperature-guess network (use_mlp = 1: every cell;
// 2: cells without a previous temperature, Tin <= 0), written to Tg; the other
// cells get their previous temperature.  Warp-collective BF16 tensor-core
// inference; kept out of the Newton kernel so that one keeps few registers.
__global__ void k_mlp_guess(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                            const float *__restrict__ dU, const float *__restrict__ dB,
                            const double *__restrict__ Tin, double *__restrict__ Tg) {
  int c[3];
  const bool in = cell3(box, c);
  if (!in) { c[0] = box.lo[0]; c[1] = box.lo[1]; c[2] = box.lo[2]; }   // harmless stand-in for the warp
  const long p = sidx(G, c[0], c[1], c[2]);
  const double T = Tin[p];
  const bool need = G.use_mlp == 1 || !(T > 0.0);
  if (!__any_sync(0xffffffffu, in && need)) {
    if (in) Tg[p] = T;
    return;
  }
  const CellState s = cell_state(G, p, U, Bf, dU, dB);
  const bool ok_in = in && s.rho > 0.0 && s.eint > 0.0;
  const float lr = ok_in ? (float)log10(s.rho) : G.mlp.c[0];
  const float le = ok_in ? (float)log10(s.eint) : G.mlp.c[1];
  const float x0 = ok_in ? (float)(s.X[0] / (s.X[0] + (G.nspec > 1 ? s.X[1] : 0.0))) : G.mlp.c[2];
  const float lt = mlp::guess_log10T(G.mlp, lr, le, x0);
  if (in) Tg[p] = need ? exp10((double)lt) : T;
}

// Interior cells: conserved -> primitives with the EOS.  FP64 path (R = double):
// FP64 Newton.  Mixed path (R = float): FP64 Newton from a guess within 1e-4,
// else FP32 Newton iterations to about 1e-5 finished in FP64 to the same
// tolerance.  First guess: Tg (the network's, with use_mlp) or Tin; with the
// network the previous temperature is the fallback.  Writes W and T_out.
// One interior cell of k_eos_cells: inversion, deviations, and (rate) the
// CFL sum of the cell, returned (0 otherwise).
// pm (mixed form, G.pred): 1 writes the record of each cell's inversion,
// 2 also starts from the previous one's (eos_invert_rec; a cleared record,
// 1/c_v = 0, gives the plain start), 0 neither.
template <typename R>
__device__ __forceinline__ double eos_cell_step(const DevGeo &G, const int *c, const double *__restrict__ U,
                                                const double *__restrict__ Bf, const float *__restrict__ dU,
                                                const float *__restrict__ dB, const double *__restrict__ Tin,
                                                double *__restrict__ Tout, R *__restrict__ W, int *dflag,
                                                bool rate, int pm) {
  const long p = sidx(G, c[0], c[1], c[2]);
  const CellState cs = cell_state(G, p, U, Bf, dU, dB);
  const double rho = cs.rho, eint = cs.eint;
  const double vx = cs.v[0], vy = cs.v[1], vz = cs.v[2], bx = cs.b[0], by = cs.b[1], bz = cs.b[2];
  double X[PHL_NSPEC_MAX];
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l) X[l] = cs.X[l];
  double abar, ye, iab;
  mixture<double>(G, X, abar, ye, &iab);
  double T = G.use_mlp ? Tout[p] : Tin[p];   // Tout holds the network's guesses (k_mlp_guess)
  eos::EosOut<double> o;
  int it;
  if (sizeof(R) == 4 && pm) {
    const long pl = G.plane;
    eos::Pred pr{};
    double *rp = G.pred + p;
    if (pm == 2) pr = eos::Pred{rp[0], rp[pl], rp[2 * pl], rp[3 * pl], rp[4 * pl], rp[5 * pl], rp[6 * pl], rp[7 * pl]};
    it = eos::eos_invert_rec(G.tab, rho, cs.irho, eint, abar, iab, ye, T, G.newton_tol, G.newton_maxit, o, pr,
                             pm == 2);
    rp[0] = pr.rho; rp[pl] = pr.e; rp[2 * pl] = pr.icv; rp[3 * pl] = pr.er;
    rp[4 * pl] = pr.lnT; rp[5 * pl] = pr.iT; rp[6 * pl] = pr.x; rp[7 * pl] = pr.ine;
  } else {
    it = sizeof(R) == 8 ? eos::eos_invert<double>(G.tab, rho, eint, abar, ye, T, G.newton_tol, G.newton_maxit, o)
                        : eos::eos_invert_mixed(G.tab, rho, eint, abar, ye, T, G.newton_tol, G.newton_maxit, o);
  }
  if (it < 0 && G.use_mlp) {   // the plain Newton from the previous temperature is the fallback
    T = Tin[p];
    it = sizeof(R) == 8 ? eos::eos_invert<double>(G.tab, rho, eint, abar, ye, T, G.newton_tol, G.newton_maxit, o)
                        : eos::eos_invert_mixed(G.tab, rho, eint, abar, ye, T, G.newton_tol, G.newton_maxit, o);
  }
  if (G.niter) {   // warp sum, one atomic per warp
    const unsigned m = __activemask();
    const unsigned tot = __reduce_add_sync(m, it > 0 ? (unsigned)it : 0u);
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(G.niter, (unsigned long long)tot);
  }
  if (it < 0 || !(o.P > 0.0) || !(rho > 0.0)) atomicOr(dflag, it < 0 ? FLAG_NEWTON : FLAG_NEG);
  Tout[p] = T;
  const Bg b = bg_cell(G, c[2]);
  const long q = widx(G, c[0], c[1], c[2]);
  const long wt = G.wtot;
  if constexpr (sizeof(R) == 4) {
    // FP32 deviations in the mixed form's power-of-two units, converted on
    // the integer pipe (d2f_scaled: the unit scale folded into the exponent)
    const int ev = G.e_m - G.e_rho;   // v_s = rho_s v_s / rho_s
    W[wix<R>(G, W_RHO, q)] = d2f_scaled(rho - b.rho, -G.e_rho);
    W[wix<R>(G, W_VX, q)] = d2f_scaled(vx, -ev); W[wix<R>(G, W_VY, q)] = d2f_scaled(vy, -ev);
    W[wix<R>(G, W_VZ, q)] = d2f_scaled(vz, -ev);
    W[wix<R>(G, W_BX, q)] = d2f_scaled(bx, -G.e_b); W[wix<R>(G, W_BY, q)] = d2f_scaled(by, -G.e_b);
    W[wix<R>(G, W_BZ, q)] = d2f_scaled(bz, -G.e_b);
    W[wix<R>(G, W_P, q)] = d2f_scaled(o.P - b.p, -G.e_e);
    W[wix<R>(G, W_GE, q)] = d2f_scaled(o.ge - b.ge, 0);
    W[wix<R>(G, W_GC, q)] = d2f_scaled(o.gc - b.gc, 0);
#pragma unroll
    for (int l = 0; l < PHL_NSPEC_MAX; ++l)
      if (l < G.nspec) W[wix<R>(G, W_X0 + l, q)] = d2f_scaled(X[l], 0);
  } else {
    W[wix<R>(G, W_RHO, q)] = rho - b.rho;
    W[wix<R>(G, W_VX, q)] = vx; W[wix<R>(G, W_VY, q)] = vy; W[wix<R>(G, W_VZ, q)] = vz;
    W[wix<R>(G, W_BX, q)] = bx; W[wix<R>(G, W_BY, q)] = by; W[wix<R>(G, W_BZ, q)] = bz;
    W[wix<R>(G, W_P, q)] = o.P - b.p;
    W[wix<R>(G, W_GE, q)] = o.ge - b.ge;
    W[wix<R>(G, W_GC, q)] = o.gc - b.gc;
#pragma unroll
    for (int l = 0; l < PHL_NSPEC_MAX; ++l)
      if (l < G.nspec) W[wix<R>(G, W_X0 + l, q)] = X[l];
  }
  if constexpr (sizeof(R) == 4) {
    float w[W_P + 1];
#pragma unroll
    for (int v = 0; v <= W_P; ++v) w[v] = W[wix<float>(G, v, q)];
    write_aux(G, W, q, w);
  }
  if (!rate) return 0.0;
  // CFL sum of the cell (as k_dt_stellar, from this stage's inversion)
  if constexpr (sizeof(R) == 4) {
    // the mixed form's CFL step needs a few digits: FP32 (CGS magnitudes stay
    // inside its range: a^2 ~ 1e17, (a^2 + b^2)^2 ~ 1e34), the FP64 values
    // converted on the integer pipe
    const float fr = d2f_scaled(rho, 0), ifr = 1.0f / fr;
    const float a2 = d2f_scaled(o.gc * o.P, 0) * ifr;
    const float fv[3] = {d2f_scaled(vx, 0), d2f_scaled(vy, 0), d2f_scaled(vz, 0)};
    const float fb[3] = {d2f_scaled(bx, 0), d2f_scaled(by, 0), d2f_scaled(bz, 0)};
    const float b2 = (fb[0] * fb[0] + fb[1] * fb[1] + fb[2] * fb[2]) * ifr;
    float sum = 0.0f;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const float bd2 = fb[d] * fb[d] * ifr;
      const float disc = fmaxf((a2 + b2) * (a2 + b2) - 4.0f * a2 * bd2, 0.0f);
      sum += (fabsf(fv[d]) + sqrtf(0.5f * (a2 + b2 + sqrtf(disc)))) * (float)G.idx[d];
    }
    return (sum == sum) ? (double)sum : INFINITY;
  } else {
    const double a2 = o.gc * o.P / rho, b2 = (bx * bx + by * by + bz * bz) / rho;
    const double vv[3] = {vx, vy, vz}, bb[3] = {bx, by, bz};
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const double bd2 = bb[d] * bb[d] / rho;
      const double disc = fmax((a2 + b2) * (a2 + b2) - 4.0 * a2 * bd2, 0.0);
      sum += (fabs(vv[d]) + sqrt(0.5 * (a2 + b2 + sqrt(disc)))) / G.dx[d];
    }
    return (sum == sum) ? sum : INFINITY;
  }
}

template <typename R>
__global__ void __launch_bounds__(256, 2) k_eos_cells(DevGeo G, Box box, const double *__restrict__ U,
                                                       const double *__restrict__ Bf, const float *__restrict__ dU,
                                                       const float *__restrict__ dB, const double *__restrict__ Tin,
                                                       double *__restrict__ Tout, R *__restrict__ W, int *dflag,
                                                       unsigned long long *cfl_dmax, int pm) {
  int c[3];
  const bool in = cell3(box, c);
  if (cfl_dmax) {   // the CFL rate of the step's own state (Eq. cfl), from this inversion
    double m = 0.0;
    if (in) m = eos_cell_step<R>(G, c, U, Bf, dU, dB, Tin, Tout, W, dflag, true, pm);
    for (int o2 = 16; o2 > 0; o2 >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o2));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
      atomicMax(cfl_dmax, (unsigned long long)__double_as_longlong(v));
    }
    return;
  }
  if (!in) return;
  eos_cell_step<R>(G, c, U, Bf, dU, dB, Tin, Tout, W, dflag, false, pm);
}

// Cells of the work layout outside the interior take the deviations of the
// interior cell their data comes from (Table bcs), with the reflecting flips.
template <typename R>
__global__ void k_ghost_fill(DevGeo G, Box box, R *__restrict__ W) {
  int c[3];
  if (!cell3(box, c)) return;
  int s[3];
  bool fl[3], ghost = false;
  for (int d = 0; d < 3; ++d) {
    fl[d] = false;
    s[d] = G.act[d] ? cell_src(c[d], G.n[d], G.bc[d][0], G.bc[d][1], fl[d]) : 0;
    ghost |= s[d] != c[d];
  }
  if (!ghost) return;
  const long qd = widx(G, c[0], c[1], c[2]), qs = widx(G, s[0], s[1], s[2]);
  const long wt = G.wtot;
#pragma unroll
  for (int v = 0; v < NW_MAX; ++v) {
    if (v >= G.nw) continue;
    R x = W[wix<R>(G, v, qs)];
    const bool flip = (v >= W_VX && v <= W_VZ && fl[v - W_VX]) || (v >= W_BX && v <= W_BZ && fl[v - W_BX]);
    W[wix<R>(G, v, qd)] = flip ? -x : x;
  }
  if constexpr (sizeof(R) == 4) {   // the ghost's auxiliaries from its (flipped) values
    float w[W_P + 1];
#pragma unroll
    for (int v = 0; v <= W_P; ++v) w[v] = W[wix<float>(G, v, qd)];
    write_aux(G, W, qd, w);
  }
}

// CFL condition with the stellar EOS (T guesses read, not written).
template <typename R>
__global__ void k_dt_stellar(DevGeo G, Box box, const double *__restrict__ U, const double *__restrict__ Bf,
                             const double *__restrict__ Tin, unsigned long long *dmax, int *dflag) {
  int c[3];
  double m = 0.0;
  if (cell3(box, c)) {
    const long p = sidx(G, c[0], c[1], c[2]);
    const long pl = G.plane;
    const double rho = U[p];
    const double v[3] = {U[pl + p] / rho, U[2 * pl + p] / rho, U[3 * pl + p] / rho};
    const double bc[3] = {0.5 * (Bf[p] + Bf[p + 1]), 0.5 * (Bf[pl + p] + Bf[pl + p + G.sy]),
                          0.5 * (Bf[2 * pl + p] + Bf[2 * pl + p + G.sz])};
    const double b2 = bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2];
    const double eint = U[4 * pl + p] / rho - 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - 0.5 * b2 / rho;
    double X[PHL_NSPEC_MAX];
#pragma unroll
    for (int l = 0; l < PHL_NSPEC_MAX; ++l)
      if (l < G.nspec) X[l] = U[(5 + l) * pl + p] / rho;
    double abar, ye;
    mixture<double>(G, X, abar, ye);
    R T = (R)Tin[p];
    eos::EosOut<R> o;
    if (sizeof(R) == 8) {
      if (eos::eos_invert<R>(G.tab, (R)rho, (R)eint, (R)abar, (R)ye, T, (R)G.newton_tol, G.newton_maxit, o) < 0)
        atomicOr(dflag, FLAG_NEWTON);
    } else {
      // the CFL step needs c_s to a few digits: FP32 Newton to 1e-5 (FP32's own
      // floor for ln n, ln T is ~1e-6); a stalled iteration keeps its last,
      // bracketed iterate
      if (eos::eos_invert<R>(G.tab, (R)rho, (R)eint, (R)abar, (R)ye, T, (R)1e-5, 16, o) < 0 &&
          !eos::eos_rt<R>(G.tab, (R)rho, T, (R)abar, (R)ye, o))
        atomicOr(dflag, FLAG_NEWTON);
    }
    const double a2 = (double)o.gc * (double)o.P / rho, bb = b2 / rho;
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (!G.act[d]) continue;
      const double bd2 = bc[d] * bc[d] / rho;
      const double disc = fmax((a2 + bb) * (a2 + bb) - 4.0 * a2 * bd2, 0.0);
      s += (fabs(v[d]) + sqrt(0.5 * (a2 + bb + sqrt(disc)))) / G.dx[d];
    }
    m = (s == s) ? s : INFINITY;
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o2));
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
    atomicMax(dmax, (unsigned long long)__double_as_longlong(v));
  }
}

__global__ void k_dt_finalize_st(double cfl, unsigned long long *dmax, double *dt) {
  *dt = cfl / __longlong_as_double((long long)*dmax);
  *dmax = 0ull;
}

// P -> T at fixed rho (Newton on P, bracketed in the table's range).
__device__ bool p_to_T(const DevGeo &G, double rho, double P, double abar, double ye, double &T,
                       eos::EosOut<double> &o) {
  double lo = exp(G.tab.y0), hi = exp(G.tab.y0 + (G.tab.ny - 1) * G.tab.dy);
  if (!(T > lo && T < hi)) T = sqrt(lo * hi);
  for (int it = 0; it < 200; ++it) {
    if (!eos::eos_rt<double>(G.tab, rho, T, abar, ye, o)) return false;
    const double dp = P - o.P;
    if (fabs(dp) <= 1e-14 * P) return true;
    if (dp > 0.0) lo = T; else hi = T;
    double Tn = T + dp / o.PT;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    T = Tn;
  }
  return false;
}

// Background of the stellar path: T_hat, gamma_e, gamma_c at centres and
// z-faces and E_hat = rho_hat e(rho_hat, T_hat) at centres, from rho_hat, P_hat.
__global__ void k_bg_stellar(DevGeo G, int L, double *bg, double *bgX, int *fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * L) return;
  const bool face = i >= L;
  const int q = face ? i - L : i;
  if (!face && q == L - 1) return;          // centres have one value fewer
  const double rho = bg[(face ? 2 : 0) * L + q], P = bg[(face ? 3 : 1) * L + q];
  double abar, ye;
  mixture<double>(G, bgX, abar, ye);
  double T = 1e9;
  eos::EosOut<double> o;
  if (!p_to_T(G, rho, P, abar, ye, T, o)) { atomicOr(fail, 1); return; }
  bg[(face ? 6 : 4) * L + q] = o.ge;
  bg[(face ? 7 : 5) * L + q] = o.gc;
  if (!face) bg[8 * L + q] = rho * o.e;
}

// Primitive state (rho, v, P, X) -> conserved state and temperature.
__global__ void k_prim_to_cons(DevGeo G, Box box, const double *__restrict__ prim, long np_,
                               double *__restrict__ U, const double *__restrict__ Bf, double *__restrict__ T,
                               int *dflag) {
  int c[3];
  if (!cell3(box, c)) return;
  const long a = c[0] + (long)G.n[0] * (c[1] + (long)G.n[1] * c[2]);   // ABI index
  const long p = sidx(G, c[0], c[1], c[2]);
  const long pl = G.plane;
  const double rho = prim[a], P = prim[4 * np_ + a];
  const double v[3] = {prim[np_ + a], prim[2 * np_ + a], prim[3 * np_ + a]};
  double X[PHL_NSPEC_MAX];
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) X[l] = prim[(5 + l) * np_ + a];
  const double bc[3] = {0.5 * (Bf[p] + Bf[p + 1]), 0.5 * (Bf[pl + p] + Bf[pl + p + G.sy]),
                        0.5 * (Bf[2 * pl + p] + Bf[2 * pl + p + G.sz])};
  double e;
  double Tc = 0.0;
  if (G.eos == 0) {
    e = P / ((G.gamma - 1.0) * rho);
  } else {
    double abar, ye;
    mixture<double>(G, X, abar, ye);
    Tc = 1e9;
    eos::EosOut<double> o;
    if (!p_to_T(G, rho, P, abar, ye, Tc, o)) atomicOr(dflag, FLAG_NEWTON);
    e = o.e;
  }
  U[p] = rho;
  for (int d = 0; d < 3; ++d) U[(1 + d) * pl + p] = rho * v[d];
  U[4 * pl + p] = rho * e + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) +
                  0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
#pragma unroll
  for (int l = 0; l < PHL_NSPEC_MAX; ++l)
    if (l < G.nspec) U[(5 + l) * pl + p] = rho * X[l];
  if (T) T[p] = Tc;
}

}  // namespace

template <typename R>
void launch_eos_cells(const DevGeo &G, const double *U, const double *Bf, const float *dU, const float *dB,
                      const double *Tin, double *Tout, R *W, int *dflag, cudaStream_t s, int *nl, Prof *prof,
                      unsigned long long *cfl_dmax, double *dt, int pm) {
  Box bi = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  if (G.use_mlp) {
    PHL_LAUNCH(KC_PRIM, prof, s, k_mlp_guess<<<grid3(bi), block3(bi), 0, s>>>(G, bi, U, Bf, dU, dB, Tin, Tout));
    if (nl) *nl += 1;
  }
  PHL_LAUNCH(KC_PRIM, prof, s,
             k_eos_cells<R><<<grid3(bi), block3(bi), 0, s>>>(G, bi, U, Bf, dU, dB, Tin, Tout, W, dflag, cfl_dmax,
                                                             G.pred ? pm : 0));
  if (cfl_dmax) {   // the step's CFL step from the rates this inversion folded in
    PHL_LAUNCH(KC_DT, prof, s, k_dt_finalize_st<<<1, 1, 0, s>>>(G.cfl, cfl_dmax, dt));
    if (nl) *nl += 1;
  }
  int l[3], h[3];
  for (int d = 0; d < 3; ++d) {
    if (G.act[d]) { l[d] = -G.ge[d]; h[d] = G.n[d] + G.ge[d]; } else { l[d] = 0; h[d] = 1; }
  }
  Box be = make_box(l[0], h[0], l[1], h[1], l[2], h[2]);
  PHL_LAUNCH(KC_PRIM, prof, s, k_ghost_fill<R><<<grid3(be), block3(be), 0, s>>>(G, be, W));
  if (nl) *nl += 2;
}
template void launch_eos_cells<double>(const DevGeo &, const double *, const double *, const float *, const float *,
                                       const double *, double *, double *, int *, cudaStream_t, int *, Prof *,
                                       unsigned long long *, double *, int);
template void launch_eos_cells<float>(const DevGeo &, const double *, const double *, const float *, const float *,
                                      const double *, double *, float *, int *, cudaStream_t, int *, Prof *,
                                      unsigned long long *, double *, int);

void launch_dt_stellar(const DevGeo &G, bool fp32, const double *U, const double *Bf, const double *T,
                       unsigned long long *dmax, double *dt, int *dflag, cudaStream_t s, int *nl, Prof *prof) {
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  if (fp32)
    PHL_LAUNCH(KC_DT, prof, s, k_dt_stellar<float><<<grid3(b), block3(b), 0, s>>>(G, b, U, Bf, T, dmax, dflag));
  else
    PHL_LAUNCH(KC_DT, prof, s, k_dt_stellar<double><<<grid3(b), block3(b), 0, s>>>(G, b, U, Bf, T, dmax, dflag));
  PHL_LAUNCH(KC_DT, prof, s, k_dt_finalize_st<<<1, 1, 0, s>>>(G.cfl, dmax, dt));
  if (nl) *nl += 2;
}

cudaError_t stellar_background(const DevGeo &G, int L, double *bg, const double *bgX_host) {
  double *dX = nullptr;
  int *fail = nullptr;
  cudaError_t e = cudaMalloc(&dX, PHL_NSPEC_MAX * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&fail, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dX, bgX_host, PHL_NSPEC_MAX * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(fail, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_bg_stellar<<<(2 * L + 63) / 64, 64>>>(G, L, bg, dX, fail);
    int f = 0;
    e = cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && f) e = cudaErrorInvalidValue;
  }
  cudaFree(dX);
  cudaFree(fail);
  return e;
}

void launch_prim_to_cons(const DevGeo &G, const double *prim, double *U, const double *Bf, double *T, int *dflag,
                         cudaStream_t s) {
  Box b = make_box(0, G.n[0], 0, G.n[1], 0, G.n[2]);
  k_prim_to_cons<<<grid3(b), block3(b), 0, s>>>(G, b, prim, b.n, U, Bf, T, dflag);
}

}  // namespace phl
