/* diffusion.c -- thermal diffusion by RKL2 super-time-stepping (Sect. 2.10),
 * the oracle's plain FP64 version.  Test infrastructure only: used by the
 * tests and the benchmark's CPU legs, never by the library.
 *
 * Operator (Sect. 2.10, Eq. diffusion_eint): with the density, velocity,
 * magnetic field and mass fractions held fixed,
 *     rho d(e_int)/dt = div(K grad T),
 * for an ideal gas with T = e_int / c_v (code units), and a conductivity
 * K = k0 T^nT / rho^nR (nT, nR small non-negative integers: a constant K has
 * nT = nR = 0; radiative diffusion with a constant opacity, K = 4acT^3 / (3
 * kappa rho), has nT = 3, nR = 1).
 *
 * Space (Sect. 2.10): the face flux is the centred difference
 * -K_f (T_R - T_L) / dx with K_f the harmonic mean 2 K_L K_R / (K_L + K_R) of
 * the two cells' conductivities (zero where both vanish); summed over the six
 * faces this is the conservative seven-point form.  Reading: a side that is not
 * periodic carries no flux (the reflecting mirror and the outflow copy both
 * give the ghost the cell's own temperature).
 *
 * Option (Sect. 2.10, last paragraph): with delta_T the operator acts on the
 * deviation from the background temperature, div(K grad (T - T_hat)), T_hat =
 * P_hat / ((gamma - 1) rho_hat c_v) of the well-balancing background at the
 * cell centres; K stays that of the full temperature.
 *
 * Time: RKL2 (Meyer, Balsara & Aslam 2012) over the whole step dt, in the
 * paper's stage form (items i-iv of Sect. 2.10), with the paper's count
 *     N_STS = max(1 + floor((sqrt(9 + 16 dt / dt_p) - 1) / 2), 3),
 *     dt_p  = 1/2 [max_cells sum_s D / dx_s^2]^-1,  D = K / (rho c_v),
 * evaluated from the state at the start of the step.  The total energy takes
 * the change rho (e_int^(N) - e_int^(0)).
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

#define BG_GHOST 3   /* the background profiles carry nz + 6 values: three ghost layers per side */

/* RKL2 coefficients of an s-stage step (Meyer, Balsara & Aslam 2012), index
 * j = 1..s: b_0 = b_1 = b_2 = 1/3, b_j = (j^2 + j - 2) / (2 j (j + 1)),
 * a_j = 1 - b_j, w_1 = 4 / (s^2 + s - 2), mu~_1 = b_1 w_1, and for j >= 2
 * mu_j = (2j - 1)/j b_j / b_{j-1}, nu_j = -(j - 1)/j b_j / b_{j-2},
 * mu~_j = mu_j w_1, gamma~_j = -a_{j-1} mu~_j. */
void ora_rkl2_coeffs(int s, double *mu, double *nu, double *mut, double *gat) {
  double *b = (double *)malloc((size_t)(s + 1) * sizeof(double));
  for (int j = 0; j <= s; ++j)
    b[j] = j <= 2 ? 1.0 / 3.0 : (double)(j * j + j - 2) / (2.0 * j * (j + 1));
  const double w1 = 4.0 / (double)(s * s + s - 2);
  for (int j = 0; j <= s; ++j) { mu[j] = 0.0; nu[j] = 0.0; mut[j] = 0.0; gat[j] = 0.0; }
  mut[1] = b[1] * w1;
  for (int j = 2; j <= s; ++j) {
    mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1];
    nu[j] = -(j - 1.0) / j * b[j] / b[j - 2];
    mut[j] = mu[j] * w1;
    gat[j] = -(1.0 - b[j - 1]) * mut[j];
  }
  free(b);
}

/* The RKL2 step's amplification factor for y' = lambda y with z = lambda dt
 * (the same recurrence applied to a scalar). */
double ora_rkl2_amp(int s, double z) {
  double *mu = (double *)malloc(4 * (size_t)(s + 1) * sizeof(double));
  double *nu = mu + s + 1, *mut = nu + s + 1, *gat = mut + s + 1;
  ora_rkl2_coeffs(s, mu, nu, mut, gat);
  const double y0 = 1.0, l0 = z * y0;
  double ym2 = y0, ym1 = y0 + mut[1] * l0;
  for (int j = 2; j <= s; ++j) {
    const double y = mu[j] * ym1 + nu[j] * ym2 + (1.0 - mu[j] - nu[j]) * y0 + mut[j] * z * ym1 + gat[j] * l0;
    ym2 = ym1;
    ym1 = y;
  }
  free(mu);
  return ym1;
}

int ora_sts_stages(double dt, double dt_p) {
  const int n = 1 + (int)floor(0.5 * (sqrt(9.0 + 16.0 * dt / dt_p) - 1.0));
  return n < 3 ? 3 : n;
}

typedef struct {
  int n[3], act[3], per[3];
  double dx[3];
  long nc;
  const double *That;   /* background temperature per z layer (NULL: none subtracted) */
} dgrid;

static long cidx(const dgrid *g, int i, int j, int k) { return i + (long)g->n[0] * (j + (long)g->n[1] * k); }

static double powi(double x, int n) {
  double r = 1.0;
  for (int q = 0; q < n; ++q) r *= x;
  return r;
}

static double conductivity(const ora_diff *p, double T, double rho) {
  return p->k0 * powi(T, p->nT) / powi(rho, p->nR);
}

/* L(Y) = div(K grad T(Y)) / rho with T = Y / c_v */
static void diff_op(const dgrid *g, const ora_diff *p, const double *rho, const double *Y, double *K, double *out) {
  for (long q = 0; q < g->nc; ++q) K[q] = conductivity(p, Y[q] / p->cv, rho[q]);
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) {
        const int c[3] = {i, j, k};
        const long q = cidx(g, i, j, k);
        const double Tc = Y[q] / p->cv;
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (!g->act[d]) continue;
          double flux_sum = 0.0;   /* (K grad T) at the upper face minus at the lower face */
          for (int side = -1; side <= 1; side += 2) {
            int cc[3] = {c[0], c[1], c[2]};
            cc[d] += side;
            if (cc[d] < 0 || cc[d] >= g->n[d]) {
              if (!g->per[d]) continue;   /* no flux through a wall or an outflow side */
              cc[d] = (cc[d] + g->n[d]) % g->n[d];
            }
            const long qn = cidx(g, cc[0], cc[1], cc[2]);
            const double Ks = K[q] + K[qn];
            const double Kf = Ks > 0.0 ? 2.0 * K[q] * K[qn] / Ks : 0.0;   /* harmonic mean */
            double dT = Y[qn] / p->cv - Tc;
            if (g->That) dT -= g->That[cc[2]] - g->That[k];   /* the deviation T - T_hat */
            const double gradT = dT / g->dx[d];   /* toward the neighbour */
            flux_sum += Kf * gradT;
          }
          s += flux_sum / g->dx[d];
        }
        out[q] = s / rho[q];
      }
}

int ora_diffuse(const ora_cfg *cfg, double *cons, const double *bx, const double *by, const double *bz,
                const ora_diff *p, double dt, int max_stages, int *nsts_out) {
  dgrid g;
  g.nc = 1;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = cfg->n[d];
    g.act[d] = cfg->n[d] > 1;
    g.per[d] = cfg->bc[d][0] == ORA_PERIODIC;
    g.dx[d] = (cfg->hi[d] - cfg->lo[d]) / cfg->n[d];
    g.nc *= g.n[d];
  }
  if (!(p->cv > 0.0) || !(p->k0 >= 0.0) || p->nT < 0 || p->nR < 0 || !(dt > 0.0)) return -1;
  if (p->delta_T && !cfg->bg_rho_c) return -1;
  g.That = NULL;
  double *That = NULL;
  if (p->delta_T) {
    That = (double *)malloc((size_t)g.n[2] * sizeof(double));
    for (int k = 0; k < g.n[2]; ++k)
      That[k] = cfg->bg_p_c[k + BG_GHOST] / ((cfg->gamma - 1.0) * cfg->bg_rho_c[k + BG_GHOST] * p->cv);
    g.That = That;
  }
  const long nc = g.nc;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  double *buf = (double *)malloc(8 * (size_t)nc * sizeof(double));
  if (!buf) { free(That); return -1; }
  double *rho = buf, *Y0 = buf + nc, *L0 = buf + 2 * nc, *Ym2 = buf + 3 * nc, *Ym1 = buf + 4 * nc,
         *Y = buf + 5 * nc, *L = buf + 6 * nc, *K = buf + 7 * nc;
  /* e_int of the state, with rho, u and the cell-centred field fixed */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long q = cidx(&g, i, j, k);
        const double r = cons[q];
        const double ux = cons[nc + q] / r, uy = cons[2 * nc + q] / r, uz = cons[3 * nc + q] / r;
        const double bcx = 0.5 * (bx[i + (long)(nx + 1) * (j + (long)ny * k)] +
                                  bx[i + 1 + (long)(nx + 1) * (j + (long)ny * k)]);
        const double bcy = 0.5 * (by[i + (long)nx * (j + (long)(ny + 1) * k)] +
                                  by[i + (long)nx * (j + 1 + (long)(ny + 1) * k)]);
        const double bcz = 0.5 * (bz[i + (long)nx * (j + (long)ny * k)] + bz[i + (long)nx * (j + (long)ny * (k + 1))]);
        rho[q] = r;
        Y0[q] = cons[4 * nc + q] / r - 0.5 * (ux * ux + uy * uy + uz * uz) - 0.5 * (bcx * bcx + bcy * bcy + bcz * bcz) / r;
        if (!(r > 0.0) || !(Y0[q] > 0.0)) { free(buf); free(That); return -2; }
      }
  /* parabolic step limit and the number of stages */
  double dmax = 0.0;
  for (long q = 0; q < nc; ++q) {
    const double D = conductivity(p, Y0[q] / p->cv, rho[q]) / (rho[q] * p->cv);
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
      if (g.act[d]) s += D / (g.dx[d] * g.dx[d]);
    if (s > dmax) dmax = s;
  }
  int s = 3;
  if (dmax > 0.0) s = ora_sts_stages(dt, 0.5 / dmax);
  if (nsts_out) *nsts_out = s;
  if (s > max_stages) { free(buf); free(That); return -4; }
  double *co = (double *)malloc(4 * (size_t)(s + 1) * sizeof(double));
  double *mu = co, *nu = co + s + 1, *mut = nu + s + 1, *gat = mut + s + 1;
  ora_rkl2_coeffs(s, mu, nu, mut, gat);
  /* stages (Sect. 2.10, items i-iv) */
  diff_op(&g, p, rho, Y0, K, L0);
  for (long q = 0; q < nc; ++q) { Ym2[q] = Y0[q]; Ym1[q] = Y0[q] + mut[1] * dt * L0[q]; }
  for (int jst = 2; jst <= s; ++jst) {
    diff_op(&g, p, rho, Ym1, K, L);
    for (long q = 0; q < nc; ++q)
      Y[q] = mu[jst] * Ym1[q] + nu[jst] * Ym2[q] + (1.0 - mu[jst] - nu[jst]) * Y0[q] + mut[jst] * dt * L[q] +
             gat[jst] * dt * L0[q];
    double *t = Ym2; Ym2 = Ym1; Ym1 = Y; Y = t;
  }
  for (long q = 0; q < nc; ++q) cons[4 * nc + q] += rho[q] * (Ym1[q] - Y0[q]);
  free(co);
  free(buf);
  free(That);
  return 0;
}
