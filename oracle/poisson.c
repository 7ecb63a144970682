/* poisson.c -- the Poisson solver for the gravitational potential (Sect.
 * 2.12), the oracle's plain FP64 version.  Test infrastructure only: used by
 * the tests and the benchmark's CPU legs, never by the library.
 *
 * Grid: Cartesian, each axis stretched independently; the caller gives the
 * n_d + 1 face coordinates of every axis.  Reading: cell centres are the
 * midpoints of their faces; the ghost centre beyond a boundary face is the
 * mirror image of the first (last) centre in that face.
 *
 * Discretisation (Eq. poisson-FD): per axis, with dm = x_i - x_{i-1} and
 * dp = x_{i+1} - x_i between centres,
 *     L1 = 2 / (dm (dm + dp)),  L2 = -2 / (dm dp),  L3 = 2 / (dp (dm + dp)),
 * and sum_axes (L1 phi_{i-1} + L2 phi_i + L3 phi_{i+1}) = 4 pi G rho_i.  Ghost
 * potentials (boundary values) come from a multipole expansion of the mass in
 * the domain and move to the right-hand side, so the unknowns see the
 * operator A with zero ghosts.
 *
 * Boundary values (reading; the paper names the expansion, not its terms):
 * the exterior expansion of 1/|r - r'| about the centre of mass X of the cell
 * masses m = rho V, so the dipole vanishes; with R = r - X, x = r' - X,
 *     phi(R) = -G [ M/|R| + (1/2) Q_ij R_i R_j / |R|^5
 *                        + (1/6) O_ijk R_i R_j R_k / |R|^7 ],
 *     Q_ij  = sum m (3 x_i x_j - |x|^2 d_ij),
 *     O_ijk = sum m (15 x_i x_j x_k - 3 |x|^2 (x_i d_jk + x_j d_ik + x_k d_ij)),
 * the monopole always, the quadrupole for lmax >= 2, the octupole for lmax >= 3.
 *
 * Solver: BiCGSTAB (van der Vorst 1992) with the Jacobi preconditioner
 * diag(A)^-1 applied on the right, in the order of the preconditioned
 * algorithm of Barrett et al. (Templates, 1994); the residual recurrence is
 * the unpreconditioned one.  Stop when the RMS of the (weighted) residual is
 * below tol: weights 1/(4 pi G rho) (Eq. poisson-eps; needs rho > 0) or 1 (the
 * absolute RMS the paper uses for its sphere test); checked after the half
 * step (on s) and after the full step (on r).
 *
 * Gravity (Eq. grav_x..grav_z): g = -grad phi by the second-order central
 * difference for non-uniform spacing, ghost potentials at the boundaries.
 * (Reading: the last coefficient of the printed g_z uses dx_-, read as dz_-,
 * the form of the x and y components.)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define PI 3.14159265358979323846

typedef struct {
  int n[3];
  long nc;
  double *xc[3];            /* centres, index -1..n (n + 2 values, offset by one) */
  double *L1[3], *L2[3], *L3[3];
} pgrid;

static void pgrid_free(pgrid *g) {
  for (int d = 0; d < 3; ++d) {
    free(g->xc[d]);
    free(g->L1[d]);
    free(g->L2[d]);
    free(g->L3[d]);
  }
}

static int pgrid_init(pgrid *g, const ora_poisson *p) {
  memset(g, 0, sizeof(*g));
  g->nc = 1;
  for (int d = 0; d < 3; ++d) {
    const int n = p->n[d];
    if (n < 2) return -1;
    g->n[d] = n;
    g->nc *= n;
    for (int i = 0; i < n; ++i)
      if (!(p->xf[d][i + 1] > p->xf[d][i])) return -1;
    g->xc[d] = (double *)malloc((size_t)(n + 2) * sizeof(double));
    g->L1[d] = (double *)malloc((size_t)n * sizeof(double));
    g->L2[d] = (double *)malloc((size_t)n * sizeof(double));
    g->L3[d] = (double *)malloc((size_t)n * sizeof(double));
    double *xc = g->xc[d] + 1;   /* xc[-1..n] */
    for (int i = 0; i < n; ++i) xc[i] = 0.5 * (p->xf[d][i] + p->xf[d][i + 1]);
    xc[-1] = 2.0 * p->xf[d][0] - xc[0];
    xc[n] = 2.0 * p->xf[d][n] - xc[n - 1];
    for (int i = 0; i < n; ++i) {
      const double dm = xc[i] - xc[i - 1], dp = xc[i + 1] - xc[i];
      g->L1[d][i] = 2.0 / (dm * (dm + dp));
      g->L2[d][i] = -2.0 / (dm * dp);
      g->L3[d][i] = 2.0 / (dp * (dm + dp));
    }
  }
  return 0;
}

static double centre(const pgrid *g, int d, int i) { return g->xc[d][i + 1]; }   /* i = -1..n */

static long cid(const pgrid *g, int i, int j, int k) { return i + (long)g->n[0] * (j + (long)g->n[1] * k); }

/* ghost potential arrays: x faces [2][nz][ny], y faces [2][nz][nx], z faces [2][ny][nx] */
long ora_poisson_nghost(const int *n) { return 2L * ((long)n[1] * n[2] + (long)n[0] * n[2] + (long)n[0] * n[1]); }

static double *gh_x(const pgrid *g, double *gh, int side) { return gh + (long)side * g->n[1] * g->n[2]; }
static double *gh_y(const pgrid *g, double *gh, int side) {
  return gh + 2L * g->n[1] * g->n[2] + (long)side * g->n[0] * g->n[2];
}
static double *gh_z(const pgrid *g, double *gh, int side) {
  return gh + 2L * g->n[1] * g->n[2] + 2L * g->n[0] * g->n[2] + (long)side * g->n[0] * g->n[1];
}

/* mass, centre of mass, Q_ij and O_ijk (full index ranges) of the cell masses */
int ora_multipole_moments(const ora_poisson *p, const double *rho, double *M, double *X, double *Q, double *O) {
  pgrid g;
  if (pgrid_init(&g, p) != 0) { pgrid_free(&g); return -1; }
  double m0 = 0.0, mx[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const double V = (p->xf[0][i + 1] - p->xf[0][i]) * (p->xf[1][j + 1] - p->xf[1][j]) *
                         (p->xf[2][k + 1] - p->xf[2][k]);
        const double m = rho[cid(&g, i, j, k)] * V;
        const double r[3] = {centre(&g, 0, i), centre(&g, 1, j), centre(&g, 2, k)};
        m0 += m;
        for (int a = 0; a < 3; ++a) mx[a] += m * r[a];
      }
  *M = m0;
  for (int a = 0; a < 3; ++a) X[a] = m0 != 0.0 ? mx[a] / m0 : 0.0;
  for (int a = 0; a < 9; ++a) Q[a] = 0.0;
  for (int a = 0; a < 27; ++a) O[a] = 0.0;
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const double V = (p->xf[0][i + 1] - p->xf[0][i]) * (p->xf[1][j + 1] - p->xf[1][j]) *
                         (p->xf[2][k + 1] - p->xf[2][k]);
        const double m = rho[cid(&g, i, j, k)] * V;
        const double x[3] = {centre(&g, 0, i) - X[0], centre(&g, 1, j) - X[1], centre(&g, 2, k) - X[2]};
        const double x2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            Q[3 * a + b] += m * (3.0 * x[a] * x[b] - (a == b ? x2 : 0.0));
            for (int c = 0; c < 3; ++c)
              O[9 * a + 3 * b + c] += m * (15.0 * x[a] * x[b] * x[c] -
                                           3.0 * x2 * ((b == c ? x[a] : 0.0) + (a == c ? x[b] : 0.0) +
                                                       (a == b ? x[c] : 0.0)));
          }
      }
  pgrid_free(&g);
  return 0;
}

double ora_multipole_phi(double G, int lmax, double M, const double *X, const double *Q, const double *O, double x,
                         double y, double z) {
  const double R[3] = {x - X[0], y - X[1], z - X[2]};
  const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  double s = M / r;
  if (lmax >= 2) {
    double q = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) q += Q[3 * a + b] * R[a] * R[b];
    s += 0.5 * q / pow(r, 5);
  }
  if (lmax >= 3) {
    double o = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) o += O[9 * a + 3 * b + c] * R[a] * R[b] * R[c];
    s += o / 6.0 / pow(r, 7);
  }
  return -G * s;
}

/* ghost potentials from the multipole expansion of rho */
int ora_poisson_boundary(const ora_poisson *p, const double *rho, double *ghost) {
  pgrid g;
  if (pgrid_init(&g, p) != 0) { pgrid_free(&g); return -1; }
  double M, X[3], Q[9], O[27];
  ora_multipole_moments(p, rho, &M, X, Q, O);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  for (int side = 0; side < 2; ++side) {
    const int ix = side ? nx : -1, iy = side ? ny : -1, iz = side ? nz : -1;
    double *gx = gh_x(&g, ghost, side), *gy = gh_y(&g, ghost, side), *gz = gh_z(&g, ghost, side);
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        gx[j + (long)ny * k] = M != 0.0 ? ora_multipole_phi(p->G, p->lmax, M, X, Q, O, centre(&g, 0, ix),
                                                             centre(&g, 1, j), centre(&g, 2, k))
                                        : 0.0;
    for (int k = 0; k < nz; ++k)
      for (int i = 0; i < nx; ++i)
        gy[i + (long)nx * k] = M != 0.0 ? ora_multipole_phi(p->G, p->lmax, M, X, Q, O, centre(&g, 0, i),
                                                             centre(&g, 1, iy), centre(&g, 2, k))
                                        : 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        gz[i + (long)nx * j] = M != 0.0 ? ora_multipole_phi(p->G, p->lmax, M, X, Q, O, centre(&g, 0, i),
                                                             centre(&g, 1, j), centre(&g, 2, iz))
                                        : 0.0;
  }
  pgrid_free(&g);
  return 0;
}

/* neighbour value along axis d (side -1 / +1) of cell (i, j, k): the cell's,
 * or the ghost potential (ghost may be NULL: zero) */
static double nb(const pgrid *g, const double *phi, const double *ghost, int i, int j, int k, int d, int side) {
  int c[3] = {i, j, k};
  c[d] += side;
  if (c[d] >= 0 && c[d] < g->n[d]) return phi[cid(g, c[0], c[1], c[2])];
  if (!ghost) return 0.0;
  const int s = side > 0;
  if (d == 0) return gh_x(g, (double *)ghost, s)[j + (long)g->n[1] * k];
  if (d == 1) return gh_y(g, (double *)ghost, s)[i + (long)g->n[0] * k];
  return gh_z(g, (double *)ghost, s)[i + (long)g->n[0] * j];
}

static void apply(const pgrid *g, const double *phi, const double *ghost, double *out) {
  for (int k = 0; k < g->n[2]; ++k)
    for (int j = 0; j < g->n[1]; ++j)
      for (int i = 0; i < g->n[0]; ++i) {
        const int c[3] = {i, j, k};
        double s = 0.0;
        for (int d = 0; d < 3; ++d)
          s += g->L1[d][c[d]] * nb(g, phi, ghost, i, j, k, d, -1) + g->L2[d][c[d]] * phi[cid(g, i, j, k)] +
               g->L3[d][c[d]] * nb(g, phi, ghost, i, j, k, d, +1);
        out[cid(g, i, j, k)] = s;
      }
}

/* the discrete Laplacian with the given ghost potentials (NULL: zero) */
int ora_poisson_apply(const ora_poisson *p, const double *phi, const double *ghost, double *out) {
  pgrid g;
  if (pgrid_init(&g, p) != 0) { pgrid_free(&g); return -1; }
  apply(&g, phi, ghost, out);
  pgrid_free(&g);
  return 0;
}

int ora_gravity(const ora_poisson *p, const double *phi, const double *ghost, double *gx, double *gy, double *gz) {
  pgrid g;
  if (pgrid_init(&g, p) != 0) { pgrid_free(&g); return -1; }
  double *out[3] = {gx, gy, gz};
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const int c[3] = {i, j, k};
        for (int d = 0; d < 3; ++d) {
          const double dm = centre(&g, d, c[d]) - centre(&g, d, c[d] - 1);
          const double dp = centre(&g, d, c[d] + 1) - centre(&g, d, c[d]);
          const double fp = nb(&g, phi, ghost, i, j, k, d, +1), fm = nb(&g, phi, ghost, i, j, k, d, -1);
          out[d][cid(&g, i, j, k)] = -dm / (dp * (dp + dm)) * fp - (dp - dm) / (dp * dm) * phi[cid(&g, i, j, k)] +
                                     dp / (dm * (dp + dm)) * fm;
        }
      }
  pgrid_free(&g);
  return 0;
}

static double dot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long q = 0; q < n; ++q) s += a[q] * b[q];
  return s;
}

static double rms(long n, const double *w, const double *r) {
  double s = 0.0;
  for (long q = 0; q < n; ++q) s += (w[q] * r[q]) * (w[q] * r[q]);
  return sqrt(s / (double)n);
}

/* Solve for phi (in: the initial guess, out: the solution).  Returns 0 on
 * convergence, 1 when max_iter is reached, -1 on bad input, -2 on a
 * breakdown (a vanishing inner product).  ghost_out (nullable) receives the
 * boundary potentials. */
int ora_poisson_solve(const ora_poisson *p, const double *rho, double *phi, double *ghost_out, int *iters,
                      double *resid) {
  pgrid g;
  if (pgrid_init(&g, p) != 0) { pgrid_free(&g); return -1; }
  const long n = g.nc;
  for (long q = 0; q < n; ++q)
    if (p->criterion == ORA_POISSON_RELATIVE && !(rho[q] > 0.0)) { pgrid_free(&g); return -1; }
  double *buf = (double *)malloc(11 * (size_t)n * sizeof(double));
  double *ghost = (double *)malloc((size_t)ora_poisson_nghost(g.n) * sizeof(double));
  double *b = buf, *r = buf + n, *rh = buf + 2 * n, *pv = buf + 3 * n, *v = buf + 4 * n, *s = buf + 5 * n,
         *t = buf + 6 * n, *ph = buf + 7 * n, *sh = buf + 8 * n, *dinv = buf + 9 * n, *w = buf + 10 * n;
  ora_poisson_boundary(p, rho, ghost);
  /* right-hand side: 4 pi G rho minus the ghost terms of the boundary cells */
  double *zero = (double *)calloc((size_t)n, sizeof(double));
  apply(&g, zero, ghost, b);   /* = the ghost terms alone */
  free(zero);
  for (long q = 0; q < n; ++q) b[q] = 4.0 * PI * p->G * rho[q] - b[q];
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const long q = cid(&g, i, j, k);
        dinv[q] = 1.0 / (g.L2[0][i] + g.L2[1][j] + g.L2[2][k]);
        w[q] = p->criterion == ORA_POISSON_RELATIVE ? 1.0 / (4.0 * PI * p->G * rho[q]) : 1.0;
      }
  /* BiCGSTAB */
  apply(&g, phi, NULL, r);
  for (long q = 0; q < n; ++q) {
    r[q] = b[q] - r[q];
    rh[q] = r[q];
    pv[q] = 0.0;
    v[q] = 0.0;
  }
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0, status = 1;
  double res = rms(n, w, r);
  if (res < p->tol) status = 0;
  while (status == 1 && it < p->max_iter) {
    ++it;
    const double rho_i = dot(n, rh, r);
    if (rho_i == 0.0) { status = -2; break; }
    if (it == 1) {
      for (long q = 0; q < n; ++q) pv[q] = r[q];
    } else {
      const double beta = (rho_i / rho_old) * (alpha / omega);
      for (long q = 0; q < n; ++q) pv[q] = r[q] + beta * (pv[q] - omega * v[q]);
    }
    for (long q = 0; q < n; ++q) ph[q] = dinv[q] * pv[q];
    apply(&g, ph, NULL, v);
    const double rv = dot(n, rh, v);
    if (rv == 0.0) { status = -2; break; }
    alpha = rho_i / rv;
    for (long q = 0; q < n; ++q) s[q] = r[q] - alpha * v[q];
    res = rms(n, w, s);
    if (res < p->tol) {
      for (long q = 0; q < n; ++q) {
        phi[q] += alpha * ph[q];
        r[q] = s[q];
      }
      status = 0;
      break;
    }
    for (long q = 0; q < n; ++q) sh[q] = dinv[q] * s[q];
    apply(&g, sh, NULL, t);
    const double tt = dot(n, t, t);
    if (tt == 0.0) { status = -2; break; }
    omega = dot(n, t, s) / tt;
    for (long q = 0; q < n; ++q) {
      phi[q] += alpha * ph[q] + omega * sh[q];
      r[q] = s[q] - omega * t[q];
    }
    rho_old = rho_i;
    res = rms(n, w, r);
    if (res < p->tol) { status = 0; break; }
    if (omega == 0.0) { status = -2; break; }
  }
  if (iters) *iters = it;
  if (resid) *resid = res;
  if (ghost_out) memcpy(ghost_out, ghost, (size_t)ora_poisson_nghost(g.n) * sizeof(double));
  free(ghost);
  free(buf);
  pgrid_free(&g);
  return status;
}
