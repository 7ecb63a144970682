/*
 * eos.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).  Stellar EOS of the oracle.
 *
 * Fully ionised ions (ideal gas), radiation in LTE (Eqs. prad, erad) and an
 * electron-positron gas of arbitrary degeneracy and relativity in pair
 * equilibrium (Sect. 2.2, item ii), written from the textbook phase-space
 * integrals:
 *   n   = K_n b^(3/2) [F_1/2 + b F_3/2],      (b = kT / m_e c^2)
 *   P   = K_p b^(5/2) [F_3/2 + b/2 F_5/2],
 *   E_k = K_e b^(5/2) [F_3/2 + b F_5/2],
 *   F_k(eta, b) = int_0^inf x^k sqrt(1 + b x / 2) / (exp(x - eta) + 1) dx,
 * positrons with eta+ = -eta - 2/b, charge neutrality n- - n+ = rho Y_e N_A,
 * pair rest mass 2 m_e c^2 n+ counted in the energy.
 *
 * The e-/e+ part is tabulated as its Helmholtz free-energy density
 * f(ln n, ln T) = n eta kT - P together with f_x = n eta k T, f_y = -T s and
 * f_xy (x = ln n, y = ln T), and interpolated with bicubic Hermite
 * polynomials; P, e, c_v and dP/drho, dP/dT all follow from that one
 * interpolant, so the thermodynamic identities hold to round-off (the paper's
 * Helmholtz table interpolates the free energy biquintically, Sect. 2.2; this
 * table is computed here from the integrals above).
 *
 * Temperature from e_int: Newton T <- T + (e - e_EoS) / c_v until
 * |de|/e < tol (Sect. 2.2), then one more Newton step; steps are kept inside
 * the table by bisection with a bracket.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define PI 3.14159265358979323846
/* CODATA 2018, CGS */
#define K_B 1.380649e-16
#define ME_C2 8.1871057769e-7          /* m_e c^2, erg */
#define H_PLANCK 6.62607015e-27
#define C_LIGHT 2.99792458e10
#define N_AVO 6.02214076e23
#define A_RAD 7.565733250e-15          /* 4 sigma / c */
#define R_GAS (K_B * N_AVO)

static double lambda3(void) {          /* (m_e c / h)^3 */
  double me = ME_C2 / (C_LIGHT * C_LIGHT);
  double l = me * C_LIGHT / H_PLANCK;
  return l * l * l;
}

/* ---------------- generalised Fermi-Dirac integrals ---------------- */
/* 24-point Gauss-Legendre nodes/weights on [-1, 1] (computed once). */
static double gl_x[24], gl_w[24];
static int gl_ready = 0;
static void gl_init(void) {
  if (gl_ready) return;
  const int n = 24;
  for (int i = 0; i < n; ++i) {
    double x = cos(PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

/* Integrals of one species at (eta, b), by x = t^2 and composite
 * Gauss-Legendre panels.  The panel edges sit at fixed distances (in units
 * of kT) from the Fermi edge x = max(eta, 0), so the Fermi function varies by
 * at most a factor e^3 ... e^24 across a panel and is below e^-48 where the
 * first panel ends: the quadrature error stays at rounding level for every
 * degeneracy (a panel ending only a few kT before the edge leaves the
 * exponential tail unresolved, an O(e^-8) relative error at strong
 * degeneracy).
 *   out[0..2] = F_1/2, F_3/2, F_5/2
 *   out[3..4] = dF_1/2/deta, dF_3/2/deta
 *   out[5..6] = dF_1/2/db,   dF_3/2/db */
static void fd_set(double eta, double b, double *out) {
  gl_init();
  for (int q = 0; q < 7; ++q) out[q] = 0.0;
  static const double off[12] = {-48.0, -24.0, -12.0, -6.0, -3.0, 0.0, 3.0, 6.0, 12.0, 24.0, 48.0, 100.0};
  const double base = eta > 0.0 ? eta : 0.0;
  double e[13];
  int ne = 0;
  e[ne++] = 0.0;
  for (int q = 0; q < 12; ++q) {
    double x = base + off[q];
    if (x > 0.0) e[ne++] = sqrt(x);   /* t-space edge */
  }
  for (int pnl = 0; pnl + 1 < ne; ++pnl) {
    double a = e[pnl], c = e[pnl + 1];
    if (c - a <= 0.0) continue;
    int nsub = 2;
    for (int s = 0; s < nsub; ++s) {
      double lo = a + (c - a) * s / nsub, hi = a + (c - a) * (s + 1) / nsub;
      double hm = 0.5 * (hi - lo), cm = 0.5 * (hi + lo);
      for (int g = 0; g < 24; ++g) {
        double t = cm + hm * gl_x[g], wt = hm * gl_w[g];
        double x = t * t, u = x - eta;
        double f, ff;   /* Fermi function and f (1 - f) */
        if (u > 0.0) { double z = exp(-u); f = z / (1.0 + z); ff = z / ((1.0 + z) * (1.0 + z)); }
        else { double z = exp(u); f = 1.0 / (1.0 + z); ff = z / ((1.0 + z) * (1.0 + z)); }
        double S = sqrt(1.0 + 0.5 * b * x);
        double jac = 2.0 * t * wt;         /* dx = 2 t dt */
        double x12 = t;                    /* x^(1/2) */
        double x32 = x * t, x52 = x * x * t;
        out[0] += jac * x12 * S * f;
        out[1] += jac * x32 * S * f;
        out[2] += jac * x52 * S * f;
        out[3] += jac * x12 * S * ff;
        out[4] += jac * x32 * S * ff;
        out[5] += jac * x32 * 0.25 / S * f;   /* d/db sqrt(1 + b x/2) = x / (4 S) */
        out[6] += jac * x52 * 0.25 / S * f;
      }
    }
  }
}

double ora_fd(double k, double eta, double beta) {
  double o[7];
  fd_set(eta, beta, o);
  if (k == 0.5) return o[0];
  if (k == 1.5) return o[1];
  if (k == 2.5) return o[2];
  return NAN;
}

/* number density of one species and its eta / b derivatives */
static void species_n(double eta, double b, double *n, double *n_eta, double *n_b, double *o) {
  double Kn = 8.0 * PI * sqrt(2.0) * lambda3();
  fd_set(eta, b, o);
  double b12 = sqrt(b), b32 = b * b12;
  *n = Kn * b32 * (o[0] + b * o[1]);
  *n_eta = Kn * b32 * (o[3] + b * o[4]);
  *n_b = Kn * (1.5 * b12 * (o[0] + b * o[1]) + b32 * (o[5] + o[1] + b * o[6]));
}

/* Solve charge neutrality for eta at net electron density nnet and b. */
static int solve_eta(double nnet, double b, double *eta_out) {
  double lo = -700.0, hi = 1e7, eta;
  /* starting guess: nondegenerate or degenerate limit */
  double Kn = 8.0 * PI * sqrt(2.0) * lambda3();
  double nd = Kn * pow(b, 1.5) * 0.886226925452758;   /* K_n b^1.5 sqrt(pi)/2 */
  double xf = pow(3.0 * nnet / (8.0 * PI * lambda3()), 1.0 / 3.0);
  double eta_deg = (sqrt(1.0 + xf * xf) - 1.0) / b;
  eta = log(nnet / nd);
  if (eta_deg > eta) eta = eta_deg;
  if (eta < lo) eta = lo + 1.0;
  double o[7];
  for (int it = 0; it < 200; ++it) {
    double nm, nm_e, nm_b, np, np_e, np_b;
    species_n(eta, b, &nm, &nm_e, &nm_b, o);
    species_n(-eta - 2.0 / b, b, &np, &np_e, &np_b, o);
    double r = nm - np - nnet;
    double dr = nm_e + np_e;
    if (r > 0.0) hi = eta; else lo = eta;
    double step = r / dr;
    double en = eta - step;
    if (!(en > lo && en < hi)) en = 0.5 * (lo + hi);
    if (fabs(en - eta) <= 1e-15 * (fabs(eta) + 1.0) || hi - lo < 1e-14 * (fabs(eta) + 1.0)) { eta = en; *eta_out = eta; return 0; }
    eta = en;
  }
  *eta_out = eta;
  return -1;
}

/* e-/e+ free energy density and derivatives at (nnet, T):
 * f, fx = n eta k T, fy = -T s, fxy (x = ln n, y = ln T); also P, e (vol). */
static int ep_node(double nnet, double T, double *fv, double *P, double *evol, double *s_out,
                   double *eta_out, double *npos) {
  double b = K_B * T / ME_C2, eta;
  if (solve_eta(nnet, b, &eta)) return -1;
  double lam = lambda3();
  double Kp = 16.0 * PI * sqrt(2.0) / 3.0 * lam * ME_C2;
  double Ke = 8.0 * PI * sqrt(2.0) * lam * ME_C2;
  double om[7], op[7], nm, nm_e, nm_b, np, np_e, np_b;
  double etap = -eta - 2.0 / b;
  species_n(eta, b, &nm, &nm_e, &nm_b, om);
  species_n(etap, b, &np, &np_e, &np_b, op);
  double b52 = b * b * sqrt(b);
  double Pm = Kp * b52 * (om[1] + 0.5 * b * om[2]), Pp = Kp * b52 * (op[1] + 0.5 * b * op[2]);
  double Em = Ke * b52 * (om[1] + b * om[2]), Ep = Ke * b52 * (op[1] + b * op[2]);
  double kT = K_B * T;
  double s = (Em + Pm - eta * kT * nm) / T + (Ep + Pp - etap * kT * np) / T;
  double Ptot = Pm + Pp;
  double E = Em + Ep + 2.0 * ME_C2 * np;
  double f = nnet * eta * kT - Ptot;
  /* d eta / db at fixed nnet: n = n-(eta) - n+(-eta - 2/b) */
  double dn_deta = nm_e + np_e;
  double dn_db = nm_b - (np_b + np_e * 2.0 / (b * b));
  double deta_db = -dn_db / dn_deta;
  double deta_dlnT = deta_db * b;
  fv[0] = f;
  fv[1] = nnet * eta * kT;
  fv[2] = -T * s;
  fv[3] = nnet * kT * (eta + deta_dlnT);
  if (P) *P = Ptot;
  if (evol) *evol = E;
  if (s_out) *s_out = s;
  if (eta_out) *eta_out = eta;
  if (npos) *npos = np;
  return 0;
}

int ora_ep_direct(double rho, double ye, double T, double *P, double *e, double *s, double *eta,
                  double *npos) {
  double fv[4], evol, sv;
  double nnet = rho * ye * N_AVO;
  if (ep_node(nnet, T, fv, P, &evol, &sv, eta, npos)) return -1;
  if (e) *e = evol / rho;
  if (s) *s = sv / rho;
  return 0;
}

/* ---------------- table and bicubic Hermite interpolation ---------------- */
struct ora_eos_table {
  int nx, ny;
  double x0, dx, y0, dy;     /* x = ln(n_net), y = ln T */
  double *v;                 /* [ny][nx][4]: f, fx, fy, fxy */
};

ora_eos_table *ora_eos_table_build(double lrho_lo, double lrho_hi, int nrho,
                                   double lT_lo, double lT_hi, int nT) {
  /* lrho_*: log10(rho Y_e); lT_*: log10 T */
  ora_eos_table *t = calloc(1, sizeof(*t));
  t->nx = nrho; t->ny = nT;
  t->x0 = log(pow(10.0, lrho_lo) * N_AVO);
  t->dx = (lrho_hi - lrho_lo) * log(10.0) / (nrho - 1);
  t->y0 = lT_lo * log(10.0);
  t->dy = (lT_hi - lT_lo) * log(10.0) / (nT - 1);
  t->v = calloc((size_t)nrho * nT * 4, sizeof(double));
  for (int j = 0; j < nT; ++j)
    for (int i = 0; i < nrho; ++i) {
      double n = exp(t->x0 + i * t->dx), T = exp(t->y0 + j * t->dy);
      if (ep_node(n, T, &t->v[((size_t)j * nrho + i) * 4], NULL, NULL, NULL, NULL, NULL)) {
        ora_eos_table_free(t);
        return NULL;
      }
    }
  return t;
}

void ora_eos_table_free(ora_eos_table *t) {
  if (!t) return;
  free(t->v);
  free(t);
}

long ora_eos_table_size(const ora_eos_table *t) { return 6 + (long)t->nx * t->ny * 4; }

int ora_eos_table_export(const ora_eos_table *t, double *out, long nout) {
  if (nout < ora_eos_table_size(t)) return -1;
  out[0] = t->nx; out[1] = t->ny; out[2] = t->x0; out[3] = t->dx; out[4] = t->y0; out[5] = t->dy;
  memcpy(out + 6, t->v, sizeof(double) * t->nx * t->ny * 4);
  return 0;
}

/* cubic Hermite basis on [0,1] and its first two derivatives */
static void hermite(double u, double *h, double *d1, double *d2) {
  double u2 = u * u, u3 = u2 * u;
  h[0] = 2 * u3 - 3 * u2 + 1; h[1] = u3 - 2 * u2 + u; h[2] = -2 * u3 + 3 * u2; h[3] = u3 - u2;
  d1[0] = 6 * u2 - 6 * u; d1[1] = 3 * u2 - 4 * u + 1; d1[2] = -6 * u2 + 6 * u; d1[3] = 3 * u2 - 2 * u;
  d2[0] = 12 * u - 6; d2[1] = 6 * u - 4; d2[2] = -12 * u + 6; d2[3] = 6 * u - 2;
}

/* f and its x/y derivatives up to second order at (x, y); -1 outside. */
static int table_eval(const ora_eos_table *t, double x, double y, double *o /* f,fx,fy,fxx,fyy,fxy */) {
  double gx = (x - t->x0) / t->dx, gy = (y - t->y0) / t->dy;
  if (!(gx >= 0.0 && gx <= t->nx - 1 && gy >= 0.0 && gy <= t->ny - 1)) return -1;
  int i = (int)gx, j = (int)gy;
  if (i > t->nx - 2) i = t->nx - 2;
  if (j > t->ny - 2) j = t->ny - 2;
  double u = gx - i, v = gy - j;
  double hu[4], du[4], ddu[4], hv[4], dv[4], ddv[4];
  hermite(u, hu, du, ddu);
  hermite(v, hv, dv, ddv);
  /* corner values, ordered (i,j), (i+1,j), (i,j+1), (i+1,j+1) */
  const double *c[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) c[a][b] = &t->v[((size_t)(j + b) * t->nx + (i + a)) * 4];
  double hx = t->dx, hy = t->dy;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      /* basis index: value 2a, slope 2a+1 (position a) */
      int iv = 2 * a, is = 2 * a + 1, jv = 2 * b, js = 2 * b + 1;
      const double *q = c[a][b];
      double coef[4] = {q[0], q[1] * hx, q[2] * hy, q[3] * hx * hy};
      int ii[4] = {iv, is, iv, is}, jj[4] = {jv, jv, js, js};
      for (int m = 0; m < 4; ++m) {
        acc[0] += coef[m] * hu[ii[m]] * hv[jj[m]];
        acc[1] += coef[m] * du[ii[m]] * hv[jj[m]];
        acc[2] += coef[m] * hu[ii[m]] * dv[jj[m]];
        acc[3] += coef[m] * ddu[ii[m]] * hv[jj[m]];
        acc[4] += coef[m] * hu[ii[m]] * ddv[jj[m]];
        acc[5] += coef[m] * du[ii[m]] * dv[jj[m]];
      }
    }
  o[0] = acc[0];
  o[1] = acc[1] / hx;
  o[2] = acc[2] / hy;
  o[3] = acc[3] / (hx * hx);
  o[4] = acc[4] / (hy * hy);
  o[5] = acc[5] / (hx * hy);
  return 0;
}

static void composition(const ora_cfg *c, const double *X, double *abar, double *ye) {
  double sa = 0.0, sz = 0.0, sx = 0.0;
  for (int l = 0; l < c->nspec; ++l) { sx += X[l]; }
  for (int l = 0; l < c->nspec; ++l) {
    double x = X[l] / sx;
    sa += x / c->A[l];
    sz += c->Z[l] * x / c->A[l];
  }
  *abar = 1.0 / sa;
  *ye = sz;
}

int ora_eos_rt(const ora_cfg *cfg, double rho, double T, const double *X,
               double *P, double *e, double *cv, double *dPdr, double *dPdT,
               double *ge, double *gc) {
  double abar, ye;
  composition(cfg, X, &abar, &ye);
  double Pe, ee, cve, Pe_T, Pe_r;
  if (cfg->eos_table) {
    double o[6];
    double x = log(rho * ye * N_AVO), y = log(T);
    if (table_eval((const ora_eos_table *)cfg->eos_table, x, y, o)) return -3;
    Pe = o[1] - o[0];
    ee = (o[0] - o[2]) / rho;
    cve = (o[2] - o[4]) / (rho * T);
    Pe_T = (o[5] - o[2]) / T;
    Pe_r = (o[3] - o[1]) / rho;
  } else {
    /* direct quadrature: derivatives by the same relations from ep_node */
    double fv[4], evol;
    if (ep_node(rho * ye * N_AVO, T, fv, &Pe, &evol, NULL, NULL, NULL)) return -3;
    ee = evol / rho;
    /* c_v and dP/dT, dP/drho by centred differences in ln T, ln rho */
    double h = 1e-4, Pp, Pm, ep_, em_, fvp[4], fvm[4];
    ep_node(rho * ye * N_AVO, T * exp(h), fvp, &Pp, &ep_, NULL, NULL, NULL);
    ep_node(rho * ye * N_AVO, T * exp(-h), fvm, &Pm, &em_, NULL, NULL, NULL);
    cve = (ep_ - em_) / (rho * 2.0 * h * T);
    Pe_T = (Pp - Pm) / (2.0 * h * T);
    ep_node(rho * ye * N_AVO * exp(h), T, fvp, &Pp, NULL, NULL, NULL, NULL);
    ep_node(rho * ye * N_AVO * exp(-h), T, fvm, &Pm, NULL, NULL, NULL, NULL);
    Pe_r = (Pp - Pm) / (2.0 * h * rho);
  }
  double Pi = rho * R_GAS * T / abar, ei = 1.5 * R_GAS * T / abar;
  double Pr = A_RAD * T * T * T * T / 3.0, er = A_RAD * T * T * T * T / rho;
  double Pt = Pe + Pi + Pr, et = ee + ei + er;
  double cvt = cve + 1.5 * R_GAS / abar + 4.0 * A_RAD * T * T * T / rho;
  double PT = Pe_T + rho * R_GAS / abar + 4.0 / 3.0 * A_RAD * T * T * T;
  double Pr_ = Pe_r + R_GAS * T / abar;
  if (P) *P = Pt;
  if (e) *e = et;
  if (cv) *cv = cvt;
  if (dPdT) *dPdT = PT;
  if (dPdr) *dPdr = Pr_;
  /* auxiliary indices (Sect. 2.6): gamma_e = P/(rho e) + 1, gamma_c = rho c_s^2 / P,
   * c_s^2 = dP/drho|_T + T (dP/dT)^2 / (rho^2 c_v)  (adiabatic sound speed) */
  double cs2 = Pr_ + T * PT * PT / (rho * rho * cvt);
  if (ge) *ge = Pt / (rho * et) + 1.0;
  if (gc) *gc = rho * cs2 / Pt;
  return 0;
}

int ora_eos_invert(const ora_cfg *cfg, double rho, double eint, const double *X,
                   double *T_inout, double *P, double *ge, double *gc, int *iters) {
  const ora_eos_table *tb = (const ora_eos_table *)cfg->eos_table;
  double Tlo = 1e3, Thi = 1e12;
  if (tb) { Tlo = exp(tb->y0); Thi = exp(tb->y0 + (tb->ny - 1) * tb->dy); }
  double tol = cfg->newton_tol > 0.0 ? cfg->newton_tol : 1e-11;
  int maxit = cfg->newton_maxit > 0 ? cfg->newton_maxit : 50;
  double T = (T_inout && *T_inout > 0.0) ? *T_inout : sqrt(Tlo * Thi);
  if (T < Tlo) T = Tlo;
  if (T > Thi) T = Thi;
  double lo = Tlo, hi = Thi;
  int it, converged = 0;
  for (it = 1; it <= maxit; ++it) {
    double e, cv;
    if (ora_eos_rt(cfg, rho, T, X, NULL, &e, &cv, NULL, NULL, NULL, NULL)) return -3;
    double de = eint - e;
    if (fabs(de) / fabs(eint) < tol) {   /* converged: one more Newton step */
      T = T + de / cv;
      converged = 1;
      break;
    }
    if (de > 0.0) lo = T; else hi = T;
    double Tn = T + de / cv;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    T = Tn;
  }
  if (!converged) return -3;
  if (T_inout) *T_inout = T;
  if (iters) *iters = it;
  return ora_eos_rt(cfg, rho, T, X, P, NULL, NULL, NULL, NULL, ge, gc);
}
