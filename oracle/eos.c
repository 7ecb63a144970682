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
 * f(ln n, ln T) = n eta kT - P, and the table is interpolated biquintically in
 * (x, y) = (ln n, ln T) as the paper does with its Helmholtz table (Sect. 2.2):
 * each node holds f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy and f_xxyy (the
 * derivatives from the integrals above by truncated Taylor arithmetic), and
 * the interpolant is the tensor product of quintic Hermite polynomials, which
 * matches f and its derivatives up to second order in each variable at the
 * nodes (Timmes & Swesty 2000).  P, e, c_v and dP/drho, dP/dT all follow from
 * that one interpolant, so the thermodynamic identities hold to round-off,
 * and the second-derivative quantities (c_v, gamma_c) are continuous.
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

/* e-/e+ gas at (nnet, T) by direct quadrature: P, E (per volume, pair rest
 * mass included), s (per volume), eta, n+, and the free-energy density with
 * its first derivatives f, f_x = n eta k T, f_y = -T s and
 * f_xy = n k T (eta + d eta / d ln T) (x = ln n, y = ln T), each from its own
 * combination of the integrals (checks of the Taylor-mode derivatives below). */
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
  if (fv) {
    fv[0] = f;
    fv[1] = nnet * eta * kT;
    fv[2] = -T * s;
    fv[3] = nnet * kT * (eta + deta_dlnT);
  }
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

int ora_ep_first(double nnet, double T, double *fv) {
  return ep_node(nnet, T, fv, NULL, NULL, NULL, NULL, NULL);
}

/* ---------------- derivatives of the free energy up to f_xxyy ----------------
 * The biquintic Hermite table needs, at each node (x, y) = (ln n, ln T), the
 * derivatives f_{x^i y^j}, i, j <= 2, of f = n eta k T - P.  They are taken
 * exactly (to rounding) in truncated Taylor arithmetic: every quantity is a
 * polynomial in the offsets (dx, dy) from the node, keeping the coefficients
 * of dx^i dy^j with i, j <= 2, so that
 *   f(x + dx, y + dy) = sum c[i][j] dx^i dy^j,  f_{x^i y^j} = i! j! c[i][j].
 * The integrals are written in the kinetic energy xi = b x (units of m_e c^2)
 * and psi = eta b, the Fermi kinetic energy:
 *   n = K_n [G_1/2 + G_3/2],  P = K_p [G_3/2 + G_5/2 / 2],
 *   G_k(psi, b) = int xi^k sqrt(1 + xi/2) f((xi - psi) / b) dxi,
 * f(u) = 1/(e^u + 1), positrons at psi+ = -psi - 2.  In these variables a
 * degenerate gas keeps psi nearly fixed as T changes, and the temperature
 * enters only through the width b of the Fermi edge: the Taylor coefficients
 * carry no large cancelling terms (in (eta, b) they would, since d eta/d ln T
 * ~ -eta there).  With w = 1/b, u0 = (xi - psi0) w0 and r = w / w0 - 1,
 *   u - u0 = u0 r - w0 (1 + r) dpsi,
 * and the Fermi factor's Taylor series needs the scalar moments
 *   M[k][p][i] = int xi^k sqrt(1 + xi/2) u0^i f^(p)(u0) / p! dxi,
 * computed once per node by quadrature; the offset dpsi is found from charge
 * neutrality N(psi) = e^x by Newton's method in this arithmetic with the
 * node's dN/dpsi (each iteration makes one more order exact; four exist). */
typedef struct { double c[3][3]; } jet;   /* c[i][j]: coefficient of dx^i dy^j */

static jet j_const(double a) { jet r; memset(&r, 0, sizeof r); r.c[0][0] = a; return r; }
static jet j_add(jet a, jet b) {
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) a.c[i][j] += b.c[i][j];
  return a;
}
static jet j_scale(jet a, double s) {
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) a.c[i][j] *= s;
  return a;
}
static jet j_mul(jet a, jet b) {
  jet r = j_const(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int i1 = 0; i1 <= i; ++i1)
        for (int j1 = 0; j1 <= j; ++j1) r.c[i][j] += a.c[i1][j1] * b.c[i - i1][j - j1];
  return r;
}
/* c0 exp(s dx) and c0 exp(s dy) */
static jet j_expx(double c0, double s) {
  jet r = j_const(0.0);
  double t = c0;
  for (int i = 0; i < 3; ++i) { r.c[i][0] = t; t *= s / (i + 1); }
  return r;
}
static jet j_expy(double c0, double s) {
  jet r = j_const(0.0);
  double t = c0;
  for (int j = 0; j < 3; ++j) { r.c[0][j] = t; t *= s / (j + 1); }
  return r;
}

/* M[k][p][i] (k = 1/2, 3/2, 5/2 as 0..2; p = 0..4; i = 0..2) of one species
 * with degeneracy parameter eta at b, on the panels of fd_set (in x = xi / b).
 * Derivatives of the Fermi function in terms of f, g = f (1 - f) and
 * t = 1 - 2 f:  f' = -g, f'' = g t, f''' = 2 g^2 - g t^2,
 * f'''' = g t^3 - 8 g^2 t. */
static void fd_moments(double eta, double b, double M[3][5][3]) {
  gl_init();
  memset(M, 0, sizeof(double) * 45);
  static const double off[12] = {-48.0, -24.0, -12.0, -6.0, -3.0, 0.0, 3.0, 6.0, 12.0, 24.0, 48.0, 100.0};
  static const double ifact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};
  const double base = eta > 0.0 ? eta : 0.0;
  double e[13];
  int ne = 0;
  e[ne++] = 0.0;
  for (int q = 0; q < 12; ++q) {
    double x = base + off[q];
    if (x > 0.0) e[ne++] = sqrt(x);
  }
  for (int pnl = 0; pnl + 1 < ne; ++pnl) {
    double a = e[pnl], c = e[pnl + 1];
    if (c - a <= 0.0) continue;
    for (int sub = 0; sub < 2; ++sub) {
      double lo = a + (c - a) * sub / 2, hi = a + (c - a) * (sub + 1) / 2;
      double hm = 0.5 * (hi - lo), cm = 0.5 * (hi + lo);
      for (int gq = 0; gq < 24; ++gq) {
        double tt = cm + hm * gl_x[gq], wt = hm * gl_w[gq];
        double x = tt * tt, u = x - eta;
        double z = exp(-fabs(u));
        double f = u > 0.0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
        double g = z / ((1.0 + z) * (1.0 + z));
        double t = u > 0.0 ? (1.0 - z) / (1.0 + z) : (z - 1.0) / (1.0 + z);
        double fk[5] = {f, -g, g * t, 2.0 * g * g - g * t * t, g * t * t * t - 8.0 * g * g * t};
        double xi = b * x, sxi = sqrt(xi);
        double S = sqrt(1.0 + 0.5 * xi);
        double jac = b * 2.0 * tt * wt;                     /* dxi = b dx = b 2 t dt */
        double phi[3] = {sxi * S, xi * sxi * S, xi * xi * sxi * S};
        double ui[3] = {1.0, u, u * u};
        for (int k = 0; k < 3; ++k)
          for (int p = 0; p < 5; ++p)
            for (int i = 0; i < 3; ++i) M[k][p][i] += jac * phi[k] * ui[i] * fk[p] * ifact[p];
      }
    }
  }
}

/* G_k (k = 1/2, 3/2, 5/2) of one species as Taylor polynomials, given the
 * offset dpsi of its psi, r = w / w0 - 1 and w0:
 *   G = sum_{p, j} C(p, j) M[k][p][p - j] r^(p - j) (-w0 (1 + r) dpsi)^j
 * (r has no constant term and at most dy^2: r^3 = 0, so p - j <= 2). */
static void g_jets(double M[3][5][3], jet dpsi, jet r, double w0, jet *G) {
  static const double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  jet rp[3], qp[5];
  rp[0] = j_const(1.0);
  for (int i = 1; i < 3; ++i) rp[i] = j_mul(rp[i - 1], r);
  const jet q = j_scale(j_mul(j_add(j_const(1.0), r), dpsi), -w0);
  qp[0] = j_const(1.0);
  for (int j = 1; j < 5; ++j) qp[j] = j_mul(qp[j - 1], q);
  for (int k = 0; k < 3; ++k) {
    G[k] = j_const(0.0);
    for (int p = 0; p < 5; ++p)
      for (int j = p >= 2 ? p - 2 : 0; j <= p; ++j)
        G[k] = j_add(G[k], j_scale(j_mul(rp[p - j], qp[j]), binom[p][j] * M[k][p][p - j]));
  }
}

/* f and its derivatives at (nnet, T): out = f, f_x, f_y, f_xx, f_yy, f_xy,
 * f_xxy, f_xyy, f_xxyy.  Returns 0 or -1 (no neutrality root). */
int ora_ep_derivs(double nnet, double T, double *out) {
  const double b0 = K_B * T / ME_C2, w0 = 1.0 / b0;
  double eta0;
  if (solve_eta(nnet, b0, &eta0)) return -1;
  const double lam = lambda3();
  const double Kn = 8.0 * PI * sqrt(2.0) * lam;
  const double Kp = 16.0 * PI * sqrt(2.0) / 3.0 * lam * ME_C2;
  const double psi0 = eta0 * b0;
  double Mm[3][5][3], Mp[3][5][3];
  fd_moments(eta0, b0, Mm);
  fd_moments(-eta0 - 2.0 / b0, b0, Mp);                         /* positrons: psi+ = -psi - 2 */
  const jet r = j_add(j_expy(1.0, -1.0), j_const(-1.0));        /* w / w0 - 1 = e^-dy - 1 */
  const jet n = j_expx(nnet, 1.0);                              /* n = nnet e^dx */
  /* dN/dpsi at the node: d/dpsi f((xi - psi) w) = -w f'; the positron psi
   * moves against the electron one */
  const double Npsi = -Kn * w0 * ((Mm[0][1][0] + Mm[1][1][0]) + (Mp[0][1][0] + Mp[1][1][0]));
  jet dpsi = j_const(0.0), Gm[3], Gp[3];
  for (int it = 0; it < 7; ++it) {
    g_jets(Mm, dpsi, r, w0, Gm);
    g_jets(Mp, j_scale(dpsi, -1.0), r, w0, Gp);
    jet R = j_add(j_scale(j_add(j_add(Gm[0], Gm[1]), j_scale(j_add(Gp[0], Gp[1]), -1.0)), Kn), j_scale(n, -1.0));
    R.c[0][0] = 0.0;   /* psi0 is the root at the node itself */
    dpsi = j_add(dpsi, j_scale(R, -1.0 / Npsi));
  }
  g_jets(Mm, dpsi, r, w0, Gm);
  g_jets(Mp, j_scale(dpsi, -1.0), r, w0, Gp);
  jet P = j_add(j_add(Gm[1], j_scale(Gm[2], 0.5)), j_add(Gp[1], j_scale(Gp[2], 0.5)));
  P = j_scale(P, Kp);
  /* f = n eta k T - P = n m_e c^2 psi - P */
  const jet f = j_add(j_scale(j_mul(n, j_add(dpsi, j_const(psi0))), ME_C2), j_scale(P, -1.0));
  out[0] = f.c[0][0];
  out[1] = f.c[1][0];
  out[2] = f.c[0][1];
  out[3] = 2.0 * f.c[2][0];
  out[4] = 2.0 * f.c[0][2];
  out[5] = f.c[1][1];
  out[6] = 2.0 * f.c[2][1];
  out[7] = 2.0 * f.c[1][2];
  out[8] = 4.0 * f.c[2][2];
  return 0;
}

/* ---------------- table and biquintic Hermite interpolation ---------------- */
#define NQ 9   /* values per node: f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy */
struct ora_eos_table {
  int nx, ny;
  double x0, dx, y0, dy;     /* x = ln(n_net), y = ln T */
  double *v;                 /* [ny][nx][NQ] */
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
  t->v = calloc((size_t)nrho * nT * NQ, sizeof(double));
  for (int j = 0; j < nT; ++j)
    for (int i = 0; i < nrho; ++i) {
      double n = exp(t->x0 + i * t->dx), T = exp(t->y0 + j * t->dy);
      if (ora_ep_derivs(n, T, &t->v[((size_t)j * nrho + i) * NQ])) {
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

long ora_eos_table_size(const ora_eos_table *t) { return 6 + (long)t->nx * t->ny * NQ; }

int ora_eos_table_export(const ora_eos_table *t, double *out, long nout) {
  if (nout < ora_eos_table_size(t)) return -1;
  out[0] = t->nx; out[1] = t->ny; out[2] = t->x0; out[3] = t->dx; out[4] = t->y0; out[5] = t->dy;
  memcpy(out + 6, t->v, sizeof(double) * t->nx * t->ny * NQ);
  return 0;
}

/* Quintic Hermite basis on [0, 1]: h[a][q] is the polynomial whose q-th
 * derivative is 1 at end a (0 or 1) while its value and first two
 * derivatives vanish otherwise at both ends; d1, d2 are its derivatives.  At
 * end 1 the functions are (-1)^q times those of end 0 evaluated at 1 - u. */
static void quintic(double u, double h[2][3], double d1[2][3], double d2[2][3]) {
  for (int a = 0; a < 2; ++a) {
    const double w = a == 0 ? u : 1.0 - u, sg = a == 0 ? 1.0 : -1.0;
    const double w2 = w * w, w3 = w2 * w, w4 = w3 * w, w5 = w4 * w;
    const double p[3] = {1.0 - 10.0 * w3 + 15.0 * w4 - 6.0 * w5, w - 6.0 * w3 + 8.0 * w4 - 3.0 * w5,
                         0.5 * (w2 - 3.0 * w3 + 3.0 * w4 - w5)};
    const double p1[3] = {-30.0 * w2 + 60.0 * w3 - 30.0 * w4, 1.0 - 18.0 * w2 + 32.0 * w3 - 15.0 * w4,
                          0.5 * (2.0 * w - 9.0 * w2 + 12.0 * w3 - 5.0 * w4)};
    const double p2[3] = {-60.0 * w + 180.0 * w2 - 120.0 * w3, -36.0 * w + 96.0 * w2 - 60.0 * w3,
                          0.5 * (2.0 - 18.0 * w + 36.0 * w2 - 20.0 * w3)};
    for (int q = 0; q < 3; ++q) {
      const double s = (a == 1 && (q & 1)) ? -1.0 : 1.0;
      h[a][q] = s * p[q];
      d1[a][q] = s * sg * p1[q];   /* d/du = sg d/dw */
      d2[a][q] = s * p2[q];
    }
  }
}

/* The 2 x 2 corner values c[a][b] of a quantity enter the tensor product as
 * sum c[a][b] X_a Y_b.  Written in differences across the interval,
 *   sum c[a][b] X_a Y_b = sum D[a][b] X~_a Y~_b,  D[0][0] = c00,
 *   D[1][0] = c10 - c00, D[0][1] = c01 - c00, D[1][1] = (c11 - c10) - (c01 - c00),
 *   X~_0 = X_0 + X_1, X~_1 = X_1 (the same in y),
 * an identity; for the value functions (q = 0) X~_0 is exactly 1 for the
 * value and 0 for the derivatives (the value functions sum to one).  This
 * form avoids the cancellation of two large node values in a derivative
 * (f_y from f alone would otherwise lose ~|f| / dy to rounding). */
static void to_difference_basis(double b[2][3], int deriv) {
  for (int q = 0; q < 3; ++q) b[0][q] = (q == 0) ? (deriv == 0 ? 1.0 : 0.0) : b[0][q] + b[1][q];
}

/* f and its x/y derivatives up to second order at (x, y); -1 outside.  The
 * node derivative of order (p, q) enters with the factor dx^p dy^q. */
static int table_eval(const ora_eos_table *t, double x, double y, double *o /* f,fx,fy,fxx,fyy,fxy */) {
  double gx = (x - t->x0) / t->dx, gy = (y - t->y0) / t->dy;
  if (!(gx >= 0.0 && gx <= t->nx - 1 && gy >= 0.0 && gy <= t->ny - 1)) return -1;
  int i = (int)gx, j = (int)gy;
  if (i > t->nx - 2) i = t->nx - 2;
  if (j > t->ny - 2) j = t->ny - 2;
  double u = gx - i, v = gy - j;
  double hu[2][3], du[2][3], eu[2][3], hv[2][3], dv[2][3], ev[2][3];
  quintic(u, hu, du, eu);
  quintic(v, hv, dv, ev);
  to_difference_basis(hu, 0); to_difference_basis(du, 1); to_difference_basis(eu, 2);
  to_difference_basis(hv, 0); to_difference_basis(dv, 1); to_difference_basis(ev, 2);
  static const int slot[3][3] = {{0, 2, 4}, {1, 5, 7}, {3, 6, 8}};   /* node slot of d^(p+q)f / dx^p dy^q */
  double hx = t->dx, hy = t->dy;
  double hxp[3] = {1.0, hx, hx * hx}, hyp[3] = {1.0, hy, hy * hy};
  const double *c00 = &t->v[((size_t)j * t->nx + i) * NQ], *c10 = c00 + NQ;
  const double *c01 = &t->v[((size_t)(j + 1) * t->nx + i) * NQ], *c11 = c01 + NQ;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < 3; ++p)
    for (int r = 0; r < 3; ++r) {
      const int k = slot[p][r];
      double D[2][2];
      D[0][0] = c00[k];
      D[1][0] = c10[k] - c00[k];
      D[0][1] = c01[k] - c00[k];
      D[1][1] = (c11[k] - c10[k]) - (c01[k] - c00[k]);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          double c = D[a][b] * hxp[p] * hyp[r];
          acc[0] += c * hu[a][p] * hv[b][r];
          acc[1] += c * du[a][p] * hv[b][r];
          acc[2] += c * hu[a][p] * dv[b][r];
          acc[3] += c * eu[a][p] * hv[b][r];
          acc[4] += c * hu[a][p] * ev[b][r];
          acc[5] += c * du[a][p] * dv[b][r];
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
    /* direct quadrature: the same relations on the exact derivatives at the point */
    double d9[NQ];
    if (ora_ep_derivs(rho * ye * N_AVO, T, d9)) return -3;
    Pe = d9[1] - d9[0];
    ee = (d9[0] - d9[2]) / rho;
    cve = (d9[2] - d9[4]) / (rho * T);
    Pe_T = (d9[5] - d9[2]) / T;
    Pe_r = (d9[3] - d9[1]) / rho;
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
