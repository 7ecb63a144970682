/*
 * mhd.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain FP64 restatement of the explicit MHD stage of PHLEGETHON
 * (arXiv 2604.12672).  Loops follow the paper's order:
 *   boundary ghosts (Sect. 2.11, Table bcs) -> primitives + EOS (Sect. 2.2)
 *   -> deviations dW = W - W_hat (Sect. 2.8) -> shock flags (Sect. 2.7)
 *   -> van Leer PLM per direction (Sect. 2.5) -> LHLLD / HLL flux (Sect. 2.6)
 *   -> F - F_hat (Eq. wb1) -> Contact-CT edge EMFs (Sect. 2.4)
 *   -> residual with sources S - S_hat (Eqs. fv, spatres, wb2)
 *   -> SSP-RK stage (Sect. 2.9); CFL step (Eq. cfl).
 * No blocking, fusion or reordering beyond those definitions.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NG 3
enum { W_RHO = 0, W_VX, W_VY, W_VZ, W_BX, W_BY, W_BZ, W_P, W_GE, W_GC, W_X0 };
enum { U_RHO = 0, U_MX, U_MY, U_MZ, U_E, U_X0 };
/* flux components (global frame) */
enum { F_RHO = 0, F_MX, F_MY, F_MZ, F_E, F_BX, F_BY, F_BZ, F_X0 };

typedef struct {
  const ora_cfg *c;
  int n[3], act[3], g[3];
  long s[3], ntot;
  double dx[3];
  int nv, nw, nf;
} geo;

static void geo_init(geo *G, const ora_cfg *c) {
  G->c = c;
  for (int d = 0; d < 3; ++d) {
    G->n[d] = c->n[d];
    G->act[d] = c->n[d] > 1;
    G->g[d] = G->act[d] ? NG : 0;
    G->dx[d] = (c->hi[d] - c->lo[d]) / c->n[d];
  }
  G->s[0] = 1;
  G->s[1] = G->n[0] + 2 * G->g[0] + 1;
  G->s[2] = G->s[1] * (G->n[1] + 2 * G->g[1] + 1);
  G->ntot = G->s[2] * (G->n[2] + 2 * G->g[2] + 1);
  G->nv = 5 + c->nspec;
  G->nw = 10 + c->nspec;
  G->nf = 8 + c->nspec;
}

static inline long IX(const geo *G, int i, int j, int k) {
  return (long)(i + G->g[0]) + (long)(j + G->g[1]) * G->s[1] + (long)(k + G->g[2]) * G->s[2];
}
static inline long IXv(const geo *G, const int *c) { return IX(G, c[0], c[1], c[2]); }

/* ABI (unpadded) indices */
static inline long AC(const geo *G, int i, int j, int k) {
  return (long)i + (long)G->n[0] * (j + (long)G->n[1] * k);
}
static inline long AF(const geo *G, int d, int i, int j, int k) {
  long nx = G->n[0] + (d == 0), ny = G->n[1] + (d == 1);
  return (long)i + nx * (j + ny * (long)k);
}
static long abi_cells(const geo *G) { return (long)G->n[0] * G->n[1] * G->n[2]; }
static long abi_faces(const geo *G, int d) {
  return (long)(G->n[0] + (d == 0)) * (G->n[1] + (d == 1)) * (G->n[2] + (d == 2));
}

/* ---------------- background (Sect. 2.8) ---------------- */
typedef struct { double rho, p, ge, gc; } bgstate;

static bgstate bg_cell(const geo *G, int k) {
  const ora_cfg *c = G->c;
  bgstate b = {0, 0, 0, 0};
  if (!c->bg_rho_c) return b;
  b.rho = c->bg_rho_c[k + NG];
  b.p = c->bg_p_c[k + NG];
  b.ge = c->bg_ge_c ? c->bg_ge_c[k + NG] : c->gamma;
  b.gc = c->bg_gc_c ? c->bg_gc_c[k + NG] : c->gamma;
  return b;
}
/* z-face k-1/2 */
static bgstate bg_zface(const geo *G, int k) {
  const ora_cfg *c = G->c;
  bgstate b = {0, 0, 0, 0};
  if (!c->bg_rho_c) return b;
  b.rho = c->bg_rho_f[k + NG];
  b.p = c->bg_p_f[k + NG];
  b.ge = c->bg_ge_f ? c->bg_ge_f[k + NG] : c->gamma;
  b.gc = c->bg_gc_f ? c->bg_gc_f[k + NG] : c->gamma;
  return b;
}

/* ---------------- EOS hook (Sect. 2.2) ---------------- */
/* From conserved quantities of one cell: returns primitive deviations. */
static int cell_prims(const geo *G, const double *u, const double *bc, int k,
                      double *Tcell, double *w) {
  const ora_cfg *c = G->c;
  double rho = u[U_RHO];
  if (!(rho > 0.0)) return -2;
  double vx = u[U_MX] / rho, vy = u[U_MY] / rho, vz = u[U_MZ] / rho;
  double eint = u[U_E] / rho - 0.5 * (vx * vx + vy * vy + vz * vz)
              - 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]) / rho;
  double X[ORA_MAXSPEC];
  for (int l = 0; l < c->nspec; ++l) X[l] = u[U_X0 + l] / rho;
  double P, ge, gc;
  if (c->eos == ORA_EOS_IDEAL) {
    P = (c->gamma - 1.0) * rho * eint;
    ge = c->gamma;
    gc = c->gamma;
  } else {
    int it;
    int rc = ora_eos_invert(c, rho, eint, X, Tcell, &P, &ge, &gc, &it);
    if (rc) return rc;
  }
  if (!(P > 0.0)) return -2;
  bgstate b = bg_cell(G, k);
  w[W_RHO] = rho - b.rho;
  w[W_VX] = vx; w[W_VY] = vy; w[W_VZ] = vz;
  w[W_BX] = bc[0]; w[W_BY] = bc[1]; w[W_BZ] = bc[2];
  w[W_P] = P - b.p;
  w[W_GE] = ge - b.ge;
  w[W_GC] = gc - b.gc;
  for (int l = 0; l < c->nspec; ++l) w[W_X0 + l] = X[l];
  return 0;
}

/* ---------------- ghost mapping (Table bcs) ---------------- */
/* Source cell index along a dimension for a ghost index; *flip = 1 if the
 * reflecting mirror applies. */
static int ghost_src(int i, int n, int bclo, int bchi, int *flip) {
  *flip = 0;
  if (i < 0) {
    if (bclo == ORA_PERIODIC) return ((i % n) + n) % n;
    if (bclo == ORA_REFLECT) { *flip = 1; return -1 - i; }
    return 0;
  }
  if (i >= n) {
    if (bchi == ORA_PERIODIC) return i % n;
    if (bchi == ORA_REFLECT) { *flip = 1; return 2 * n - 1 - i; }
    return n - 1;
  }
  return i;
}

/* Ghost values of the face-normal field along its own direction (face index f). */
static int ghost_face_src(int f, int n, int bclo, int bchi, double *sign) {
  *sign = 1.0;
  if (f < 0) {
    if (bclo == ORA_PERIODIC) return f + n;
    if (bclo == ORA_REFLECT) { *sign = -1.0; return -f; }
    return 0;
  }
  if (f > n) {
    if (bchi == ORA_PERIODIC) return f - n;
    if (bchi == ORA_REFLECT) { *sign = -1.0; return 2 * n - f; }
    return n;
  }
  return f;
}

/* Fill ghost layers of cell-centred arrays a[0..na-1].  Dimensions are done
 * in the order x, y, z, each pass spanning the ghosts of the dimensions already
 * done, so edge and corner ghosts are filled too.  flipcomp[d][q] = 1: array q
 * changes sign under a reflection across a d-boundary. */
static void fill_cell_ghosts(const geo *G, double **a, int na, int flipcomp[3][16]) {
  for (int d = 0; d < 3; ++d) {
    if (!G->act[d]) continue;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      if (e <= d) { lo[e] = -G->g[e]; hi[e] = G->n[e] + G->g[e]; }
      else { lo[e] = 0; hi[e] = G->n[e]; }
    }
    int c[3];
    for (c[2] = lo[2]; c[2] < hi[2]; ++c[2])
      for (c[1] = lo[1]; c[1] < hi[1]; ++c[1])
        for (c[0] = lo[0]; c[0] < hi[0]; ++c[0]) {
          if (c[d] >= 0 && c[d] < G->n[d]) continue;
          int s[3] = {c[0], c[1], c[2]};
          int flip;
          s[d] = ghost_src(c[d], G->n[d], G->c->bc[d][0], G->c->bc[d][1], &flip);
          long dst = IXv(G, c), src = IXv(G, s);
          for (int q = 0; q < na; ++q) {
            double v = a[q][src];
            if (flip && flipcomp[d][q]) v = -v;
            a[q][dst] = v;
          }
        }
  }
}

/* Fill ghosts of the three face arrays.  The component normal to a reflecting
 * boundary is mirrored with a sign change about the wall face; tangential
 * components are mirrored like cell data. */
static void fill_face_ghosts(const geo *G, double **B) {
  for (int d = 0; d < 3; ++d) {
    if (!G->act[d]) continue;
    for (int comp = 0; comp < 3; ++comp) {
      int lo[3], hi[3];
      for (int e = 0; e < 3; ++e) {
        int extra = (e == comp);
        if (e <= d) { lo[e] = -G->g[e]; hi[e] = G->n[e] + G->g[e] + extra; }
        else { lo[e] = 0; hi[e] = G->n[e] + extra; }
      }
      int c[3];
      for (c[2] = lo[2]; c[2] < hi[2]; ++c[2])
        for (c[1] = lo[1]; c[1] < hi[1]; ++c[1])
          for (c[0] = lo[0]; c[0] < hi[0]; ++c[0]) {
            int s[3] = {c[0], c[1], c[2]};
            double sg = 1.0;
            if (comp == d) {
              if (c[d] >= 0 && c[d] <= G->n[d]) continue;
              s[d] = ghost_face_src(c[d], G->n[d], G->c->bc[d][0], G->c->bc[d][1], &sg);
            } else {
              int flip;
              if (c[d] >= 0 && c[d] < G->n[d]) continue;
              s[d] = ghost_src(c[d], G->n[d], G->c->bc[d][0], G->c->bc[d][1], &flip);
            }
            B[comp][IXv(G, c)] = sg * B[comp][IXv(G, s)];
          }
    }
  }
}

/* ---------------- van Leer limited slope (Sect. 2.5, item i) ---------------- */
static inline double vl_slope(double a, double b, double c) {
  double dm = b - a, dp = c - b;
  if (dm * dp > 0.0) return 2.0 * dm * dp / (dm + dp);
  return 0.0;
}

/* ---------------- PPH reconstruction (Sect. 2.5, item ii) ----------------
 * Third order on the three-cell stencil: the parabola whose averages over
 * cells i-1, i, i+1 are the three cell values, evaluated at the cell's faces.
 * Its right-face value is (-W_{i-1} + 5 W_i + 2 W_{i+1}) / 6 and its
 * left-face value (2 W_{i-1} + 5 W_i - W_{i+1}) / 6.  Unlimited for every
 * primitive variable except the mass fractions.  Those take the limited
 * parabola (reading: the monotonicity constraints of the piecewise parabolic
 * method of Colella & Woodward 1984 -- each face value clipped to the range
 * of the two cells sharing the face; a cell that is a local extremum stays
 * constant; a parabola that would overshoot inside the cell has its far face
 * value pulled back so that it is monotone there). */
static inline double pph_right(double a, double b, double c) { return (-a + 5.0 * b + 2.0 * c) / 6.0; }
static inline double pph_left(double a, double b, double c) { return (2.0 * a + 5.0 * b - c) / 6.0; }
static inline double clip(double v, double x, double y) {
  double lo = x < y ? x : y, hi = x < y ? y : x;
  return v < lo ? lo : (v > hi ? hi : v);
}
/* limited left and right face values of the cell with value b between a and c */
static inline void pph_limited(double a, double b, double c, double *fl, double *fr) {
  if ((b - a) * (c - b) <= 0.0) { *fl = b; *fr = b; return; }
  double l = clip(pph_left(a, b, c), a, b), r = clip(pph_right(a, b, c), b, c);
  const double d = r - l, a6 = 6.0 * (b - 0.5 * (l + r));
  if (d * a6 > d * d) l = 3.0 * b - 2.0 * r;
  else if (d * a6 < -d * d) r = 3.0 * b - 2.0 * l;
  *fl = l; *fr = r;
}

/* Limited fifth-order reconstruction (Sect. 2.5, item iii: a limited
 * fifth-order polynomial reconstruction following the PQH method of the cited
 * Leidi et al. 2024, applied to every variable; that method is not printed,
 * reading): the face value of the degree-4 polynomial whose averages over the
 * five cells i-2..i+2 are the cell values,
 *   right face (2a - 13b + 47c + 27d - 3e) / 60 (the left face mirrored),
 * limited by the monotonicity-preserving bounds of Suresh & Huynh (1997):
 * kept where it lies between the cell value and the monotone bound
 * c + minmod(d - c, 4 (c - b)); otherwise moved to the nearest point of an
 * interval built from the neighbouring values and curvature estimates, which
 * contains the smooth extrema a plain clip would flatten. */
static inline double minmod2(double x, double y) {
  return (x > 0.0 && y > 0.0) ? (x < y ? x : y) : ((x < 0.0 && y < 0.0) ? (x > y ? x : y) : 0.0);
}
static inline double minmod4(double w, double x, double y, double z) {
  return minmod2(minmod2(w, x), minmod2(y, z));
}
static inline double mn3(double x, double y, double z) { double m = x < y ? x : y; return m < z ? m : z; }
static inline double mx3(double x, double y, double z) { double m = x > y ? x : y; return m > z ? m : z; }
/* the limited value at the face between c and d of the cells a b c d e */
static double mp5_face(double a, double b, double c, double d, double e) {
  const double vor = (2.0 * a - 13.0 * b + 47.0 * c + 27.0 * d - 3.0 * e) / 60.0;
  const double vmp = c + minmod2(d - c, 4.0 * (c - b));
  if ((vor - c) * (vor - vmp) <= 0.0) return vor;
  const double djm1 = a - 2.0 * b + c, dj = b - 2.0 * c + d, djp1 = c - 2.0 * d + e;
  const double dm4p = minmod4(4.0 * dj - djp1, 4.0 * djp1 - dj, dj, djp1);
  const double dm4m = minmod4(4.0 * dj - djm1, 4.0 * djm1 - dj, dj, djm1);
  const double vul = c + 4.0 * (c - b);
  const double vav = 0.5 * (c + d);
  const double vmd = vav - 0.5 * dm4p;
  const double vlc = c + 0.5 * (c - b) + 4.0 / 3.0 * dm4m;
  const double lo = fmax(mn3(c, d, vmd), mn3(c, vul, vlc));
  const double hi = fmin(mx3(c, d, vmd), mx3(c, vul, vlc));
  return vor + minmod2(lo - vor, hi - vor);
}
/* left and right face values of cell c (stencil a b c d e) */
static inline void pqh_limited(double a, double b, double c, double d, double e, double *fl, double *fr) {
  *fr = mp5_face(a, b, c, d, e);
  *fl = mp5_face(e, d, c, b, a);
}

/* Face values of the centre cell w[2] of five cells, for tests: recon, and
 * species != 0 for a mass fraction (PPH limits only those). */
void ora_recon_cell(int recon, int species, const double *w, double *fl, double *fr) {
  if (recon == ORA_RECON_PQH) { pqh_limited(w[0], w[1], w[2], w[3], w[4], fl, fr); return; }
  if (recon == ORA_RECON_PPH) {
    if (species) { pph_limited(w[1], w[2], w[3], fl, fr); return; }
    *fl = pph_left(w[1], w[2], w[3]);
    *fr = pph_right(w[1], w[2], w[3]);
    return;
  }
  const double sl = vl_slope(w[1], w[2], w[3]);
  *fl = w[2] - 0.5 * sl;
  *fr = w[2] + 0.5 * sl;
}

/* ---------------- Riemann solvers (Sect. 2.6) ---------------- */
/* Normal-frame state: rho, un, ut1, ut2, Bt1, Bt2, P, ge, gc, X.. */
enum { R_RHO = 0, R_UN, R_UT1, R_UT2, R_BT1, R_BT2, R_P, R_GE, R_GC, R_X0 };
/* flux/conserved normal-frame: rho, mn, mt1, mt2, E, Bt1, Bt2, rhoX.. */
enum { Q_RHO = 0, Q_MN, Q_MT1, Q_MT2, Q_E, Q_BT1, Q_BT2, Q_X0 };

typedef struct {
  double rho, un, ut1, ut2, bn, bt1, bt2, p, ge, gc;
  double pt, e, cf, cs;
  double U[7], F[7];
} rstate;

static void rstate_init(rstate *s, const double *w, double bn) {
  s->rho = w[R_RHO]; s->un = w[R_UN]; s->ut1 = w[R_UT1]; s->ut2 = w[R_UT2];
  s->bn = bn; s->bt1 = w[R_BT1]; s->bt2 = w[R_BT2]; s->p = w[R_P];
  s->ge = w[R_GE]; s->gc = w[R_GC];
  double b2 = bn * bn + s->bt1 * s->bt1 + s->bt2 * s->bt2;
  double u2 = s->un * s->un + s->ut1 * s->ut1 + s->ut2 * s->ut2;
  s->pt = s->p + 0.5 * b2;
  /* e_int = P / (rho (gamma_e - 1))  (Sect. 2.6, reconstructed gamma_e) */
  s->e = s->p / (s->ge - 1.0) + 0.5 * s->rho * u2 + 0.5 * b2;
  double a2 = s->gc * s->p / s->rho;
  double bb = b2 / s->rho, bnn = bn * bn / s->rho;
  double disc = (a2 + bb) * (a2 + bb) - 4.0 * a2 * bnn;
  if (disc < 0.0) disc = 0.0;
  s->cf = sqrt(0.5 * (a2 + bb + sqrt(disc)));
  s->cs = sqrt(a2);
  double vb = s->un * bn + s->ut1 * s->bt1 + s->ut2 * s->bt2;
  s->U[Q_RHO] = s->rho; s->U[Q_MN] = s->rho * s->un; s->U[Q_MT1] = s->rho * s->ut1;
  s->U[Q_MT2] = s->rho * s->ut2; s->U[Q_E] = s->e; s->U[Q_BT1] = s->bt1; s->U[Q_BT2] = s->bt2;
  s->F[Q_RHO] = s->rho * s->un;
  s->F[Q_MN] = s->rho * s->un * s->un + s->pt - bn * bn;
  s->F[Q_MT1] = s->rho * s->un * s->ut1 - bn * s->bt1;
  s->F[Q_MT2] = s->rho * s->un * s->ut2 - bn * s->bt2;
  s->F[Q_E] = (s->e + s->pt) * s->un - bn * vb;
  s->F[Q_BT1] = s->un * s->bt1 - s->ut1 * bn;
  s->F[Q_BT2] = s->un * s->bt2 - s->ut2 * bn;
}

/* One side's single-star state (Miyoshi & Kusano 2005 HLLD). */
static void star_state(const rstate *s, double S, double SM, double pts, double *Us,
                       double *vs1, double *vs2, double *bs1, double *bs2) {
  double rhos = s->rho * (S - s->un) / (S - SM);
  double den = s->rho * (S - s->un) * (S - SM) - s->bn * s->bn;
  double scale = s->rho * (S - s->un) * (S - s->un) + s->bn * s->bn;
  if (fabs(den) < 1e-12 * scale) {
    *vs1 = s->ut1; *vs2 = s->ut2; *bs1 = s->bt1; *bs2 = s->bt2;
  } else {
    double fv = s->bn * (SM - s->un) / den;
    double fb = (s->rho * (S - s->un) * (S - s->un) - s->bn * s->bn) / den;
    *vs1 = s->ut1 - s->bt1 * fv;
    *vs2 = s->ut2 - s->bt2 * fv;
    *bs1 = s->bt1 * fb;
    *bs2 = s->bt2 * fb;
  }
  double vb = s->un * s->bn + s->ut1 * s->bt1 + s->ut2 * s->bt2;
  double vbs = SM * s->bn + *vs1 * *bs1 + *vs2 * *bs2;
  double es = ((S - s->un) * s->e - s->pt * s->un + pts * SM + s->bn * (vb - vbs)) / (S - SM);
  Us[Q_RHO] = rhos; Us[Q_MN] = rhos * SM; Us[Q_MT1] = rhos * *vs1; Us[Q_MT2] = rhos * *vs2;
  Us[Q_E] = es; Us[Q_BT1] = *bs1; Us[Q_BT2] = *bs2;
}

/* Low-dissipation factor xi (Sect. 2.6, Eq. after pstar): max(M_L, M_R) if it
 * is below the threshold, 1 otherwise; M = |u| / c_s. */
static double ld_xi(const rstate *L, const rstate *R, double mthr) {
  double ml = sqrt(L->un * L->un + L->ut1 * L->ut1 + L->ut2 * L->ut2) / L->cs;
  double mr = sqrt(R->un * R->un + R->ut1 * R->ut1 + R->ut2 * R->ut2) / R->cs;
  double m = ml > mr ? ml : mr;
  return m < mthr ? m : 1.0;
}

/* Direction of the contact used by Contact-CT upwinding: the sign of the mass
 * flux, or 0 when |F_rho| is below 1e-12 rho max|S| -- a mass flux at the
 * rounding level of the face's flux scale carries no direction, and the
 * Contact-CT rule for a zero mass flux (average of both sides) applies. */
static int contact_dir(double frho, double rhol, double rhor, double SL, double SR) {
  double scale = 1e-12 * fmax(rhol, rhor) * fmax(fabs(SL), fabs(SR));
  return frho > scale ? 1 : (frho < -scale ? -1 : 0);
}

/* Contact-CT corner EMF (Sect. 2.4; Gardiner & Stone 2005) of the edge at the
 * corner (a-1/2, b-1/2): Ea1, Ea0 the face EMFs of the a-faces above and
 * below the corner, Eb1, Eb0 those of the b-faces right and left of it, Eij
 * the cell reference EMFs of cells (c_a - 1 + i, c_b - 1 + j), m* the contact
 * directions of the four faces.  The corner averages the four face values
 * and their extrapolations to the corner; each half-cell derivative is taken
 * from the upwind cell of the face's mass flux, the mean of both with none. */
static double ct_corner(double Ea1, double Ea0, double Eb1, double Eb0, double E00, double E10, double E01,
                        double E11, int ma1, int ma0, int mb1, int mb0) {
  /* derivatives along b on the a-faces, upwinded in a */
  double lo_l = Eb0 - E00, lo_r = Eb1 - E10;    /* below the corner */
  double up_l = E01 - Eb0, up_r = E11 - Eb1;    /* above the corner */
  double dlo = ma0 > 0 ? lo_l : (ma0 < 0 ? lo_r : 0.5 * (lo_l + lo_r));
  double dup = ma1 > 0 ? up_l : (ma1 < 0 ? up_r : 0.5 * (up_l + up_r));
  /* derivatives along a on the b-faces, upwinded in b */
  double le_d = Ea0 - E00, le_u = Ea1 - E01;    /* left of the corner  */
  double ri_d = E10 - Ea0, ri_u = E11 - Ea1;    /* right of the corner */
  double dle = mb0 > 0 ? le_d : (mb0 < 0 ? le_u : 0.5 * (le_d + le_u));
  double dri = mb1 > 0 ? ri_d : (mb1 < 0 ? ri_u : 0.5 * (ri_d + ri_u));
  return 0.25 * (Ea1 + Ea0 + Eb1 + Eb0) + 0.25 * (dlo - dup) + 0.25 * (dle - dri);
}

double ora_ct_corner(const double *Ef, const double *Ec, const double *F, double rho, double smax) {
  int m[4];
  for (int q = 0; q < 4; ++q) m[q] = contact_dir(F[q], rho, rho, -smax, smax);
  return ct_corner(Ef[0], Ef[1], Ef[2], Ef[3], Ec[0], Ec[1], Ec[2], Ec[3], m[0], m[1], m[2], m[3]);
}

static void riemann_core(const double *wl, const double *wr, double bn, int nspec,
                         int solver, double mach_thr, double *f, int *up);

void ora_riemann(const double *wl, const double *wr, double bn, int nspec,
                 int solver, double mach_thr, double *f) {
  int up;
  riemann_core(wl, wr, bn, nspec, solver, mach_thr, f, &up);
}

void ora_riemann_up(const double *wl, const double *wr, double bn, int nspec,
                    int solver, double mach_thr, double *f, int *up) {
  riemann_core(wl, wr, bn, nspec, solver, mach_thr, f, up);
}

static void riemann_core(const double *wl, const double *wr, double bn, int nspec,
                         int solver, double mach_thr, double *f, int *up) {
  rstate L, R;
  rstate_init(&L, wl, bn);
  rstate_init(&R, wr, bn);
  double SL = fmin(L.un - L.cf, R.un - R.cf);
  double SR = fmax(L.un + L.cf, R.un + R.cf);
  double xl[ORA_MAXSPEC], xr[ORA_MAXSPEC];
  /* consistent multi-fluid advection: rescale X_l by their sum (Sect. 2.9) */
  double sl = 0.0, sr = 0.0;
  for (int l = 0; l < nspec; ++l) { sl += wl[R_X0 + l]; sr += wr[R_X0 + l]; }
  for (int l = 0; l < nspec; ++l) { xl[l] = wl[R_X0 + l] / sl; xr[l] = wr[R_X0 + l] / sr; }

  if (solver == ORA_HLL) {
    if (SL >= 0.0) {
      for (int q = 0; q < 7; ++q) f[q] = L.F[q];
      for (int l = 0; l < nspec; ++l) f[Q_X0 + l] = L.F[Q_RHO] * xl[l];
    } else if (SR <= 0.0) {
      for (int q = 0; q < 7; ++q) f[q] = R.F[q];
      for (int l = 0; l < nspec; ++l) f[Q_X0 + l] = R.F[Q_RHO] * xr[l];
    } else {
      for (int q = 0; q < 7; ++q)
        f[q] = (SR * L.F[q] - SL * R.F[q] + SL * SR * (R.U[q] - L.U[q])) / (SR - SL);
      for (int l = 0; l < nspec; ++l) {
        double ul = L.rho * xl[l], ur = R.rho * xr[l];
        f[Q_X0 + l] = (SR * L.F[Q_RHO] * xl[l] - SL * R.F[Q_RHO] * xr[l] + SL * SR * (ur - ul)) / (SR - SL);
      }
    }
    *up = contact_dir(f[Q_RHO], L.rho, R.rho, SL, SR);
    return;
  }

  double xi = (solver == ORA_LHLLD) ? ld_xi(&L, &R, mach_thr) : 1.0;
  double D = (SR - R.un) * R.rho - (SL - L.un) * L.rho;
  double SM = ((SR - R.un) * R.rho * R.un - (SL - L.un) * L.rho * L.un - R.pt + L.pt) / D;
  /* total pressure of the HLLD intermediate states: central part + dissipative
   * part proportional to (u_R - u_L) (the HLLD analogue of Eq. pstar) */
  double pdis = L.rho * R.rho * (SR - R.un) * (SL - L.un) * (R.un - L.un) / D;
  double pts = ((SR - R.un) * R.rho * L.pt - (SL - L.un) * L.rho * R.pt) / D + pdis;
  double UsL[7], UsR[7], vL1, vL2, bL1, bL2, vR1, vR2, bR1, bR2;
  star_state(&L, SL, SM, pts, UsL, &vL1, &vL2, &bL1, &bL2);
  star_state(&R, SR, SM, pts, UsR, &vR1, &vR2, &bR1, &bR2);
  double sqL = sqrt(UsL[Q_RHO]), sqR = sqrt(UsR[Q_RHO]);
  double sgn = bn >= 0.0 ? 1.0 : -1.0;
  double SsL = SM - fabs(bn) / sqL, SsR = SM + fabs(bn) / sqR;
  double FsL[7], FsR[7];
  for (int q = 0; q < 7; ++q) {
    FsL[q] = L.F[q] + SL * (UsL[q] - L.U[q]);
    FsR[q] = R.F[q] + SR * (UsR[q] - R.U[q]);
  }
  double F[7];
  int left;
  if (SL >= 0.0) { for (int q = 0; q < 7; ++q) F[q] = L.F[q]; left = 1; }
  else if (SsL >= 0.0) { for (int q = 0; q < 7; ++q) F[q] = FsL[q]; left = 1; }
  else if (SsR < 0.0 && SR >= 0.0) { for (int q = 0; q < 7; ++q) F[q] = FsR[q]; left = 0; }
  else if (SR < 0.0) { for (int q = 0; q < 7; ++q) F[q] = R.F[q]; left = 0; }
  else {
    /* double-star states between the Alfven waves */
    double den = sqL + sqR;
    double vss1 = (sqL * vL1 + sqR * vR1 + (bR1 - bL1) * sgn) / den;
    double vss2 = (sqL * vL2 + sqR * vR2 + (bR2 - bL2) * sgn) / den;
    double bss1 = (sqL * bR1 + sqR * bL1 + sqL * sqR * (vR1 - vL1) * sgn) / den;
    double bss2 = (sqL * bR2 + sqR * bL2 + sqL * sqR * (vR2 - vL2) * sgn) / den;
    double vbss = SM * bn + vss1 * bss1 + vss2 * bss2;
    if (SM >= 0.0) {
      double vbs = SM * bn + vL1 * bL1 + vL2 * bL2;
      double Uss[7];
      Uss[Q_RHO] = UsL[Q_RHO]; Uss[Q_MN] = UsL[Q_RHO] * SM;
      Uss[Q_MT1] = UsL[Q_RHO] * vss1; Uss[Q_MT2] = UsL[Q_RHO] * vss2;
      Uss[Q_E] = UsL[Q_E] - sqL * (vbs - vbss) * sgn;
      Uss[Q_BT1] = bss1; Uss[Q_BT2] = bss2;
      for (int q = 0; q < 7; ++q) F[q] = FsL[q] + SsL * (Uss[q] - UsL[q]);
      left = 1;
    } else {
      double vbs = SM * bn + vR1 * bR1 + vR2 * bR2;
      double Uss[7];
      Uss[Q_RHO] = UsR[Q_RHO]; Uss[Q_MN] = UsR[Q_RHO] * SM;
      Uss[Q_MT1] = UsR[Q_RHO] * vss1; Uss[Q_MT2] = UsR[Q_RHO] * vss2;
      Uss[Q_E] = UsR[Q_E] + sqR * (vbs - vbss) * sgn;
      Uss[Q_BT1] = bss1; Uss[Q_BT2] = bss2;
      for (int q = 0; q < 7; ++q) F[q] = FsR[q] + SsR * (Uss[q] - UsR[q]);
      left = 0;
    }
  }
  /* LHLLD: inside the Riemann fan the interface total pressure carries the
   * dissipative part scaled by xi (Sect. 2.6).  The intermediate states stay
   * those of HLLD; the pressure acting in the normal-momentum flux and its
   * work in the energy flux are corrected by (xi - 1) * pdis. */
  if (xi != 1.0 && SL < 0.0 && SR > 0.0) {
    F[Q_MN] += (xi - 1.0) * pdis;
    F[Q_E] += (xi - 1.0) * pdis * SM;
  }
  for (int q = 0; q < 7; ++q) f[q] = F[q];
  for (int l = 0; l < nspec; ++l) f[Q_X0 + l] = F[Q_RHO] * (left ? xl[l] : xr[l]);
  *up = contact_dir(F[Q_RHO], L.rho, R.rho, SL, SR);
}

/* ---------------- one stage ---------------- */
typedef struct {
  geo G;
  double *W[10 + ORA_MAXSPEC];
  double *B[3];
  double *F[3][8 + ORA_MAXSPEC];
  double *E[3];
  signed char *up[3];        /* contact direction per face (Contact-CT upwinding) */
  unsigned char *raw, *flag;
  double *fhat_c, *fhat_f;   /* per-k normal-frame background fluxes (7 + nspec) */
} work;

static int work_alloc(work *w, const ora_cfg *c) {
  memset(w, 0, sizeof(*w));
  geo_init(&w->G, c);
  long n = w->G.ntot;
  for (int q = 0; q < w->G.nw; ++q) if (!(w->W[q] = calloc(n, sizeof(double)))) return -1;
  for (int d = 0; d < 3; ++d) if (!(w->B[d] = calloc(n, sizeof(double)))) return -1;
  for (int d = 0; d < 3; ++d) {
    if (!w->G.act[d]) continue;
    for (int q = 0; q < w->G.nf; ++q) if (!(w->F[d][q] = calloc(n, sizeof(double)))) return -1;
  }
  for (int d = 0; d < 3; ++d) if (!(w->E[d] = calloc(n, sizeof(double)))) return -1;
  for (int d = 0; d < 3; ++d) if (!(w->up[d] = calloc(n, 1))) return -1;
  w->raw = calloc(n, 1);
  w->flag = calloc(n, 1);
  int nz = c->n[2];
  w->fhat_c = calloc((size_t)(nz + 2 * NG) * 16, sizeof(double));
  w->fhat_f = calloc((size_t)(nz + 2 * NG + 1) * 16, sizeof(double));
  return 0;
}

static void work_free(work *w) {
  for (int q = 0; q < 10 + ORA_MAXSPEC; ++q) free(w->W[q]);
  for (int d = 0; d < 3; ++d) {
    free(w->B[d]); free(w->E[d]); free(w->up[d]);
    for (int q = 0; q < 8 + ORA_MAXSPEC; ++q) free(w->F[d][q]);
  }
  free(w->raw); free(w->flag); free(w->fhat_c); free(w->fhat_f);
}

/* Normal-frame face state from a background (u = 0, B = 0). */
static void bg_rstate(const geo *G, bgstate b, double *w) {
  memset(w, 0, sizeof(double) * (R_X0 + ORA_MAXSPEC));
  w[R_RHO] = b.rho; w[R_P] = b.p; w[R_GE] = b.ge; w[R_GC] = b.gc;
  /* species of the background flux carry no mass flux; give them a valid sum */
  for (int l = 0; l < G->c->nspec; ++l) w[R_X0 + l] = 1.0 / G->c->nspec;
}

static int compute_rhs(work *w, const double *cons, const double *bx, const double *by,
                       const double *bz, double *T, double *R, double *RB[3]) {
  geo *G = &w->G;
  const ora_cfg *c = G->c;
  const double *bin[3] = {bx, by, bz};
  int nspec = c->nspec;
  int solver = c->riemann;
  int rc = 0;

  /* (1) face fields with ghosts */
  for (int d = 0; d < 3; ++d) {
    int ext[3] = {G->n[0] + (d == 0), G->n[1] + (d == 1), G->n[2] + (d == 2)};
    for (int k = 0; k < ext[2]; ++k)
      for (int j = 0; j < ext[1]; ++j)
        for (int i = 0; i < ext[0]; ++i)
          w->B[d][IX(G, i, j, k)] = bin[d][AF(G, d, i, j, k)];
  }
  fill_face_ghosts(G, w->B);

  /* (2) primitives + EOS on interior cells, as deviations from the background */
#pragma omp parallel for reduction(min : rc) schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        double u[5 + ORA_MAXSPEC], bc[3], ww[10 + ORA_MAXSPEC];
        long a = AC(G, i, j, k), p = IX(G, i, j, k);
        for (int v = 0; v < G->nv; ++v) u[v] = cons[v * abi_cells(G) + a];
        bc[0] = 0.5 * (w->B[0][p] + w->B[0][p + G->s[0]]);
        bc[1] = 0.5 * (w->B[1][p] + w->B[1][p + G->s[1]]);
        bc[2] = 0.5 * (w->B[2][p] + w->B[2][p + G->s[2]]);
        int r = cell_prims(G, u, bc, k, T ? &T[a] : NULL, ww);
        if (r) rc = r;
        for (int q = 0; q < G->nw; ++q) w->W[q][p] = ww[q];
      }
  if (rc) return rc;
  /* (3) ghost deviations: mirror with normal velocity / field negated */
  {
    int flip[3][16];
    memset(flip, 0, sizeof(flip));
    for (int d = 0; d < 3; ++d) { flip[d][W_VX + d] = 1; flip[d][W_BX + d] = 1; }
    fill_cell_ghosts(G, w->W, G->nw, flip);
  }

  /* (4) shock flags (Sect. 2.7) on interior cells, dilated over 5^ndim */
  memset(w->raw, 0, G->ntot);
  memset(w->flag, 0, G->ntot);
  if (c->eps_sf > 0.0) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          long p = IX(G, i, j, k);
          double P0 = w->W[W_P][p] + bg_cell(G, k).p;
          double sum = 0.0;
          for (int d = 0; d < 3; ++d) {
            if (!G->act[d]) continue;
            int kp = k + (d == 2), km = k - (d == 2);
            double Pp = w->W[W_P][p + G->s[d]] + bg_cell(G, kp).p;
            double Pm = w->W[W_P][p - G->s[d]] + bg_cell(G, km).p;
            sum += fabs(Pp - Pm);
          }
          w->raw[p] = (sum / (c->eps_sf * P0) > 1.0);
        }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          int f = 0;
          int r0 = G->act[0] ? 2 : 0, r1 = G->act[1] ? 2 : 0, r2 = G->act[2] ? 2 : 0;
          for (int dk = -r2; dk <= r2 && !f; ++dk)
            for (int dj = -r1; dj <= r1 && !f; ++dj)
              for (int di = -r0; di <= r0 && !f; ++di) {
                int cc[3] = {i + di, j + dj, k + dk}, ok = 1;
                for (int d = 0; d < 3; ++d) {
                  if (cc[d] < 0 || cc[d] >= G->n[d]) {
                    int per = (cc[d] < 0 ? c->bc[d][0] : c->bc[d][1]) == ORA_PERIODIC;
                    if (!per) { ok = 0; break; }
                    cc[d] = ((cc[d] % G->n[d]) + G->n[d]) % G->n[d];
                  }
                }
                if (ok && w->raw[IXv(G, cc)]) f = 1;
              }
          w->flag[IX(G, i, j, k)] = (unsigned char)f;
        }
    /* ghosts carry the flag of the cell their data comes from */
    double *tmp = calloc(G->ntot, sizeof(double));
    for (long p = 0; p < G->ntot; ++p) tmp[p] = w->flag[p];
    int noflip[3][16];
    memset(noflip, 0, sizeof(noflip));
    fill_cell_ghosts(G, &tmp, 1, noflip);
    for (long p = 0; p < G->ntot; ++p) w->flag[p] = tmp[p] != 0.0;
    free(tmp);
  }

  /* background fluxes F_hat = F(W_hat, W_hat) with the same solver (Sect. 2.8) */
  int has_bg = c->bg_rho_c != NULL;
  if (has_bg) {
    double wb[R_X0 + ORA_MAXSPEC], fb[Q_X0 + ORA_MAXSPEC];
    for (int k = -NG; k < G->n[2] + NG; ++k) {
      bg_rstate(G, bg_cell(G, k), wb);
      ora_riemann(wb, wb, 0.0, nspec, solver, c->mach_thr, fb);
      for (int q = 0; q < 7 + nspec; ++q) w->fhat_c[(k + NG) * 16 + q] = fb[q];
    }
    for (int k = -NG; k <= G->n[2] + NG; ++k) {
      bg_rstate(G, bg_zface(G, k), wb);
      ora_riemann(wb, wb, 0.0, nspec, solver, c->mach_thr, fb);
      for (int q = 0; q < 7 + nspec; ++q) w->fhat_f[(k + NG) * 16 + q] = fb[q];
    }
  }

  /* (5) fluxes per direction: PLM of deviations, add W_hat at the face, Riemann */
  for (int d = 0; d < 3; ++d) {
    if (!G->act[d]) continue;
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      if (e == d) { lo[e] = 0; hi[e] = G->n[e] + 1; }
      else if (G->act[e]) { lo[e] = -1; hi[e] = G->n[e] + 1; }
      else { lo[e] = 0; hi[e] = 1; }
    }
#pragma omp parallel for reduction(min : rc) schedule(static)
    for (int kz = lo[2]; kz < hi[2]; ++kz)
      for (int ky = lo[1]; ky < hi[1]; ++ky)
        for (int kx = lo[0]; kx < hi[0]; ++kx) {
          int c3[3] = {kx, ky, kz};
          long pR = IXv(G, c3), pL = pR - G->s[d];
          long sd = G->s[d];
          double wl[10 + ORA_MAXSPEC], wr[10 + ORA_MAXSPEC];
          /* shock flattening (Sect. 2.7): a flagged cell reconstructs with van Leer */
          const int vlL = c->recon == ORA_RECON_VANLEER || w->flag[pL];
          const int vlR = c->recon == ORA_RECON_VANLEER || w->flag[pR];
          for (int q = 0; q < G->nw; ++q) {
            const double a = w->W[q][pL - sd], b = w->W[q][pL], cc = w->W[q][pR], e = w->W[q][pR + sd];
            if (c->recon == ORA_RECON_PQH && (!vlL || !vlR)) {
              double fl_, fr_, pl, pr;
              const double a2 = w->W[q][pL - 2 * sd], e2 = w->W[q][pR + 2 * sd];
              pqh_limited(a2, a, b, cc, e, &fl_, &fr_);   /* cell pL */
              pl = fr_;
              pqh_limited(a, b, cc, e, e2, &fl_, &fr_);   /* cell pR */
              pr = fl_;
              wl[q] = vlL ? b + 0.5 * vl_slope(a, b, cc) : pl;
              wr[q] = vlR ? cc - 0.5 * vl_slope(b, cc, e) : pr;
            } else if (!vlL || !vlR) {   /* PPH: left state from cell pL's right face, right state from pR's left face */
              double pl, pr;
              if (q < W_X0) { pl = pph_right(a, b, cc); pr = pph_left(b, cc, e); }
              else {
                double fl_, fr_;
                pph_limited(a, b, cc, &fl_, &fr_);
                pl = fr_;
                pph_limited(b, cc, e, &fl_, &fr_);
                pr = fl_;
              }
              wl[q] = vlL ? b + 0.5 * vl_slope(a, b, cc) : pl;
              wr[q] = vlR ? cc - 0.5 * vl_slope(b, cc, e) : pr;
            } else {
              double sL = vl_slope(a, b, cc);
              double sR = vl_slope(b, cc, e);
              wl[q] = b + 0.5 * sL;
              wr[q] = cc - 0.5 * sR;
            }
          }
          int k = c3[2];
          bgstate bf = (d == 2) ? bg_zface(G, k) : bg_cell(G, k);
          double rl[R_X0 + ORA_MAXSPEC], rr[R_X0 + ORA_MAXSPEC];
          rl[R_RHO] = wl[W_RHO] + bf.rho; rr[R_RHO] = wr[W_RHO] + bf.rho;
          rl[R_UN] = wl[W_VX + d]; rr[R_UN] = wr[W_VX + d];
          rl[R_UT1] = wl[W_VX + t1]; rr[R_UT1] = wr[W_VX + t1];
          rl[R_UT2] = wl[W_VX + t2]; rr[R_UT2] = wr[W_VX + t2];
          rl[R_BT1] = wl[W_BX + t1]; rr[R_BT1] = wr[W_BX + t1];
          rl[R_BT2] = wl[W_BX + t2]; rr[R_BT2] = wr[W_BX + t2];
          rl[R_P] = wl[W_P] + bf.p; rr[R_P] = wr[W_P] + bf.p;
          rl[R_GE] = wl[W_GE] + bf.ge; rr[R_GE] = wr[W_GE] + bf.ge;
          rl[R_GC] = wl[W_GC] + bf.gc; rr[R_GC] = wr[W_GC] + bf.gc;
          for (int l = 0; l < nspec; ++l) { rl[R_X0 + l] = wl[W_X0 + l]; rr[R_X0 + l] = wr[W_X0 + l]; }
          if (!(rl[R_RHO] > 0.0 && rr[R_RHO] > 0.0 && rl[R_P] > 0.0 && rr[R_P] > 0.0)) rc = -2;
          double bn = w->B[d][pR];
          int sol = (w->flag[pL] || w->flag[pR]) ? ORA_HLL : solver;
          double fq[Q_X0 + ORA_MAXSPEC];
          int updir;
          riemann_core(rl, rr, bn, nspec, sol, c->mach_thr, fq, &updir);
          if (has_bg) {
            const double *fh = (d == 2) ? &w->fhat_f[(k + NG) * 16] : &w->fhat_c[(k + NG) * 16];
            for (int q = 0; q < 7 + nspec; ++q) fq[q] -= fh[q];
          }
          /* A reflecting wall face is a symmetry plane of its Riemann problem
           * (Table bcs: u_n = 0, B_n = 0): every flux component except the
           * normal momentum vanishes there.  Set them to zero instead of to the
           * solver's rounding residue. */
          if ((c3[d] == 0 && c->bc[d][0] == ORA_REFLECT) || (c3[d] == G->n[d] && c->bc[d][1] == ORA_REFLECT))
            for (int q = 0; q < 7 + nspec; ++q) {
              if (q != Q_MN) fq[q] = 0.0;
              updir = 0;
            }
          w->up[d][pR] = (signed char)updir;
          w->F[d][F_RHO][pR] = fq[Q_RHO];
          w->F[d][F_MX + d][pR] = fq[Q_MN];
          w->F[d][F_MX + t1][pR] = fq[Q_MT1];
          w->F[d][F_MX + t2][pR] = fq[Q_MT2];
          w->F[d][F_E][pR] = fq[Q_E];
          w->F[d][F_BX + d][pR] = 0.0;
          w->F[d][F_BX + t1][pR] = fq[Q_BT1];
          w->F[d][F_BX + t2][pR] = fq[Q_BT2];
          for (int l = 0; l < nspec; ++l) w->F[d][F_X0 + l][pR] = fq[Q_X0 + l];
        }
  }
  if (rc) return rc;

  /* (6) Contact-CT edge EMFs (Sect. 2.4; Gardiner & Stone 2005).
   * Edge along d sits at the lower corner (a-1/2, b-1/2) of cell (.., a, b),
   * with (d, a, b) cyclic.  E_d = -F_a(B_b) on a-faces, +F_b(B_a) on b-faces,
   * cell reference E_d = -(u_a B_b - u_b B_a).  The corner value averages the
   * extrapolations from the four adjacent faces; each half-cell derivative is
   * upwinded by the mass flux through the face it is taken on. */
  for (int d = 0; d < 3; ++d) {
    int a = (d + 1) % 3, b = (d + 2) % 3;
    int hi[3];
    hi[d] = G->n[d];
    hi[a] = G->act[a] ? G->n[a] + 1 : 1;
    hi[b] = G->act[b] ? G->n[b] + 1 : 1;
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < hi[2]; ++kz)
      for (int ky = 0; ky < hi[1]; ++ky)
        for (int kx = 0; kx < hi[0]; ++kx) {
          int cc[3] = {kx, ky, kz};
          long p = IXv(G, cc);
          double Ed = 0.0;
          if (G->act[a] && G->act[b]) {
            long sa = G->s[a], sb = G->s[b];
            /* face EMFs */
            double Ea1 = -w->F[a][F_BX + b][p];          /* a-face (c_a, c_b)   */
            double Ea0 = -w->F[a][F_BX + b][p - sb];     /* a-face (c_a, c_b-1) */
            double Eb1 = w->F[b][F_BX + a][p];           /* b-face (c_a, c_b)   */
            double Eb0 = w->F[b][F_BX + a][p - sa];      /* b-face (c_a-1, c_b) */
            /* contact directions (signs of the mass fluxes) on those faces */
            int ma1 = w->up[a][p], ma0 = w->up[a][p - sb];
            int mb1 = w->up[b][p], mb0 = w->up[b][p - sa];
            /* cell reference EMFs at (c_a-1|c_a, c_b-1|c_b) */
            long q00 = p - sa - sb, q10 = p - sb, q01 = p - sa, q11 = p;
#define ECELL(q) (-(w->W[W_VX + a][q] * w->W[W_BX + b][q] - w->W[W_VX + b][q] * w->W[W_BX + a][q]))
            double E00 = ECELL(q00), E10 = ECELL(q10), E01 = ECELL(q01), E11 = ECELL(q11);
#undef ECELL
            Ed = ct_corner(Ea1, Ea0, Eb1, Eb0, E00, E10, E01, E11, ma1, ma0, mb1, mb0);
          } else if (G->act[a]) {
            Ed = -w->F[a][F_BX + b][p];
          } else if (G->act[b]) {
            Ed = w->F[b][F_BX + a][p];
          }
          /* An edge lying on a reflecting wall: u_n = 0 and B_n = 0 there
           * (Table bcs) make the tangential EMF -(u x B)_t vanish. */
          if ((G->act[a] && ((cc[a] == 0 && c->bc[a][0] == ORA_REFLECT) ||
                             (cc[a] == G->n[a] && c->bc[a][1] == ORA_REFLECT))) ||
              (G->act[b] && ((cc[b] == 0 && c->bc[b][0] == ORA_REFLECT) ||
                             (cc[b] == G->n[b] && c->bc[b][1] == ORA_REFLECT))))
            Ed = 0.0;
          w->E[d][p] = Ed;
        }
  }

  /* (7) cell residual R = div F - (S - S_hat) (Eqs. fv, spatres, wb2) */
  long nc = abi_cells(G);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long p = IX(G, i, j, k), a = AC(G, i, j, k);
        double r[5 + ORA_MAXSPEC];
        int map[5 + ORA_MAXSPEC];
        map[U_RHO] = F_RHO; map[U_MX] = F_MX; map[U_MY] = F_MY; map[U_MZ] = F_MZ; map[U_E] = F_E;
        for (int l = 0; l < nspec; ++l) map[U_X0 + l] = F_X0 + l;
        for (int v = 0; v < G->nv; ++v) {
          double s = 0.0;
          for (int d = 0; d < 3; ++d) {
            if (!G->act[d]) continue;
            s += (w->F[d][map[v]][p + G->s[d]] - w->F[d][map[v]][p]) / G->dx[d];
          }
          r[v] = s;
        }
        double rho = cons[U_RHO * nc + a];
        double rhohat = bg_cell(G, k).rho;
        double se = 0.0;
        for (int d = 0; d < 3; ++d) {
          r[U_MX + d] -= (rho - rhohat) * c->g[d];
          se += cons[(U_MX + d) * nc + a] * c->g[d];
        }
        if (c->heat) se += c->heat[k];
        r[U_E] -= se;
        for (int v = 0; v < G->nv; ++v) R[v * nc + a] = r[v];
      }

  /* (8) face residuals: dB_d/dt = -(d_a E_b - d_b E_a), (d, a, b) cyclic */
  for (int d = 0; d < 3; ++d) {
    int a = (d + 1) % 3, b = (d + 2) % 3;
    int ext[3] = {G->n[0] + (d == 0), G->n[1] + (d == 1), G->n[2] + (d == 2)};
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < ext[2]; ++kz)
      for (int ky = 0; ky < ext[1]; ++ky)
        for (int kx = 0; kx < ext[0]; ++kx) {
          int cc[3] = {kx, ky, kz};
          int e[3] = {cc[0], cc[1], cc[2]};
          if (!G->act[d]) e[d] = 0;
          long p = IXv(G, e);
          double r = 0.0;
          if (G->act[a]) r += (w->E[b][p + G->s[a]] - w->E[b][p]) / G->dx[a];
          if (G->act[b]) r -= (w->E[a][p + G->s[b]] - w->E[a][p]) / G->dx[b];
          RB[d][AF(G, d, cc[0], cc[1], cc[2])] = r;
        }
  }
  return 0;
}

int ora_stage(const ora_cfg *cfg, const double *cons_in, const double *bx_in,
              const double *by_in, const double *bz_in, double *T,
              const double *cons_base, const double *bx_base, const double *by_base,
              const double *bz_base, double a, double b, double dt,
              double *cons_out, double *bx_out, double *by_out, double *bz_out) {
  work w;
  if (work_alloc(&w, cfg)) { work_free(&w); return -1; }
  geo *G = &w.G;
  long nc = abi_cells(G);
  double *R = calloc((size_t)nc * G->nv, sizeof(double));
  double *RB[3];
  for (int d = 0; d < 3; ++d) RB[d] = calloc(abi_faces(G, d), sizeof(double));
  int rc = compute_rhs(&w, cons_in, bx_in, by_in, bz_in, T, R, RB);
  if (!rc) {
    for (long q = 0; q < nc * G->nv; ++q)
      cons_out[q] = a * cons_base[q] + b * cons_in[q] - b * dt * R[q];
    const double *bi[3] = {bx_in, by_in, bz_in}, *bb[3] = {bx_base, by_base, bz_base};
    double *bo[3] = {bx_out, by_out, bz_out};
    for (int d = 0; d < 3; ++d)
      for (long q = 0; q < abi_faces(G, d); ++q)
        bo[d][q] = a * bb[d][q] + b * bi[d][q] - b * dt * RB[d][q];
  }
  free(R);
  for (int d = 0; d < 3; ++d) free(RB[d]);
  work_free(&w);
  return rc;
}

/* ---------------- CFL step (Eq. cfl) ---------------- */
double ora_dt(const ora_cfg *cfg, const double *cons, const double *bx,
              const double *by, const double *bz, double *T) {
  geo G;
  geo_init(&G, cfg);
  long nc = abi_cells(&G);
  double mx = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : mx) reduction(max : bad) schedule(static)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        long a = AC(&G, i, j, k);
        double u[5 + ORA_MAXSPEC], bc[3], w[10 + ORA_MAXSPEC];
        for (int v = 0; v < G.nv; ++v) u[v] = cons[v * nc + a];
        bc[0] = 0.5 * (bx[AF(&G, 0, i, j, k)] + bx[AF(&G, 0, i + 1, j, k)]);
        bc[1] = 0.5 * (by[AF(&G, 1, i, j, k)] + by[AF(&G, 1, i, j + 1, k)]);
        bc[2] = 0.5 * (bz[AF(&G, 2, i, j, k)] + bz[AF(&G, 2, i, j, k + 1)]);
        double Tl = T ? T[a] : 0.0;    /* the step's Newton guesses are left untouched */
        if (cell_prims(&G, u, bc, k, T ? &Tl : NULL, w)) { bad = 1; continue; }
        bgstate b = bg_cell(&G, k);
        double rho = w[W_RHO] + b.rho, P = w[W_P] + b.p, gc = w[W_GC] + b.gc;
        double a2 = gc * P / rho;
        double b2 = (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]) / rho;
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (!G.act[d]) continue;
          double bd2 = bc[d] * bc[d] / rho;
          double disc = (a2 + b2) * (a2 + b2) - 4.0 * a2 * bd2;
          if (disc < 0.0) disc = 0.0;
          double cf = sqrt(0.5 * (a2 + b2 + sqrt(disc)));
          s += (fabs(w[W_VX + d]) + cf) / G.dx[d];
        }
        if (s > mx) mx = s;
      }
  if (bad) return -1.0;
  return cfg->cfl / mx;
}

/* ---------------- SSP-RK driver (Sect. 2.9) ---------------- */
int ora_run(const ora_cfg *cfg, double *cons, double *bx, double *by, double *bz,
            double *T, int nsteps, double dt_fixed, double *t, double *dt_last) {
  geo G;
  geo_init(&G, cfg);
  long nc = abi_cells(&G) * G.nv;
  long nf[3] = {abi_faces(&G, 0), abi_faces(&G, 1), abi_faces(&G, 2)};
  double *c0 = malloc(nc * sizeof(double)), *c1 = malloc(nc * sizeof(double));
  double *b0[3], *b1[3];
  for (int d = 0; d < 3; ++d) { b0[d] = malloc(nf[d] * sizeof(double)); b1[d] = malloc(nf[d] * sizeof(double)); }
  int rc = 0;
  for (int s = 0; s < nsteps && !rc; ++s) {
    double dt = dt_fixed > 0.0 ? dt_fixed : ora_dt(cfg, cons, bx, by, bz, T);
    if (!(dt > 0.0)) { rc = -2; break; }
    memcpy(c0, cons, nc * sizeof(double));
    memcpy(b0[0], bx, nf[0] * sizeof(double));
    memcpy(b0[1], by, nf[1] * sizeof(double));
    memcpy(b0[2], bz, nf[2] * sizeof(double));
    if (cfg->rk == 2) {
      rc = ora_stage(cfg, c0, b0[0], b0[1], b0[2], T, c0, b0[0], b0[1], b0[2], 0.0, 1.0, dt,
                     c1, b1[0], b1[1], b1[2]);
      if (!rc) rc = ora_stage(cfg, c1, b1[0], b1[1], b1[2], T, c0, b0[0], b0[1], b0[2], 0.5, 0.5, dt,
                              cons, bx, by, bz);
    } else {
      rc = ora_stage(cfg, c0, b0[0], b0[1], b0[2], T, c0, b0[0], b0[1], b0[2], 0.0, 1.0, dt,
                     c1, b1[0], b1[1], b1[2]);
      if (!rc) rc = ora_stage(cfg, c1, b1[0], b1[1], b1[2], T, c0, b0[0], b0[1], b0[2], 0.75, 0.25, dt,
                              c1, b1[0], b1[1], b1[2]);
      if (!rc) rc = ora_stage(cfg, c1, b1[0], b1[1], b1[2], T, c0, b0[0], b0[1], b0[2],
                              1.0 / 3.0, 2.0 / 3.0, dt, cons, bx, by, bz);
    }
    if (t) *t += dt;
    if (dt_last) *dt_last = dt;
  }
  free(c0); free(c1);
  for (int d = 0; d < 3; ++d) { free(b0[d]); free(b1[d]); }
  return rc;
}

double ora_divb(const ora_cfg *cfg, const double *bx, const double *by, const double *bz) {
  geo G;
  geo_init(&G, cfg);
  const double *b[3] = {bx, by, bz};
  double mx = 0.0, hmin = 1e300;
  for (int d = 0; d < 3; ++d) if (G.act[d] && G.dx[d] < hmin) hmin = G.dx[d];
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (!G.act[d]) continue;
          int c1[3] = {i, j, k};
          c1[d] += 1;
          s += (b[d][AF(&G, d, c1[0], c1[1], c1[2])] - b[d][AF(&G, d, i, j, k)]) / G.dx[d];
        }
        if (fabs(s) > mx) mx = fabs(s);
      }
  return mx * hmin;
}
