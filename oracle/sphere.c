/*
 * sphere.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).  The explicit MHD
 * stage of the oracle on a cubed-sphere shell: six equiangular patches of
 * N x N angular cells times Nr radial cells between r_in and r_out.
 *
 * The paper runs hydrodynamics on the cubed sphere (Sect. 2.3, with the
 * grid of Calhoun et al. 2008) but not MHD (the footnote there).  The
 * extension written here keeps the paper's scheme and its readings (see the
 * Cartesian stage in mhd.c) and adds only what the geometry needs:
 *
 *  - The mesh is treated as an unstructured hexahedral mesh: vertices on
 *    patch edges are shared exactly (their cube-surface coordinates are +-1
 *    or +-tan of an angle computed from |2i - N| with the sign applied), so a
 *    seam face or seam edge is one object seen by two (three at a cube
 *    corner) patches.  Fluxes through a seam face and EMFs on a seam edge are
 *    therefore computed once and enter both sides: mass, energy and the
 *    discrete div B are conserved across seams by construction.
 *  - Momentum and the field are Cartesian vectors, so no vector rotation is
 *    needed across seams, and the finite-volume balance
 *      dU/dt = -(1/V) sum_f F_f . S_f + S
 *    carries no geometric source terms (the divergence theorem on each cell,
 *    Eq. fv with the face area vectors S_f).
 *  - Reconstruction (van Leer PLM, Sect. 2.5) runs along the mesh's lines:
 *    the stencil of a face is its two cells and the cells across their
 *    opposite faces, in whatever patch those lie (logical index space, as the
 *    paper reconstructs on its logically rectangular grids).
 *  - The Riemann problem of a face (LHLLD, Sect. 2.6) is solved in the frame
 *    (n, t1, t2) of its unit normal; the background flux of the face's
 *    hydrostatic state is removed (deviation form, Sect. 2.8).
 *  - The field is stored as the magnetic flux Phi_f through each face and
 *    advanced by the circulation of the edge EMFs (Eq. induction):
 *      dPhi_f/dt = -sum_e sigma_fe l_e E_e.
 *    The edge EMF is Contact-CT (Sect. 2.4) on the values of E . l_e: the
 *    face EMF E_f = -n x F_B (F_B the face's transverse B-flux) and the cell
 *    EMF -u x B, around the four faces of the edge, upwinded by their mass
 *    fluxes; an edge with three faces (a radial edge at a cube corner) takes
 *    the mean of their EMFs; an edge on a reflecting wall has none.
 *  - The cell-centred field is (1/V) sum_f s_f Phi_f x_f, the divergence
 *    theorem applied to B x (exact for a uniform field on planar faces).
 *  - The radial walls reflect (Table bcs): mirrored deviations with the
 *    normal velocity and field negated, a symmetry-plane flux.
 *  - Gravity is radial, g(r) per shell; the source is (rho - rho_hat) g on
 *    the momentum and rho u . g on the energy (Eq. wb2), plus heating.
 *
 * ABI layout (per patch p = 0..5, as the library's phl_sphere calls):
 *   cons[v][p][k][j][i] (v = rho, m_x, m_y, m_z, E), N x N x Nr per patch;
 *   phi_a[p][k][j][i], i = 0..N (faces normal to +alpha), N x N x Nr;
 *   phi_b[p][k][j][i], j = 0..N (faces normal to +beta);
 *   phi_r[p][k][j][i], k = 0..Nr (faces normal to +r).
 * Magnetic fluxes through the faces, each in its patch's orientation; the
 * two copies of a seam face must agree (the lower patch's is read).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define PI_S 3.14159265358979323846

void ora_riemann_up(const double *wl, const double *wr, double bn, int nspec, int solver, double mach_thr,
                    double *f, int *up);

/* patch frames: centre direction c, alpha axis a, beta axis b (a x b = c) */
static const double PC[6][3] = {{1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double PA[6][3] = {{0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 1, 0}};
static const double PB[6][3] = {{0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {0, 0, 1}, {-1, 0, 0}, {1, 0, 0}};

typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double nrm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / nrm(a)); }

struct ora_sphere {
  int N, Nr;
  double r_in, r_out, gamma, cfl, mach_thr;
  int riemann;
  double *r;                     /* Nr + 1 shell radii */
  const double *rho_c, *p_c, *rho_f, *p_f, *g_c, *heat;   /* caller's profiles (may be NULL) */
  /* angular vertices */
  int nav;
  v3 *adir;                      /* unit directions */
  int *avid;                     /* [6][N+1][N+1] -> angular vertex id */
  /* cells: [p][k][j][i] */
  long nc;
  double *vol;
  v3 *xc;
  int *cface;                    /* [nc][6] face ids in the order -a, +a, -b, +b, -r, +r */
  signed char *csign;            /* [nc][6] +1 when the face's normal points out of the cell */
  /* faces */
  long nf;
  v3 *S, *xf, *fn, *ft1, *ft2;   /* area vector, centre, unit normal and tangents */
  double *farea;
  int *fL, *fR;                  /* cells on the -n and +n side; -1 beyond a wall */
  int *fkind;                    /* 0 angular (alpha or beta) face, 1 radial face */
  int *fk;                       /* shell (angular faces) or radius index (radial faces) */
  int *fedge;                    /* [nf][4] edge ids */
  signed char *fesign;           /* [nf][4] orientation of each edge in the face's boundary */
  /* ABI face maps: per patch face -> (unique face, sign) */
  long *abi_face;                /* [n_abi_faces] */
  signed char *abi_fsign;
  char *abi_own;                 /* the copy that owns the unique face */
  long nabi_a, nabi_b, nabi_r;
  /* edges */
  long ne;
  v3 *ldir, *xe;
  double *elen;
  int *ekind;                    /* 0: four faces (Contact-CT), 1: three faces, 2: on a wall (no EMF) */
  int *ecell;                    /* [ne][4] c00, c10, c11, c01 (or three cells) */
  int *eface;                    /* [ne][4] fa0, fb1, fa1, fb0 (or three faces) */
  signed char *eside;            /* [ne][4] mass-flux sign: +1 when the face's normal runs a0/b1/a1/b0-wise */
  /* stellar EOS (ora_sphere_set_stellar).  The composition is uniform and
   * stays so (a passive scalar that starts uniform is carried uniform by a
   * conservative scheme), so it enters as constants; code density and
   * pressure are rho_u and p_u times the EOS's g/cm^3 and erg/cm^3. */
  int stellar;
  ora_cfg ecfg;
  double X[ORA_MAXSPEC];
  double rho_u, p_u;
  double *ge_c, *gc_c, *ge_f, *gc_f;   /* background gamma_e, gamma_c: shell middles (Nr), radii (Nr + 1) */
  double *T;                     /* [nc] cell temperatures (K): each inversion's guess and result */
};

/* --------------------------------------------------------------------------
 * mesh construction */

/* tan of the equiangular grid line m of N: argument (2m - N) pi / (4N),
 * exactly odd in (2m - N) and exactly +-1 at the patch edges */
static double tline(int m, int N) {
  int q = 2 * m - N;
  if (q == N) return 1.0;
  if (q == -N) return -1.0;
  double t = tan((double)(q < 0 ? -q : q) * (PI_S / (4.0 * N)));
  return q < 0 ? -t : t;
}

typedef struct { double k[3]; int id; } vkey;
static int vkey_cmp(const void *a, const void *b) {
  const vkey *x = a, *y = b;
  for (int q = 0; q < 3; ++q) {
    if (x->k[q] < y->k[q]) return -1;
    if (x->k[q] > y->k[q]) return 1;
  }
  return x->id - y->id;
}

typedef struct { long k[4]; long id; } fkey;
static int fkey_cmp(const void *a, const void *b) {
  const fkey *x = a, *y = b;
  for (int q = 0; q < 4; ++q) {
    if (x->k[q] < y->k[q]) return -1;
    if (x->k[q] > y->k[q]) return 1;
  }
  return (x->id > y->id) - (x->id < y->id);
}
static void sort4(long *a) {
  for (int i = 1; i < 4; ++i)
    for (int j = i; j > 0 && a[j - 1] > a[j]; --j) { long t = a[j]; a[j] = a[j - 1]; a[j - 1] = t; }
}

static long cid(const ora_sphere *s, int p, int i, int j, int k) {
  return (((long)p * s->Nr + k) * s->N + j) * s->N + i;
}
static int avid(const ora_sphere *s, int p, int i, int j) { return s->avid[(p * (s->N + 1) + j) * (s->N + 1) + i]; }

/* solid angle of the spherical triangle (a, b, c) (Van Oosterom & Strackee) */
static double tri_omega(v3 a, v3 b, v3 c) {
  double num = fabs(dot(a, cross(b, c)));
  double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
  return 2.0 * atan2(num, den);
}
/* vector area of the unit spherical polygon with great-circle edges, corners in
 * counter-clockwise order: (1/2) sum over edges of angle * unit normal of the
 * edge's plane */
static v3 sph_vector_area(const v3 *d, int n) {
  v3 s = mk(0, 0, 0);
  for (int q = 0; q < n; ++q) {
    v3 u = d[q], w = d[(q + 1) % n];
    v3 c = cross(u, w);
    double th = atan2(nrm(c), dot(u, w));
    s = add(s, scl(unit(c), 0.5 * th));
  }
  return s;
}

/* Radial, alpha and beta edges are identified by their vertex pair. */
typedef struct { long a, b; long id; } ekey;
static int ekey_cmp(const void *x, const void *y) {
  const ekey *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return (p->id > q->id) - (p->id < q->id);
}

static void free_all(ora_sphere *s) {
  if (!s) return;
  free(s->r); free(s->adir); free(s->avid); free(s->vol); free(s->xc); free(s->cface); free(s->csign);
  free(s->S); free(s->xf); free(s->fn); free(s->ft1); free(s->ft2); free(s->farea); free(s->fL); free(s->fR);
  free(s->fkind); free(s->fk); free(s->fedge); free(s->fesign); free(s->abi_face); free(s->abi_fsign);
  free(s->abi_own);
  free(s->ldir); free(s->xe); free(s->elen); free(s->ekind); free(s->ecell); free(s->eface); free(s->eside);
  free(s->T); free(s->ge_c); free(s->gc_c); free(s->ge_f); free(s->gc_f);
  free(s);
}

void ora_sphere_free(ora_sphere *s) { free_all(s); }

ora_sphere *ora_sphere_create(int N, int Nr, double r_in, double r_out, double gamma, const double *rho_c,
                              const double *p_c, const double *rho_f, const double *p_f, const double *g_c,
                              const double *heat, double cfl, int riemann, double mach_thr) {
  if (N < 2 || Nr < 2 || !(r_out > r_in) || !(r_in > 0.0)) return NULL;
  ora_sphere *s = calloc(1, sizeof(*s));
  s->N = N; s->Nr = Nr; s->r_in = r_in; s->r_out = r_out; s->gamma = gamma; s->cfl = cfl;
  s->riemann = riemann; s->mach_thr = mach_thr;
  s->rho_c = rho_c; s->p_c = p_c; s->rho_f = rho_f; s->p_f = p_f; s->g_c = g_c; s->heat = heat;
  s->r = malloc(sizeof(double) * (Nr + 1));
  for (int k = 0; k <= Nr; ++k) s->r[k] = r_in + (r_out - r_in) * k / Nr;

  /* (1) angular vertices: cube-surface points, deduplicated exactly */
  const int NA = 6 * (N + 1) * (N + 1);
  vkey *vk = malloc(sizeof(vkey) * NA);
  for (int p = 0; p < 6; ++p)
    for (int j = 0; j <= N; ++j)
      for (int i = 0; i <= N; ++i) {
        double ti = tline(i, N), tj = tline(j, N);
        int q = (p * (N + 1) + j) * (N + 1) + i;
        for (int c = 0; c < 3; ++c) vk[q].k[c] = PC[p][c] + ti * PA[p][c] + tj * PB[p][c];
        vk[q].id = q;
      }
  qsort(vk, NA, sizeof(vkey), vkey_cmp);
  s->avid = malloc(sizeof(int) * NA);
  s->adir = malloc(sizeof(v3) * NA);
  int nav = 0;
  for (int q = 0; q < NA; ++q) {
    if (q == 0 || memcmp(vk[q].k, vk[q - 1].k, sizeof(vk[q].k)) != 0) {
      s->adir[nav] = unit(mk(vk[q].k[0], vk[q].k[1], vk[q].k[2]));
      ++nav;
    }
    s->avid[vk[q].id] = nav - 1;
  }
  free(vk);
  s->nav = nav;   /* 6 N^2 + 2 */

  /* (2) cells */
  s->nc = 6L * N * N * Nr;
  s->vol = malloc(sizeof(double) * s->nc);
  s->xc = malloc(sizeof(v3) * s->nc);
  s->cface = malloc(sizeof(int) * 6 * s->nc);
  s->csign = malloc(6 * s->nc);
  for (int p = 0; p < 6; ++p)
    for (int k = 0; k < Nr; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          long c = cid(s, p, i, j, k);
          v3 d00 = s->adir[avid(s, p, i, j)], d10 = s->adir[avid(s, p, i + 1, j)];
          v3 d11 = s->adir[avid(s, p, i + 1, j + 1)], d01 = s->adir[avid(s, p, i, j + 1)];
          double om = tri_omega(d00, d10, d11) + tri_omega(d00, d11, d01);
          double r0 = s->r[k], r1 = s->r[k + 1];
          s->vol[c] = (r1 * r1 * r1 - r0 * r0 * r0) / 3.0 * om;
          s->xc[c] = scl(unit(add(add(d00, d10), add(d11, d01))), 0.5 * (r0 + r1));
        }

  /* (3) faces: every patch face, then deduplicated by its four 3-D vertex ids */
  const long na = 6L * Nr * N * (N + 1), nb = na, nr = 6L * (Nr + 1) * N * N;
  s->nabi_a = na; s->nabi_b = nb; s->nabi_r = nr;
  const long nall = na + nb + nr;
  fkey *fk = malloc(sizeof(fkey) * nall);
  long q = 0;
#define V3D(p, i, j, k) ((long)avid(s, p, i, j) * (Nr + 1) + (k))
  for (int p = 0; p < 6; ++p)   /* alpha faces */
    for (int k = 0; k < Nr; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i <= N; ++i, ++q) {
          long v[4] = {V3D(p, i, j, k), V3D(p, i, j + 1, k), V3D(p, i, j, k + 1), V3D(p, i, j + 1, k + 1)};
          sort4(v);
          memcpy(fk[q].k, v, sizeof(v));
          fk[q].id = q;
        }
  for (int p = 0; p < 6; ++p)   /* beta faces */
    for (int k = 0; k < Nr; ++k)
      for (int j = 0; j <= N; ++j)
        for (int i = 0; i < N; ++i, ++q) {
          long v[4] = {V3D(p, i, j, k), V3D(p, i + 1, j, k), V3D(p, i, j, k + 1), V3D(p, i + 1, j, k + 1)};
          sort4(v);
          memcpy(fk[q].k, v, sizeof(v));
          fk[q].id = q;
        }
  for (int p = 0; p < 6; ++p)   /* radial faces */
    for (int k = 0; k <= Nr; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i, ++q) {
          long v[4] = {V3D(p, i, j, k), V3D(p, i + 1, j, k), V3D(p, i, j + 1, k), V3D(p, i + 1, j + 1, k)};
          sort4(v);
          memcpy(fk[q].k, v, sizeof(v));
          fk[q].id = q;
        }
  qsort(fk, nall, sizeof(fkey), fkey_cmp);
  /* unique faces in key order; the first (lowest ABI index, so lowest patch)
   * occurrence is the face's owner and sets its orientation */
  long *owner = malloc(sizeof(long) * nall);
  long nf = 0;
  s->abi_face = malloc(sizeof(long) * nall);
  s->abi_fsign = malloc(nall);
  s->abi_own = calloc(nall, 1);
  for (long t = 0; t < nall; ++t) {
    if (t == 0 || memcmp(fk[t].k, fk[t - 1].k, sizeof(fk[t].k)) != 0) owner[nf++] = fk[t].id;
    s->abi_face[fk[t].id] = nf - 1;
  }
  free(fk);
  s->nf = nf;
  s->S = malloc(sizeof(v3) * nf); s->xf = malloc(sizeof(v3) * nf); s->fn = malloc(sizeof(v3) * nf);
  s->ft1 = malloc(sizeof(v3) * nf); s->ft2 = malloc(sizeof(v3) * nf); s->farea = malloc(sizeof(double) * nf);
  s->fL = malloc(sizeof(int) * nf); s->fR = malloc(sizeof(int) * nf); s->fkind = malloc(sizeof(int) * nf);
  s->fk = malloc(sizeof(int) * nf);
  for (long f = 0; f < nf; ++f) { s->fL[f] = -1; s->fR[f] = -1; }
  /* geometry of an ABI face in its patch's orientation, and its two cells */
  for (long t = 0; t < nall; ++t) {
    int p, i, j, k, kind;   /* kind 0 alpha, 1 beta, 2 radial */
    long u = t;
    if (u < na) { kind = 0; i = u % (N + 1); u /= (N + 1); j = u % N; u /= N; k = u % Nr; p = (int)(u / Nr); }
    else if ((u -= na) < nb) { kind = 1; i = u % N; u /= N; j = u % (N + 1); u /= (N + 1); k = u % Nr; p = (int)(u / Nr); }
    else { u -= nb; kind = 2; i = u % N; u /= N; j = u % N; u /= N; k = u % (Nr + 1); p = (int)(u / (Nr + 1)); }
    v3 S, xf;
    int lo, hi;   /* cells on the -n and +n side in this patch (-1 outside it) */
    if (kind == 2) {
      v3 d[4] = {s->adir[avid(s, p, i, j)], s->adir[avid(s, p, i + 1, j)], s->adir[avid(s, p, i + 1, j + 1)],
                 s->adir[avid(s, p, i, j + 1)]};
      double rk = s->r[k];
      S = scl(sph_vector_area(d, 4), rk * rk);
      xf = scl(unit(add(add(d[0], d[1]), add(d[2], d[3]))), rk);
      lo = k > 0 ? (int)cid(s, p, i, j, k - 1) : -1;
      hi = k < Nr ? (int)cid(s, p, i, j, k) : -1;
    } else {
      v3 d0, d1, ax;
      if (kind == 0) { d0 = s->adir[avid(s, p, i, j)]; d1 = s->adir[avid(s, p, i, j + 1)]; ax = mk(PA[p][0], PA[p][1], PA[p][2]); }
      else { d0 = s->adir[avid(s, p, i, j)]; d1 = s->adir[avid(s, p, i + 1, j)]; ax = mk(PB[p][0], PB[p][1], PB[p][2]); }
      v3 n = unit(cross(d0, d1));
      if (dot(n, ax) < 0.0) n = scl(n, -1.0);
      double th = atan2(nrm(cross(d0, d1)), dot(d0, d1));
      double r0 = s->r[k], r1 = s->r[k + 1];
      S = scl(n, 0.5 * (r1 * r1 - r0 * r0) * th);
      xf = scl(unit(add(d0, d1)), 0.5 * (r0 + r1));
      if (kind == 0) { lo = i > 0 ? (int)cid(s, p, i - 1, j, k) : -1; hi = i < N ? (int)cid(s, p, i, j, k) : -1; }
      else { lo = j > 0 ? (int)cid(s, p, i, j - 1, k) : -1; hi = j < N ? (int)cid(s, p, i, j, k) : -1; }
    }
    long f = s->abi_face[t];
    if (owner[f] == t) {   /* the owner's orientation */
      s->abi_own[t] = 1;
      s->S[f] = S;
      s->xf[f] = xf;
      s->fkind[f] = kind == 2;
      s->fk[f] = k;
      s->abi_fsign[t] = 1;
      if (lo >= 0) s->fL[f] = lo;
      if (hi >= 0) s->fR[f] = hi;
    }
  }
  /* the other side of seam faces, and the copies' signs */
  for (long t = 0; t < nall; ++t) {
    long f = s->abi_face[t];
    if (owner[f] == t) continue;
    int p, i, j, k, kind;
    long u = t;
    if (u < na) { kind = 0; i = u % (N + 1); u /= (N + 1); j = u % N; u /= N; k = u % Nr; p = (int)(u / Nr); }
    else if ((u -= na) < nb) { kind = 1; i = u % N; u /= N; j = u % (N + 1); u /= (N + 1); k = u % Nr; p = (int)(u / Nr); }
    else { u -= nb; kind = 2; i = u % N; u /= N; j = u % N; u /= N; k = u % (Nr + 1); p = (int)(u / (Nr + 1)); }
    /* this patch's normal direction for the face */
    v3 ax = kind == 0 ? mk(PA[p][0], PA[p][1], PA[p][2]) : mk(PB[p][0], PB[p][1], PB[p][2]);
    int sg = dot(s->S[f], ax) > 0.0 ? 1 : -1;
    s->abi_fsign[t] = (signed char)sg;
    int lo, hi;
    if (kind == 0) { lo = i > 0 ? (int)cid(s, p, i - 1, j, k) : -1; hi = i < N ? (int)cid(s, p, i, j, k) : -1; }
    else { lo = j > 0 ? (int)cid(s, p, i, j - 1, k) : -1; hi = j < N ? (int)cid(s, p, i, j, k) : -1; }
    int in = lo >= 0 ? lo : hi;   /* this patch's cell at the seam */
    /* in this patch's orientation the cell is on the -n side if lo >= 0 */
    int on_minus = (lo >= 0) == (sg > 0);
    if (on_minus) s->fL[f] = in; else s->fR[f] = in;
  }
  free(owner);
  for (long f = 0; f < nf; ++f) {
    s->farea[f] = nrm(s->S[f]);
    v3 n = scl(s->S[f], 1.0 / s->farea[f]);
    s->fn[f] = n;
    /* tangent basis: the Cartesian axis least aligned with n */
    double an[3] = {fabs(n.x), fabs(n.y), fabs(n.z)};
    int m = 0;
    if (an[1] < an[m]) m = 1;
    if (an[2] < an[m]) m = 2;
    v3 e = mk(m == 0, m == 1, m == 2);
    v3 t1 = unit(cross(e, n));
    s->ft1[f] = t1;
    s->ft2[f] = cross(n, t1);
  }
  /* cells' faces and signs */
  for (int p = 0; p < 6; ++p)
    for (int k = 0; k < Nr; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          long c = cid(s, p, i, j, k);
          long t6[6] = {((((long)p * Nr + k) * N + j) * (N + 1) + i), ((((long)p * Nr + k) * N + j) * (N + 1) + i + 1),
                        na + ((((long)p * Nr + k) * (N + 1) + j) * N + i), na + ((((long)p * Nr + k) * (N + 1) + j + 1) * N + i),
                        na + nb + ((((long)p * (Nr + 1) + k) * N + j) * N + i),
                        na + nb + ((((long)p * (Nr + 1) + k + 1) * N + j) * N + i)};
          for (int m = 0; m < 6; ++m) {
            long f = s->abi_face[t6[m]];
            s->cface[6 * c + m] = (int)f;
            s->csign[6 * c + m] = s->fL[f] == c ? 1 : -1;
          }
        }

  /* (4) edges: radial (vertex, k) and angular (vertex pair, k); the face's
   * four edges in its ABI patch order */
  const long nre = (long)nav * Nr;            /* radial edges */
  long nang = 0;                              /* angular edge keys collected from the faces */
  ekey *ek = malloc(sizeof(ekey) * (size_t)(4 * nf));
  /* angular edges: key (min vertex, max vertex) of the 3-D vertex ids at one radius */
  s->fedge = malloc(sizeof(int) * 4 * nf);
  s->fesign = malloc(4 * nf);
  /* walk the patch faces once per unique face, recording its four edges */
  char *done = calloc(nf, 1);
  for (long t = 0; t < nall; ++t) {
    long f = s->abi_face[t];
    if (done[f]) continue;
    done[f] = 1;
    int p, i, j, k, kind;
    long u = t;
    if (u < na) { kind = 0; i = u % (N + 1); u /= (N + 1); j = u % N; u /= N; k = u % Nr; p = (int)(u / Nr); }
    else if ((u -= na) < nb) { kind = 1; i = u % N; u /= N; j = u % (N + 1); u /= (N + 1); k = u % Nr; p = (int)(u / Nr); }
    else { u -= nb; kind = 2; i = u % N; u /= N; j = u % N; u /= N; k = u % (Nr + 1); p = (int)(u / (Nr + 1)); }
    long a0, a1, e[4][2];
    int rad[4];
    if (kind == 2) {   /* four angular edges at radius k */
      long v00 = avid(s, p, i, j), v10 = avid(s, p, i + 1, j), v11 = avid(s, p, i + 1, j + 1), v01 = avid(s, p, i, j + 1);
      long vv[4][2] = {{v00, v10}, {v10, v11}, {v11, v01}, {v01, v00}};
      for (int m = 0; m < 4; ++m) { e[m][0] = vv[m][0]; e[m][1] = vv[m][1]; rad[m] = 0; }
    } else {           /* two radial edges and two angular edges */
      if (kind == 0) { a0 = avid(s, p, i, j); a1 = avid(s, p, i, j + 1); }
      else { a0 = avid(s, p, i, j); a1 = avid(s, p, i + 1, j); }
      e[0][0] = a0; e[0][1] = a1; rad[0] = 0;            /* at radius k */
      e[1][0] = a1; e[1][1] = -1; rad[1] = 1;            /* radial at a1 */
      e[2][0] = a0; e[2][1] = a1; rad[2] = 2;            /* at radius k + 1 */
      e[3][0] = a0; e[3][1] = -1; rad[3] = 1;            /* radial at a0 */
    }
    for (int m = 0; m < 4; ++m) {
      ekey *x = &ek[nang];
      if (rad[m] == 1) { x->a = -1 - e[m][0]; x->b = k; }   /* radial edges: negative first key */
      else {
        long lo = e[m][0] < e[m][1] ? e[m][0] : e[m][1], hi = e[m][0] < e[m][1] ? e[m][1] : e[m][0];
        int kk = kind == 2 ? k : (rad[m] == 2 ? k + 1 : k);
        x->a = lo * (Nr + 1) + kk;
        x->b = hi;
      }
      x->id = 4 * f + m;
      ++nang;
    }
  }
  free(done);
  qsort(ek, nang, sizeof(ekey), ekey_cmp);
  long ne = 0;
  for (long t = 0; t < nang; ++t) {
    if (t == 0 || ek[t].a != ek[t - 1].a || ek[t].b != ek[t - 1].b) ++ne;
    s->fedge[ek[t].id] = (int)(ne - 1);
  }
  (void)nre;
  s->ne = ne;
  s->ldir = malloc(sizeof(v3) * ne); s->xe = malloc(sizeof(v3) * ne); s->elen = malloc(sizeof(double) * ne);
  s->ekind = malloc(sizeof(int) * ne);
  s->ecell = malloc(sizeof(int) * 4 * ne); s->eface = malloc(sizeof(int) * 4 * ne); s->eside = malloc(4 * ne);
  {
    long e = -1;
    for (long t = 0; t < nang; ++t) {
      if (!(t == 0 || ek[t].a != ek[t - 1].a || ek[t].b != ek[t - 1].b)) continue;
      ++e;
      if (ek[t].a < 0) {   /* radial edge at angular vertex -1 - a, from r_k to r_(k+1) */
        long v = -1 - ek[t].a;
        int k = (int)ek[t].b;
        s->ldir[e] = s->adir[v];
        s->xe[e] = scl(s->adir[v], 0.5 * (s->r[k] + s->r[k + 1]));
        s->elen[e] = s->r[k + 1] - s->r[k];
      } else {             /* angular edge between two angular vertices at radius kk */
        long lo = ek[t].a / (Nr + 1);
        int kk = (int)(ek[t].a % (Nr + 1));
        long hi = ek[t].b;
        v3 u = s->adir[lo], w = s->adir[hi];
        double th = atan2(nrm(cross(u, w)), dot(u, w));
        s->ldir[e] = unit(sub(w, u));   /* the chord: parallel to the arc at its midpoint */
        s->xe[e] = scl(unit(add(u, w)), s->r[kk]);
        s->elen[e] = s->r[kk] * th;
      }
    }
  }
  free(ek);
  /* orientation of each edge in its face's boundary (counter-clockwise about n) */
  for (long f = 0; f < nf; ++f)
    for (int m = 0; m < 4; ++m) {
      int e = s->fedge[4 * f + m];
      v3 tang = cross(s->fn[f], sub(s->xe[e], s->xf[f]));
      s->fesign[4 * f + m] = dot(s->ldir[e], tang) > 0.0 ? 1 : -1;
    }
  /* cells and faces around each edge */
  int *nfe = calloc(ne, sizeof(int)), *fel = malloc(sizeof(int) * 4 * ne);
  for (long f = 0; f < nf; ++f)
    for (int m = 0; m < 4; ++m) {
      int e = s->fedge[4 * f + m];
      if (nfe[e] < 4) fel[4 * e + nfe[e]] = (int)f;
      nfe[e]++;
    }
  for (long e = 0; e < ne; ++e) {
    int nfc = nfe[e];
    int *F = &fel[4 * e];
    /* an edge on a wall: one of its faces is a radial face without a cell on one side */
    int wall = 0;
    for (int m = 0; m < nfc && m < 4; ++m) if (s->fL[F[m]] < 0 || s->fR[F[m]] < 0) wall = 1;
    for (int m = 0; m < 4; ++m) { s->ecell[4 * e + m] = -1; s->eface[4 * e + m] = -1; s->eside[4 * e + m] = 0; }
    if (wall) { s->ekind[e] = 2; continue; }
    if (nfc == 3) {
      s->ekind[e] = 1;
      for (int m = 0; m < 3; ++m) s->eface[4 * e + m] = F[m];
      continue;
    }
    s->ekind[e] = 0;
    /* the four cells: each face gives two; order them cyclically */
    int cells[4], ncl = 0;
    for (int m = 0; m < 4; ++m) {
      int c2[2] = {s->fL[F[m]], s->fR[F[m]]};
      for (int h = 0; h < 2; ++h) {
        int seen = 0;
        for (int q2 = 0; q2 < ncl; ++q2) seen |= cells[q2] == c2[h];
        if (!seen && ncl < 4) cells[ncl++] = c2[h];
      }
    }
    /* face between two cells (or -1) */
    #define FACE_BETWEEN(x, y, out) do { out = -1; for (int mm = 0; mm < 4; ++mm) { int a_ = s->fL[F[mm]], b_ = s->fR[F[mm]]; if ((a_ == (x) && b_ == (y)) || (a_ == (y) && b_ == (x))) out = F[mm]; } } while (0)
    int c00 = cells[0], X = -1, Y = -1;
    for (int q2 = 1; q2 < 4; ++q2) {
      int fb;
      FACE_BETWEEN(c00, cells[q2], fb);
      if (fb >= 0) { if (X < 0) X = cells[q2]; else Y = cells[q2]; }
    }
    int c11 = -1;
    for (int q2 = 1; q2 < 4; ++q2) if (cells[q2] != X && cells[q2] != Y) c11 = cells[q2];
    v3 da = sub(s->xc[X], s->xc[c00]), db = sub(s->xc[Y], s->xc[c00]);
    int c10 = X, c01 = Y;
    if (dot(s->ldir[e], cross(da, db)) < 0.0) { c10 = Y; c01 = X; }
    int fa0, fb1, fa1, fb0;
    FACE_BETWEEN(c00, c10, fa0);
    FACE_BETWEEN(c10, c11, fb1);
    FACE_BETWEEN(c01, c11, fa1);
    FACE_BETWEEN(c00, c01, fb0);
    #undef FACE_BETWEEN
    int cc[4] = {c00, c10, c11, c01}, ff[4] = {fa0, fb1, fa1, fb0};
    int from[4] = {c00, c10, c01, c00};   /* mass-flux sign: positive from this cell across the face */
    for (int m = 0; m < 4; ++m) {
      s->ecell[4 * e + m] = cc[m];
      s->eface[4 * e + m] = ff[m];
      s->eside[4 * e + m] = s->fL[ff[m]] == from[m] ? 1 : -1;
    }
  }
  free(nfe);
  free(fel);
  return s;
}

long ora_sphere_ncells(const ora_sphere *s) { return s->nc; }
long ora_sphere_nfaces(const ora_sphere *s) { return s->nf; }
long ora_sphere_nedges(const ora_sphere *s) { return s->ne; }
long ora_sphere_nabi_faces(const ora_sphere *s) { return s->nabi_a + s->nabi_b + s->nabi_r; }

int ora_sphere_geometry(const ora_sphere *s, double *vol, double *xc, double *S, double *xf, double *csum) {
  for (long c = 0; c < s->nc; ++c) {
    if (vol) vol[c] = s->vol[c];
    if (xc) { xc[3 * c] = s->xc[c].x; xc[3 * c + 1] = s->xc[c].y; xc[3 * c + 2] = s->xc[c].z; }
    if (csum) {   /* sum of outward area vectors of the cell */
      v3 t = mk(0, 0, 0);
      for (int m = 0; m < 6; ++m) t = add(t, scl(s->S[s->cface[6 * c + m]], s->csign[6 * c + m]));
      csum[3 * c] = t.x; csum[3 * c + 1] = t.y; csum[3 * c + 2] = t.z;
    }
  }
  for (long f = 0; f < s->nf; ++f) {
    if (S) { S[3 * f] = s->S[f].x; S[3 * f + 1] = s->S[f].y; S[3 * f + 2] = s->S[f].z; }
    if (xf) { xf[3 * f] = s->xf[f].x; xf[3 * f + 1] = s->xf[f].y; xf[3 * f + 2] = s->xf[f].z; }
  }
  return 0;
}

/* --------------------------------------------------------------------------
 * the stage */

/* deviations: drho, u(3), B(3), dP, dgamma_e, dgamma_c */
enum { SW_RHO = 0, SW_U = 1, SW_B = 4, SW_P = 7, SW_GE = 8, SW_GC = 9, SW_N = 10 };

static double bg_rho_cell(const ora_sphere *s, int k) { return s->rho_c ? s->rho_c[k] : 0.0; }
static double bg_p_cell(const ora_sphere *s, int k) { return s->p_c ? s->p_c[k] : 0.0; }
/* the background's gamma_e, gamma_c at shell k's middle (face 0) or radius k (face 1) */
static double bg_ge(const ora_sphere *s, int k, int face) {
  const double *a = face ? s->ge_f : s->ge_c;
  return s->stellar && a ? a[k] : s->gamma;
}
static double bg_gc(const ora_sphere *s, int k, int face) {
  const double *a = face ? s->gc_f : s->gc_c;
  return s->stellar && a ? a[k] : s->gamma;
}

static void load_phi(const ora_sphere *s, const double *pa, const double *pb, const double *pr, double *phi);

/* T with P_EoS(rho, T) = P at fixed rho (EOS units): Newton on P from T,
 * bracketed in [1e7, 1e10] K */
static int p_to_T(const ora_cfg *cfg, double rho, double P, const double *X, double *T) {
  double lo = 1e7, hi = 1e10, t = *T > lo && *T < hi ? *T : 1e9;
  for (int it = 0; it < 200; ++it) {
    double Pt, e, cv, dPdr, dPdT, ge, gc;
    if (ora_eos_rt(cfg, rho, t, X, &Pt, &e, &cv, &dPdr, &dPdT, &ge, &gc)) return -1;
    double dp = P - Pt;
    if (fabs(dp) <= 1e-14 * P) { *T = t; return 0; }
    if (dp > 0.0) lo = t; else hi = t;
    double tn = t + dp / dPdT;
    t = tn > lo && tn < hi ? tn : 0.5 * (lo + hi);
  }
  return -1;
}

int ora_sphere_set_stellar(ora_sphere *s, const ora_cfg *eos, const double *X, double rho_u, double p_u) {
  if (!s || !eos || !eos->eos_table || !X || !(rho_u > 0.0) || !(p_u > 0.0)) return -1;
  if (eos->nspec < 1 || eos->nspec > ORA_MAXSPEC) return -1;
  s->stellar = 1;
  s->ecfg = *eos;
  s->ecfg.eos = ORA_EOS_STELLAR;
  for (int l = 0; l < eos->nspec; ++l) s->X[l] = X[l];
  s->rho_u = rho_u; s->p_u = p_u;
  if (!s->T) s->T = calloc(s->nc, sizeof(double));
  if (s->rho_c) {   /* the background's gamma_e, gamma_c from its (rho_hat, P_hat) */
    const int Nr = s->Nr;
    double **dst[4] = {&s->ge_c, &s->gc_c, &s->ge_f, &s->gc_f};
    for (int q = 0; q < 4; ++q) { free(*dst[q]); *dst[q] = malloc(sizeof(double) * (Nr + 1)); }
    for (int face = 0; face < 2; ++face) {
      double T = 1e9;
      for (int k = 0; k < Nr + face; ++k) {
        double rho = (face ? s->rho_f[k] : s->rho_c[k]) * rho_u, P = (face ? s->p_f[k] : s->p_c[k]) * p_u;
        double Pt, e, cv, dPdr, dPdT, ge, gc;
        if (p_to_T(&s->ecfg, rho, P, s->X, &T) ||
            ora_eos_rt(&s->ecfg, rho, T, s->X, &Pt, &e, &cv, &dPdr, &dPdT, &ge, &gc))
          return -1;
        (face ? s->ge_f : s->ge_c)[k] = ge;
        (face ? s->gc_f : s->gc_c)[k] = gc;
      }
    }
  }
  return 0;
}

static v3 cell_field(const ora_sphere *s, const double *phi, long c) {
  v3 Bc = mk(0, 0, 0);
  for (int m = 0; m < 6; ++m) {
    int f = s->cface[6 * c + m];
    Bc = add(Bc, scl(s->xf[f], s->csign[6 * c + m] * phi[f]));
  }
  return scl(Bc, 1.0 / s->vol[c]);
}

int ora_sphere_from_prims(ora_sphere *s, const double *rho, const double *vel, const double *P, const double *pa,
                          const double *pb, const double *pr, double *cons) {
  if (!s || !rho || !vel || !P || !pa || !pb || !pr || !cons) return -1;
  const long nc = s->nc;
  double *phi = malloc(sizeof(double) * s->nf);
  load_phi(s, pa, pb, pr, phi);
  int rc = 0;
  for (long c = 0; c < nc && !rc; ++c) {
    v3 u = mk(vel[3 * c], vel[3 * c + 1], vel[3 * c + 2]), Bc = cell_field(s, phi, c);
    double eden;   /* rho e_int */
    if (s->stellar) {
      double T = s->T[c] > 0.0 ? s->T[c] : 1e9, Pt, e, cv, dPdr, dPdT, ge, gc;
      if (p_to_T(&s->ecfg, rho[c] * s->rho_u, P[c] * s->p_u, s->X, &T) ||
          ora_eos_rt(&s->ecfg, rho[c] * s->rho_u, T, s->X, &Pt, &e, &cv, &dPdr, &dPdT, &ge, &gc)) {
        rc = -3;
        break;
      }
      s->T[c] = T;
      eden = rho[c] * e * (s->rho_u / s->p_u);
    } else {
      eden = P[c] / (s->gamma - 1.0);
    }
    cons[c] = rho[c];
    cons[nc + c] = rho[c] * u.x; cons[2 * nc + c] = rho[c] * u.y; cons[3 * nc + c] = rho[c] * u.z;
    cons[4 * nc + c] = eden + 0.5 * rho[c] * dot(u, u) + 0.5 * dot(Bc, Bc);
  }
  free(phi);
  return rc;
}

int ora_sphere_set_T(ora_sphere *s, const double *T) {
  if (!s || !s->T || !T) return -1;
  memcpy(s->T, T, sizeof(double) * s->nc);
  return 0;
}

int ora_sphere_get_T(const ora_sphere *s, double *T) {
  if (!s || !s->T || !T) return -1;
  memcpy(T, s->T, sizeof(double) * s->nc);
  return 0;
}
static int cell_k(const ora_sphere *s, long c) { return (int)((c / ((long)s->N * s->N)) % s->Nr); }

/* Load (ABI) face fluxes into the unique faces: the owner's copy. */
static void load_phi(const ora_sphere *s, const double *pa, const double *pb, const double *pr, double *phi) {
  const long na = s->nabi_a, nb = s->nabi_b, nall = na + nb + s->nabi_r;
  for (long t = 0; t < nall; ++t) {
    if (!s->abi_own[t]) continue;   /* the owner's copy */
    long f = s->abi_face[t];
    double v = t < na ? pa[t] : (t < na + nb ? pb[t - na] : pr[t - na - nb]);
    phi[f] = v;
  }
}
static void store_phi(const ora_sphere *s, const double *phi, double *pa, double *pb, double *pr) {
  const long na = s->nabi_a, nb = s->nabi_b, nall = na + nb + s->nabi_r;
  for (long t = 0; t < nall; ++t) {
    double v = s->abi_fsign[t] * phi[s->abi_face[t]];
    if (t < na) pa[t] = v; else if (t < na + nb) pb[t - na] = v; else pr[t - na - nb] = v;
  }
}

/* primitive deviations of every cell from the conserved state and face fluxes */
static int sphere_prims(const ora_sphere *s, const double *cons, const double *phi, double *W) {
  const long nc = s->nc;
  int rc = 0;
  for (long c = 0; c < nc; ++c) {
    v3 Bc = cell_field(s, phi, c);
    double rho = cons[c];
    v3 u = mk(cons[nc + c] / rho, cons[2 * nc + c] / rho, cons[3 * nc + c] / rho);
    double eden = cons[4 * nc + c] - 0.5 * rho * dot(u, u) - 0.5 * dot(Bc, Bc);   /* rho e_int */
    double P, ge = s->gamma, gc = s->gamma;
    if (!s->stellar) {
      P = (s->gamma - 1.0) * eden;
    } else {   /* the EOS in its own units: e_int per gram, T by Newton from the cell's last T */
      double Pe;
      int it;
      if (!(rho > 0.0) || ora_eos_invert(&s->ecfg, rho * s->rho_u, eden / rho * (s->p_u / s->rho_u), s->X, &s->T[c],
                                         &Pe, &ge, &gc, &it)) {
        rc = -3;
        continue;
      }
      P = Pe / s->p_u;
    }
    if (!(rho > 0.0) || !(P > 0.0)) rc = -2;
    int k = cell_k(s, c);
    double *w = &W[SW_N * c];
    w[SW_RHO] = rho - bg_rho_cell(s, k);
    w[SW_U] = u.x; w[SW_U + 1] = u.y; w[SW_U + 2] = u.z;
    w[SW_B] = Bc.x; w[SW_B + 1] = Bc.y; w[SW_B + 2] = Bc.z;
    w[SW_P] = P - bg_p_cell(s, k);
    w[SW_GE] = ge - bg_ge(s, k, 0);
    w[SW_GC] = gc - bg_gc(s, k, 0);
  }
  return rc;
}

/* deviations mirrored at a wall with unit normal n: u_n and B_n negated */
static void mirror(const double *w, v3 n, double *o) {
  memcpy(o, w, sizeof(double) * SW_N);
  v3 u = mk(w[SW_U], w[SW_U + 1], w[SW_U + 2]), b = mk(w[SW_B], w[SW_B + 1], w[SW_B + 2]);
  u = sub(u, scl(n, 2.0 * dot(u, n)));
  b = sub(b, scl(n, 2.0 * dot(b, n)));
  o[SW_U] = u.x; o[SW_U + 1] = u.y; o[SW_U + 2] = u.z;
  o[SW_B] = b.x; o[SW_B + 1] = b.y; o[SW_B + 2] = b.z;
}

/* the neighbour of cell c across the face opposite to face f (or -1 at a wall) */
static int across_opposite(const ora_sphere *s, int c, int f) {
  int m = -1;
  for (int q = 0; q < 6; ++q) if (s->cface[6 * c + q] == f) m = q;
  int g = s->cface[6 * c + (m ^ 1)];
  return s->fL[g] == c ? s->fR[g] : s->fL[g];
}

static double vl(double a, double b, double c) {
  double dm = b - a, dp = c - b;
  if (dm * dp > 0.0) return 2.0 * dm * dp / (dm + dp);
  return 0.0;
}

/* fluxes (integrated over the face) FC[f][5] (rho, m(3), E), face EMF vector
 * EF[f][3] and the face's contact direction UP[f] */
static int sphere_fluxes(const ora_sphere *s, const double *W, const double *phi, double *FC, double *EF, int *UP) {
  int rc = 0;
  for (long f = 0; f < s->nf; ++f) {
    int L = s->fL[f], R = s->fR[f];
    v3 n = s->fn[f], t1 = s->ft1[f], t2 = s->ft2[f];
    double wL[SW_N], wR[SW_N], wLL[SW_N], wRR[SW_N];
    const int wall = L < 0 || R < 0;
    if (!wall) {
      int LL = across_opposite(s, L, (int)f), RR = across_opposite(s, R, (int)f);
      memcpy(wL, &W[SW_N * L], sizeof(wL));
      memcpy(wR, &W[SW_N * R], sizeof(wR));
      if (LL >= 0) memcpy(wLL, &W[SW_N * LL], sizeof(wLL));
      else {   /* L touches a wall on its far side: the mirror of L across that wall */
        int g = s->cface[6 * L + 0];
        for (int q = 0; q < 6; ++q) if (s->cface[6 * L + q] == (int)f) g = s->cface[6 * L + (q ^ 1)];
        mirror(wL, s->fn[g], wLL);
      }
      if (RR >= 0) memcpy(wRR, &W[SW_N * RR], sizeof(wRR));
      else {
        int g = s->cface[6 * R + 0];
        for (int q = 0; q < 6; ++q) if (s->cface[6 * R + q] == (int)f) g = s->cface[6 * R + (q ^ 1)];
        mirror(wR, s->fn[g], wRR);
      }
    } else {   /* a wall face: the ghost side mirrors the cell (and its neighbour) */
      int in = L >= 0 ? L : R;
      int nb = across_opposite(s, in, (int)f);
      double wi[SW_N], wn[SW_N], mi[SW_N], mn[SW_N];
      memcpy(wi, &W[SW_N * in], sizeof(wi));
      memcpy(wn, &W[SW_N * nb], sizeof(wn));
      mirror(wi, n, mi);
      mirror(wn, n, mn);
      if (L >= 0) { memcpy(wL, wi, sizeof(wL)); memcpy(wLL, wn, sizeof(wLL)); memcpy(wR, mi, sizeof(wR)); memcpy(wRR, mn, sizeof(wRR)); }
      else { memcpy(wR, wi, sizeof(wR)); memcpy(wRR, wn, sizeof(wRR)); memcpy(wL, mi, sizeof(wL)); memcpy(wLL, mn, sizeof(wLL)); }
    }
    double ql[SW_N], qr[SW_N];
    for (int v = 0; v < SW_N; ++v) {
      ql[v] = wL[v] + 0.5 * vl(wLL[v], wL[v], wR[v]);
      qr[v] = wR[v] - 0.5 * vl(wL[v], wR[v], wRR[v]);
    }
    /* the face's background: radial faces at their radius, angular faces at the shell's middle */
    double brho, bp;
    if (s->fkind[f]) { brho = s->rho_f ? s->rho_f[s->fk[f]] : 0.0; bp = s->p_f ? s->p_f[s->fk[f]] : 0.0; }
    else { brho = bg_rho_cell(s, s->fk[f]); bp = bg_p_cell(s, s->fk[f]); }
    const double bge = bg_ge(s, s->fk[f], s->fkind[f]), bgc = bg_gc(s, s->fk[f], s->fkind[f]);
    double rl[9], rr[9];
    v3 ul = mk(ql[SW_U], ql[SW_U + 1], ql[SW_U + 2]), ur = mk(qr[SW_U], qr[SW_U + 1], qr[SW_U + 2]);
    v3 bl = mk(ql[SW_B], ql[SW_B + 1], ql[SW_B + 2]), br = mk(qr[SW_B], qr[SW_B + 1], qr[SW_B + 2]);
    rl[0] = ql[SW_RHO] + brho; rr[0] = qr[SW_RHO] + brho;
    rl[1] = dot(ul, n); rl[2] = dot(ul, t1); rl[3] = dot(ul, t2);
    rr[1] = dot(ur, n); rr[2] = dot(ur, t1); rr[3] = dot(ur, t2);
    rl[4] = dot(bl, t1); rl[5] = dot(bl, t2);
    rr[4] = dot(br, t1); rr[5] = dot(br, t2);
    rl[6] = ql[SW_P] + bp; rr[6] = qr[SW_P] + bp;
    rl[7] = ql[SW_GE] + bge; rl[8] = ql[SW_GC] + bgc;
    rr[7] = qr[SW_GE] + bge; rr[8] = qr[SW_GC] + bgc;
    if (!(rl[0] > 0.0 && rr[0] > 0.0 && rl[6] > 0.0 && rr[6] > 0.0)) rc = -2;
    double bn = phi[f] / s->farea[f];
    double fq[7], fh[7];
    int up;
    ora_riemann_up(rl, rr, bn, 0, s->riemann, s->mach_thr, fq, &up);
    if (s->rho_c) {   /* the flux of the face's hydrostatic state, F(W_hat, W_hat) */
      double wh[9] = {brho, 0, 0, 0, 0, 0, bp, bge, bgc};
      ora_riemann(wh, wh, 0.0, 0, s->riemann, s->mach_thr, fh);
      for (int q = 0; q < 7; ++q) fq[q] -= fh[q];
    }
    if (wall) {   /* a symmetry plane: only the normal-momentum flux survives */
      for (int q = 0; q < 7; ++q) if (q != 1) fq[q] = 0.0;
      up = 0;
    }
    double A = s->farea[f];
    v3 fm = add(add(scl(n, fq[1]), scl(t1, fq[2])), scl(t2, fq[3]));
    v3 fb = add(scl(t1, fq[5]), scl(t2, fq[6]));
    FC[5 * f + 0] = A * fq[0];
    FC[5 * f + 1] = A * fm.x; FC[5 * f + 2] = A * fm.y; FC[5 * f + 3] = A * fm.z;
    FC[5 * f + 4] = A * fq[4];
    v3 ef = scl(cross(n, fb), -1.0);   /* E_f = -n x F_B */
    EF[3 * f] = ef.x; EF[3 * f + 1] = ef.y; EF[3 * f + 2] = ef.z;
    UP[f] = up;
  }
  return rc;
}

/* edge EMFs E . l (line averages along each edge) */
static void sphere_emfs(const ora_sphere *s, const double *W, const double *EF, const int *UP, double *EE) {
  for (long e = 0; e < s->ne; ++e) {
    if (s->ekind[e] == 2) { EE[e] = 0.0; continue; }
    v3 l = s->ldir[e];
    if (s->ekind[e] == 1) {
      double t = 0.0;
      for (int m = 0; m < 3; ++m) {
        int f = s->eface[4 * e + m];
        t += dot(mk(EF[3 * f], EF[3 * f + 1], EF[3 * f + 2]), l);
      }
      EE[e] = t / 3.0;
      continue;
    }
    double Ec[4], Ef[4];
    int ms[4];
    for (int m = 0; m < 4; ++m) {
      int c = s->ecell[4 * e + m], f = s->eface[4 * e + m];
      const double *w = &W[SW_N * c];
      v3 u = mk(w[SW_U], w[SW_U + 1], w[SW_U + 2]), b = mk(w[SW_B], w[SW_B + 1], w[SW_B + 2]);
      Ec[m] = dot(scl(cross(u, b), -1.0), l);
      Ef[m] = dot(mk(EF[3 * f], EF[3 * f + 1], EF[3 * f + 2]), l);
      ms[m] = s->eside[4 * e + m] * UP[f];
    }
    /* cells c00, c10, c11, c01; faces a0 (c00|c10), b1 (c10|c11), a1 (c01|c11), b0 (c00|c01) */
    double E00 = Ec[0], E10 = Ec[1], E11 = Ec[2], E01 = Ec[3];
    double Ea0 = Ef[0], Eb1 = Ef[1], Ea1 = Ef[2], Eb0 = Ef[3];
    int ma0 = ms[0], mb1 = ms[1], ma1 = ms[2], mb0 = ms[3];
    double lo_l = Eb0 - E00, lo_r = Eb1 - E10;
    double up_l = E01 - Eb0, up_r = E11 - Eb1;
    double dlo = ma0 > 0 ? lo_l : (ma0 < 0 ? lo_r : 0.5 * (lo_l + lo_r));
    double dup = ma1 > 0 ? up_l : (ma1 < 0 ? up_r : 0.5 * (up_l + up_r));
    double le_d = Ea0 - E00, le_u = Ea1 - E01;
    double ri_d = E10 - Ea0, ri_u = E11 - Ea1;
    double dle = mb0 > 0 ? le_d : (mb0 < 0 ? le_u : 0.5 * (le_d + le_u));
    double dri = mb1 > 0 ? ri_d : (mb1 < 0 ? ri_u : 0.5 * (ri_d + ri_u));
    EE[e] = 0.25 * (Ea1 + Ea0 + Eb1 + Eb0) + 0.25 * (dlo - dup) + 0.25 * (dle - dri);
  }
}

/* R = (1/V) sum_f s_f F_f - S per cell, RB = -sum_e sigma l E per face */
static int sphere_rhs(const ora_sphere *s, const double *cons, const double *phi, double *R, double *RB) {
  const long nc = s->nc, nf = s->nf;
  double *W = malloc(sizeof(double) * SW_N * nc);
  double *FC = malloc(sizeof(double) * 5 * nf), *EF = malloc(sizeof(double) * 3 * nf), *EE = malloc(sizeof(double) * s->ne);
  int *UP = malloc(sizeof(int) * nf);
  int rc = sphere_prims(s, cons, phi, W);
  if (!rc) rc = sphere_fluxes(s, W, phi, FC, EF, UP);
  if (!rc) {
    sphere_emfs(s, W, EF, UP, EE);
    for (long c = 0; c < nc; ++c) {
      double r[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < 6; ++m) {
        int f = s->cface[6 * c + m];
        for (int v = 0; v < 5; ++v) r[v] += s->csign[6 * c + m] * FC[5 * f + v];
      }
      for (int v = 0; v < 5; ++v) r[v] /= s->vol[c];
      int k = cell_k(s, c);
      double g = s->g_c ? s->g_c[k] : 0.0;
      v3 gv = scl(unit(s->xc[c]), -g);   /* radial, inward */
      double rho = cons[c], drho = rho - bg_rho_cell(s, k);
      r[1] -= drho * gv.x; r[2] -= drho * gv.y; r[3] -= drho * gv.z;
      double se = cons[nc + c] * gv.x + cons[2 * nc + c] * gv.y + cons[3 * nc + c] * gv.z;
      if (s->heat) se += s->heat[k];
      r[4] -= se;
      for (int v = 0; v < 5; ++v) R[v * nc + c] = r[v];
    }
    for (long f = 0; f < nf; ++f) {
      double t = 0.0;
      for (int m = 0; m < 4; ++m) {
        int e = s->fedge[4 * f + m];
        t += s->fesign[4 * f + m] * s->elen[e] * EE[e];
      }
      RB[f] = t;   /* dPhi/dt = -(circulation of E about the face) */
    }
  }
  free(W); free(FC); free(EF); free(EE); free(UP);
  return rc;
}

double ora_sphere_dt(const ora_sphere *s, const double *cons, const double *pa, const double *pb, const double *pr) {
  const long nc = s->nc;
  double *phi = malloc(sizeof(double) * s->nf), *W = malloc(sizeof(double) * SW_N * nc);
  load_phi(s, pa, pb, pr, phi);
  if (sphere_prims(s, cons, phi, W)) { free(phi); free(W); return -1.0; }
  double mx = 0.0;
  for (long c = 0; c < nc; ++c) {
    const double *w = &W[SW_N * c];
    int k = cell_k(s, c);
    double rho = w[SW_RHO] + bg_rho_cell(s, k), P = w[SW_P] + bg_p_cell(s, k);
    v3 u = mk(w[SW_U], w[SW_U + 1], w[SW_U + 2]), b = mk(w[SW_B], w[SW_B + 1], w[SW_B + 2]);
    double a2 = (w[SW_GC] + bg_gc(s, k, 0)) * P / rho, b2 = dot(b, b) / rho;
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {   /* the cell's three logical directions */
      int f0 = s->cface[6 * c + 2 * d], f1 = s->cface[6 * c + 2 * d + 1];
      v3 span = sub(s->xf[f1], s->xf[f0]);
      double width = nrm(span);
      v3 ed = scl(span, 1.0 / width);
      double bd = dot(b, ed);
      double disc = (a2 + b2) * (a2 + b2) - 4.0 * a2 * bd * bd / rho;
      if (disc < 0.0) disc = 0.0;
      double cf = sqrt(0.5 * (a2 + b2 + sqrt(disc)));
      sum += (fabs(dot(u, ed)) + cf) / width;
    }
    if (sum > mx) mx = sum;
  }
  free(phi); free(W);
  return s->cfl / mx;
}

int ora_sphere_run(const ora_sphere *s, double *cons, double *pa, double *pb, double *pr, int nsteps,
                   double dt_fixed, double *dt_last) {
  const long nc = s->nc, nf = s->nf;
  double *phi = malloc(sizeof(double) * nf);
  double *c0 = malloc(sizeof(double) * 5 * nc), *c1 = malloc(sizeof(double) * 5 * nc);
  double *p0 = malloc(sizeof(double) * nf), *p1 = malloc(sizeof(double) * nf);
  double *R = malloc(sizeof(double) * 5 * nc), *RB = malloc(sizeof(double) * nf);
  load_phi(s, pa, pb, pr, phi);
  int rc = 0;
  static const double A3[3] = {0.0, 0.75, 1.0 / 3.0}, B3[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int n = 0; n < nsteps && !rc; ++n) {
    double dt = dt_fixed;
    if (!(dt > 0.0)) {
      double *tpa = malloc(sizeof(double) * s->nabi_a), *tpb = malloc(sizeof(double) * s->nabi_b),
             *tpr = malloc(sizeof(double) * s->nabi_r);
      store_phi(s, phi, tpa, tpb, tpr);
      dt = ora_sphere_dt(s, cons, tpa, tpb, tpr);
      free(tpa); free(tpb); free(tpr);
      if (!(dt > 0.0)) { rc = -2; break; }
    }
    memcpy(c0, cons, sizeof(double) * 5 * nc);
    memcpy(p0, phi, sizeof(double) * nf);
    memcpy(c1, cons, sizeof(double) * 5 * nc);
    memcpy(p1, phi, sizeof(double) * nf);
    for (int st = 0; st < 3 && !rc; ++st) {   /* Shu-Osher SSP-RK3 (Sect. 2.9) */
      rc = sphere_rhs(s, c1, p1, R, RB);
      if (rc) break;
      for (long q = 0; q < 5 * nc; ++q) c1[q] = A3[st] * c0[q] + B3[st] * (c1[q] - dt * R[q]);
      for (long f = 0; f < nf; ++f) p1[f] = A3[st] * p0[f] + B3[st] * (p1[f] - dt * RB[f]);
    }
    if (!rc) {
      memcpy(cons, c1, sizeof(double) * 5 * nc);
      memcpy(phi, p1, sizeof(double) * nf);
    }
    if (dt_last) *dt_last = dt;
  }
  store_phi(s, phi, pa, pb, pr);
  free(phi); free(c0); free(c1); free(p0); free(p1); free(R); free(RB);
  return rc;
}

/* discrete divergence sum_f s_f Phi_f of every cell (flux units) */
int ora_sphere_divb(const ora_sphere *s, const double *pa, const double *pb, const double *pr, double *div) {
  double *phi = malloc(sizeof(double) * s->nf);
  load_phi(s, pa, pb, pr, phi);
  for (long c = 0; c < s->nc; ++c) {
    double t = 0.0;
    for (int m = 0; m < 6; ++m) t += s->csign[6 * c + m] * phi[s->cface[6 * c + m]];
    div[c] = t;
  }
  free(phi);
  return 0;
}
