/*
 * oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of one explicit finite-volume MHD
 * update of PHLEGETHON (arXiv 2604.12672, Sect. 2): primitive recovery and EOS
 * (Sect. 2.2), deviation well-balancing (Sect. 2.8), van Leer PLM (Sect. 2.5),
 * LHLLD / HLL Riemann fluxes (Sect. 2.6), shock flattening (Sect. 2.7),
 * Contact-CT (Sect. 2.4), SSP-RK stages and the CFL step (Sect. 2.9); thermal
 * diffusion by RKL2 super-time-stepping (Sect. 2.10); the Poisson solver for
 * the gravitational potential (Sect. 2.12).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library; both
 * consume the same seeded inputs (workloads/).  Compiled with
 * -ffp-contract=off so that every operation rounds as written.
 *
 * Array layout (same as the library's ABI, x fastest, no ghosts):
 *   cons[v][nz][ny][nx], v = rho, mx, my, mz, E, rhoX_0..;
 *   bx[nz][ny][nx+1], by[nz][ny+1][nx], bz[nz+1][ny][nx]; T[nz][ny][nx].
 */
#ifndef PHL_ORACLE_H
#define PHL_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_PERIODIC = 0, ORA_REFLECT = 1, ORA_OUTFLOW = 2 };
enum { ORA_EOS_IDEAL = 0, ORA_EOS_STELLAR = 1 };
enum { ORA_LHLLD = 0, ORA_HLLD = 1, ORA_HLL = 2 };
enum { ORA_RECON_VANLEER = 0, ORA_RECON_PPH = 1, ORA_RECON_PQH = 2 };
#define ORA_MAXSPEC 4

typedef struct {
  int n[3];                 /* cells per dimension; a dimension with n = 1 is inactive */
  double lo[3], hi[3];
  int bc[3][2];             /* ORA_PERIODIC / ORA_REFLECT / ORA_OUTFLOW */
  int eos;                  /* ORA_EOS_IDEAL or ORA_EOS_STELLAR */
  double gamma;
  int nspec;
  double A[ORA_MAXSPEC], Z[ORA_MAXSPEC];
  double g[3];              /* constant gravitational acceleration */
  /* background along z with 3 ghost layers (NULL: no well-balancing) */
  const double *bg_rho_c, *bg_p_c;   /* nz+6 */
  const double *bg_rho_f, *bg_p_f;   /* nz+7 */
  const double *bg_ge_c, *bg_gc_c, *bg_ge_f, *bg_gc_f; /* NULL: gamma */
  const double *heat;       /* NULL or volumetric heating per z-cell [nz] */
  double cfl;
  int rk;                   /* 2 or 3 */
  int riemann;              /* ORA_LHLLD / ORA_HLLD / ORA_HLL */
  double eps_sf;            /* 0: no shock flattening */
  double mach_thr;          /* LHLLD threshold (0.6) */
  double newton_tol;        /* stellar EOS */
  int newton_maxit;
  const void *eos_table;    /* stellar EOS table (ora_eos_table_build) */
  int recon;                /* ORA_RECON_VANLEER (limited linear), _PPH, _PQH (limited fifth order) */
} ora_cfg;

/* Thermal diffusion (Sect. 2.10): conductivity K = k0 T^nT / rho^nR with
 * T = e_int / cv (ideal gas, code units). */
typedef struct {
  double k0;
  int nT, nR;
  double cv;
  int delta_T;              /* 1: diffuse only T - T_hat, the deviation from the */
                            /* background temperature P_hat / ((gamma-1) rho_hat cv) */
} ora_diff;

/* RKL2 coefficients mu_j, nu_j, mu~_j, gamma~_j (j = 1..s; arrays of s + 1),
 * the amplification factor of an s-stage step at z = lambda dt, and the
 * paper's stage count for a step dt against the parabolic limit dt_p. */
void ora_rkl2_coeffs(int s, double *mu, double *nu, double *mut, double *gat);
double ora_rkl2_amp(int s, double z);
int ora_sts_stages(double dt, double dt_p);

/* One RKL2 super step of length dt of rho d(e_int)/dt = div(K grad T) with
 * rho, u, B fixed, on the ABI-layout state (cons updated in place: E only).
 * *nsts_out receives the stage count.  Returns 0, -1 (bad input), -2
 * (non-positive rho or e_int) or -4 (more than max_stages stages needed). */
int ora_diffuse(const ora_cfg *cfg, double *cons, const double *bx, const double *by, const double *bz,
                const ora_diff *p, double dt, int max_stages, int *nsts_out);

/* Face values (left, right) of the centre cell w[2] of five cells under a
 * reconstruction; species != 0: a mass fraction. */
void ora_recon_cell(int recon, int species, const double *w, double *fl, double *fr);

/* Poisson solver for the gravitational potential (poisson.c, Sect. 2.12).
 * xf[d]: the n[d] + 1 increasing face coordinates of axis d; rho, phi: cell
 * arrays [nz][ny][nx]; ghost potentials: x faces [2][nz][ny], then y faces
 * [2][nz][nx], then z faces [2][ny][nx] (lower side first). */
enum { ORA_POISSON_RELATIVE = 0, ORA_POISSON_ABSOLUTE = 1 };
typedef struct {
  int n[3];
  const double *xf[3];
  double G;
  int lmax;                 /* 0: monopole; 2: + quadrupole; 3: + octupole */
  int criterion;            /* ORA_POISSON_RELATIVE (Eq. poisson-eps) / _ABSOLUTE */
  double tol;
  int max_iter;
} ora_poisson;

long ora_poisson_nghost(const int *n);
int ora_multipole_moments(const ora_poisson *p, const double *rho, double *M, double *X, double *Q, double *O);
double ora_multipole_phi(double G, int lmax, double M, const double *X, const double *Q, const double *O, double x,
                         double y, double z);
int ora_poisson_boundary(const ora_poisson *p, const double *rho, double *ghost);
int ora_poisson_apply(const ora_poisson *p, const double *phi, const double *ghost, double *out);
int ora_gravity(const ora_poisson *p, const double *phi, const double *ghost, double *gx, double *gy, double *gz);
int ora_poisson_solve(const ora_poisson *p, const double *rho, double *phi, double *ghost_out, int *iters,
                      double *resid);

/* Advance nsteps SSP-RK steps in place.  dt_fixed > 0 uses that step;
 * otherwise each step's dt comes from the CFL condition on U^n.
 * t (nullable) accumulates time; dt_last (nullable) receives the last dt.
 * Returns 0 or a negative code (-1 bad input, -2 non-positive rho/P, -3 Newton). */
int ora_run(const ora_cfg *cfg, double *cons, double *bx, double *by, double *bz,
            double *T, int nsteps, double dt_fixed, double *t, double *dt_last);

/* CFL time step of the state (Eq. cfl). */
double ora_dt(const ora_cfg *cfg, const double *cons, const double *bx,
              const double *by, const double *bz, double *T);

/* One stage: out = a*base + b*(in - dt*R(in)) for cells and faces. */
int ora_stage(const ora_cfg *cfg, const double *cons_in, const double *bx_in,
              const double *by_in, const double *bz_in, double *T,
              const double *cons_base, const double *bx_base, const double *by_base,
              const double *bz_base, double a, double b, double dt,
              double *cons_out, double *bx_out, double *by_out, double *bz_out);

/* Single-face Riemann flux in the face-normal frame.
 * wl, wr: rho, un, ut1, ut2, Bt1, Bt2, P, gamma_e, gamma_c, X_0..X_{nspec-1}
 * f: rho, mn, mt1, mt2, E, Bt1, Bt2, rhoX_0.. */
void ora_riemann(const double *wl, const double *wr, double bn, int nspec,
                 int solver, double mach_thr, double *f);

/* Contact-CT corner EMF (Sect. 2.4): Ef = face EMFs Ea1, Ea0, Eb1, Eb0; Ec =
 * cell reference EMFs E00, E10, E01, E11; F = mass fluxes through the same
 * four faces; rho, smax: the density and fastest signal speed of the faces
 * (the contact direction's deadband is 1e-12 rho smax). */
double ora_ct_corner(const double *Ef, const double *Ec, const double *F, double rho, double smax);

/* Divergence max|div B| * min(dx) over interior cells (Eq. divb). */
double ora_divb(const ora_cfg *cfg, const double *bx, const double *by, const double *bz);

/* ---------------- stellar EOS (eos.c) ---------------- */
typedef struct ora_eos_table ora_eos_table;
ora_eos_table *ora_eos_table_build(double lrho_lo, double lrho_hi, int nrho,
                                   double lT_lo, double lT_hi, int nT);
void ora_eos_table_free(ora_eos_table *t);
int ora_eos_table_export(const ora_eos_table *t, double *out, long nout);
long ora_eos_table_size(const ora_eos_table *t);

/* Direct (quadrature) electron-positron gas at (rho*Ye, T): P, e (per gram of
 * the mixture with Ye), free energy f = e - T s, s, eta.  Returns 0 or -1. */
int ora_ep_direct(double rho, double ye, double T, double *P, double *e,
                  double *s, double *eta, double *npos);
/* Free-energy density f(x, y) of the e-/e+ gas, x = ln nnet, y = ln T:
 * ora_ep_first: f, f_x, f_y, f_xy from the integrals' own combinations;
 * ora_ep_derivs: f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy by
 * truncated Taylor arithmetic (the biquintic table's node values). */
int ora_ep_first(double nnet, double T, double *fv);
int ora_ep_derivs(double nnet, double T, double *out);
/* Generalised Fermi-Dirac integral F_k(eta, beta). */
double ora_fd(double k, double eta, double beta);

/* Full stellar EOS (ions + radiation + e-/e+) at (rho, T, X):
 * P, e_int, c_v, dP/drho|T, dP/dT|rho, gamma_e, gamma_c.  table NULL: direct. */
int ora_eos_rt(const ora_cfg *cfg, double rho, double T, const double *X,
               double *P, double *e, double *cv, double *dPdr, double *dPdT,
               double *ge, double *gc);
/* Newton inversion e_int -> T (Sect. 2.2); T_inout holds the guess. */
int ora_eos_invert(const ora_cfg *cfg, double rho, double eint, const double *X,
                   double *T_inout, double *P, double *ge, double *gc, int *iters);

/* ---------------- cubed-sphere shell (sphere.c) ----------------
 * Six equiangular patches of N x N angular cells times Nr radial cells, r in
 * [r_in, r_out] uniform; ideal gas (or the stellar EOS, ora_sphere_set_stellar);
 * per-shell background rho_c, p_c (Nr, at
 * the shell's middle radius) and rho_f, p_f (Nr + 1, at the shell radii), or
 * NULL (no well-balancing); inward gravity g_c (Nr) and heating (Nr) or NULL.
 * Layouts: see sphere.c. */
typedef struct ora_sphere ora_sphere;
ora_sphere *ora_sphere_create(int N, int Nr, double r_in, double r_out, double gamma, const double *rho_c,
                              const double *p_c, const double *rho_f, const double *p_f, const double *g_c,
                              const double *heat, double cfl, int riemann, double mach_thr);
void ora_sphere_free(ora_sphere *s);
long ora_sphere_ncells(const ora_sphere *s);
long ora_sphere_nfaces(const ora_sphere *s);
long ora_sphere_nedges(const ora_sphere *s);
long ora_sphere_nabi_faces(const ora_sphere *s);
/* vol[nc], xc[nc][3], S[nf][3] (unique faces), xf[nf][3], csum[nc][3] (sum of a
 * cell's outward area vectors); any may be NULL */
int ora_sphere_geometry(const ora_sphere *s, double *vol, double *xc, double *S, double *xf, double *csum);
double ora_sphere_dt(const ora_sphere *s, const double *cons, const double *pa, const double *pb, const double *pr);
int ora_sphere_run(const ora_sphere *s, double *cons, double *pa, double *pb, double *pr, int nsteps,
                   double dt_fixed, double *dt_last);
int ora_sphere_divb(const ora_sphere *s, const double *pa, const double *pb, const double *pr, double *div);
/* The stellar EOS on the shell (Sect. 2.2): eos supplies the table, the
 * species' A, Z and the Newton settings; X the uniform mass fractions (the
 * composition stays uniform, so Abar and Y_e are constants of the run);
 * code density and pressure are rho_u and p_u times g/cm^3 and erg/cm^3.
 * The background's gamma_e, gamma_c come from the EOS at (rho_hat, P_hat).
 * Returns 0 or -1. */
int ora_sphere_set_stellar(ora_sphere *s, const ora_cfg *eos, const double *X, double rho_u, double p_u);
/* Conserved cells (5 x cells, ABI order) from primitives rho, vel[cells][3],
 * P and the face fluxes (the cell field is the method's (1/V) sum s_f Phi_f
 * x_f); with the stellar EOS T by P -> T and E from e(rho, T), kept as the
 * cells' temperatures.  Returns 0, -1 or -3 (no temperature). */
int ora_sphere_from_prims(ora_sphere *s, const double *rho, const double *vel, const double *P, const double *pa,
                          const double *pb, const double *pr, double *cons);
/* Cell temperatures (ABI order): each stellar inversion's guess and result. */
int ora_sphere_set_T(ora_sphere *s, const double *T);
int ora_sphere_get_T(const ora_sphere *s, double *T);
void ora_riemann_up(const double *wl, const double *wr, double bn, int nspec, int solver, double mach_thr,
                    double *f, int *up);

/* ---------------- MLP (mlp.c) ---------------- */
void ora_mlp_forward(const double *w, int nin, int nh, const double *x, long n,
                     double *y);
double ora_mlp_loss_grad(const double *w, int nin, int nh, const double *x,
                         const double *t, long n, double *grad);

#ifdef __cplusplus
}
#endif
#endif
