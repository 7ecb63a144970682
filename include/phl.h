/*
 * phl.h -- C ABI of the GB300 explicit-MHD stage library (libphl.so).
 *
 * The library advances the equations of fully compressible ideal MHD with
 * gravity and heating sources (arXiv 2604.12672, Sect. 2.1, Eqs. mass
 * conservation .. energy) with the paper's explicit finite-volume scheme:
 *   - primitive recovery and the equation of state (Sect. 2.2),
 *   - deviation well-balancing against a hydrostatic background (Sect. 2.8,
 *     Eqs. wb, wb1, wb2),
 *   - van Leer limited piecewise-linear reconstruction (Sect. 2.5, item i),
 *   - the low-dissipation LHLLD Riemann flux with the HLL shock-flattening
 *     fallback (Sects. 2.6-2.7, Eqs. flux-hlld, pstar),
 *   - Contact-CT edge EMFs and the face-centred B update (Sect. 2.4, Eqs.
 *     induction, divb),
 *   - SSP-RK2/RK3 stages and the CFL time step (Sect. 2.9, Eqs. spatres, cfl).
 *
 * Conventions shared by every entry point
 *   Units: Heaviside-Lorentz (no 4 pi), Sect. 2.1.
 *   Layout of state arrays (x fastest, no ghost cells):
 *     cons[v][nz][ny][nx], v = rho, rho*u_x, rho*u_y, rho*u_z, rho*e, rho*X_l...
 *       (nv = 5 + nspec doubles per cell; rho*e is the total energy density);
 *     bx[nz][ny][nx+1] normal B on x-faces i-1/2 (i = 0..nx),
 *     by[nz][ny+1][nx], bz[nz+1][ny][nx] likewise;
 *     T[nz][ny][nx] temperature (stellar EOS only; the Newton first guess).
 *   A dimension with n = 1 is inactive; its face array holds two equal layers.
 *   Periodic boundaries: the duplicate faces (index 0 and n) must be equal.
 *   Pointers: "where" = PHL_HOST means ordinary (pageable or pinned) host
 *     memory; PHL_DEVICE means device memory of the current CUDA device.  No
 *     call keeps a caller's pointer after it returns.
 *   Streams: all device work of a grid is ordered on desc.stream (a
 *     cudaStream_t; NULL = legacy default stream).
 *   Errors: every call returns a phl_status; a message for the last failure
 *     of the calling thread is available from phl_last_error().  Invalid
 *     states found on the device (rho <= 0, P <= 0, NaN, Newton failure) set
 *     a device flag that is reported by the next call that synchronises
 *     (phl_compute_dt, phl_get_state, phl_check).  Nothing aborts.
 *   Threads: a grid may be used by one host thread at a time.
 */
#ifndef PHL_H
#define PHL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PHL_OK = 0,
  PHL_EINVAL = 1,        /* bad argument                                  */
  PHL_ECUDA = 2,         /* CUDA runtime error                            */
  PHL_ENOMEM = 3,        /* device allocation failed                      */
  PHL_ENEGATIVE = 4,     /* rho <= 0 or P <= 0 in a cell or at a face     */
  PHL_ENAN = 5,          /* non-finite value                              */
  PHL_ENEWTON = 6,       /* EOS temperature inversion did not converge    */
  PHL_ETIMEOUT = 7,      /* a bounded device wait gave up                 */
  PHL_EUNSUPPORTED = 8,  /* option combination not built                  */
  PHL_ENOCONV = 9        /* iterative solver did not converge / broke down */
} phl_status;

enum { PHL_PERIODIC = 0, PHL_REFLECT = 1, PHL_OUTFLOW = 2 };
enum { PHL_EOS_IDEAL = 0, PHL_EOS_STELLAR = 1 };
enum { PHL_LHLLD = 0, PHL_HLLD = 1, PHL_HLL = 2 };
enum { PHL_RECON_VANLEER = 0, PHL_RECON_PPH = 1, PHL_RECON_PQH = 2 };
enum { PHL_FP64 = 0, PHL_MIXED = 1 };
enum { PHL_HOST = 0, PHL_DEVICE = 1 };
#define PHL_MAXSPEC 4

typedef struct phl_grid phl_grid;   /* opaque; owns all its device buffers */

typedef struct {
  int n[3];                 /* cells per dimension (1 = inactive)              */
  double lo[3], hi[3];      /* domain; uniform spacing (hi-lo)/n               */
  int bc[3][2];             /* PHL_PERIODIC / PHL_REFLECT / PHL_OUTFLOW        */
  int eos;                  /* PHL_EOS_IDEAL / PHL_EOS_STELLAR                 */
  double gamma;             /* ideal-gas adiabatic index                       */
  int nspec;                /* advected mass fractions (0..PHL_MAXSPEC)        */
  double A[PHL_MAXSPEC], Z[PHL_MAXSPEC];
  double g[3];              /* constant gravitational acceleration             */
  /* Hydrostatic background along z for the deviation method (Sect. 2.8),
   * host arrays copied at creation, with 3 ghost layers each side:
   *   *_c: cell centres k = -3..nz+2 (nz+6 values, index k+3)
   *   *_f: z-faces k-1/2, k = -3..nz+3 (nz+7 values, index k+3)
   * bg_rho_c == NULL: no background (plain scheme).  The gamma_e/gamma_c
   * profiles may be NULL (then gamma is used). */
  const double *bg_rho_c, *bg_p_c, *bg_rho_f, *bg_p_f;
  const double *bg_ge_c, *bg_gc_c, *bg_ge_f, *bg_gc_f;
  const double *heat;       /* host, per z-cell volumetric heating rate, or NULL */
  double cfl;               /* Eq. cfl                                          */
  int rk;                   /* 2 or 3 (SSP-RK)                                  */
  int riemann;              /* PHL_LHLLD / PHL_HLLD / PHL_HLL                   */
  double eps_sf;            /* shock-flattening threshold (0.2); 0 = off        */
  double mach_thr;          /* LHLLD Mach threshold (0.6)                       */
  int precision;            /* PHL_FP64 / PHL_MIXED                             */
  double newton_tol;        /* stellar EOS Newton tolerance (1e-11)             */
  int newton_maxit;
  int use_mlp;              /* stellar EOS, Newton first guess from desc.mlp:   */
                            /* 1: always (previous T as fallback); 2: only where */
                            /* no previous T exists (cold start); 0: never       */
  void *stream;             /* cudaStream_t                                     */
  const struct phl_eos_table *eos_table;  /* stellar EOS table (not owned)      */
  const struct phl_mlp *mlp;  /* temperature-guess network when use_mlp (not owned) */
  double bg_X[PHL_MAXSPEC]; /* stellar: mass fractions of the background        */
  /* Reconstruction (Sect. 2.5): PHL_RECON_VANLEER, limited linear (van Leer
   * slope, item i; the default, 0); PHL_RECON_PPH, the three-cell parabola of
   * item ii -- unlimited for the primitive variables, limited for the mass
   * fractions (the piecewise-parabolic method's monotonicity constraints).
   * Both use the same three-cell stencil per face side.  PHL_RECON_PQH, the
   * limited fifth-order reconstruction of item iii for every variable: the
   * face value of the degree-4 polynomial through five cell averages, limited
   * by the monotonicity-preserving bounds of Suresh & Huynh (1997); five-cell
   * stencil, three ghost layers, not on the fused tile kernel (phl_set_fused
   * declines it).  Under every scheme, cells flagged by the shock flattener
   * reconstruct with van Leer (Sect. 2.7). */
  int recon;
} phl_grid_desc;

typedef struct {
  long steps;               /* completed RK steps                               */
  double t;                 /* accumulated time (only when dt is read back)     */
  double last_dt;
  int device_flags;         /* bit 0: rho/P <= 0, bit 1: NaN, bit 2: Newton     */
  int kernels_per_step;     /* CUDA kernel launches per RK step                 */
  size_t device_bytes;      /* device memory owned by the grid                  */
  long newton_iters;        /* stellar EOS: Newton iterations summed over cells */
} phl_stats;

/* Create a grid: validates the description, allocates the state (padded SoA
 * FP64) and the work buffers on the current device.  *out receives the
 * handle.  Errors: PHL_EINVAL (dimensions, BCs, cfl, rk...), PHL_ENOMEM,
 * PHL_EUNSUPPORTED, PHL_ECUDA. */
phl_status phl_create_grid(const phl_grid_desc *desc, phl_grid **out);

/* Load the state (layout above).  T (stellar EOS: Newton first guesses) may
 * be NULL: the first inversion then starts from the network's guess
 * (use_mlp) or from the table's mid-range temperature.  where = PHL_HOST or
 * PHL_DEVICE.  Stream-ordered; host sources are copied before return. */
phl_status phl_set_state(phl_grid *g, const double *cons, const double *bx,
                         const double *by, const double *bz, const double *T,
                         int where);

/* The mixed stellar form's inversion record (Sect. 2.2 Newton inversion):
 * per cell rho, e_int, 1/c_v, de/drho at fixed T, ln T, 1/T, ln(n_e N_A) and
 * n_e = rho Y_e of the cell's last inversion, rec[8][nz][ny][nx]; each
 * inversion starts from the first-order guess they give.  set_state and
 * set_state_prim clear it (the next inversions start plainly); restoring it
 * with the state and T makes a resumed run repeat the uninterrupted one bit
 * for bit.  PHL_EINVAL on grids without one (FP64 or ideal gas). */
phl_status phl_get_eos_record(phl_grid *g, double *rec, int where);
phl_status phl_set_eos_record(phl_grid *g, const double *rec, int where);

/* Load the state from primitive fields: prim[(5 + nspec)][nz][ny][nx] =
 * rho, u_x, u_y, u_z, P, X_l (mass fractions), plus the face fields.  The
 * conserved energy is rho e(rho, T) + rho u^2/2 + B^2/2 with T from
 * P_EoS(rho, T, X) = P (stellar EOS: Newton on P; ideal gas: direct);
 * the temperatures become the Newton first guesses.  Host or device arrays. */
phl_status phl_set_state_prim(phl_grid *g, const double *prim, const double *bx, const double *by,
                              const double *bz, int where);

/* Store the state into caller arrays (layout above); T may be NULL.
 * Synchronises the grid's stream and reports device flags. */
phl_status phl_get_state(phl_grid *g, double *cons, double *bx, double *by,
                         double *bz, double *T, int where);

/* CFL step of the current state (Eq. cfl): dt = cfl / max over cells of
 * sum_s (|u_s| + c_f,s) / dx_s, c_f the fast magnetosonic speed.  Writes the
 * host value to *dt_out (synchronises). */
phl_status phl_compute_dt(phl_grid *g, double *dt_out);

/* Advance nsteps SSP-RK steps (Sect. 2.9).  dt > 0: fixed step; dt <= 0: each
 * step's dt is computed on the device from U^n (no host round trip).  Launches
 * are asynchronous on the grid's stream; errors found on the device are
 * reported by the next synchronising call. */
phl_status phl_step(phl_grid *g, double dt, int nsteps);

/* Synchronise and report device error flags. */
phl_status phl_check(phl_grid *g);

/* Replace the stream used by the grid. */
phl_status phl_set_stream(phl_grid *g, void *stream);

phl_status phl_get_stats(phl_grid *g, phl_stats *st);

/* Per-kernel device timing.  When enabled, every kernel launch of the grid is
 * bracketed by CUDA events on the grid's stream; phl_kernel_times folds the
 * recorded pairs (synchronising) into per-kernel totals since the last reset.
 * Kernel classes are named ("prim", "flux_x", "stage_mixed", ...). */
typedef struct {
  char name[32];
  long launches;
  double ms;                /* summed device time of those launches */
} phl_kernel_time;

phl_status phl_set_timing(phl_grid *g, int on);
/* Fills up to max entries, *n receives the number of kernel classes seen;
 * reset != 0 clears the totals afterwards. */
phl_status phl_kernel_times(phl_grid *g, phl_kernel_time *out, int max, int *n, int reset);

/* Thermal diffusion (Sect. 2.10): ideal gas with T = e_int / cv (code
 * units) and conductivity K = k0 T^nT / rho^nR (nT = 0..4, nR = 0..2; a
 * constant K: nT = nR = 0; radiative diffusion with a constant opacity,
 * K = 4acT^3 / (3 kappa rho): nT = 3, nR = 1, k0 = 4ac / (3 kappa)). */
enum { PHL_DIFF_GRID = 0, PHL_DIFF_FP64 = 1, PHL_DIFF_MIXED = 2 };
typedef struct {
  double k0;
  int nT, nR;
  double cv;
  int precision;            /* PHL_DIFF_GRID: the grid's precision mode;       */
                            /* PHL_DIFF_FP64: stages in double;                */
                            /* PHL_DIFF_MIXED: stages in float on the change   */
                            /* of e_int (face differences of e_int^(0) taken   */
                            /* in double), either grid                         */
  int tile_z;               /* mixed stage kernel: planes per CTA (0: 16), a    */
                            /* tuning knob; results do not depend on it        */
  int delta_T;              /* 1: diffuse only T - T_hat, the deviation from the */
                            /* well-balancing background's temperature         */
                            /* P_hat / ((gamma-1) rho_hat cv) (Sect. 2.10); K  */
                            /* stays that of the full T; needs a background    */
} phl_diffusion;

/* Advance rho d(e_int)/dt = div(K grad T) over dt with the density,
 * velocity, magnetic field and mass fractions held fixed, by one RKL2 super
 * step (Meyer, Balsara & Aslam 2012; Sect. 2.10 items i-iv), and add
 * rho times the change of e_int to the total energy.  The stage count is the
 * paper's N_STS = max(1 + floor((sqrt(9 + 16 dt/dt_p) - 1)/2), 3) with the
 * parabolic limit dt_p = 1/2 [max sum_s D/dx_s^2]^-1, D = K/(rho cv), of the
 * state at the start of the step: the call reads that maximum back (one
 * synchronisation of the grid's stream) and then enqueues the stage kernels
 * (3 N_STS + 2 in FP64, N_STS + 2 mixed).  Space: conservative seven-point
 * operator, face conductivity the harmonic mean of the two cells' (Sect.
 * 2.10), no flux through sides that are not periodic.  Call between MHD
 * steps (e.g. Strang splitting: half dt, phl_step, half dt).  The first call
 * allocates the grid's diffusion arrays (eleven doubles per cell).
 *   max_stages: PHL_EINVAL when N_STS would exceed it; *nsts_out (nullable)
 *   receives N_STS.  PHL_EINVAL also for bad parameters and for delta_T on a
 *   grid without a background; PHL_EUNSUPPORTED for the stellar EOS and for
 *   the mixed form on 2^32 cells or more.  A cell with rho <= 0 or
 *   e_int <= 0 sets the device flag (PHL_ENEGATIVE at the next synchronising
 *   call). */
phl_status phl_diffuse(phl_grid *g, const phl_diffusion *p, double dt, int max_stages, int *nsts_out);

/* Selects how a mixed-precision grid evaluates a stage (Sects. 2.4-2.9; the
 * arithmetic is the same, only the kernel decomposition differs).
 *   on = 1: the fused tile kernel -- each CTA stages an 8x8x8 tile of the
 *           primitive deviations with two ghost layers by TMA, computes the
 *           faces of all three directions in shared memory and applies the
 *           cell update; the primitives, raw shock flags and their dilation
 *           before it and the Contact-CT EMFs and face updates after it run as
 *           one kernel each (six launches per stage).  Needs
 *           precision = PHL_MIXED, an ideal gas, nspec = 0 and at least four
 *           cells along each of three active dimensions (PHL_EUNSUPPORTED
 *           otherwise).  Default where eligible.
 *   on = 2..9: the same kernel in other launch shapes (threads per CTA,
 *           CTAs per SM, faces of one direction at a time through a smaller
 *           shared buffer; 5 to 7 evaluate two faces per thread on packed
 *           FP32x2 arithmetic; 8 and 9 pair the left and right states of
 *           each face on FP32x2 arithmetic), for tuning; 1 selects the
 *           default shape.
 *   on = 201..209: shapes 1..9 with the stage in three launches: (i) the
 *           tile kernel, which dilates the raw shock flags of its tile in
 *           shared memory; (ii) Contact-CT: the edge EMFs an 8^3 tile of
 *           sites needs, in shared memory, and the update of the tile's own
 *           faces; (iii) the next stage's primitive deviations for a 16x16x8
 *           tile of cells with their ghost images, the raw flags from the
 *           pressures of a one-cell halo, and in the last stage the CFL rate
 *           of the new state folded into the next step's maximum (a step
 *           with the device CFL step adds one one-thread launch).  The first
 *           step after the state was set from outside (phl_set_state,
 *           phl_set_state_prim, phl_diffuse, a host phl_get_state, an
 *           ensemble step, this call) forms the primitives, raw flags and
 *           CFL step in their own kernels first.  Ten launches per step
 *           instead of twenty, but slower per cell on this GPU (the flag
 *           dilation no longer overlaps the tile's copy; the halo primitives
 *           and the small CT tiles cost more than they save).
 *   on = 0: one kernel per direction for the faces, then EMFs and updates.
 * Results of all of these agree to FP32 rounding of the deviations.  Call
 * between steps only (no stage of the grid in flight on its stream).
 * PHL_EINVAL for on outside 0..9 and 201..209. */
phl_status phl_set_fused(phl_grid *g, int on);

/* Test of the failure path of the fused tile kernel's bounded wait.  With
 * on != 0, each tile announces 16 bytes more to its TMA completion barrier than
 * its copy delivers: the copy itself completes (nothing is left in flight),
 * the barrier's phase never does, every CTA gives up after its bounded waits
 * (1 s each), sets the timeout bit and returns without writing its cells, and
 * the next synchronising call (phl_check, phl_compute_dt, phl_get_state)
 * returns PHL_ETIMEOUT.  The context stays usable: with on = 0 and the state
 * reloaded (phl_set_state clears the error bits) the grid steps normally.
 * Meant for tiny grids (each affected stage waits ~2 s per wave of CTAs).
 * PHL_EUNSUPPORTED if the grid does not run the fused kernel. */
phl_status phl_test_tile_wait_timeout(phl_grid *g, int on);

/* Test of the two forms of the mixed stage's primitive deviations (Sect. 2.8,
 * the deviations from the hydrostatic background of the stage-input state):
 * forms W for the whole work box (interior cells and their ghost images) of a
 * mixed ideal-gas grid and copies it to the host.
 *   form       0: one cell per thread; 1: two cells of a row per thread from
 *              aligned FP64 pairs (grids with an even number of cells along x
 *              and no species); 2 / 3: forms 0 / 1 of the first stage, with the
 *              CFL rate of U^n taken from the same deviations
 *   increments != 0 (forms 0 and 1): add the grid's current FP32 stage
 *              increments, as the second and third stages do
 *   w_out      host, cap floats; receives (wstr + 4) x wtot floats: the W
 *              planes and their auxiliary planes in the work layout (two ghost
 *              layers per active axis, x fastest), zero where no cell is formed
 *              (phl_test_prims_size gives the count)
 *   rate_out   host, optional: the largest CFL rate in scaled units (forms 2, 3;
 *              0 otherwise)
 * W is clobbered (the next phl_step forms it again).  Synchronous on the
 * grid's stream.  PHL_EUNSUPPORTED for FP64 or stellar grids, or form 1 / 3 on
 * a grid without the pair form; PHL_EINVAL for a bad form or a short buffer. */
phl_status phl_test_prims(phl_grid *g, int form, int increments, float *w_out, long cap, float *rate_out);
/* The number of floats phl_test_prims writes (0 for an FP64 grid). */
phl_status phl_test_prims_size(phl_grid *g, long *nfloat);

/* Test of the two forms of the raw shock flags (Sect. 2.7: sum over the axes
 * of |P_(i+1) - P_(i-1)| against eps_sf P_i) of a mixed grid, from the W that
 * the last phl_test_prims formed.
 *   form     0: one cell per thread; 1: four cells of a row per thread (n_x a
 *            multiple of 4)
 *   out      host, cap bytes; receives nx*ny*nz flags (0 / 1), x fastest
 *   any_out  host, optional: the kernel's vote, 1 if some cell is flagged
 * The grid's flag buffers are clobbered (the next phl_step forms them again).
 * Synchronous on the grid's stream.  PHL_EUNSUPPORTED for an FP64 grid or
 * form 1 on a grid without the four-cell form; PHL_EINVAL for a bad form or a
 * short buffer. */
phl_status phl_test_raw_flags(phl_grid *g, int form, unsigned char *out, long cap, int *any_out);

/* Device pointer of the last computed dt (double), valid for the grid's
 * lifetime; lets callers enqueue reads without a synchronisation. */
phl_status phl_dt_device_ptr(phl_grid *g, const double **ptr);

/* The mixed form's FP64 <-> FP32 boundary conversions, for unit tests: for
 * each x[i], f[i] = x[i] * 2^k rounded to the nearest FP32 (ties away from
 * zero; magnitudes below 2^-126 flush to zero, above the FP32 range give
 * +-inf; NaN stays NaN) and back[i] = f[i] * 2^-k in FP64 (exact).  The
 * kernels apply their power-of-two unit scales this way, on the integer
 * pipe.  Host arrays of n values; |k| < 800 (PHL_EINVAL otherwise). */
phl_status phl_convert_batch(long n, const double *x, int k, float *f, double *back);

/* Evaluate the library's face flux (the device Riemann solver of the stage)
 * for n independent faces -- for unit tests of the solver itself.
 *   wl, wr  [n][9 + nspec] normal-frame primitive deviations, in order
 *           rho, u_n, u_t1, u_t2, B_t1, B_t2, P, gamma_e, gamma_c, X_l...
 *           (full values when the background is zero);
 *   bn      [n] face-normal field;
 *   bg      [n][4] background at the face: rho, P, gamma_e, gamma_c (zeros
 *           for none);
 *   f       [n][7 + nspec] output F - F_hat: rho, m_n, m_t1, m_t2, E, B_t1,
 *           B_t2, rho*X_l...
 * solver = PHL_LHLLD / PHL_HLLD / PHL_HLL; precision = PHL_FP64 evaluates in
 * double, PHL_MIXED in float (inputs rounded to float), 2 in float with the
 * ideal-gas solver of the fused stage kernel, two faces per thread on packed
 * FP32x2 arithmetic, 3 in float with the ideal-gas solver that pairs the left
 * and right states of each face on FP32x2 arithmetic (2 and 3: nspec = 0
 * only; gamma taken from bg[.][2] (of the first face of each pair for 2), so
 * all faces must share one gamma; gamma_e and gamma_c deviations are
 * ignored).  All pointers are host memory; the call is
 * synchronous on the legacy default stream. */
phl_status phl_riemann_batch(long n, const double *wl, const double *wr, const double *bn,
                             const double *bg, int nspec, int solver, double mach_thr,
                             int precision, double *f);

/* Arithmetic-throughput probe: the current GPU's fused multiply-add rate in
 * TFLOP/s (2 flop per FMA), kind 0 = FP32, 1 = FP64, from register-only
 * kernels of independent FMA chains over all SMs (best of three timed runs
 * after a warm-up, CUDA events on `stream`; synchronous).  It gives the
 * measured denominators of the ALU rooflines (no counterpart in the paper).
 * Errors: PHL_EINVAL, PHL_ECUDA. */
phl_status phl_probe_alu(int kind, double *tflops, void *stream);

/* CFL step (same definition as phl_compute_dt) computed without allocating
 * any device memory.  No counterpart in the paper: it exists for callers that
 * cannot let a library call cudaMalloc/cudaFree -- a host program whose own
 * memory pool owns all device memory, or a driver loop that must not pay the
 * device-wide synchronisation those calls may imply.
 *   desc     geometry and physics (n, lo, hi, gamma, cfl; ideal EOS only);
 *            no other field is read and no grid is needed;
 *   cons, bx, by, bz  device pointers, ABI layout above (read only):
 *            cons (5 + nspec) nx ny nz doubles, bx (nx+1) ny nz, by nx (ny+1) nz,
 *            bz nx ny (nz+1); the caller keeps them alive until the kernels end;
 *   dt_out   device pointer to one double that receives cfl / max(...);
 *   stream   cudaStream_t the two kernels are queued on (asynchronous).
 * Pointers that are not device (or managed) memory of the current device are
 * rejected with PHL_EINVAL before anything is launched; sizes cannot be
 * checked from a pointer and must match desc.
 * Invalid states: unlike phl_compute_dt, which returns PHL_ENEGATIVE or
 * PHL_ENAN, this call keeps no error word: a cell with rho <= 0, P <= 0 or any
 * non-finite value makes dt_out exactly 0 (the call itself returns PHL_OK), so
 * a caller checks dt_out > 0 before using it.
 * Scratch: a library-owned __device__ array of PHL_DT_NOALLOC_MAX_CELLS / 4096
 * doubles (128 KiB), present on every GPU that loads the library until the
 * process exits; grids above PHL_DT_NOALLOC_MAX_CELLS cells are rejected with
 * PHL_EINVAL ("too many cells").  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the current
 * CUDA context; a call under another context (after cudaDeviceReset, or a
 * non-primary context) looks it up again.  Make the first call in each
 * context before any stream capture.  Every call shares the array and leaves
 * its partial results in it; calls whose kernels overlap on the GPU race on
 * it.
 * Errors: PHL_EINVAL, PHL_EUNSUPPORTED (stellar EOS), PHL_ECUDA. */
#define PHL_DT_NOALLOC_MAX_CELLS 67108864L
phl_status phl_cfl_dt_noalloc(const phl_grid_desc *desc, const double *cons, const double *bx,
                              const double *by, const double *bz, double *dt_out, void *stream);

/* ---------------- stellar equation of state (Sect. 2.2, item ii) --------
 * Ions (ideal gas), radiation (Eqs. prad, erad) and an electron-positron gas
 * of arbitrary degeneracy and relativity in pair equilibrium.  The e-/e+ part
 * is a table of its Helmholtz free-energy density f over (x, y) =
 * (ln n_e, ln T), n_e = rho Y_e N_A, holding f, f_x, f_y, f_xx, f_yy, f_xy,
 * f_xxy, f_xyy and f_xxyy at each node, computed on the device from
 * generalised Fermi-Dirac integrals, and interpolated biquintically (tensor
 * product of quintic Hermite polynomials) as the paper does with its
 * Helmholtz free-energy table; P, e, c_v and the pressure derivatives all
 * derive from that one interpolant.  At 80 nodes per decade in both
 * variables the interpolated P, e, gamma_e agree with direct quadrature to
 * ~1e-8 and c_v, gamma_c to ~4e-7; at 40 per decade (the bindings' default)
 * to ~1e-7 and ~7e-6.  CGS units. */
typedef struct phl_eos_table phl_eos_table;

/* Build the table on the current device: log10(rho Y_e) in [lrhoye_lo,
 * lrhoye_hi] with nrho nodes, log10 T in [lT_lo, lT_hi] with nT nodes.
 * Errors: PHL_EINVAL, PHL_ENOMEM, PHL_ENEWTON (a node did not converge). */
phl_status phl_eos_table_create(double lrhoye_lo, double lrhoye_hi, int nrho, double lT_lo,
                                double lT_hi, int nT, phl_eos_table **out);
void phl_eos_table_destroy(phl_eos_table *t);
/* Copy the node data to host: [nx, ny, x0, dx, y0, dy, then per node (x
 * fastest) f, f_x, f_y, f_xx, f_yy, f_xy, f_xxy, f_xyy, f_xxyy] (6 + 9 nx ny
 * doubles); for tests. */
phl_status phl_eos_table_export(const phl_eos_table *t, double *out, long nout);

/* Batch EOS: for each i, temperature from (rho, e_int) by Newton
 * T <- T + (e - e_EoS) / c_v until |de|/e < tol, then one more step
 * (Sect. 2.2); T_inout holds the first guess and receives T.  Outputs (may
 * be NULL except T_inout): P, gamma_e = P/(rho e) + 1, gamma_c = rho c_s^2 / P,
 * c_s, Newton iterations (-1: no convergence).  abar, ye: mean mass number
 * and electron fraction per element.  precision = PHL_FP64: FP64 Newton;
 * PHL_MIXED: FP32 Newton to about 1e-5, finished by FP64 Newton to tol (the
 * iteration count sums both phases).  The iterations evaluate e and c_v
 * only; P, gamma_e, gamma_c once, at the final T.  where = PHL_HOST (host
 * arrays, synchronous) or PHL_DEVICE (device arrays, asynchronous on stream). */
phl_status phl_eos(const phl_eos_table *t, long n, const double *rho, const double *eint,
                   const double *abar, const double *ye, double *T_inout, double *P,
                   double *gamma_e, double *gamma_c, double *cs, int *iters, int precision,
                   double tol, int maxit, int where, void *stream);

/* ---------------------------------------------------------------------------
 * Temperature-guess network for the EOS inversion (not in the paper; the
 * Newton iteration of Sect. 2.2 alone decides the converged T).
 * y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with 3 inputs, two hidden layers
 * of PHL_MLP_HIDDEN units, one output.  Inputs x = ((log10 rho - c0) s0,
 * (log10 e_int - c1) s1, (X_0 - c2) s2), X_0 the first species' mass
 * fraction; output log10 T = c3 + y / s3.  Training runs on the device in
 * FP32 (master weights, Adam); inference uses BF16 weights on the tensor
 * cores with FP32 accumulation, fused into the grid's EOS kernel when
 * desc.use_mlp is set.  Flat FP32 weight layout (PHL_MLP_NPARAM values):
 * W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3. */
#define PHL_MLP_HIDDEN 64
#define PHL_MLP_NPARAM 4481
typedef struct phl_mlp phl_mlp;

typedef struct {
  long nsamples;            /* EOS samples (5% held out for validation)         */
  int epochs;
  long batch;               /* minibatch size                                  */
  double lr;                /* peak Adam step (cosine decay to 0)              */
  unsigned long long seed;  /* SplitMix64 counter-based sample generator       */
  double lrho[2], lT[2];    /* log10 rho and log10 T ranges (uniform)          */
  double A[2], Z[2];        /* the two species; X_0 uniform in [0, 1]          */
} phl_mlp_train_cfg;

typedef struct {
  double final_loss;        /* last minibatch MSE (normalised target)          */
  double val_rms_log10T;    /* held-out error of the BF16 network, in log10 T   */
  double val_max_log10T;
  long steps;
  double seconds;
} phl_mlp_train_stats;

/* Glorot-uniform weights from seed, zero biases.  Errors: PHL_ENOMEM. */
phl_status phl_mlp_create(unsigned long long seed, phl_mlp **out);
void phl_mlp_destroy(phl_mlp *m);
/* Host FP32 weights in the layout above (set also rebuilds the BF16 copy and
 * resets the optimiser state). */
phl_status phl_mlp_set_weights(phl_mlp *m, const float *w);
phl_status phl_mlp_get_weights(const phl_mlp *m, float *w);
/* Affine input/output maps c[4], s[4] (host arrays). */
phl_status phl_mlp_set_norm(phl_mlp *m, const double *c, const double *s);
phl_status phl_mlp_get_norm(const phl_mlp *m, double *c, double *s);
/* Mean squared error over n samples (x[n][3] normalised inputs, t[n] targets)
 * and its gradient (PHL_MLP_NPARAM floats) from the FP32 forward and backward
 * kernels.  where: PHL_HOST or PHL_DEVICE for x, t, grad; loss is host. */
phl_status phl_mlp_loss_grad(phl_mlp *m, long n, const float *x, const float *t, double *loss,
                             float *grad, int where);
/* BF16 tensor-core forward pass on normalised inputs x[n][3] -> y[n]. */
phl_status phl_mlp_forward(const phl_mlp *m, long n, const float *x, float *y, int where);
/* Temperature guesses T[n] (clamped to the table's range) for (rho, e_int, X_0). */
phl_status phl_mlp_guess_temperature(const phl_mlp *m, const phl_eos_table *t, long n, const double *rho,
                           const double *eint, const double *X0, double *T, int where);
/* Generate cfg->nsamples (rho, T, X_0) -> e_int samples with the device EOS
 * on table t, set the affine maps from their ranges, and train.  st may be
 * NULL.  Errors: PHL_EINVAL (arguments, ranges outside the table). */
phl_status phl_mlp_train(phl_mlp *m, const phl_eos_table *t, const phl_mlp_train_cfg *cfg,
                         phl_mlp_train_stats *st);

/* ---------------------------------------------------------------------------
 * Ensembles of independent boxes of uneven sizes (mixed form, ideal gas, no
 * species, SSP-RK3).  Each box is a grid of its own (state I/O through
 * phl_ensemble_grid + phl_set_state / phl_get_state; each box keeps its own
 * CFL step).  phl_ensemble_step runs one persistent cooperative launch per RK
 * stage covering every box and every step of the stage (phases separated by
 * grid-wide barriers); the step's three launches are captured as one CUDA
 * graph and replayed.  Alternatively each phase of a stage is its own launch
 * over all boxes (mode 1), or each box runs its own chain of per-kernel
 * launches on one of several concurrent streams (mode 2); or (mode 3) one
 * persistent cooperative launch per stage runs the fused tile stage over a
 * list of every box's 8^3 tiles, each tile staged by TMA from its box's own
 * tensor map (primitives, raw shock flags, tiles with the flag dilation, edge
 * EMFs and face updates as phases between grid-wide barriers; offered when
 * every box runs the fused stage).  The step is one graph in every mode.
 * The mode and launch shape are chosen by phl_ensemble_autotune or set
 * explicitly. */
typedef struct phl_ensemble phl_ensemble;

typedef struct {
  int mode;                 /* 0: persistent stage kernel; 1: one launch per     */
                            /* phase of the stage (all boxes per launch); 2:     */
                            /* each box's own kernel chain, concurrent streams; */
                            /* 3: persistent stage kernel on the fused tiles    */
  int block;                /* threads per block (128 or 256; modes 0, 1; 288   */
                            /* in mode 3)                                        */
  int blocks_per_sm;        /* modes 0, 3: persistent blocks per SM (mode 3:    */
                            /* fixed by its occupancy)                           */
  int streams;              /* mode 2: concurrent streams                       */
  double ms_per_step;       /* measured (autotune)                              */
} phl_tune_entry;

typedef struct {
  int nbox;
  long cells;               /* total cells of all boxes                         */
  int mode, block, blocks_per_sm, streams;   /* current launch shape            */
  int graph;                /* 1 when the step runs as a captured CUDA graph    */
  int launches_per_step;    /* kernel launches per step (inside the graph)      */
} phl_ensemble_info;

/* descs[nbox]: one description per box (precision PHL_MIXED, PHL_EOS_IDEAL,
 * nspec 0, rk 3, one shared stream; NULL: the ensemble creates a blocking
 * stream of its own, which the default stream's work is ordered with).
 * use_graph != 0 captures the step.
 * Errors: PHL_EINVAL, PHL_EUNSUPPORTED, PHL_ENOMEM, PHL_ECUDA. */
phl_status phl_ensemble_create(const phl_grid_desc *descs, int nbox, int use_graph, phl_ensemble **out);
/* Grid handle of box `box` (owned by the ensemble; do not destroy). */
phl_status phl_ensemble_grid(phl_ensemble *e, int box, phl_grid **g);
phl_status phl_ensemble_step(phl_ensemble *e, int nsteps);
/* Device flags of every box (as phl_check). */
phl_status phl_ensemble_check(phl_ensemble *e);
phl_status phl_ensemble_set_shape(phl_ensemble *e, int mode, int block, int blocks_per_sm, int streams);
/* Time every launch shape for trial_steps steps (state saved and restored)
 * and keep the fastest; out[max] receives the timings (*n entries). */
phl_status phl_ensemble_autotune(phl_ensemble *e, int trial_steps, phl_tune_entry *out, int max, int *n);
phl_status phl_ensemble_get_info(const phl_ensemble *e, phl_ensemble_info *info);
void phl_ensemble_destroy(phl_ensemble *e);

void phl_destroy(phl_grid *g);

/* Message describing the calling thread's last failure ("" if none). */
const char *phl_last_error(void);

/* ---------------------------------------------------------------------
 * Poisson solver for the gravitational potential (Sect. 2.12).
 *
 * Solves sum_axes (L1 phi_{i-1} + L2 phi_i + L3 phi_{i+1}) = 4 pi G rho_i on a
 * Cartesian grid whose axes are stretched independently (Eq. poisson-FD:
 * L1 = 2/(dm (dm+dp)), L2 = -2/(dm dp), L3 = 2/(dp (dm+dp)) with dm, dp the
 * spacings to the neighbouring cell centres), by BiCGSTAB with the Jacobi
 * preconditioner (Sect. 2.12), in FP64 on the device.  Cell centres are the
 * midpoints of the given faces; the ghost centre beyond a side is the mirror
 * image of the first (last) centre in that side.  Boundary values: the
 * multipole expansion of the cell masses rho V about their centre of mass
 * (monopole always; quadrupole for lmax >= 2; octupole for lmax = 3).
 * Convergence: the RMS over cells of the residual weighted by 1/(4 pi G rho)
 * (PHL_POISSON_RELATIVE, Eq. poisson-eps; needs rho > 0 everywhere) or
 * unweighted (PHL_POISSON_ABSOLUTE) below tol, checked after each half and
 * full BiCGSTAB step.
 *
 * Arrays: rho, phi, gx, gy, gz are cell arrays [nz][ny][nx] (x fastest) of
 * doubles in host or device memory as `where` says (PHL_HOST / PHL_DEVICE);
 * the library copies them, never keeps the caller's pointers.  Ghost
 * potentials: x sides [2][nz][ny], then y sides [2][nz][nx], then z sides
 * [2][ny][nx], the lower side first: 2 (ny nz + nx nz + nx ny) doubles. */
enum { PHL_POISSON_RELATIVE = 0, PHL_POISSON_ABSOLUTE = 1 };
typedef struct {
  int n[3];                 /* cells per axis, >= 2 each; at most 2^32 - 2^24 cells */
  const double *xf[3];      /* host: n[d] + 1 increasing face coordinates (read */
                            /* at creation only)                               */
  double G;                 /* gravitational constant, > 0                      */
  int lmax;                 /* 0, 2 or 3                                       */
  int criterion;            /* PHL_POISSON_RELATIVE / PHL_POISSON_ABSOLUTE      */
  double tol;               /* > 0 (the paper's default: 1e-4, relative)        */
  int max_iter;             /* >= 1                                            */
  void *stream;             /* cudaStream_t (null: the legacy default stream)   */
} phl_poisson_desc;
typedef struct phl_poisson phl_poisson;

/* Allocates the solver (12 doubles per cell plus the ghost potentials).
 * PHL_EINVAL (dimensions, faces, lmax, criterion, tol, max_iter, G),
 * PHL_EUNSUPPORTED (more than 2^32 - 2^24 cells), PHL_ENOMEM. */
phl_status phl_poisson_create(const phl_poisson_desc *d, phl_poisson **out);
phl_status phl_poisson_destroy(phl_poisson *p);
/* phi: in, the initial guess; out, the solution.  *iters (nullable): the
 * BiCGSTAB iterations taken; *resid (nullable): the last residual RMS.
 * Synchronous on the solver's stream (it reads the convergence state back
 * once per 16 iterations).  PHL_ENOCONV: max_iter reached (phi holds the
 * last iterate) or a breakdown; PHL_EINVAL: relative criterion with a cell
 * rho <= 0. */
phl_status phl_poisson_solve(phl_poisson *p, const double *rho, double *phi, int where, int *iters, double *resid);
/* The ghost potentials of the last solve (PHL_EINVAL before any solve). */
phl_status phl_poisson_ghost(phl_poisson *p, double *ghost, int where);
/* g = -grad phi at the cell centres by the non-uniform central difference
 * (Eqs. grav_x..grav_z), with the last solve's ghost potentials at the
 * sides.  Synchronous. */
phl_status phl_poisson_gravity(phl_poisson *p, const double *phi, double *gx, double *gy, double *gz, int where);

/* ---------------------------------------------------------------------
 * MHD on a cubed-sphere shell (the stage of Sects. 2.4-2.9 on the grid of
 * Sect. 2.3, in FP64).
 *
 * The shell r_in < r < r_out is covered by six equiangular patches of N x N
 * angular cells (Sect. 2.3) times Nr uniform radial cells.  Patch p has the
 * centre direction c_p, the alpha axis a_p and the beta axis b_p (a x b = c):
 *   p:   0     1     2     3     4     5
 *   c:  +x    +y    -x    -y    +z    -z
 *   a:  +y    -x    -y    +x    +y    +y
 *   b:  +z    +z    +z    +z    -x    +x
 * and the cube-surface point of the angles (alpha, beta) in [-pi/4, pi/4]^2
 * is c + tan(alpha) a + tan(beta) b; grid line m of N sits at the angle
 * (2m - N) pi / (4N).  The paper runs hydrodynamics on this grid; the field
 * here is its extension: magnetic fluxes through the faces advanced by the
 * circulation of Contact-CT edge EMFs (Sect. 2.4, Eq. induction), momentum
 * and field as Cartesian vectors, van Leer PLM along the mesh lines (Sect.
 * 2.5), LHLLD / HLLD / HLL (Sect. 2.6) in each face's normal frame, the
 * deviation form with a radial background (Sect. 2.8), radial gravity and
 * heating, SSP-RK3 (Sect. 2.9), reflecting radial walls.  Ideal gas, or the
 * stellar EOS (Sect. 2.2: ions, radiation, the e-/e+ table) with a uniform
 * composition: a passive scalar that starts uniform stays uniform under a
 * conservative scheme, so the mass fractions enter as constants and are not
 * transported.  The shell's density and pressure are code values; the EOS
 * sees rho * rho_unit (g/cm^3) and P * p_unit (erg/cm^3).
 *
 * State layout (doubles, host or device as `where` says):
 *   cons  [5][6][Nr][N][N]: rho, m_x, m_y, m_z, E (Cartesian components);
 *   pa    [6][Nr][N][N+1]: flux through the alpha faces (i = 0..N), along +a_p;
 *   pb    [6][Nr][N+1][N]: flux through the beta faces (j = 0..N), along +b_p;
 *   pr    [6][Nr+1][N][N]: flux through the radial faces (k = 0..Nr), outwards.
 * A face on a seam between two patches has a copy in each; set_state reads
 * the copy of the lower-numbered array position (alpha before beta, then
 * patch, shell, j, i), get_state writes both, each in its patch's direction.
 * The library copies the arrays; it keeps no caller pointer. */
typedef struct {
  int N, Nr;                /* angular cells per patch side, radial cells; >= 2 */
  double r_in, r_out;       /* 0 < r_in < r_out                                 */
  double gamma;             /* > 1                                              */
  double cfl;               /* Courant number (Eq. cfl), > 0                    */
  int riemann;              /* PHL_LHLLD / PHL_HLLD / PHL_HLL                   */
  double mach_thr;          /* LHLLD Mach threshold, > 0                        */
  int precision;            /* PHL_FP64, or PHL_MIXED: FP64 U^n and face fluxes */
                            /* (FP64 face stages, circulations summed in FP64),*/
                            /* FP32 cell increments, deviations, fluxes, EMFs  */
  const double *rho_c, *p_c;  /* host: hydrostatic background at the shell    */
                              /* middles (Nr each), or both null with rho_f,  */
                              /* p_f: no background (full-state fluxes)       */
  const double *rho_f, *p_f;  /* host: the background at the Nr + 1 radii     */
  const double *g_c;        /* host, nullable: inward gravity per shell (Nr)    */
  const double *heat;       /* host, nullable: heating per unit volume (Nr)     */
  void *stream;             /* cudaStream_t (null: the legacy default stream)   */
  /* stellar EOS (eos = PHL_EOS_STELLAR; zero-initialised fields: ideal gas) */
  int eos;                  /* PHL_EOS_IDEAL (gamma) or PHL_EOS_STELLAR         */
  const struct phl_eos_table *eos_table;  /* the EOS table (not owned)        */
  int nspec;                /* species of the uniform composition, 1..4         */
  double A[PHL_MAXSPEC], Z[PHL_MAXSPEC], X[PHL_MAXSPEC];  /* mass number,    */
                            /* charge, mass fraction of each species            */
  double rho_unit, p_unit;  /* g/cm^3 and erg/cm^3 per code density, pressure   */
  double newton_tol;        /* Newton tolerance (0: 1e-11)                      */
  int newton_maxit;         /* (0: 50)                                          */
  const struct phl_mlp *mlp;  /* nullable: temperature-guess network for cells */
                              /* without a temperature (cold start only)      */
} phl_sphere_desc;
typedef struct phl_sphere phl_sphere;

/* Builds the mesh on the host and uploads it (profiles are read here only).
 * PHL_EINVAL (sizes, radii, gamma, cfl, solver, precision, a partial
 * background, more than 2^31 faces or edges), PHL_ENOMEM.  Device memory:
 * FP64 about 450 bytes per cell, mixed about 270. */
phl_status phl_sphere_create(const phl_sphere_desc *d, phl_sphere **out);
void phl_sphere_destroy(phl_sphere *s);
/* Unique cells, faces (seam faces once) and edges of the mesh. */
phl_status phl_sphere_counts(const phl_sphere *s, long *cells, long *faces, long *edges);
/* Loads a state (layout above).  Host sources: synchronous; device sources:
 * stream-ordered.  Clears the error flags. */
phl_status phl_sphere_set_state(phl_sphere *s, const double *cons, const double *pa, const double *pb,
                                const double *pr, int where);
/* Writes the state back and synchronises the stream; returns PHL_ENEGATIVE or
 * PHL_ENAN when a kernel since set_state met rho <= 0, P <= 0 or a
 * non-finite value. */
phl_status phl_sphere_get_state(phl_sphere *s, double *cons, double *pa, double *pb, double *pr, int where);
/* Loads a state given in primitives (stellar shells are given so: the
 * energy and temperature depend on the EOS): rho, P [6][Nr][N][N] (code
 * units), vel [6][Nr][N][N][3], the fluxes as in set_state.  The cell field
 * is the method's (1/V) sum_f s_f Phi_f x_f; with the stellar EOS each cell's
 * T solves P_EoS(rho, T) = P (Newton on P, bracketed in the table's range)
 * and E = rho e(rho, T) + rho u^2 / 2 + B^2 / 2.  PHL_ENEWTON when a
 * temperature was not found.  Host sources: synchronous. */
phl_status phl_sphere_set_prims(phl_sphere *s, const double *rho, const double *vel, const double *P,
                                const double *pa, const double *pb, const double *pr, int where);
/* Cell temperatures (K) of a stellar shell, [6][Nr][N][N]: each inversion's
 * Newton guess and result.  set: values <= 0 mark cells without one (a cold
 * start: the network's guess where desc.mlp is given, else the shell
 * background's temperature); set_state leaves every cell cold.  get:
 * synchronous for host memory.  PHL_EINVAL on an ideal-gas shell. */
phl_status phl_sphere_set_temperature(phl_sphere *s, const double *T, int where);
phl_status phl_sphere_get_temperature(phl_sphere *s, double *T, int where);
/* The mixed stellar shell's inversion record, rec[8][6][Nr][N][N] (the
 * eight values of phl_get_eos_record per cell); set_state, set_prims and
 * set_temperature clear it.  PHL_EINVAL without one. */
phl_status phl_sphere_get_eos_record(phl_sphere *s, double *rec, int where);
phl_status phl_sphere_set_eos_record(phl_sphere *s, const double *rec, int where);
/* The CFL step of the current state (Eq. cfl with the fast speed along each
 * cell's three mesh directions over the distance between its opposite face
 * centres), to host memory; synchronous. */
phl_status phl_sphere_compute_dt(phl_sphere *s, double *dt_out);
/* nsteps SSP-RK3 steps of size dt (dt <= 0: each step takes its CFL step
 * on the device); asynchronous on the stream.  Errors show in
 * phl_sphere_check / get_state. */
phl_status phl_sphere_step(phl_sphere *s, double dt, int nsteps);
/* on != 0: phl_sphere_step replays one captured CUDA graph per step (the
 * step's launches, captured at the first step of each dt mode: the device
 * CFL step, or a fixed dt, whose value is part of the capture); the
 * results are those of the direct launches.  Needs desc.stream; not used
 * while per-kernel timing is on or for a cold start's first step. */
phl_status phl_sphere_set_graph(phl_sphere *s, int on);
/* Synchronises the stream; PHL_ENEGATIVE / PHL_ENAN as in get_state,
 * PHL_ENEWTON when a stellar inversion did not converge. */
phl_status phl_sphere_check(phl_sphere *s);
/* Per-kernel CUDA-event timing of the sphere's launches, as phl_set_timing /
 * phl_kernel_times for a grid (classes "sph_prim", "sph_flux", "sph_emf",
 * "sph_update_faces", "sph_update_cells", "sph_dt", "set_scalar"). */
phl_status phl_sphere_set_timing(phl_sphere *s, int on);
phl_status phl_sphere_kernel_times(phl_sphere *s, phl_kernel_time *out, int max, int *n, int reset);

#ifdef __cplusplus
}
#endif
#endif /* PHL_H */
