/*
 * fitgb.h -- C ABI of the GB300 FIT leapfrog + ParaExp library (libfitgb.so).
 *
 * Method: Merkel, Niyonzima, Schoeps, "ParaExp using Leapfrog as Integrator
 * for High-Frequency Electromagnetic Simulations".
 *   - Sec. II   FIT grid pair, curls C and C~ = C^T, material matrices
 *               (eq. maxwell_grid1-3), the CFL estimate (eq. cfl), and the
 *               interleaved discrete energy (eq. energy).
 *   - Sec. II-A leapfrog update.
 *   - Sec. III  ParaExp: zero-initial-value window problems, homogeneous
 *               problems, superposition (Algorithm 1, eqs. solution-
 *               particular-paraexp, solution-homogeneous-paraexp,
 *               solution-particular-para, averaging1/2); here the homogeneous
 *               problems are integrated by leapfrog as well.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: nx*ny*nz cells of size dx*dy*dz [m]; PEC walls on all six sides.
 * Per-cell arrays (eps_r, mu_r, sigma, gradients): nx*ny*nz values,
 *   x fastest: c(i,j,k) = i + nx*(j + ny*k).
 * Field arrays ("compact FIT layout"): component-major, then x fastest;
 *   e = [e_x | e_y | e_z], h = [h_x | h_y | h_z], each component nx*ny*nz
 *   values indexed like the cells.
 *   e_a(i,j,k) is the voltage [V] on the primal edge from point (i,j,k) to
 *   (i,j,k)+u_a.  h_a(i,j,k) is the magnetic voltage [A] on the dual edge
 *   through the primal face normal to a whose lowest corner is (i,j,k).
 *   The canonical FIT arrays of the paper have (nx+1)(ny+1)(nz+1) entries
 *   per component; the entries with index nx, ny or nz along any axis are
 *   identically zero under PEC (edges/faces in a wall or outside the box)
 *   and are not stored.  Entries that are not degrees of freedom (e
 *   tangential to a wall, h normal to a wall) are ignored on input and
 *   returned as zero.
 * Precision: a grid is created for FP32, FP64, FP32-with-residual or
 *   compensated-FP32 fields; field arrays passed to it (e_io, h_io) are float
 *   for FP32 and double otherwise.  Probe traces,
 *   energies, superposed fields, J and gradients are always double.
 * Pointers: every array argument may be a host or a device pointer; the
 *   library finds out with cudaPointerGetAttributes.  Device pointers must
 *   be memory of the current device (or managed memory): memory of another
 *   GPU gives FIT_ERR_ARG.  The caller owns all
 *   argument buffers; the library owns the grid and its device workspaces.
 * Streams: work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 *   default stream).  A call whose outputs include a host pointer returns
 *   after the results are on the host; otherwise it may return before the
 *   device work ends.  Errors raised by the device after a call returned
 *   are reported by the next call on that grid or by fit_sync().
 * Errors: every entry point returns a fit_status (0 = success); nothing is
 *   thrown across the ABI.  fit_strerror() describes a status.
 * Threads: a grid is not thread-safe; calls on one grid must not overlap.
 *   Different grids may be used from different threads.  The batched entry
 *   point and the CUDA-graph option synchronize the stream before returning.
 */
#ifndef FITGB_H
#define FITGB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fit_grid fit_grid; /* opaque; owns device state */

typedef enum {
    FIT_OK = 0,
    FIT_ERR_ARG = -1,       /* bad argument (size, index, pointer, count)   */
    FIT_ERR_CFL = -2,       /* dt above the CFL estimate of eq. (cfl)       */
    FIT_ERR_OOM = -3,       /* device allocation failed                     */
    FIT_ERR_CUDA = -4,      /* CUDA runtime error                           */
    FIT_ERR_TIMEOUT = -5,   /* a bounded device wait gave up                */
    FIT_ERR_NONFINITE = -6, /* non-finite or non-positive material value    */
    FIT_ERR_UNSUPPORTED = -7/* valid request the library does not implement */
} fit_status;

/* Source waveforms i(t) [A] of an edge current. */
enum {
    FIT_WAVE_GAUSS_SINE = 0, /* amp*sin(2 pi f0 (t-delay))*exp(-4((t-delay)/width)^2) */
    FIT_WAVE_GAUSS = 1,      /* amp*exp(-4((t-delay)/width)^2), eq. (line_current)    */
    FIT_WAVE_SINE = 2        /* amp*sin(2 pi f0 t)                                    */
};

/* An edge current source: j^{m+1/2} = i(t_{m+1/2}) on the edge along `axis`
 * starting at point (i,j,k).  It must be a degree of freedom (not in a PEC
 * wall).  It enters Ampere's law as  M_eps de/dt = C~h - M_sigma e - j. */
typedef struct {
    int axis, i, j, k;
    int waveform;
    double amp, f0, width, delay;
} fit_source;

/* A probe records the edge voltage e [V] on the edge along `axis` starting
 * at point (i,j,k) (the field value is e / edge length). */
typedef struct {
    int axis, i, j, k;
} fit_probe;

/* Run options; pass NULL for the defaults given in brackets. */
typedef struct {
    int tile_x, tile_y, tile_z; /* CTA tile in cells [0 = autotuned/default] */
    int autotune;               /* 1: time candidate tiles once per shape [0] */
    int use_graph;              /* 1: capture the step loop in CUDA graphs [0]*/
    int sigma_scheme;           /* 0: sigma at (e^n+e^{n+1})/2, 1: at e^n [0] */
    int sum_mode;               /* superposition: 0 FP64, 1 Kahan FP32 [0]    */
    int members_per_pass;       /* ParaExp members advanced per launch;
                                   0 = all K at once (batched), or fewer when
                                   their states pass 96 GiB (larger launches
                                   run slower) or the free device memory;
                                   1 = one member after another (plain
                                   per-window runs) [0]                       */
    int force_dt;               /* 1: accept dt above the CFL estimate [0]    */
    int profile;                /* 1: time every step launch with CUDA events
                                   on the run's stream (fit_last_stats) [0]   */
    int kernel;                 /* step kernel: 1 shared-memory staging by
                                   plain loads, 2 TMA pipeline (FP32 and
                                   precision 40: two cells per thread), 3 the
                                   TMA pipeline with one cell per thread
                                   [0 = 2]                                    */
    int stages;                 /* TMA ring depth in planes, 3 or 4 (FP32
                                   TMA kernels; 0 = the tile's default)       */
    int debug_wait_limit;       /* test hook: polls before a TMA-kernel wait
                                   gives up [0 = about a second]              */
    int debug_extra_tx;         /* test hook: bytes announced on top of the
                                   first plane's copies of every tile, so its
                                   wait can never complete and must time out
                                   (the TMA step kernels, one or two steps per
                                   launch, and the fused Leja pair kernel) [0] */
    int homogeneous;            /* propagator of the homogeneous ParaExp
                                   problems: FIT_HOMOG_LEAPFROG, _LEJA or
                                   _TAYLOR (see paraexp_run) [LEAPFROG]       */
    int expo_substep;           /* Leja/Taylor: substep length in leapfrog
                                   steps (q) [0 = planned, fit_expo_plan]     */
    int expo_degree;            /* Leja/Taylor: even polynomial degree m
                                   [0 = planned]                              */
    double expo_tol;            /* Leja/Taylor: backward-error tolerance
                                   eps_A of ||Delta A|| <= eps_A ||A||
                                   [0 = 1e-12 for FP64 grids, 1e-6 for FP32]  */
    int steps_per_launch;       /* FP32 leapfrog and ParaExp runs without
                                   energy output: 2 advances every member two
                                   steps per launch (temporal blocking: the
                                   fields are read and written once per two
                                   steps), 1 one step [0 = 1]                 */
    int adjoint_mem_mb;         /* fit_adjoint_grad on FP32 grids: device
                                   memory (MiB) it may use to keep the forward
                                   sweep's e^{n+1} - e^n of its last checkpoint
                                   segments, which then need no recompute
                                   (3 floats per cell and kept step) [0]      */
} fit_run_opts;

/* Propagators of the homogeneous problems w_j (opts->homogeneous). */
enum {
    FIT_HOMOG_LEAPFROG = 0, /* leapfrog continued source-free                 */
    FIT_HOMOG_LEJA = 1,     /* Newton interpolation of exp at conjugate Leja
                               points of the spectral interval (Sec. III-B)   */
    FIT_HOMOG_TAYLOR = 2    /* the same with every point at 0: truncated
                               Taylor series (the method of Sec. III-B that
                               the paper reports as the slower one)           */
};

/* Counters of the last leapfrog / ParaExp run on a grid.  step_ms is the
 * summed device time of the fused step launches (only with opts->profile);
 * alg_bytes is the algorithmic DRAM traffic of those launches: per launch,
 * every active member's e and h read once and written once, plus the
 * coefficient arrays read once (shared by all members of the launch). */
typedef struct {
    long long step_launches;    /* fused step kernels launched               */
    long long kernel_launches;  /* all kernels launched by the run           */
    long long cell_updates;     /* sum over launches of cells x members      */
    double alg_bytes;           /* algorithmic bytes of the step launches    */
    double step_ms;             /* device time of the step launches (profile)*/
    long long expo_launches;    /* operator launches of Leja/Taylor runs     */
    long long expo_applications;/* sum over them of cells x members / cells:
                                   applications of the operator A per member
                                   (the SMVP count of the paper)             */
    double expo_alg_bytes;      /* algorithmic bytes of those launches       */
    double expo_ms;             /* their device time (opts->profile)         */
} fit_run_stats;

/* Grid flags */
#define FIT_FLAG_NONE 0u
/* Round the leapfrog coefficients ca, cb, ch to float even on an FP64 grid.
 * FP32 and compensated grids always store float coefficients; with this flag
 * an FP64 grid runs exactly their discretization, so comparing with it
 * measures only the error of the field arithmetic. */
#define FIT_FLAG_COEF_FLOAT 1u

/* Create a grid and upload its per-cell materials.
 *   eps_r (required), mu_r (NULL = 1), sigma [S/m] (NULL = 0): nx*ny*nz.
 *   precision: 32 (float fields), 64 (double fields), 40 or 48:
 *     40: FP32 fields that carry a residual: each value is hi + lo, hi a
 *     float and lo the rounding residual of hi stored as a bfloat16 (6 bytes
 *     per value).  Updates are FP32 arithmetic: the increment is summed into
 *     hi by a fast two-sum and the residual kept; the curl C e of the
 *     magnetic update is formed from two same-component differences made
 *     error-free by two-sums (so a large curl-free part of e cancels
 *     exactly); products with the coefficients are split by one FMA.  About
 *     10x smaller field error than 32 for 1.5x its field bytes.
 *     48: compensated FP32 fields, each value an unevaluated sum hi + lo of
 *     two floats (about 48 significant bits), advanced in FP32 arithmetic
 *     with error-free sums and products.
 *     The field arrays of 40 and 48 (e_io, h_io, e0, h0) are double.  Both
 *     run fit_leapfrog_run and paraexp_run (FP64 superposition, sum_mode 0)
 *     with a TMA kernel; fit_adjoint_grad, fit_expo_propagate and the
 *     exponential homogeneous propagators return FIT_ERR_UNSUPPORTED for
 *     them, and paraexp_run_batched runs their problems one after another.
 * Material matrices (Sec. II, eq. maxwell_grid3): M_eps on an edge is eps0
 * times the area-weighted mean of eps_r over the four cells around it, times
 * dual area / length; M_sigma likewise; M_mu on a face is mu0 times the
 * harmonic mean of mu_r of the two cells sharing it, times area / dual
 * length.  Returns FIT_ERR_NONFINITE if any eps_r or mu_r is not a positive
 * finite number or any sigma is negative or non-finite. */
int fit_grid_create(int nx, int ny, int nz, double dx, double dy, double dz,
                    const float *eps_r, const float *mu_r, const float *sigma,
                    int precision, unsigned flags, fit_grid **out);

/* A graded (tensor-product) grid: cell (i,j,k) measures dx[i] x dy[j] x dz[k]
 * (host arrays of nx, ny, nz sizes [m]); everything else as fit_grid_create.
 * Material matrices with the local sizes (Sec. II, eq. maxwell_grid3):
 *   M_eps(edge along a at q) = eps0 / d_a[q_a] * sum over the four cells
 *     around the edge of eps_r * d_b * d_c / 4 (each cell's part of the dual
 *     facet); M_sigma likewise;
 *   M_mu(face normal to a at q) = mu0 d_b[q_b] d_c[q_c] / s,
 *     s = (d_a[q_a-1]/2)/mu_r(q-u_a) + (d_a[q_a]/2)/mu_r(q).
 * fit_cfl_dt returns eq. (cfl) with each cell's own sizes.  The exponential
 * propagators interpolate on i[-beta, beta] with beta = ||A||_1 (the largest
 * absolute row sum of A, a bound on ||A||_2), since eq. (cfl) is only an
 * estimate on such grids. */
int fit_grid_create_graded(int nx, int ny, int nz, const double *dx, const double *dy, const double *dz,
                           const float *eps_r, const float *mu_r, const float *sigma,
                           int precision, unsigned flags, fit_grid **out);

/* The bound beta >= ||A||_2 of the grid's skew system matrix that the
 * exponential propagators use: 2/dt_CFL on a uniform grid (the bound eq. (cfl)
 * is derived from), ||A||_1 on a graded one. */
int fit_spectral_bound(const fit_grid *g, double *beta);

/* Free the grid and every workspace it owns, after the device has finished
 * all work (cudaDeviceSynchronize).  NULL is accepted. */
void fit_grid_destroy(fit_grid *g);

/* Eq. (cfl): dt_CFL = min over cells of sqrt(eps mu / (1/dx^2+1/dy^2+1/dz^2)).
 * Returns the value in *dt_out. */
int fit_cfl_dt(const fit_grid *g, double *dt_out);

/* Number of cells / field precision of a grid. */
int fit_grid_info(const fit_grid *g, int *nx, int *ny, int *nz, int *precision, int *lossy);

/* Leapfrog run (Sec. II-A), nsteps steps from absolute step step0:
 *   h^{n+1/2} = h^{n-1/2} - dt M_mu^{-1} C e^n
 *   e^{n+1}   = ca e^n + cb (C~ h^{n+1/2} - j^{n+1/2}),
 *   sigma_scheme 0: a = dt M_sigma/(2 M_eps), ca = (1-a)/(1+a),
 *                   cb = dt/(M_eps (1+a));   1: ca = 1-2a, cb = dt/M_eps,
 * with j^{n+1/2} taken at t = (step0 + n + 1/2) dt.
 *   e_io, h_io: 3*nx*ny*nz float/double each; on entry (e^{step0},
 *     h^{step0-1/2}), on exit the final state.  NULL = zero initial state
 *     and no copy-out.
 *   probe_out: nsteps*nprb doubles (row n = e^{step0+n+1} on each probe) or NULL.
 *   energy_out: nsteps doubles, W^n = e^n' M_eps e^n + h^{n-1/2}' M_mu h^{n+1/2}
 *     (interleaved discrete energy, eq. energy) for n = step0..step0+nsteps-1,
 *     or NULL.
 * Fails with FIT_ERR_CFL if dt > fit_cfl_dt unless opts->force_dt. */
int fit_leapfrog_run(fit_grid *g, double dt, long nsteps, long step0,
                     const fit_source *src, int nsrc, const fit_probe *prb, int nprb,
                     double *probe_out, double *energy_out,
                     void *e_io, void *h_io, const fit_run_opts *opts, void *stream);

/* ParaExp with leapfrog members (Sec. III, Algorithm 1).
 *   win: K+1 increasing absolute step bounds W_0 < ... < W_K; window j is
 *     [W_{j-1}, W_j).  Member j (1..K) starts from zero at W_{j-1}, carries
 *     the sources only inside its window (v_j) and continues source-free to
 *     W_K (w_{j+1}).  If e0 or h0 is non-NULL an extra member propagates
 *     that initial state from W_0 with no source (w_1).
 *   probe_out: (W_K-W_0)*nprb doubles, row m = the superposed e at absolute
 *     step W_0+m+1 (the sum of all members, eq. solution-particular-para
 *     with the staggered reconstruction of eqs. averaging1/2).
 *   e_final, h_final: 3*nx*ny*nz doubles each, e^{W_K} and h^{W_K-1/2} of
 *     the sum (either may be NULL).
 *   e0, h0: float/double initial state (grid precision) or NULL.
 * All members are advanced together (coefficients read once per tile for
 * all of them) unless opts->members_per_pass = 1.  Superposition sums are
 * FP64 (or Kahan-compensated FP32 with opts->sum_mode = 1) in a fixed
 * member order, so results do not depend on scheduling.
 * opts->homogeneous = FIT_HOMOG_LEJA or _TAYLOR (lossless FP32/FP64 grids):
 * member j runs leapfrog over its window only (v_j), ending in
 * (e^{W_j}, h^{W_j-1/2}); h is brought to the time of e by a half magnetic
 * step, h^{W_j} = h^{W_j-1/2} - (dt/2) M_mu^{-1} C e^{W_j}, and that state
 * is propagated to W_K by fit_expo_propagate's propagator (w_{j+1});
 * w_1 starts from (e0, h0) the same way.  The homogeneous solutions enter
 * the superposition with e at integer steps and h at half steps (eqs.
 * averaging1/2): h_final holds them at W_K - 1/2.  sum_mode must be 0 and
 * members_per_pass is ignored. */
int paraexp_run(fit_grid *g, double dt, int K, const long *win,
                const fit_source *src, int nsrc, const fit_probe *prb, int nprb,
                double *probe_out, double *e_final, double *h_final,
                const void *e0, const void *h0, const fit_run_opts *opts, void *stream);

/* Exponential propagators (Sec. III-B, "Approximation of the matrix
 * exponential").  On a lossless grid the transformed system of eq.
 * (FIT_ode_2) has the skew matrix A, whose spectrum lies in i[-beta, beta],
 * beta = ||A||_2 <= fit_spectral_bound (2/dt_CFL on uniform grids, the
 * bound behind eq. (cfl)).  With X = (2/beta) A, a substep of q leapfrog
 * steps is exp(c X), c = q dt beta/2 (= q dt/dt_CFL on uniform grids),
 * replaced by the Newton interpolant p_m of exp(c z) at m+1 points of
 * i[-2, 2]:
 *   Leja:   xi_0 = 0, then conjugate pairs +-i eta_j, eta_j the first
 *           maximiser over eta = 2l/2^15 (l = 0..2^15) of the product of
 *           distances to the points chosen before;
 *   Taylor: every point 0.
 * Applied in real arithmetic as
 *   p_m(X) b = b + sum_{j=1}^{m/2} R_{j-1}(X) b (alpha_j + gamma_j X),
 *   R_0 = X, R_j = (X^2 + eta_j^2) R_{j-1},
 * alpha_j = d_{2j-1} - i eta_j d_{2j} and gamma_j = d_{2j}, d_k the divided
 * differences (both real for conjugate points).  Since polynomials of A and
 * of M^{-1}K are similar, the library applies X in the untransformed
 * voltages: X (e, h) = (2/(beta dt)) (cb C~h, -ch C e) on a lossless grid.
 *
 * fit_expo_plan: the substep q (leapfrog steps) and degree m for
 * dt_ratio = dt beta/2, the tolerance eps_A and the field precision
 * (32, 64).  The condition ||Delta A|| <= eps_A ||A|| of Sec. III-D, with
 * ||A|| replaced by beta, holds for a normal A when
 *   max_{z in i[-2,2]} |log(p_m(z) e^{-cz})| + u_p H_m <= 2 c eps_A,
 * evaluated at z = i 2l/4096 (l = 0..4096); H_m = max_z sum_k |d_k w_k(z)|
 * bounds the rounding of the Newton sum (u_p: unit roundoff of the
 * precision); the same must hold with tau c for every output fraction
 * tau = i/q.  Over q with q dt beta/2 <= 32 and even m <= 120 the least m/q
 * wins (ties: smaller q).  Host only (no device work); FIT_ERR_ARG if no
 * pair meets the tolerance. */
int fit_expo_plan(int kind, double dt_ratio, double tol, int precision, int *substep, int *degree);

/* The real coefficients alpha_j, gamma_j, eta_j^2 (j = 1..degree/2) of the
 * interpolant of exp(a z) of the given kind and even degree (a = tau c).
 * Divided differences are the first column of exp(a Z), Z the bidiagonal
 * matrix of the points (Opitz), by scaling and squaring.  Host only. */
int fit_expo_coeffs(int kind, int degree, double a, double *alpha, double *gamma, double *eta2);

/* w(t) = exp((t - t0) A) (e, h): propagate a synchronised state (e and h at
 * the same time t0) over nsteps leapfrog steps with the propagator
 * opts->homogeneous (LEJA or TAYLOR; LEAPFROG is FIT_ERR_ARG).
 *   e_io, h_io: 3*nx*ny*nz float/double (grid precision), the state at t0
 *     on entry and at t0 + nsteps dt on exit.
 *   probe_out: nsteps*nprb doubles, row n = e at t0 + (n+1) dt (dense
 *     output: the Newton basis of a substep serves every step inside it),
 *     or NULL.
 * Lossless FP32/FP64 grids only (FIT_ERR_UNSUPPORTED otherwise). */
int fit_expo_propagate(fit_grid *g, double dt, long nsteps, const fit_probe *prb, int nprb,
                       double *probe_out, void *e_io, void *h_io, const fit_run_opts *opts,
                       void *stream);

/* One ParaExp problem of a batch. */
typedef struct {
    fit_grid *grid;
    double dt;
    int K;
    const long *win;            /* K+1 bounds                               */
    const fit_source *src;
    int nsrc;
    const fit_probe *prb;
    int nprb;
    double *probe_out;          /* (win[K]-win[0])*nprb or NULL             */
    double *e_final, *h_final;  /* 3*ncells each or NULL                    */
} fit_paraexp_problem;

/* Many independent ParaExp problems (grids of any size) advanced together:
 * every member of every problem is one work item of a single persistent,
 * CUDA-graph-captured launch per block of iterations.  Results equal
 * paraexp_run on each problem alone.  With opts->homogeneous set to LEJA or
 * TAYLOR, or opts->steps_per_launch = 2, the problems run one after another
 * through paraexp_run instead. */
int paraexp_run_batched(const fit_paraexp_problem *probs, int nprobs,
                        const fit_run_opts *opts, void *stream);

/* Adjoint gradient of the probe functional
 *   J = sum_{n=1..N} sum_p (e_p^n / L_p)^2      (L_p: length of probe edge p)
 * of a leapfrog run of N = nsteps steps from zero state, with respect to the
 * per-cell eps_r.  The reverse sweep transposes the leapfrog step (derived
 * from Sec. II-A); states are recomputed from checkpoints of (e, h) taken
 * every ckpt_every steps (0 = about sqrt(N)).  J_out: 1 double; grad_eps_r:
 * nx*ny*nz doubles (dJ/d eps_r per cell); both may be host or device, and
 * either may be NULL.  With grad_eps_r NULL only the forward run and J are
 * computed (no checkpoints, no reverse sweep).
 * On a graded grid L_p is the size of the cell the probe edge runs through
 * along its axis, and each cell's share of an edge's M_eps is its own
 * d_b d_c / 4 (the material matrices of fit_grid_create_graded). */
int fit_adjoint_grad(fit_grid *g, double dt, long nsteps,
                     const fit_source *src, int nsrc, const fit_probe *prb, int nprb,
                     int ckpt_every, double *J_out, double *grad_eps_r,
                     const fit_run_opts *opts, void *stream);

/* Counters of the last run on `g` (see fit_run_stats). */
int fit_last_stats(const fit_grid *g, fit_run_stats *out);

/* FP32 leapfrog run that allocates no device memory, for callers that cannot
 * call cudaMalloc (a fixed memory budget handed out up front, a real-time loop
 * where an allocation may block or fail, a plugin that must not grow the
 * process's footprint).  The paper has no counterpart: this is a deployment
 * variant of fit_leapfrog_run for mu_r = 1 and the semi-implicit sigma scheme,
 * without energy output.
 *   eps_r, sigma (NULL = 0): device, nx*ny*nz per-cell values.
 *   e_io, h_io: device, 3*nx*ny*nz floats each (compact layout), the initial
 *     state on entry and the final one on exit (both required).
 *   probe_out: device, nsteps*nprb doubles, or NULL.  src, prb: host arrays.
 * Every workspace lives in one fixed __device__ array of about 30 MiB held
 * by each GPU that loads the library until the process exits, so grids are
 * limited to ceil4(nx)*ny*nz <= 393216 cells (e.g. 64 x 64 x 96); larger
 * grids, more than 8 sources or 32 probes, host pointers or pointers to
 * another GPU's memory, and non-finite spacings or dt give FIT_ERR_ARG.
 * Every call looks the array's address up on the current device
 * (cudaGetSymbolAddress); the first call on a device also loads the
 * library's device code there and should come before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU race on it and
 * must be serialized by the caller.  Returns after the run has finished
 * (FIT_ERR_CFL / FIT_ERR_NONFINITE as fit_leapfrog_run). */
int fit_leapfrog_run_static(int nx, int ny, int nz, double dx, double dy, double dz,
                            const float *eps_r, const float *sigma, double dt, long nsteps, long step0,
                            const fit_source *src, int nsrc, const fit_probe *prb, int nprb,
                            double *probe_out, float *e_io, float *h_io, void *stream);

/* Test hook for the out-of-memory paths: the device allocation `after`
 * allocations from now (0 = the next one) fails as if the device were out of
 * memory, without calling cudaMalloc; every other allocation is made
 * normally.  A negative value turns the hook off.  The failing call returns
 * FIT_ERR_OOM and leaves its grid usable.  The paper has no counterpart. */
int fit_debug_fail_alloc(long long after);

/* Test hook for the z chunk length of the single-grid step launches (host
 * only, no device call): the chunk length, at most kz_max planes, that the
 * library takes for an nx x ny x nz grid cut into tile_x x tile_y tile
 * columns when a launch advances nmem members and `slots` CTAs of the step
 * kernel are resident on the GPU at once.  It minimizes ceil(CTAs / slots) x
 * (chunk + 2), the longest chunk on ties; slots <= 0 gives the fallback rule
 * (halving from kz_max to 8 planes while the launch has fewer than 4 CTAs per
 * SM of 152 SMs).  Returns the length, or FIT_ERR_ARG for a size below 1. */
int fit_debug_chunk_length(int nx, int ny, int nz, int tile_x, int tile_y, int kz_max, int nmem, long long slots);

/* Wait for the grid's outstanding work on `stream` and return the first
 * deferred device error, if any. */
int fit_sync(fit_grid *g, void *stream);

/* Human-readable text of a status (static storage). */
const char *fit_strerror(int status);

/* Library version string (static storage). */
const char *fit_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FITGB_H */
