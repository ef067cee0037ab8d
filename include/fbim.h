/*
 * fbim.h -- C ABI of the GB300 fluctuating boundary integral method (FBIM) library.
 *
 * The library applies the periodic 2D single-layer Stokeslet matrix M of
 * Bao, Rachh, Keaveny, Greengard & Donev, "A fluctuating boundary integral
 * method for Brownian suspensions" (J. Comput. Phys. 2018), by the positively
 * split Ewald sum (Sec. 3.2), solves the first-kind mobility problem (Sec. 3.1,
 * Eq. discreteSaddlePoint) with block-diagonal preconditioned GMRES (Sec. 3.4),
 * draws the random slip M^1/2 W (Sec. 3.3) and advances Brownian rigid bodies
 * with the Euler-Maruyama and Adams-Bashforth random-finite-difference steps (Sec. 4.4,
 * Eqs. EM-RFD, AB2-RFD).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Bodies are indexed beta = 0..n_b-1 and carry the same reference shape,
 *   sampled at n_p equispaced parameters s_j = 2 pi j / n_p (Sec. 3.1).  Node
 *   m = beta * n_p + j sits at x_m = q_beta + R(theta_beta) gamma_ref(s_j).
 * - Q (body coordinates) is double [n_b][3] = (q_x, q_y, theta); F (forces and
 *   torques) and U (velocities and angular velocities) are double [n_b][3].
 * - Node vectors (forces mu, velocities v, slips) are double [n_b * n_p][2],
 *   body-major.  mu_m is the force carried by node m (Sec. 3.1, mu = psi Ds).
 * - "_dev" pointers are device pointers on the handle's device; "_host"
 *   pointers are host memory.  The caller owns every array it passes; the
 *   library owns only its workspace, released by fbim_destroy.
 * - Work is enqueued on the handle's stream (fbim_params.stream).  Calls that
 *   return scalars (iteration counts, residuals) synchronise that stream.
 * - Every call returns an fbim_status; no call aborts the process or throws.
 *   The text of the last error is available from fbim_last_error.
 * - Viscosity eta and kT enter as given; the paper's tests use eta = kT = 1.
 */
#ifndef FBIM_H
#define FBIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbim_handle_s* fbim_handle;

typedef enum {
    FBIM_OK = 0,
    FBIM_ERR_INVALID_ARG = 1,   /* bad size, pointer or parameter                          */
    FBIM_ERR_CUDA = 2,          /* a CUDA / cuFFT / cuBLAS call failed                       */
    FBIM_ERR_OOM = 3,           /* device allocation failed                                  */
    FBIM_ERR_OVERLAP = 4,       /* two bodies' nodes closer than allowed (quadrature breaks) */
    FBIM_ERR_NONFINITE = 5,     /* NaN or Inf in an input or an iterate                      */
    FBIM_ERR_NOT_CONVERGED = 6, /* iteration cap reached; partial result written             */
    FBIM_ERR_TIMEOUT = 7,       /* a bounded device wait expired                             */
    FBIM_ERR_SETUP = 8          /* precomputation failed (rule, eigen gap, ...)             */
} fbim_status;

typedef enum { FBIM_FP64 = 0, FBIM_FP32 = 1 } fbim_precision;

typedef struct {
    int    precision;     /* fbim_precision of the Ewald operator (pairs, spread, FFT, interp).
                             Krylov vectors, residuals and the Alpert band are always FP64.   */
    int    alpert_order;  /* 4 (default) or 8: order of the log-singular correction, Sec. 4.1 */
    int    grid;          /* FFT grid side M (even); <= 0 selects it from tol, Sec. 3.2        */
    int    support;       /* Gaussian support P (odd);  <= 0 selects it from tol, Sec. 3.2     */
    double eta;           /* viscosity, default 1                                               */
    void*  stream;        /* cudaStream_t to enqueue on; NULL = the legacy default stream       */
    int    device;        /* CUDA device ordinal, default 0                                     */
    int    restart;       /* GMRES restart length, default 60                                   */
    int    autotune;      /* wave-space kernels: 1 (default) time both variants at setup and keep
                             the faster; 0 shared-memory tile kernels; 2 warp-per-node kernels */
    int    grid_tune;     /* 1 (default): when grid <= 0, time the FFT of a few admissible sides in
                             [M_min, 1.3 M_min] and keep the cheapest (any side >= the rule's M_min
                             meets tol); 0: use M_min                                          */
    int    split_tune;    /* 0 (default): use r_c as given.  1: treat r_c > 0 as the smallest cutoff
                             and time candidate cutoffs up to 2.2 r_c (xi then follows from r_c and
                             tol; the given xi is ignored) on throwaway handles, keeping the one with
                             the least 25 FP32 + 1 FP64 operator applications + 1 geometry update
                             (one mixed-precision solve; 25 FP64 + 1 update for FBIM_FP64).  Set-up
                             then costs a few handle set-ups more.                               */
    int    fp32_support;  /* Gaussian support of the FP32 operator's wave space (odd; FBIM_FP32
                             handles), at most the FP64 support.  <= 0 (default): the support rule
                             e^{-pi P/2} <= max(tol, 1e-7) -- the FP32 operator's own rounding is
                             ~3e-7, and its refinement corrections need ~1e-4.  Grid, xi and tiles
                             stay those of the FP64 operator.                                    */
    int    tensor_cores;  /* FBIM_FP32 handles: 1 (default) apply the block-diagonal body operators
                             (the preconditioner's M_ref^+ block with its body solve, the square
                             root's G_ref and G_ref^+ blocks) as one tcgen05 tensor-core kernel
                             each, in three-term TF32 (FP32 accuracy), for 2 n_p <= 256; 0 the
                             library GEMM between rotation and body-solve kernels              */
} fbim_params;

/* Ewald parameters the library settled on (fbim_get_info). */
typedef struct {
    int    n_b, n_p, n_nodes;
    double L, xi, r_c, tol;
    int    n_box;         /* cells per side, r_c = L / n_box                      */
    int    grid;          /* M                                                     */
    int    support;       /* P                                                     */
    double eta_s;         /* Gaussian shape parameter of the spreading kernel      */
    double h;             /* grid spacing L / M                                    */
    int    alpert_order, alpert_nodes, alpert_window, alpert_band;
    int    precision;
    int    tile;          /* wave-space tile side (divides grid)                   */
    long long pair_entries;  /* stored real-space pair entries of the handle's precision
                                (ordered pairs within r_c plus sliced-ELL padding)     */
    int    wave_variant;     /* spread kernel in use: 0 tile, 1 warp-per-node          */
    double variant_ms[2];    /* autotuner timings (ms) of the spread per variant       */
    long long launches;      /* kernels this library has launched for the handle so far
                                (library calls such as cuFFT and cuBLAS not included)  */
    int    grid_min;         /* the grid rule's smallest admissible side M_min          */
    double grid_tune_ms;     /* tuned cost (ms) of the chosen side's FFT pair, 0 if untuned */
    int    split_candidates; /* cutoffs the split tuner timed (0: r_c as given)          */
    double split_cost_ms;    /* the chosen cutoff's cost per solve-equivalent (ms)      */
    int    interp_variant;   /* interpolation kernel in use: 0 tile, 1 warp-per-node   */
    double interp_ms[2];     /* autotuner timings (ms) of the interpolation per variant */
    int    support32;        /* Gaussian support of the FP32 operator (FP32 handles; P otherwise) */
    double eta_s32;          /* its Gaussian shape parameter                            */
    int    fp64_fft;         /* transforms and Fourier scale of the FP64 operator: 1 float-
                                float kernels (FP32 handles with an even 5-smooth grid),
                                -1 cuFFT double, 0 not yet set up (first FP64 use)      */
    int    coarse_fallbacks; /* GMRES cycles in which the learned coarse level stagnated
                                (no tenfold residual drop in 20 steps), after which the
                                solve went on with the block-diagonal preconditioner and
                                the coarse level stayed off until the next move          */
} fbim_info;

/* Fill *p with defaults: FP64, order 4, automatic grid and support, eta = 1,
 * default stream, device 0, restart 60. */
fbim_status fbim_default_params(fbim_params* p);

/* Parameter rules of Sec. 3.2 (host only, no device needed).
 * Given the box side L, the cutoff r_c (<= 0: L / 3) and the tolerance tol:
 *   n_box = floor(L / r_c) (>= 3), r_c = L / n_box,
 *   xi    = sqrt(ln(C_r / tol)) / r_c with C_r = 100       (real-space error C_r e^{-xi^2 r_c^2} <= tol),
 *   grid  = smallest even 2^a 3^b 5^c 7^d >= k_max L / pi, with k_max the smallest
 *           wavenumber where C_w H^(k_max) = C_w (1 + q) e^{-q} <= tol, q = k_max^2/4xi^2,
 *           C_w = 1 (the paper's wave-space bound C_w e^{-q} <= tol, with the Hasimoto
 *           prefactor 1 + q kept),
 *   P     = smallest odd >= 2 ln(1/tol) / pi               (NUFFT error e^{-pi P/2} <= tol),
 *   eta_s = (2 w xi / m)^2 with w = P h / 2, m = sqrt(pi P) (Gaussian shape; grid is refined
 *                                                          until eta_s < 1).
 * xi_in > 0 overrides xi.  Any output pointer may be NULL. */
fbim_status fbim_choose_ewald(double L, double r_c, double tol, double xi_in,
                              int* n_box, double* r_c_out, double* xi, int* grid,
                              int* support, double* eta_s);

/* Create a handle for n_b bodies of one shape.
 *   ref_nodes_host: double [n_p][2], gamma_ref(s_j) relative to the tracking point.
 *   Q_host:         double [n_b][3], initial body coordinates.
 *   L:              periodic box side.  r_c: real-space cutoff (<= 0: automatic).
 *   xi:             splitting parameter (<= 0: from tol).  tol: Ewald tolerance.
 *   opt:            NULL for defaults.
 * Precomputes the Alpert band of the reference body (Sec. 3.2, rotated per body),
 * sorts the nodes into cells, plans the FFTs.  Returns FBIM_ERR_OVERLAP if two
 * bodies' nodes are closer than 1e-12 L. */
fbim_status fbim_setup(fbim_handle* out, int n_b, int n_p, const double* ref_nodes_host,
                       const double* Q_host, double L, double r_c, double xi, double tol,
                       const fbim_params* opt);

/* Move the bodies: Q_dev double [n_b][3] (device).  Rebuilds node positions, cells and
 * pair lists, and synchronises the stream to report FBIM_ERR_NONFINITE (non-finite
 * coordinates) or FBIM_ERR_OVERLAP (two nodes coincide). */
fbim_status fbim_update_config(fbim_handle h, const double* Q_dev);

/* Move the bodies to Q + a W (the displaced configurations Q +- delta/2 W~ of the random
 * finite difference, Sec. 4.4, Eq. EM-RFD): Q_dev, W_dev double [n_b][3] (device), the
 * sum formed on the device.  Otherwise as fbim_update_config. */
fbim_status fbim_update_config_displaced(fbim_handle h, const double* Q_dev, double a, const double* W_dev);

/* v = M mu with M = M(t) + M(a)_sym + M(w) (Sec. 3.2).  mu_dev, v_dev: double [N][2]. */
fbim_status fbim_apply_stokeslet(fbim_handle h, const double* mu_dev, double* v_dev);

/* v = M(r) mu = (M(t) + M(a)_sym) mu, the real-space part only (Sec. 3.2, Eq. Mreal-decompose). */
fbim_status fbim_apply_real(fbim_handle h, const double* mu_dev, double* v_dev);

/* v = M(w) mu, the wave-space part only (Sec. 3.2, Eq. Mwave-factorization). */
fbim_status fbim_apply_wave(fbim_handle h, const double* mu_dev, double* v_dev);

/* First-kind mobility solve (Sec. 3.1, Eq. discreteSaddlePoint):
 *     [[M, -K], [-K^T, 0]] [mu; U] = -[slip; F]
 * by right-preconditioned flexible GMRES with the block-diagonal preconditioner
 * of Sec. 3.4.  FP64 handles iterate on the FP64 operator; FP32 handles run
 * iterative refinement (FP64 residual b - A x, FP32-operator corrections).
 *   F_dev:    double [n_b][3] forces and torques (device).
 *   slip_dev: double [N][2] random slip, or NULL for none.
 *   tol:      relative residual |b - A x| / |b| to reach.
 *   max_iter: cap on GMRES iterations (all refinement steps together).
 *   U_dev:    double [n_b][3] output velocities (device).  mu_dev: NULL or double [N][2].
 *   iters, rel_residual: NULL or outputs.  Synchronises the stream.
 * The returned residual: an FBIM_FP64 handle measures it with the FP64 operator at exit.
 * An FBIM_FP32 handle measures it with the FP64 operator after each correction taken
 * from a residual above max(1e-3, 5e4 tol), and afterwards ESTIMATES it: the residual is
 * advanced by r - A_32 d and the last correction's inner GMRES estimate, which saves one
 * FP64 operator application per solve.  That estimate misses (A_64 - A_32) d; the solve
 * bounds it by 3 e32 |d| summed over the estimated corrections (e32 = |(A_32 - A_64) v| /
 * |v|, measured once per handle on a probe vector) and accepts convergence on the
 * estimate only when estimate + bound <= tol, measuring the residual otherwise.
 * fbim_set_residual_audit makes every solve also measure its final residual with the
 * FP64 operator, for checking the estimate.
 * Returns FBIM_ERR_NOT_CONVERGED (with the partial result written) if the cap is hit. */
fbim_status fbim_mobility_solve(fbim_handle h, const double* F_dev, const double* slip_dev, double tol,
                                int max_iter, double* U_dev, double* mu_dev, int* iters,
                                double* rel_residual);

/* One application of the block-diagonal preconditioner of Sec. 3.4 (Eqs.
 * preconditionerGMRES, approximate-body-mobility, M-block-inverse), the one
 * fbim_mobility_solve applies at every GMRES step: per body b, the system
 * [[M~_bb, -K_b], [-K_b^T, 0]] [mu_b; U_b] = [r_mu,b; r_U,b] with M~_bb^+ = R_b M_ref^+ R_b^T
 * (M_ref: the reference body alone in the box), through N~_b = (K_b^T M~_bb^+ K_b)^-1.
 *   in_dev:  double [2N + 3 n_b] = [r_mu (N x 2, body-major); r_U (n_b x 3)] (device).
 *   out_dev: double [2N + 3 n_b] = [mu; U] (device).  Both 16-byte aligned.
 * The handle's precision and kernels, as in the solve (FBIM_FP32 handles: FP32 block
 * operator, on the tensor cores unless fbim_params.tensor_cores = 0; the learned coarse
 * level when it is on).  For a user's own Krylov solver or for tests.  Synchronises. */
fbim_status fbim_precondition(fbim_handle h, const double* in_dev, double* out_dev);

/* Residual audit (tracing; the paper has no counterpart).  With on = 1 every mobility
 * solve of the handle -- also the three inside fbim_rfd_step -- ends with one more
 * FP64 operator application that measures its true relative residual |b - A x| / |b|
 * of the returned [mu; U], and records it beside the residual the solve reports
 * (fbim_mobility_solve: measured or estimated).  The solve's iterates and results are
 * unchanged.  Turning the audit on or off clears the records. */
fbim_status fbim_set_residual_audit(fbim_handle h, int on);

/* The last min(n, kept) audit records, oldest first, into the host arrays reported[n]
 * and measured[n]; *count (NULL allowed) = the number written.  The handle keeps the
 * last 64 records. */
fbim_status fbim_residual_audit(fbim_handle h, int n, double* reported, double* measured, int* count);

/* Random slip v = M^1/2 W with <v v^T> = (2 kT / dt) M by the positive split (Sec. 3.3,
 * Eq. sqrtM-split): sqrt(2 kT/dt) [G^+ (G M(r) G^T)^1/2 W(r) + (M(w))^1/2 W(w)], the
 * near field by preconditioned Lanczos (Sec. 3.4, Eq. preconditioned-real-part) to
 * relative tolerance tol, the far field on the Fourier grid (Eq. sqrtMwave).
 *   W_r_dev: double [N][2] standard normals, or NULL to draw them from Philox
 *            (seed, stream 0, counter) at index 2 m + c.
 *   Z_w_dev: double [M][M][2][2] standard normals (grid index j_y, j_x, component,
 *            real/imaginary; M = fbim_info.grid), or NULL to draw them from Philox
 *            (seed, stream 1, counter) at index ((j_y M + j_x) 2 + comp) 2 + re/im.
 *   Drawn normals are those of fbim_philox_normals; an FBIM_FP32 handle takes the
 *   Box-Muller transform of the same uniforms in FP32 (normals to FP32 rounding).
 *   slip_dev: double [N][2] output.  lanczos_iters: NULL or output.  Synchronises. */
fbim_status fbim_brownian_slip(fbim_handle h, uint64_t seed, uint64_t counter, double kT, double dt,
                               const double* W_r_dev, const double* Z_w_dev, double tol, int max_iter,
                               double* slip_dev, int* lanczos_iters);

/* One Euler-Maruyama step with a random finite difference (Sec. 4.4, Eq. EM-RFD):
 *   Q <- Q + dt N F + sqrt(2 kT dt) N^1/2 W + dt kT/delta [N(Q + delta/2 W~) - N(Q - delta/2 W~)] W~,
 * three saddle solves to tol (the velocity with slip and force, and the two displaced
 * solves with force W~).  The slip's normals are W_r_dev / Z_w_dev or, when NULL, Philox
 * (seed, streams 0 and 1, counter 3 step); W~ is W_t_dev (double [n_b][3]) or Philox
 * (seed, stream 2, counter step).  Q_dev (double [n_b][3], device) is read and
 * overwritten; the handle is left at the new configuration.  iters: NULL or the GMRES
 * iterations of the three solves.  Synchronises the stream. */
fbim_status fbim_rfd_step(fbim_handle h, const double* F_dev, double dt, double kT, double delta, uint64_t seed,
                          uint64_t step, const double* W_r_dev, const double* Z_w_dev, const double* W_t_dev,
                          double tol, int max_iter, double* Q_dev, int* iters);

/* Brownian dynamics step schemes of Sec. 4.4 (fbim_bd_step).  FBIM_EM_NO_RFD is the
 * biased Euler-Maruyama scheme of Sec. 4.4.1 (Eq. EM-noRFD) that omits the stochastic
 * drift; it is there to show what the drift term does (its equilibrium distribution is
 * Eq. biased-dist instead of the Gibbs-Boltzmann one). */
typedef enum { FBIM_EM = 0, FBIM_AB2 = 1, FBIM_EM_NO_RFD = 2 } fbim_scheme;

/* One Brownian dynamics step with a random finite difference (Sec. 4.4):
 *   FBIM_EM  (Eq. EM-RFD): as fbim_rfd_step, three solves.
 *   FBIM_EM_NO_RFD (Eq. EM-noRFD with the force term): Q <- Q + dt N F + sqrt(2 kT dt) N^1/2 W,
 *            one solve (delta, tol_rfd and W~ unused; W~ is not drawn).
 *   FBIM_AB2 (Eq. AB2-RFD): Q <- Q + dt (3/2 N F - 1/2 N_prev F_prev) + sqrt(2 kT dt) N^1/2 W
 *            + dt kT/delta [N(Q + delta/2 W~) - N(Q - delta/2 W~)] W~, four solves (N F, the
 *            slip's velocity with force zero, the RFD pair).
 * The RFD pair is solved to tol_rfd, the other solves to tol (Sec. 4.4.2 uses 1e-3 and
 * 1e-6; tol_rfd = tol reproduces fbim_rfd_step for FBIM_EM).  NF_dev (double [n_b][3],
 * device; FBIM_AB2 only, NULL allowed for FBIM_EM): on entry N_prev F_prev of the previous
 * step when have_prev != 0 (have_prev = 0: the first step, dt N F for the deterministic
 * part), on exit N F of this step.  Noise arguments, Q_dev and iters as in fbim_rfd_step
 * (the slip's Philox counter is 3 step, W~'s counter step).  Synchronises the stream. */
fbim_status fbim_bd_step(fbim_handle h, int scheme, const double* F_dev, double dt, double kT, double delta,
                         uint64_t seed, uint64_t step, const double* W_r_dev, const double* Z_w_dev,
                         const double* W_t_dev, double tol, double tol_rfd, int max_iter, double* NF_dev,
                         int have_prev, double* Q_dev, int* iters);

/* The position update of Eqs. EM-RFD and EM-noRFD for velocities solved elsewhere (for
 * instance by fbim_batch_solve for many independent trajectories at once):
 *   Q[i] += dt U[i] + c (Up[i] - Um[i]),  i < n,   c = dt kT / delta,
 * or Q[i] += dt U[i] when Up_dev and Um_dev are both NULL.  U_dev: the velocities of the
 * solve with the slip and the force; Up_dev, Um_dev: those of the solves with force W~
 * at Q + delta/2 W~ and Q - delta/2 W~.  All device arrays of doubles; asynchronous on
 * stream (a cudaStream_t, NULL = the legacy default stream) of the current device. */
fbim_status fbim_bd_update(void* stream, size_t n, double dt, double c, const double* U_dev, const double* Up_dev,
                           const double* Um_dev, double* Q_dev);

/* n standard normals of (seed, stream, counter) from Philox4x32-10 and Box-Muller:
 * normal i is element i mod 2 of block i / 2, counter block = (i/2 low, i/2 high,
 * stream, counter), key = (seed low, seed high).  out_dev: double [n] (device). */
fbim_status fbim_philox_normals(fbim_handle h, uint64_t seed, uint32_t stream, uint32_t counter, size_t n,
                                double* out_dev);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent suspensions (handles), each with one or more
 * right-hand sides, through one captured CUDA graph per operator application.
 * The batched form of fbim_mobility_solve (Sec. 3.1, Eq. discreteSaddlePoint with
 * the Sec. 3.4 block-diagonal preconditioner): every system (handle k, right-hand
 * side r) is solved to the same relative residual as a single solve would be.
 * ------------------------------------------------------------------------- */
typedef struct fbim_batch_s* fbim_batch;

typedef struct {
    int       n_handles, n_systems;  /* suspensions, systems (handle, right-hand side)          */
    long long n_unknowns;            /* length of the stacked Krylov vectors                    */
    int       restart;               /* GMRES restart of the batch (smallest of the handles')   */
    int       branches;              /* concurrent branches of the captured graphs              */
    long long graph_kernels[7];      /* this library's kernels in each graph: precondition +
                                        saddle FP32, the same FP64, saddle FP32, saddle FP64,
                                        the slip's G M(r) G^T, G^+ and G^+ G (handles' precision)
                                        (0 until the graph is first captured)                   */
    long long launches;              /* this library's kernels run by the batch so far,
                                        graph nodes included (cuFFT, cuBLAS not counted)        */
    long long graph_launches;        /* graph replays so far                                    */
} fbim_batch_info;

/* Group n_handles distinct handles into a batch; handle k gets n_rhs[k] >= 1
 * right-hand sides (n_rhs NULL: one each).  All handles must share device, stream
 * and precision.  Systems are ordered handle-major: system i = (k, r) for k in
 * order and r < n_rhs[k].  The handles stay owned by the caller and must outlive
 * the batch; they may be moved (fbim_update_config, fbim_rfd_step) between batched
 * solves, and the batch recaptures its graphs when a move reallocated a buffer.
 * Allocates the stacked Krylov workspace ((2 restart + 9) doubles per unknown). */
fbim_status fbim_batch_create(fbim_batch* out, int n_handles, const fbim_handle* handles, const int* n_rhs);

/* Solve every system of the batch.
 *   F_dev:    double, the systems' [n_b][3] force blocks stacked in system order (device).
 *   slip_dev: NULL or double, the systems' [N][2] slip blocks stacked the same way.
 *   tol:      relative residual each system must reach (its FP64 operator defines the residual)
 *             (FP32 handles refine: FP64 residuals, FP32-operator corrections).
 *   max_iter: cap on each system's GMRES iterations (all refinement steps together).
 *   U_dev:    double output, the systems' [n_b][3] velocity blocks stacked like F_dev.
 *   iters, rel_residual: NULL or host arrays [n_systems] (iterations and the final
 *             relative residual of every system: measured with the FP64 operators for
 *             FBIM_FP64 handles, estimated after the last small correction for FBIM_FP32
 *             handles, as in fbim_mobility_solve).
 * Synchronises the stream.  FBIM_ERR_NOT_CONVERGED (results written) when a system
 * misses tol within max_iter. */
fbim_status fbim_batch_solve(fbim_batch b, const double* F_dev, const double* slip_dev, double tol, int max_iter,
                             double* U_dev, int* iters, double* rel_residual);

/* Brownian slip of every system of the batch (Sec. 3.3, Eq. sqrtM-split, with the
 * Sec. 3.4 block-diagonal G): system i gets the slip fbim_brownian_slip gives its
 * handle with seed seeds[i] and this counter (Philox normals), up to rounding: the
 * same Lanczos iteration and stopping test per system, run for all systems at once
 * (one graph of G M(r) G^T per step, segmented FP64 Gram-Schmidt, each system frozen
 * once it stops), then a graph of G^+ and each system's far-field noise.
 *   seeds:    host array [n_systems] (distinct seeds give independent slips).
 *   counter:  Philox call counter of every system (fbim_rfd_step uses 3 step).
 *   kT, dt, tol, max_iter: as in fbim_brownian_slip (max_iter <= 1000).
 *   slip_dev: double output [N][2] blocks stacked in system order (the layout of
 *             fbim_batch_solve's slip_dev).
 *   lanczos_iters: NULL or host array [n_systems].
 * Keeps a Lanczos basis of (max_iter + 2) stacked vectors (grown on demand, freed
 * with the batch).  Synchronises the stream.  A system that has not met tol after
 * max_iter steps gets its last iterate, as in fbim_brownian_slip. */
fbim_status fbim_batch_slip(fbim_batch b, const uint64_t* seeds, uint64_t counter, double kT, double dt, double tol,
                            int max_iter, double* slip_dev, int* lanczos_iters);

fbim_status fbim_batch_get_info(fbim_batch b, fbim_batch_info* info);

/* Release the batch's workspace and graphs (not the handles).  NULL is accepted. */
void fbim_batch_destroy(fbim_batch b);

/* Text of the last error of the batch (of the last failed fbim_batch_create when NULL). */
const char* fbim_batch_last_error(fbim_batch b);

/* ---------------------------------------------------------------------------
 * Learned coarse level (an option on top of the Sec. 3.4 block-diagonal
 * preconditioner; the paper has no network).  A multilayer perceptron
 * 6 -> 128 -> 128 -> 128 -> 36 (tanh hidden layers, linear output) maps the
 * geometry of a close body pair to a 6x6 pair-mobility correction C, which the
 * preconditioner adds to the block-diagonal body mobilities.  Matrix products
 * run on the tensor cores with bfloat16 operands and FP32 accumulation; the
 * parameters, activations, gradients and Adam moments are FP32.
 *
 * Parameter vector (float, fbim_mlp_param_count() = 38564 entries): for layers
 * l = 1..4, W_l [n_l][n_(l-1)] row-major then b_l [n_l], widths 6, 128, 128, 128, 36.
 * Network inputs are normalised features x_n = (x - in_shift) / in_scale; outputs y
 * are the normalised 6x6 correction, C = sym(reshape(y * out_scale, 6, 6)).
 * ------------------------------------------------------------------------- */
typedef struct fbim_mlp_s* fbim_mlp;

int fbim_mlp_param_count(void);

/* Create a network for batches of up to max_batch samples on `stream` (cudaStream_t,
 * NULL = legacy default) of `device`.  Parameters start at zero. */
fbim_status fbim_mlp_create(fbim_mlp* out, int max_batch, void* stream, int device);
void fbim_mlp_destroy(fbim_mlp m);
const char* fbim_mlp_last_error(fbim_mlp m);

/* Copy the parameter vector from / to host memory (float [38564]).  Setting the
 * parameters resets the Adam moments and step count.  Synchronises the stream. */
fbim_status fbim_mlp_set_params(fbim_mlp m, const float* theta_host);
fbim_status fbim_mlp_get_params(fbim_mlp m, float* theta_host);

/* Feature normalisation used by the coarse level (host arrays float [6], [6], [36];
 * in_scale > 0). */
fbim_status fbim_mlp_set_normalization(fbim_mlp m, const float* in_shift, const float* in_scale,
                                       const float* out_scale);

/* Y [n][36] = network(X [n][6]) for n <= max_batch (device, float). */
fbim_status fbim_mlp_forward(fbim_mlp m, int n, const float* X_dev, float* Y_dev);

/* Loss (1 / (36 n)) sum (Y - T)^2 of the batch X [n][6], T [n][36] (device, float) and
 * its gradient with respect to the parameter vector into grad_dev (float [38564],
 * device; NULL to skip the copy).  *loss (host, NULL allowed).  Synchronises. */
fbim_status fbim_mlp_gradient(fbim_mlp m, int n, const float* X_dev, const float* T_dev, float* grad_dev,
                              double* loss);

/* One Adam step (Kingma & Ba, Algorithm 1) on the batch's loss gradient: moments
 * m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, theta <- theta - lr m^ / (sqrt(v^) + eps)
 * with m^ = m / (1 - b1^t), v^ = v / (1 - b2^t).  *loss: the loss before the step. */
fbim_status fbim_mlp_adam_step(fbim_mlp m, int n, const float* X_dev, const float* T_dev, float lr, float beta1,
                               float beta2, float eps, double* loss);

/* Kernels the network has launched so far. */
long long fbim_mlp_launches(fbim_mlp m);

/* Close pairs of the handle's current configuration: pairs (a < b, alpha-major) whose
 * smallest node-to-node distance (minimum image) is below g_c, and their features
 * (dx, dy, |d|, cos phi, sin phi, gap): d = q_b - q_a (minimum image) rotated into
 * body a's frame, phi = theta_b - theta_a.  pairs_dev int [max][2], feat_dev double
 * [max][6] (device, either may be NULL); *n_pairs = the number found (all of them
 * even when more than max_pairs; only the first max_pairs are written).  Synchronises. */
fbim_status fbim_coarse_pairs(fbim_handle h, double g_c, int max_pairs, int* pairs_dev, double* feat_dev,
                              int* n_pairs);

/* Turn the learned coarse level on (model non-NULL) or off (NULL).  With it on, every
 * preconditioner application replaces each body's velocity U_b = N~_b a_b by
 * U_b = N~_b a_b + sum over close pairs (p, q) containing b of (C_pq [a_p; a_q])_b and
 * recomputes the body's traction from that U (the body solve of Sec. 3.4 with the
 * mobility N~ + sum C).  C comes from the network at every new configuration; a
 * pair's correction is dropped when blockdiag(N~_p, N~_q) + C_pq is not positive
 * definite or not finite.  A GMRES cycle that does not cut its residual tenfold within
 * 20 steps with the coarse level on falls back to the block-diagonal preconditioner for
 * the rest of the solve and the current configuration (fbim_info.coarse_fallbacks counts
 * these).  The model must outlive its use by the handle and is evaluated on the handle's
 * stream. */
fbim_status fbim_coarse_enable(fbim_handle h, fbim_mlp model, double g_c);

/* Pairs in use and pairs dropped at the last coarse-level setup (NULL allowed). */
fbim_status fbim_coarse_stats(fbim_handle h, int* n_pairs, int* n_rejected);

/* v = (M(t) + M(a)_sym) mu, the same operator as fbim_apply_real, computed without
 * allocating any device memory (the paper has no counterpart: this is a library
 * service).  It is for callers that must not allocate once running, such as a host
 * that gives all device memory to its own pool at start-up or a time-critical loop.
 * Works in FP64 on the handle's cell list (FBIM_FP32 and FBIM_FP64 handles alike:
 * fbim_setup builds the FP64 cell offsets of every handle), with its scratch in a
 * fixed device array of the library (4 MiB per device, held until exit); the handle
 * may have at most 131072 nodes, larger handles get FBIM_ERR_INVALID_ARG.
 * fbim_setup does this entry point's set-up on the handle's device: it looks up the
 * array's address and loads the entry point's kernels (under CUDA's lazy module
 * loading that load would otherwise allocate at the first call), so the call itself
 * neither loads code nor allocates.  All calls share the array and it keeps the last
 * call's contents: calls whose work overlaps on the GPU race and must be serialised
 * by the caller.  Coincident nodes contribute nothing (fbim_setup and
 * fbim_update_config report them as FBIM_ERR_OVERLAP).
 * mu_dev, v_dev: double [N][2], 16-byte aligned. */
fbim_status fbim_apply_real_noalloc(fbim_handle h, const double* mu_dev, double* v_dev);

/* v = M mu with the handle's FP64 operator whatever its precision: the operator of the
 * FP64 refinement residuals (Sec. 3.2 as fbim_apply_stokeslet).  On an FBIM_FP32 handle
 * its real-space kernel values come from the FP32 pair list's pairs, evaluated in
 * float-float arithmetic (about 1e-13 relative); on an FBIM_FP64 handle this is
 * fbim_apply_stokeslet. */
fbim_status fbim_apply_stokeslet_fp64(fbim_handle h, const double* mu_dev, double* v_dev);

/* ---------------------------------------------------------------------------
 * Second-kind reference solver (App. B): the completed double-layer formulation,
 *     u + omega (x - q)^perp = 1/2 phi + D phi + sum_b [G(x - q_b) f_b + R(x - q_b) tau_b],
 *     u = (1/|Gamma|) int phi dS,  omega = (1/W) int phi . (x - q)^perp dS,
 * periodised with the Hasimoto split of the Stokeslet, rotlet and stresslet (App. B),
 * trapezoidal rule at the handle's nodes (spectrally accurate on smooth, separated
 * bodies), FP64 throughout, GMRES without preconditioning.  It reuses the handle's
 * geometry, cells, r_c, xi and FP64 wave grid (M, P, eta_s); the stresslet and rotlet
 * decay one power of k slower in wave space than the Stokeslet, so a grid somewhat
 * finer than the first kind's keeps the same tolerance.  Needs n_box >= 3.  The state
 * (FFT plans, workspace: about (restart + 6) vectors of 2N + 3N_b doubles plus 8 M^2
 * doubles) is built on first use and freed with the handle.  Readings: S_lm =
 * phi_l n_m dS with n pointing into the body; the mean-flow term (1/V) sum x_s (phi . n)
 * dS; the trapezoidal self term -(1/4 pi) 2 kappa (t t^T) phi dS; perp counter-clockwise.
 * ------------------------------------------------------------------------- */

/* Solve the second-kind mobility problem for forces and torques F_dev [n_b][3]: U_dev
 * [n_b][3] velocities, phi_dev NULL or [N][2] double-layer density.  iters: GMRES
 * iterations; rel_residual: the measured |b - A x| / |b|.  FBIM_ERR_NOT_CONVERGED
 * (results written) when tol is missed within max_iter.  Synchronises the stream. */
fbim_status fbim_second_kind_solve(fbim_handle h, const double* F_dev, double tol, int max_iter, double* U_dev,
                                   double* phi_dev, int* iters, double* rel_residual);

/* y = A x for x = [phi (2N); U (3 n_b)] (device, not aliased): node rows
 * u + omega (x - q)^perp - 1/2 phi - D phi, closure rows |Gamma| u - int phi dS and
 * W omega - int phi . (x - q)^perp dS.  Synchronises the stream. */
fbim_status fbim_second_kind_apply(fbim_handle h, const double* x_dev, double* y_dev);

/* b = [C F; 0] (2N + 3 n_b doubles, device): the periodic Stokeslets and rotlets of the
 * bodies' forces and torques at every node.  Synchronises the stream. */
fbim_status fbim_second_kind_rhs(fbim_handle h, const double* F_dev, double* b_dev);

/* Information about the handle's parameters. */
fbim_status fbim_get_info(fbim_handle h, fbim_info* info);

/* Per-stage CUDA-event timers of the operator (tracing).  With timing on, every
 * operator call records an event after each stage on the handle's stream and
 * synchronises at its end; fbim_stage_times returns the accumulated milliseconds
 * and call counts of the stages, in this order: gather, spread, forward FFT,
 * Fourier scale, inverse FFT, real-space pairs, interpolation, finish (scatter +
 * Alpert band).  Turning timing on or off resets the accumulators. */
fbim_status fbim_set_timing(fbim_handle h, int on);
fbim_status fbim_stage_times(fbim_handle h, double* ms, long long* calls, int n);

/* Release the handle and its device workspace.  NULL is accepted. */
void fbim_destroy(fbim_handle h);

/* Text of the last error on h (or of the last failed fbim_setup when h is NULL). */
const char* fbim_last_error(fbim_handle h);

/* Host E1(z) as used by the library's setup (exponential integral, Sec. 3.2 Eq. expint);
 * exported so that its accuracy can be tested without a GPU. */
double fbim_host_expint_e1(double z);

/* Nodes v_k and weights w_k of the library's log-singular end correction (Sec. 3.1) and
 * its window a; v and w must hold order - 1 doubles.  Host only. */
fbim_status fbim_host_alpert_rule(int order, double* v, double* w, int* a);

/* Coefficients c = wnorm f(T) e_1, f = sqrt with negative Ritz values clipped to zero, of
 * the Lanczos approximation V c to A^1/2 w (Sec. 3.3) from the k x k symmetric tridiagonal
 * T (alpha[k] diagonal, beta[k - 1] off-diagonal): the host routine of fbim_brownian_slip
 * and fbim_batch_slip, exported so that it can be tested without a GPU.  out: double [k].
 * FBIM_ERR_INVALID_ARG for k < 1 or NULL pointers.  Host only. */
fbim_status fbim_host_lanczos_sqrt(const double* alpha, const double* beta, int k, double wnorm, double* out);

#ifdef __cplusplus
}
#endif
#endif /* FBIM_H */
