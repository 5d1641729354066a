/*
 * rlbm.h -- C ABI of librlbm.so: the fused streaming + Anderson-Witting
 * collision step of the relativistic lattice Boltzmann method for a massless
 * gas in (2+1) dimensions (Bazzanini, Gabbana, Simeoni, Succi, Tripiccione,
 * arXiv 2011.06856), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: lattice units, dx = dy = dt = 1, c = 1 (Sec. 2).  tau is the
 *   relaxation time in time steps; tau = +INFINITY is the free-streaming
 *   (ballistic) limit used in Fig. 2 and Appendix A.
 * Quadrature (Sec. 2.3, Eq. off-lattice-quad): order N, N+1 radial
 *   Gauss-Laguerre nodes p_r (roots of L_{N+1}), K angles per shell,
 *   theta_rj = (j + r/(N+1)) 2 pi / K, N_pop = K (N+1), shell-major
 *   population index i = r K + j.  Requires N >= 2 (the collision conserves
 *   N^0 and T^{0 nu} only from N = 2 on) and K >= 2N+1.
 * Populations: structure of arrays f[i][y][x], x fastest, S = nx * ny sites.
 *   Precision RLBM_FP64 / RLBM_FP32 stores f_i itself.  The 16-bit forms
 *   store f_i relative to the rest equilibrium at n = 1, T = 1, for which
 *   f^rest_i = w_i / (2 pi) exactly: *_DEV stores s_i = f_i / f^rest_i - 1,
 *   *_NORM stores s_i = f_i / f^rest_i; arithmetic in FP32.  Steps write them
 *   with stochastic rounding (counter-based random bits, reproducible: the
 *   stream of random bits is a function of site, population and step number,
 *   so a run resumed from a checkpoint at step k repeats the original run);
 *   the initial state is rounded to nearest.
 * Macroscopic fields: double arrays of S values, [y][x].  Velocities are
 *   given as beta = (u_x, u_y), |beta| < 1; U^a = gamma (1, beta).
 * Pointers: "host" pointers are ordinary CPU memory, "device" pointers are
 *   CUDA global memory on the handle's device.  Host arrays are owned by the
 *   caller and only accessed during the call.
 * Streams: all GPU work of a handle is issued on the stream given at
 *   creation (NULL: a private non-blocking stream the library creates).
 *   Entry points that take or return host data synchronise that stream.
 * Errors: every entry point returns an rlbm_status; nothing aborts or traps.
 *   rlbm_last_error() gives the message of the latest failure of a handle.
 *   A non-physical cell (no timelike eigenvector, n <= 0 or eps <= 0) sets a
 *   device status word; the next synchronising call returns
 *   RLBM_ERR_UNPHYSICAL (and clears it).
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlbm rlbm_t; /* opaque handle, owned by the library */

typedef enum {
    RLBM_OK = 0,
    RLBM_ERR_ARG = 1,        /* invalid argument; nothing was changed */
    RLBM_ERR_CUDA = 2,       /* a CUDA runtime call failed; see rlbm_last_error */
    RLBM_ERR_OOM = 3,        /* device allocation failed */
    RLBM_ERR_UNPHYSICAL = 4, /* a cell had no physical Landau frame */
    RLBM_ERR_TIMEOUT = 5,    /* a bounded device wait ran out */
    RLBM_ERR_UNSUPPORTED = 6 /* valid but not built (e.g. an (N, K) with no kernel) */
} rlbm_status;

/* Storage precision and the arithmetic that goes with it.  The per-site part
 * of a step is the moment fold (Eq. discrete_sum_moments), the Landau frame
 * (Sec. 2.2) and the equilibrium coefficients (Eq. mj-feq-expansion-truncated).
 *  - RLBM_FP64: FP64 throughout.
 *  - RLBM_FP32: FP32 per-population arithmetic; the per-site part at FP64-class
 *    accuracy (double-float, pairs of FP32, in the two-sites-per-lane kernels;
 *    FP64 in the others).  In FP32 it would carry the conserved moments to a
 *    relative bias of about 4e-7 per step, which the collision accumulates.
 *  - 16-bit forms: FP32 per-population arithmetic and moment accumulation,
 *    the Landau frame solved in double-float (the storage rounding, about
 *    3e-4 over a run, sets their error). */
typedef enum {
    RLBM_FP64 = 0,      /* FP64 storage and arithmetic */
    RLBM_FP32 = 1,      /* FP32 storage and per-population arithmetic */
    RLBM_FP16_DEV = 2,  /* FP16 s = f / f^rest - 1 (deviation from the rest equilibrium) */
    RLBM_BF16_DEV = 3,  /* BF16 s = f / f^rest - 1 */
    RLBM_FP16_NORM = 4, /* FP16 s = f / f^rest (normalised by the rest equilibrium) */
    RLBM_BF16_NORM = 5  /* BF16 s = f / f^rest */
} rlbm_precision;

typedef enum { RLBM_BC_PERIODIC = 0, RLBM_BC_COPYOUT = 1 } rlbm_bc;

/* Grid and boundary conditions.  Periodic wraps the source index of the
 * streaming pull; copy-out clamps it into the grid (zero-gradient ghost cell). */
typedef struct {
    int nx, ny;
    int bc_x, bc_y; /* rlbm_bc */
} rlbm_grid;

/* Quadrature tables of Sec. 2.3, Eq. (off-lattice-quad): for N >= 0 and
 * K >= 2N+1, writes N_pop = K (N+1) values to each host array:
 * p0 = p_r, vx = cos theta_rj, vy = sin theta_rj, w = w^(p)_r 2 pi / K with
 * w^(p)_r = p_r / ((N+2)^2 L_{N+2}(p_r)^2).  Any pointer may be NULL. */
rlbm_status rlbm_quadrature(int order_N, int angles_K, double *p0, double *vx, double *vy,
                            double *w);

/* Bytes of ONE population buffer (N_pop * nx * ny elements of the storage
 * type); the handle uses two of them (ping-pong, pull streaming). */
size_t rlbm_population_bytes(rlbm_grid grid, int order_N, int angles_K, int precision);

/* Create a handle for one problem.  Validates N >= 2, K >= 2N+1, nx, ny >= 1,
 * tau > 0 (or +INFINITY), bc values and precision; RLBM_ERR_ARG otherwise.
 * RLBM_ERR_UNSUPPORTED for N > 5 (the kernels are compiled for N = 2..5; the
 * two-sites-per-lane, TMA-staged and batched kernels for N = 2, 3) and for K
 * beyond one population group per warp in 16-bit storage
 * (rlbm_population_groups).
 * dev_buffers: optional caller-owned device memory of at least
 * 2 * rlbm_population_bytes() bytes, 256-byte aligned, holding both
 * population buffers (it must outlive the handle); NULL makes the library
 * allocate and own them.  The handle always allocates its small constant
 * tables and a status word.  cuda_stream: a cudaStream_t or NULL. */
rlbm_status rlbm_create(rlbm_t **out, rlbm_grid grid, int order_N, int angles_K, double tau,
                        int precision, void *cuda_stream, void *dev_buffers,
                        size_t dev_buffer_bytes);

/* Create a handle for the on-lattice rule of Sec. 2.3 (Fig. 1, left; the
 * quadrature with prescribed abscissas): order N = 3, the 12 integer stencil
 * vectors n of length 5 ((+-5,0), (0,+-5), (+-3,+-4), (+-4,+-3)) on each of the 4
 * Gauss-Laguerre energy shells, N_pop = 48, momenta p_r (1, n/5), weights
 * satisfying the orthonormal conditions (Eq. mj-orthogonal-conditions) as a
 * product of the radial Gauss-Laguerre weights and two angular weights (axis and
 * off-axis vectors).  Populations are shell-major, i = 12 r + j, the vectors
 * ordered by angle from 0.  Streaming is perfect: population i moves by its
 * stencil vector n_i, 5 cells per step, with no interpolation (so the speed of
 * light is 5 cells per step; boundary conditions as for rlbm_create: periodic
 * wrap or copy-out clamp of the source cell).  Equilibrium, Landau frame and
 * collision are those of rlbm_create.  FP32 and FP64 storage only
 * (RLBM_ERR_UNSUPPORTED otherwise: the 16-bit forms scale by one weight per
 * shell); the per-tile kernel with 12 populations per warp only (rlbm_set_tiling
 * refuses anything else).  Other arguments and errors as for rlbm_create. */
rlbm_status rlbm_create_onlattice(rlbm_t **out, rlbm_grid grid, double tau, int precision,
                                  void *cuda_stream, void *dev_buffers, size_t dev_buffer_bytes);

/* 1 if the handle uses the on-lattice rule, 0 if the off-lattice one, -1 for NULL. */
int rlbm_is_onlattice(const rlbm_t *h);

/* Equilibrium statistic of Eq. (feq_dist), f^eq = g / (z^-1 exp(U.p/T) + s):
 * statistics s = 0 Maxwell-Juttner (the default; g unused), +1 Fermi-Dirac,
 * -1 Bose-Einstein (Sec. 2.1: the quadratures apply unchanged).  For s != 0 the
 * Landau frame gives n and the energy density e, and the per-site step solves
 * n = 2 pi g T^2 phi_2(z), e = 4 pi g T^3 phi_3(z) for (T, z) (phi_s = -Li_s(-z)
 * or Li_s(z)); the projection weights of the truncated equilibrium use the
 * radial moments 2 pi g T^(k+1) phi_{k+1}(z).  rlbm_init takes (n, T) and finds z
 * from n; rlbm_moments reports this T.  A Bose-Einstein state beyond
 * condensation (no z < 1) is RLBM_ERR_UNPHYSICAL, as a failed Landau frame.
 * Needs g > 0 (RLBM_ERR_ARG); FP64 or FP32 storage, N = 2 or 3 and the
 * off-lattice rule (RLBM_ERR_UNSUPPORTED otherwise).  The per-site part runs in
 * FP64 and the per-tile kernel is used.  Synchronises the stream; the stored
 * populations are kept (call rlbm_init afterwards to start from an equilibrium
 * of the new statistic). */
rlbm_status rlbm_set_statistics(rlbm_t *h, int statistics, double g);

/* The handle's statistic (0, 1, -1), or -2 for NULL. */
int rlbm_statistics(const rlbm_t *h);

/* Host evaluation of the routine the kernels use for the quantum statistics:
 * phi_s(z) at eta = ln z, s = 0..6, statistics +1 (-Li_s(-z)) or -1 (Li_s(z),
 * eta < 0).  NaN for arguments outside that range.  No GPU needed. */
double rlbm_quantum_phi(int s, double eta, int statistics);

/* Host evaluation of the kernels' (eta, T) solve for the quantum statistics:
 * the equilibrium of statistics +1 / -1 and degeneracy g > 0 with density
 * n > 0 and energy density e > 0 (2 pi g T^2 phi_2 = n, 4 pi g T^3 phi_3 = e).
 * eta0: a start (the previous step's eta of a site), or NaN for the
 * Maxwell-Boltzmann start.  fp32_storage != 0: the stopping rule of the
 * FP32-storage kernels (FP64 Newton steps stop below 1e-5 (1 + |eta|): eta
 * within about 1e-12 from a start near the root, 1e-9 from a cold one), else
 * that of FP64 storage (below 1e-10: exact to rounding).  Writes eta and T (neither may be NULL) and returns 1, or 0 where
 * no equilibrium exists (Bose-Einstein beyond condensation) or the input is
 * not physical (eta and T are then written but meaningless).  No GPU needed. */
int rlbm_quantum_solve(double n, double e, double g, int statistics, double eta0, int fp32_storage,
                       double *eta, double *T);

void rlbm_destroy(rlbm_t *h);

/* Message of the most recent failure on h (or of the last failed create when
 * h is NULL).  Valid until the next call on h. */
const char *rlbm_last_error(const rlbm_t *h);

/* Equilibrium initial state, f_i = f^eq_i(n, T, U) of Eq.
 * (mj-feq-expansion-truncated) at every site, from host fields (S doubles
 * each).  Resets the step counter.  Synchronises the stream. */
rlbm_status rlbm_init(rlbm_t *h, const double *n, const double *T, const double *beta_x,
                      const double *beta_y);

/* Same from device fields; asynchronous on the handle's stream. */
rlbm_status rlbm_init_device(rlbm_t *h, const double *d_n, const double *d_T,
                             const double *d_beta_x, const double *d_beta_y);

/* Advance nsteps >= 0 time steps, asynchronously.  One step is Sec. 2.2 in
 * order: bilinear pull streaming (Eqs. streaming, interpolation), moments
 * N^a, T^ab of the streamed populations (Eq. discrete_sum_moments), the
 * Landau frame eps U^a = T^ab U_b with n = U_a N^a and T = eps/(2n), the
 * truncated equilibrium, and relaxation f <- f* - (p.U / p^0 tau)(f* - f^eq)
 * (Eq. discrete-rbe), fused in one kernel per step (one read and one write
 * of every population).  Steps are replayed from a captured CUDA graph. */
rlbm_status rlbm_step(rlbm_t *h, int nsteps);

/* Landau-frame fields of the stored populations (no streaming): n, eps, T,
 * U^0, U^x, U^y, S doubles each.  Host pointers; synchronises; reports and
 * clears RLBM_ERR_UNPHYSICAL. */
rlbm_status rlbm_moments(rlbm_t *h, double *n, double *eps, double *T, double *U0, double *Ux,
                         double *Uy);

/* Same into device pointers, asynchronously (no status check). */
rlbm_status rlbm_moments_device(rlbm_t *h, double *d_n, double *d_eps, double *d_T,
                                double *d_U0, double *d_Ux, double *d_Uy);

/* Checkpoint / resume: copy the current population buffer (raw storage
 * format, rlbm_population_bytes() bytes) to or from host memory.  Both
 * synchronise.  set also restores the step counter to `step`. */
rlbm_status rlbm_get_populations(rlbm_t *h, void *host, size_t bytes);
rlbm_status rlbm_set_populations(rlbm_t *h, const void *host, size_t bytes, long long step);

/* Device address of the current population buffer (valid until the next
 * rlbm_step) and the number of completed steps. */
void *rlbm_current_buffer(rlbm_t *h);
long long rlbm_steps_done(const rlbm_t *h);

/* Wait for the handle's stream; returns RLBM_ERR_UNPHYSICAL (and clears the
 * flag) if any cell was non-physical since the last check. */
rlbm_status rlbm_sync(rlbm_t *h);

/* Number of kernel launches the handle has issued (graph replays count
 * every kernel node). */
long long rlbm_kernel_launches(const rlbm_t *h);

/* Which step kernel the handle uses: 1 = persistent TMA-staged kernel
 * (row pitch a multiple of 16 bytes and nx >= one box), 2 = two sites per
 * lane (64-site tiles, packed f32x2 arithmetic; FP32 arithmetic, finite tau,
 * nx even, K a multiple of P in {8, 12, 16, 24, 32}, at most 16 warps),
 * 3 = the same with its first pass staged through shared memory by
 * cp.async.bulk on interior tiles (row pitch a multiple of 16 bytes; bounded
 * mbarrier waits), 4 = the same arithmetic with the whole 64-site tile staged
 * into shared memory by TMA at the CTA's start (cp.async.bulk.tensor: the
 * centre row and the upwind pull row of every population, the pull rows in
 * chunks of 4 or 8 populations that share sgn(v_y); row pitch a multiple of
 * 16 bytes, nx >= 64 + 32 bytes of halo, one population group; bounded
 * mbarrier wait; 16-bit stores round stochastically with cvt.rs),
 * 0 = per-tile kernel. */
int rlbm_step_kernel_variant(const rlbm_t *h);

/* Select the tiling and step kernel directly (no counterpart in the paper:
 * a performance choice that does not change what a step computes beyond
 * rounding).  P = populations per warp (one of 8, 12, 16, 24, 32, 48, 64 that
 * fits K and N); kind = 0 per-tile, 1 persistent TMA-staged, 2 two sites per
 * lane, 3 two sites per lane with bulk-staged loads, 4 two sites per lane
 * with the tile staged by TMA.  RLBM_ERR_UNSUPPORTED if the kernel is not
 * possible for this handle (the handle then keeps tiling P with the per-tile
 * kernel); RLBM_ERR_ARG for a kind outside 0..4.
 * Synchronises the stream; the state is kept. */
rlbm_status rlbm_set_tiling(rlbm_t *h, int P, int kind);

/* Populations per warp of the handle's current tiling (the tile is 32 sites
 * of one row x all populations; G = ceil(K / P) (N+1) warps per CTA). */
int rlbm_tile_populations(const rlbm_t *h);

/* Groups of P populations each warp of the per-tile kernel owns: 1, unless K
 * exceeds what one group per warp holds (K > 64 floor(16 / (N+1)), e.g. the
 * paper's K = 600 reference runs with N = 3).  Then floor(16 / (N+1)) warps
 * per shell own ceil(K / (warps P)) groups each; the streamed values of all
 * but the last group are parked in the output buffer between the two passes
 * (FP32 and FP64 storage; rlbm_create refuses such K in 16-bit storage).
 * The per-tile kernel and, in FP32 storage with K a multiple of P, the
 * two-sites-per-lane kernel (without staging) apply.  -1 for a NULL handle. */
int rlbm_population_groups(const rlbm_t *h);

/* Autotuner: time every compiled tiling of the step kernel (P populations per
 * warp in {8,12,16,24,32,48,64} that fits K and N, each with the four
 * two-sites-per-lane forms and the persistent TMA-staged kernel where
 * possible and with the per-tile kernel) on this
 * handle's own problem, launches_per_trial launches each, and keep the
 * fastest.  The populations of the current state are not modified (trials
 * read the current buffer and write the other one).  Results are cached per
 * (grid, N, K, precision, boundary conditions) for the life of the process.
 * best_ms (may be NULL) receives the time of one step launch with the chosen
 * tiling.  Synchronises the stream. */
rlbm_status rlbm_autotune(rlbm_t *h, int launches_per_trial, float *best_ms);

/* Bound, in SM clock cycles, of every mbarrier wait in the TMA-staged, the
 * tile-staged and the bulk-staged step kernels (default 4e9, about 2 s).  A wait that runs out
 * makes the kernel record RLBM_ERR_TIMEOUT, drain its own copies (bounded) and
 * skip its stores; the next synchronising call reports it.  cycles >= 1000. */
rlbm_status rlbm_set_wait_limit(rlbm_t *h, long long cycles);

/* Test hook for the timeout path: the next step launch expects 16 bytes more
 * than its copies deliver, so its waits run out after the wait limit.
 * RLBM_ERR_UNSUPPORTED when the step kernel has no device waits (per-tile,
 * two sites per lane without staging). */
rlbm_status rlbm_test_stall_next_step(rlbm_t *h);

/* ------------------------------------------------------------------ */
/* Batched persistent form: many independent problems, one launch       */
/* ------------------------------------------------------------------ */

typedef struct rlbm_batch rlbm_batch_t; /* opaque, owned by the library */

/* One problem of a batch: grid, boundary conditions, K angles, tau. */
typedef struct {
    int nx, ny;
    int bc_x, bc_y;
    int angles_K;
    double tau;
} rlbm_problem;

/* Bytes of device memory holding both population buffers of every problem
 * (each problem's pair starts on a 256-byte boundary). */
size_t rlbm_batch_arena_bytes(const rlbm_problem *problems, int count, int order_N, int precision);

/* Create a batch of `count` independent problems sharing the order N and the
 * storage precision (RLBM_FP64 or RLBM_FP32).  Every problem needs a tiling
 * whose warps per tile divide the 6-warp CTA: N = 2 with K <= 64 (N = 3 has
 * none: RLBM_ERR_UNSUPPORTED).  dev_arena: caller-owned device memory of
 * rlbm_batch_arena_bytes() bytes, 256-byte aligned, or NULL (the library
 * allocates).  The problems are also reachable as single handles through
 * rlbm_batch_problem() for init, moments and checkpoints. */
rlbm_status rlbm_batch_create(rlbm_batch_t **out, const rlbm_problem *problems, int count,
                              int order_N, int precision, void *cuda_stream, void *dev_arena,
                              size_t arena_bytes);
void rlbm_batch_destroy(rlbm_batch_t *b);
const char *rlbm_batch_last_error(const rlbm_batch_t *b);
int rlbm_batch_count(const rlbm_batch_t *b);

/* Handle of problem i (owned by the batch; do not destroy).  Use rlbm_init,
 * rlbm_init_device, rlbm_moments, rlbm_get/set_populations on it; do not call
 * rlbm_step on it while the batch is in use. */
rlbm_t *rlbm_batch_problem(rlbm_batch_t *b, int i);

/* Advance every problem nsteps time steps (Sec. 2.2, the same fused step as
 * rlbm_step).  Mode 0 (the default): ONE persistent cooperative kernel
 * launch, replayed from a CUDA graph captured per nsteps; work units (tiles
 * of 32 sites of one row of one problem) are taken dynamically from a
 * counter; time steps are separated by a grid barrier whose waits are
 * bounded (RLBM_ERR_TIMEOUT at the next rlbm_batch_sync).  Mode 1: the
 * problems are independent, so each runs its own single-problem step kernel
 * (its own tiling), all nsteps steps back to back, on one of 16 streams
 * forked from and joined back to the batch stream (problems balanced over
 * the streams by size).  Asynchronous. */
rlbm_status rlbm_batch_step(rlbm_batch_t *b, int nsteps);

/* Select the execution mode (0 persistent launch, 1 stream pool; no
 * counterpart in the paper: a scheduling choice that does not change what a
 * step computes beyond rounding).  Re-tiles every problem; synchronises.
 * RLBM_ERR_ARG for another value. */
rlbm_status rlbm_batch_set_mode(rlbm_batch_t *b, int mode);
int rlbm_batch_mode(const rlbm_batch_t *b);

/* Wait for the stream; reports a barrier timeout or a non-physical cell. */
rlbm_status rlbm_batch_sync(rlbm_batch_t *b);
long long rlbm_batch_kernel_launches(const rlbm_batch_t *b);

/* Autotuner of the batched form: for each class of problems with the same K,
 * time the persistent kernel with one and with two warps per energy shell
 * (P populations per warp, 1 or 2 tiles per CTA), then the stream-pool mode
 * with each two-sites-per-lane tiling P in {8, 12, 16, 24, 32} that the
 * class allows, steps_per_trial steps each; keep the faster mode with its
 * best tilings.  It initialises every problem with a uniform rest state
 * first, so call it before rlbm_init.  best_ms (may be NULL): time of one
 * batched step with the chosen mode and shapes. */
rlbm_status rlbm_batch_autotune(rlbm_batch_t *b, int steps_per_trial, float *best_ms);

/* Bound of each grid-barrier wait in SM cycles (default 4e9) and a test hook
 * making the next rlbm_batch_step's barrier wait for one CTA too many, so
 * that every wait runs out and RLBM_ERR_TIMEOUT is reported (mode 0 only:
 * RLBM_ERR_UNSUPPORTED in mode 1, which has no barrier). */
rlbm_status rlbm_batch_set_wait_limit(rlbm_batch_t *b, long long cycles);
rlbm_status rlbm_batch_test_stall_next_step(rlbm_batch_t *b);

/* ------------------------------------------------------------------ */
/* Learned angular closure (an extension; the paper has no counterpart)  */
/* ------------------------------------------------------------------ */
/* A small MLP corrects a coarse-angle run toward the fine-angle solution.
 * Per site: features x = (N^a, T^ab)/N^0 (9 values), a scalar kn,
 * f_i/(w_i N^0) (N_pop values).  kn is the caller's: the Python driver passes
 * tau / L_train, the Knudsen number of the run's relaxation time on the
 * training grid (equal to Kn on that grid); y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3 with hidden
 * width 64 and N_pop outputs; the correction d_i = y_i w_i N^0 minus its
 * weighted least-squares component along p^0, p^0 p^0, p^0 p^x, p^0 p^y is
 * added to the post-collision populations, so N^0, T^00, T^0x, T^0y of every
 * site are kept.  Weights are BF16 in the forward passes (FP32 master copy,
 * Adam), products accumulate in FP32.  Activations are feature-major
 * [feature][column] device arrays with leading dimension ld; coarse
 * populations are FP32 [i][site].  Parameters are one flat FP32 array:
 * W1 [F][64], b1 [64], W2 [64][64], b2 [64], W3 [64][N_pop], b3 [N_pop],
 * F = 10 + N_pop (input-major matrices). */
typedef struct rlbm_closure rlbm_closure_t;

rlbm_status rlbm_closure_create(rlbm_closure_t **out, int order_N, int angles_K,
                                unsigned long long seed, void *cuda_stream);
void rlbm_closure_destroy(rlbm_closure_t *c);
const char *rlbm_closure_last_error(const rlbm_closure_t *c);
size_t rlbm_closure_param_count(const rlbm_closure_t *c);
rlbm_status rlbm_closure_get_params(rlbm_closure_t *c, float *host, size_t n);
rlbm_status rlbm_closure_set_params(rlbm_closure_t *c, const float *host, size_t n);

/* Features of `sites` sites of coarse FP32 populations d_f into columns
 * [off, off + sites) of d_x (F rows, leading dimension ld). */
rlbm_status rlbm_closure_features(rlbm_closure_t *c, const float *d_f, long long sites, double kn,
                                  float *d_x, long long ld, long long off);
/* Training target (d_fr - d_fc) / (w_i N^0(d_fc)) into columns of d_t. */
rlbm_status rlbm_closure_target(rlbm_closure_t *c, const float *d_fr, const float *d_fc,
                                long long sites, float *d_t, long long ld, long long off);
/* Angular restriction of fine FP32 populations (fine_K angles per shell) to
 * the closure's coarse rule: per shell, the angular function f / w is cut to
 * its Fourier modes |m| <= (K - 1) / 2 and evaluated at the coarse angles
 * (exact for equilibria; keeps N^a, T^00, T^0x, T^0y). */
rlbm_status rlbm_closure_restrict(rlbm_closure_t *c, int fine_K, const float *d_ff,
                                  long long sites, float *d_fc);
/* Network output for columns [off, off + count) of d_x into d_y (N_pop rows,
 * leading dimension ld, columns from 0). */
rlbm_status rlbm_closure_forward(rlbm_closure_t *c, const float *d_x, long long ld, long long off,
                                 int count, float *d_y);
/* Device work array size (floats) for gradient / training on ld columns. */
size_t rlbm_closure_work_floats(const rlbm_closure_t *c, long long ld);
/* Mean-squared-error gradient over columns [off, off + count); host_grad
 * (param_count floats, may be NULL) and loss (may be NULL). */
rlbm_status rlbm_closure_gradient(rlbm_closure_t *c, const float *d_x, const float *d_t,
                                  long long ld, long long off, int count, float *d_work,
                                  float *host_grad, float *loss);
/* One Adam step (beta 0.9, 0.999) on the same loss. */
rlbm_status rlbm_closure_train_step(rlbm_closure_t *c, const float *d_x, const float *d_t,
                                    long long ld, long long off, int count, float lr,
                                    float *d_work, float *loss);
/* Features + network + conservative projection + update of `sites` sites of
 * coarse FP32 populations d_f, in place (one fused kernel). */
rlbm_status rlbm_closure_apply_buffer(rlbm_closure_t *c, float *d_f, long long sites, double kn);
/* Choose the kernel of rlbm_closure_apply_buffer: tensor cores (BF16
 * mma.sync, activations rounded to BF16; the default when N_pop <= 80) or one
 * thread per site with FP32 activations (tensor_cores = 0). */
rlbm_status rlbm_closure_set_apply_path(rlbm_closure_t *c, int tensor_cores);
/* Choose the kernels of rlbm_closure_gradient / rlbm_closure_train_step:
 * tensor cores (the default for the specialised rules N = 2 with K = 16 or
 * 24, and N = 3 with K = 16: one fused forward + backward + weight-gradient
 * kernel, BF16 mma.sync with FP32 accumulation; the layer inputs x, h1, h2
 * and the back-propagated deltas dY, dz2, dz1 are rounded to BF16 as they
 * enter a product; the work array is not used) or one thread per site with
 * FP32 activations and deltas (tensor_cores = 0; the work array holds the
 * pre-activations and dY). */
rlbm_status rlbm_closure_set_train_path(rlbm_closure_t *c, int tensor_cores);

/* ------------------------------------------------------------------ */
/* Allocation-free single step                                          */
/* ------------------------------------------------------------------ */

/* One fused time step (the same step as rlbm_step) from d_fin to d_fout,
 * caller-owned device buffers of N_pop * nx * ny elements each (FP64 or FP32
 * storage, f[i][y][x]; the two byte ranges must not overlap, else
 * RLBM_ERR_ARG), on cuda_stream (NULL: the default stream).  The per-site part
 * runs in FP64 for both storages (a handle's FP32-storage steps run it in
 * double-float; the two agree to about 1e-6 over two steps).  This entry
 * point has no counterpart in the paper: it exists for callers that cannot
 * let a library allocate device memory -- their memory comes from their own
 * pool or framework allocator, or they run under a fixed budget -- so it calls
 * no cudaMalloc, cudaFree or other allocating routine.  Its constant tables
 * and status word live in one file-scope __device__ array of 32 KB that every
 * GPU loading the library holds until the process exits; the first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, kept per
 * device) with the device current.  A call cannot be captured into a CUDA graph: it copies from pageable host
 * memory and synchronises its stream (below).  Limits: N in {2, 3}, K (N+1) <= 256 populations; larger sizes
 * return RLBM_ERR_ARG.  Every call rewrites the array and clears its status
 * word, so calls that overlap on the GPU race: serialise them.  Every call
 * copies the tables in from host memory and synchronises the stream to read
 * the status word back; it returns RLBM_ERR_UNPHYSICAL if a cell had no
 * physical Landau frame.  rlbm_noalloc_last_error() gives the message of the
 * calling thread's latest failure. */
rlbm_status rlbm_step_noalloc(rlbm_grid grid, int order_N, int angles_K, double tau, int precision,
                              const void *d_fin, void *d_fout, void *cuda_stream);
const char *rlbm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_H */
