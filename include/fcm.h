/*
 * libfcm - fast force-coupling method (FCM) mobility product on one GB300 GPU.
 *
 * Computes (U, W) = M (F, T) for N spheres of radius a in a periodic box, where
 * M is the FCM mobility matrix (Su & Keaveny, Sections 2 and 3.4), evaluated by
 * the fast FCM algorithm of Section 4:
 *   1. spatial hashing and sort by key (Section 4, steps 1-2),
 *   2. spread of forces and torques with the modified kernels (Section 3.1,
 *      eq. force_kernel_mod and eq. torque_kernel_mod),
 *   3. the inverse Stokes operator on the grid by FFT (Section 2.1, step 2),
 *   4. interpolation back to the particles (eq. avg_particle_vel_mod and
 *      eq. avg_particle_rot_mod),
 *   5. the pairwise correction for pairs closer than r_c (eq. correction_VF,
 *      eq. correction_WF, eq. correction_WT) and the self correction of
 *      Appendix B.
 *
 * Conventions for every entry point:
 *   - Particle arrays are caller-owned, row-major (n, 3), contiguous, in DEVICE
 *     memory, of the handle's precision (float for FCM_FP32, double for
 *     FCM_FP64). The library never frees or retains caller memory.
 *   - Calls are asynchronous on the caller's CUDA stream (cudaStream_t passed
 *     as void*, NULL = legacy default stream); no call synchronises unless its
 *     comment says so. Inputs are not modified. Positions may lie outside
 *     [0, L) and are wrapped. Outputs are in input order.
 *   - Every call returns an fcm_status; on failure fcm_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - The library allocates all its device workspace in fcm_create (or
 *     fcm_create_batch) and frees it in fcm_destroy; fcm_apply and
 *     fcm_batch_apply allocate nothing.
 *   - A handle may be used from one host thread at a time. Two calls on
 *     different streams with the same handle race on its workspace.
 */
#ifndef FCM_H_
#define FCM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fcm_status {
  FCM_OK = 0,
  FCM_ERR_ARG = 1,      /* invalid parameter or size (message says which)          */
  FCM_ERR_OOM = 2,      /* device allocation failed                                */
  FCM_ERR_CUDA = 3,     /* a CUDA runtime call failed                              */
  FCM_ERR_CUFFT = 4,    /* a cuFFT call failed                                     */
  FCM_ERR_TIMEOUT = 5,  /* a bounded wait ran out                                  */
  FCM_ERR_INPUT = 6,    /* the device flagged bad input (non-finite position)      */
  FCM_ERR_BUSY = 7,     /* the request is already running (fcm_server_cancel)      */
  FCM_ERR_CANCELED = 8, /* the request was canceled before it ran                  */
  FCM_ERR_NOT_CONVERGED = 9 /* an iterative solve reached max_iter above its tolerance */
} fcm_status;

typedef enum fcm_precision {
  FCM_FP32 = 0,  /* float I/O; tiled spread/gather, FP32 FFT; pair corrections from  */
                 /* piecewise cubics fitted in FP64 to the closed forms, a Taylor    */
                 /* series below sigma/2, per-particle pair sums compensated across  */
                 /* candidate chunks                                                 */
  FCM_FP64 = 1   /* double I/O; the plain path: global FP64 atomics, FP64 FFT        */
} fcm_precision;

/* Parameters of one periodic system (Sections 2.1, 3, 4 and 5). */
typedef struct fcm_params {
  double L[3];       /* box edges L_x, L_y, L_z (> 0)                                   */
  int M[3];          /* grid points per dimension, h_i = L_i / M_i; FFT-friendly sizes   */
  double a;          /* hydrodynamic radius; sigma = a/sqrt(pi), sigma_D = a/(6 sqrt(pi))^(1/3) */
  double eta;        /* viscosity (> 0)                                                  */
  double Sigma;      /* modified force-kernel width, Sigma >= sigma; Sigma == sigma is    */
                     /* standard FCM (no correction)                                     */
  double Sigma_D;    /* modified torque-kernel width; 0 means Sigma_D = Sigma             */
  double r_c;        /* pair-correction cutoff, 0 < r_c <= min(L)/2 (ignored when         */
                     /* Sigma == sigma)                                                   */
  int M_G;           /* grid support per dimension, 1 <= M_G <= min(M), M_G <= 24         */
  int precision;     /* fcm_precision                                                    */
  int max_n;         /* capacity: largest n accepted by fcm_apply                         */
  int tile[3];       /* FP32 spread/gather tile in grid points per dimension; 0 = choose */
  int spread_kernel; /* FP32 spread: 0 = choose (the pencil kernel: register rows      */
                     /* carried along x-pencils of tiles), 1 = row-stationary per pair   */
                     /* of tiles (needs tile[0] == 8 and M_G <= 16), 2 = shared atomics, */
                     /* 3 = tensor cores per pair of tiles, 4 = tensor cores along       */
                     /* pencils (3 and 4: tcgen05 kind::tf32, operands split in three    */
                     /* products for FP32 accuracy; 8^3 tiles and M_G in {10, 12, 14},   */
                     /* 4 also Sigma_D == Sigma; otherwise as 0)                         */
} fcm_params;

typedef struct fcm_handle fcm_handle;

/* Library and ABI version, major*10000 + minor*100 + patch. (No counterpart
 * in the paper.) */
int fcm_version(void);

/* Fills p with a = eta = 1 (the paper keeps eta symbolic), Sigma_D = 0 (the end
 * of Section 3.4 sets Sigma_D = Sigma), tile = 0 and precision FCM_FP32; the
 * caller sets L, M, Sigma, r_c, M_G and max_n. Returns FCM_ERR_ARG if p is NULL. */
int fcm_params_default(fcm_params* p);

/* Validates p and builds a handle on CUDA device `device`: workspace for max_n
 * particles, the grid, cuFFT plans and an internal stream. The parameters are
 * those the paper sets per system: box and grid (Section 2.1), the modified
 * widths Sigma, Sigma_D (Section 3.1, end of Section 3.4), the cutoff r_c and
 * the cell list it implies (Section 4, step 1) and the grid support M_G
 * (Section 5.1, Table 1). On failure *out is NULL and nothing is leaked.
 * Synchronous. */
int fcm_create(const fcm_params* p, int device, fcm_handle** out);

/* Releases everything fcm_create allocated; NULL is a no-op. Synchronises the
 * handle's device. (Resource management: no counterpart in the paper.) */
int fcm_destroy(fcm_handle* h);

/* (U, W) = M (F, T) for n particles (0 <= n <= max_n): the fast FCM algorithm
 * of Section 4 (steps 1-6): hashing and sort, spread with the modified kernels
 * (eq. force_kernel_mod, eq. torque_kernel_mod), the Stokes solve by FFT
 * (Section 2.1, step 2), interpolation (eq. avg_particle_vel_mod,
 * eq. avg_particle_rot_mod) and the pairwise and self corrections
 * (eq. correction_VF, eq. correction_WF, eq. correction_WT, Appendix B).
 *   pos : (n, 3) positions                       [device, read]
 *   F   : (n, 3) forces                          [device, read]
 *   T   : (n, 3) torques, or NULL for zero       [device, read]
 *   U   : (n, 3) velocities                      [device, write]
 *   W   : (n, 3) angular velocities, or NULL     [device, write]
 * With T == NULL and W == NULL the forces-only kernels run. A non-finite
 * position sets the handle's device status (see fcm_check); the call still
 * completes without touching memory out of bounds. */
int fcm_apply(fcm_handle* h, int n, const void* pos, const void* F, const void* T,
              void* U, void* W, void* stream);

/* Stage selection for fcm_apply_stages (bit mask). */
enum {
  FCM_STAGE_GRID = 1,  /* spread, FFT Stokes solve, interpolation (M~)       */
  FCM_STAGE_PAIR = 2,  /* pairwise and self corrections (M - M~)            */
  FCM_STAGE_ALL = 3
};

/* fcm_apply restricted to the stages in `stages`; the outputs hold the sum of
 * the selected parts: the grid part M~ and the correction M - M~ of the
 * splitting M = M~ + (M - M~) (Section 3.2, Section 3.4). Used to check each
 * part of the product on its own. */
int fcm_apply_stages(fcm_handle* h, int n, const void* pos, const void* F, const void* T,
                     void* U, void* W, int stages, void* stream);

/* ---- Brownian increments (positive splitting) ------------------------------
 * Section 3.3 shows that both M~ (grid part) and M - M~ (pairwise correction)
 * are symmetric positive definite, which is what Brownian displacements need;
 * Section 7 proposes fluctuating FCM for the grid part and a Lanczos square
 * root for the pairwise part. fcm_brownian returns a velocity increment whose
 * covariance over the random inputs is 2 kT (M~ + (M - M~)_VF):
 *   grid part : u_B = sqrt(2 kT / h^3) G^{1/2} xi, G^{1/2} = F^-1 (I - k k^T/k^2)
 *               / (sqrt(eta) |k|) F (k = 0 and Nyquist modes zero), interpolated
 *               like the deterministic grid velocity (translation and rotation);
 *   pair part : sqrt(2 kT) (M - M~)^{1/2} z for the force-velocity block (the
 *               paper proves positive splitting for it; the torque blocks are
 *               left out), by Lanczos iteration on the pair kernel.
 *   kT    : thermal energy (> 0)
 *   xi    : 3 M_x M_y M_z values (layout [c][z][y][x]), i.i.d. N(0, 1), or NULL
 *           to leave out the grid part                             [device, read]
 *   z     : (n, 3) i.i.d. N(0, 1), or NULL to leave out the pair part [device, read]
 *   U     : (n, 3) translational increment velocity                [device, write]
 *   W     : (n, 3) rotational (grid part only), or NULL            [device, write]
 *   max_iter, tol : Lanczos limits (1 <= max_iter <= FCM_LANCZOS_MAX_ITER); it
 *           stops when successive approximations differ by less than tol
 *           (relative); *iterations receives the iterations used (may be NULL).
 * Single-system use of any handle (system 0 of a batch handle). Synchronous:
 * the Lanczos recurrence reads two scalars per iteration. Allocates its Lanczos
 * basis ((max_iter + 1) x 3n values) on first use and keeps it until
 * fcm_destroy. FCM_ERR_INPUT if the correction is not positive definite on the
 * Krylov space. */
#define FCM_LANCZOS_MAX_ITER 64
int fcm_brownian(fcm_handle* h, int n, const void* pos, double kT, const void* xi, const void* z, void* U, void* W,
                 int max_iter, double tol, int* iterations, void* stream);

/* ---- Rigid bodies made of FCM particles (Section 6.1) -----------------------
 * The rod suspensions of Section 6.1 build each rod from FCM particles that move
 * as one rigid body. Body b owns particles body_off[b] .. body_off[b+1]-1, has
 * reference point X_b and lever arms r_i = Y_i - X_b (minimum image). Given each
 * body's force f_b and torque tau_b, fcm_rigid_solve finds the particle forces F
 * and body velocities (U_b, Gamma_b) with
 *   V = M^VF F               (fast-FCM product of forces only, eq. U)
 *   V_i = U_b + Gamma_b x r_i                   (rigid motion, eq. ui)
 *   sum_b F_i = f_b, sum_b r_i x F_i = tau_b    (eqs. Fn, Tn)
 * by Broyden's method (inverse "good" update, full steps) started from the
 * Jacobian of the diagonal mobility 1/(6 pi eta a) I, as the paper does. All
 * vectors stay on the device; each iteration is one fast-FCM product plus a few
 * vector kernels, and the host reads one residual norm per iteration.
 * Unknowns x = (F, W / mu) and residual R = ((V - K W) / mu, K^T F - ft) with
 * mu = 1/(6 pi eta a): both blocks in force units. Converged when
 * ||R||_2 <= tol ||ft||_2.
 *   n        : particles (0 < n <= max_n)
 *   pos      : (n, 3) particle positions                               [device, read]
 *   n_bodies : bodies (1 <= n_bodies <= n)
 *   body_off : n_bodies + 1 ints, body_off[0] = 0, increasing, body_off[n_bodies]
 *              = n; each body needs 3 particles not on one line (else its 6 x 6
 *              K^T K is singular)                                   [device, read]
 *   X        : (n_bodies, 3) reference points                          [device, read]
 *   ft       : (n_bodies, 6) rows (f_b, tau_b)                         [device, read]
 *   F        : (n, 3) particle forces                 [device, write; read if warm]
 *   UG       : (n_bodies, 6) rows (U_b, Gamma_b)      [device, write; read if warm]
 *   max_iter : 1 <= max_iter <= FCM_BROYDEN_MAX_ITER
 *   tol      : relative residual tolerance (> 0; the paper uses 1e-4)
 *   precond  : the Jacobian Broyden starts from. FCM_RIGID_PRECOND_DIAGONAL: that
 *              of the diagonal mobility mu I (the paper's choice). FCM_RIGID_PRECOND_BODY
 *              (not in the paper): that of the block-diagonal mobility keeping each
 *              body's own free-space FCM interactions, J0 = [[M_bb / mu, -K], [K^T, 0]]
 *              per body (M_bb from S(x; sigma sqrt 2), Section 2.2), inverted once per
 *              call on the device (bodies of at most FCM_RIGID_BODY_MAX particles;
 *              (3k + 6)^2 values per body of k particles); for separated rods it takes
 *              about a third of the diagonal start's steps to the same solution
 *   warm     : nonzero: start from the F and UG passed in (a previous step's
 *              solution); zero: start from F = 0, UG = 0
 *   iterations, residual : Broyden steps taken (one fast-FCM product each; a
 *              warm start costs one more product) and the final ||R|| / ||ft||
 *              (either may be NULL)
 * Single-system use of any handle (system 0 of a batch handle), in the handle's
 * precision. Synchronous. Allocates its workspace (about max_iter + 4 vectors of
 * 3n + 6 n_bodies values) on first use and keeps it until fcm_destroy.
 * FCM_ERR_INPUT if body_off is invalid or a body is degenerate (checked on the
 * device before the first product); FCM_ERR_NOT_CONVERGED if max_iter products
 * leave ||R|| above tol ||ft|| (F and UG then hold the last iterate). ft = 0 with
 * warm = 0 returns F = 0, UG = 0 after 0 iterations. */
#define FCM_BROYDEN_MAX_ITER 256
#define FCM_RIGID_PRECOND_DIAGONAL 0
#define FCM_RIGID_PRECOND_BODY 1
#define FCM_RIGID_BODY_MAX 32
int fcm_rigid_solve(fcm_handle* h, int n, const void* pos, int n_bodies, const int* body_off, const void* X,
                    const void* ft, void* F, void* UG, int max_iter, double tol, int precond, int warm,
                    int* iterations, double* residual, void* stream);

/* ---- Batched systems (many independent systems in one pass) ----------------
 * The paper treats one periodic system at a time; running many small systems
 * one call each leaves the GPU idle between launches. A batch handle holds up
 * to max_systems systems that share every parameter in p (box, grid, kernel
 * widths, cutoff, precision), stacked along the particle axis: every stage is
 * one launch over all systems' tiles, cells and grids, and the FFT is one
 * batched cuFFT plan. Results equal those of one fcm_apply per system (each
 * system's arithmetic is unchanged; only the launch covers more of them). */
#define FCM_MAX_BATCH 1024

/* fcm_create for batches: p->max_n bounds the TOTAL number of particles of one
 * batch; the grid, spectrum and bins are allocated max_systems times
 * (1 <= max_systems <= FCM_MAX_BATCH). FP64 handles hold one grid and run a
 * batch one system after another. fcm_create(p, d, out) is
 * fcm_create_batch(p, 1, d, out). Synchronous. */
int fcm_create_batch(const fcm_params* p, int max_systems, int device, fcm_handle** out);

/* (U, W) = M (F, T) for n_sys independent systems (0 <= n_sys <= max_systems).
 *   offsets : HOST array of n_sys + 1 ints [read during the call only]:
 *             offsets[0] = 0, nondecreasing, offsets[n_sys] <= max_n; system s
 *             owns rows offsets[s] .. offsets[s+1]-1 of every particle array
 *   pos, F, T, U, W : stacked (offsets[n_sys], 3) arrays, as for fcm_apply
 * Systems do not interact: each sees only its own particles and its own
 * periodic images. Empty systems are allowed. Bad offsets give FCM_ERR_ARG
 * before any work is enqueued. Asynchronous on `stream`. */
int fcm_batch_apply(fcm_handle* h, int n_sys, const int* offsets, const void* pos, const void* F,
                    const void* T, void* U, void* W, void* stream);

/* fcm_batch_apply restricted to `stages` (FCM_STAGE_GRID, FCM_STAGE_PAIR). */
int fcm_batch_apply_stages(fcm_handle* h, int n_sys, const int* offsets, const void* pos, const void* F,
                           const void* T, void* U, void* W, int stages, void* stream);

/* max_systems of the handle (1 for fcm_create), 0 for NULL. (No counterpart in
 * the paper.) */
int fcm_max_systems(const fcm_handle* h);

/* Copies the handle's real grid (the periodic grid of Section 2.1; 3 components,
 * layout [c][z][y][x], x fastest,
 * M_x*M_y*M_z values per component, the handle's precision) to device memory
 * `dst`. After fcm_apply_stages(FCM_STAGE_GRID) it holds the grid velocity u;
 * after fcm_spread it holds the spread force density f. A batch handle copies
 * the grid of system 0. */
int fcm_copy_grid(fcm_handle* h, void* dst, void* stream);

/* Sort and spread only: afterwards the grid holds f (Section 4, steps 1-3;
 * eq. force_kernel_mod and eq. torque_kernel_mod). */
int fcm_spread(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* stream);

/* Bits of the device status word that fcm_check reports. */
#define FCM_STATUS_NONFINITE 1    /* a non-finite position was seen (clamped, no fault)        */
#define FCM_STATUS_WAIT_TIMEOUT 2 /* a bounded wait inside a kernel ran out: that pass's result */
                                  /* is incomplete                                              */

/* Failure detection, no counterpart in the paper. Waits (bounded by
 * timeout_ms, polling) for all work the handle enqueued on
 * `stream`, then reads and clears the device status word into *flags
 * (FCM_STATUS_* bits). Returns FCM_ERR_TIMEOUT if the wait ran out,
 * FCM_ERR_INPUT if flags != 0. */
int fcm_check(fcm_handle* h, void* stream, int timeout_ms, int* flags);

/* Per-stage timing with CUDA events recorded on the stream each stage runs on
 * (the stages of the algorithm of Section 4; the paper times whole applies,
 * Section 5.2).
 * Stage ids: 0 binning (key/count, scan, scatter kernels), 1 spread kernel
 * (the grid zero-fill before it is not included), 2 FFT + projection +
 * inverse FFT, 3 gather kernel, 4 pair-correction kernel (side stream),
 * 5 whole apply. */
#define FCM_NUM_STAGES 6
int fcm_set_timing(fcm_handle* h, int enable);
/* Synchronises the handle's streams, then reports for each stage the summed
 * milliseconds and the number of timed launches since the last reset, and
 * resets the sums. ms and counts must hold FCM_NUM_STAGES entries. */
int fcm_read_timing(fcm_handle* h, double* ms, long long* counts);

/* (No counterpart in the paper.) Number of kernels of this library launched
 * through the handle so far
 * (library kernels only; cuFFT's own kernels are not counted). */
long long fcm_launch_count(const fcm_handle* h);

/* Device bytes the handle holds (workspace, grid, spectrum, cuFFT work area);
 * the paper's memory estimate for the grid is in Section 2.1. */
size_t fcm_workspace_bytes(const fcm_handle* h);

/* Parameter rule of the autotuner, the tolerance-related cutoff of Section 4
 * (Section 5.2, Table 2 for its measured slopes): the smallest r with every
 * normalised block
 * of the pairwise correction below `tol` for all larger separations
 * (VF relative to 1/(6 pi eta a); with torques != 0 also WT relative to
 * 1/(8 pi eta a^3) and WF relative to their geometric mean). Host only. */
int fcm_cutoff_radius(double Sigma, double Sigma_D, double a, double eta, double tol,
                      int torques, double* r_c);

/* ---- Serving engine --------------------------------------------------------
 * A request queue in front of the batched path, for many independent systems
 * of mixed sizes and boxes submitted from any host threads. The paper has no
 * counterpart; each request is computed exactly as fcm_apply would compute it.
 *   - Requests whose parameters agree (box, grid, Sigma, Sigma_D, r_c, M_G, a,
 *     eta, precision, and whether torques act: a "grid class") and that wait at
 *     the same time run as one fcm_batch_apply pass (up to max_batch systems).
 *   - Batch handles are cached per grid class and capacity, so repeated classes
 *     neither allocate nor plan. The device bytes of cached handles and staging
 *     stay within hbm_budget: idle handles are evicted least recently used
 *     first; a request whose handle alone would exceed it fails with
 *     FCM_ERR_OOM (admission control).
 *   - Four launch slots (own stream, pinned staging) let passes overlap: one
 *     pass's copies and kernels run beside the next ones'.
 *   - FP32 passes are captured once per (cached handle, power-of-two bucket of
 *     systems, staging set) into a CUDA graph and replayed (each handle has two
 *     staging sets, used alternately): the pass reads its offsets and
 *     particle count from device memory, so one graph serves every batch that
 *     fits the bucket and the handle's capacity.
 *   - One worker thread issues all GPU work; submit/poll/cancel/stats may be
 *     called from any thread, fcm_server_destroy from one thread after all
 *     other calls have returned. */
typedef struct fcm_server fcm_server;

typedef struct fcm_request {
  fcm_params params;  /* the system; max_n, tile and spread_kernel are ignored        */
  int n;              /* particles, >= 0                                              */
  const void* pos;    /* HOST (n, 3) positions, params.precision                      */
  const void* F;      /* HOST (n, 3) forces                                           */
  const void* T;      /* HOST (n, 3) torques, or NULL                                 */
  void* U;            /* HOST (n, 3) velocities                                       */
  void* W;            /* HOST (n, 3) angular velocities, or NULL                      */
} fcm_request;        /* the caller keeps all five arrays alive until the request is  */
                      /* done; inputs are read when it launches, outputs written      */
                      /* before it completes                                          */

typedef struct fcm_server_stats {
  long long submitted, completed, rejected, canceled, failed, pending;
  long long batches;           /* passes launched                                    */
  long long batched_requests;  /* requests those passes carried                      */
  long long handles_created, handles_evicted;
  long long graph_passes;      /* passes replayed from a captured CUDA graph         */
  size_t hbm_bytes;            /* device bytes held by cached handles and staging    */
  size_t hbm_budget;
  double latency_p50_us, latency_p99_us, latency_max_us;  /* submit to completion,  */
                                                           /* last 131072 requests  */
} fcm_server_stats;

/* Starts a server on `device` (worker thread, two streams). hbm_budget > 0 bytes;
 * 1 <= max_batch <= FCM_MAX_BATCH systems per pass. */
int fcm_server_create(int device, size_t hbm_budget, int max_batch, fcm_server** out);

/* Queues a request; returns at once with its id. Parameters are checked as
 * fcm_create checks them: an invalid request returns FCM_ERR_ARG and is not
 * queued. n == 0 completes immediately. */
int fcm_server_submit(fcm_server* s, const fcm_request* r, long long* id);

/* Waits up to timeout_us (0: no wait) for request `id`. Returns FCM_OK once it
 * is done, with *status its result (FCM_OK, FCM_ERR_OOM when the budget
 * refused it, FCM_ERR_CANCELED, FCM_ERR_CUDA ...), and forgets the id;
 * FCM_ERR_TIMEOUT if it is still queued or running; FCM_ERR_ARG for an
 * unknown id. */
int fcm_server_poll(fcm_server* s, long long id, long long timeout_us, int* status);

/* Removes a request that has not launched yet (it completes with
 * FCM_ERR_CANCELED); FCM_ERR_BUSY if it already launched or finished. */
int fcm_server_cancel(fcm_server* s, long long id);

/* Counters, HBM use and latency percentiles. */
int fcm_server_get_stats(fcm_server* s, fcm_server_stats* out);

/* Clears the latency window (counters are kept). */
int fcm_server_reset_latency(fcm_server* s);

/* Cancels queued requests, waits for passes in flight, frees everything. */
int fcm_server_destroy(fcm_server* s);

/* Capacity of fcm_pair_correction_noalloc's fixed scratch. */
#define FCM_NOALLOC_MAX_N 65536
#define FCM_NOALLOC_MAX_CELLS 65536

/* The pairwise and self corrections (M - M~)(F, T) of one FP32 system, like
 * fcm_apply_stages(..., FCM_STAGE_PAIR), for callers that cannot allocate
 * device memory: code whose memory pool or arena owns the whole device (a
 * cudaMalloc beside it would fail or fragment the pool), and hosts that
 * allocate everything at start-up and forbid cudaMalloc afterwards.
 * The paper has no counterpart: this entry point exists for those callers.
 *   p      : L, a, eta, Sigma, Sigma_D, r_c of the system (precision must be
 *            FCM_FP32; M, M_G, max_n and tile are not used)
 *   n      : 0 <= n <= FCM_NOALLOC_MAX_N; the pair cells, max(int(L_i/r_c), 3)
 *            per dimension, must number at most FCM_NOALLOC_MAX_CELLS
 *   pos, F, T (T may be NULL), U, W (W may be NULL): as for fcm_apply, on the
 *            current CUDA device
 * It allocates nothing: all scratch (about 7.7 MB) is one fixed file-scope
 * device array, held by every CUDA context that loads the library's device
 * code (normally one per GPU) until the process exits. With lazy module
 * loading the context reserves it at the first call made in it: make that
 * first call before a pool or arena takes the device's memory, and before any
 * stream capture. Each call looks up the array's address in the context
 * current at the time (addresses are per context; nothing is cached). Every
 * call shares the array and clears its counters first; calls whose work
 * overlaps on the GPU race on it. Non-finite positions are not reported (there
 * is no status word to read; the result is then meaningless). Sizes beyond the
 * limits return FCM_ERR_ARG with a message. */
int fcm_pair_correction_noalloc(const fcm_params* p, int n, const void* pos, const void* F, const void* T,
                                void* U, void* W, void* stream);

/* Message of the last failed call on this thread ("" if none). (Error
 * reporting: no counterpart in the paper.) */
const char* fcm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FCM_H_ */
