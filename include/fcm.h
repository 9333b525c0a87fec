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
 *   - The library allocates all its device workspace in fcm_create and frees it
 *     in fcm_destroy; fcm_apply allocates nothing.
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
  FCM_ERR_INPUT = 6     /* the device flagged bad input (non-finite position)      */
} fcm_status;

typedef enum fcm_precision {
  FCM_FP32 = 0,  /* float I/O; tiled spread/gather, FP32 FFT, FP32 pair closed form */
                 /* with the small-r series, compensated per-particle pair sums      */
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
  int spread_kernel; /* FP32 spread: 0 = choose, 1 = row-stationary (registers, no      */
                     /* atomics; needs tile[0] == 8 and M_G <= 16), 2 = shared atomics   */
} fcm_params;

typedef struct fcm_handle fcm_handle;

/* Library and ABI version, major*10000 + minor*100 + patch. */
int fcm_version(void);

/* Fills p with a = eta = 1, Sigma_D = 0, tile = 0 and precision FCM_FP32; the
 * caller sets L, M, Sigma, r_c, M_G and max_n. Returns FCM_ERR_ARG if p is NULL. */
int fcm_params_default(fcm_params* p);

/* Validates p and builds a handle on CUDA device `device`: workspace for max_n
 * particles, the grid, cuFFT plans and an internal stream. On failure *out is
 * NULL and nothing is leaked. Synchronous. */
int fcm_create(const fcm_params* p, int device, fcm_handle** out);

/* Releases everything fcm_create allocated; NULL is a no-op. Synchronises the
 * handle's device. */
int fcm_destroy(fcm_handle* h);

/* (U, W) = M (F, T) for n particles (0 <= n <= max_n).
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
 * the selected parts. Used to check each part of the product on its own. */
int fcm_apply_stages(fcm_handle* h, int n, const void* pos, const void* F, const void* T,
                     void* U, void* W, int stages, void* stream);

/* Copies the handle's real grid (3 components, layout [c][z][y][x], x fastest,
 * M_x*M_y*M_z values per component, the handle's precision) to device memory
 * `dst`. After fcm_apply_stages(FCM_STAGE_GRID) it holds the grid velocity u;
 * after fcm_spread it holds the spread force density f. */
int fcm_copy_grid(fcm_handle* h, void* dst, void* stream);

/* Sort and spread only: afterwards the grid holds f (Section 4, steps 1-3). */
int fcm_spread(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* stream);

/* Waits (bounded by timeout_ms, polling) for all work the handle enqueued on
 * `stream`, then reads and clears the device status word into *flags
 * (bit 0: a non-finite position was seen). Returns FCM_ERR_TIMEOUT if the
 * wait ran out, FCM_ERR_INPUT if flags != 0. */
int fcm_check(fcm_handle* h, void* stream, int timeout_ms, int* flags);

/* Per-stage timing with CUDA events recorded on the stream each stage runs on.
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

/* Number of kernels of this library launched through the handle so far
 * (library kernels only; cuFFT's own kernels are not counted). */
long long fcm_launch_count(const fcm_handle* h);

/* Device bytes the handle holds (workspace, grid, spectrum, cuFFT work area). */
size_t fcm_workspace_bytes(const fcm_handle* h);

/* Parameter rule of the autotuner: the smallest r with every normalised block
 * of the pairwise correction below `tol` for all larger separations
 * (VF relative to 1/(6 pi eta a); with torques != 0 also WT relative to
 * 1/(8 pi eta a^3) and WF relative to their geometric mean). Host only. */
int fcm_cutoff_radius(double Sigma, double Sigma_D, double a, double eta, double tol,
                      int torques, double* r_c);

/* Capacity of fcm_pair_correction_noalloc's fixed scratch. */
#define FCM_NOALLOC_MAX_N 65536
#define FCM_NOALLOC_MAX_CELLS 65536

/* The pairwise and self corrections (M - M~)(F, T) of one FP32 system, like
 * fcm_apply_stages(..., FCM_STAGE_PAIR), for callers that cannot allocate
 * device memory (an allocator or arena that owns the device, code running
 * while a graph is captured, hosts that forbid cudaMalloc after start-up).
 * The paper has no counterpart: this entry point exists for those callers.
 *   p      : L, a, eta, Sigma, Sigma_D, r_c of the system (precision must be
 *            FCM_FP32; M, M_G, max_n and tile are not used)
 *   n      : 0 <= n <= FCM_NOALLOC_MAX_N; the pair cells, max(int(L_i/r_c), 3)
 *            per dimension, must number at most FCM_NOALLOC_MAX_CELLS
 *   pos, F, T (T may be NULL), U, W (W may be NULL): as for fcm_apply, on the
 *            current CUDA device
 * It allocates nothing: all scratch (about 7.7 MB) is one fixed file-scope
 * device array, held by every GPU that loads the library until the process
 * exits. The first call on a device looks up that array's address with the
 * device current; make it before any stream capture. Every call shares the
 * array and clears its counters first; calls whose work overlaps on the GPU
 * race on it. Sizes beyond the limits return FCM_ERR_ARG with a message. */
int fcm_pair_correction_noalloc(const fcm_params* p, int n, const void* pos, const void* F, const void* T,
                                void* U, void* W, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* fcm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FCM_H_ */
