// Internal declarations of libfcm: device parameter blocks, index rules, the
// pairwise-correction closed forms and the kernel launchers of each stage.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <stdint.h>
#include <math.h>

namespace fcm {

constexpr double kPi = 3.14159265358979323846;
constexpr int kSeriesTerms = 10;   // Taylor terms of the small-r branch
constexpr int kMaxMG = 24;         // largest grid support the kernels accept

// Status bits written by kernels into the handle's device status word (FCM_STATUS_* in fcm.h).
// kStatusWaitTimeout: a bounded wait inside a kernel ran out (that kernel's output is incomplete).
enum : int { kStatusNonFinite = 1, kStatusWaitTimeout = 2 };

// ---------------------------------------------------------------- vectors
template <typename R> struct Vec4;
template <> struct alignas(16) Vec4<float> { float x, y, z, w; };
template <> struct alignas(32) Vec4<double> { double x, y, z, w; };

__host__ __device__ inline float as_real_bits(int i, float) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i);
#else
  union { int i; float f; } u; u.i = i; return u.f;
#endif
}
__host__ __device__ inline double as_real_bits(int i, double) { return (double)i; }
__device__ inline int index_from_w(float w) { return __float_as_int(w); }
__device__ inline int index_from_w(double w) { return (int)w; }

// ---------------------------------------------------------------- math wrappers
__host__ __device__ inline float  x_erfc(float v)  { return erfcf(v); }
__host__ __device__ inline double x_erfc(double v) { return erfc(v); }
__host__ __device__ inline float  x_exp(float v)   { return expf(v); }
__host__ __device__ inline double x_exp(double v)  { return exp(v); }
__host__ __device__ inline float  x_sqrt(float v)  { return sqrtf(v); }
__host__ __device__ inline double x_sqrt(double v) { return sqrt(v); }
__host__ __device__ inline float  x_floor(float v) { return floorf(v); }
__host__ __device__ inline double x_floor(double v){ return floor(v); }
__device__ inline float  x_mul_rn(float a, float b)   { return __fmul_rn(a, b); }
__device__ inline double x_mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ---------------------------------------------------------------- geometry
// Everything the index rules need, in the handle's precision.
template <typename R>
struct Geometry {
  R L[3];        // box edges
  R h[3];        // grid spacing L_i / M_i
  R inv_h[3];    // M_i / L_i
  R cellw_inv[3];// m_i / L_i (pair cells)
  int M[3];      // grid points
  int MG;        // grid support per dimension
  int tile[3];   // spread/gather tile in grid points
  int ntile[3];  // ceil(M_i / tile_i)
  int mcell[3];  // pair cells per dimension, max(int(L_i / r_c), 3)
  int shift;     // 1 if every mcell >= 4: the 27-cell neighbourhood never meets itself, so a
                 // neighbour cell's periodic image relative to the centre cell is unique
  // Batched launches: nsys systems with these parameters, stacked. Tile t of the launch belongs
  // to system t / tiles_per, pair cell c to system c / cells_per, and system s's grid starts
  // grid_stride reals after system s-1's. nsys <= 1 is one system (the other fields unused).
  int nsys;
  int tiles_per;       // ntile[0] ntile[1] ntile[2]
  int cells_per;       // mcell[0] mcell[1] mcell[2]
  long long grid_stride;  // 3 M_x M_y M_z
};

// Position wrapped into [0, L): y - L floor(y / L), with the product rounded on
// its own so the value does not depend on contraction into an FMA.
template <typename R>
__device__ inline R wrap_coord(R y, R L, int* bad) {
  if (!(y == y) || y - y != R(0)) { *bad = 1; return R(0); }   // NaN or +-inf
  R w = y - x_mul_rn(L, x_floor(y / L));
  if (w >= L) w -= L;
  if (w < R(0)) w = R(0);
  return w;
}

// First grid index of the M_G-point window: floor(y/h - M_G/2) + 1 (unwrapped),
// from s = y/h. The FP32 path forms s = y * (1/h) with the product rounded on its
// own (no contraction of y * (1/h) - M_G/2 into one FMA, which would move the
// floor for a particle on a grid point), the FP64 path s = y / h; every site of
// one precision goes through window_start_d, so they all agree.
template <typename R>
__device__ inline int window_start_scaled(R s, int MG) {
  R v = x_floor(s - R(0.5) * R(MG));
  v = v < R(-(1 << 29)) ? R(-(1 << 29)) : (v > R(1 << 29) ? R(1 << 29) : v);
  return (int)v + 1;
}
// a[d] for a runtime d by selects: indexing a kernel-parameter array with a runtime index
// makes the compiler copy the whole parameter block to local memory.
template <typename T>
__host__ __device__ inline T sel3(const T (&a)[3], int d) { return d == 0 ? a[0] : (d == 1 ? a[1] : a[2]); }

__device__ inline int window_start_d(const Geometry<float>& g, int d, float y) {
  return window_start_scaled(x_mul_rn(y, sel3(g.inv_h, d)), g.MG);
}
__device__ inline int window_start_d(const Geometry<double>& g, int d, double y) {
  return window_start_scaled(y / sel3(g.h, d), g.MG);
}

// i mod M for i in (-M, 2M): one correction instead of an integer division.
__host__ __device__ inline int wrap_once(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

__host__ __device__ inline int pmod(int i, int m) { int r = i % m; return r < 0 ? r + m : r; }

template <typename R>
__device__ inline int cell_coord(R yw, R winv, int m) {
  int c = (int)(yw * winv);
  return c < 0 ? 0 : (c >= m ? m - 1 : c);
}

// ---------------------------------------------------------------- kernel constants
// Spread/gather constants of the modified kernels (Section 3.1 and 3.4):
//   Delta~(d; Sigma) = nrm exp(-|d|^2/(2 Sigma^2)) (A + B |d|^2),
//   A = 1 - 3 dd / (2 Sigma^2), B = dd / (2 Sigma^4), dd = sigma^2 - Sigma^2;
//   torque part  -(1/2) T x grad Delta(d; Sigma_D) = nrmD/(2 Sigma_D^2) exp(..) (T x d).
template <typename R>
struct KernelConsts {
  R inv2S2;      // 1 / (2 Sigma^2)
  R inv2SD2;     // 1 / (2 Sigma_D^2)
  R nrm;         // (2 pi Sigma^2)^-3/2
  R A, B;
  R tq;          // (2 pi Sigma_D^2)^-3/2 / (2 Sigma_D^2)
  R h3;          // h_x h_y h_z
  int same_width;// Sigma_D == Sigma
};

// ---------------------------------------------------------------- pair correction
// Radial form of the correction blocks (Section 3.2, 3.4), x = Y_n - Y_m:
//   M_VF - M~_VF = al I + bt x x^T
//   M_WF - M~_WF = M_VT - M~_VT = cr (-x cross)
//   M_WT - M~_WT = gm I + dl x x^T
// For r^2 < rs2 the coefficients come from their Taylor series in r^2, whose
// terms are Gaussian moments of the Fourier kernels (no cancellation at small r);
// at r = 0 the series gives the Appendix B self corrections.
template <typename R>
struct PairConsts {
  R eta;
  R sg2, Sg2, dd;                  // sigma^2, Sigma^2, sigma^2 - Sigma^2
  R inv2sg, inv2Sg;                // 1/(2 sigma), 1/(2 Sigma)
  R nA, eA, nB, eB;                // Delta(r; sigma sqrt2), Delta(r; Sigma sqrt2): n exp(-e r^2)
  R sg4, Sg4;
  R k1, k2;                        // 1/(s1 sqrt2), 1/(s2 sqrt2), s1^2 = sigma^2 + sigma_D^2, s2^2 = Sigma^2 + Sigma_D^2
  R s1sq, s2sq, n1, e1, n2, e2;    // Delta(r; s1), Delta(r; s2)
  R inv2sD, inv2SD;                // 1/(2 sigma_D), 1/(2 Sigma_D)
  R sD2, SD2;                      // sigma_D^2, Sigma_D^2
  R nDa, eDa, nDb, eDb;            // Delta(r; sigma_D sqrt2), Delta(r; Sigma_D sqrt2)
  R selfVF, selfWT;                // Appendix B
  R rs2;                           // series below this r^2
  R rc2;                           // cutoff squared
  R ser_al[kSeriesTerms], ser_bt[kSeriesTerms], ser_cr[kSeriesTerms];
  R ser_gm[kSeriesTerms], ser_dl[kSeriesTerms];
};

template <typename R>
__host__ __device__ inline R horner(const R* c, R x) {
  R s = c[kSeriesTerms - 1];
#pragma unroll
  for (int j = kSeriesTerms - 2; j >= 0; --j) s = s * x + c[j];
  return s;
}

template <typename R>
__host__ __device__ inline void pair_coeffs(R r2, const PairConsts<R>& C, R& al, R& bt, R& cr,
                                            R& gm, R& dl) {
  if (r2 < C.rs2) {
    al = horner(C.ser_al, r2);
    bt = horner(C.ser_bt, r2);
    cr = horner(C.ser_cr, r2);
    gm = horner(C.ser_gm, r2);
    dl = horner(C.ser_dl, r2);
    return;
  }
  const R pi = R(kPi);
  R r = x_sqrt(r2);
  R ir = R(1) / r, ir2 = ir * ir, ir3 = ir2 * ir;
  R ieta = R(1) / C.eta;
  // VF: (G + sigma^2 lap G)(erf(r/2sigma) - erf(r/2Sigma)) + S3 terms - dd Q2 - dd^2/4 T
  R E = x_erfc(r * C.inv2Sg) - x_erfc(r * C.inv2sg);
  R DA = C.nA * x_exp(-r2 * C.eA);
  R DB = C.nB * x_exp(-r2 * C.eB);
  R t1 = E * ir * ieta / (R(8) * pi);
  R t2 = E * C.sg2 * ir3 * ieta / (R(4) * pi);
  R s3 = (C.sg4 * DA - C.Sg4 * DB) * ir2 * ieta;
  R q = C.dd * DB * ieta;
  R tt = C.dd * C.dd * DB * ieta / (R(8) * C.Sg2);
  R rho = r2 / (R(2) * C.Sg2);
  al = t1 + t2 - R(2) * s3 + q * (R(1) + R(2) * C.Sg2 * ir2) - tt * (R(2) - rho);
  R be = t1 - R(3) * t2 + R(6) * s3 - q * (R(1) + R(6) * C.Sg2 * ir2) - tt * rho;
  bt = be * ir2;
  // WF: R(x; s1) - R(x; s2) - dd/2 K(x; s2)
  R Ef = x_erfc(r * C.k2) - x_erfc(r * C.k1);
  R D1 = C.n1 * x_exp(-r2 * C.e1);
  R D2 = C.n2 * x_exp(-r2 * C.e2);
  cr = (Ef - R(4) * pi * r * (C.s1sq * D1 - C.s2sq * D2)) * ir3 * ieta / (R(8) * pi)
       + R(0.5) * C.dd * D2 * ieta / (R(2) * C.s2sq);
  // WT: (P(x; sigma_D sqrt2) - P(x; Sigma_D sqrt2)) / 2
  R Et = x_erfc(r * C.inv2SD) - x_erfc(r * C.inv2sD);
  R Da = C.nDa * x_exp(-r2 * C.eDa);
  R Db = C.nDb * x_exp(-r2 * C.eDb);
  R w1 = Et * ir3 * ieta / (R(8) * pi);
  R w2 = ir2 * ieta * R(0.5);
  gm = R(0.5) * (-w1 + ((R(2) * C.sD2 + r2) * Da - (R(2) * C.SD2 + r2) * Db) * w2);
  R de = R(0.5) * (R(3) * w1 - ((R(6) * C.sD2 + r2) * Da - (R(6) * C.SD2 + r2) * Db) * w2);
  dl = de * ir2;
}

// Piecewise-cubic tables of the five radial coefficients for the FP32 pair
// kernel: interval i covers r in [r0 + i h, r0 + (i+1) h); coef[5 i + f] holds
// (c0, c1, c2, c3) of function f (al, bt, cr, gm, dl) in u = (r - r0)/h - i.
// Built on the host in FP64 from the closed form through four points per interval.
// The interval count keeps h <= sigma/10 (cubic error below about 1e-7 of each
// function's largest value), between 64 and kPairTableIntervals: a small table
// stays in L1, where the per-lane lookups at random r are served.
constexpr int kPairTableIntervals = 1024;
struct PairTable {
  const float4* coef;
  float r0, inv_h;
  int n;
};

__host__ inline int pair_table_intervals(double r_lo, double r_hi, double sigma) {
  const double n = std::ceil((r_hi - r_lo) / (0.1 * sigma));
  return (int)std::min(std::max(n, 64.0), (double)kPairTableIntervals);
}

__device__ inline float cubic(float4 c, float u) { return fmaf(u, fmaf(u, fmaf(u, c.w, c.z), c.y), c.x); }

__device__ inline void pair_coeffs_table(float r2, const PairConsts<float>& C, const PairTable& t, float& al,
                                         float& bt, float& cr, float& gm, float& dl) {
  if (r2 < C.rs2) {
    pair_coeffs<float>(r2, C, al, bt, cr, gm, dl);
    return;
  }
  float u = (sqrtf(r2) - t.r0) * t.inv_h;
  int i = min(max((int)u, 0), t.n - 1);
  u -= (float)i;
  const float4* c = t.coef + 5 * i;
  al = cubic(__ldg(c + 0), u);
  bt = cubic(__ldg(c + 1), u);
  cr = cubic(__ldg(c + 2), u);
  gm = cubic(__ldg(c + 3), u);
  dl = cubic(__ldg(c + 4), u);
}

// Host-side construction of the constants (double), then narrowing.
void make_pair_consts(double a, double eta, double Sigma, double Sigma_D, double r_c,
                      double r_series, PairConsts<double>* out);
void narrow_pair_consts(const PairConsts<double>& in, PairConsts<float>* out);
// Fills host memory coef[5 * n] (float4 each) for r in [r_lo, r_hi] with n intervals.
void build_pair_table(const PairConsts<double>& pd, double r_lo, double r_hi, int n, float4* coef);

// ---------------------------------------------------------------- launch API
// Binning: wraps positions, computes tile and cell keys, counts and ranks,
// scans, then scatters pos/F/T into tile-sorted and cell-sorted Vec4 arrays
// whose w field carries the original index.
struct BinBuffers {
  unsigned* tile_key; unsigned* tile_rank; unsigned* cell_key; unsigned* cell_rank;
  int* tile_count; int* tile_start; int* cell_count; int* cell_start;
  int ntiles; int ncells;
  void* t_pos; void* t_F; void* t_T;   // tile-sorted Vec4<R>
  void* c_pos; void* c_F; void* c_T;   // cell-sorted Vec4<R>
  int* status;
  // Batched launches: particles of system s are rows sys_off[s] .. sys_off[s+1]-1 of the stacked
  // inputs (device array of nsys + 1 ints); nsys <= 1 or sys_off == nullptr is one system.
  const int* sys_off; int nsys;
  // Non-null for passes replayed from a CUDA graph: the particle count is read here (device) at
  // run time and the particle kernels are launched for the capacity.
  const int* n_dev;
};

// Largest number of systems in one batched pass.
constexpr int kMaxBatch = 1024;
struct SysOffsets { int off[kMaxBatch + 1]; };
// Writes the first n + 1 offsets into device memory (a kernel, so graph capture can record it).
void launch_write_offsets(const SysOffsets& o, int n, int* dst, cudaStream_t s, long long* launches);

template <typename R>
void launch_binning(const Geometry<R>& g, int n, const R* pos, const R* F, const R* T,
                    const BinBuffers& b, bool need_cells, cudaStream_t s, long long* launches);

template <typename R>
void launch_projection(const Geometry<R>& g, R eta, void* spectrum, cudaStream_t s, long long* launches);
// factor (I - k k^T/k^2) / (sqrt(eta) |k| M) in place, same zero modes (one system).
template <typename R>
void launch_projection_sqrt(const Geometry<R>& g, R eta, R factor, void* spectrum, cudaStream_t s,
                            long long* launches);

// Vector kernels of the Lanczos iteration (length m, FP64 accumulation of dot products).
constexpr int kLanczosMax = 64;
struct LanczosCoef { double c[kLanczosMax]; };
template <typename R>
void launch_dot(const R* a, const R* b, size_t m, double* out, cudaStream_t s, long long* launches);
template <typename R>   // y = alpha x + beta y
void launch_axpby(R* y, double alpha, const R* x, double beta, size_t m, cudaStream_t s, long long* launches);
template <typename R>   // out = sum_j c_j V[j] (+ out when accumulate), V[j] = V + j m
void launch_combine(R* out, const R* V, const LanczosCoef& c, int k, size_t m, bool accumulate, cudaStream_t s,
                    long long* launches);

// Rigid-body solve (rigid.cu). Unknown and step vectors have length m = 3n + 6 nb, laid out
// (F of n particles, W/mu of nb bodies); step j of the Broyden history sits at S + j * stride.
constexpr int kBroydenMax = 256;
template <typename R>   // lever arms (3n) and, unless ginv is NULL, (K^T K)^-1 (36 nb); flags[0]: bad offsets, [1]: singular
void launch_rigid_setup(const R* pos, const int* body_off, const R* X, int n, int nb, const double L[3], R* arm,
                        R* ginv, int* flags, cudaStream_t s, long long* launches);
template <typename R>   // z = -J0^-1 R(x) for V = M F, *norm2 += ||R||^2
void launch_rigid_residual(const R* V, const R* x, const R* ft, const R* arm, const R* ginv, const int* body_off,
                           int n, int nb, double inv_mu, R* z, double* norm2, cudaStream_t s, long long* launches);
// Body preconditioner (not the paper's): per body (3k + 6)^2 inverse of [[M_bb / mu, -K], [K^T, 0]],
// stored transposed with stride ms = 3 kmax + 6; bodies of at most kRigidBodyMax particles.
constexpr int kRigidBodyMax = 32;
template <typename R>
void launch_body_precond(const R* arm, const int* body_off, int nb, int kmax, const double L[3], double a, double eta,
                         R* aT, int* flags, cudaStream_t s, long long* launches);
template <typename R>
void launch_rigid_residual_body(const R* V, const R* x, const R* ft, const R* arm, const R* aT, int ms,
                                const int* body_off, int n, int nb, double inv_mu, R* z, double* norm2, cudaStream_t s,
                                long long* launches);
template <typename R>   // out[j] += a . (S + j stride), j < k
void launch_multi_dot(const R* a, const R* S, size_t m, size_t stride, int k, double* out, cudaStream_t s,
                      long long* launches);
// coef of the next Broyden step from d (n + 1 values) and the Gram rows G (row stride ld); flags[2]: breakdown
void launch_broyden_coef(const double* d, const double* G, int ld, int n, double* coef, int* flags, cudaStream_t s,
                         long long* launches);
template <typename R>   // s_out = coef[0] z + sum_{j<n} coef[1+j] S_{j+1}; x += s_out
void launch_broyden_step(const R* z, const R* S, size_t m, size_t stride, int n, const double* coef, R* s_out, R* x,
                         cudaStream_t s, long long* launches);

// FP32 tiled spread / gather (tile accumulation, halo flush).
size_t tile_smem_bytes(const int tile[3], int MG);      // extended region (gather, atomic spread)
size_t spread_smem_bytes(const int tile[3], int MG);    // whichever spread kernel the tile selects
bool spread_uses_rows(const int tile[3], int MG);       // row-stationary spread applies
int tile_smem_limit();
// spread_kernel: 0 = choose, 1 = row-stationary, 2 = shared atomics, 3 = tensor cores where eligible
// (fcm_params.spread_kernel).
void launch_spread_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, int spread_kernel,
                       const BinBuffers& b, float* grid, cudaStream_t s, long long* launches);
// Tensor-core spread along x-pencils (spread_tc.cu): 8^3 tiles, M_G in {10, 12, 14}, Sigma_D = Sigma.
bool spread_tc_eligible(const int tile[3], int MG, bool same_width);
void launch_spread_tc(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, const BinBuffers& b,
                      float* grid, cudaStream_t s);
// Tensor-core spread per pair of tiles (spread_mma.cu): 8^3 tiles and M_G in {10, 12, 14}.
bool spread_mma_eligible(const int tile[3], int MG);
void launch_spread_mma(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, const BinBuffers& b,
                       float* grid, cudaStream_t s);
// SMs of the current device (launch sizing of the pencil kernels).
inline int device_sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}
void launch_gather_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque,
                       const BinBuffers& b, const float* grid, const float* upair, const float* wpair,
                       float* U, float* W, cudaStream_t s, long long* launches);
void launch_pair_f32(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab, bool torque,
                     const BinBuffers& b, int n, float* upair, float* wpair, cudaStream_t s,
                     long long* launches);

// FP64 plain path (block per particle, global FP64 atomics; thread per particle pairs).
void launch_spread_f64(const Geometry<double>& g, const KernelConsts<double>& kc, bool torque,
                       const BinBuffers& b, int n, double* grid, cudaStream_t s, long long* launches);
void launch_gather_f64(const Geometry<double>& g, const KernelConsts<double>& kc, bool torque,
                       const BinBuffers& b, int n, const double* grid, const double* upair,
                       const double* wpair, double* U, double* W, cudaStream_t s, long long* launches);
void launch_pair_f64(const Geometry<double>& g, const PairConsts<double>& pc, bool torque,
                     const BinBuffers& b, int n, double* upair, double* wpair, cudaStream_t s,
                     long long* launches);

// Sets the message fcm_last_error() returns on this thread; returns code.
int record_error(int code, const char* msg);

// Zero-fill of a device range (a kernel of this library, counted as a launch).
void launch_zero(void* p, size_t bytes, cudaStream_t s, long long* launches);

// U[k] += up[k] for k < count, and W[k] += wp[k] when W is non-null (the join of the grid part
// and the pair sums, both in input order).
template <typename R>
void launch_add(R* U, const R* up, R* W, const R* wp, size_t count, cudaStream_t s, long long* launches,
                const int* n_dev = nullptr);   // n_dev: count = 3 * (*n_dev), read on the device

}  // namespace fcm
