// Pair correction with no device allocation.
//
// Some callers cannot allocate device memory: code that runs inside a memory
// pool or arena that owns the whole device (a cudaMalloc beside it would fail
// or fragment the pool), or host environments that allocate everything at
// start-up and forbid cudaMalloc afterwards.
// fcm_pair_correction_noalloc serves them: it computes the pairwise and self
// corrections (M - M~)(F, T) of one FP32 system with the library's binning and
// pair kernels, and keeps every intermediate (sort keys, cell lists, sorted
// particles, coefficient table) in one fixed-size file-scope device array.
//
// That array exists once per CUDA context that loads the library's device code
// (normally one per GPU, the primary context) and stays allocated until the
// process exits. With lazy module loading, the context reserves it at the first
// call made in it: make that call before a pool or arena takes the device's
// memory, and before any stream capture. Host code cannot use the array's name
// as a device address; every call looks the address up with
// cudaGetSymbolAddress in the context that is current at the time, so a
// caller that switches contexts, or resets the device, gets the address valid
// in the context it runs in (nothing is cached across calls). Every call
// shares the array: the counters are cleared at the start of each call, and
// two calls whose work overlaps on the GPU (different streams, no ordering)
// race on it. Non-finite positions are clamped by the binning kernels as on
// the handle path, but this entry point has no status word for the caller to
// read: they go undetected and the result is meaningless.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/fcm.h"
#include "fcm_internal.cuh"

namespace fcm {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

constexpr size_t kN = FCM_NOALLOC_MAX_N;
constexpr size_t kCells = FCM_NOALLOC_MAX_CELLS;
constexpr size_t kKeysBytes = align_up(4 * sizeof(unsigned) * kN);
constexpr size_t kTileCountBytes = align_up(2 * sizeof(int) * 2);
constexpr size_t kCellCountBytes = align_up(2 * sizeof(int) * (kCells + 1));
constexpr size_t kSortedBytes = align_up(6 * sizeof(float4) * kN);
constexpr size_t kTableBytes = align_up(5 * sizeof(float4) * kPairTableIntervals);
constexpr size_t kStatusBytes = kAlign;
constexpr size_t kScratchBytes = kKeysBytes + kTileCountBytes + kCellCountBytes + kSortedBytes + kTableBytes + kStatusBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

int fail(int code, const std::string& msg) { return record_error(code, msg.c_str()); }

// The coefficient table, built on the device in FP64 (one thread per interval),
// the same construction as the host table of fcm_create.
__global__ void build_table_kernel(PairConsts<double> pd, double r_lo, double h, int n, float4* coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  PairConsts<double> c = pd;
  c.rs2 = 0.0;
  double v[4][5];
  for (int k = 0; k < 4; ++k) {
    const double r = r_lo + (i + k / 3.0) * h;
    pair_coeffs<double>(r * r, c, v[k][0], v[k][1], v[k][2], v[k][3], v[k][4]);
  }
  for (int f = 0; f < 5; ++f) {
    const double d1 = v[1][f] - v[0][f];
    const double d2 = v[2][f] - 2.0 * v[1][f] + v[0][f];
    const double d3 = v[3][f] - 3.0 * v[2][f] + 3.0 * v[1][f] - v[0][f];
    coef[5 * i + f] = make_float4((float)v[0][f], (float)(3.0 * (d1 - 0.5 * d2 + d3 / 3.0)),
                                  (float)(9.0 * (0.5 * d2 - 0.5 * d3)), (float)(27.0 * d3 / 6.0));
  }
}

// Device address of g_noalloc_scratch in the current context (looked up on every call: an address
// is valid only in the context it was taken in).
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return fail(FCM_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                  cudaGetErrorString(e));
  }
  *out = static_cast<unsigned char*>(p);
  return FCM_OK;
}

}  // namespace
}  // namespace fcm

using namespace fcm;

#pragma GCC visibility push(default)
extern "C" int fcm_pair_correction_noalloc(const fcm_params* p, int n, const void* pos, const void* F,
                                           const void* T, void* U, void* W, void* stream) {
  if (!p) return fail(FCM_ERR_ARG, "params is NULL");
  if (p->precision != FCM_FP32) return fail(FCM_ERR_ARG, "the no-alloc pair correction is FP32 only");
  if (n < 0 || n > FCM_NOALLOC_MAX_N)
    return fail(FCM_ERR_ARG, "n = " + std::to_string(n) + " outside [0, " + std::to_string(FCM_NOALLOC_MAX_N) +
                                 "] (the fixed scratch of the no-alloc path)");
  for (int d = 0; d < 3; ++d)
    if (!(std::isfinite(p->L[d]) && p->L[d] > 0)) return fail(FCM_ERR_ARG, "L must be finite and > 0");
  if (!(p->a > 0) || !(p->eta > 0)) return fail(FCM_ERR_ARG, "a and eta must be > 0");
  const double pi = kPi;
  const double sg = p->a / std::sqrt(pi), sD = p->a / std::cbrt(6.0 * std::sqrt(pi));
  const double Sigma = p->Sigma;
  const double SigmaD = (p->Sigma_D == 0.0) ? Sigma : p->Sigma_D;
  if (!(Sigma >= sg * (1 - 1e-12)) || !std::isfinite(Sigma)) return fail(FCM_ERR_ARG, "Sigma must be >= sigma");
  if (!(SigmaD >= sD * (1 - 1e-12)) || !std::isfinite(SigmaD)) return fail(FCM_ERR_ARG, "Sigma_D must be >= sigma_D");
  const double Lmin = std::fmin(p->L[0], std::fmin(p->L[1], p->L[2]));
  if (!(p->r_c > 0) || !(p->r_c <= 0.5 * Lmin)) return fail(FCM_ERR_ARG, "r_c must satisfy 0 < r_c <= min(L)/2");
  double cells_d = 1.0;
  for (int d = 0; d < 3; ++d) cells_d *= std::fmax(std::floor(p->L[d] / p->r_c), 3.0);
  if (cells_d > (double)FCM_NOALLOC_MAX_CELLS)
    return fail(FCM_ERR_ARG, "the pair cells, max(int(L_i/r_c), 3) per dimension, exceed " +
                                 std::to_string(FCM_NOALLOC_MAX_CELLS) +
                                 " (the fixed scratch of the no-alloc path); r_c is too small for this box");
  Geometry<float> g{};
  long long cells = 1;
  for (int d = 0; d < 3; ++d) {
    g.L[d] = (float)p->L[d];
    g.M[d] = 1;  // one spread tile covering everything: only the pair cells are used here
    g.h[d] = (float)p->L[d];
    g.inv_h[d] = (float)(1.0 / p->L[d]);
    g.tile[d] = 1;
    g.ntile[d] = 1;
    g.mcell[d] = std::max((int)(p->L[d] / p->r_c), 3);
    g.cellw_inv[d] = (float)(g.mcell[d] / p->L[d]);
    cells *= g.mcell[d];
  }
  g.MG = 1;
  g.shift = (g.mcell[0] >= 4 && g.mcell[1] >= 4 && g.mcell[2] >= 4) ? 1 : 0;
  if (cells > (long long)FCM_NOALLOC_MAX_CELLS)
    return fail(FCM_ERR_ARG, std::to_string(cells) + " pair cells exceed " + std::to_string(FCM_NOALLOC_MAX_CELLS) +
                                 " (the fixed scratch of the no-alloc path); r_c is too small for this box");
  if (n > 0 && (!pos || !F || !U)) return fail(FCM_ERR_ARG, "pos, F and U must be non-NULL when n > 0");
  if (n == 0) return FCM_OK;

  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FCM_OK) return rc;

  BinBuffers b{};
  unsigned char* q = base;
  b.tile_key = (unsigned*)q;
  b.tile_rank = b.tile_key + kN;
  b.cell_key = b.tile_rank + kN;
  b.cell_rank = b.cell_key + kN;
  q += kKeysBytes;
  b.tile_count = (int*)q;
  b.tile_start = b.tile_count + 2;
  q += kTileCountBytes;
  b.cell_count = (int*)q;
  b.cell_start = b.cell_count + (kCells + 1);
  q += kCellCountBytes;
  float4* sorted = (float4*)q;
  b.t_pos = sorted;
  b.t_F = sorted + kN;
  b.t_T = sorted + 2 * kN;
  b.c_pos = sorted + 3 * kN;
  b.c_F = sorted + 4 * kN;
  b.c_T = sorted + 5 * kN;
  q += kSortedBytes;
  float4* table = (float4*)q;
  q += kTableBytes;
  b.status = (int*)q;
  b.ntiles = 1;
  b.ncells = (int)cells;

  PairConsts<double> pd;
  const double r_lo = 0.5 * sg;
  make_pair_consts(p->a, p->eta, Sigma, SigmaD, p->r_c, r_lo, &pd);
  PairConsts<float> pf;
  narrow_pair_consts(pd, &pf);
  const double r_hi = std::fmax(p->r_c, r_lo + 1e-3);
  PairTable tab;
  tab.coef = table;
  tab.r0 = (float)r_lo;
  tab.inv_h = (float)(kPairTableIntervals / (r_hi - r_lo));
  tab.n = kPairTableIntervals;

  cudaStream_t s = (cudaStream_t)stream;
  long long launches = 0;
  // counters must start at zero; the scan leaves them at zero, but a call may follow an error
  launch_zero(b.tile_count, kTileCountBytes, s, &launches);
  launch_zero(b.cell_count, sizeof(int) * (size_t)(cells + 1), s, &launches);
  launch_zero(b.status, kStatusBytes, s, &launches);
  build_table_kernel<<<(kPairTableIntervals + 127) / 128, 128, 0, s>>>(pd, r_lo, (r_hi - r_lo) / kPairTableIntervals,
                                                                      kPairTableIntervals, table);
  launch_binning<float>(g, n, (const float*)pos, (const float*)F, (const float*)T, b, true, s, &launches);
  const bool torque = (T != nullptr) || (W != nullptr);
  launch_pair_f32(g, pf, tab, torque, b, n, (float*)U, (float*)W, s, &launches);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FCM_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return FCM_OK;
}
#pragma GCC visibility pop
