// libfcm C-ABI: handle lifetime, parameter checks, workspace, and the launch
// sequence of one mobility product (Section 4):
//
//   caller stream : bin ─► zero grid ─► spread ─┬─► R2C ─► project ─► C2R ─► gather ─┬─► add ─► U, W
//   side stream   :                             └─► pair ────────────────────────────┘
//
// The pair correction only needs the cell-sorted particles. It is forked onto
// the handle's side stream after the spread, where it runs beside the FFT
// chain and the gather (the spread fills every SM's registers, so overlapping
// it gains nothing). The gather writes the grid part of U and W in input
// order, the pair kernel its sums, and a small kernel adds them after the
// join. The fork/join uses events only, so a caller may capture fcm_apply into
// a CUDA graph.
#include <cufft.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/fcm.h"
#include "fcm_internal.cuh"

using namespace fcm;

namespace {

thread_local std::string g_error;

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

#define FCM_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? FCM_ERR_OOM : FCM_ERR_CUDA,              \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

#define FCM_CUFFT(call)                                                                      \
  do {                                                                                       \
    cufftResult r_ = (call);                                                                 \
    if (r_ != CUFFT_SUCCESS) return fail(FCM_ERR_CUFFT, std::string(#call) + " failed: " +   \
                                              std::to_string((int)r_));                      \
  } while (0)

struct StageEvents {
  cudaEvent_t a, b;
  int stage;
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() { cudaSetDevice(prev_); }
 private:
  int prev_ = 0;
};

double gauss_moment(double s2, int m) {  // int_0^inf exp(-s2 k^2) k^(2m) dk
  return std::tgamma(m + 0.5) / (2.0 * std::pow(s2, m + 0.5));
}

double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

double double_factorial(int k) {
  double f = 1.0;
  for (int i = k; i > 1; i -= 2) f *= i;
  return f;
}

}  // namespace

namespace fcm {

// Constants of pair_coeffs, and the Taylor coefficients of each radial
// function: the correction blocks are Fourier integrals of radial kernels
// (Appendix A for VF), so expanding exp(i k.x) in powers of k.x gives series in
// r^2 whose coefficients are angular averages times Gaussian moments of the kernels.
void make_pair_consts(double a, double eta, double Sigma, double Sigma_D, double r_c, double r_series,
                      PairConsts<double>* o) {
  const double pi = kPi;
  const double sg = a / std::sqrt(pi);
  const double sD = a / std::cbrt(6.0 * std::sqrt(pi));
  std::memset(o, 0, sizeof(*o));
  o->eta = eta;
  o->sg2 = sg * sg;
  o->Sg2 = Sigma * Sigma;
  o->dd = sg * sg - Sigma * Sigma;
  o->inv2sg = 1.0 / (2.0 * sg);
  o->inv2Sg = 1.0 / (2.0 * Sigma);
  o->nA = std::pow(4.0 * pi * sg * sg, -1.5);
  o->eA = 1.0 / (4.0 * sg * sg);
  o->nB = std::pow(4.0 * pi * Sigma * Sigma, -1.5);
  o->eB = 1.0 / (4.0 * Sigma * Sigma);
  o->sg4 = o->sg2 * o->sg2;
  o->Sg4 = o->Sg2 * o->Sg2;
  const double s1 = std::sqrt(sg * sg + sD * sD), s2 = std::sqrt(Sigma * Sigma + Sigma_D * Sigma_D);
  o->k1 = 1.0 / (s1 * std::sqrt(2.0));
  o->k2 = 1.0 / (s2 * std::sqrt(2.0));
  o->s1sq = s1 * s1;
  o->s2sq = s2 * s2;
  o->n1 = std::pow(2.0 * pi * s1 * s1, -1.5);
  o->e1 = 1.0 / (2.0 * s1 * s1);
  o->n2 = std::pow(2.0 * pi * s2 * s2, -1.5);
  o->e2 = 1.0 / (2.0 * s2 * s2);
  o->inv2sD = 1.0 / (2.0 * sD);
  o->inv2SD = 1.0 / (2.0 * Sigma_D);
  o->sD2 = sD * sD;
  o->SD2 = Sigma_D * Sigma_D;
  o->nDa = std::pow(4.0 * pi * sD * sD, -1.5);
  o->eDa = 1.0 / (4.0 * sD * sD);
  o->nDb = std::pow(4.0 * pi * Sigma_D * Sigma_D, -1.5);
  o->eDb = 1.0 / (4.0 * Sigma_D * Sigma_D);
  const double dd = o->dd;
  const double sp = Sigma * std::sqrt(pi);
  o->selfVF = 1.0 / (6.0 * pi * eta * a) - 1.0 / (6.0 * pi * eta * sp) + dd / (12.0 * eta * sp * sp * sp) -
              dd * dd / (32.0 * eta * std::pow(Sigma, 5) * std::pow(pi, 1.5));
  const double spD = Sigma_D * std::sqrt(pi);
  o->selfWT = 1.0 / (8.0 * pi * eta * a * a * a) - 1.0 / (48.0 * eta * spD * spD * spD);
  o->rs2 = r_series * r_series;
  o->rc2 = r_c * r_c;
  // Taylor series
  const double S2 = Sigma * Sigma, SD2 = Sigma_D * Sigma_D;
  const double e1sq = 0.5 * (sg * sg + sD * sD), e2sq = 0.5 * (S2 + SD2);
  auto mVF = [&](int j) {
    return gauss_moment(sg * sg, j) - gauss_moment(S2, j) + dd * gauss_moment(S2, j + 1) -
           0.25 * dd * dd * gauss_moment(S2, j + 2);
  };
  auto mWT = [&](int j) { return gauss_moment(sD * sD, j + 1) - gauss_moment(SD2, j + 1); };
  auto mWF = [&](int j) {
    return gauss_moment(e1sq, j + 1) - gauss_moment(e2sq, j + 1) + 0.5 * dd * gauss_moment(e2sq, j + 2);
  };
  for (int j = 0; j <= kSeriesTerms; ++j) {
    const double sgn = (j % 2 == 0) ? 1.0 : -1.0;
    const double ang = 1.0 / ((2.0 * j + 1.0) * (2.0 * j + 3.0));
    const double base_vf = sgn * mVF(j) / (factorial(2 * j) * 2.0 * pi * pi * eta) * ang;
    const double base_wt = sgn * mWT(j) / (factorial(2 * j) * 8.0 * pi * pi * eta) * ang;
    if (j < kSeriesTerms) {
      o->ser_al[j] = base_vf * (2.0 * j + 2.0);
      o->ser_gm[j] = base_wt * (2.0 * j + 2.0);
      o->ser_cr[j] = sgn * mWF(j) / (4.0 * pi * pi * eta * std::pow(2.0, j) * factorial(j) * double_factorial(2 * j + 3));
    }
    if (j >= 1) {
      o->ser_bt[j - 1] = -base_vf * (2.0 * j);
      o->ser_dl[j - 1] = -base_wt * (2.0 * j);
    }
  }
}

void narrow_pair_consts(const PairConsts<double>& in, PairConsts<float>* o) {
  const double* src = reinterpret_cast<const double*>(&in);
  float* dst = reinterpret_cast<float*>(o);
  static_assert(sizeof(PairConsts<double>) == 2 * sizeof(PairConsts<float>), "layout");
  for (size_t k = 0; k < sizeof(PairConsts<float>) / sizeof(float); ++k) dst[k] = (float)src[k];
}

int record_error(int code, const char* msg) { return fail(code, msg); }

void build_pair_table(const PairConsts<double>& pd, double r_lo, double r_hi, int n, float4* coef) {
  PairConsts<double> c = pd;
  c.rs2 = 0.0;  // the closed form throughout the tabulated range
  const double h = (r_hi - r_lo) / n;
  for (int i = 0; i < n; ++i) {
    double v[4][5];
    for (int k = 0; k < 4; ++k) {
      const double r = r_lo + (i + k / 3.0) * h;
      pair_coeffs<double>(r * r, c, v[k][0], v[k][1], v[k][2], v[k][3], v[k][4]);
    }
    for (int f = 0; f < 5; ++f) {
      // Newton differences on s = 3u in {0, 1, 2, 3}, rewritten in powers of u
      const double d1 = v[1][f] - v[0][f];
      const double d2 = v[2][f] - 2.0 * v[1][f] + v[0][f];
      const double d3 = v[3][f] - 3.0 * v[2][f] + 3.0 * v[1][f] - v[0][f];
      float4 q;
      q.x = (float)v[0][f];
      q.y = (float)(3.0 * (d1 - 0.5 * d2 + d3 / 3.0));
      q.z = (float)(9.0 * (0.5 * d2 - 0.5 * d3));
      q.w = (float)(27.0 * d3 / 6.0);
      coef[5 * i + f] = q;
    }
  }
}

}  // namespace fcm

struct fcm_handle {
  fcm_params p{};
  int device = 0;
  bool fp64 = false;
  bool pairs_on = false;
  Geometry<float> gf{};
  Geometry<double> gd{};
  KernelConsts<float> kf{};
  KernelConsts<double> kd{};
  PairConsts<float> pf{};
  PairConsts<double> pd{};
  PairTable ptab{};
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  BinBuffers bb{};
  void* grid = nullptr;
  void* spec = nullptr;
  void* upair = nullptr;
  void* wpair = nullptr;
  void* wscratch = nullptr;
  size_t grid_bytes = 0;
  // FFT plans per batch bucket (1, 2, 4, ... systems, and max_systems), sharing one work area
  struct Plan { int systems; cufftHandle r2c, c2r; };
  std::vector<Plan> plans;
  void* fft_work = nullptr;
  int max_systems = 1;
  int* sys_off = nullptr;       // device offsets of the current batched pass
  size_t spec_bytes = 0;        // one system's spectra
  void* lz = nullptr;           // Lanczos basis and work vector (fcm_brownian), grown on demand
  size_t lz_bytes = 0;
  double* lz_dot = nullptr;     // device scalar of the Lanczos dot products
  void* rg = nullptr;           // rigid-solve vectors, Broyden steps and scalars, grown on demand
  size_t rg_bytes = 0;
  void* rgp = nullptr;          // rigid-solve body preconditioner (inverse blocks), grown on demand
  size_t rgp_bytes = 0;
  size_t bytes = 0;
  long long launches = 0;
  std::vector<void*> allocs;
  bool timing = false;
  std::vector<StageEvents> pool;
  std::vector<int> pending;
  size_t next_event = 0;
  double ms[FCM_NUM_STAGES] = {0};
  long long counts[FCM_NUM_STAGES] = {0};
};

namespace {

int halloc(fcm_handle* h, void** out, size_t bytes) {
  bytes = (bytes + 255) / 256 * 256;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(FCM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  h->allocs.push_back(p);
  h->bytes += bytes;
  *out = p;
  return FCM_OK;
}

void release(fcm_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (auto& pl : h->plans) {
    cufftDestroy(pl.r2c);
    cufftDestroy(pl.c2r);
  }
  for (auto& ev : h->pool) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  for (void* p : h->allocs) cudaFree(p);
  if (h->lz) cudaFree(h->lz);
  if (h->lz_dot) cudaFree(h->lz_dot);
  if (h->rg) cudaFree(h->rg);
  if (h->rgp) cudaFree(h->rgp);
  delete h;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

// FP32 tile: (8, t, t) with the largest t in {8, 4, 2} whose extended (y, z)
// rows fit the row-stationary spread; otherwise the largest tile whose
// extended region fits shared memory (atomic spread).
void choose_tile(const fcm_params& p, int tile[3]) {
  if (p.tile[0] > 0 && p.tile[1] > 0 && p.tile[2] > 0) {
    for (int d = 0; d < 3; ++d) tile[d] = std::min(p.tile[d], p.M[d]);
    return;
  }
  for (int t : {8, 4, 2}) {
    int c[3] = {std::min(8, p.M[0]), std::min(t, p.M[1]), std::min(t, p.M[2])};
    if (spread_uses_rows(c, p.M_G) && tile_smem_bytes(c, p.M_G) <= (size_t)tile_smem_limit() &&
        spread_smem_bytes(c, p.M_G) <= (size_t)tile_smem_limit()) {
      tile[0] = c[0]; tile[1] = c[1]; tile[2] = c[2];
      return;
    }
  }
  static const int cands[][3] = {{8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {4, 4, 4}, {4, 4, 2}, {4, 2, 2},
                                 {2, 2, 2}, {2, 2, 1}, {2, 1, 1}, {1, 1, 1}};
  const size_t budgets[2] = {113 * 1024, (size_t)tile_smem_limit()};
  for (size_t budget : budgets) {
    for (auto& c : cands) {
      int t[3] = {std::min(c[0], p.M[0]), std::min(c[1], p.M[1]), std::min(c[2], p.M[2])};
      if (tile_smem_bytes(t, p.M_G) <= budget) {
        tile[0] = t[0]; tile[1] = t[1]; tile[2] = t[2];
        return;
      }
    }
  }
  tile[0] = tile[1] = tile[2] = 1;
}

// Pair cells: side max(r_c, s_occ) with s_occ = (kCellTarget / rho)^(1/3), rho the capacity's number
// density (max_n particles over `systems` boxes). Any side >= r_c keeps every pair within the 27
// neighbouring cells (Section 4 step 1 uses side r_c); in dilute systems an r_c cell holds about one
// particle, and a CTA per cell would then stage 27 cells for a single particle.
constexpr double kCellTarget = 8.0;

double cell_side(const fcm_params& p, int systems) {
  const double V = p.L[0] * p.L[1] * p.L[2];
  const double rho = (double)std::max(p.max_n, 1) / ((double)std::max(systems, 1) * V);
  return std::max(p.r_c, std::cbrt(kCellTarget / rho));
}

template <typename R>
void fill_geometry(const fcm_params& p, const int tile[3], Geometry<R>* g, int systems = 1) {
  const double side = (p.r_c > 0) ? cell_side(p, systems) : 0.0;
  for (int d = 0; d < 3; ++d) {
    g->L[d] = (R)p.L[d];
    g->h[d] = (R)(p.L[d] / p.M[d]);
    g->inv_h[d] = (R)(p.M[d] / p.L[d]);
    g->M[d] = p.M[d];
    g->tile[d] = tile[d];
    g->ntile[d] = (p.M[d] + tile[d] - 1) / tile[d];
    // cells per dimension max(int(L/side), 3), clamped before the integer conversion
    const double m = (p.r_c > 0) ? std::floor(p.L[d] / side) : 3.0;
    g->mcell[d] = (int)std::min(std::max(m, 3.0), 1048576.0);
    g->cellw_inv[d] = (R)(g->mcell[d] / p.L[d]);
  }
  g->shift = (g->mcell[0] >= 4 && g->mcell[1] >= 4 && g->mcell[2] >= 4) ? 1 : 0;
  g->MG = p.M_G;
  g->nsys = 1;
  g->tiles_per = g->ntile[0] * g->ntile[1] * g->ntile[2];
  g->cells_per = g->mcell[0] * g->mcell[1] * g->mcell[2];
  g->grid_stride = 3LL * p.M[0] * p.M[1] * p.M[2];
}

template <typename R>
void fill_kernel_consts(const fcm_params& p, double SigmaD, KernelConsts<R>* k) {
  const double pi = kPi;
  const double sg = p.a / std::sqrt(pi);
  const double S = p.Sigma, dd = sg * sg - S * S;
  k->inv2S2 = (R)(1.0 / (2.0 * S * S));
  k->inv2SD2 = (R)(1.0 / (2.0 * SigmaD * SigmaD));
  k->nrm = (R)std::pow(2.0 * pi * S * S, -1.5);
  k->A = (R)(1.0 - 3.0 * dd / (2.0 * S * S));
  k->B = (R)(dd / (2.0 * S * S * S * S));
  k->tq = (R)(std::pow(2.0 * pi * SigmaD * SigmaD, -1.5) / (2.0 * SigmaD * SigmaD));
  k->h3 = (R)((p.L[0] / p.M[0]) * (p.L[1] / p.M[1]) * (p.L[2] / p.M[2]));
  k->same_width = (SigmaD == S) ? 1 : 0;
}

int validate(const fcm_params* p, std::string* why) {
  for (int d = 0; d < 3; ++d) {
    if (!finite_pos(p->L[d])) { *why = "L must be finite and > 0"; return 0; }
    if (p->M[d] < 1 || p->M[d] > (1 << 14)) { *why = "M must be in [1, 16384]"; return 0; }
    if (p->M_G > p->M[d]) { *why = "M_G must not exceed M in any dimension"; return 0; }
  }
  if (p->M_G < 1 || p->M_G > 24) { *why = "M_G must be in [1, 24]"; return 0; }
  if (!finite_pos(p->a)) { *why = "a must be finite and > 0"; return 0; }
  if (!finite_pos(p->eta)) { *why = "eta must be finite and > 0"; return 0; }
  const double sg = p->a / std::sqrt(kPi), sD = p->a / std::cbrt(6.0 * std::sqrt(kPi));
  if (!finite_pos(p->Sigma) || p->Sigma < sg * (1 - 1e-12)) { *why = "Sigma must be >= sigma = a/sqrt(pi)"; return 0; }
  if (!(p->Sigma_D == 0.0 || (std::isfinite(p->Sigma_D) && p->Sigma_D >= sD * (1 - 1e-12)))) {
    *why = "Sigma_D must be 0 or >= sigma_D = a/(6 sqrt(pi))^(1/3)";
    return 0;
  }
  if (p->precision != FCM_FP32 && p->precision != FCM_FP64) { *why = "precision must be FCM_FP32 or FCM_FP64"; return 0; }
  if (p->max_n < 0) { *why = "max_n must be >= 0"; return 0; }
  if (p->spread_kernel < 0 || p->spread_kernel > 4) { *why = "spread_kernel must be 0, 1, 2, 3 or 4"; return 0; }
  return 1;
}

int fold_pending(fcm_handle* h) {
  for (int idx : h->pending) {
    StageEvents& ev = h->pool[idx];
    FCM_CUDA(cudaEventSynchronize(ev.b));
    float t = 0.f;
    FCM_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
    h->ms[ev.stage] += t;
    h->counts[ev.stage] += 1;
  }
  h->pending.clear();
  h->next_event = 0;
  return FCM_OK;
}

// Stage timing: stage_begin records the start event of a free pair and returns
// its slot (-1 when timing is off); stage_end records the stop event.
int stage_begin(fcm_handle* h, int stage, cudaStream_t s, int* slot) {
  *slot = -1;
  if (!h->timing) return FCM_OK;
  if (h->next_event >= h->pool.size()) {
    int rc = fold_pending(h);
    if (rc) return rc;
  }
  StageEvents& ev = h->pool[h->next_event];
  ev.stage = stage;
  FCM_CUDA(cudaEventRecord(ev.a, s));
  *slot = (int)h->next_event++;
  return FCM_OK;
}

int stage_end(fcm_handle* h, int slot, cudaStream_t s) {
  if (slot < 0) return FCM_OK;
  FCM_CUDA(cudaEventRecord(h->pool[slot].b, s));
  h->pending.push_back(slot);
  return FCM_OK;
}

// Forks the pair correction onto the side stream (it needs only the cell-sorted
// particles); the caller joins on ev_join before the gather.
template <typename R>
int launch_pair_stage(fcm_handle* h, const Geometry<R>& g, const BinBuffers& bb, int n, R* U, R* Wout, bool torque,
                      bool grid_on, cudaStream_t s) {
  int rc, t_pair;
  R* up = grid_on ? (R*)h->upair : U;
  R* wp = grid_on ? (R*)h->wpair : Wout;
  FCM_CUDA(cudaEventRecord(h->ev_fork, s));
  FCM_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  if ((rc = stage_begin(h, 4, h->side, &t_pair))) return rc;
  if constexpr (std::is_same<R, double>::value)
    launch_pair_f64(g, h->pd, torque, bb, n, up, wp, h->side, &h->launches);
  else
    launch_pair_f32(g, h->pf, h->ptab, torque, bb, n, up, wp, h->side, &h->launches);
  if ((rc = stage_end(h, t_pair, h->side))) return rc;
  FCM_CUDA(cudaGetLastError());
  FCM_CUDA(cudaEventRecord(h->ev_join, h->side));
  return FCM_OK;
}

const fcm_handle::Plan* plan_for(const fcm_handle* h, int nsys) {
  for (const auto& pl : h->plans)
    if (pl.systems >= nsys) return &pl;
  return nullptr;
}

// One pass over nsys stacked systems (nsys > 1 only on the FP32 path; h->sys_off then holds
// the offsets). Plans cover a bucket of systems >= nsys: the bucket's extra grids are zeroed
// with the others, so their transforms stay zero.
template <typename R>
int run(fcm_handle* h, int nsys, int n, const R* pos, const R* F, const R* T, R* U, R* W, int stages,
        bool spread_only, cudaStream_t s, const int* n_dev = nullptr) {
  const bool torque = (T != nullptr) || (W != nullptr);
  R* Wout = W ? W : (torque ? (R*)h->wscratch : nullptr);
  const bool grid_on = spread_only || (stages & FCM_STAGE_GRID);
  const bool pair_on = !spread_only && (stages & FCM_STAGE_PAIR) && h->pairs_on;
  Geometry<R> g = *reinterpret_cast<const Geometry<R>*>(h->fp64 ? (const void*)&h->gd : (const void*)&h->gf);
  BinBuffers bb = h->bb;
  const fcm_handle::Plan* plan = plan_for(h, nsys);
  if (!plan) return fail(FCM_ERR_ARG, "no FFT plan for " + std::to_string(nsys) + " systems");
  g.nsys = nsys;
  bb.nsys = nsys;
  bb.sys_off = nsys > 1 ? h->sys_off : nullptr;
  bb.n_dev = n_dev;
  bb.ntiles = nsys * g.tiles_per;
  bb.ncells = pair_on ? nsys * g.cells_per : bb.ncells;
  int rc, t_all, t_bin, t_spread, t_fft, t_gather;
  if ((rc = stage_begin(h, 5, s, &t_all))) return rc;
  if ((rc = stage_begin(h, 0, s, &t_bin))) return rc;
  launch_binning<R>(g, n, pos, F, T, bb, pair_on, s, &h->launches);
  if ((rc = stage_end(h, t_bin, s))) return rc;
  FCM_CUDA(cudaGetLastError());
  if (grid_on) {
    launch_zero(h->grid, h->grid_bytes * plan->systems, s, &h->launches);
    if ((rc = stage_begin(h, 1, s, &t_spread))) return rc;
    if constexpr (std::is_same<R, double>::value)
      launch_spread_f64(g, h->kd, torque, bb, n, (double*)h->grid, s, &h->launches);
    else
      launch_spread_f32(g, h->kf, torque, h->p.spread_kernel, bb, (float*)h->grid, s, &h->launches);
    if ((rc = stage_end(h, t_spread, s))) return rc;
    FCM_CUDA(cudaGetLastError());
    if (pair_on && !spread_only) {
      if ((rc = launch_pair_stage(h, g, bb, n, U, Wout, torque, grid_on, s))) return rc;
    }
    if (!spread_only) {
      // FFT chain and gather on the caller's stream, beside the pair kernel on the side stream.
      // (Giving them a higher stream priority than the pair made the step slower: the pair then
      // ran mostly after the gather instead of beside the FFT.)
      cudaStream_t m = s;
      if ((rc = stage_begin(h, 2, m, &t_fft))) return rc;
      FCM_CUFFT(cufftSetStream(plan->r2c, m));
      FCM_CUFFT(cufftSetStream(plan->c2r, m));
      if constexpr (std::is_same<R, double>::value) {
        FCM_CUFFT(cufftExecD2Z(plan->r2c, (cufftDoubleReal*)h->grid, (cufftDoubleComplex*)h->spec));
        launch_projection<double>(g, h->p.eta, h->spec, m, &h->launches);
        FCM_CUFFT(cufftExecZ2D(plan->c2r, (cufftDoubleComplex*)h->spec, (cufftDoubleReal*)h->grid));
      } else {
        FCM_CUFFT(cufftExecR2C(plan->r2c, (cufftReal*)h->grid, (cufftComplex*)h->spec));
        launch_projection<float>(g, (float)h->p.eta, h->spec, m, &h->launches);
        FCM_CUFFT(cufftExecC2R(plan->c2r, (cufftComplex*)h->spec, (cufftReal*)h->grid));
      }
      if ((rc = stage_end(h, t_fft, m))) return rc;
      FCM_CUDA(cudaGetLastError());
      // the gather writes the grid part; the pair sums, which run beside the FFT and the gather,
      // are added once both are done
      if ((rc = stage_begin(h, 3, m, &t_gather))) return rc;
      if constexpr (std::is_same<R, double>::value)
        launch_gather_f64(g, h->kd, torque, bb, n, (const double*)h->grid, nullptr, nullptr, U, Wout, m,
                          &h->launches);
      else
        launch_gather_f32(g, h->kf, torque, bb, (const float*)h->grid, nullptr, nullptr, U, Wout, m, &h->launches);
      if ((rc = stage_end(h, t_gather, m))) return rc;
      FCM_CUDA(cudaGetLastError());
      if (pair_on) {
        FCM_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
        launch_add<R>(U, (const R*)h->upair, Wout, (const R*)h->wpair, 3 * (size_t)n, s, &h->launches, n_dev);
        FCM_CUDA(cudaGetLastError());
      }
    }
  } else if (pair_on) {
    if ((rc = launch_pair_stage(h, g, bb, n, U, Wout, torque, grid_on, s))) return rc;
    FCM_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
  } else if (!spread_only) {  // only the correction requested and it is identically zero
    launch_zero(U, sizeof(R) * 3 * (size_t)n, s, &h->launches);
    if (W) launch_zero(W, sizeof(R) * 3 * (size_t)n, s, &h->launches);
  }
  if ((rc = stage_end(h, t_all, s))) return rc;
  FCM_CUDA(cudaGetLastError());
  return FCM_OK;
}

int apply_common(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* U, void* W,
                 int stages, bool spread_only, void* stream) {
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  if (n < 0 || n > h->p.max_n)
    return fail(FCM_ERR_ARG, "n = " + std::to_string(n) + " outside [0, max_n = " + std::to_string(h->p.max_n) + "]");
  if (n > 0 && (!pos || !F || (!spread_only && !U)))
    return fail(FCM_ERR_ARG, "pos, F and U must be non-NULL when n > 0");
  if (stages < 1 || stages > FCM_STAGE_ALL) return fail(FCM_ERR_ARG, "stages must be a non-empty subset of FCM_STAGE_ALL");
  if (n == 0) return FCM_OK;
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->fp64)
    return run<double>(h, 1, n, (const double*)pos, (const double*)F, (const double*)T, (double*)U, (double*)W,
                       stages, spread_only, s);
  return run<float>(h, 1, n, (const float*)pos, (const float*)F, (const float*)T, (float*)U, (float*)W, stages,
                    spread_only, s);
}

// Stacked systems: FP32 runs them as one pass; the FP64 plain path runs them one after another.
int batch_common(fcm_handle* h, int nsys, const int* offsets, const void* pos, const void* F, const void* T,
                 void* U, void* W, int stages, void* stream) {
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  if (nsys < 0 || nsys > h->max_systems)
    return fail(FCM_ERR_ARG, "n_sys = " + std::to_string(nsys) + " outside [0, max_systems = " +
                                 std::to_string(h->max_systems) + "]");
  if (nsys == 0) return FCM_OK;
  if (!offsets) return fail(FCM_ERR_ARG, "offsets is NULL");
  if (offsets[0] != 0) return fail(FCM_ERR_ARG, "offsets[0] must be 0");
  for (int k = 0; k < nsys; ++k)
    if (offsets[k + 1] < offsets[k]) return fail(FCM_ERR_ARG, "offsets must be nondecreasing");
  const int n = offsets[nsys];
  if (n > h->p.max_n)
    return fail(FCM_ERR_ARG, "offsets[n_sys] = " + std::to_string(n) + " exceeds max_n = " + std::to_string(h->p.max_n));
  if (n > 0 && (!pos || !F || !U)) return fail(FCM_ERR_ARG, "pos, F and U must be non-NULL when particles are present");
  if (stages < 1 || stages > FCM_STAGE_ALL) return fail(FCM_ERR_ARG, "stages must be a non-empty subset of FCM_STAGE_ALL");
  if (n == 0) return FCM_OK;
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->fp64) {
    for (int k = 0; k < nsys; ++k) {
      const int nk = offsets[k + 1] - offsets[k];
      if (nk == 0) continue;
      const size_t o = 3 * (size_t)offsets[k];
      int rc = run<double>(h, 1, nk, (const double*)pos + o, (const double*)F + o, T ? (const double*)T + o : nullptr,
                           (double*)U + o, W ? (double*)W + o : nullptr, stages, false, s);
      if (rc) return rc;
    }
    return FCM_OK;
  }
  if (nsys > 1) {
    SysOffsets so;
    for (int k = 0; k <= nsys; ++k) so.off[k] = offsets[k];
    launch_write_offsets(so, nsys, h->sys_off, s, &h->launches);
  }
  return run<float>(h, nsys, n, (const float*)pos, (const float*)F, (const float*)T, (float*)U, (float*)W, stages,
                    false, s);
}

}  // namespace

namespace fcm {

// Captures one FP32 batched pass over `bucket` systems (a plan bucket of the handle) into a CUDA
// graph, for callers that replay the same pass shape many times. Before each replay the caller
// copies bucket + 1 offsets into handle_sys_off(h) on the replay stream (systems past the real
// ones repeat the total, so they are empty); the particle kernels read the total from there, and
// pos/F/T/U/W are the given device addresses (capacity max_n rows each).
int capture_batch_graph(fcm_handle* h, int bucket, const void* pos, const void* F, const void* T, void* U, void* W,
                        cudaStream_t s, cudaGraphExec_t* out) {
  *out = nullptr;
  if (!h || h->fp64) return fail(FCM_ERR_ARG, "graph capture needs an FP32 handle");
  const fcm_handle::Plan* plan = plan_for(h, bucket);
  if (bucket < 1 || bucket > h->max_systems || !plan || plan->systems != bucket)
    return fail(FCM_ERR_ARG, "bucket must be one of the handle's FFT plan buckets");
  if (h->timing) return fail(FCM_ERR_ARG, "stage timing is on; graphs are captured without it");
  DeviceGuard guard(h->device);
  FCM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  const int rc = run<float>(h, bucket, std::max(h->p.max_n, 1), (const float*)pos, (const float*)F, (const float*)T,
                            (float*)U, (float*)W, FCM_STAGE_ALL, false, s, h->sys_off + bucket);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || rc != FCM_OK || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (rc != FCM_OK) return rc;
    return fail(FCM_ERR_CUDA, std::string("graph capture failed: ") +
                                  cudaGetErrorString(e != cudaSuccess ? e : ee));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(FCM_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
  }
  return FCM_OK;
}

int handle_max_n(const fcm_handle* h) { return h ? h->p.max_n : 0; }

int* handle_sys_off(fcm_handle* h) { return h ? h->sys_off : nullptr; }

// Host checks of fcm_create (without touching a device): parameter ranges and the cutoff rule.
int check_params(const fcm_params* p, std::string* why) {
  if (!p) { *why = "params is NULL"; return 0; }
  if (!validate(p, why)) return 0;
  const double sg = p->a / std::sqrt(kPi), sD = p->a / std::cbrt(6.0 * std::sqrt(kPi));
  const double SigmaD = (p->Sigma_D == 0.0) ? p->Sigma : p->Sigma_D;
  const bool pairs_on = (p->Sigma > sg * (1 + 1e-12)) || (SigmaD > sD * (1 + 1e-12));
  if (pairs_on) {
    const double Lmin = std::min(p->L[0], std::min(p->L[1], p->L[2]));
    if (!(p->r_c > 0) || !(p->r_c <= 0.5 * Lmin)) { *why = "r_c must satisfy 0 < r_c <= min(L)/2"; return 0; }
    double cells = 1.0;
    for (int d = 0; d < 3; ++d) cells *= std::min(std::max(std::floor(p->L[d] / p->r_c), 3.0), 1048576.0);
    if (cells > (double)(1u << 26)) { *why = "too many pair cells (r_c too small for L)"; return 0; }
  }
  return 1;
}

// Device bytes fcm_create_batch(p, max_systems) would allocate (cuFFT work area estimated by cuFFT).
size_t workspace_estimate(const fcm_params& p, int max_systems) {
  const bool fp64 = p.precision == FCM_FP64;
  const int gsys = fp64 ? 1 : max_systems;
  int tile[3];
  if (fp64) { tile[0] = tile[1] = tile[2] = std::min(8, std::min(p.M[0], std::min(p.M[1], p.M[2]))); }
  else choose_tile(p, tile);
  Geometry<double> g{};
  fill_geometry(p, tile, &g, max_systems);
  const size_t n = (size_t)std::max(p.max_n, 1);
  const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
  const size_t v4 = fp64 ? sizeof(Vec4<double>) : sizeof(Vec4<float>);
  const size_t mtot = (size_t)p.M[0] * p.M[1] * p.M[2];
  const size_t ncplx = (size_t)(p.M[0] / 2 + 1) * p.M[1] * p.M[2];
  const size_t ntiles = (size_t)g.tiles_per * gsys, ncells = (size_t)g.cells_per * gsys;
  size_t b = 16 * n + 8 * (2 * ntiles + 1) + 8 * (ncells + 1) + 6 * v4 * n + 256 + 4 * (kMaxBatch + 1) + 9 * rsz * n;
  b += (3 * rsz * mtot + 6 * rsz * ncplx) * gsys + sizeof(float4) * 5 * kPairTableIntervals;
  int dims[3] = {p.M[2], p.M[1], p.M[0]};
  size_t w1 = 0, w2 = 0;
  if (cufftEstimateMany(3, dims, nullptr, 1, (int)mtot, nullptr, 1, (int)ncplx, fp64 ? CUFFT_D2Z : CUFFT_R2C,
                        3 * gsys, &w1) != CUFFT_SUCCESS)
    w1 = 6 * rsz * ncplx * gsys;
  if (cufftEstimateMany(3, dims, nullptr, 1, (int)ncplx, nullptr, 1, (int)mtot, fp64 ? CUFFT_Z2D : CUFFT_C2R,
                        3 * gsys, &w2) != CUFFT_SUCCESS)
    w2 = w1;
  return b + std::max(w1, w2) + 24 * 256;
}

}  // namespace fcm

namespace {

// Eigen-decomposition of a small symmetric matrix (row-major n x n) by cyclic Jacobi rotations:
// A = Q diag(w) Q^T. Used on the Lanczos tridiagonal matrix (n <= kLanczosMax).
void jacobi_eig(std::vector<double> A, int n, std::vector<double>* w, std::vector<double>* Q) {
  Q->assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) (*Q)[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = (*Q)[(size_t)k * n + p], qkq = (*Q)[(size_t)k * n + q];
          (*Q)[(size_t)k * n + p] = c * qkp - sn * qkq;
          (*Q)[(size_t)k * n + q] = sn * qkp + c * qkq;
        }
      }
  }
  w->resize(n);
  for (int i = 0; i < n; ++i) (*w)[i] = A[(size_t)i * n + i];
}

static_assert(kLanczosMax == FCM_LANCZOS_MAX_ITER, "the Lanczos coefficient block holds every iteration");
static_assert(kStatusNonFinite == FCM_STATUS_NONFINITE && kStatusWaitTimeout == FCM_STATUS_WAIT_TIMEOUT,
              "device status bits as the header names them");

// Lanczos coefficients c = |z| T^{1/2} e_1 for the k x k tridiagonal T (diagonal alpha, off-diagonal
// beta): the square root applied to z is then V c. False if T is not positive definite.
bool lanczos_coef(const std::vector<double>& alpha, const std::vector<double>& beta, int k, double znorm,
                  std::vector<double>* c) {
  std::vector<double> T((size_t)k * k, 0.0), w, Q;
  for (int i = 0; i < k; ++i) {
    T[(size_t)i * k + i] = alpha[i];
    if (i + 1 < k) T[(size_t)i * k + i + 1] = T[(size_t)(i + 1) * k + i] = beta[i];
  }
  jacobi_eig(T, k, &w, &Q);
  c->assign(k, 0.0);
  for (int j = 0; j < k; ++j) {
    if (!(w[j] > 0.0)) return false;
    const double s = std::sqrt(w[j]) * Q[(size_t)0 * k + j] * znorm;   // (Q^T e_1)_j = Q[0][j]
    for (int i = 0; i < k; ++i) (*c)[i] += Q[(size_t)i * k + j] * s;
  }
  return true;
}

// Grid part: white grid noise xi -> u_B = sqrt(2 kT / h^3) G^{1/2} xi -> interpolated (U, W).
template <typename R>
int brownian_grid(fcm_handle* h, int n, const R* pos, const R* xi, double kT, R* U, R* W, cudaStream_t s) {
  Geometry<R> g = *reinterpret_cast<const Geometry<R>*>(h->fp64 ? (const void*)&h->gd : (const void*)&h->gf);
  g.nsys = 1;
  BinBuffers bb = h->bb;
  bb.nsys = 1;
  bb.sys_off = nullptr;
  bb.n_dev = nullptr;
  bb.ntiles = g.tiles_per;
  const fcm_handle::Plan* plan = plan_for(h, 1);
  if (!plan) return fail(FCM_ERR_ARG, "no FFT plan for one system");
  launch_binning<R>(g, n, pos, pos, nullptr, bb, false, s, &h->launches);   // tile order (forces unused)
  FCM_CUDA(cudaMemcpyAsync(h->grid, xi, h->grid_bytes, cudaMemcpyDeviceToDevice, s));
  const double h3 = (h->p.L[0] / h->p.M[0]) * (h->p.L[1] / h->p.M[1]) * (h->p.L[2] / h->p.M[2]);
  const R factor = (R)std::sqrt(2.0 * kT / h3);
  FCM_CUFFT(cufftSetStream(plan->r2c, s));
  FCM_CUFFT(cufftSetStream(plan->c2r, s));
  if constexpr (std::is_same<R, double>::value) {
    FCM_CUFFT(cufftExecD2Z(plan->r2c, (cufftDoubleReal*)h->grid, (cufftDoubleComplex*)h->spec));
    launch_projection_sqrt<double>(g, h->p.eta, factor, h->spec, s, &h->launches);
    FCM_CUFFT(cufftExecZ2D(plan->c2r, (cufftDoubleComplex*)h->spec, (cufftDoubleReal*)h->grid));
    launch_gather_f64(g, h->kd, W != nullptr, bb, n, (const double*)h->grid, nullptr, nullptr, U, W, s, &h->launches);
  } else {
    FCM_CUFFT(cufftExecR2C(plan->r2c, (cufftReal*)h->grid, (cufftComplex*)h->spec));
    launch_projection_sqrt<float>(g, (float)h->p.eta, factor, h->spec, s, &h->launches);
    FCM_CUFFT(cufftExecC2R(plan->c2r, (cufftComplex*)h->spec, (cufftReal*)h->grid));
    launch_gather_f32(g, h->kf, W != nullptr, bb, (const float*)h->grid, nullptr, nullptr, U, W, s, &h->launches);
  }
  FCM_CUDA(cudaGetLastError());
  return FCM_OK;
}

int read_dot(fcm_handle* h, cudaStream_t s, double* v) {
  FCM_CUDA(cudaMemcpyAsync(v, h->lz_dot, sizeof(double), cudaMemcpyDeviceToHost, s));
  FCM_CUDA(cudaStreamSynchronize(s));
  return FCM_OK;
}

// Pair part: U += sqrt(2 kT) (M - M~)^{1/2} z by Lanczos (Krylov basis V, tridiagonal T), the
// matrix-vector product being the pair stage applied to forces.
template <typename R>
int brownian_pair(fcm_handle* h, int n, const R* pos, const R* z, double kT, R* U, int max_iter, double tol,
                  int* iterations, cudaStream_t s) {
  const size_t m = 3 * (size_t)n;
  const size_t need = sizeof(R) * m * (size_t)(max_iter + 1);
  if (h->lz_bytes < need) {
    if (h->lz) cudaFree(h->lz);
    h->lz = nullptr;
    h->lz_bytes = 0;
    cudaError_t e = cudaMalloc(&h->lz, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(FCM_ERR_OOM, "Lanczos workspace of " + std::to_string(need) + " bytes: " + cudaGetErrorString(e));
    }
    h->lz_bytes = need;
  }
  if (!h->lz_dot) FCM_CUDA(cudaMalloc((void**)&h->lz_dot, sizeof(double)));
  R* V = (R*)h->lz;
  R* w = V + m * (size_t)max_iter;
  int rc;
  double zz = 0.0;
  launch_dot<R>(z, z, m, h->lz_dot, s, &h->launches);
  if ((rc = read_dot(h, s, &zz))) return rc;
  *iterations = 0;
  if (!(zz > 0.0)) return FCM_OK;
  const double znorm = std::sqrt(zz);
  launch_axpby<R>(V, 1.0 / znorm, z, 0.0, m, s, &h->launches);
  std::vector<double> alpha, beta, c, cprev;
  int k = 0;
  for (int j = 0; j < max_iter; ++j) {
    R* vj = V + m * (size_t)j;
    if ((rc = run<R>(h, 1, n, pos, vj, nullptr, w, nullptr, FCM_STAGE_PAIR, false, s))) return rc;
    if (j > 0) launch_axpby<R>(w, -beta[j - 1], V + m * (size_t)(j - 1), 1.0, m, s, &h->launches);
    double a = 0.0, bb2 = 0.0;
    launch_dot<R>(w, vj, m, h->lz_dot, s, &h->launches);
    if ((rc = read_dot(h, s, &a))) return rc;
    launch_axpby<R>(w, -a, vj, 1.0, m, s, &h->launches);
    launch_dot<R>(w, w, m, h->lz_dot, s, &h->launches);
    if ((rc = read_dot(h, s, &bb2))) return rc;
    alpha.push_back(a);
    k = j + 1;
    if (!lanczos_coef(alpha, beta, k, znorm, &c))
      return fail(FCM_ERR_INPUT, "the pairwise correction is not positive definite on this Krylov space");
    double diff = 0.0, cn = 0.0;
    for (int i = 0; i < k; ++i) {
      const double d = c[i] - (i < (int)cprev.size() ? cprev[i] : 0.0);
      diff += d * d;
      cn += c[i] * c[i];
    }
    cprev = c;
    const double b = std::sqrt(std::max(bb2, 0.0));
    if ((j > 0 && diff <= tol * tol * cn) || b <= 1e-14 * std::fabs(a) || j + 1 == max_iter) break;
    beta.push_back(b);
    launch_axpby<R>(V + m * (size_t)(j + 1), 1.0 / b, w, 0.0, m, s, &h->launches);
  }
  LanczosCoef lc{};
  const double amp = std::sqrt(2.0 * kT);
  for (int i = 0; i < k; ++i) lc.c[i] = amp * c[i];
  launch_combine<R>(U, V, lc, k, m, true, s, &h->launches);
  FCM_CUDA(cudaGetLastError());
  *iterations = k;
  return FCM_OK;
}

template <typename R>
int brownian(fcm_handle* h, int n, const R* pos, double kT, const R* xi, const R* z, R* U, R* W, int max_iter,
             double tol, int* iterations, cudaStream_t s) {
  int rc;
  if (xi) {
    if ((rc = brownian_grid<R>(h, n, pos, xi, kT, U, W, s))) return rc;
  } else {
    launch_zero(U, sizeof(R) * 3 * (size_t)n, s, &h->launches);
    if (W) launch_zero(W, sizeof(R) * 3 * (size_t)n, s, &h->launches);
  }
  int it = 0;
  if (z && h->pairs_on) {
    if ((rc = brownian_pair<R>(h, n, pos, z, kT, U, max_iter, tol, &it, s))) return rc;
  }
  if (iterations) *iterations = it;
  FCM_CUDA(cudaStreamSynchronize(s));
  return FCM_OK;
}

// Rigid-body mobility solve (Section 6.1) by Broyden's method from the diagonal-mobility
// Jacobian. Workspace carve-up of h->rg (256-byte aligned pieces):
//   arm 3n R | ginv 36 nb R | x, z: m R | V 3n R | steps (max_iter + 1) x stride R |
//   scalars: norm2[max_iter + 2], d rows (max_iter + 1) x ld, Gram rows (max_iter + 1) x ld,
//   coef[ld], one, ftnorm2, flags[4]
template <typename R>
int rigid_solve(fcm_handle* h, int n, const R* pos, int nb, const int* body_off, const R* X, const R* ft, R* F,
                R* UG, int max_iter, double tol, int precond, bool warm, int* iterations, double* residual,
                cudaStream_t s) {
  const size_t m = 3 * (size_t)n + 6 * (size_t)nb;
  const size_t stride = (m + 63) / 64 * 64;
  const int ld = max_iter + 2;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_arm = up(sizeof(R) * 3 * n), b_ginv = up(sizeof(R) * 36 * (size_t)nb);
  const size_t b_vec = up(sizeof(R) * m), b_V = b_arm, b_S = sizeof(R) * stride * (size_t)(max_iter + 1);
  const size_t n_scal = (size_t)ld + 2 * (size_t)(max_iter + 1) * ld + ld + 2;
  const size_t b_scal = up(sizeof(double) * n_scal + 4 * sizeof(int));
  const size_t need = b_arm + b_ginv + 2 * b_vec + b_V + up(b_S) + b_scal;
  if (h->rg_bytes < need) {
    if (h->rg) cudaFree(h->rg);
    h->rg = nullptr;
    h->rg_bytes = 0;
    cudaError_t e = cudaMalloc(&h->rg, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(FCM_ERR_OOM, "rigid-solve workspace of " + std::to_string(need) + " bytes: " + cudaGetErrorString(e));
    }
    h->rg_bytes = need;
  }
  char* p = (char*)h->rg;
  R* arm = (R*)p; p += b_arm;
  R* ginv = (R*)p; p += b_ginv;
  R* x = (R*)p; p += b_vec;
  R* z = (R*)p; p += b_vec;
  R* V = (R*)p; p += b_V;
  R* S = (R*)p; p += up(b_S);
  double* scal = (double*)p;
  double* norm2 = scal;
  double* drow = norm2 + ld;
  double* gram = drow + (size_t)(max_iter + 1) * ld;
  double* coef = gram + (size_t)(max_iter + 1) * ld;
  double* one = coef + ld;
  double* ftn2 = one + 1;
  int* flags = (int*)(ftn2 + 1);
  const double mu = 1.0 / (6.0 * kPi * h->p.eta * h->p.a);
  const double onev = 1.0;
  FCM_CUDA(cudaMemsetAsync(scal, 0, b_scal, s));
  FCM_CUDA(cudaMemcpyAsync(one, &onev, sizeof(double), cudaMemcpyHostToDevice, s));
  launch_rigid_setup<R>(pos, body_off, X, n, nb, h->p.L, arm, precond == FCM_RIGID_PRECOND_BODY ? nullptr : ginv,
                        flags, s, &h->launches);
  launch_dot<R>(ft, ft, 6 * (size_t)nb, ftn2, s, &h->launches);
  int hf[4] = {0, 0, 0, 0};
  double hft2 = 0.0;
  FCM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
  FCM_CUDA(cudaMemcpyAsync(&hft2, ftn2, sizeof(double), cudaMemcpyDeviceToHost, s));
  FCM_CUDA(cudaStreamSynchronize(s));
  if (hf[0]) return fail(FCM_ERR_INPUT, "body_off invalid at body " + std::to_string(hf[0] - 1));
  if (hf[1])
    return fail(FCM_ERR_INPUT, "body " + std::to_string(hf[1] - 1) + " is degenerate (K^T K singular: fewer than "
                               "3 particles off one line)");
  if (!std::isfinite(hft2)) return fail(FCM_ERR_INPUT, "ft is not finite");
  // body preconditioner: the inverse of [[M_bb / mu, -K], [K^T, 0]] per body, ms x ms each
  R* aT = nullptr;
  int ms = 0;
  if (precond == FCM_RIGID_PRECOND_BODY) {
    const int kmax = hf[3];
    if (kmax > kRigidBodyMax)
      return fail(FCM_ERR_INPUT, "the body preconditioner takes bodies of at most " + std::to_string(kRigidBodyMax) +
                                     " particles (largest: " + std::to_string(kmax) + ")");
    ms = 3 * kmax + 6;
    const size_t pneed = sizeof(R) * (size_t)ms * ms * (size_t)nb;
    if (h->rgp_bytes < pneed) {
      if (h->rgp) cudaFree(h->rgp);
      h->rgp = nullptr;
      h->rgp_bytes = 0;
      cudaError_t e = cudaMalloc(&h->rgp, pneed);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FCM_ERR_OOM, "body preconditioner of " + std::to_string(pneed) + " bytes: " + cudaGetErrorString(e));
      }
      h->rgp_bytes = pneed;
    }
    aT = (R*)h->rgp;
    launch_body_precond<R>(arm, body_off, nb, kmax, h->p.L, h->p.a, h->p.eta, aT, flags, s, &h->launches);
    FCM_CUDA(cudaGetLastError());
    FCM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    FCM_CUDA(cudaStreamSynchronize(s));
    if (hf[1])
      return fail(FCM_ERR_INPUT, "body " + std::to_string(hf[1] - 1) + ": its preconditioner block is singular");
  }
  auto residual_launch = [&](double* nrm) {
    if (aT)
      launch_rigid_residual_body<R>(V, x, ft, arm, aT, ms, body_off, n, nb, 1.0 / mu, z, nrm, s, &h->launches);
    else
      launch_rigid_residual<R>(V, x, ft, arm, ginv, body_off, n, nb, 1.0 / mu, z, nrm, s, &h->launches);
  };
  const double tau = tol * std::sqrt(hft2);
  int rc;
  auto finish = [&](int it, double nrm2) -> int {
    launch_axpby<R>(F, 1.0, x, 0.0, 3 * (size_t)n, s, &h->launches);
    launch_axpby<R>(UG, mu, x + 3 * (size_t)n, 0.0, 6 * (size_t)nb, s, &h->launches);
    FCM_CUDA(cudaGetLastError());
    FCM_CUDA(cudaStreamSynchronize(s));
    if (iterations) *iterations = it;
    if (residual) *residual = hft2 > 0.0 ? std::sqrt(nrm2 / hft2) : std::sqrt(nrm2);
    return FCM_OK;
  };
  if (!warm && hft2 == 0.0) {
    launch_zero(x, sizeof(R) * m, s, &h->launches);
    return finish(0, 0.0);
  }
  if (warm) {
    launch_axpby<R>(x, 1.0, F, 0.0, 3 * (size_t)n, s, &h->launches);
    launch_axpby<R>(x + 3 * (size_t)n, 1.0 / mu, UG, 0.0, 6 * (size_t)nb, s, &h->launches);
    if ((rc = run<R>(h, 1, n, pos, x, nullptr, V, nullptr, FCM_STAGE_ALL, false, s))) return rc;
  } else {
    launch_zero(x, sizeof(R) * m, s, &h->launches);
    launch_zero(V, sizeof(R) * 3 * (size_t)n, s, &h->launches);
  }
  auto read_norm = [&](int k, double* v, int* breakdown) -> int {
    FCM_CUDA(cudaMemcpyAsync(v, norm2 + k, sizeof(double), cudaMemcpyDeviceToHost, s));
    FCM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    FCM_CUDA(cudaStreamSynchronize(s));
    *breakdown = hf[2];
    return FCM_OK;
  };
  double nrm2 = 0.0;
  int brk = 0;
  residual_launch(norm2);
  if ((rc = read_norm(0, &nrm2, &brk))) return rc;
  if (!std::isfinite(nrm2)) return fail(FCM_ERR_INPUT, "non-finite residual (check F and UG of a warm start)");
  if (std::sqrt(nrm2) <= tau) return finish(0, nrm2);
  // s_0 = z (coefficient 1), x += s_0, Gram row 0
  launch_broyden_step<R>(z, S, m, stride, 0, one, S, x, s, &h->launches);
  launch_multi_dot<R>(S, S, m, stride, 1, gram, s, &h->launches);
  for (int it = 0; it < max_iter; ++it) {
    const int nstep = it;   // steps s_0 .. s_nstep are stored, and x already includes s_nstep
    if ((rc = run<R>(h, 1, n, pos, x, nullptr, V, nullptr, FCM_STAGE_ALL, false, s))) return rc;
    residual_launch(norm2 + it + 1);
    if ((rc = read_norm(it + 1, &nrm2, &brk))) return rc;
    if (!std::isfinite(nrm2)) return fail(FCM_ERR_INPUT, "non-finite residual in the Broyden iteration");
    if (brk) {
      finish(it + 1, nrm2);
      return fail(FCM_ERR_NOT_CONVERGED, "Broyden update broke down (s_n . z = |s_n|^2) after " +
                                             std::to_string(it + 1) + " iterations");
    }
    if (std::sqrt(nrm2) <= tau) return finish(it + 1, nrm2);
    if (it + 1 == max_iter) break;
    double* d = drow + (size_t)it * ld;
    launch_multi_dot<R>(z, S, m, stride, nstep + 1, d, s, &h->launches);
    launch_broyden_coef(d, gram, ld, nstep, coef, flags, s, &h->launches);
    R* snext = S + (size_t)(nstep + 1) * stride;
    launch_broyden_step<R>(z, S, m, stride, nstep, coef, snext, x, s, &h->launches);
    launch_multi_dot<R>(snext, S, m, stride, nstep + 2, gram + (size_t)(nstep + 1) * ld, s, &h->launches);
  }
  if ((rc = finish(max_iter, nrm2))) return rc;
  return fail(FCM_ERR_NOT_CONVERGED, "relative residual " + std::to_string(std::sqrt(nrm2 / hft2)) + " above tol " +
                                         std::to_string(tol) + " after " + std::to_string(max_iter) + " iterations");
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

int fcm_brownian(fcm_handle* h, int n, const void* pos, double kT, const void* xi, const void* z, void* U, void* W,
                 int max_iter, double tol, int* iterations, void* stream) {
  if (iterations) *iterations = 0;
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  if (n < 0 || n > h->p.max_n)
    return fail(FCM_ERR_ARG, "n = " + std::to_string(n) + " outside [0, max_n = " + std::to_string(h->p.max_n) + "]");
  if (!(kT > 0.0) || !std::isfinite(kT)) return fail(FCM_ERR_ARG, "kT must be finite and > 0");
  if (max_iter < 1 || max_iter > FCM_LANCZOS_MAX_ITER)
    return fail(FCM_ERR_ARG, "max_iter must be in [1, " + std::to_string(FCM_LANCZOS_MAX_ITER) + "]");
  if (!(tol > 0.0)) return fail(FCM_ERR_ARG, "tol must be > 0");
  if (n > 0 && (!pos || !U)) return fail(FCM_ERR_ARG, "pos and U must be non-NULL when n > 0");
  if (n == 0) return FCM_OK;
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->fp64)
    return brownian<double>(h, n, (const double*)pos, kT, (const double*)xi, (const double*)z, (double*)U,
                            (double*)W, max_iter, tol, iterations, s);
  return brownian<float>(h, n, (const float*)pos, kT, (const float*)xi, (const float*)z, (float*)U, (float*)W,
                         max_iter, tol, iterations, s);
}

int fcm_rigid_solve(fcm_handle* h, int n, const void* pos, int n_bodies, const int* body_off, const void* X,
                    const void* ft, void* F, void* UG, int max_iter, double tol, int precond, int warm,
                    int* iterations, double* residual, void* stream) {
  if (iterations) *iterations = 0;
  if (residual) *residual = 0.0;
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  if (n < 1 || n > h->p.max_n)
    return fail(FCM_ERR_ARG, "n = " + std::to_string(n) + " outside [1, max_n = " + std::to_string(h->p.max_n) + "]");
  if (n_bodies < 1 || n_bodies > n)
    return fail(FCM_ERR_ARG, "n_bodies = " + std::to_string(n_bodies) + " outside [1, n]");
  if (max_iter < 1 || max_iter > FCM_BROYDEN_MAX_ITER)
    return fail(FCM_ERR_ARG, "max_iter must be in [1, " + std::to_string(FCM_BROYDEN_MAX_ITER) + "]");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(FCM_ERR_ARG, "tol must be finite and > 0");
  if (precond != FCM_RIGID_PRECOND_DIAGONAL && precond != FCM_RIGID_PRECOND_BODY)
    return fail(FCM_ERR_ARG, "precond must be FCM_RIGID_PRECOND_DIAGONAL or FCM_RIGID_PRECOND_BODY");
  if (!pos || !body_off || !X || !ft || !F || !UG)
    return fail(FCM_ERR_ARG, "pos, body_off, X, ft, F and UG must be non-NULL");
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->fp64)
    return rigid_solve<double>(h, n, (const double*)pos, n_bodies, body_off, (const double*)X, (const double*)ft,
                               (double*)F, (double*)UG, max_iter, tol, precond, warm != 0, iterations, residual, s);
  return rigid_solve<float>(h, n, (const float*)pos, n_bodies, body_off, (const float*)X, (const float*)ft,
                            (float*)F, (float*)UG, max_iter, tol, precond, warm != 0, iterations, residual, s);
}

}  // extern "C"

extern "C" {

int fcm_version(void) { return 10000; }

int fcm_params_default(fcm_params* p) {
  if (!p) return fail(FCM_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->a = 1.0;
  p->eta = 1.0;
  p->precision = FCM_FP32;
  return FCM_OK;
}

int fcm_create(const fcm_params* p, int device, fcm_handle** out) { return fcm_create_batch(p, 1, device, out); }

int fcm_create_batch(const fcm_params* p, int max_systems, int device, fcm_handle** out) {
  if (!out) return fail(FCM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return fail(FCM_ERR_ARG, "params is NULL");
  if (max_systems < 1 || max_systems > FCM_MAX_BATCH)
    return fail(FCM_ERR_ARG, "max_systems must be in [1, " + std::to_string(FCM_MAX_BATCH) + "]");
  std::string why;
  if (!check_params(p, &why)) return fail(FCM_ERR_ARG, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(FCM_ERR_CUDA, "CUDA device " + std::to_string(device) + " is not available");
  }
  const double sg = p->a / std::sqrt(kPi), sD = p->a / std::cbrt(6.0 * std::sqrt(kPi));
  const double SigmaD = (p->Sigma_D == 0.0) ? p->Sigma : p->Sigma_D;
  const bool pairs_on = (p->Sigma > sg * (1 + 1e-12)) || (SigmaD > sD * (1 + 1e-12));
  if (pairs_on) {
    const double Lmin = std::min(p->L[0], std::min(p->L[1], p->L[2]));
    if (!(p->r_c > 0) || !(p->r_c <= 0.5 * Lmin)) return fail(FCM_ERR_ARG, "r_c must satisfy 0 < r_c <= min(L)/2");
  }
  fcm_handle* h = new fcm_handle();
  h->p = *p;
  h->p.Sigma_D = SigmaD;
  h->device = device;
  h->fp64 = (p->precision == FCM_FP64);
  h->pairs_on = pairs_on;
  h->max_systems = max_systems;
  const int gsys = h->fp64 ? 1 : max_systems;   // the FP64 path runs a batch one system at a time
  DeviceGuard guard(device);
  int tile[3];
  if (h->fp64) { tile[0] = tile[1] = tile[2] = std::min(8, std::min(p->M[0], std::min(p->M[1], p->M[2]))); }
  else choose_tile(*p, tile);
  for (int d = 0; d < 3; ++d) h->p.tile[d] = tile[d];
  fill_geometry(h->p, tile, &h->gf, max_systems);
  fill_geometry(h->p, tile, &h->gd, max_systems);
  fill_kernel_consts(h->p, SigmaD, &h->kf);
  fill_kernel_consts(h->p, SigmaD, &h->kd);
  make_pair_consts(p->a, p->eta, p->Sigma, SigmaD, pairs_on ? p->r_c : 0.0, 0.5 * sg, &h->pd);
  narrow_pair_consts(h->pd, &h->pf);
  if (!h->fp64 && (tile_smem_bytes(tile, p->M_G) > (size_t)tile_smem_limit() ||
                   spread_smem_bytes(tile, p->M_G) > (size_t)tile_smem_limit())) {
    release(h);
    return fail(FCM_ERR_ARG, "M_G too large for the FP32 tile kernels");
  }
  int rc = FCM_OK;
  auto A = [&](void** q, size_t bytes) { if (rc == FCM_OK) rc = halloc(h, q, bytes); };
  const size_t n = (size_t)std::max(p->max_n, 1);
  const size_t rsz = h->fp64 ? sizeof(double) : sizeof(float);
  const size_t v4 = h->fp64 ? sizeof(Vec4<double>) : sizeof(Vec4<float>);
  const size_t mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  const size_t ncplx = (size_t)(p->M[0] / 2 + 1) * p->M[1] * p->M[2];
  BinBuffers& b = h->bb;
  const double ntiles_d = (double)h->gf.ntile[0] * h->gf.ntile[1] * h->gf.ntile[2] * gsys;
  const double ncells_d = (double)h->gf.mcell[0] * h->gf.mcell[1] * h->gf.mcell[2] * gsys;
  if (pairs_on && ncells_d > (double)(1u << 26)) {
    release(h);
    return fail(FCM_ERR_ARG, "too many pair cells (r_c too small for L)");
  }
  if (ntiles_d > (double)(1u << 28)) {
    release(h);
    return fail(FCM_ERR_ARG, "too many tiles for one pass (grid or max_systems too large)");
  }
  b.ntiles = (int)ntiles_d;
  b.ncells = pairs_on ? (int)ncells_d : 1;
  A((void**)&b.tile_key, 4 * n); A((void**)&b.tile_rank, 4 * n);
  A((void**)&b.cell_key, 4 * n); A((void**)&b.cell_rank, 4 * n);
  A((void**)&b.tile_count, 4 * (size_t)(2 * b.ntiles + 1)); A((void**)&b.tile_start, 4 * (size_t)(2 * b.ntiles + 1));
  A((void**)&b.cell_count, 4 * (size_t)(b.ncells + 1)); A((void**)&b.cell_start, 4 * (size_t)(b.ncells + 1));
  A(&b.t_pos, v4 * n); A(&b.t_F, v4 * n); A(&b.t_T, v4 * n);
  A(&b.c_pos, v4 * n); A(&b.c_F, v4 * n); A(&b.c_T, v4 * n);
  A((void**)&b.status, 256);
  A((void**)&h->sys_off, sizeof(int) * (kMaxBatch + 1));
  A(&h->upair, 3 * rsz * n); A(&h->wpair, 3 * rsz * n); A(&h->wscratch, 3 * rsz * n);
  h->grid_bytes = 3 * rsz * mtot;
  h->spec_bytes = 3 * 2 * rsz * ncplx;
  A(&h->grid, h->grid_bytes * gsys);
  A(&h->spec, h->spec_bytes * gsys);
  void* table = nullptr;
  if (!h->fp64 && pairs_on) A(&table, sizeof(float4) * 5 * kPairTableIntervals);
  if (rc != FCM_OK) { std::string e = g_error; release(h); return fail(rc, e); }
  if (table) {
    const int nint = pair_table_intervals(0.5 * sg, std::max(p->r_c, 0.5 * sg + 1e-3), sg);
    std::vector<float4> host(5 * (size_t)nint);
    const double r_lo = 0.5 * sg;
    const double r_hi = std::max(p->r_c, r_lo + 1e-3);  // below r_lo only the series is used
    build_pair_table(h->pd, r_lo, r_hi, nint, host.data());
    if (cudaMemcpy(table, host.data(), sizeof(float4) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      release(h);
      return fail(FCM_ERR_CUDA, "copy of the pair table failed");
    }
    h->ptab.coef = (const float4*)table;
    h->ptab.r0 = (float)r_lo;
    h->ptab.inv_h = (float)(nint / (r_hi - r_lo));
    h->ptab.n = nint;
  }
  cudaError_t ce = cudaMemset(b.tile_count, 0, 4 * (size_t)(2 * b.ntiles + 1));
  if (ce == cudaSuccess) ce = cudaMemset(b.cell_count, 0, 4 * (size_t)(b.ncells + 1));
  if (ce == cudaSuccess) ce = cudaMemset(b.status, 0, 256);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (ce != cudaSuccess) { release(h); return fail(FCM_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(ce)); }
  // One R2C and one C2R plan per bucket of systems (3 transforms per system), all with one work
  // area of the largest size any of them needs.
  int dims[3] = {p->M[2], p->M[1], p->M[0]};
  std::vector<int> buckets;
  for (int k = 1; k < gsys; k *= 2) buckets.push_back(k);
  buckets.push_back(gsys);
  size_t work = 0;
  for (int nb : buckets) {
    fcm_handle::Plan pl{nb, 0, 0};
    size_t w1 = 0, w2 = 0;
    cufftResult fr = cufftCreate(&pl.r2c);
    if (fr == CUFFT_SUCCESS) {
      fr = cufftCreate(&pl.c2r);
      if (fr != CUFFT_SUCCESS) cufftDestroy(pl.r2c);
    }
    if (fr == CUFFT_SUCCESS) {
      h->plans.push_back(pl);
      fr = cufftSetAutoAllocation(pl.r2c, 0);
      if (fr == CUFFT_SUCCESS) fr = cufftSetAutoAllocation(pl.c2r, 0);
      if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(pl.r2c, 3, dims, nullptr, 1, (int)mtot, nullptr, 1, (int)ncplx,
                               h->fp64 ? CUFFT_D2Z : CUFFT_R2C, 3 * nb, &w1);
      if (fr == CUFFT_SUCCESS)
        fr = cufftMakePlanMany(pl.c2r, 3, dims, nullptr, 1, (int)ncplx, nullptr, 1, (int)mtot,
                               h->fp64 ? CUFFT_Z2D : CUFFT_C2R, 3 * nb, &w2);
    }
    if (fr != CUFFT_SUCCESS) {
      release(h);
      return fail(FCM_ERR_CUFFT, "cuFFT plan for " + std::to_string(nb) + " systems failed: " + std::to_string((int)fr));
    }
    work = std::max(work, std::max(w1, w2));
  }
  A(&h->fft_work, work);
  if (rc != FCM_OK) { std::string e = g_error; release(h); return fail(rc, e); }
  for (auto& pl : h->plans) {
    if (cufftSetWorkArea(pl.r2c, h->fft_work) != CUFFT_SUCCESS || cufftSetWorkArea(pl.c2r, h->fft_work) != CUFFT_SUCCESS) {
      release(h);
      return fail(FCM_ERR_CUFFT, "cufftSetWorkArea failed");
    }
  }
  // extra grids of a bucket start at zero and stay zero (every pass zeroes the bucket's grids)
  if (cudaMemset(h->grid, 0, h->grid_bytes * gsys) != cudaSuccess) {
    release(h);
    return fail(FCM_ERR_CUDA, "grid initialisation failed");
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { release(h); return fail(FCM_ERR_CUDA, "setup synchronisation failed"); }
  *out = h;
  return FCM_OK;
}

int fcm_destroy(fcm_handle* h) {
  release(h);
  return FCM_OK;
}

int fcm_apply(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* U, void* W, void* stream) {
  return apply_common(h, n, pos, F, T, U, W, FCM_STAGE_ALL, false, stream);
}

int fcm_apply_stages(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* U, void* W,
                     int stages, void* stream) {
  return apply_common(h, n, pos, F, T, U, W, stages, false, stream);
}

int fcm_batch_apply(fcm_handle* h, int n_sys, const int* offsets, const void* pos, const void* F, const void* T,
                    void* U, void* W, void* stream) {
  return batch_common(h, n_sys, offsets, pos, F, T, U, W, FCM_STAGE_ALL, stream);
}

int fcm_batch_apply_stages(fcm_handle* h, int n_sys, const int* offsets, const void* pos, const void* F,
                           const void* T, void* U, void* W, int stages, void* stream) {
  return batch_common(h, n_sys, offsets, pos, F, T, U, W, stages, stream);
}

int fcm_max_systems(const fcm_handle* h) { return h ? h->max_systems : 0; }

int fcm_spread(fcm_handle* h, int n, const void* pos, const void* F, const void* T, void* stream) {
  return apply_common(h, n, pos, F, T, nullptr, nullptr, FCM_STAGE_GRID, true, stream);
}

int fcm_copy_grid(fcm_handle* h, void* dst, void* stream) {
  if (!h || !dst) return fail(FCM_ERR_ARG, "handle and dst must be non-NULL");
  DeviceGuard guard(h->device);
  FCM_CUDA(cudaMemcpyAsync(dst, h->grid, h->grid_bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return FCM_OK;
}

int fcm_check(fcm_handle* h, void* stream, int timeout_ms, int* flags) {
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev;
  FCM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, s);
  cudaEventRecord(h->ev_fork, h->side);
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t a = cudaEventQuery(ev), b = cudaEventQuery(h->ev_fork);
    if (a == cudaSuccess && b == cudaSuccess) break;
    if ((a != cudaSuccess && a != cudaErrorNotReady) || (b != cudaSuccess && b != cudaErrorNotReady)) {
      cudaEventDestroy(ev);
      return fail(FCM_ERR_CUDA, std::string("device error: ") + cudaGetErrorString(a != cudaSuccess && a != cudaErrorNotReady ? a : b));
    }
    auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_ms) {
      cudaEventDestroy(ev);
      return fail(FCM_ERR_TIMEOUT, "work did not finish within " + std::to_string(timeout_ms) + " ms");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  int v = 0;
  FCM_CUDA(cudaMemcpy(&v, h->bb.status, sizeof(int), cudaMemcpyDeviceToHost));
  FCM_CUDA(cudaMemset(h->bb.status, 0, sizeof(int)));
  if (flags) *flags = v;
  if (v) return fail(FCM_ERR_INPUT, "non-finite particle position seen");
  return FCM_OK;
}

int fcm_set_timing(fcm_handle* h, int enable) {
  if (!h) return fail(FCM_ERR_ARG, "handle is NULL");
  DeviceGuard guard(h->device);
  if (enable && h->pool.empty()) {
    h->pool.resize(6 * 256);
    for (auto& ev : h->pool) {
      FCM_CUDA(cudaEventCreate(&ev.a));
      FCM_CUDA(cudaEventCreate(&ev.b));
    }
  }
  h->timing = enable != 0;
  return FCM_OK;
}

int fcm_read_timing(fcm_handle* h, double* ms, long long* counts) {
  if (!h || !ms || !counts) return fail(FCM_ERR_ARG, "handle, ms and counts must be non-NULL");
  DeviceGuard guard(h->device);
  int rc = fold_pending(h);
  if (rc) return rc;
  for (int k = 0; k < FCM_NUM_STAGES; ++k) {
    ms[k] = h->ms[k];
    counts[k] = h->counts[k];
    h->ms[k] = 0.0;
    h->counts[k] = 0;
  }
  return FCM_OK;
}

long long fcm_launch_count(const fcm_handle* h) { return h ? h->launches : 0; }

size_t fcm_workspace_bytes(const fcm_handle* h) { return h ? h->bytes : 0; }

int fcm_cutoff_radius(double Sigma, double Sigma_D, double a, double eta, double tol, int torques, double* r_c) {
  if (!r_c) return fail(FCM_ERR_ARG, "r_c is NULL");
  if (!(a > 0) || !(eta > 0) || !(tol > 0) || !(Sigma > 0)) return fail(FCM_ERR_ARG, "a, eta, tol, Sigma must be > 0");
  if (Sigma_D == 0.0) Sigma_D = Sigma;
  PairConsts<double> C;
  make_pair_consts(a, eta, Sigma, Sigma_D, 1e300, 0.0, &C);
  const double pi = kPi;
  const double nvf = 6 * pi * eta * a, nwt = 8 * pi * eta * a * a * a, nwf = std::sqrt(nvf * nwt);
  auto norm = [&](double r) {
    double al, bt, cr, gm, dl;
    pair_coeffs<double>(r * r, C, al, bt, cr, gm, dl);
    double v = std::max(std::fabs(al), std::fabs(al + bt * r * r)) * nvf;
    if (torques) {
      v = std::max(v, std::max(std::fabs(gm), std::fabs(gm + dl * r * r)) * nwt);
      v = std::max(v, std::fabs(cr) * r * nwf);
    }
    return v;
  };
  const double rmax = 40.0 * std::max(Sigma, Sigma_D);
  const int steps = 40000;
  double prev = rmax;
  double lo = -1, hi = -1;
  for (int k = 0; k < steps; ++k) {
    double r = rmax - (rmax - 1e-3) * k / (steps - 1);
    if (norm(r) >= tol) {
      if (k == 0) return fail(FCM_ERR_ARG, "correction still above tol at 40 Sigma");
      lo = r;
      hi = prev;
      break;
    }
    prev = r;
  }
  if (lo < 0) { *r_c = 0.0; return FCM_OK; }
  for (int it = 0; it < 80; ++it) {
    double mid = 0.5 * (lo + hi);
    if (norm(mid) >= tol) lo = mid; else hi = mid;
  }
  *r_c = hi;
  return FCM_OK;
}

const char* fcm_last_error(void) { return g_error.c_str(); }

}  // extern "C"
#pragma GCC visibility pop
