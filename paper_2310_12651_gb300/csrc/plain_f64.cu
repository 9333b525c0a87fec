// FP64 plain path: the same operators as the FP32 path, written the direct way.
//
// * spread: one block per particle; the 3 M_G one-dimensional kernel factors
//   sit in shared memory and each thread adds a row of M_G points to the grid
//   with global FP64 atomics (the block-per-particle scheme of Appendix C);
// * gather: one block per particle, thread partial sums then a block reduction;
// * pair correction: one thread per particle over the 27 neighbour cells with
//   the closed form in FP64 (Taylor series below r_series).
// Formulas as in grid_f32.cu and pair_f32.cu.
#include "fcm_internal.cuh"

namespace fcm {

constexpr int kBpp = 128;

struct Tables64 {
  double d[3][kMaxMG];
  double gS[3][kMaxMG];   // exp(-d^2/(2 Sigma^2))
  double gD[3][kMaxMG];   // exp(-d^2/(2 Sigma_D^2))
  int i0[3];
};

__device__ inline void fill_tables(const Geometry<double>& g, const KernelConsts<double>& kc,
                                   const Vec4<double>& y, Tables64& t) {
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    const double yd = d == 0 ? y.x : (d == 1 ? y.y : y.z);
    t.i0[d] = window_start_d(g, d, yd);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * g.MG; k += blockDim.x) {
    const int d = k / g.MG, j = k - d * g.MG;
    const double yd = d == 0 ? y.x : (d == 1 ? y.y : y.z);
    const double dd = (double)(t.i0[d] + j) * sel3(g.h, d) - yd;
    t.d[d][j] = dd;
    t.gS[d][j] = exp(-dd * dd * kc.inv2S2);
    t.gD[d][j] = exp(-dd * dd * kc.inv2SD2);
  }
  __syncthreads();
}

template <bool TORQUE>
__global__ void __launch_bounds__(kBpp) spread_bpp_f64(Geometry<double> g, KernelConsts<double> kc, int n,
                                                       const Vec4<double>* __restrict__ pos,
                                                       const Vec4<double>* __restrict__ Fv,
                                                       const Vec4<double>* __restrict__ Tv,
                                                       double* __restrict__ grid) {
  __shared__ Tables64 t;
  const int p = blockIdx.x;
  const Vec4<double> y = pos[p];
  const Vec4<double> f = Fv[p];
  Vec4<double> tq = {0.0, 0.0, 0.0, 0.0};
  if (TORQUE) tq = Tv[p];
  fill_tables(g, kc, y, t);
  const int MG = g.MG;
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  for (int r = threadIdx.x; r < MG * MG; r += blockDim.x) {
    const int jz = r / MG, jy = r - jz * MG;
    const double dy = t.d[1][jy], dz = t.d[2][jz];
    const double G = kc.nrm * t.gS[1][jy] * t.gS[2][jz];
    const double H = kc.tq * t.gD[1][jy] * t.gD[2][jz];
    const int gy_ = pmod(t.i0[1] + jy, g.M[1]);
    const int gz_ = pmod(t.i0[2] + jz, g.M[2]);
    double* row = grid + ((size_t)gz_ * g.M[1] + gy_) * g.M[0];
    for (int jx = 0; jx < MG; ++jx) {
      const double dx = t.d[0][jx];
      const double w = G * t.gS[0][jx] * (kc.A + kc.B * (dx * dx + dy * dy + dz * dz));
      double fx = f.x * w, fy = f.y * w, fz = f.z * w;
      if (TORQUE) {
        const double wt = H * t.gD[0][jx];
        fx += wt * (tq.y * dz - tq.z * dy);
        fy += wt * (tq.z * dx - tq.x * dz);
        fz += wt * (tq.x * dy - tq.y * dx);
      }
      const int gx_ = pmod(t.i0[0] + jx, g.M[0]);
      atomicAdd(row + gx_, fx);
      atomicAdd(row + Mtot + gx_, fy);
      atomicAdd(row + 2 * Mtot + gx_, fz);
    }
  }
}

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

template <bool TORQUE>
__global__ void __launch_bounds__(kBpp) gather_bpp_f64(Geometry<double> g, KernelConsts<double> kc, int n,
                                                       const Vec4<double>* __restrict__ pos,
                                                       const double* __restrict__ grid,
                                                       const double* __restrict__ upair,
                                                       const double* __restrict__ wpair,
                                                       double* __restrict__ U, double* __restrict__ W) {
  __shared__ Tables64 t;
  __shared__ double red[kBpp / 32];
  const int p = blockIdx.x;
  const Vec4<double> y = pos[p];
  fill_tables(g, kc, y, t);
  const int MG = g.MG;
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int r = threadIdx.x; r < MG * MG; r += blockDim.x) {
    const int jz = r / MG, jy = r - jz * MG;
    const double dy = t.d[1][jy], dz = t.d[2][jz];
    const double G = kc.nrm * t.gS[1][jy] * t.gS[2][jz];
    const double H = kc.tq * t.gD[1][jy] * t.gD[2][jz];
    const int gy_ = pmod(t.i0[1] + jy, g.M[1]);
    const int gz_ = pmod(t.i0[2] + jz, g.M[2]);
    const double* row = grid + ((size_t)gz_ * g.M[1] + gy_) * g.M[0];
    for (int jx = 0; jx < MG; ++jx) {
      const double dx = t.d[0][jx];
      const int gx_ = pmod(t.i0[0] + jx, g.M[0]);
      const double ux = row[gx_], uy = row[Mtot + gx_], uz = row[2 * Mtot + gx_];
      const double w = G * t.gS[0][jx] * (kc.A + kc.B * (dx * dx + dy * dy + dz * dz));
      acc[0] += w * ux; acc[1] += w * uy; acc[2] += w * uz;
      if (TORQUE) {
        const double wt = H * t.gD[0][jx];
        acc[3] += wt * (dy * uz - dz * uy);
        acc[4] += wt * (dz * ux - dx * uz);
        acc[5] += wt * (dx * uy - dy * ux);
      }
    }
  }
  double tot[6];
  for (int c = 0; c < (TORQUE ? 6 : 3); ++c) tot[c] = block_sum(acc[c], red);
  if (threadIdx.x == 0) {
    const size_t o = 3 * (size_t)index_from_w(y.w);
    for (int c = 0; c < 3; ++c) U[o + c] = kc.h3 * tot[c] + (upair ? upair[o + c] : 0.0);
    if (TORQUE && W)
      for (int c = 0; c < 3; ++c) W[o + c] = kc.h3 * tot[3 + c] + (wpair ? wpair[o + c] : 0.0);
  }
}

__device__ inline double min_image64(double d, double L) {
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

template <bool TORQUE>
__global__ void __launch_bounds__(128) pair_thread_f64(Geometry<double> g, PairConsts<double> pc, int n,
                                                       const Vec4<double>* __restrict__ cpos,
                                                       const Vec4<double>* __restrict__ cF,
                                                       const Vec4<double>* __restrict__ cT,
                                                       const int* __restrict__ cstart,
                                                       double* __restrict__ Uo, double* __restrict__ Wo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Vec4<double> yi = cpos[i];
  const int cx = cell_coord(yi.x, g.cellw_inv[0], g.mcell[0]);
  const int cy = cell_coord(yi.y, g.cellw_inv[1], g.mcell[1]);
  const int cz = cell_coord(yi.z, g.cellw_inv[2], g.mcell[2]);
  double u[3] = {0, 0, 0}, w[3] = {0, 0, 0};
  for (int ddz = -1; ddz <= 1; ++ddz)
    for (int ddy = -1; ddy <= 1; ++ddy)
      for (int ddx = -1; ddx <= 1; ++ddx) {
        const int c = pmod(cx + ddx, g.mcell[0]) +
                      g.mcell[0] * (pmod(cy + ddy, g.mcell[1]) + g.mcell[1] * pmod(cz + ddz, g.mcell[2]));
        for (int j = cstart[c]; j < cstart[c + 1]; ++j) {
          if (j == i) continue;
          const Vec4<double> yj = cpos[j];
          const double dx = min_image64(yi.x - yj.x, g.L[0]);
          const double dy = min_image64(yi.y - yj.y, g.L[1]);
          const double dz = min_image64(yi.z - yj.z, g.L[2]);
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < pc.rc2)) continue;
          double al, bt, cr, gm, dl;
          pair_coeffs<double>(r2, pc, al, bt, cr, gm, dl);
          const Vec4<double> Fj = cF[j];
          const double xF = dx * Fj.x + dy * Fj.y + dz * Fj.z;
          u[0] += al * Fj.x + bt * xF * dx;
          u[1] += al * Fj.y + bt * xF * dy;
          u[2] += al * Fj.z + bt * xF * dz;
          if (TORQUE) {
            const Vec4<double> Tj = cT[j];
            u[0] += cr * (Tj.y * dz - Tj.z * dy);
            u[1] += cr * (Tj.z * dx - Tj.x * dz);
            u[2] += cr * (Tj.x * dy - Tj.y * dx);
            const double xT = dx * Tj.x + dy * Tj.y + dz * Tj.z;
            w[0] += cr * (Fj.y * dz - Fj.z * dy) + gm * Tj.x + dl * xT * dx;
            w[1] += cr * (Fj.z * dx - Fj.x * dz) + gm * Tj.y + dl * xT * dy;
            w[2] += cr * (Fj.x * dy - Fj.y * dx) + gm * Tj.z + dl * xT * dz;
          }
        }
      }
  const Vec4<double> Fi = cF[i];
  const size_t o = 3 * (size_t)index_from_w(yi.w);
  Uo[o + 0] = u[0] + pc.selfVF * Fi.x;
  Uo[o + 1] = u[1] + pc.selfVF * Fi.y;
  Uo[o + 2] = u[2] + pc.selfVF * Fi.z;
  if (TORQUE && Wo) {
    const Vec4<double> Ti = cT[i];
    Wo[o + 0] = w[0] + pc.selfWT * Ti.x;
    Wo[o + 1] = w[1] + pc.selfWT * Ti.y;
    Wo[o + 2] = w[2] + pc.selfWT * Ti.z;
  }
}

void launch_spread_f64(const Geometry<double>& g, const KernelConsts<double>& kc, bool torque,
                       const BinBuffers& b, int n, double* grid, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  if (torque)
    spread_bpp_f64<true><<<n, kBpp, 0, s>>>(g, kc, n, (const Vec4<double>*)b.t_pos, (const Vec4<double>*)b.t_F,
                                            (const Vec4<double>*)b.t_T, grid);
  else
    spread_bpp_f64<false><<<n, kBpp, 0, s>>>(g, kc, n, (const Vec4<double>*)b.t_pos, (const Vec4<double>*)b.t_F,
                                             (const Vec4<double>*)b.t_T, grid);
  *launches += 1;
}

void launch_gather_f64(const Geometry<double>& g, const KernelConsts<double>& kc, bool torque,
                       const BinBuffers& b, int n, const double* grid, const double* up, const double* wp,
                       double* U, double* W, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  if (torque)
    gather_bpp_f64<true><<<n, kBpp, 0, s>>>(g, kc, n, (const Vec4<double>*)b.t_pos, grid, up, wp, U, W);
  else
    gather_bpp_f64<false><<<n, kBpp, 0, s>>>(g, kc, n, (const Vec4<double>*)b.t_pos, grid, up, wp, U, W);
  *launches += 1;
}

void launch_pair_f64(const Geometry<double>& g, const PairConsts<double>& pc, bool torque, const BinBuffers& b,
                     int n, double* upair, double* wpair, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  const int blocks = (n + 127) / 128;
  if (torque)
    pair_thread_f64<true><<<blocks, 128, 0, s>>>(g, pc, n, (const Vec4<double>*)b.c_pos,
                                                 (const Vec4<double>*)b.c_F, (const Vec4<double>*)b.c_T,
                                                 b.cell_start, upair, wpair);
  else
    pair_thread_f64<false><<<blocks, 128, 0, s>>>(g, pc, n, (const Vec4<double>*)b.c_pos,
                                                  (const Vec4<double>*)b.c_F, (const Vec4<double>*)b.c_T,
                                                  b.cell_start, upair, wpair);
  *launches += 1;
}

}  // namespace fcm
