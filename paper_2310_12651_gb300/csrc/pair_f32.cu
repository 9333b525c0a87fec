// FP32 pairwise correction (Section 4 step 6, eq. correction_VF / WF / WT, Appendix B).
//
// For particle n and every m with minimum-image r = |Y_n - Y_m| < r_c:
//   U_n += al F_m + bt x (x.F_m) + cr (T_m x x)
//   W_n += cr (F_m x x) + gm T_m + dl x (x.T_m)
// with x = Y_n - Y_m and the radial coefficients of the closed form, read from
// piecewise-cubic tables built in FP64 (Taylor series for r < r_series, which
// also covers coincident points), plus the self correction. Candidates come
// from the 27 cells around n's cell (Section 4 step 1); cells adjacent in x are
// contiguous in the cell-sorted arrays, so a warp walks at most 9 ranges (more
// only where x wraps).
//
// GB300 decomposition: one warp per particle n. Lanes test 32 candidates at a
// time; hits are compacted with a ballot into a per-warp shared-memory queue,
// and the correction is evaluated when 32 hits are queued, so that work runs
// with every lane busy although only ~15% of candidates are within r_c.
// Per-lane sums are compensated (Neumaier); the warp reduction is a tree.
#include "fcm_internal.cuh"

namespace fcm {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kPairWarps = 8;
constexpr int kQueue = 64;

struct Neu {
  float s, c;
  __device__ inline void add(float v) {
    float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ inline float value() const { return s + c; }
};

__device__ inline float min_image(float d, float L) {
  if (d > 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return d;
}

template <bool TORQUE>
__device__ inline void eval_pair(const PairConsts<float>& pc, const PairTable& tab, float4 dq, float4 Fj, float4 Tj,
                                 Neu* u, Neu* w) {
  float al, bt, cr, gm, dl;
  pair_coeffs_table(dq.w, pc, tab, al, bt, cr, gm, dl);
  const float dx = dq.x, dy = dq.y, dz = dq.z;
  const float xF = dx * Fj.x + dy * Fj.y + dz * Fj.z;
  float u0 = al * Fj.x + bt * xF * dx;
  float u1 = al * Fj.y + bt * xF * dy;
  float u2 = al * Fj.z + bt * xF * dz;
  if (TORQUE) {
    // U += cr (T x x)
    u0 += cr * (Tj.y * dz - Tj.z * dy);
    u1 += cr * (Tj.z * dx - Tj.x * dz);
    u2 += cr * (Tj.x * dy - Tj.y * dx);
    const float xT = dx * Tj.x + dy * Tj.y + dz * Tj.z;
    // W += cr (F x x) + gm T + dl x (x.T)
    w[0].add(cr * (Fj.y * dz - Fj.z * dy) + gm * Tj.x + dl * xT * dx);
    w[1].add(cr * (Fj.z * dx - Fj.x * dz) + gm * Tj.y + dl * xT * dy);
    w[2].add(cr * (Fj.x * dy - Fj.y * dx) + gm * Tj.z + dl * xT * dz);
  }
  u[0].add(u0);
  u[1].add(u1);
  u[2].add(u2);
}

template <bool TORQUE>
__global__ void __launch_bounds__(kPairWarps * 32) pair_warp_kernel(Geometry<float> g, PairConsts<float> pc, PairTable tab, int n,
                                                                    const float4* __restrict__ cpos,
                                                                    const float4* __restrict__ cF,
                                                                    const float4* __restrict__ cT,
                                                                    const int* __restrict__ cstart,
                                                                    float* __restrict__ Uo,
                                                                    float* __restrict__ Wo) {
  __shared__ float4 qd[kPairWarps][kQueue];
  __shared__ int qj[kPairWarps][kQueue];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kPairWarps + warp;
  if (i >= n) return;
  const float4 yi = cpos[i];
  const int cx = cell_coord(yi.x, g.cellw_inv[0], g.mcell[0]);
  const int cy = cell_coord(yi.y, g.cellw_inv[1], g.mcell[1]);
  const int cz = cell_coord(yi.z, g.cellw_inv[2], g.mcell[2]);
  const int mx = g.mcell[0], my = g.mcell[1], mz = g.mcell[2];
  const unsigned lt = (1u << lane) - 1u;
  Neu u[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  Neu w[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  int qh = 0, qn = 0;
  for (int ddz = -1; ddz <= 1; ++ddz) {
    const int zc = pmod(cz + ddz, mz);
    for (int ddy = -1; ddy <= 1; ++ddy) {
      const int yc = pmod(cy + ddy, my);
      const int rowbase = mx * (yc + my * zc);
      // x neighbours cx-1, cx, cx+1 as at most two contiguous cell ranges
      int ra[2], rb[2], np = 0;
      if (cx - 1 >= 0 && cx + 1 < mx) { ra[0] = cx - 1; rb[0] = cx + 1; np = 1; }
      else if (cx - 1 < 0) { ra[0] = mx - 1; rb[0] = mx - 1; ra[1] = 0; rb[1] = 1; np = 2; }
      else { ra[0] = mx - 2; rb[0] = mx - 1; ra[1] = 0; rb[1] = 0; np = 2; }
      for (int piece = 0; piece < np; ++piece) {
        const int a = cstart[rowbase + ra[piece]];
        const int b = cstart[rowbase + rb[piece] + 1];
        for (int base = a; base < b; base += 32) {
          const int j = base + lane;
          bool hit = false;
          float4 dq = make_float4(0.f, 0.f, 0.f, 0.f);
          if (j < b && j != i) {
            const float4 yj = cpos[j];
            dq.x = min_image(yi.x - yj.x, g.L[0]);
            dq.y = min_image(yi.y - yj.y, g.L[1]);
            dq.z = min_image(yi.z - yj.z, g.L[2]);
            dq.w = dq.x * dq.x + dq.y * dq.y + dq.z * dq.z;
            hit = dq.w < pc.rc2;
          }
          const unsigned m = __ballot_sync(kFullMask, hit);
          if (hit) {
            const int slot = (qh + qn + __popc(m & lt)) & (kQueue - 1);
            qd[warp][slot] = dq;
            qj[warp][slot] = j;
          }
          qn += __popc(m);
          __syncwarp();
          if (qn >= 32) {
            const int slot = (qh + lane) & (kQueue - 1);
            const float4 e = qd[warp][slot];
            const int jj = qj[warp][slot];
            const float4 Fj = cF[jj];
            float4 Tj = make_float4(0.f, 0.f, 0.f, 0.f);
            if (TORQUE) Tj = cT[jj];
            eval_pair<TORQUE>(pc, tab, e, Fj, Tj, u, w);
            qh = (qh + 32) & (kQueue - 1);
            qn -= 32;
            __syncwarp();
          }
        }
      }
    }
  }
  if (lane < qn) {
    const int slot = (qh + lane) & (kQueue - 1);
    const float4 e = qd[warp][slot];
    const int jj = qj[warp][slot];
    const float4 Fj = cF[jj];
    float4 Tj = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TORQUE) Tj = cT[jj];
    eval_pair<TORQUE>(pc, tab, e, Fj, Tj, u, w);
  }
  float r[6] = {u[0].value(), u[1].value(), u[2].value(), w[0].value(), w[1].value(), w[2].value()};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 6; ++c) r[c] += __shfl_xor_sync(kFullMask, r[c], o);
  }
  if (lane == 0) {
    const float4 Fi = cF[i];
    const size_t o = 3 * (size_t)index_from_w(yi.w);
    Uo[o + 0] = r[0] + pc.selfVF * Fi.x;
    Uo[o + 1] = r[1] + pc.selfVF * Fi.y;
    Uo[o + 2] = r[2] + pc.selfVF * Fi.z;
    if (TORQUE && Wo) {
      const float4 Ti = cT[i];
      Wo[o + 0] = r[3] + pc.selfWT * Ti.x;
      Wo[o + 1] = r[4] + pc.selfWT * Ti.y;
      Wo[o + 2] = r[5] + pc.selfWT * Ti.z;
    }
  }
}

void launch_pair_f32(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab, bool torque,
                     const BinBuffers& b, int n, float* upair, float* wpair, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  const int blocks = (n + kPairWarps - 1) / kPairWarps;
  if (torque)
    pair_warp_kernel<true><<<blocks, kPairWarps * 32, 0, s>>>(g, pc, tab, n, (const float4*)b.c_pos,
                                                              (const float4*)b.c_F, (const float4*)b.c_T,
                                                              b.cell_start, upair, wpair);
  else
    pair_warp_kernel<false><<<blocks, kPairWarps * 32, 0, s>>>(g, pc, tab, n, (const float4*)b.c_pos,
                                                               (const float4*)b.c_F, (const float4*)b.c_T,
                                                               b.cell_start, upair, wpair);
  *launches += 1;
}

}  // namespace fcm
