// FP32 spread (J~^dagger + N~^dagger) and interpolation (J~ + N~) on tiles.
//
// Spread, Section 3.1 / 3.4 with the modified kernels:
//   f(x_g) += F Delta~(x_g - Y; Sigma) - (1/2) T x grad Delta(x_g - Y; Sigma_D)
// over the particle's M_G^3 window. Interpolation, the trapezoidal rule of
// Section 2.1 step 3:
//   U = h^3 sum_g u Delta~,  W = h^3 sum_g Delta(.; Sigma_D) (d x u) / (2 Sigma_D^2).
//
// Work decomposition (GB300): one CTA per grid tile of tile[0] x tile[1] x
// tile[2] points; its particles are the tile-sorted range whose window starts
// in the tile, so the windows all fall inside the tile extended by M_G - 1
// points. Spread accumulates into that extended region in shared memory
// (shared-memory atomics), then flushes it to the grid once with global
// reductions (the halo flush); the grid sees one reduction per extended point
// instead of one per particle point. Gather stages the extended region of u in
// shared memory once per tile. Inside a CTA a warp owns a particle; lanes own
// rows (y, z) of the window and walk x. The Gaussian is separable, so the M_G
// x-weights (and their d and d^2 moments) are computed by M_G lanes and
// broadcast into registers with warp shuffles; per point the force part costs
// 2 FMA per component and the torque part 1 more for two of them.
#include "fcm_internal.cuh"

namespace fcm {

constexpr unsigned kFull = 0xffffffffu;

struct TileCoords {
  int ox0, oy0, oz0, EX, EY, EZ, E;
};

__device__ inline TileCoords tile_coords(const Geometry<float>& g, int t) {
  TileCoords c;
  int tx = t % g.ntile[0];
  int ty = (t / g.ntile[0]) % g.ntile[1];
  int tz = t / (g.ntile[0] * g.ntile[1]);
  c.ox0 = tx * g.tile[0];
  c.oy0 = ty * g.tile[1];
  c.oz0 = tz * g.tile[2];
  c.EX = g.tile[0] + g.MG - 1;
  c.EY = g.tile[1] + g.MG - 1;
  c.EZ = g.tile[2] + g.MG - 1;
  c.E = c.EX * c.EY * c.EZ;
  return c;
}

__device__ inline int wrap_index(int i, int M) {
  while (i >= M) i -= M;
  return i;
}

// Per-particle window data held by the lanes of the warp that owns it.
struct WindowLane {
  int ox, oy, oz;        // window start inside the extended region
  float dx, dy, dz;      // displacement of this lane's point (lane < MG) per dimension
  float gx, gy, gz;      // exp(-d^2 / (2 Sigma^2)) per dimension
  float gdx, gdy, gdz;   // exp(-d^2 / (2 Sigma_D^2)) per dimension
};

template <bool SAMEW>
__device__ inline WindowLane window_lane(const Geometry<float>& g, const KernelConsts<float>& kc,
                                         const TileCoords& tc, float4 y, int lane) {
  WindowLane w;
  int i0x = window_start(y.x, g.h[0], g.MG);
  int i0y = window_start(y.y, g.h[1], g.MG);
  int i0z = window_start(y.z, g.h[2], g.MG);
  w.ox = min(max(pmod(i0x, g.M[0]) - tc.ox0, 0), g.tile[0] - 1);
  w.oy = min(max(pmod(i0y, g.M[1]) - tc.oy0, 0), g.tile[1] - 1);
  w.oz = min(max(pmod(i0z, g.M[2]) - tc.oz0, 0), g.tile[2] - 1);
  w.dx = (float)(i0x + lane) * g.h[0] - y.x;
  w.dy = (float)(i0y + lane) * g.h[1] - y.y;
  w.dz = (float)(i0z + lane) * g.h[2] - y.z;
  w.gx = expf(-w.dx * w.dx * kc.inv2S2);
  w.gy = expf(-w.dy * w.dy * kc.inv2S2);
  w.gz = expf(-w.dz * w.dz * kc.inv2S2);
  if (!SAMEW) {
    w.gdx = expf(-w.dx * w.dx * kc.inv2SD2);
    w.gdy = expf(-w.dy * w.dy * kc.inv2SD2);
    w.gdz = expf(-w.dz * w.dz * kc.inv2SD2);
  } else {
    w.gdx = w.gx; w.gdy = w.gy; w.gdz = w.gz;
  }
  return w;
}

template <int MGT, bool TORQUE, bool SAMEW>
__global__ void __launch_bounds__(256) spread_tile_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                          const float4* __restrict__ pos,
                                                          const float4* __restrict__ Fv,
                                                          const float4* __restrict__ Tv,
                                                          const int* __restrict__ tstart,
                                                          float* __restrict__ grid) {
  extern __shared__ float acc[];
  const int t = blockIdx.x;
  const int p0 = tstart[t], p1 = tstart[t + 1];
  if (p0 >= p1) return;
  const TileCoords tc = tile_coords(g, t);
  for (int k = threadIdx.x; k < 3 * tc.E; k += blockDim.x) acc[k] = 0.f;
  __syncthreads();

  const int MG = g.MG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int p = p0 + warp; p < p1; p += nwarp) {
    const float4 y = pos[p];
    const float4 f = Fv[p];
    float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TORQUE) tq = Tv[p];
    const WindowLane w = window_lane<SAMEW>(g, kc, tc, y, lane);
    float gx[MGT], gx2[MGT], gx1[MGT], gdx[MGT];
#pragma unroll
    for (int j = 0; j < MGT; ++j) {
      float gj = __shfl_sync(kFull, w.gx, j);
      float dj = __shfl_sync(kFull, w.dx, j);
      gx[j] = gj;
      gx2[j] = dj * dj * gj;
      if (TORQUE) {
        float gdj = SAMEW ? gj : __shfl_sync(kFull, w.gdx, j);
        gdx[j] = gdj;
        gx1[j] = dj * gdj;
      }
    }
    const int nrows = MG * MG;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
      const int r = r0 + lane;
      const bool active = r < nrows;
      const int rr = active ? r : 0;
      const int jz = rr / MG, jy = rr - jz * MG;
      const float dy = __shfl_sync(kFull, w.dy, jy);
      const float gy = __shfl_sync(kFull, w.gy, jy);
      const float dz = __shfl_sync(kFull, w.dz, jz);
      const float gz = __shfl_sync(kFull, w.gz, jz);
      float gdy = gy, gdz = gz;
      if (TORQUE && !SAMEW) {
        gdy = __shfl_sync(kFull, w.gdy, jy);
        gdz = __shfl_sync(kFull, w.gdz, jz);
      }
      if (!active) continue;
      const float G = kc.nrm * gy * gz;
      const float Q = kc.A + kc.B * (dy * dy + dz * dz);
      float ax = f.x * G * Q, ay = f.y * G * Q, az = f.z * G * Q;
      const float bx = f.x * G * kc.B, by = f.y * G * kc.B, bz = f.z * G * kc.B;
      float* row = acc + ((w.oz + jz) * tc.EY + (w.oy + jy)) * tc.EX + w.ox;
      if (TORQUE) {
        const float H = kc.tq * gdy * gdz;
        const float cx = H * (tq.y * dz - tq.z * dy);  // times gdx
        const float cy = -H * tq.x * dz;                // times gdx
        const float cz = H * tq.x * dy;                 // times gdx
        const float ky = H * tq.z;                      // times d gdx
        const float kz = -H * tq.y;                     // times d gdx
        if (SAMEW) {
          ax += cx; ay += cy; az += cz;
#pragma unroll
          for (int j = 0; j < MGT; ++j) {
            if (j < MG) {
              atomicAdd(row + j, ax * gx[j] + bx * gx2[j]);
              atomicAdd(row + tc.E + j, ay * gx[j] + by * gx2[j] + ky * gx1[j]);
              atomicAdd(row + 2 * tc.E + j, az * gx[j] + bz * gx2[j] + kz * gx1[j]);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < MGT; ++j) {
            if (j < MG) {
              atomicAdd(row + j, ax * gx[j] + bx * gx2[j] + cx * gdx[j]);
              atomicAdd(row + tc.E + j, ay * gx[j] + by * gx2[j] + cy * gdx[j] + ky * gx1[j]);
              atomicAdd(row + 2 * tc.E + j, az * gx[j] + bz * gx2[j] + cz * gdx[j] + kz * gx1[j]);
            }
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < MGT; ++j) {
          if (j < MG) {
            atomicAdd(row + j, ax * gx[j] + bx * gx2[j]);
            atomicAdd(row + tc.E + j, ay * gx[j] + by * gx2[j]);
            atomicAdd(row + 2 * tc.E + j, az * gx[j] + bz * gx2[j]);
          }
        }
      }
    }
  }
  __syncthreads();
  // halo flush: one global reduction per non-zero point of the extended region
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  const int EXY = tc.EX * tc.EY;
  for (int k = threadIdx.x; k < 3 * tc.E; k += blockDim.x) {
    const float v = acc[k];
    if (v == 0.f) continue;
    const int c = k / tc.E;
    const int e = k - c * tc.E;
    const int ez = e / EXY;
    const int ey = (e - ez * EXY) / tc.EX;
    const int ex = e - ez * EXY - ey * tc.EX;
    const int gx_ = wrap_index(tc.ox0 + ex, g.M[0]);
    const int gy_ = wrap_index(tc.oy0 + ey, g.M[1]);
    const int gz_ = wrap_index(tc.oz0 + ez, g.M[2]);
    atomicAdd(grid + c * Mtot + ((size_t)gz_ * g.M[1] + gy_) * g.M[0] + gx_, v);
  }
}

template <int MGT, bool TORQUE, bool SAMEW>
__global__ void __launch_bounds__(256) gather_tile_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                          const float4* __restrict__ pos,
                                                          const int* __restrict__ tstart,
                                                          const float* __restrict__ grid,
                                                          const float* __restrict__ upair,
                                                          const float* __restrict__ wpair,
                                                          float* __restrict__ U, float* __restrict__ W) {
  extern __shared__ float acc[];
  const int t = blockIdx.x;
  const int p0 = tstart[t], p1 = tstart[t + 1];
  if (p0 >= p1) return;
  const TileCoords tc = tile_coords(g, t);
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  const int EXY = tc.EX * tc.EY;
  for (int k = threadIdx.x; k < 3 * tc.E; k += blockDim.x) {
    const int c = k / tc.E;
    const int e = k - c * tc.E;
    const int ez = e / EXY;
    const int ey = (e - ez * EXY) / tc.EX;
    const int ex = e - ez * EXY - ey * tc.EX;
    const int gx_ = wrap_index(tc.ox0 + ex, g.M[0]);
    const int gy_ = wrap_index(tc.oy0 + ey, g.M[1]);
    const int gz_ = wrap_index(tc.oz0 + ez, g.M[2]);
    acc[k] = grid[c * Mtot + ((size_t)gz_ * g.M[1] + gy_) * g.M[0] + gx_];
  }
  __syncthreads();

  const int MG = g.MG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int p = p0 + warp; p < p1; p += nwarp) {
    const float4 y = pos[p];
    const WindowLane w = window_lane<SAMEW>(g, kc, tc, y, lane);
    float gx[MGT], gx2[MGT], gx1[MGT], gdx[MGT];
#pragma unroll
    for (int j = 0; j < MGT; ++j) {
      float gj = __shfl_sync(kFull, w.gx, j);
      float dj = __shfl_sync(kFull, w.dx, j);
      gx[j] = gj;
      gx2[j] = dj * dj * gj;
      if (TORQUE) {
        float gdj = SAMEW ? gj : __shfl_sync(kFull, w.gdx, j);
        gdx[j] = gdj;
        gx1[j] = dj * gdj;
      }
    }
    float u0 = 0.f, u1 = 0.f, u2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
    const int nrows = MG * MG;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
      const int r = r0 + lane;
      const bool active = r < nrows;
      const int rr = active ? r : 0;
      const int jz = rr / MG, jy = rr - jz * MG;
      const float dy = __shfl_sync(kFull, w.dy, jy);
      const float gy = __shfl_sync(kFull, w.gy, jy);
      const float dz = __shfl_sync(kFull, w.dz, jz);
      const float gz = __shfl_sync(kFull, w.gz, jz);
      float gdy = gy, gdz = gz;
      if (TORQUE && !SAMEW) {
        gdy = __shfl_sync(kFull, w.gdy, jy);
        gdz = __shfl_sync(kFull, w.gdz, jz);
      }
      if (!active) continue;
      const float* row = acc + ((w.oz + jz) * tc.EY + (w.oy + jy)) * tc.EX + w.ox;
      float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, sx2 = 0.f, sy2 = 0.f, sz2 = 0.f;
      float dx0 = 0.f, dy0 = 0.f, dz0 = 0.f, dy1 = 0.f, dz1 = 0.f;
#pragma unroll
      for (int j = 0; j < MGT; ++j) {
        if (j < MG) {
          const float ux = row[j], uy = row[tc.E + j], uz = row[2 * tc.E + j];
          sx0 += gx[j] * ux; sy0 += gx[j] * uy; sz0 += gx[j] * uz;
          sx2 += gx2[j] * ux; sy2 += gx2[j] * uy; sz2 += gx2[j] * uz;
          if (TORQUE) {
            if (!SAMEW) { dx0 += gdx[j] * ux; dy0 += gdx[j] * uy; dz0 += gdx[j] * uz; }
            dy1 += gx1[j] * uy; dz1 += gx1[j] * uz;
          }
        }
      }
      const float G = kc.nrm * gy * gz;
      const float Q = kc.A + kc.B * (dy * dy + dz * dz);
      u0 += G * (Q * sx0 + kc.B * sx2);
      u1 += G * (Q * sy0 + kc.B * sy2);
      u2 += G * (Q * sz0 + kc.B * sz2);
      if (TORQUE) {
        if (SAMEW) { dx0 = sx0; dy0 = sy0; dz0 = sz0; }
        const float H = kc.tq * gdy * gdz;
        w0 += H * (dy * dz0 - dz * dy0);
        w1 += H * (dz * dx0 - dz1);
        w2 += H * (dy1 - dy * dx0);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      u0 += __shfl_xor_sync(kFull, u0, o);
      u1 += __shfl_xor_sync(kFull, u1, o);
      u2 += __shfl_xor_sync(kFull, u2, o);
      if (TORQUE) {
        w0 += __shfl_xor_sync(kFull, w0, o);
        w1 += __shfl_xor_sync(kFull, w1, o);
        w2 += __shfl_xor_sync(kFull, w2, o);
      }
    }
    if (lane == 0) {
      const size_t o = 3 * (size_t)index_from_w(y.w);
      float a0 = kc.h3 * u0, a1 = kc.h3 * u1, a2 = kc.h3 * u2;
      if (upair) { a0 += upair[o]; a1 += upair[o + 1]; a2 += upair[o + 2]; }
      U[o] = a0; U[o + 1] = a1; U[o + 2] = a2;
      if (TORQUE && W) {
        float b0 = kc.h3 * w0, b1 = kc.h3 * w1, b2 = kc.h3 * w2;
        if (wpair) { b0 += wpair[o]; b1 += wpair[o + 1]; b2 += wpair[o + 2]; }
        W[o] = b0; W[o + 1] = b1; W[o + 2] = b2;
      }
    }
  }
}

size_t tile_smem_bytes(const int tile[3], int MG) {
  return (size_t)3 * sizeof(float) * (tile[0] + MG - 1) * (tile[1] + MG - 1) * (tile[2] + MG - 1);
}

int tile_smem_limit() { return 227 * 1024; }

template <int MGT, bool TORQUE, bool SAMEW>
static void spread_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b,
                           float* grid, cudaStream_t s) {
  size_t smem = tile_smem_bytes(g.tile, g.MG);
  auto k = spread_tile_kernel<MGT, TORQUE, SAMEW>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<b.ntiles, 256, smem, s>>>(g, kc, (const float4*)b.t_pos, (const float4*)b.t_F, (const float4*)b.t_T,
                                b.tile_start, grid);
}

template <int MGT, bool TORQUE, bool SAMEW>
static void gather_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b,
                           const float* grid, const float* up, const float* wp, float* U, float* W,
                           cudaStream_t s) {
  size_t smem = tile_smem_bytes(g.tile, g.MG);
  auto k = gather_tile_kernel<MGT, TORQUE, SAMEW>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<b.ntiles, 256, smem, s>>>(g, kc, (const float4*)b.t_pos, b.tile_start, grid, up, wp, U, W);
}

#define FCM_DISPATCH_MG(MG, CALL)                 \
  if ((MG) <= 8) { CALL(8); }                     \
  else if ((MG) <= 12) { CALL(12); }              \
  else if ((MG) <= 16) { CALL(16); }              \
  else if ((MG) <= 20) { CALL(20); }              \
  else { CALL(24); }

void launch_spread_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque,
                       const BinBuffers& b, float* grid, cudaStream_t s, long long* launches) {
#define SPREAD_CALL(MGT)                                                        \
  if (!torque) spread_variant<MGT, false, true>(g, kc, b, grid, s);             \
  else if (kc.same_width) spread_variant<MGT, true, true>(g, kc, b, grid, s);   \
  else spread_variant<MGT, true, false>(g, kc, b, grid, s);
  FCM_DISPATCH_MG(g.MG, SPREAD_CALL)
#undef SPREAD_CALL
  *launches += 1;
}

void launch_gather_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque,
                       const BinBuffers& b, const float* grid, const float* up, const float* wp,
                       float* U, float* W, cudaStream_t s, long long* launches) {
#define GATHER_CALL(MGT)                                                                  \
  if (!torque) gather_variant<MGT, false, true>(g, kc, b, grid, up, wp, U, W, s);         \
  else if (kc.same_width) gather_variant<MGT, true, true>(g, kc, b, grid, up, wp, U, W, s); \
  else gather_variant<MGT, true, false>(g, kc, b, grid, up, wp, U, W, s);
  FCM_DISPATCH_MG(g.MG, GATHER_CALL)
#undef GATHER_CALL
  *launches += 1;
}

}  // namespace fcm
