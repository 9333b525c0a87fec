// FP32 interpolation J~ + N~ on tiles (trapezoidal rule of Section 2.1 step 3,
// eq. avg_particle_vel_mod and eq. avg_particle_rot_mod):
//   U = h^3 sum_g u(x_g) Delta~(x_g - Y; Sigma)
//   W = h^3 sum_g Delta(x_g - Y; Sigma_D) (d_g x u(x_g)) / (2 Sigma_D^2),  d_g = x_g - Y
// (the second line is (1/2) int (curl u) Delta after one integration by parts,
// the exact adjoint of the torque spread).
//
// One CTA per z-pencil of tiles, taking the tiles in turn: the extended region of u is held in
// shared memory as a ring of its z planes, and each step copies only the tile's new planes
// (tile_z of the E_Z, with asynchronous 4-byte copies, no register round trip); a warp owns a
// particle and its lanes own window rows; the M_G x-profiles are computed by
// M_G lanes and broadcast into registers with warp shuffles. Per point: a 4-byte
// load (x) and an 8-byte load (y, z interleaved) from shared memory and 8 FMA.
// The pair-correction sums, when present, are added when U and W are written
// in input order.
#include "grid_common.cuh"

namespace fcm {

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW>
__global__ void __launch_bounds__(256) gather_tile_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                          const float4* __restrict__ pos,
                                                          const int* __restrict__ tstart,
                                                          const float* __restrict__ grid,
                                                          const float* __restrict__ upair,
                                                          const float* __restrict__ wpair,
                                                          float* __restrict__ U, float* __restrict__ W,
                                                          int segl) {
  extern __shared__ float4 sm4[];
  float* acc = reinterpret_cast<float*>(sm4);
  // the CTA's segment (segl tiles) of a z-pencil of tiles (tx, ty, 0 .. ntile_z - 1) of one system, walked in z
  const int ntx = g.ntile[0], nty = g.ntile[1], ntz = g.ntile[2];
  const int per = ntx * nty;
  const int nseg = (ntz + segl - 1) / segl;
  const int sys = blockIdx.x / (per * nseg);
  const int rem = blockIdx.x - sys * per * nseg;
  const int pcl = rem / nseg;
  const int z0 = (rem - pcl * nseg) * segl, z1 = min(ntz, z0 + segl);
  const int tx = pcl % ntx, ty = pcl / ntx;
  const int tbase = sys * g.tiles_per + pcl;   // tile (tx, ty, 0): tiles are numbered x fastest
  if (g.nsys > 1) grid += (size_t)sys * (size_t)g.grid_stride;
  const int MG = GUARD ? g.MG : MGT;
  const ExtLayout l = ext_layout(g.tile, MG);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  TileOrigin pen;   // the pencil's origin: region plane ez of tile tz is pencil plane tz tile_z + ez
  pen.ox0 = tx * g.tile[0];
  pen.oy0 = ty * g.tile[1];
  pen.oz0 = 0;
  int staged = 0;   // pencil planes below this are in the ring (plane P in slot P mod E_Z)
  for (int tz = z0; tz < z1; ++tz) {
    const int t = tbase + per * tz;
    const int p0 = tstart[t], p1 = tstart[t + 1];
    if (p0 >= p1) continue;
    const int zlo = tz * g.tile[2];
    __syncthreads();   // every warp is done with the planes this step replaces
    stage_region_async(g, pen, l, grid, acc, max(staged, zlo), zlo + l.EZ);
    staged = zlo + l.EZ;
    __syncthreads();
    TileOrigin o = pen;
    o.oz0 = zlo;
    const int zs = zlo % l.EZ;   // ring slot of the tile's region plane 0

    for (int p = p0 + warp; p < p1; p += nwarp) {
      const float4 y = pos[p];
      const int3 i0 = window_starts(g, y);
      const int4 off = window_offset(g, o, i0);
      const float dxl = (float)(i0.x + lane) * g.h[0] - y.x;
      const float dyl = (float)(i0.y + lane) * g.h[1] - y.y;
      const float dzl = (float)(i0.z + lane) * g.h[2] - y.z;
      const float gxl = expf(-dxl * dxl * kc.inv2S2);
      const float gyl = expf(-dyl * dyl * kc.inv2S2);
      const float gzl = expf(-dzl * dzl * kc.inv2S2);
      const float gdxl = SAMEW ? gxl : expf(-dxl * dxl * kc.inv2SD2);
      const float gdyl = SAMEW ? gyl : expf(-dyl * dyl * kc.inv2SD2);
      const float gdzl = SAMEW ? gzl : expf(-dzl * dzl * kc.inv2SD2);
      float gx[MGT], gx2[MGT], gx1[MGT], gdx[MGT];
#pragma unroll
      for (int j = 0; j < MGT; ++j) {
        const float gj = __shfl_sync(kFullMask32, gxl, j);
        const float dj = __shfl_sync(kFullMask32, dxl, j);
        const float gdj = SAMEW ? gj : __shfl_sync(kFullMask32, gdxl, j);
        gx[j] = gj;
        gx2[j] = dj * dj * gj;
        gdx[j] = gdj;
        gx1[j] = dj * gdj;
      }
      float u0 = 0.f, u1 = 0.f, u2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
      // one window row (jy, jz) of this particle: x sums over the row, times the row's y, z factors
      auto row_update = [&](const float* row, int sy, int sz, bool active) {
        const float dy = __shfl_sync(kFullMask32, dyl, sy);
        const float gy = __shfl_sync(kFullMask32, gyl, sy);
        const float dz = __shfl_sync(kFullMask32, dzl, sz);
        const float gz = __shfl_sync(kFullMask32, gzl, sz);
        const float gdy = SAMEW ? gy : __shfl_sync(kFullMask32, gdyl, sy);
        const float gdz = SAMEW ? gz : __shfl_sync(kFullMask32, gdzl, sz);
        if (!active) return;
        if (!TORQUE) {   // forces only: one weight per point, w = GQ g + GB d^2 g, for the three components
          const float G = kc.nrm * gy * gz;
          const float GQ = G * fmaf(kc.B, fmaf(dy, dy, dz * dz), kc.A);
          const float GB = G * kc.B;
          float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
          for (int j = 0; j < MGT; ++j) {
            if (!GUARD || j < MG) {
              const float w = fmaf(GB, gx2[j], GQ * gx[j]);
              const float ux = row[j];
              const float2 uyz = reinterpret_cast<const float2*>(acc + yz_plane_offset(l))[(row - acc) + j];
              a0 = fmaf(w, ux, a0);
              a1 = fmaf(w, uyz.x, a1);
              a2 = fmaf(w, uyz.y, a2);
            }
          }
          u0 += a0;
          u1 += a1;
          u2 += a2;
          return;
        }
        float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, sx2 = 0.f, sy2 = 0.f, sz2 = 0.f;
        float dx0 = 0.f, dy0 = 0.f, dz0 = 0.f, dy1 = 0.f, dz1 = 0.f;
#pragma unroll
        for (int j = 0; j < MGT; ++j) {
          if (!GUARD || j < MG) {
            const float ux = row[j];
            const float2 uyz = reinterpret_cast<const float2*>(acc + yz_plane_offset(l))[(row - acc) + j];
            const float uy = uyz.x, uz = uyz.y;
            sx0 = fmaf(gx[j], ux, sx0); sy0 = fmaf(gx[j], uy, sy0); sz0 = fmaf(gx[j], uz, sz0);
            sx2 = fmaf(gx2[j], ux, sx2); sy2 = fmaf(gx2[j], uy, sy2); sz2 = fmaf(gx2[j], uz, sz2);
            if (TORQUE) {
              if (!SAMEW) { dx0 = fmaf(gdx[j], ux, dx0); dy0 = fmaf(gdx[j], uy, dy0); dz0 = fmaf(gdx[j], uz, dz0); }
              dy1 = fmaf(gx1[j], uy, dy1);
              dz1 = fmaf(gx1[j], uz, dz1);
            }
          }
        }
        const float G = kc.nrm * gy * gz;
        const float GQ = G * fmaf(kc.B, fmaf(dy, dy, dz * dz), kc.A);
        const float GB = G * kc.B;
        u0 = fmaf(GQ, sx0, fmaf(GB, sx2, u0));
        u1 = fmaf(GQ, sy0, fmaf(GB, sy2, u1));
        u2 = fmaf(GQ, sz0, fmaf(GB, sz2, u2));
        if (TORQUE) {
          if (SAMEW) { dx0 = sx0; dy0 = sy0; dz0 = sz0; }
          const float H = kc.tq * gdy * gdz;
          w0 = fmaf(H, dy * dz0 - dz * dy0, w0);
          w1 = fmaf(H, dz * dx0 - dz1, w1);
          w2 = fmaf(H, dy1 - dy * dx0, w2);
        }
      };
      if (!GUARD) {
        // window row r = jy + M_G jz of lane and pass it: fixed per lane, so the row offsets inside the
        // staged region (jz Q + jy P) are loop invariants of the particle loop
        int zb = zs + off.z;   // ring slot of the window's first plane
        if (zb >= l.EZ) zb -= l.EZ;
        const float* pbase = acc + off.y * l.P + off.x;
        constexpr int NFULL = MGT * MGT / 32, TAIL = MGT * MGT % 32;
        constexpr bool SPLIT_TAIL = TAIL > 0 && TAIL * MGT <= 64;   // a short last pass: split it by points
#pragma unroll
        for (int it = 0; it < (SPLIT_TAIL ? NFULL : (MGT * MGT + 31) / 32); ++it) {
          const int r = 32 * it + lane;
          const bool active = r < MGT * MGT;
          const int jz = active ? r / MGT : 0, jy = active ? r - (r / MGT) * MGT : 0;
          int sl = zb + jz;
          if (sl >= l.EZ) sl -= l.EZ;
          row_update(pbase + sl * l.Q + jy * l.P, jy, jz, active);
        }
        if (SPLIT_TAIL) {
          // the last TAIL rows have TAIL * M_G (row, point) items: each lane takes up to two and applies
          // the row's y, z factors to each item itself
#pragma unroll
          for (int pass = 0; pass < 2; ++pass) {
            const int e = lane + 32 * pass;
            const bool valid = e < TAIL * MGT;
            const int t = valid ? e / MGT : 0, j = valid ? e - (e / MGT) * MGT : 0;
            const int r = 32 * NFULL + t;
            const int jz = r / MGT, jy = r - jz * MGT;
            const float gj = __shfl_sync(kFullMask32, gxl, j);
            const float dj = __shfl_sync(kFullMask32, dxl, j);
            const float gdj = SAMEW ? gj : __shfl_sync(kFullMask32, gdxl, j);
            const float dy = __shfl_sync(kFullMask32, dyl, jy);
            const float gy = __shfl_sync(kFullMask32, gyl, jy);
            const float dz = __shfl_sync(kFullMask32, dzl, jz);
            const float gz = __shfl_sync(kFullMask32, gzl, jz);
            const float gdy = SAMEW ? gy : __shfl_sync(kFullMask32, gdyl, jy);
            const float gdz = SAMEW ? gz : __shfl_sync(kFullMask32, gdzl, jz);
            if (valid) {
              int sl = zb + jz;
              if (sl >= l.EZ) sl -= l.EZ;
              const float* row = pbase + sl * l.Q + jy * l.P;
              const float ux = row[j];
            const float2 uyz = reinterpret_cast<const float2*>(acc + yz_plane_offset(l))[(row - acc) + j];
            const float uy = uyz.x, uz = uyz.y;
              const float G = kc.nrm * gy * gz;
              const float GQ = G * fmaf(kc.B, fmaf(dy, dy, dz * dz), kc.A);
              const float GB = G * kc.B;
              const float wgt = fmaf(GB, dj * dj * gj, GQ * gj);
              u0 = fmaf(wgt, ux, u0);
              u1 = fmaf(wgt, uy, u1);
              u2 = fmaf(wgt, uz, u2);
              if (TORQUE) {
                const float H = kc.tq * gdy * gdz;
                const float g1 = dj * gdj;
                w0 = fmaf(H, gdj * (dy * uz - dz * uy), w0);
                w1 = fmaf(H, dz * gdj * ux - g1 * uz, w1);
                w2 = fmaf(H, g1 * uy - dy * gdj * ux, w2);
              }
            }
          }
        }
      } else {
        int jy = lane, jz = 0;
        while (jy >= MG) { jy -= MG; ++jz; }
        for (int r0 = 0; r0 < MG * MG; r0 += 32) {
          const bool active = r0 + lane < MG * MG;
          const int sy = active ? jy : 0, sz = active ? jz : 0;
          int sl = zs + off.z + sz;
          while (sl >= l.EZ) sl -= l.EZ;
          row_update(acc + sl * l.Q + (off.y + sy) * l.P + off.x, sy, sz, active);
          jy += 32;
          while (jy >= MG) { jy -= MG; ++jz; }
        }
      }
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        u0 += __shfl_xor_sync(kFullMask32, u0, s);
        u1 += __shfl_xor_sync(kFullMask32, u1, s);
        u2 += __shfl_xor_sync(kFullMask32, u2, s);
        if (TORQUE) {
          w0 += __shfl_xor_sync(kFullMask32, w0, s);
          w1 += __shfl_xor_sync(kFullMask32, w1, s);
          w2 += __shfl_xor_sync(kFullMask32, w2, s);
        }
      }
      if (lane == 0) {
        const size_t oi = 3 * (size_t)index_from_w(y.w);
        float a0 = kc.h3 * u0, a1 = kc.h3 * u1, a2 = kc.h3 * u2;
        if (upair) { a0 += upair[oi]; a1 += upair[oi + 1]; a2 += upair[oi + 2]; }
        U[oi] = a0; U[oi + 1] = a1; U[oi + 2] = a2;
        if (TORQUE && W) {
          float b0 = kc.h3 * w0, b1 = kc.h3 * w1, b2 = kc.h3 * w2;
          if (wpair) { b0 += wpair[oi]; b1 += wpair[oi + 1]; b2 += wpair[oi + 2]; }
          W[oi] = b0; W[oi + 1] = b1; W[oi + 2] = b2;
        }
      }
    }
  }
}

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW>
static void gather_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b,
                           const float* grid, const float* up, const float* wp, float* U, float* W,
                           cudaStream_t s) {
  const size_t smem = tile_smem_bytes(g.tile, g.MG);
  auto k = gather_tile_kernel<MGT, GUARD, TORQUE, SAMEW>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nsys = g.nsys > 1 ? g.nsys : 1;
  const int pencils = nsys * g.ntile[0] * g.ntile[1];
  // one CTA per z-pencil of tiles; pencils are split into segments when there are too few of them for
  // two waves of two CTAs per SM
  const int nseg = std::min(g.ntile[2], std::max(1, (4 * device_sm_count() + pencils - 1) / pencils));
  const int segl = (g.ntile[2] + nseg - 1) / nseg;
  const int blocks = pencils * ((g.ntile[2] + segl - 1) / segl);
  k<<<blocks, 256, smem, s>>>(g, kc, (const float4*)b.t_pos, b.tile_start, grid, up, wp, U, W, segl);
}

void launch_gather_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque,
                       const BinBuffers& b, const float* grid, const float* up, const float* wp,
                       float* U, float* W, cudaStream_t s, long long* launches) {
#define GATHER_CALL(MGT, GUARD)                                                                     \
  if (!torque) gather_variant<MGT, GUARD, false, true>(g, kc, b, grid, up, wp, U, W, s);           \
  else if (kc.same_width) gather_variant<MGT, GUARD, true, true>(g, kc, b, grid, up, wp, U, W, s); \
  else gather_variant<MGT, GUARD, true, false>(g, kc, b, grid, up, wp, U, W, s);
  FCM_DISPATCH_MG(g.MG, GATHER_CALL)
#undef GATHER_CALL
  *launches += 1;
}

}  // namespace fcm
