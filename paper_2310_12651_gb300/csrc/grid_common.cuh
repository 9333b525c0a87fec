// Shared pieces of the FP32 tile kernels (spread_f32.cu, gather_f32.cu).
//
// A tile is tile[0] x tile[1] x tile[2] grid points; its particles are the
// tile-sorted range whose windows start in the tile, so all their windows lie
// in the tile extended by M_G - 1 points (the extended region, EX x EY x EZ).
// Along a grid row (fixed y, z) each particle's contribution is a combination
// of three x profiles of its separable Gaussian: g(x), d^2 g(x), d g_D(x)
// (plus g_D(x) when the torque width differs); per point that is 8 FMA for
// force + torque with Sigma_D = Sigma.
#pragma once

#include "fcm_internal.cuh"

namespace fcm {

constexpr unsigned kFullMask32 = 0xffffffffu;
constexpr int kRowsMaxThreads = 512;   // row-stationary spread: one thread per extended (y, z) row
constexpr int kRowsChunk = 32;         // particles staged per pass

// Shared layout of the extended region: row pitch P (odd) and plane pitch Q
// with Q = P M_G (mod 32), so the 32 lanes of a warp, which own 32 consecutive
// window rows (jy + M_G jz), hit 32 different banks.
struct ExtLayout {
  int EX, EY, EZ;
  int P, Q, C;  // row pitch, plane pitch, component stride (floats)
};

__host__ __device__ inline ExtLayout ext_layout(const int tile[3], int MG) {
  ExtLayout l;
  l.EX = tile[0] + MG - 1;
  l.EY = tile[1] + MG - 1;
  l.EZ = tile[2] + MG - 1;
  l.P = l.EX | 1;
  const int q = l.P * l.EY;
  const int want = (l.P * MG) & 31;
  l.Q = q + ((want - (q & 31)) & 31);
  l.C = l.Q * l.EZ;
  return l;
}

struct TileOrigin {
  int ox0, oy0, oz0;
};

__device__ inline TileOrigin tile_origin(const Geometry<float>& g, int t) {
  TileOrigin o;
  const int tx = t % g.ntile[0];
  const int ty = (t / g.ntile[0]) % g.ntile[1];
  const int tz = t / (g.ntile[0] * g.ntile[1]);
  o.ox0 = tx * g.tile[0];
  o.oy0 = ty * g.tile[1];
  o.oz0 = tz * g.tile[2];
  return o;
}

__device__ inline int wrap_index(int i, int M) {
  while (i >= M) i -= M;
  return i;
}

// Window start of a particle inside the extended region (clamped into the tile).
__device__ inline int4 window_offset(const Geometry<float>& g, const TileOrigin& o, float4 y) {
  int4 off;
  off.x = min(max(pmod(window_start(y.x, g.h[0], g.MG), g.M[0]) - o.ox0, 0), g.tile[0] - 1);
  off.y = min(max(pmod(window_start(y.y, g.h[1], g.MG), g.M[1]) - o.oy0, 0), g.tile[1] - 1);
  off.z = min(max(pmod(window_start(y.z, g.h[2], g.MG), g.M[2]) - o.oz0, 0), g.tile[2] - 1);
  off.w = 0;
  return off;
}

// Rows (c, z, y) of the extended region visited by one warp as a contiguous
// block: one division at the start, then carries. gy, gz are the wrapped grid
// coordinates of the row. Lane l owns x offset l (EX <= 31).
struct RowWalk {
  int c, ez, ey, gy, gz, r, r1;
};

__device__ inline RowWalk row_walk_begin(const Geometry<float>& g, const TileOrigin& o, const ExtLayout& l) {
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int rows = 3 * l.EY * l.EZ;
  const int per = (rows + nwarp - 1) / nwarp;
  RowWalk w;
  w.r = min(warp * per, rows);
  w.r1 = min(w.r + per, rows);
  w.c = w.r / (l.EY * l.EZ);
  const int rem = w.r - w.c * l.EY * l.EZ;
  w.ez = rem / l.EY;
  w.ey = rem - w.ez * l.EY;
  w.gy = wrap_index(o.oy0 + w.ey, g.M[1]);
  w.gz = wrap_index(o.oz0 + w.ez, g.M[2]);
  return w;
}

__device__ inline void row_walk_next(const Geometry<float>& g, const TileOrigin& o, const ExtLayout& l, RowWalk& w) {
  ++w.r;
  if (++w.ey == l.EY) {
    w.ey = 0;
    w.gy = wrap_index(o.oy0, g.M[1]);
    if (++w.ez == l.EZ) {
      w.ez = 0;
      ++w.c;
      w.gz = wrap_index(o.oz0, g.M[2]);
    } else {
      w.gz = (w.gz + 1 == g.M[2]) ? 0 : w.gz + 1;
    }
  } else {
    w.gy = (w.gy + 1 == g.M[1]) ? 0 : w.gy + 1;
  }
}

// Global reduction of four consecutive floats (16-byte aligned address).
__device__ inline void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Per-particle profile tables staged in shared memory (row-stationary spread).
struct RowTables {
  float4* xt;   // [chunk][MGT] {g, d^2 g, d g_D, g_D} along x
  float4* yt;   // [chunk][MGT] {g, d, g_D, 0} along y
  float4* zt;   // [chunk][MGT] {g, d, g_D, 0} along z
  float4* pf;   // [chunk] force
  float4* pt;   // [chunk] torque
  int4* po;     // [chunk] window start inside the extended region
};

template <int MGT>
__device__ inline RowTables row_tables(float4* sm) {
  RowTables t;
  t.xt = sm;
  t.yt = t.xt + kRowsChunk * MGT;
  t.zt = t.yt + kRowsChunk * MGT;
  t.pf = t.zt + kRowsChunk * MGT;
  t.pt = t.pf + kRowsChunk;
  t.po = reinterpret_cast<int4*>(t.pt + kRowsChunk);
  return t;
}

__host__ __device__ constexpr size_t row_tables_bytes(int MGT) {
  return sizeof(float4) * (3 * (size_t)kRowsChunk * MGT + 2 * kRowsChunk) + sizeof(int4) * kRowsChunk;
}

// Kernel variants: MGT is the compiled support; GUARD says whether the runtime
// M_G may be smaller (then every point is guarded by j < M_G).
#define FCM_DISPATCH_MG(MG, CALL)                                              \
  switch (MG) {                                                                \
    case 10: CALL(10, false); break;                                           \
    case 12: CALL(12, false); break;                                           \
    case 14: CALL(14, false); break;                                           \
    case 16: CALL(16, false); break;                                           \
    default:                                                                   \
      if ((MG) <= 8) { CALL(8, true); }                                        \
      else if ((MG) <= 12) { CALL(12, true); }                                 \
      else if ((MG) <= 16) { CALL(16, true); }                                 \
      else if ((MG) <= 20) { CALL(20, true); }                                 \
      else { CALL(24, true); }                                                 \
  }

#define FCM_DISPATCH_ROWS(MG, CALL)                                            \
  switch (MG) {                                                                \
    case 10: CALL(10, false); break;                                           \
    case 12: CALL(12, false); break;                                           \
    case 14: CALL(14, false); break;                                           \
    case 16: CALL(16, false); break;                                           \
    default:                                                                   \
      if ((MG) <= 8) { CALL(8, true); }                                        \
      else if ((MG) <= 12) { CALL(12, true); }                                 \
      else { CALL(16, true); }                                                 \
  }

}  // namespace fcm
