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
constexpr int kRowsChunk = 64;         // particles staged per pass

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

// Tile t of a (possibly batched) launch: the tile's index inside its system, and in *grid_off
// the offset (reals) of that system's grid.
__device__ inline int local_tile(const Geometry<float>& g, int t, size_t* grid_off) {
  if (g.nsys > 1) {
    const int s = t / g.tiles_per;
    *grid_off = (size_t)s * (size_t)g.grid_stride;
    return t - s * g.tiles_per;
  }
  *grid_off = 0;
  return t;
}

__device__ inline int wrap_index(int i, int M) {
  while (i >= M) i -= M;
  return i;
}

// Window start (unwrapped grid index) of a particle along each axis.
__device__ inline int3 window_starts(const Geometry<float>& g, float4 y) {
  return make_int3(window_start_d(g, 0, y.x), window_start_d(g, 1, y.y), window_start_d(g, 2, y.z));
}

// Window start inside the extended region (clamped into the tile). Positions are
// wrapped into [0, L), so the window start lies in (-M, M) and one correction wraps it.
__device__ inline int4 window_offset(const Geometry<float>& g, const TileOrigin& o, int3 i0) {
  int4 off;
  off.x = min(max(wrap_once(i0.x, g.M[0]) - o.ox0, 0), g.tile[0] - 1);
  off.y = min(max(wrap_once(i0.y, g.M[1]) - o.oy0, 0), g.tile[1] - 1);
  off.z = min(max(wrap_once(i0.z, g.M[2]) - o.oz0, 0), g.tile[2] - 1);
  off.w = 0;
  return off;
}

// Offset (floats) of the interleaved (y, z) plane of the gather's staged region: after the x
// plane, rounded up to 8 bytes.
__host__ __device__ inline int yz_plane_offset(const ExtLayout& l) { return (l.C + 1) & ~1; }

// Copies z planes [pa, pb) of the extended region of the grid (3 components) into shared memory
// with asynchronous 4-byte copies: warps take (component, z) planes, lanes take x, rows advance by
// pointer increments (the y range is split at its periodic wrap, so no per-row wrap test). Plane
// ez is taken at grid z = o.oz0 + ez and goes to plane slot ez mod E_Z, so a CTA that walks a
// z-pencil of tiles keeps the region as a ring of E_Z planes and copies only the planes a step
// adds (pa, pb may exceed E_Z there; the default copies the whole region). Layout: the x component
// as one plane (index slot Q + ey P + ex), then the y and z components interleaved as float2 at
// the same index from yz_plane_offset, so the gather reads them with one 8-byte load.
__device__ inline void stage_region_async(const Geometry<float>& g, const TileOrigin& o, const ExtLayout& l,
                                          const float* __restrict__ grid, float* ext, int pa = 0, int pb = -1) {
  if (pb < 0) pb = l.EZ;
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int np = pb - pa;
  if (lane < l.EX && np > 0) {
    const int gx = wrap_index(o.ox0 + lane, g.M[0]);
    const int gy0 = wrap_index(o.oy0, g.M[1]);
    const int n1 = min(l.EY, g.M[1] - gy0);   // rows before the periodic wrap in y
    const size_t row = (size_t)g.M[0];
    for (int pl = warp; pl < 3 * np; pl += nwarp) {
      const int c = pl >= 2 * np ? 2 : (pl >= np ? 1 : 0);
      const int ez = pa + (pl - c * np);
      const int gz = wrap_index(o.oz0 + ez, g.M[2]);
      const int slot = ez % l.EZ;
      const float* gplane = grid + c * Mtot + (size_t)gz * g.M[1] * g.M[0] + gx;
      const int idx = slot * l.Q + lane;
      float* dst = c == 0 ? ext + idx : ext + yz_plane_offset(l) + 2 * idx + (c - 1);
      unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
      const unsigned sstep = (c == 0 ? 4u : 8u) * (unsigned)l.P;
      // rows gy0 .. gy0 + n1 - 1, then rows 0 .. EY - n1 - 1: pointers advance by one row each
      const float* src = gplane + (size_t)gy0 * row;
#pragma unroll 4
      for (int ey = 0; ey < n1; ++ey) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
        sa += sstep;
        src += row;
      }
      src = gplane;
      for (int ey = n1; ey < l.EY; ++ey) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
        sa += sstep;
        src += row;
      }
    }
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Adds the extended region held in shared memory to the grid: warps take
// (component, z) planes, lanes take x, coalesced global reductions, zeros skipped.
__device__ inline void flush_region(const Geometry<float>& g, const TileOrigin& o, const ExtLayout& l,
                                    const float* ext, float* __restrict__ grid) {
  const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (lane >= l.EX) return;
  const int gx = wrap_index(o.ox0 + lane, g.M[0]);
  const int gy0 = wrap_index(o.oy0, g.M[1]);
  for (int pl = warp; pl < 3 * l.EZ; pl += nwarp) {
    const int c = pl / l.EZ;
    const int ez = pl - c * l.EZ;
    const int gz = wrap_index(o.oz0 + ez, g.M[2]);
    float* gplane = grid + c * Mtot + (size_t)gz * g.M[1] * g.M[0] + gx;
    const float* splane = ext + c * l.C + ez * l.Q + lane;
    int gy = gy0;
    for (int ey = 0; ey < l.EY; ++ey) {
      const float v = splane[ey * l.P];
      if (v != 0.f) atomicAdd(gplane + (size_t)gy * g.M[0], v);
      gy = (gy + 1 == g.M[1]) ? 0 : gy + 1;
    }
  }
}

// TX = 8: one binning tile per CTA. TX = 16: two x-adjacent binning tiles (8 points each) per CTA;
// their particles are contiguous in the tile-sorted order (tiles are numbered x fastest), and the
// wider rows add about a third less halo to the grid per grid point.
template <int TX>
__device__ inline bool spread_tile_range(const Geometry<float>& g, const int* __restrict__ tstart, int b, int* p0,
                                         int* p1, TileOrigin* o, size_t* goff) {
  if (TX == 8) {
    *p0 = tstart[b];
    *p1 = tstart[b + 1];
    if (*p0 >= *p1) return false;
    *o = tile_origin(g, local_tile(g, b, goff));
    return true;
  }
  const int ntx = g.ntile[0], nsx = (ntx + 1) >> 1;
  const int sper = nsx * g.ntile[1] * g.ntile[2];
  const int sys = b / sper;
  const int sl = b - sys * sper;
  const int sx = sl % nsx, rest = sl / nsx;
  const int t0 = sys * g.tiles_per + 2 * sx + ntx * rest;
  const int t1 = t0 + ((2 * sx + 1 < ntx) ? 2 : 1);
  *p0 = tstart[t0];
  *p1 = tstart[t1];
  if (*p0 >= *p1) return false;
  *goff = (size_t)sys * (size_t)g.grid_stride;
  o->ox0 = 2 * sx * g.tile[0];
  o->oy0 = (rest % g.ntile[1]) * g.tile[1];
  o->oz0 = (rest / g.ntile[1]) * g.tile[2];
  return true;
}

// Global reduction of four consecutive floats (16-byte aligned address).
__device__ inline void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Pairs of x points per particle in the row-stationary spread: the window's M_G points placed on
// even-aligned pairs of the row (one zero in front when the window starts on an odd point, one
// behind when it starts on an even one), M_G / 2 + 1 pairs.
__host__ __device__ constexpr int row_pairs(int MGT) { return MGT / 2 + 1; }

// Per-particle profile tables staged in shared memory (row-stationary spread).
struct RowTables {
  float4* xp;   // [chunk][pairs][2] {g, g', d^2 g, (d^2 g)'}, {d g_D, (d g_D)', g_D, g_D'} along x, ' = next point
  float4* yt;   // [chunk][MGT] {g, d, g_D, 0} along y
  float4* zt;   // [chunk][MGT] {g, d, g_D, 0} along z
  float4* pf;   // [chunk] force
  float4* pt;   // [chunk] torque
  int4* po;     // [chunk] window start inside the extended region
};

template <int MGT>
__device__ inline RowTables row_tables(float4* sm) {
  RowTables t;
  t.xp = sm;
  t.yt = t.xp + kRowsChunk * 2 * row_pairs(MGT);
  t.zt = t.yt + kRowsChunk * MGT;
  t.pf = t.zt + kRowsChunk * MGT;
  t.pt = t.pf + kRowsChunk;
  t.po = reinterpret_cast<int4*>(t.pt + kRowsChunk);
  return t;
}

__host__ __device__ constexpr size_t row_tables_bytes(int MGT) {
  return sizeof(float4) * ((size_t)kRowsChunk * (2 * row_pairs(MGT) + 2 * MGT) + 2 * kRowsChunk) +
         sizeof(int4) * kRowsChunk;
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
