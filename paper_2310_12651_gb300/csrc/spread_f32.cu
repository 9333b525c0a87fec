// FP32 spread J~^dagger + N~^dagger on tiles (Section 3.1, Section 3.4):
//   f(x_g) += F Delta~(x_g - Y; Sigma) - (1/2) T x grad Delta(x_g - Y; Sigma_D)
// with Delta~ = Delta(.; Sigma) (A + B |d|^2), A = 1 - 3 dd/(2 Sigma^2),
// B = dd/(2 Sigma^4), over each particle's M_G^3 window.
//
// spread_rows_kernel (default, M_G <= 16): every thread owns one (y, z) row of
// the tile's extended region and keeps its EX x 3 sums in registers (for
// M_G <= 14 a CTA takes two x-adjacent binning tiles, 16-point rows: a third
// less halo per grid point). All
// threads walk the tile's particles together; each particle's x/y/z profiles
// are staged once in shared memory and read as broadcasts. No two threads add
// to the same point, so there are no atomics and the order of the sum over
// particles is fixed. At the end each thread adds its row to the grid with
// 16-byte global reductions (the halo flush).
//
// spread_tile_kernel (any M_G): warp per particle, lanes on window rows, shared
// memory atomics into the extended region (bank-conflict-free layout), then
// the same flush from shared memory with coalesced reductions.
#include "grid_common.cuh"

namespace fcm {

// The row update works on pairs of x points with packed FP32 instructions (__ffma2_rn: two
// correctly rounded FMAs per instruction, the same operations in the same order as one FMA per
// point). Forces only: the row's weight at each point, w = GQ g + GB d^2 g, is formed once and scaled
// by the three force components; with torques the terms are kept per component.
template <int OXP, int NP, int EXT2, bool TORQUE, bool SAMEW>
__device__ __forceinline__ void add_row2(const float4* __restrict__ xp, float2 (&sx)[EXT2], float2 (&sy)[EXT2],
                                         float2 (&sz)[EXT2], float ax, float ay, float az, float bx, float by,
                                         float bz, float cx, float cy, float cz, float ky, float kz, float gq,
                                         float gb, float4 f) {
  static_assert(OXP + NP <= EXT2, "pair window beyond the row");
  const float2 AX = make_float2(ax, ax), AY = make_float2(ay, ay), AZ = make_float2(az, az);
  const float2 BX = make_float2(bx, bx), BY = make_float2(by, by), BZ = make_float2(bz, bz);
#pragma unroll
  for (int jp = 0; jp < NP; ++jp) {
    const float4 p0 = xp[2 * jp];
    const float2 g2 = make_float2(p0.x, p0.y), q2 = make_float2(p0.z, p0.w);
    if (!TORQUE) {
      const float2 w = __ffma2_rn(make_float2(gb, gb), q2, __fmul2_rn(make_float2(gq, gq), g2));
      sx[OXP + jp] = __ffma2_rn(make_float2(f.x, f.x), w, sx[OXP + jp]);
      sy[OXP + jp] = __ffma2_rn(make_float2(f.y, f.y), w, sy[OXP + jp]);
      sz[OXP + jp] = __ffma2_rn(make_float2(f.z, f.z), w, sz[OXP + jp]);
      continue;
    }
    const float4 p1 = xp[2 * jp + 1];
    const float2 k2 = make_float2(p1.x, p1.y);
    float2 vx = __ffma2_rn(BX, q2, __ffma2_rn(AX, g2, sx[OXP + jp]));
    float2 vy = __ffma2_rn(BY, q2, __ffma2_rn(AY, g2, sy[OXP + jp]));
    float2 vz = __ffma2_rn(BZ, q2, __ffma2_rn(AZ, g2, sz[OXP + jp]));
    vy = __ffma2_rn(make_float2(ky, ky), k2, vy);
    vz = __ffma2_rn(make_float2(kz, kz), k2, vz);
    if (!SAMEW) {
      const float2 d2 = make_float2(p1.z, p1.w);
      vx = __ffma2_rn(make_float2(cx, cx), d2, vx);
      vy = __ffma2_rn(make_float2(cy, cy), d2, vy);
      vz = __ffma2_rn(make_float2(cz, cz), d2, vz);
    }
    sx[OXP + jp] = vx;
    sy[OXP + jp] = vy;
    sz[OXP + jp] = vz;
  }
}

// Adds a row of EX points (held as pairs) to the grid row starting at x = o.ox0.
template <int EXT2>
__device__ inline void flush_row2(const Geometry<float>& g, const TileOrigin& o, int EX, float* __restrict__ row,
                                  const float2 (&s)[EXT2]) {
  const bool vec = (o.ox0 + EX <= g.M[0]) && ((g.M[0] & 3) == 0);
  if (vec) {
    float* p = row + o.ox0;
#pragma unroll
    for (int k = 0; k + 1 < EXT2; k += 2) {   // points 2k .. 2k + 3
      if (2 * k + 3 < EX) {
        if (s[k].x != 0.f || s[k].y != 0.f || s[k + 1].x != 0.f || s[k + 1].y != 0.f)
          red_add_v4(p + 2 * k, s[k].x, s[k].y, s[k + 1].x, s[k + 1].y);
      } else {
        const float v[4] = {s[k].x, s[k].y, s[k + 1].x, s[k + 1].y};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (2 * k + e < EX && v[e] != 0.f) atomicAdd(p + 2 * k + e, v[e]);
      }
    }
    if (EXT2 & 1) {
      const int k = EXT2 - 1;
      if (2 * k < EX && s[k].x != 0.f) atomicAdd(p + 2 * k, s[k].x);
      if (2 * k + 1 < EX && s[k].y != 0.f) atomicAdd(p + 2 * k + 1, s[k].y);
    }
  } else {
#pragma unroll
    for (int k = 0; k < EXT2; ++k) {
      if (2 * k < EX && s[k].x != 0.f) atomicAdd(row + wrap_index(o.ox0 + 2 * k, g.M[0]), s[k].x);
      if (2 * k + 1 < EX && s[k].y != 0.f) atomicAdd(row + wrap_index(o.ox0 + 2 * k + 1, g.M[0]), s[k].y);
    }
  }
}

// Threads of the rows kernel: one per extended (y, z) row, at most (7 + M_G)^2
// with an 8-point tile (M_G = 16 uses a 4-point tile in y and z).
constexpr int rows_threads(int MGT) {
  return MGT <= 14 ? (((7 + MGT) * (7 + MGT) + 31) / 32) * 32 : kRowsMaxThreads;
}

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW, int TX>
__global__ void __launch_bounds__(rows_threads(MGT), 1) spread_rows_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                                        const float4* __restrict__ pos,
                                                                        const float4* __restrict__ Fv,
                                                                        const float4* __restrict__ Tv,
                                                                        const int* __restrict__ tstart,
                                                                        float* __restrict__ grid) {
  constexpr int EXT = TX + MGT - 1;
  constexpr int NP = row_pairs(MGT);
  constexpr int EXT2 = (TX + 2 * NP - 1) / 2;   // pairs of the row: window pairs start at pair (window start) / 2
  static_assert(2 * EXT2 >= EXT, "row pairs");
  extern __shared__ float4 sm4[];
  int p0, p1;
  size_t goff;
  TileOrigin o;
  if (!spread_tile_range<TX>(g, tstart, blockIdx.x, &p0, &p1, &o, &goff)) return;
  grid += goff;
  const int MG = GUARD ? g.MG : MGT;
  const int EY = g.tile[1] + MG - 1, EZ = g.tile[2] + MG - 1;
  const int R = EY * EZ;
  const int row = threadIdx.x;
  const bool has_row = row < R;
  const int ez = has_row ? row / EY : 0;
  const int ey = has_row ? row - ez * EY : 0;
  float2 sx[EXT2], sy[EXT2], sz[EXT2];
#pragma unroll
  for (int k = 0; k < EXT2; ++k) {
    sx[k] = make_float2(0.f, 0.f);
    sy[k] = make_float2(0.f, 0.f);
    sz[k] = make_float2(0.f, 0.f);
  }
  const RowTables tb = row_tables<MGT>(sm4);

  for (int base = p0; base < p1; base += kRowsChunk) {
    const int np = min(kRowsChunk, p1 - base);
    __syncthreads();
    // y and z profiles {g, d, g_D, 0}
    for (int k = threadIdx.x; k < np * 2 * MGT; k += blockDim.x) {
      const int q = k / (2 * MGT);
      const int rem = k - q * 2 * MGT;
      const int d = 1 + rem / MGT;
      const int j = rem - (d - 1) * MGT;
      const float4 y = pos[base + q];
      const float yd = d == 1 ? y.y : y.z;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < MG) {
        const float dd = (float)(window_start_d(g, d, yd) + j) * sel3(g.h, d) - yd;
        const float gs = expf(-dd * dd * kc.inv2S2);
        const float gd = SAMEW ? gs : expf(-dd * dd * kc.inv2SD2);
        v = make_float4(gs, dd, gd, 0.f);
      }
      (d == 1 ? tb.yt : tb.zt)[q * MGT + j] = v;
    }
    // x profiles on even-aligned pairs: slot 2 jp + e holds window point j = 2 jp + e - (start & 1)
    for (int k = threadIdx.x; k < np * 2 * NP; k += blockDim.x) {
      const int q = k / (2 * NP);
      const int slot = k - q * 2 * NP;
      const float4 y = pos[base + q];
      const int i0 = window_start_d(g, 0, y.x);
      const int ox = TX == 8 ? min(max(wrap_once(i0, g.M[0]) - o.ox0, 0), g.tile[0] - 1)
                             : min(max(wrap_once(i0, g.M[0]) - o.ox0, 0), TX - 1);
      const int j = slot - (ox & 1);
      float gs = 0.f, q2 = 0.f, dg = 0.f, gd = 0.f;
      if (j >= 0 && j < MG) {
        const float dd = (float)(i0 + j) * g.h[0] - y.x;
        gs = expf(-dd * dd * kc.inv2S2);
        gd = SAMEW ? gs : expf(-dd * dd * kc.inv2SD2);
        q2 = dd * dd * gs;
        dg = dd * gd;
      }
      float* e = reinterpret_cast<float*>(tb.xp + (size_t)(q * NP + (slot >> 1)) * 2) + (slot & 1);
      e[0] = gs;
      e[2] = q2;
      e[4] = dg;
      e[6] = gd;
    }
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      int4 off = window_offset(g, o, window_starts(g, pos[base + q]));
      if (TX != 8) {   // window start inside the (wider) row: recomputed without the 8-point clamp
        const int3 i0 = window_starts(g, pos[base + q]);
        off.x = min(max(wrap_once(i0.x, g.M[0]) - o.ox0, 0), TX - 1);
      }
      tb.po[q] = off;
      tb.pf[q] = Fv[base + q];
      tb.pt[q] = TORQUE ? Tv[base + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (!has_row) continue;
    for (int q = 0; q < np; ++q) {
      const int4 off = tb.po[q];
      const int jy = ey - off.y, jz = ez - off.z;
      if ((unsigned)jy >= (unsigned)MG || (unsigned)jz >= (unsigned)MG) continue;
      const float4 yv = tb.yt[q * MGT + jy];
      const float4 zv = tb.zt[q * MGT + jz];
      const float4 f = tb.pf[q];
      const float G = kc.nrm * yv.x * zv.x;
      const float GQ = G * fmaf(kc.B, fmaf(yv.y, yv.y, zv.y * zv.y), kc.A);
      const float GB = G * kc.B;
      float ax = f.x * GQ, ay = f.y * GQ, az = f.z * GQ;
      const float bx = f.x * GB, by = f.y * GB, bz = f.z * GB;
      float cx = 0.f, cy = 0.f, cz = 0.f, ky = 0.f, kz = 0.f;
      if (TORQUE) {
        const float4 tq = tb.pt[q];
        const float H = kc.tq * yv.z * zv.z;
        const float dy = yv.y, dz = zv.y;
        cx = H * (tq.y * dz - tq.z * dy);
        cy = -H * tq.x * dz;
        cz = H * tq.x * dy;
        ky = H * tq.z;
        kz = -H * tq.y;
        if (SAMEW) { ax += cx; ay += cy; az += cz; }
      }
      const float4* xp = tb.xp + (size_t)q * 2 * NP;
#define FCM_ROW_CASE(OXP)                                                                                 \
  case OXP:                                                                                               \
    add_row2<OXP, NP, EXT2, TORQUE, SAMEW>(xp, sx, sy, sz, ax, ay, az, bx, by, bz, cx, cy, cz, ky, kz, GQ, GB, \
                                           f);                                                            \
    break;
      switch (off.x >> 1) {
        FCM_ROW_CASE(0) FCM_ROW_CASE(1) FCM_ROW_CASE(2) FCM_ROW_CASE(3)
        default:
          if (TX > 8) {
            switch (off.x >> 1) {
              FCM_ROW_CASE(4 % (TX / 2)) FCM_ROW_CASE(5 % (TX / 2)) FCM_ROW_CASE(6 % (TX / 2))
              FCM_ROW_CASE(7 % (TX / 2))
              default: break;
            }
          }
          break;
      }
#undef FCM_ROW_CASE
    }
  }
  if (has_row) {
    const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
    const int gy = wrap_index(o.oy0 + ey, g.M[1]);
    const int gz = wrap_index(o.oz0 + ez, g.M[2]);
    float* r0 = grid + ((size_t)gz * g.M[1] + gy) * g.M[0];
    const int EX = TX + MG - 1;
    flush_row2<EXT2>(g, o, EX, r0, sx);
    flush_row2<EXT2>(g, o, EX, r0 + Mtot, sy);
    flush_row2<EXT2>(g, o, EX, r0 + 2 * Mtot, sz);
  }
}

// ---------------------------------------------------------------- pencil kernel
//
// spread_pencil_kernel (default for M_G <= 16 with 8-point tiles in x): one CTA walks a whole
// x-pencil of binning tiles (all tiles with the same (y, z) tile index of one system; they are
// contiguous in the tile-sorted order). Every thread owns one (y, z) row of the pencil's extended
// (y, z) region and keeps a register row of EXT2 point pairs per component, anchored at the current
// half tile's x origin x0 = 4 s. The binning orders each tile's particles by the half of the tile
// their window starts in, so the particles of half tile s, taken in order, have window starts in
// [x0, x0 + 4): once the walk passes to half tile s + 1 the points x0 .. x0 + 3 are complete for this
// pencil, they are added to the grid (two pairs per component) and the register row shifts by two
// pairs. Walking half tiles keeps the row at M_G / 2 + 2 pairs (a window starts at one of two pairs)
// instead of M_G / 2 + 4. The x halo is thus carried along the pencil in registers instead of being
// added to the grid, and only the (y, z) halo is flushed with global reductions. A particle's row update is predicated (coefficients
// zero outside its window): a warp skips a particle only when none of its rows is in the window, so
// no lane diverges.
//
// The row update regroups the kernel's terms by their x profile. With G = g(dy) g(dz), the modified
// kernel's polynomial P = A + B (dy^2 + dz^2), F' = nrm F and U' = tq T, a particle adds to its row
//   f_c(x) += G alpha_c g(x) + G w_c(x),
//   alpha = (F'x P + U'y dz - U'z dy, F'y P - U'x dz, F'z P + U'x dy),
//   w = (B F'x d^2 g, B F'y d^2 g + U'z d g, B F'z d^2 g - U'y d g)      (d = x - Y_x, g = g(d))
// for Sigma_D = Sigma: the x profiles g and w_c are staged once per particle, the row coefficients
// G alpha_c and G once per particle-row, and a point takes six FMAs (three packed pairs per two
// points). Forces only: f_c(x) += G F'_c (P g + B d^2 g). Sigma_D != Sigma keeps the torque terms on
// their own profiles d g_D and g_D with the row factor H = tq g_D(dy) g_D(dz).

// Particles staged per pass of the pencil kernel. The profile tables are double-buffered: while
// the row updates of pass c read one table set, the same threads build the tables of pass c + 1 in
// the other (a warp whose rows finish early starts on them at once), and the raw rows (position,
// force, torque) of pass c + 2 arrive by asynchronous copies. One CTA barrier per pass. Passes of
// 128 particles where both table sets fit shared memory (one width and M_G <= 14), else 64.
enum { kPencilForces = 0, kPencilSameWidth = 1, kPencilTwoWidths = 2 };

__host__ __device__ constexpr int pencil_chunk(int MGT, int MODE) {
  return (MODE != kPencilTwoWidths && MGT <= 14) ? 128 : 64;
}

// Register pairs of a pencil row: the walk steps half a tile (4 points) at a time, so window pairs start at
// pair ox / 2 with ox in [0, 4) (the binning puts each tile's particles with ox < 4 first).
__host__ __device__ constexpr int pencil_pairs(int MGT) { return row_pairs(MGT) + 1; }

// Per-particle tables of the pencil kernel (one staged chunk).
struct PencilTables {
  float4* xa;   // [chunk][NP] {g, g', q, q'} (q = d^2 g; same width: q -> w_x = B F'x d^2 g), ' = next point
  float4* xb;   // [chunk][NP] same width: {w_y, w_y', w_z, w_z'}
  float4* yt;   // [chunk][MGT] {g, d, A + B d^2, g_D} along y
  float4* zt;   // [chunk][MGT] {g, d, B d^2, g_D} along z
  float4* pf;   // [chunk] F' = nrm F (two widths: F)
  float4* pt;   // [chunk] U' = tq T (two widths: T)
  int4* po;     // [chunk] (x offset in the tile, y and z window start in the region, tile step)
  float* xk;    // two widths: [chunk][4 NK] d g_D along x, two pairs per float4
  float* xd;    // two widths: [chunk][2 NP] g_D along x
};

// float4 of one table set: the float4 tables, then (two widths) the float tables rounded up.
__host__ __device__ constexpr int pencil_set_f4(int MGT, int MODE) {
  return pencil_chunk(MGT, MODE) * (2 * row_pairs(MGT) + 2 * MGT + 3) +
         (MODE == kPencilTwoWidths
              ? (pencil_chunk(MGT, MODE) * (4 * ((row_pairs(MGT) + 1) / 2) + 2 * row_pairs(MGT)) + 3) / 4
              : 0);
}

// Table set t (0 or 1); the raw rows [2][3][chunk] follow both sets.
template <int MGT, int MODE>
__device__ inline PencilTables pencil_tables(float4* sm, int t) {
  constexpr int NP = row_pairs(MGT), NK = (NP + 1) / 2;
  constexpr int C = pencil_chunk(MGT, MODE);
  PencilTables s;
  s.xa = sm + (size_t)t * pencil_set_f4(MGT, MODE);
  s.xb = s.xa + C * NP;
  s.yt = s.xb + C * NP;
  s.zt = s.yt + C * MGT;
  s.pf = s.zt + C * MGT;
  s.pt = s.pf + C;
  s.po = reinterpret_cast<int4*>(s.pt + C);
  s.xk = reinterpret_cast<float*>(s.po + C);
  s.xd = s.xk + C * 4 * NK;
  return s;
}

template <int MGT, int MODE>
__device__ inline float4* pencil_raw(float4* sm, int buf) {
  return sm + 2 * (size_t)pencil_set_f4(MGT, MODE) + (size_t)buf * 3 * pencil_chunk(MGT, MODE);
}

__host__ __device__ constexpr size_t pencil_tables_bytes(int MGT, int MODE) {
  return sizeof(float4) * (2 * (size_t)pencil_set_f4(MGT, MODE) + 6 * (size_t)pencil_chunk(MGT, MODE));
}

// Asynchronous 16-byte copy global -> shared (the raw rows of a later pass).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// Raw rows of particles [base, base + np) into raw buffer r ([3][C]).
template <bool TORQUE, int C>
__device__ __forceinline__ void pencil_fetch(float4* r, int base, int np, const float4* __restrict__ pos,
                                             const float4* __restrict__ Fv, const float4* __restrict__ Tv) {
  for (int k = threadIdx.x; k < (TORQUE ? 3 : 2) * np; k += blockDim.x) {
    const int a = k >= 2 * np ? 2 : (k >= np ? 1 : 0), q = k - a * np;
    const float4* src = (a == 0 ? pos : (a == 1 ? Fv : Tv)) + base + q;
    cp_async16(r + a * C + q, src);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

template <int OXP, int NP, int EXT2, int MODE>
__device__ __forceinline__ void pencil_row(const float4* __restrict__ xa, const float4* __restrict__ xb,
                                           const float4* __restrict__ xk, const float2* __restrict__ xd,
                                           float2 (&sx)[EXT2], float2 (&sy)[EXT2], float2 (&sz)[EXT2],
                                           float c0, float c1, float c2, float c3, float c4, float c5,
                                           float c6, float c7, float c8, float c9, float c10) {
  static_assert(OXP + NP <= EXT2, "pair window beyond the row");
  if (MODE == kPencilSameWidth) {   // c0 = G, c1..c3 = G alpha
    const float2 G2 = dup2(c0), AX = dup2(c1), AY = dup2(c2), AZ = dup2(c3);
#pragma unroll
    for (int jp = 0; jp < NP; ++jp) {
      const float4 p0 = xa[jp], p1 = xb[jp];
      const float2 g2 = make_float2(p0.x, p0.y);
      sx[OXP + jp] = __ffma2_rn(G2, make_float2(p0.z, p0.w), __ffma2_rn(AX, g2, sx[OXP + jp]));
      sy[OXP + jp] = __ffma2_rn(G2, make_float2(p1.x, p1.y), __ffma2_rn(AY, g2, sy[OXP + jp]));
      sz[OXP + jp] = __ffma2_rn(G2, make_float2(p1.z, p1.w), __ffma2_rn(AZ, g2, sz[OXP + jp]));
    }
  } else if (MODE == kPencilForces) {   // c0 = P, c1 = B, c2..c4 = G F'
    const float2 P2 = dup2(c0), B2 = dup2(c1), FX = dup2(c2), FY = dup2(c3), FZ = dup2(c4);
#pragma unroll
    for (int jp = 0; jp < NP; ++jp) {
      const float4 p0 = xa[jp];
      const float2 w = __ffma2_rn(B2, make_float2(p0.z, p0.w), __fmul2_rn(P2, make_float2(p0.x, p0.y)));
      sx[OXP + jp] = __ffma2_rn(FX, w, sx[OXP + jp]);
      sy[OXP + jp] = __ffma2_rn(FY, w, sy[OXP + jp]);
      sz[OXP + jp] = __ffma2_rn(FZ, w, sz[OXP + jp]);
    }
  } else {   // two widths: c0..c2 = a, c3..c5 = b, c6..c8 = c, c9 = ky, c10 = kz
    const float2 AX = dup2(c0), AY = dup2(c1), AZ = dup2(c2), BX = dup2(c3), BY = dup2(c4), BZ = dup2(c5);
    const float2 CX = dup2(c6), CY = dup2(c7), CZ = dup2(c8), KY = dup2(c9), KZ = dup2(c10);
    float4 k4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int jp = 0; jp < NP; ++jp) {
      const float4 p0 = xa[jp];
      const float2 g2 = make_float2(p0.x, p0.y), q2 = make_float2(p0.z, p0.w);
      if ((jp & 1) == 0) k4 = xk[jp >> 1];
      const float2 k2 = (jp & 1) ? make_float2(k4.z, k4.w) : make_float2(k4.x, k4.y);
      const float2 d2 = xd[jp];
      float2 vx = __ffma2_rn(BX, q2, __ffma2_rn(AX, g2, sx[OXP + jp]));
      float2 vy = __ffma2_rn(BY, q2, __ffma2_rn(AY, g2, sy[OXP + jp]));
      float2 vz = __ffma2_rn(BZ, q2, __ffma2_rn(AZ, g2, sz[OXP + jp]));
      vy = __ffma2_rn(KY, k2, vy);
      vz = __ffma2_rn(KZ, k2, vz);
      sx[OXP + jp] = __ffma2_rn(CX, d2, vx);
      sy[OXP + jp] = __ffma2_rn(CY, d2, vy);
      sz[OXP + jp] = __ffma2_rn(CZ, d2, vz);
    }
  }
}

// Adds pairs [k0, k1) of a register row to grid points x0 + 2k, x0 + 2k + 1 (wrapped into [0, M_x)):
// 16-byte reductions where four points lie inside the row and the row holds whole float4s, scalar
// atomics elsewhere; zeros are skipped.
template <int EXT2>
__device__ __forceinline__ void pencil_flush(int x0, int Mx, bool vec_rows, float* __restrict__ row,
                                             const float2 (&s)[EXT2], int k0, int k1) {
#pragma unroll
  for (int k = 0; k < EXT2; k += 2) {
    if (k < k0 || k >= k1) continue;
    const int x = x0 + 2 * k;
    const bool two = (k + 1 < EXT2) && (k + 1 < k1);
    const float v0 = s[k].x, v1 = s[k].y;
    const float v2 = two ? s[k + 1].x : 0.f, v3 = two ? s[k + 1].y : 0.f;
    if (v0 == 0.f && v1 == 0.f && v2 == 0.f && v3 == 0.f) continue;
    if (two && vec_rows && x + 3 < Mx) {
      red_add_v4(row + x, v0, v1, v2, v3);
    } else {
      const float v[4] = {v0, v1, v2, v3};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (v[e] != 0.f) atomicAdd(row + wrap_index(x + e, Mx), v[e]);
    }
  }
}

template <int EXT2>
__device__ __forceinline__ void pencil_shift(float2 (&s)[EXT2]) {
#pragma unroll
  for (int k = 0; k < EXT2; ++k) s[k] = (k + 2 < EXT2) ? s[k + 2] : make_float2(0.f, 0.f);
}

template <int MGT, bool GUARD, int MODE>
__global__ void __launch_bounds__(rows_threads(MGT), 1) spread_pencil_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                                          const float4* __restrict__ pos,
                                                                          const float4* __restrict__ Fv,
                                                                          const float4* __restrict__ Tv,
                                                                          const int* __restrict__ tstart,
                                                                          float* __restrict__ grid, int segl) {
  constexpr int NP = row_pairs(MGT);
  constexpr int NK = (NP + 1) / 2;
  constexpr int EXT2 = pencil_pairs(MGT);
  constexpr bool TORQUE = MODE != kPencilForces;
  extern __shared__ float4 sm4[];
  const int ntx = g.ntile[0], nty = g.ntile[1];
  const int per = nty * g.ntile[2];
  const int nseg = (ntx + segl - 1) / segl;              // segments of segl tiles per pencil
  const int sys = blockIdx.x / (per * nseg);
  const int rem = blockIdx.x - sys * per * nseg;
  const int pc = rem / nseg;
  const int s0 = (rem - pc * nseg) * segl, s1 = min(ntx, s0 + segl);   // this CTA's tiles of the pencil
  const int t0 = sys * g.tiles_per + ntx * pc;          // tile (0, ty, tz) of the pencil
  const int p_begin = tstart[t0 + s0], p_end = tstart[t0 + s1];
  if (p_begin >= p_end) return;
  if (g.nsys > 1) grid += (size_t)sys * (size_t)g.grid_stride;
  const int oy0 = (pc % nty) * g.tile[1], oz0 = (pc / nty) * g.tile[2];
  const int MG = GUARD ? g.MG : MGT;
  const int EY = g.tile[1] + MG - 1, EZ = g.tile[2] + MG - 1;
  const int row = threadIdx.x;
  const bool has_row = row < EY * EZ;
  const int ez = has_row ? row / EY : 0;
  const int ey = has_row ? row - ez * EY : 0;
  float2 sx[EXT2], sy[EXT2], sz[EXT2];
#pragma unroll
  for (int k = 0; k < EXT2; ++k) {
    sx[k] = make_float2(0.f, 0.f);
    sy[k] = make_float2(0.f, 0.f);
    sz[k] = make_float2(0.f, 0.f);
  }
  int cur = 2 * s0;   // half-tile step whose x origin (4 cur) anchors the register row
  constexpr int C = pencil_chunk(MGT, MODE);
  // profile tables of one pass (particles [base, base + np)) from its raw rows
  auto build = [&](const PencilTables& tb, const float4* rpos, int np) {
    const float4* rF = rpos + C;
    const float4* rT = rF + C;
    // y and z profiles {g, d, A + B d^2 (y) or B d^2 (z), g_D}
    for (int k = threadIdx.x; k < np * 2 * MGT; k += blockDim.x) {
      const int q = k / (2 * MGT);
      const int rem = k - q * 2 * MGT;
      const int d = 1 + rem / MGT;
      const int j = rem - (d - 1) * MGT;
      const float4 y = rpos[q];
      const float yd = d == 1 ? y.y : y.z;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < MG) {
        const float dd = (float)(window_start_d(g, d, yd) + j) * sel3(g.h, d) - yd;
        const float gs = expf(-dd * dd * kc.inv2S2);
        const float gd = MODE == kPencilTwoWidths ? expf(-dd * dd * kc.inv2SD2) : gs;
        const float bq = kc.B * dd * dd;
        v = make_float4(gs, dd, d == 1 ? kc.A + bq : bq, gd);
      }
      (d == 1 ? tb.yt : tb.zt)[q * MGT + j] = v;
    }
    // x profiles on even-aligned pairs: slot 2 jp + e holds window point j = 2 jp + e - (start & 1)
    for (int k = threadIdx.x; k < np * 2 * NP; k += blockDim.x) {
      const int q = k / (2 * NP);
      const int slot = k - q * 2 * NP;
      const float4 y = rpos[q];
      const int i0 = window_start_d(g, 0, y.x);
      const int j = slot - (wrap_once(i0, g.M[0]) & 1);
      float gs = 0.f, q2 = 0.f, dg = 0.f, gd = 0.f;
      if (j >= 0 && j < MG) {
        const float dd = (float)(i0 + j) * g.h[0] - y.x;
        gs = expf(-dd * dd * kc.inv2S2);
        gd = MODE == kPencilTwoWidths ? expf(-dd * dd * kc.inv2SD2) : gs;
        q2 = dd * dd * gs;
        dg = dd * gd;
      }
      float* ea = reinterpret_cast<float*>(tb.xa + (size_t)q * NP + (slot >> 1)) + (slot & 1);
      ea[0] = gs;
      if (MODE == kPencilSameWidth) {
        const float4 f = rF[q], t = rT[q];
        const float bn = kc.B * kc.nrm;
        float* eb = reinterpret_cast<float*>(tb.xb + (size_t)q * NP + (slot >> 1)) + (slot & 1);
        ea[2] = bn * f.x * q2;
        eb[0] = fmaf(bn * f.y, q2, kc.tq * t.z * dg);
        eb[2] = fmaf(bn * f.z, q2, -kc.tq * t.y * dg);
      } else {
        ea[2] = q2;
      }
      if (MODE == kPencilTwoWidths) {
        tb.xk[(size_t)q * 4 * NK + slot] = dg;
        tb.xd[(size_t)q * 2 * NP + slot] = gd;
      }
    }
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      const float4 y = rpos[q];
      const int3 i0 = window_starts(g, y);
      const int wx = wrap_once(i0.x, g.M[0]);
      const int step = min(max(wx >> 3, 0), ntx - 1);
      const int ox = min(max(wx - 8 * step, 0), 7);   // the binning's half of the tile: ox >= 4
      int4 off;
      off.x = ox & 3;
      off.y = min(max(wrap_once(i0.y, g.M[1]) - oy0, 0), g.tile[1] - 1);
      off.z = min(max(wrap_once(i0.z, g.M[2]) - oz0, 0), g.tile[2] - 1);
      off.w = 2 * step + (ox >> 2);
      tb.po[q] = off;
      const float4 f = rF[q];
      const float4 t = TORQUE ? rT[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (MODE == kPencilTwoWidths) {
        tb.pf[q] = f;
        tb.pt[q] = t;
      } else {
        tb.pf[q] = make_float4(kc.nrm * f.x, kc.nrm * f.y, kc.nrm * f.z, 0.f);
        tb.pt[q] = make_float4(kc.tq * t.x, kc.tq * t.y, kc.tq * t.z, 0.f);
      }
    }
  };
  const int npass = (p_end - p_begin + C - 1) / C;
  pencil_fetch<TORQUE, C>(pencil_raw<MGT, MODE>(sm4, 0), p_begin, min(C, p_end - p_begin), pos, Fv, Tv);
  if (npass > 1) pencil_fetch<TORQUE, C>(pencil_raw<MGT, MODE>(sm4, 1), p_begin + C, min(C, p_end - p_begin - C), pos, Fv, Tv);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  build(pencil_tables<MGT, MODE>(sm4, 0), pencil_raw<MGT, MODE>(sm4, 0), min(C, p_end - p_begin));
  __syncthreads();
  for (int pass = 0; pass < npass; ++pass) {
    const int base = p_begin + pass * C;
    const int np = min(C, p_end - base);
    // raw rows of pass + 2 into the buffer that pass's tables were built from
    if (pass + 2 < npass)
      pencil_fetch<TORQUE, C>(pencil_raw<MGT, MODE>(sm4, pass & 1), base + 2 * C, min(C, p_end - base - 2 * C), pos, Fv, Tv);
    const PencilTables tb = pencil_tables<MGT, MODE>(sm4, pass & 1);
    for (int q = 0; q < np; ++q) {
      const int4 off = tb.po[q];
      // the walk reaches the particle's half tile: complete points of the passed half tiles go to the grid
      while (cur < off.w) {
        if (has_row) {
          const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
          float* r0 = grid + ((size_t)wrap_index(oz0 + ez, g.M[2]) * g.M[1] + wrap_index(oy0 + ey, g.M[1])) * g.M[0];
          const bool vec_rows = (g.M[0] & 3) == 0;
          pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0, sx, 0, 2);
          pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0 + Mtot, sy, 0, 2);
          pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0 + 2 * Mtot, sz, 0, 2);
        }
        pencil_shift<EXT2>(sx);
        pencil_shift<EXT2>(sy);
        pencil_shift<EXT2>(sz);
        ++cur;
      }
      const int jy = ey - off.y, jz = ez - off.z;
      const bool in = has_row && (unsigned)jy < (unsigned)MG && (unsigned)jz < (unsigned)MG;
      if (!__any_sync(kFullMask32, in)) continue;
      const float4 yv = tb.yt[q * MGT + (in ? jy : 0)];
      const float4 zv = tb.zt[q * MGT + (in ? jz : 0)];
      const float4 f = tb.pf[q];
      const float P = yv.z + zv.z;
      float c[11];
      if (MODE == kPencilSameWidth) {
        const float4 u = tb.pt[q];
        const float G = in ? yv.x * zv.x : 0.f;
        const float dy = yv.y, dz = zv.y;
        c[0] = G;
        c[1] = G * fmaf(f.x, P, fmaf(u.y, dz, -u.z * dy));
        c[2] = G * fmaf(f.y, P, -u.x * dz);
        c[3] = G * fmaf(f.z, P, u.x * dy);
        for (int k = 4; k < 11; ++k) c[k] = 0.f;
      } else if (MODE == kPencilForces) {
        const float G = in ? yv.x * zv.x : 0.f;
        c[0] = P;
        c[1] = kc.B;
        c[2] = G * f.x;
        c[3] = G * f.y;
        c[4] = G * f.z;
        for (int k = 5; k < 11; ++k) c[k] = 0.f;
      } else {
        const float4 tq = tb.pt[q];
        const float G = in ? kc.nrm * yv.x * zv.x : 0.f;
        const float GQ = G * P, GB = G * kc.B;
        const float H = in ? kc.tq * yv.w * zv.w : 0.f;
        const float dy = yv.y, dz = zv.y;
        c[0] = f.x * GQ; c[1] = f.y * GQ; c[2] = f.z * GQ;
        c[3] = f.x * GB; c[4] = f.y * GB; c[5] = f.z * GB;
        c[6] = H * (tq.y * dz - tq.z * dy);
        c[7] = -H * tq.x * dz;
        c[8] = H * tq.x * dy;
        c[9] = H * tq.z;
        c[10] = -H * tq.y;
      }
      const float4* xa = tb.xa + (size_t)q * NP;
      const float4* xb = tb.xb + (size_t)q * NP;
      const float4* xk = reinterpret_cast<const float4*>(tb.xk + (size_t)q * 4 * NK);
      const float2* xd = reinterpret_cast<const float2*>(tb.xd + (size_t)q * 2 * NP);
#define FCM_PENCIL_CASE(OXP)                                                                                    \
  case OXP:                                                                                                     \
    pencil_row<OXP, NP, EXT2, MODE>(xa, xb, xk, xd, sx, sy, sz, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], \
                                    c[8], c[9], c[10]);                                                         \
    break;
      switch (off.x >> 1) {
        FCM_PENCIL_CASE(0) FCM_PENCIL_CASE(1)
        default: break;
      }
#undef FCM_PENCIL_CASE
    }
    // tables of the next pass, into the set the previous pass used
    if (pass + 1 < npass)
      build(pencil_tables<MGT, MODE>(sm4, (pass + 1) & 1), pencil_raw<MGT, MODE>(sm4, (pass + 1) & 1), min(C, p_end - base - C));
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // the next tables and the raw rows of pass + 2 are in; this pass's tables are free
  }
  if (has_row) {   // the last tile reached: every pair of the register row, x from 8 cur on
    const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
    float* r0 = grid + ((size_t)wrap_index(oz0 + ez, g.M[2]) * g.M[1] + wrap_index(oy0 + ey, g.M[1])) * g.M[0];
    const bool vec_rows = (g.M[0] & 3) == 0;
    pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0, sx, 0, EXT2);
    pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0 + Mtot, sy, 0, EXT2);
    pencil_flush<EXT2>(4 * cur, g.M[0], vec_rows, r0 + 2 * Mtot, sz, 0, EXT2);
  }
}

// ---------------------------------------------------------------- atomic kernel

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW>
__global__ void __launch_bounds__(256) spread_tile_kernel(Geometry<float> g, KernelConsts<float> kc,
                                                          const float4* __restrict__ pos,
                                                          const float4* __restrict__ Fv,
                                                          const float4* __restrict__ Tv,
                                                          const int* __restrict__ tstart,
                                                          float* __restrict__ grid) {
  extern __shared__ float4 sm4[];
  float* acc = reinterpret_cast<float*>(sm4);
  const int t = blockIdx.x;
  const int p0 = tstart[t], p1 = tstart[t + 1];
  if (p0 >= p1) return;
  size_t goff;
  const TileOrigin o = tile_origin(g, local_tile(g, t, &goff));
  grid += goff;
  const int MG = GUARD ? g.MG : MGT;
  const ExtLayout l = ext_layout(g.tile, MG);
  for (int k = threadIdx.x; k < 3 * l.C; k += blockDim.x) acc[k] = 0.f;
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int p = p0 + warp; p < p1; p += nwarp) {
    const float4 y = pos[p];
    const float4 f = Fv[p];
    float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (TORQUE) tq = Tv[p];
    const int3 i0 = window_starts(g, y);
    const int4 off = window_offset(g, o, i0);
    // lane l < MG holds the l-th point of each axis
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
    int jy = lane, jz = 0;
    while (jy >= MG) { jy -= MG; ++jz; }
    for (int r0 = 0; r0 < MG * MG; r0 += 32) {
      const bool active = r0 + lane < MG * MG;
      const int sy = active ? jy : 0, sz = active ? jz : 0;
      const float dy = __shfl_sync(kFullMask32, dyl, sy);
      const float gy = __shfl_sync(kFullMask32, gyl, sy);
      const float dz = __shfl_sync(kFullMask32, dzl, sz);
      const float gz = __shfl_sync(kFullMask32, gzl, sz);
      const float gdy = SAMEW ? gy : __shfl_sync(kFullMask32, gdyl, sy);
      const float gdz = SAMEW ? gz : __shfl_sync(kFullMask32, gdzl, sz);
      if (active) {
        const float G = kc.nrm * gy * gz;
        const float GQ = G * fmaf(kc.B, fmaf(dy, dy, dz * dz), kc.A);
        const float GB = G * kc.B;
        float ax = f.x * GQ, ay = f.y * GQ, az = f.z * GQ;
        const float bx = f.x * GB, by = f.y * GB, bz = f.z * GB;
        float* rowp = acc + (off.z + jz) * l.Q + (off.y + jy) * l.P + off.x;
        float cx = 0.f, cy = 0.f, cz = 0.f, ky = 0.f, kz = 0.f;
        if (TORQUE) {
          const float H = kc.tq * gdy * gdz;
          cx = H * (tq.y * dz - tq.z * dy);
          cy = -H * tq.x * dz;
          cz = H * tq.x * dy;
          ky = H * tq.z;
          kz = -H * tq.y;
          if (SAMEW) { ax += cx; ay += cy; az += cz; }
        }
#pragma unroll
        for (int j = 0; j < MGT; ++j) {
          if (!GUARD || j < MG) {
            float vx = fmaf(bx, gx2[j], ax * gx[j]);
            float vy = fmaf(by, gx2[j], ay * gx[j]);
            float vz = fmaf(bz, gx2[j], az * gx[j]);
            if (TORQUE) {
              vy = fmaf(ky, gx1[j], vy);
              vz = fmaf(kz, gx1[j], vz);
              if (!SAMEW) { vx = fmaf(cx, gdx[j], vx); vy = fmaf(cy, gdx[j], vy); vz = fmaf(cz, gdx[j], vz); }
            }
            atomicAdd(rowp + j, vx);
            atomicAdd(rowp + l.C + j, vy);
            atomicAdd(rowp + 2 * l.C + j, vz);
          }
        }
      }
      jy += 32;
      while (jy >= MG) { jy -= MG; ++jz; }
    }
  }
  __syncthreads();
  flush_region(g, o, l, acc, grid);
}

// ---------------------------------------------------------------- sizing and launch

size_t tile_smem_bytes(const int tile[3], int MG) {
  const ExtLayout l = ext_layout(tile, MG);
  return sizeof(float) * (3 * (size_t)l.C + 1);   // + 1: the gather's (y, z) plane starts 8-byte aligned
}

int tile_smem_limit() { return 227 * 1024; }

static int rows_mgt(int MG) {
  switch (MG) {
    case 10: case 12: case 14: case 16: return MG;
    default: return MG <= 8 ? 8 : (MG <= 12 ? 12 : (MG <= 16 ? 16 : 0));
  }
}

bool spread_uses_rows(const int tile[3], int MG) {
  const int mgt = rows_mgt(MG);
  if (tile[0] != 8 || mgt == 0) return false;
  return (tile[1] + MG - 1) * (tile[2] + MG - 1) <= rows_threads(mgt);
}

static bool rows_selected(const Geometry<float>& g, int spread_kernel) {
  if (spread_kernel == 2) return false;
  return spread_uses_rows(g.tile, g.MG);
}

template <int MGT, bool GUARD, int MODE>
static void pencil_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b, float* grid,
                           cudaStream_t s) {
  const size_t smem = pencil_tables_bytes(MGT, MODE);
  const int threads = (((g.tile[1] + g.MG - 1) * (g.tile[2] + g.MG - 1) + 31) / 32) * 32;
  const int nsys = g.nsys > 1 ? g.nsys : 1;
  const int pencils = nsys * g.ntile[1] * g.ntile[2];
  // Long pencils are split into segments when there are too few pencils for four waves of one CTA per SM
  // (thin slabs, small single systems); a segment flushes its whole register row at its end.
  const int nseg = std::min(g.ntile[0], std::max(1, (4 * device_sm_count() + pencils - 1) / pencils));
  const int segl = (g.ntile[0] + nseg - 1) / nseg;
  const int blocks = pencils * ((g.ntile[0] + segl - 1) / segl);
  auto k = spread_pencil_kernel<MGT, GUARD, MODE>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, threads, smem, s>>>(g, kc, (const float4*)b.t_pos, (const float4*)b.t_F, (const float4*)b.t_T,
                                  b.tile_start, grid, segl);
}

size_t spread_smem_bytes(const int tile[3], int MG) {
  if (!spread_uses_rows(tile, MG)) return tile_smem_bytes(tile, MG);
  const size_t tab = std::max(row_tables_bytes(rows_mgt(MG)),
                              std::max(pencil_tables_bytes(rows_mgt(MG), kPencilSameWidth),
                                       pencil_tables_bytes(rows_mgt(MG), kPencilTwoWidths)));
  const size_t ext = tile_smem_bytes(tile, MG);
  return tab > ext ? tab : ext;  // any of the kernels may be selected for this tile
}

// Row-stationary spread over pairs of x-adjacent binning tiles (16-point rows).
constexpr bool kSpreadPairTiles = true;

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW>
static void rows_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b, float* grid,
                         cudaStream_t s) {
  const size_t smem = row_tables_bytes(MGT);
  const int threads = (((g.tile[1] + g.MG - 1) * (g.tile[2] + g.MG - 1) + 31) / 32) * 32;
  const float4* pos = (const float4*)b.t_pos;
  const float4* F = (const float4*)b.t_F;
  const float4* T = (const float4*)b.t_T;
  if (kSpreadPairTiles && MGT <= 14) {   // two binning tiles per CTA (registers: 3 (16 + M_G - 1) sums)
    const int nsys = g.nsys > 1 ? g.nsys : 1;
    const int blocks = nsys * ((g.ntile[0] + 1) / 2) * g.ntile[1] * g.ntile[2];
    auto k = spread_rows_kernel<MGT, GUARD, TORQUE, SAMEW, 16>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<blocks, threads, smem, s>>>(g, kc, pos, F, T, b.tile_start, grid);
  } else {
    auto k = spread_rows_kernel<MGT, GUARD, TORQUE, SAMEW, 8>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<b.ntiles, threads, smem, s>>>(g, kc, pos, F, T, b.tile_start, grid);
  }
}

template <int MGT, bool GUARD, bool TORQUE, bool SAMEW>
static void atomic_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b,
                           float* grid, cudaStream_t s) {
  const size_t smem = tile_smem_bytes(g.tile, g.MG);
  auto k = spread_tile_kernel<MGT, GUARD, TORQUE, SAMEW>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<b.ntiles, 256, smem, s>>>(g, kc, (const float4*)b.t_pos, (const float4*)b.t_F, (const float4*)b.t_T,
                                b.tile_start, grid);
}

void launch_spread_f32(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, int spread_kernel,
                       const BinBuffers& b, float* grid, cudaStream_t s, long long* launches) {
  if (spread_kernel == 4 && spread_tc_eligible(g.tile, g.MG, !torque || kc.same_width)) {
    launch_spread_tc(g, kc, torque, b, grid, s);
  } else if (spread_kernel == 3 && spread_mma_eligible(g.tile, g.MG)) {
    launch_spread_mma(g, kc, torque, b, grid, s);
  } else if (rows_selected(g, spread_kernel) && spread_kernel != 1) {
#define PENCIL_CALL(MGT, GUARD)                                                            \
  if (!torque) pencil_variant<MGT, GUARD, kPencilForces>(g, kc, b, grid, s);              \
  else if (kc.same_width) pencil_variant<MGT, GUARD, kPencilSameWidth>(g, kc, b, grid, s); \
  else pencil_variant<MGT, GUARD, kPencilTwoWidths>(g, kc, b, grid, s);
    FCM_DISPATCH_ROWS(g.MG, PENCIL_CALL)
#undef PENCIL_CALL
  } else if (rows_selected(g, spread_kernel)) {
#define ROWS_CALL(MGT, GUARD)                                                              \
  if (!torque) rows_variant<MGT, GUARD, false, true>(g, kc, b, grid, s);                  \
  else if (kc.same_width) rows_variant<MGT, GUARD, true, true>(g, kc, b, grid, s);        \
  else rows_variant<MGT, GUARD, true, false>(g, kc, b, grid, s);
    FCM_DISPATCH_ROWS(g.MG, ROWS_CALL)
#undef ROWS_CALL
  } else {
#define ATOMIC_CALL(MGT, GUARD)                                                            \
  if (!torque) atomic_variant<MGT, GUARD, false, true>(g, kc, b, grid, s);                \
  else if (kc.same_width) atomic_variant<MGT, GUARD, true, true>(g, kc, b, grid, s);      \
  else atomic_variant<MGT, GUARD, true, false>(g, kc, b, grid, s);
    FCM_DISPATCH_MG(g.MG, ATOMIC_CALL)
#undef ATOMIC_CALL
  }
  *launches += 1;
}

}  // namespace fcm
