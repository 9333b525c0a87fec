// FP32 spread J~^dagger + N~^dagger on the tensor cores (Section 3.1, eq. force_kernel_mod;
// Section 3.4, eq. torque_kernel_mod), for M_G in {10, 12, 14} with Sigma_D = Sigma or not.
//
// Along x, each particle's contribution to a grid row (y, z) of component c is a combination of
// T x profiles X_t: g, d^2 g, d g_D (and g_D when Sigma_D != Sigma), with coefficients that depend
// only on the row and c (the same coefficients the row-stationary kernel forms per row). Over a
// CTA's extended region (two x-adjacent binning tiles: EX = 15 + M_G x points, padded to 32; EY x EZ
// rows) the spread is therefore one contraction over (particle, profile):
//   f[(row, c)][x] = sum_(p, t) A[(row, c)][(p, t)] B[(p, t)][x]
// A: the row coefficients, zero outside the particle's window; B: the x profiles placed at the
// particle's window offset, zero outside it. The CTA writes A from registers into tensor memory
// (tcgen05.st), B into shared memory, and accumulates D = A B in tensor memory with
// tcgen05.mma kind::tf32 (M = 128 rows of (row, c), N = 32 x points, K = 8 per instruction). FP32
// accuracy from TF32 operands with the split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, where
// a_hi keeps the sign, exponent and top 10 mantissa bits of a and a_lo = a - a_hi (exact): the
// dropped a_lo b_lo and the truncation of the low parts are below 2^-20 relative.
//
// Pipeline: particles in chunks of 8 (K = 8 T per chunk); for each chunk and each 128-row block
// of the region all 16 warps write one A stage (the four warps of a TMEM lane quadrant take two
// particles each), one thread issues the 3 T instructions and commits them to the stage's
// mbarrier, and the warps move on to the next stage in another TMEM buffer. D of every row block
// stays in tensor memory until the CTA's particles are done; then each warp reads its lanes
// (tcgen05.ld) and adds the rows to the grid with 16-byte global reductions, as the
// row-stationary kernel's flush does. Every mbarrier wait is bounded; a wait that runs out sets
// bit 1 of the status word, the CTA skips the rest of its work, waits (bounded) for its issued
// instructions and frees its tensor memory.
#include "grid_common.cuh"
#include "tcgen05.cuh"

namespace fcm {
namespace {

constexpr int kMmaThreads = 512;     // 16 warps, four per TMEM lane quadrant
constexpr int kMmaChunk = 8;         // particles per K chunk
constexpr int kMmaBatch = 64;        // particles staged per pass
constexpr int kMmaTx = 16;           // region x points from two binning tiles
constexpr int kMmaN = 32;            // MMA N: region x padded
constexpr int kTmemCols = 512;

template <bool TORQUE, bool SAMEW>
__host__ __device__ constexpr int mma_terms() {
  return TORQUE ? (SAMEW ? 3 : 4) : 2;
}

// Layout constants of one (M_G, T) variant.
template <int MGT, int T>
struct MmaShape {
  static constexpr int EXT = kMmaTx + MGT - 1;        // region x points (<= 29)
  static constexpr int EY = 7 + MGT, EZ = 7 + MGT;    // region rows per axis (8-point tiles in y, z)
  static constexpr int ROWS = 3 * EY * EZ;            // (row, component) pairs: M of the contraction
  static constexpr int NMB = (ROWS + 127) / 128;      // 128-row blocks
  static constexpr int KC = kMmaChunk * T;            // K of one chunk
  static constexpr int NST = T == 4 ? 2 : 3;          // A stages in tensor memory
  static constexpr int DCOL = kMmaN * NMB;            // D columns
  static constexpr int NCH = kMmaBatch / kMmaChunk;   // chunks per staged pass
  static constexpr int BFL = kMmaN * KC;              // floats of one chunk's B (hi or lo)
  static_assert(EXT <= kMmaN, "region wider than the MMA N");
  static_assert(DCOL + NST * 2 * KC <= kTmemCols, "tensor memory budget");
  // shared memory (bytes): B [NCH][hi, lo][BFL] | yt, zt [batch][MGT] float4 | pc [batch][3] float4 |
  // po [batch] int4 | NST mbarriers | TMEM address | failure flag
  static constexpr size_t B_BYTES = sizeof(float) * (size_t)NCH * 2 * BFL;
  static constexpr size_t YT_OFF = B_BYTES;
  static constexpr size_t ZT_OFF = YT_OFF + sizeof(float4) * kMmaBatch * MGT;
  static constexpr size_t PC_OFF = ZT_OFF + sizeof(float4) * kMmaBatch * MGT;
  static constexpr size_t PO_OFF = PC_OFF + sizeof(float4) * kMmaBatch * 3;
  static constexpr size_t BAR_OFF = PO_OFF + sizeof(int4) * kMmaBatch;
  static constexpr size_t SLOT_OFF = BAR_OFF + sizeof(uint64_t) * NST;
  static constexpr size_t SMEM = SLOT_OFF + 16;
};

// Offset (floats) of B element (x point i, K index k) inside one chunk: K-major core matrices of
// 8 x points by 4 K entries (128 bytes), K-adjacent core matrices contiguous.
template <int KC>
__device__ inline int b_index(int i, int k) {
  return ((i >> 3) * (KC / 4) + (k >> 2)) * 32 + (i & 7) * 4 + (k & 3);
}

template <int MGT, bool TORQUE, bool SAMEW>
__global__ void __launch_bounds__(kMmaThreads, 1)
    spread_mma_kernel(Geometry<float> g, KernelConsts<float> kc, const float4* __restrict__ pos,
                      const float4* __restrict__ Fv, const float4* __restrict__ Tv, const int* __restrict__ tstart,
                      float* __restrict__ grid, int* __restrict__ status) {
  constexpr int T = mma_terms<TORQUE, SAMEW>();
  using S = MmaShape<MGT, T>;
  constexpr int MG = MGT;
  int p0, p1;
  size_t goff;
  TileOrigin o;
  if (!spread_tile_range<kMmaTx>(g, tstart, blockIdx.x, &p0, &p1, &o, &goff)) return;
  grid += goff;

  extern __shared__ __align__(128) unsigned char smem[];
  float* Bs = reinterpret_cast<float*>(smem);
  float4* yt = reinterpret_cast<float4*>(smem + S::YT_OFF);
  float4* zt = reinterpret_cast<float4*>(smem + S::ZT_OFF);
  float4* pc = reinterpret_cast<float4*>(smem + S::PC_OFF);
  int4* po = reinterpret_cast<int4*>(smem + S::PO_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::SLOT_OFF);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp & 3, role = warp >> 2;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < S::NST; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = (uint32_t)(32 * quad) << 16;   // this warp's TMEM lane quadrant
  constexpr uint32_t idesc = idesc_tf32(128, kMmaN);

  int pend[S::NST];   // stage index whose MMAs last used buffer b (-1: none outstanding)
#pragma unroll
  for (int b = 0; b < S::NST; ++b) pend[b] = -1;
  int stage = 0, fail = 0;

  for (int base = p0; base < p1 && !fail; base += kMmaBatch) {
    const int np = min(kMmaBatch, p1 - base);
    const int nch = (np + kMmaChunk - 1) / kMmaChunk;
    if (base != p0) {   // the previous pass's MMAs read B: wait for all of them
#pragma unroll
      for (int b = 0; b < S::NST; ++b)
        if (pend[b] >= 0) {
          if (!mbar_wait(&bars[b], (uint32_t)(pend[b] / S::NST) & 1u)) fail = 1;
          pend[b] = -1;
        }
      if (__syncthreads_or(fail)) { fail = 1; break; }
    }
    // per-particle tables: y and z profiles {g, d, g_D, 0}, window offsets, component weights
    for (int k = tid; k < np * 2 * MG; k += kMmaThreads) {
      const int q = k / (2 * MG);
      const int rem = k - q * 2 * MG;
      const int d = 1 + rem / MG;
      const int j = rem - (d - 1) * MG;
      const float4 y = pos[base + q];
      const float yd = d == 1 ? y.y : y.z;
      const float dd = (float)(window_start_d(g, d, yd) + j) * sel3(g.h, d) - yd;
      const float gs = expf(-dd * dd * kc.inv2S2);
      const float gd = SAMEW ? gs : expf(-dd * dd * kc.inv2SD2);
      (d == 1 ? yt : zt)[q * MGT + j] = make_float4(gs, dd, gd, 0.f);
    }
    for (int q = tid; q < np; q += kMmaThreads) {
      const float4 y = pos[base + q];
      const int3 i0 = window_starts(g, y);
      int4 off = window_offset(g, o, i0);
      off.x = min(max(wrap_once(i0.x, g.M[0]) - o.ox0, 0), kMmaTx - 1);
      po[q] = off;
      const float4 f = Fv[base + q];
      const float4 tq = TORQUE ? Tv[base + q] : make_float4(0.f, 0.f, 0.f, 0.f);
      // {F_c, u_c, v_c, kappa_c}: torque part of the g coefficient H (u_c dy + v_c dz) (or of the g_D one),
      // coefficient of d g_D: H kappa_c
      pc[3 * q + 0] = make_float4(f.x, -tq.z, tq.y, 0.f);
      pc[3 * q + 1] = make_float4(f.y, 0.f, -tq.x, tq.z);
      pc[3 * q + 2] = make_float4(f.z, tq.x, 0.f, -tq.y);
    }
    // B: every element of the pass's chunks (zeros outside each particle's window and past np)
    for (int k = tid; k < nch * kMmaChunk * kMmaN; k += kMmaThreads) {
      const int p = k / kMmaN, i = k - p * kMmaN;
      float xv[4] = {0.f, 0.f, 0.f, 0.f};
      if (p < np) {
        const float4 y = pos[base + p];
        const int i0 = window_start_d(g, 0, y.x);
        const int ox = min(max(wrap_once(i0, g.M[0]) - o.ox0, 0), kMmaTx - 1);
        const int j = i - ox;
        if (j >= 0 && j < MG) {
          const float dd = (float)(i0 + j) * g.h[0] - y.x;
          const float gs = expf(-dd * dd * kc.inv2S2);
          const float gd = SAMEW ? gs : expf(-dd * dd * kc.inv2SD2);
          xv[0] = gs;
          xv[1] = dd * dd * gs;
          xv[2] = dd * gd;
          xv[3] = gd;
        }
      }
      float* bh = Bs + (size_t)(2 * (p / kMmaChunk)) * S::BFL;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        float hi, lo;
        split_tf32(xv[t], hi, lo);
        const int e = b_index<S::KC>(i, t * kMmaChunk + (p % kMmaChunk));
        bh[e] = hi;
        bh[S::BFL + e] = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B is read by the tensor core
    __syncthreads();

    for (int ch = 0; ch < nch && !fail; ++ch) {
      for (int mb = 0; mb < S::NMB; ++mb) {
        const int b = stage % S::NST;
        int lfail = 0;
        if (pend[b] >= 0) {
          if (!mbar_wait(&bars[b], (uint32_t)(pend[b] / S::NST) & 1u)) lfail = 1;
          pend[b] = -1;
          tc_fence_after();
        }
        // A entries of this thread's row for particles ch*8 + 2 role + {0, 1}
        float hv[T][2], lv[T][2];
        const int m = mb * 128 + quad * 32 + lane;
        const int rowid = m / 3, c = m - 3 * rowid;
        const int ez = rowid / S::EY, ey = rowid - ez * S::EY;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int p = ch * kMmaChunk + 2 * role + e;
          float v[4] = {0.f, 0.f, 0.f, 0.f};
          if (m < S::ROWS && p < np) {
            const int4 off = po[p];
            const int jy = ey - off.y, jz = ez - off.z;
            if ((unsigned)jy < (unsigned)MG && (unsigned)jz < (unsigned)MG) {
              const float4 yv = yt[p * MGT + jy];
              const float4 zv = zt[p * MGT + jz];
              const float4 w = pc[3 * p + c];
              const float G = kc.nrm * yv.x * zv.x;
              const float GQ = G * fmaf(kc.B, fmaf(yv.y, yv.y, zv.y * zv.y), kc.A);
              v[0] = w.x * GQ;
              v[1] = w.x * (G * kc.B);
              if (TORQUE) {
                const float H = kc.tq * yv.z * zv.z;
                const float ct = H * fmaf(w.y, yv.y, w.z * zv.y);
                if (SAMEW) v[0] += ct;
                else v[3] = ct;
                v[2] = H * w.w;
              }
            }
          }
#pragma unroll
          for (int t = 0; t < T; ++t) split_tf32(v[t], hv[t][e], lv[t][e]);
        }
        if (!lfail) {
          const uint32_t ta = tmem + tlane + (uint32_t)(S::DCOL + b * 2 * S::KC + 2 * role);
#pragma unroll
          for (int t = 0; t < T; ++t) {
            tmem_st2(ta + t * kMmaChunk, hv[t][0], hv[t][1]);
            tmem_st2(ta + S::KC + t * kMmaChunk, lv[t][0], lv[t][1]);
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        if (__syncthreads_or(lfail)) { fail = 1; break; }
        if (tid == 0) {
          tc_fence_after();
          const uint32_t d_t = tmem + (uint32_t)(mb * kMmaN);
          const uint32_t a_t = tmem + (uint32_t)(S::DCOL + b * 2 * S::KC);
          const uint32_t bh = smem_u32(Bs + (size_t)(2 * ch) * S::BFL);
          const uint32_t bl = bh + (uint32_t)(S::BFL * sizeof(float));
          constexpr uint32_t lbo = 128, sbo = (S::KC / 4) * 128;
          const int first = (base == p0 && ch == 0);
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const uint32_t koff = (uint32_t)(t * 2 * 128);   // K entries 8t .. 8t + 7: core matrices 2t, 2t + 1
            mma_tf32(d_t, a_t + t * kMmaChunk, smem_desc(bh + koff, lbo, sbo), idesc, !(first && t == 0));
            mma_tf32(d_t, a_t + t * kMmaChunk, smem_desc(bl + koff, lbo, sbo), idesc, 1);
            mma_tf32(d_t, a_t + S::KC + t * kMmaChunk, smem_desc(bh + koff, lbo, sbo), idesc, 1);
          }
          mma_commit(&bars[b]);
        }
        pend[b] = stage;
        ++stage;
      }
    }
  }

  // all issued MMAs done (bounded), then D to the grid
#pragma unroll
  for (int b = 0; b < S::NST; ++b)
    if (pend[b] >= 0) {
      if (!mbar_wait(&bars[b], (uint32_t)(pend[b] / S::NST) & 1u)) fail = 1;
      pend[b] = -1;
    }
  fail = __syncthreads_or(fail);
  tc_fence_after();
  if (fail) {
    if (tid == 0) atomicOr(status, kStatusWaitTimeout);
  } else {
    const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
    const bool vec = (o.ox0 + S::EXT <= g.M[0]) && ((g.M[0] & 3) == 0);
    for (int mb = role; mb < S::NMB; mb += 4) {
      float v[32];
      tmem_ld32(tmem + tlane + (uint32_t)(mb * kMmaN), v);
      const int m = mb * 128 + quad * 32 + lane;
      if (m >= S::ROWS) continue;
      const int rowid = m / 3, c = m - 3 * rowid;
      const int ez = rowid / S::EY, ey = rowid - ez * S::EY;
      const int gy = wrap_index(o.oy0 + ey, g.M[1]);
      const int gz = wrap_index(o.oz0 + ez, g.M[2]);
      float* row = grid + (size_t)c * Mtot + ((size_t)gz * g.M[1] + gy) * g.M[0];
      if (vec) {
        float* p = row + o.ox0;
#pragma unroll
        for (int k = 0; k + 3 < S::EXT; k += 4)
          if (v[k] != 0.f || v[k + 1] != 0.f || v[k + 2] != 0.f || v[k + 3] != 0.f)
            red_add_v4(p + k, v[k], v[k + 1], v[k + 2], v[k + 3]);
#pragma unroll
        for (int k = (S::EXT / 4) * 4; k < S::EXT; ++k)
          if (v[k] != 0.f) atomicAdd(p + k, v[k]);
      } else {
#pragma unroll
        for (int k = 0; k < S::EXT; ++k)
          if (v[k] != 0.f) atomicAdd(row + wrap_index(o.ox0 + k, g.M[0]), v[k]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int MGT, bool TORQUE, bool SAMEW>
void mma_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b, float* grid,
                 cudaStream_t s) {
  using S = MmaShape<MGT, mma_terms<TORQUE, SAMEW>()>;
  const int nsys = g.nsys > 1 ? g.nsys : 1;
  const int blocks = nsys * ((g.ntile[0] + 1) / 2) * g.ntile[1] * g.ntile[2];
  auto k = spread_mma_kernel<MGT, TORQUE, SAMEW>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  k<<<blocks, kMmaThreads, S::SMEM, s>>>(g, kc, (const float4*)b.t_pos, (const float4*)b.t_F,
                                         (const float4*)b.t_T, b.tile_start, grid, b.status);
}

}  // namespace

bool spread_mma_eligible(const int tile[3], int MG) {
  return tile[0] == 8 && tile[1] == 8 && tile[2] == 8 && (MG == 10 || MG == 12 || MG == 14);
}

void launch_spread_mma(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, const BinBuffers& b,
                       float* grid, cudaStream_t s) {
#define MMA_CALL(MGT)                                                              \
  if (!torque) mma_variant<MGT, false, true>(g, kc, b, grid, s);                  \
  else if (kc.same_width) mma_variant<MGT, true, true>(g, kc, b, grid, s);        \
  else mma_variant<MGT, true, false>(g, kc, b, grid, s);
  switch (g.MG) {
    case 10: MMA_CALL(10) break;
    case 12: MMA_CALL(12) break;
    default: MMA_CALL(14) break;
  }
#undef MMA_CALL
}

}  // namespace fcm
