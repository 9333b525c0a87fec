// FP32 pairwise correction (Section 4 step 6, eq. correction_VF / WF / WT, Appendix B).
//
// For particle n and every m with minimum-image r = |Y_n - Y_m| < r_c:
//   U_n += al F_m + bt x (x.F_m) + cr (T_m x x)
//   W_n += cr (F_m x x) + gm T_m + dl x (x.T_m)
// with x = Y_n - Y_m and the radial coefficients of the closed form, read from
// piecewise-cubic tables built in FP64 (Taylor series for r < r_series, which
// also covers coincident points), plus the self correction. Candidates come
// from the cells around n's cell (Section 4 step 1); cells adjacent in x are
// contiguous in the cell-sorted arrays, so a CTA stages a few x ranges.
//
// GB300 decomposition: each unordered pair is evaluated once. The coefficients
// depend on r only, so the partner's terms are the same expressions with
// x -> -x (the odd cross-product terms change sign). One CTA per pair cell
// stages its own cell and a half shell of 13 neighbour cells in shared memory;
// a warp takes one particle n at a time and pairs it with the staged candidates
// after its own slot. Lanes test 32 candidates at a time; the staged slots of
// hits are compacted with a ballot into a per-warp shared-memory queue, and the
// correction is evaluated when 32 hits are queued (each lane recomputes its
// pair's separation from the staged position), so that work runs with every
// lane busy although only ~15% of candidates are within r_c. n's sums add up
// per lane (a lane sees about three of n's pairs), by a tree across the lanes
// and compensated across candidate chunks (Neumaier); the partners' sums add
// up in shared memory (one plane per component) and
// reach the output with atomic adds, so the output is zeroed first and the
// order of those additions is not fixed.
#include "fcm_internal.cuh"

namespace fcm {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kQueue = 64;

__device__ inline float min_image(float d, float L) {
  if (d > 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return d;
}

// ---------------------------------------------------------------- half-shell cell kernel
//
// One CTA per pair cell c. Each unordered pair within r_c is evaluated once (the mobility
// correction is symmetric: the pair's coefficients are shared, and the partner's terms follow
// from x -> -x), so a CTA stages only its own cell and the 13 neighbour cells of a half shell:
// offsets (dx, dy, dz) with dz = +1, or dz = 0 and dy = +1, or dz = dy = 0 and dx = +1. Every
// unordered pair of neighbouring cells is met from exactly one side (m_i >= 3 keeps the offsets
// distinct modulo m_i). The own cell is staged first in cell order, so particle i of the cell
// pairs with the staged candidates after its own slot: same-cell pairs once, no self pair.
// Terms for i add up in the lanes and a warp reduction; terms for the partner j
// add into per-candidate shared sums, which go to the output with global atomics after the
// chunk; the output is zeroed before the launch.

constexpr int kCellWarps = 8;
constexpr int kHalfChunk = 640;   // above the half-shell candidate count of the 5% suspension (about 530)
static_assert(kHalfChunk % 32 == 0, "candidate chunks are padded to whole 32-candidate passes");
constexpr int kIBatch = 64;      // particles of a cell per pass (a cell holds about 38 at 5%)
// 51.6 KB of shared memory and at most 64 registers per thread: four 256-thread CTAs per SM
constexpr int kPieces = 10;   // x ranges staged per cell: 5 rows, each split in two where it wraps in x

template <bool TORQUE>
constexpr size_t half_kernel_smem() {
  return sizeof(float4) * (size_t)kHalfChunk * (TORQUE ? 3 : 2) +
         sizeof(float) * (size_t)kHalfChunk * (TORQUE ? 6 : 3) + sizeof(float) * 12 * kIBatch +
         sizeof(int) * kCellWarps * kQueue + sizeof(int) * 64 + sizeof(float4) * kPieces;
}

__device__ inline void neu_add(float* s, float* c, float v) {
  const float t = *s + v;
  *c += (fabsf(*s) >= fabsf(v)) ? ((*s - t) + v) : ((v - t) + *s);
  *s = t;
}

template <bool TORQUE, bool SHIFT>
__global__ void __launch_bounds__(kCellWarps * 32, 4) pair_half_kernel(Geometry<float> g, PairConsts<float> pc,
                                                                       PairTable tab,
                                                                       const float4* __restrict__ cpos,
                                                                       const float4* __restrict__ cF,
                                                                       const float4* __restrict__ cT,
                                                                       const int* __restrict__ cstart,
                                                                       float* __restrict__ Uo,
                                                                       float* __restrict__ Wo) {
  constexpr int C = TORQUE ? 6 : 3;   // partner sums per candidate
  extern __shared__ float4 sm4[];
  float4* spos = sm4;
  float4* sF = spos + kHalfChunk;
  float4* sT = sF + kHalfChunk;
  float* accj = reinterpret_cast<float*>(TORQUE ? sT + kHalfChunk : sT);   // [C][chunk]
  float* acc = accj + C * kHalfChunk;                                       // [kIBatch][12]
  int* qj = reinterpret_cast<int*>(acc + 12 * kIBatch);                     // [warps][kQueue]
  int* meta = qj + kCellWarps * kQueue;                                     // pieces: source start, prefix
  float4* pshift = reinterpret_cast<float4*>(meta + 64);                    // periodic image shift per piece

  const int cell = blockIdx.x;
  const int i_begin = cstart[cell], i_end = cstart[cell + 1];
  if (i_begin >= i_end) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mx = g.mcell[0], my = g.mcell[1], mz = g.mcell[2];
  if (warp == 0) {
    // kPieces slots, lane l describes slot l: row l / 2, part l % 2 of a row that wraps in x. Row 0 is
    // the own cell and its +x neighbour (the own cell first); rows 1 .. 4 are dy = +1 at dz = 0 and
    // dy = -1, 0, +1 at dz = +1, cells cx - 1 .. cx + 1. A slot a row does not need stays empty.
    const int cs = g.nsys > 1 ? cell / g.cells_per : 0;   // system of this cell (batched launches)
    const int cbase = cs * g.cells_per;
    const int lc = cell - cbase;
    const int cx = lc % mx, cy = (lc / mx) % my, cz = lc / (mx * my);
    const int r = lane >> 1, part = lane & 1;
    int xa = 0, xb = -1;   // cells xa .. xb of the row; empty when xb < xa
    float sx = 0.f;
    if (r == 0) {
      if (part == 0) { xa = cx; xb = (cx + 1 < mx) ? cx + 1 : cx; }
      else if (cx + 1 >= mx) { xa = 0; xb = 0; sx = g.L[0]; }
    } else if (r < 5) {
      if (cx - 1 >= 0 && cx + 1 < mx) { if (part == 0) { xa = cx - 1; xb = cx + 1; } }
      else if (cx - 1 < 0) {
        if (part == 0) { xa = mx - 1; xb = mx - 1; sx = -g.L[0]; } else { xa = 0; xb = 1; }
      } else {
        if (part == 0) { xa = mx - 2; xb = mx - 1; } else { xa = 0; xb = 0; sx = g.L[0]; }
      }
    }
    const int yu = r == 1 ? cy + 1 : cy + r - 3, zu = r <= 1 ? cz : cz + 1;   // row 0: (cy, cz)
    const int yr = r == 0 ? cy : yu;
    int a = 0, cnt = 0;
    if (lane < kPieces && xb >= xa) {
      const int rowbase = cbase + mx * (pmod(yr, my) + my * pmod(zu, mz));
      a = cstart[rowbase + xa];
      cnt = cstart[rowbase + xb + 1] - a;
    }
    int pre = cnt;   // inclusive prefix over the slots
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFullMask, pre, o);
      if (lane >= o) pre += v;
    }
    if (lane < kPieces) {
      meta[2 * lane] = a;
      meta[2 * lane + 1] = pre - cnt;
      const float sy = yr < 0 ? -g.L[1] : (yr >= my ? g.L[1] : 0.f);
      const float sz = zu < 0 ? -g.L[2] : (zu >= mz ? g.L[2] : 0.f);
      pshift[lane] = make_float4(sx, sy, sz, 0.f);
    }
    if (lane == kPieces - 1) meta[2 * kPieces + 1] = pre;   // prefix sentinel
  }
  __syncthreads();
  constexpr int npieces = kPieces;
  const int total = meta[2 * npieces + 1];
  const unsigned lt = (1u << lane) - 1u;
  int* myqj = qj + warp * kQueue;

  for (int ib = i_begin; ib < i_end; ib += kIBatch) {
    const int ni = min(kIBatch, i_end - ib);
    for (int k = threadIdx.x; k < 12 * ni; k += blockDim.x) acc[k] = 0.f;
    for (int cb = 0; cb < total; cb += kHalfChunk) {
      const int nc = min(kHalfChunk, total - cb);
      __syncthreads();
      for (int q = 0; q < npieces; ++q) {
        const int lo = max(meta[2 * q + 1], cb), hi = min(meta[2 * q + 3], cb + nc);
        const int src = meta[2 * q] + (lo - meta[2 * q + 1]);
        const float4 sh = pshift[q];
        for (int k = threadIdx.x; k < hi - lo; k += blockDim.x) {
          float4 y = cpos[src + k];
          if (SHIFT) { y.x += sh.x; y.y += sh.y; y.z += sh.z; }
          spos[lo - cb + k] = y;
          sF[lo - cb + k] = cF[src + k];
          if (TORQUE) sT[lo - cb + k] = cT[src + k];
        }
      }
      for (int k = threadIdx.x; k < C * kHalfChunk; k += blockDim.x) accj[k] = 0.f;
      // pad to whole 32-candidate passes with far-away dummies: no bounds test in the loop
      const int ncp = (nc + 31) & ~31;
      for (int k = nc + threadIdx.x; k < ncp; k += blockDim.x)
        spos[k] = make_float4(1e18f, 1e18f, 1e18f, __int_as_float(-1));
      __syncthreads();
      for (int il = warp; il < ni; il += kCellWarps) {
        // candidates after particle i's own slot (the own cell is staged first, in cell order)
        const int start = max(ib - i_begin + il + 1 - cb, 0);
        if (start >= nc) continue;
        const float4 yi = cpos[ib + il];
        const float4 Fi = cF[ib + il];
        const float4 Ti = TORQUE ? cT[ib + il] : make_float4(0.f, 0.f, 0.f, 0.f);
        float u[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f};
        // one queued pair: the separation is recomputed from the staged position; i's terms go to
        // the lane's sums, j's (x -> -x) to the candidate's shared sums
        auto eval_slot = [&](int jj) {
          const float4 yj = spos[jj];
          const float dx = SHIFT ? yi.x - yj.x : min_image(yi.x - yj.x, g.L[0]);
          const float dy = SHIFT ? yi.y - yj.y : min_image(yi.y - yj.y, g.L[1]);
          const float dz = SHIFT ? yi.z - yj.z : min_image(yi.z - yj.z, g.L[2]);
          float al, bt, cr, gm, dl;
          pair_coeffs_table(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), pc, tab, al, bt, cr, gm, dl);
          const float4 Fj = sF[jj];
          const float xFj = dx * Fj.x + dy * Fj.y + dz * Fj.z;
          const float xFi = dx * Fi.x + dy * Fi.y + dz * Fi.z;
          float ui0 = al * Fj.x + bt * xFj * dx, ui1 = al * Fj.y + bt * xFj * dy, ui2 = al * Fj.z + bt * xFj * dz;
          float uj0 = al * Fi.x + bt * xFi * dx, uj1 = al * Fi.y + bt * xFi * dy, uj2 = al * Fi.z + bt * xFi * dz;
          float* aj = accj + jj;   // component c at aj[c kHalfChunk]
          if (TORQUE) {
            const float4 Tj = sT[jj];
            // U_i += cr (T_j x x), U_j -= cr (T_i x x)
            ui0 += cr * (Tj.y * dz - Tj.z * dy);
            ui1 += cr * (Tj.z * dx - Tj.x * dz);
            ui2 += cr * (Tj.x * dy - Tj.y * dx);
            uj0 -= cr * (Ti.y * dz - Ti.z * dy);
            uj1 -= cr * (Ti.z * dx - Ti.x * dz);
            uj2 -= cr * (Ti.x * dy - Ti.y * dx);
            // W_i += cr (F_j x x) + gm T_j + dl x (x.T_j), W_j += -cr (F_i x x) + gm T_i + dl x (x.T_i)
            const float xTj = dx * Tj.x + dy * Tj.y + dz * Tj.z;
            const float xTi = dx * Ti.x + dy * Ti.y + dz * Ti.z;
            w[0] += (cr * (Fj.y * dz - Fj.z * dy) + gm * Tj.x + dl * xTj * dx);
            w[1] += (cr * (Fj.z * dx - Fj.x * dz) + gm * Tj.y + dl * xTj * dy);
            w[2] += (cr * (Fj.x * dy - Fj.y * dx) + gm * Tj.z + dl * xTj * dz);
            atomicAdd(aj + 3 * kHalfChunk, gm * Ti.x + dl * xTi * dx - cr * (Fi.y * dz - Fi.z * dy));
            atomicAdd(aj + 4 * kHalfChunk, gm * Ti.y + dl * xTi * dy - cr * (Fi.z * dx - Fi.x * dz));
            atomicAdd(aj + 5 * kHalfChunk, gm * Ti.z + dl * xTi * dz - cr * (Fi.x * dy - Fi.y * dx));
          }
          u[0] += ui0;
          u[1] += ui1;
          u[2] += ui2;
          atomicAdd(aj + 0 * kHalfChunk, uj0);
          atomicAdd(aj + 1 * kHalfChunk, uj1);
          atomicAdd(aj + 2 * kHalfChunk, uj2);
        };
        int qn = 0;   // queued pairs (the same in every lane); the queue starts at slot 0
        for (int base = start & ~31; base < ncp; base += 32) {
          const int k = base + lane;
          const float4 yj = spos[k];
          const float dx = SHIFT ? yi.x - yj.x : min_image(yi.x - yj.x, g.L[0]);
          const float dy = SHIFT ? yi.y - yj.y : min_image(yi.y - yj.y, g.L[1]);
          const float dz = SHIFT ? yi.z - yj.z : min_image(yi.z - yj.z, g.L[2]);
          const bool hit = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < pc.rc2 && k >= start;
          const unsigned m = __ballot_sync(kFullMask, hit);
          if (m == 0u) continue;
          if (hit) myqj[qn + __popc(m & lt)] = k;   // qn < 32 here, so the slot is < 64
          qn += __popc(m);
          if (qn >= 32) {
            __syncwarp();
            eval_slot(myqj[lane]);
            __syncwarp();
            if (lane < qn - 32) myqj[lane] = myqj[32 + lane];   // the overflow moves to the front
            qn -= 32;
            __syncwarp();
          }
        }
        __syncwarp();
        if (lane < qn) eval_slot(myqj[lane]);
        __syncwarp();
        float r[6] = {u[0], u[1], u[2], w[0], w[1], w[2]};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int c = 0; c < 6; ++c) r[c] += __shfl_xor_sync(kFullMask, r[c], o);
        }
        if (lane == 0) {
          float* a = acc + 12 * il;
#pragma unroll
          for (int c = 0; c < 6; ++c) neu_add(a + c, a + 6 + c, r[c]);
        }
      }
      __syncthreads();
      // the partners' sums of this chunk to the output
      for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        const float* aj = accj + k;
        const size_t o = 3 * (size_t)index_from_w(spos[k].w);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (aj[c * kHalfChunk] != 0.f) atomicAdd(Uo + o + c, aj[c * kHalfChunk]);
        if (TORQUE && Wo) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (aj[(3 + c) * kHalfChunk] != 0.f) atomicAdd(Wo + o + c, aj[(3 + c) * kHalfChunk]);
        }
      }
    }
    __syncthreads();
    for (int il = threadIdx.x; il < ni; il += blockDim.x) {
      const int i = ib + il;
      const float* a = acc + 12 * il;
      const float4 Fi = cF[i];
      const size_t o = 3 * (size_t)index_from_w(cpos[i].w);
      atomicAdd(Uo + o + 0, (a[0] + a[6]) + pc.selfVF * Fi.x);
      atomicAdd(Uo + o + 1, (a[1] + a[7]) + pc.selfVF * Fi.y);
      atomicAdd(Uo + o + 2, (a[2] + a[8]) + pc.selfVF * Fi.z);
      if (TORQUE && Wo) {
        const float4 Ti = cT[i];
        atomicAdd(Wo + o + 0, (a[3] + a[9]) + pc.selfWT * Ti.x);
        atomicAdd(Wo + o + 1, (a[4] + a[10]) + pc.selfWT * Ti.y);
        atomicAdd(Wo + o + 2, (a[5] + a[11]) + pc.selfWT * Ti.z);
      }
    }
    __syncthreads();
  }
}

template <bool TORQUE, bool SHIFT>
static void half_variant(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab,
                         const BinBuffers& b, float* upair, float* wpair, cudaStream_t s) {
  const size_t smem = half_kernel_smem<TORQUE>();
  auto k = pair_half_kernel<TORQUE, SHIFT>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<b.ncells, kCellWarps * 32, smem, s>>>(g, pc, tab, (const float4*)b.c_pos, (const float4*)b.c_F,
                                            (const float4*)b.c_T, b.cell_start, upair, wpair);
}

void launch_pair_f32(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab, bool torque,
                     const BinBuffers& b, int n, float* upair, float* wpair, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  // every particle's sums arrive by atomic adds from its own CTA and its neighbours'
  launch_zero(upair, sizeof(float) * 3 * (size_t)n, s, launches);
  if (torque && wpair) launch_zero(wpair, sizeof(float) * 3 * (size_t)n, s, launches);
  if (torque) {
    if (g.shift) half_variant<true, true>(g, pc, tab, b, upair, wpair, s);
    else half_variant<true, false>(g, pc, tab, b, upair, wpair, s);
  } else {
    if (g.shift) half_variant<false, true>(g, pc, tab, b, upair, wpair, s);
    else half_variant<false, false>(g, pc, tab, b, upair, wpair, s);
  }
  *launches += 1;
}

}  // namespace fcm
