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
// GB300 decomposition: one CTA per pair cell stages the candidates of the 27
// neighbour cells in shared memory; a warp takes one particle n at a time.
// Lanes test 32 candidates at a time; the staged slots of hits are compacted
// with a ballot into a per-warp shared-memory queue, and the correction is
// evaluated when 32 hits are queued (each lane recomputes its pair's
// separation from the staged position), so that work runs with every lane busy
// although only ~15% of candidates are within r_c. Per-lane sums are
// compensated (Kahan), the warp reduction is a tree, and the per-particle
// totals over candidate chunks are compensated again (Neumaier).
#include "fcm_internal.cuh"

namespace fcm {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kQueue = 64;

// Compensated (Kahan) running sum: c carries the low-order part lost by s.
struct Kahan {
  float s, c;
  __device__ inline void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ inline float value() const { return s - c; }
};

__device__ inline float min_image(float d, float L) {
  if (d > 0.5f * L) d -= L;
  else if (d < -0.5f * L) d += L;
  return d;
}

template <bool TORQUE>
__device__ inline void eval_pair(const PairConsts<float>& pc, const PairTable& tab, float4 dq, float4 Fj, float4 Tj,
                                 Kahan* u, Kahan* w) {
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

// ---------------------------------------------------------------- cell-tiled kernel
//
// One CTA per pair cell. The candidates of its 27 neighbour cells are staged
// once in shared memory (positions, forces, torques; chunks of kCandChunk),
// then each warp takes particles of the cell and runs the same ballot
// compaction over the staged candidates: candidate reads are shared-memory
// loads instead of L2 traffic repeated for every particle of the cell.

constexpr int kCellWarps = 8;
constexpr int kCandChunk = 1280;   // above the 27-cell candidate count of the 5% suspension (about 1,025)
static_assert(kCandChunk % 32 == 0, "candidate chunks are padded to whole 32-candidate passes");
constexpr int kIBatch = 128;
constexpr int kMaxPieces = 18;

template <bool TORQUE>
constexpr size_t cell_kernel_smem() {
  return sizeof(float4) * (size_t)kCandChunk * (TORQUE ? 3 : 2) + sizeof(float) * 12 * kIBatch +
         sizeof(int) * kCellWarps * kQueue + sizeof(int) * 64 + sizeof(float4) * kMaxPieces;
}

__device__ inline void neu_add(float* s, float* c, float v) {
  const float t = *s + v;
  *c += (fabsf(*s) >= fabsf(v)) ? ((*s - t) + v) : ((v - t) + *s);
  *s = t;
}

template <bool TORQUE, bool SHIFT>
__global__ void __launch_bounds__(kCellWarps * 32, 3) pair_cell_kernel(Geometry<float> g, PairConsts<float> pc,
                                                                       PairTable tab,
                                                                       const float4* __restrict__ cpos,
                                                                       const float4* __restrict__ cF,
                                                                       const float4* __restrict__ cT,
                                                                       const int* __restrict__ cstart,
                                                                       float* __restrict__ Uo,
                                                                       float* __restrict__ Wo) {
  extern __shared__ float4 sm4[];
  float4* spos = sm4;
  float4* sF = spos + kCandChunk;
  float4* sT = sF + kCandChunk;
  float* acc = reinterpret_cast<float*>(TORQUE ? sT + kCandChunk : sT);   // [kIBatch][12]
  int* qj = reinterpret_cast<int*>(acc + 12 * kIBatch);                     // [warps][kQueue]
  int* meta = qj + kCellWarps * kQueue;                                     // pieces: source start, prefix
  float4* pshift = reinterpret_cast<float4*>(meta + 64);                    // periodic image shift per piece

  const int cell = blockIdx.x;
  const int i_begin = cstart[cell], i_end = cstart[cell + 1];
  if (i_begin >= i_end) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mx = g.mcell[0], my = g.mcell[1], mz = g.mcell[2];
  if (threadIdx.x == 0) {
    const int cs = g.nsys > 1 ? cell / g.cells_per : 0;   // system of this cell (batched launches)
    const int cbase = cs * g.cells_per;
    const int lc = cell - cbase;
    const int cx = lc % mx, cy = (lc / mx) % my, cz = lc / (mx * my);
    int np = 0, total = 0;
    for (int ddz = -1; ddz <= 1; ++ddz) {
      const int zu = cz + ddz;
      const int zc = pmod(zu, mz);
      const float sz = zu < 0 ? -g.L[2] : (zu >= mz ? g.L[2] : 0.f);
      for (int ddy = -1; ddy <= 1; ++ddy) {
        const int yu = cy + ddy;
        const float sy = yu < 0 ? -g.L[1] : (yu >= my ? g.L[1] : 0.f);
        const int rowbase = cbase + mx * (pmod(yu, my) + my * zc);
        int ra[2], rb[2], k = 0;
        float sx[2] = {0.f, 0.f};
        if (cx - 1 >= 0 && cx + 1 < mx) { ra[0] = cx - 1; rb[0] = cx + 1; k = 1; }
        else if (cx - 1 < 0) { ra[0] = mx - 1; rb[0] = mx - 1; sx[0] = -g.L[0]; ra[1] = 0; rb[1] = 1; k = 2; }
        else { ra[0] = mx - 2; rb[0] = mx - 1; ra[1] = 0; rb[1] = 0; sx[1] = g.L[0]; k = 2; }
        for (int q = 0; q < k; ++q) {
          const int a = cstart[rowbase + ra[q]], b = cstart[rowbase + rb[q] + 1];
          meta[2 * np] = a;
          meta[2 * np + 1] = total;
          pshift[np] = make_float4(sx[q], sy, sz, 0.f);
          total += b - a;
          ++np;
        }
      }
    }
    meta[2 * np + 1] = total;   // prefix sentinel
    meta[63] = np;
  }
  __syncthreads();
  const int npieces = meta[63];
  const int total = meta[2 * npieces + 1];
  const unsigned lt = (1u << lane) - 1u;
  int* myqj = qj + warp * kQueue;

  for (int ib = i_begin; ib < i_end; ib += kIBatch) {
    const int ni = min(kIBatch, i_end - ib);
    for (int k = threadIdx.x; k < 12 * ni; k += blockDim.x) acc[k] = 0.f;
    for (int cb = 0; cb < total; cb += kCandChunk) {
      const int nc = min(kCandChunk, total - cb);
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
      // pad to whole 32-candidate passes with far-away dummies (index -1): no bounds test in the loop
      const int ncp = (nc + 31) & ~31;
      for (int k = nc + threadIdx.x; k < ncp; k += blockDim.x)
        spos[k] = make_float4(1e18f, 1e18f, 1e18f, __int_as_float(-1));
      __syncthreads();
      for (int il = warp; il < ni; il += kCellWarps) {
        const float4 yi = cpos[ib + il];
        const int self = __float_as_int(yi.w);
        Kahan u[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        Kahan w[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        // one queued hit: the separation is recomputed from the staged position
        auto eval_slot = [&](int jj) {
          const float4 yj = spos[jj];
          float4 dq;
          dq.x = SHIFT ? yi.x - yj.x : min_image(yi.x - yj.x, g.L[0]);
          dq.y = SHIFT ? yi.y - yj.y : min_image(yi.y - yj.y, g.L[1]);
          dq.z = SHIFT ? yi.z - yj.z : min_image(yi.z - yj.z, g.L[2]);
          dq.w = fmaf(dq.x, dq.x, fmaf(dq.y, dq.y, dq.z * dq.z));
          eval_pair<TORQUE>(pc, tab, dq, sF[jj], TORQUE ? sT[jj] : make_float4(0.f, 0.f, 0.f, 0.f), u, w);
        };
        int qn = 0;   // queued hits (the same in every lane); the queue starts at slot 0
        for (int base = 0; base < ncp; base += 32) {
          const float4 yj = spos[base + lane];
          const float dx = SHIFT ? yi.x - yj.x : min_image(yi.x - yj.x, g.L[0]);
          const float dy = SHIFT ? yi.y - yj.y : min_image(yi.y - yj.y, g.L[1]);
          const float dz = SHIFT ? yi.z - yj.z : min_image(yi.z - yj.z, g.L[2]);
          const bool hit = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < pc.rc2 && __float_as_int(yj.w) != self;
          const unsigned m = __ballot_sync(kFullMask, hit);
          if (m == 0u) continue;
          if (hit) myqj[qn + __popc(m & lt)] = base + lane;   // qn < 32 here, so the slot is < 64
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
        float r[6] = {u[0].value(), u[1].value(), u[2].value(), w[0].value(), w[1].value(), w[2].value()};
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
    }
    __syncthreads();
    for (int il = threadIdx.x; il < ni; il += blockDim.x) {
      const int i = ib + il;
      const float* a = acc + 12 * il;
      const float4 Fi = cF[i];
      const size_t o = 3 * (size_t)index_from_w(cpos[i].w);
      Uo[o + 0] = (a[0] + a[6]) + pc.selfVF * Fi.x;
      Uo[o + 1] = (a[1] + a[7]) + pc.selfVF * Fi.y;
      Uo[o + 2] = (a[2] + a[8]) + pc.selfVF * Fi.z;
      if (TORQUE && Wo) {
        const float4 Ti = cT[i];
        Wo[o + 0] = (a[3] + a[9]) + pc.selfWT * Ti.x;
        Wo[o + 1] = (a[4] + a[10]) + pc.selfWT * Ti.y;
        Wo[o + 2] = (a[5] + a[11]) + pc.selfWT * Ti.z;
      }
    }
    __syncthreads();
  }
}

template <bool TORQUE, bool SHIFT>
static void cell_variant(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab,
                         const BinBuffers& b, float* upair, float* wpair, cudaStream_t s) {
  const size_t smem = cell_kernel_smem<TORQUE>();
  auto k = pair_cell_kernel<TORQUE, SHIFT>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<b.ncells, kCellWarps * 32, smem, s>>>(g, pc, tab, (const float4*)b.c_pos, (const float4*)b.c_F,
                                            (const float4*)b.c_T, b.cell_start, upair, wpair);
}

void launch_pair_f32(const Geometry<float>& g, const PairConsts<float>& pc, const PairTable& tab, bool torque,
                     const BinBuffers& b, int n, float* upair, float* wpair, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  if (torque) {
    if (g.shift) cell_variant<true, true>(g, pc, tab, b, upair, wpair, s);
    else cell_variant<true, false>(g, pc, tab, b, upair, wpair, s);
  } else {
    if (g.shift) cell_variant<false, true>(g, pc, tab, b, upair, wpair, s);
    else cell_variant<false, false>(g, pc, tab, b, upair, wpair, s);
  }
  *launches += 1;
}

}  // namespace fcm
