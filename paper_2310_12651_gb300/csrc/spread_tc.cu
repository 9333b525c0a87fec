// FP32 spread J~^dagger + N~^dagger on the tensor cores along x-pencils (Section 3.1,
// eq. force_kernel_mod; Section 3.4, eq. torque_kernel_mod), for Sigma_D = Sigma and M_G <= 14.
//
// With G = g(dy) g(dz), s = dy^2 + dz^2, F' = nrm F and U' = tq T, a particle adds to grid row
// (y, z), component c, point x (d = x - Y_x, g = g(d)):
//   f_c(x) += G [F'_c A g + w_c] + (G s) [F'_c B g] + (G dy) [beta3_c g] + (G dz) [beta4_c g]
//   w = (B F'x d^2 g, B F'y d^2 g + U'z d g, B F'z d^2 g - U'y d g),
//   beta3 = (-U'z, 0, U'x), beta4 = (U'y, -U'x, 0)
// (forces only: the first two terms, w = B F' d^2 g). Over a pencil's extended (y, z) region this is
// one contraction over (particle, term):
//   D[row][(c, x)] += sum_(p, t) A[row][(p, t)] B[(p, t)][(c, x)]
// with A the four row factors (G, G s, G dy, G dz; zero outside the particle's window) and B the
// bracketed x profiles. M = the region's rows in 128-row blocks, N = 3 components x 32 x positions,
// K = 4 terms x 4 particles per stage. A and B are written by the threads into shared memory
// (K-major core matrices, no swizzle), D accumulates in tensor memory (tcgen05.mma kind::tf32, FP32
// accuracy from the three-product split of the TF32 operands: a_hi b_hi + a_hi b_lo + a_lo b_hi).
//
// The CTA walks every 8-point tile of one (y, z) tile column (a pencil). Column x of component c
// lives in tensor-memory column c 32 + (x mod 32): particles of tile s write x in [8 s, 8 s + 21),
// so once the walk reaches tile s + 2 the points 8 s .. 8 s + 7 are complete: each warp reads them
// from its lanes (tcgen05.ld), adds them to the grid with 16-byte reductions and zeros the columns for
// reuse. Only the (y, z) halo goes to the grid with reductions; the x halo stays in tensor memory.
// Stages are double-buffered: the threads form stage k + 1 while the tensor core runs stage k. Every
// mbarrier wait is bounded; a wait that runs out sets bit 1 of the status word, the CTA skips the rest
// of its work, waits (bounded) for what it issued and frees its tensor memory.
#include "grid_common.cuh"
#include "tcgen05.cuh"

namespace fcm {
namespace {

constexpr int kTcProducers = 448;    // producer threads: one per region row (at most 21 x 21 = 441)
constexpr int kTcThreads = kTcProducers + 32;   // + one warp that issues the MMAs
constexpr int kTcChunk = 64;         // particles whose tables are staged per pass
constexpr int kTcStageP = 4;         // particles per MMA stage
constexpr int kTcRing = 32;          // x positions per component in tensor memory
constexpr int kTcN = 3 * kTcRing;    // MMA N
constexpr int kTcCols = 512;         // tensor-memory columns allocated (D uses NMB x 96)

template <int MGT, bool TORQUE>
struct TcShape {
  static constexpr int T = TORQUE ? 4 : 2;            // terms per particle
  static constexpr int KS = kTcStageP * T;            // K of one stage (8 or 16)
  static constexpr int KSTEPS = KS / 8;               // MMA K steps per stage
  static constexpr int EY = 7 + MGT, EZ = 7 + MGT;    // region rows per axis (8-point tiles in y, z)
  static constexpr int ROWS = EY * EZ;
  static constexpr int NPW = (ROWS + 31) / 32;        // producer warps
  static constexpr int NMB = (ROWS + 127) / 128;      // 128-row blocks
  static constexpr int AFL = 128 * KS;                // floats of one block's A (hi or lo)
  static constexpr int BFL = kTcN * KS;               // floats of B (hi or lo)
  static_assert(ROWS <= kTcProducers, "one producer thread per row");
  static_assert(NMB * kTcN <= kTcCols, "tensor memory budget");
  // shared memory (bytes): A [2][NMB][hi, lo][AFL] | B [2][hi, lo][BFL] | yt, zt, xt [chunk][MGT] float4 |
  // pf, pt [chunk] float4 | po [chunk] int4 | raw [2][3][chunk] float4 | full[2], empty[2] mbarriers |
  // stage flags [2] | TMEM address
  static constexpr size_t A_OFF = 0;
  static constexpr size_t B_OFF = A_OFF + sizeof(float) * 2 * NMB * 2 * (size_t)AFL;
  static constexpr size_t YT_OFF = B_OFF + sizeof(float) * 2 * 2 * (size_t)BFL;
  static constexpr size_t ZT_OFF = YT_OFF + sizeof(float4) * kTcChunk * MGT;
  static constexpr size_t XT_OFF = ZT_OFF + sizeof(float4) * kTcChunk * MGT;
  static constexpr size_t PF_OFF = XT_OFF + sizeof(float4) * kTcChunk * MGT;
  static constexpr size_t PT_OFF = PF_OFF + sizeof(float4) * kTcChunk;
  static constexpr size_t PO_OFF = PT_OFF + sizeof(float4) * kTcChunk;
  static constexpr size_t RAW_OFF = PO_OFF + sizeof(int4) * kTcChunk;
  static constexpr size_t BAR_OFF = RAW_OFF + sizeof(float4) * 2 * 3 * kTcChunk;
  static constexpr size_t FLAG_OFF = BAR_OFF + sizeof(uint64_t) * 4;
  static constexpr size_t SLOT_OFF = FLAG_OFF + sizeof(int) * 4;
  static constexpr size_t SMEM = SLOT_OFF + 16;
};

// Offset (floats) of element (row or column r, K index k) of a K-major operand: core matrices of
// 8 rows x 4 K entries (128 bytes), K-adjacent core matrices contiguous.
template <int KS>
__device__ inline int kmajor_index(int r, int k) {
  return ((r >> 3) * (KS / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier among the producer warps only (named barrier 1).
__device__ inline void producers_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

__device__ __forceinline__ void cp_async16_tc(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int MGT, bool TORQUE>
__global__ void __launch_bounds__(kTcThreads, 1)
    spread_pencil_tc_kernel(Geometry<float> g, KernelConsts<float> kc, const float4* __restrict__ pos,
                            const float4* __restrict__ Fv, const float4* __restrict__ Tv,
                            const int* __restrict__ tstart, float* __restrict__ grid, int* __restrict__ status) {
  using S = TcShape<MGT, TORQUE>;
  constexpr int T = S::T, KS = S::KS;
  constexpr int MG = MGT;
  constexpr int NPROD = 32 * S::NPW;   // producer threads of this variant
  const int ntx = g.ntile[0], nty = g.ntile[1];
  const int per = nty * g.ntile[2];
  const int sys = blockIdx.x / per;
  const int pc = blockIdx.x - sys * per;
  const int t0 = sys * g.tiles_per + ntx * pc;
  const int p_begin = tstart[t0], p_end = tstart[t0 + ntx];
  if (p_begin >= p_end) return;
  if (g.nsys > 1) grid += (size_t)sys * (size_t)g.grid_stride;
  const int oy0 = (pc % nty) * g.tile[1], oz0 = (pc / nty) * g.tile[2];

  extern __shared__ __align__(128) unsigned char smem[];
  float* As = reinterpret_cast<float*>(smem + S::A_OFF);
  float* Bs = reinterpret_cast<float*>(smem + S::B_OFF);
  float4* yt = reinterpret_cast<float4*>(smem + S::YT_OFF);
  float4* zt = reinterpret_cast<float4*>(smem + S::ZT_OFF);
  float4* xt = reinterpret_cast<float4*>(smem + S::XT_OFF);
  float4* pf = reinterpret_cast<float4*>(smem + S::PF_OFF);
  float4* pt = reinterpret_cast<float4*>(smem + S::PT_OFF);
  int4* po = reinterpret_cast<int4*>(smem + S::PO_OFF);
  float4* raw = reinterpret_cast<float4*>(smem + S::RAW_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::BAR_OFF);
  uint64_t* empty = full + 2;
  int* flags = reinterpret_cast<int*>(smem + S::FLAG_OFF);   // [0, 1]: stage in buffer b is real; [2]: failure
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::SLOT_OFF);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool producer = warp < S::NPW;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(S::NPW) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])) : "memory");
    }
    flags[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int fail = 0;

  if (!producer) {
    // ---- the MMA issuer: one thread; waits for a full stage, issues it, commits it to empty[b]
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, kTcN);
      constexpr uint32_t lbo = 128, sbo = (KS / 4) * 128;
      const uint64_t a0 = smem_desc(smem_u32(As), lbo, sbo), b0 = smem_desc(smem_u32(Bs), lbo, sbo);
      // descriptor offsets: the address field holds bytes / 16
      constexpr uint64_t kA = (uint64_t)(S::AFL * sizeof(float)) >> 4;   // hi -> lo, and block stride / 2
      constexpr uint64_t kB = (uint64_t)(S::BFL * sizeof(float)) >> 4;
      for (int k = 0;; ++k) {
        const int b = k & 1;
        if (!mbar_wait(&full[b], (uint32_t)(k >> 1) & 1u)) { fail = 1; break; }
        tc_fence_after();
        if (!flags[b]) break;
        const uint64_t bh = b0 + (uint64_t)b * 2 * kB, bl = bh + kB;
#pragma unroll
        for (int m = 0; m < S::NMB; ++m) {
          const uint64_t ah = a0 + (uint64_t)(b * S::NMB + m) * 2 * kA, al = ah + kA;
          const uint32_t d_t = tmem + (uint32_t)(m * kTcN);
#pragma unroll
          for (int ks = 0; ks < S::KSTEPS; ++ks) {
            const uint64_t ko = (uint64_t)(ks * 2 * 128) >> 4;   // K entries 8 ks .. 8 ks + 7
            mma_tf32_ss(d_t, ah + ko, bh + ko, idesc, 1);
            mma_tf32_ss(d_t, ah + ko, bl + ko, idesc, 1);
            mma_tf32_ss(d_t, al + ko, bh + ko, idesc, 1);
          }
        }
        mma_commit(&empty[b]);
      }
      if (fail) flags[2] = 1;
    }
    __syncwarp();
  } else {
    // ---- producers: one region row per thread
    const int row = tid;
    const bool has_row = row < S::ROWS;
    const int ez = has_row ? row / S::EY : 0, ey = has_row ? row - (row / S::EY) * S::EY : 0;
    const int mb = warp >> 2;                 // 128-row block; this warp's lanes in it: 32 (warp & 3) + lane
    const int mlane = row & 127;
    const uint32_t dcol = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mb * kTcN);
#pragma unroll
    for (int c = 0; c < kTcN; c += 8) tmem_zero8(dcol + c);   // D starts at zero
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();

    const size_t Mtot = (size_t)g.M[0] * g.M[1] * g.M[2];
    const bool vec_rows = (g.M[0] & 3) == 0;
    float* const r0 = grid + ((size_t)wrap_index(oz0 + ez, g.M[2]) * g.M[1] + wrap_index(oy0 + ey, g.M[1])) * g.M[0];
    // Adds the points x = 8 st .. 8 st + npts - 1 of this thread's row to the grid and zeros their
    // tensor-memory columns (warp-collective: every lane of the warp takes part).
    auto flush_step = [&](int st, int npts) {
      const int x0 = 8 * st;
      const uint32_t cx = (uint32_t)(x0 & (kTcRing - 1));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float v[8];
        tmem_ld8(dcol + (uint32_t)(c * kTcRing) + cx, v);
        if (has_row) {
          float* rowp = r0 + (size_t)c * Mtot;
#pragma unroll
          for (int h = 0; h < 8; h += 4) {
            if (h >= npts) continue;
            if (v[h] == 0.f && v[h + 1] == 0.f && v[h + 2] == 0.f && v[h + 3] == 0.f) continue;
            const int x = x0 + h;
            if (vec_rows && x + 3 < g.M[0] && h + 3 < npts) {
              red_add_v4(rowp + x, v[h], v[h + 1], v[h + 2], v[h + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e)
                if (h + e < npts && v[h + e] != 0.f) atomicAdd(rowp + wrap_index(x + e, g.M[0]), v[h + e]);
            }
          }
        }
        tmem_zero8(dcol + (uint32_t)(c * kTcRing) + cx);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    };
    // Raw rows (position, force, torque) of particles [base, base + n) into raw buffer `buf`.
    auto fetch = [&](int buf, int base, int n) {
      float4* r = raw + (size_t)buf * 3 * kTcChunk;
      for (int k = tid; k < (TORQUE ? 3 : 2) * n; k += NPROD) {
        const int a = k / n, q = k - a * n;
        cp_async16_tc(r + a * kTcChunk + q, (a == 0 ? pos : (a == 1 ? Fv : Tv)) + base + q);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };

    int stage = 0;             // stages handed to the issuer; stage k used buffer k & 1
    int flushed = 0;           // tile steps 0 .. flushed - 1 are in the grid
    int last_step = 0;         // highest tile step handed over
    // Waits until the issuer's commit for stage k arrived (all of this thread's waits are bounded).
    auto wait_stage = [&](int k) {
      if (k >= 0 && !mbar_wait(&empty[k & 1], (uint32_t)(k >> 1) & 1u)) fail = 1;
    };

    fetch(0, p_begin, min(kTcChunk, p_end - p_begin));
    int rb = 0;
    for (int base = p_begin; base < p_end; base += kTcChunk, rb ^= 1) {
      const int np = min(kTcChunk, p_end - base);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      producers_sync(NPROD);   // raw rows in; every producer is done with the previous tables
      if (base + np < p_end) fetch(rb ^ 1, base + np, min(kTcChunk, p_end - base - np));
      const float4* rpos = raw + (size_t)rb * 3 * kTcChunk;
      const float4* rF = rpos + kTcChunk;
      const float4* rT = rF + kTcChunk;
      // per-particle tables: y and z profiles {g, d, d^2, 0}, x profiles {g, d^2 g, d g, 0} over the window
      for (int k = tid; k < np * 3 * MG; k += NPROD) {
        const int q = k / (3 * MG);
        const int rem = k - q * 3 * MG;
        const int d = rem / MG;
        const int j = rem - d * MG;
        const float4 y = rpos[q];
        const float yd = d == 0 ? y.x : (d == 1 ? y.y : y.z);
        const float dd = (float)(window_start_d(g, d, yd) + j) * sel3(g.h, d) - yd;
        const float gs = expf(-dd * dd * kc.inv2S2);
        if (d == 0) xt[q * MGT + j] = make_float4(gs, dd * dd * gs, dd * gs, 0.f);
        else (d == 1 ? yt : zt)[q * MGT + j] = make_float4(gs, dd, dd * dd, 0.f);
      }
      for (int q = tid; q < np; q += NPROD) {
        const float4 y = rpos[q];
        const int3 i0 = window_starts(g, y);
        const int wx = wrap_once(i0.x, g.M[0]);
        const int step = min(max(wx >> 3, 0), ntx - 1);
        int4 off;
        off.x = min(max(wx - 8 * step, 0), 7);
        off.y = min(max(wrap_once(i0.y, g.M[1]) - oy0, 0), g.tile[1] - 1);
        off.z = min(max(wrap_once(i0.z, g.M[2]) - oz0, 0), g.tile[2] - 1);
        off.w = step;
        po[q] = off;
        const float4 f = rF[q];
        const float4 t = TORQUE ? rT[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        pf[q] = make_float4(kc.nrm * f.x, kc.nrm * f.y, kc.nrm * f.z, 0.f);
        pt[q] = make_float4(kc.tq * t.x, kc.tq * t.y, kc.tq * t.z, 0.f);
      }
      producers_sync(NPROD);

      for (int q0 = 0; q0 < np;) {
        // a stage: up to kTcStageP consecutive particles whose tile steps differ by at most one, so that
        // its x positions and the columns not yet in the grid span at most 29 < 32 ring positions
        const int st_lo = po[q0].w;
        int q1 = q0 + 1;
        while (q1 < np && q1 < q0 + kTcStageP && po[q1].w <= st_lo + 1) ++q1;
        const int st_hi = po[q1 - 1].w;                      // particles are in tile order
        const int b = stage & 1;
        wait_stage(stage - 2);                                // buffer b was last read by stage - 2
        // tile steps below st_hi - 1 are complete (every later particle starts at st_lo or above): once
        // the stages handed over are done they go to the grid and their columns are zeroed for reuse
        if (st_hi - 2 >= flushed) {
          wait_stage(stage - 1);
          tc_fence_after();
          if (!__any_sync(kFullMask32, fail))
            for (; flushed <= st_hi - 2; ++flushed) flush_step(flushed, 8);
          flushed = max(flushed, st_hi - 1);
        }
        last_step = st_hi;
        // A: this thread's row factors for the stage's particles (K index e T + t)
        {
          float av[kTcStageP][4];
#pragma unroll
          for (int e = 0; e < kTcStageP; ++e) {
            const int q = q0 + e;
            av[e][0] = av[e][1] = av[e][2] = av[e][3] = 0.f;
            if (q < q1 && has_row) {
              const int4 off = po[q];
              const int jy = ey - off.y, jz = ez - off.z;
              if ((unsigned)jy < (unsigned)MG && (unsigned)jz < (unsigned)MG) {
                const float4 yv = yt[q * MGT + jy];
                const float4 zv = zt[q * MGT + jz];
                const float G = yv.x * zv.x;
                av[e][0] = G;
                av[e][1] = G * (yv.z + zv.z);
                av[e][2] = G * yv.y;
                av[e][3] = G * zv.y;
              }
            }
          }
          float* ah = As + ((size_t)(b * S::NMB + mb) * 2) * S::AFL;
          float* al = ah + S::AFL;
#pragma unroll
          for (int e = 0; e < kTcStageP; e += 4 / T) {
            float h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split_tf32(av[e + u / T][u % T], h[u], l[u]);
            const int o = kmajor_index<KS>(mlane, e * T);
            *reinterpret_cast<float4*>(ah + o) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(al + o) = make_float4(l[0], l[1], l[2], l[3]);
          }
        }
        // B: (particle, term) x (component, x position mod 32)
        {
          float* bh = Bs + (size_t)(b * 2) * S::BFL;
          float* bl = bh + S::BFL;
          for (int it = tid; it < kTcStageP * kTcN; it += NPROD) {
            const int e = it / kTcN, n = it - e * kTcN;
            const int c = n / kTcRing, r = n - c * kTcRing;
            const int q = q0 + e;
            float bv[4] = {0.f, 0.f, 0.f, 0.f};
            if (q < q1) {
              const int4 off = po[q];
              const int xs = 8 * off.w + off.x;                      // window start in pencil coordinates
              const int j = ((r - xs) & (kTcRing - 1));              // x = xs + j has ring position r
              if (j < MG) {
                const float4 xv = xt[q * MGT + j];
                const float4 f = pf[q];
                const float fc = c == 0 ? f.x : (c == 1 ? f.y : f.z);
                if (!TORQUE) {
                  bv[0] = fc * fmaf(kc.B, xv.y, kc.A * xv.x);
                  bv[1] = fc * kc.B * xv.x;
                } else {
                  const float4 u = pt[q];
                  const float w = c == 0 ? kc.B * fc * xv.y
                                         : (c == 1 ? fmaf(kc.B * fc, xv.y, u.z * xv.z)
                                                   : fmaf(kc.B * fc, xv.y, -u.y * xv.z));
                  bv[0] = fmaf(fc * kc.A, xv.x, w);
                  bv[1] = fc * kc.B * xv.x;
                  bv[2] = (c == 0 ? -u.z : (c == 1 ? 0.f : u.x)) * xv.x;
                  bv[3] = (c == 0 ? u.y : (c == 1 ? -u.x : 0.f)) * xv.x;
                }
              }
            }
            const int o = kmajor_index<KS>(n, e * T);
            if (T == 4) {
              float h[4], l[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) split_tf32(bv[u], h[u], l[u]);
              *reinterpret_cast<float4*>(bh + o) = make_float4(h[0], h[1], h[2], h[3]);
              *reinterpret_cast<float4*>(bl + o) = make_float4(l[0], l[1], l[2], l[3]);
            } else {
              float h[2], l[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) split_tf32(bv[u], h[u], l[u]);
              *reinterpret_cast<float2*>(bh + o) = make_float2(h[0], h[1]);
              *reinterpret_cast<float2*>(bl + o) = make_float2(l[0], l[1]);
            }
          }
        }
        if (tid == 0) flags[b] = 1;
        // A and B are read by the tensor core; the zeroed columns by the MMAs that follow
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[b]);
        ++stage;
        q0 = q1;
      }
    }
    // end of the walk: hand the issuer an empty stage, wait for every real one, then the rest to the grid
    {
      const int b = stage & 1;
      wait_stage(stage - 2);
      if (tid == 0) flags[b] = 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[b]);
      wait_stage(stage - 1);
      tc_fence_after();
      if (!__any_sync(kFullMask32, fail))
        for (int st = flushed; st <= last_step + 2; ++st) flush_step(st, st <= last_step + 1 ? 8 : 5);
      tc_fence_before();
    }
  }
  fail = __syncthreads_or(fail || flags[2]);
  tc_fence_after();
  if (fail && tid == 0) atomicOr(status, kStatusWaitTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

template <int MGT, bool TORQUE>
void tc_variant(const Geometry<float>& g, const KernelConsts<float>& kc, const BinBuffers& b, float* grid,
                cudaStream_t s) {
  using S = TcShape<MGT, TORQUE>;
  const int nsys = g.nsys > 1 ? g.nsys : 1;
  const int blocks = nsys * g.ntile[1] * g.ntile[2];
  const int threads = 32 * (S::NPW + 1);   // producer warps + the issuer warp
  auto k = spread_pencil_tc_kernel<MGT, TORQUE>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  k<<<blocks, threads, S::SMEM, s>>>(g, kc, (const float4*)b.t_pos, (const float4*)b.t_F,
                                        (const float4*)b.t_T, b.tile_start, grid, b.status);
}

}  // namespace

bool spread_tc_eligible(const int tile[3], int MG, bool same_width) {
  return same_width && tile[0] == 8 && tile[1] == 8 && tile[2] == 8 && (MG == 10 || MG == 12 || MG == 14);
}

void launch_spread_tc(const Geometry<float>& g, const KernelConsts<float>& kc, bool torque, const BinBuffers& b,
                      float* grid, cudaStream_t s) {
#define TC_CALL(MGT)                                             \
  if (torque) tc_variant<MGT, true>(g, kc, b, grid, s);         \
  else tc_variant<MGT, false>(g, kc, b, grid, s);
  switch (g.MG) {
    case 10: TC_CALL(10) break;
    case 12: TC_CALL(12) break;
    default: TC_CALL(14) break;
  }
#undef TC_CALL
}

}  // namespace fcm
