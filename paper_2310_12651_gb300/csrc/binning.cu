// Spatial hashing, counting sort and cell lists (Section 4, steps 1-2).
//
// Two keys per particle: the spread/gather tile that holds the first point of
// its M_G^3 window, and the pair cell of Section 4 step 1 (m_i = max(int(L_i/r_c), 3)
// cells, index x_c + (y_c + z_c m_y) m_x). Counting sort by each key gives the
// tile-sorted arrays used by spread/gather and the cell-sorted arrays with
// start offsets used by the pair correction. The rank of a particle inside its
// bin is the value its atomic increment returned, so three kernels suffice:
// key+count, scan, scatter. The scan leaves the counters at zero for the next call.
// Inside a tile, particles whose window starts in the first half of the tile's x
// range come first: they count on tile_count[t], the others on tile_count[ntiles + t]
// and are placed from tile_start[ntiles + 1 + t] (the pencil spread steps half a
// tile at a time along x).
#include "fcm_internal.cuh"

namespace fcm {

// System of stacked row i: the s with sys_off[s] <= i < sys_off[s + 1] (binary search).
__device__ inline int system_of(const BinBuffers& b, int i) {
  if (b.nsys <= 1 || !b.sys_off) return 0;
  int lo = 0, hi = b.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(b.sys_off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename R>
__global__ void __launch_bounds__(256) key_count_kernel(Geometry<R> g, int n, const R* __restrict__ pos,
                                                        BinBuffers b, int need_cells) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (b.n_dev) n = min(n, *b.n_dev);
  if (i >= n) return;
  const int sys = system_of(b, i);
  int bad = 0;
  int t[3], c[3], xoff = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R y = wrap_coord(pos[3 * (size_t)i + d], g.L[d], &bad);
    int i0 = pmod(window_start_d(g, d, y), g.M[d]);
    t[d] = i0 / g.tile[d];
    if (d == 0) xoff = i0 - t[0] * g.tile[0];
    c[d] = cell_coord(y, g.cellw_inv[d], g.mcell[d]);
  }
  if (bad) atomicOr(b.status, kStatusNonFinite);
  unsigned tk = (unsigned)(t[0] + g.ntile[0] * (t[1] + g.ntile[1] * t[2]));
  if (sys) tk += (unsigned)sys * (unsigned)g.tiles_per;
  b.tile_key[i] = tk;
  const unsigned half = (g.tile[0] >= 2 && xoff >= (g.tile[0] >> 1)) ? 1u : 0u;
  const unsigned rank = (unsigned)atomicAdd(&b.tile_count[tk + (half ? (unsigned)b.ntiles : 0u)], 1);
  b.tile_rank[i] = rank | (half << 31);
  if (need_cells) {
    unsigned ck = (unsigned)(c[0] + g.mcell[0] * (c[1] + g.mcell[1] * c[2]));
    if (sys) ck += (unsigned)sys * (unsigned)g.cells_per;
    b.cell_key[i] = ck;
    b.cell_rank[i] = (unsigned)atomicAdd(&b.cell_count[ck], 1);
  }
}

// Exclusive scan of one counter array by one block, offset by base; start[nb] = base + total
// when write_end. Resets counts. With count1 (a second counter per bin, placed after the first's
// particles), bin k holds count[k] + count1[k] particles and start1[k] = start[k] + count[k].
__device__ void block_scan(int* count, int* start, int nb, int base, bool write_end, int* count1 = nullptr,
                           int* start1 = nullptr) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int chunk = (nb + nthr - 1) / nthr;
  const int lo = min(nb, tid * chunk), hi = min(nb, lo + chunk);
  int local = 0;
  for (int k = lo; k < hi; ++k) local += count[k] + (count1 ? count1[k] : 0);
  // inclusive warp scan of the per-thread sums
  int lane = tid & 31, wid = tid >> 5;
  int v = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = (nthr + 31) / 32;
    int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < nw) warp_sums[lane] = w;
    if (lane == nw - 1) carry = w;
  }
  __syncthreads();
  int excl = base + v - local + (wid > 0 ? warp_sums[wid - 1] : 0);
  for (int k = lo; k < hi; ++k) {
    const int cnt = count[k];
    start[k] = excl;
    excl += cnt;
    count[k] = 0;
    if (count1) {
      start1[k] = excl;
      excl += count1[k];
      count1[k] = 0;
    }
  }
  if (tid == 0 && write_end) start[nb] = base + carry;
}

// Block (k, s): k = 0 scans system s's tile counters, k = 1 its cell counters. A system's
// bins are contiguous and its particles are the stacked rows from sys_off[s], so each
// segment starts at sys_off[s] and the segments scan independently.
__global__ void __launch_bounds__(1024) scan_kernel(BinBuffers b, int need_cells) {
  const int sys = blockIdx.y;
  const int nsys = max(b.nsys, 1);
  const int base = (b.nsys > 1 && b.sys_off) ? b.sys_off[sys] : 0;
  const bool last = sys == nsys - 1;
  if (blockIdx.x == 0) {
    const int per = b.ntiles / nsys;
    block_scan(b.tile_count + (size_t)sys * per, b.tile_start + (size_t)sys * per, per, base, last,
               b.tile_count + (size_t)b.ntiles + (size_t)sys * per, b.tile_start + (size_t)b.ntiles + 1 + (size_t)sys * per);
  } else if (need_cells) {
    const int per = b.ncells / nsys;
    block_scan(b.cell_count + (size_t)sys * per, b.cell_start + (size_t)sys * per, per, base, last);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) scatter_kernel(Geometry<R> g, int n, const R* __restrict__ pos,
                                                      const R* __restrict__ F, const R* __restrict__ T,
                                                      BinBuffers b, int need_cells) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (b.n_dev) n = min(n, *b.n_dev);
  if (i >= n) return;
  int bad = 0;
  Vec4<R> p, f, t;
  p.x = wrap_coord(pos[3 * (size_t)i + 0], g.L[0], &bad);
  p.y = wrap_coord(pos[3 * (size_t)i + 1], g.L[1], &bad);
  p.z = wrap_coord(pos[3 * (size_t)i + 2], g.L[2], &bad);
  p.w = as_real_bits(i, R(0));
  f.x = F[3 * (size_t)i + 0]; f.y = F[3 * (size_t)i + 1]; f.z = F[3 * (size_t)i + 2]; f.w = R(0);
  if (T) { t.x = T[3 * (size_t)i + 0]; t.y = T[3 * (size_t)i + 1]; t.z = T[3 * (size_t)i + 2]; }
  else   { t.x = R(0); t.y = R(0); t.z = R(0); }
  t.w = R(0);
  // keys and ranks come from key_count_kernel; both bins are in range by construction
  const unsigned rk = b.tile_rank[i];
  int dt = b.tile_start[(rk >> 31) ? (size_t)b.ntiles + 1 + b.tile_key[i] : (size_t)b.tile_key[i]] +
           (int)(rk & 0x7fffffffu);
  dt = min(max(dt, 0), n - 1);
  ((Vec4<R>*)b.t_pos)[dt] = p;
  ((Vec4<R>*)b.t_F)[dt] = f;
  ((Vec4<R>*)b.t_T)[dt] = t;
  if (need_cells) {
    int dc = b.cell_start[b.cell_key[i]] + (int)b.cell_rank[i];
    dc = min(max(dc, 0), n - 1);
    ((Vec4<R>*)b.c_pos)[dc] = p;
    ((Vec4<R>*)b.c_F)[dc] = f;
    ((Vec4<R>*)b.c_T)[dc] = t;
  }
}

template <typename R>
void launch_binning(const Geometry<R>& g, int n, const R* pos, const R* F, const R* T,
                    const BinBuffers& b, bool need_cells, cudaStream_t s, long long* launches) {
  if (n <= 0) return;
  int blocks = (n + 255) / 256;
  key_count_kernel<R><<<blocks, 256, 0, s>>>(g, n, pos, b, need_cells ? 1 : 0);
  scan_kernel<<<dim3(2, b.nsys > 1 ? b.nsys : 1), 1024, 0, s>>>(b, need_cells ? 1 : 0);
  scatter_kernel<R><<<blocks, 256, 0, s>>>(g, n, pos, F, T, b, need_cells ? 1 : 0);
  *launches += 3;
}

template void launch_binning<float>(const Geometry<float>&, int, const float*, const float*, const float*,
                                    const BinBuffers&, bool, cudaStream_t, long long*);
template void launch_binning<double>(const Geometry<double>&, int, const double*, const double*, const double*,
                                     const BinBuffers&, bool, cudaStream_t, long long*);

__global__ void write_offsets_kernel(SysOffsets o, int n, int* dst) {
  for (int k = threadIdx.x; k <= n; k += blockDim.x) dst[k] = o.off[k];
}

void launch_write_offsets(const SysOffsets& o, int n, int* dst, cudaStream_t s, long long* launches) {
  write_offsets_kernel<<<1, 256, 0, s>>>(o, n, dst);
  *launches += 1;
}

template <typename R>
__global__ void __launch_bounds__(256) add_kernel(R* __restrict__ U, const R* __restrict__ up, R* __restrict__ W,
                                                  const R* __restrict__ wp, size_t count, const int* n_dev) {
  if (n_dev) count = min(count, 3 * (size_t)max(*n_dev, 0));
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += stride) {
    U[k] += up[k];
    if (W) W[k] += wp[k];
  }
}

template <typename R>
void launch_add(R* U, const R* up, R* W, const R* wp, size_t count, cudaStream_t s, long long* launches,
                const int* n_dev) {
  if (count == 0) return;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (count + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 8 ? want : (size_t)sms * 8);
  add_kernel<R><<<blocks, 256, 0, s>>>(U, up, W, wp, count, n_dev);
  *launches += 1;
}

template void launch_add<float>(float*, const float*, float*, const float*, size_t, cudaStream_t, long long*,
                                const int*);
template void launch_add<double>(double*, const double*, double*, const double*, size_t, cudaStream_t, long long*,
                                 const int*);

__global__ void zero_kernel(uint4* p, size_t n16, unsigned char* tail, size_t ntail) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t k = i; k < n16; k += stride) p[k] = make_uint4(0, 0, 0, 0);
  if (i < ntail) tail[i] = 0;
}

void launch_zero(void* p, size_t bytes, cudaStream_t s, long long* launches) {
  if (bytes == 0) return;
  size_t n16 = bytes / 16, ntail = bytes - n16 * 16;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t want = (n16 + 255) / 256;
  int blocks = (int)(want < (size_t)sms * 8 ? (want > 0 ? want : 1) : (size_t)sms * 8);
  zero_kernel<<<blocks, 256, 0, s>>>((uint4*)p, n16, (unsigned char*)p + n16 * 16, ntail);
  *launches += 1;
}

}  // namespace fcm
