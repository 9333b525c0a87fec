// Vector kernels of the Lanczos square root used for the pairwise part of Brownian
// increments (positive splitting, Section 3.3): dot products accumulated in FP64,
// y = alpha x + beta y, and the final combination of the Krylov basis.
#include "fcm_internal.cuh"

namespace fcm {

namespace {

int grid_blocks(size_t m) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (m + 255) / 256;
  return (int)(want < (size_t)sms * 4 ? (want > 0 ? want : 1) : (size_t)sms * 4);
}

}  // namespace

template <typename R>
__global__ void __launch_bounds__(256) dot_kernel(const R* __restrict__ a, const R* __restrict__ b, size_t m,
                                                  double* out) {
  double v = 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x)
    v += (double)a[k] * (double)b[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t);
  }
}

template <typename R>
__global__ void __launch_bounds__(256) axpby_kernel(R* __restrict__ y, double alpha, const R* __restrict__ x,
                                                    double beta, size_t m) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m; k += (size_t)gridDim.x * blockDim.x)
    y[k] = (R)(beta == 0.0 ? alpha * (double)x[k] : alpha * (double)x[k] + beta * (double)y[k]);
}

template <typename R>
__global__ void __launch_bounds__(256) combine_kernel(R* __restrict__ out, const R* __restrict__ V, LanczosCoef c,
                                                      int nk, size_t m, int accumulate) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    double v = accumulate ? (double)out[i] : 0.0;
    for (int j = 0; j < nk; ++j) v += c.c[j] * (double)V[(size_t)j * m + i];
    out[i] = (R)v;
  }
}

template <typename R>
void launch_dot(const R* a, const R* b, size_t m, double* out, cudaStream_t s, long long* launches) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  dot_kernel<R><<<grid_blocks(m), 256, 0, s>>>(a, b, m, out);
  *launches += 1;
}

template <typename R>
void launch_axpby(R* y, double alpha, const R* x, double beta, size_t m, cudaStream_t s, long long* launches) {
  axpby_kernel<R><<<grid_blocks(m), 256, 0, s>>>(y, alpha, x, beta, m);
  *launches += 1;
}

template <typename R>
void launch_combine(R* out, const R* V, const LanczosCoef& c, int k, size_t m, bool accumulate, cudaStream_t s,
                    long long* launches) {
  combine_kernel<R><<<grid_blocks(m), 256, 0, s>>>(out, V, c, k, m, accumulate ? 1 : 0);
  *launches += 1;
}

template void launch_dot<float>(const float*, const float*, size_t, double*, cudaStream_t, long long*);
template void launch_dot<double>(const double*, const double*, size_t, double*, cudaStream_t, long long*);
template void launch_axpby<float>(float*, double, const float*, double, size_t, cudaStream_t, long long*);
template void launch_axpby<double>(double*, double, const double*, double, size_t, cudaStream_t, long long*);
template void launch_combine<float>(float*, const float*, const LanczosCoef&, int, size_t, bool, cudaStream_t,
                                    long long*);
template void launch_combine<double>(double*, const double*, const LanczosCoef&, int, size_t, bool, cudaStream_t,
                                     long long*);

}  // namespace fcm
