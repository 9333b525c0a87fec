// Inverse Stokes operator in Fourier space (Section 2.1, step 2 (b)):
//   u_k = (I - k k^T / k^2) f_k / (eta k^2),
// applied in place to the three R2C spectra (layout [c][z][y][x], x halved to
// M_x/2 + 1) of each system of a launch (blockIdx.y). The factor 1/M of the
// unnormalised inverse FFT is folded in. The k = 0 mode and every mode with an
// index on a Nyquist plane (M_i/2 of an even M_i) are set to zero. One thread
// per complex mode, 3 x 2 loads and stores. The square-root variant, with the
// same zero modes, turns white grid noise into a velocity field whose covariance
// is the operator itself (Brownian increments).
#include <cuComplex.h>
#include <cmath>
#include "fcm_internal.cuh"

namespace fcm {

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 T; };
template <> struct Cplx<double> { typedef double2 T; };

template <typename R>
__device__ inline R wavenumber(int i, int M, R twopi_over_L) {
  int s = (i <= M / 2) ? i : i - M;
  return R(s) * twopi_over_L;
}

// SQRT: the square root of the operator instead, (I - k k^T / k^2) / |k| (the projector is
// idempotent), for grid noise in Brownian increments.
template <typename R, bool SQRT>
__global__ void __launch_bounds__(256) project_kernel(Geometry<R> g, R scale, typename Cplx<R>::T* spec,
                                                      size_t ncplx) {
  typedef typename Cplx<R>::T C2;
  size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= ncplx) return;
  spec += (size_t)blockIdx.y * 3 * ncplx;   // system blockIdx.y of a batched launch
  const int Mh = g.M[0] / 2 + 1;
  int ix = (int)(idx % Mh);
  size_t rest = idx / Mh;
  int iy = (int)(rest % g.M[1]);
  int iz = (int)(rest / g.M[1]);
  C2* f0 = spec + idx;
  C2* f1 = f0 + ncplx;
  C2* f2 = f1 + ncplx;
  bool nyq = ((g.M[0] & 1) == 0 && ix == g.M[0] / 2) || ((g.M[1] & 1) == 0 && iy == g.M[1] / 2) ||
             ((g.M[2] & 1) == 0 && iz == g.M[2] / 2);
  const R twopi = R(2.0 * kPi);
  R kx = R(ix) * (twopi / g.L[0]);
  R ky = wavenumber(iy, g.M[1], twopi / g.L[1]);
  R kz = wavenumber(iz, g.M[2], twopi / g.L[2]);
  R k2 = kx * kx + ky * ky + kz * kz;
  C2 a = *f0, b = *f1, c = *f2;
  if (nyq || k2 == R(0)) {
    C2 z; z.x = R(0); z.y = R(0);
    *f0 = z; *f1 = z; *f2 = z;
    return;
  }
  R ik2 = R(1) / k2;
  R dre = (kx * a.x + ky * b.x + kz * c.x) * ik2;
  R dim = (kx * a.y + ky * b.y + kz * c.y) * ik2;
  R sc = SQRT ? scale / sqrt(k2) : scale * ik2;
  a.x = (a.x - kx * dre) * sc; a.y = (a.y - kx * dim) * sc;
  b.x = (b.x - ky * dre) * sc; b.y = (b.y - ky * dim) * sc;
  c.x = (c.x - kz * dre) * sc; c.y = (c.y - kz * dim) * sc;
  *f0 = a; *f1 = b; *f2 = c;
}

template <typename R>
void launch_projection(const Geometry<R>& g, R eta, void* spectrum, cudaStream_t s, long long* launches) {
  size_t ncplx = (size_t)(g.M[0] / 2 + 1) * g.M[1] * g.M[2];
  double mtot = (double)g.M[0] * g.M[1] * g.M[2];
  R scale = R(1.0 / ((double)eta * mtot));
  unsigned blocks = (unsigned)((ncplx + 255) / 256);
  const unsigned nsys = g.nsys > 1 ? (unsigned)g.nsys : 1u;
  project_kernel<R, false><<<dim3(blocks, nsys), 256, 0, s>>>(g, scale, (typename Cplx<R>::T*)spectrum, ncplx);
  *launches += 1;
}

template <typename R>
void launch_projection_sqrt(const Geometry<R>& g, R eta, R factor, void* spectrum, cudaStream_t s,
                            long long* launches) {
  size_t ncplx = (size_t)(g.M[0] / 2 + 1) * g.M[1] * g.M[2];
  double mtot = (double)g.M[0] * g.M[1] * g.M[2];
  R scale = R((double)factor / (std::sqrt((double)eta) * mtot));
  unsigned blocks = (unsigned)((ncplx + 255) / 256);
  project_kernel<R, true><<<dim3(blocks, 1), 256, 0, s>>>(g, scale, (typename Cplx<R>::T*)spectrum, ncplx);
  *launches += 1;
}

template void launch_projection_sqrt<float>(const Geometry<float>&, float, float, void*, cudaStream_t, long long*);
template void launch_projection_sqrt<double>(const Geometry<double>&, double, double, void*, cudaStream_t,
                                             long long*);

template void launch_projection<float>(const Geometry<float>&, float, void*, cudaStream_t, long long*);
template void launch_projection<double>(const Geometry<double>&, double, void*, cudaStream_t, long long*);

}  // namespace fcm
