// Kernels of the rigid-body mobility solve (rod suspensions, Section 6.1).
//
// Body b owns particles body_off[b] .. body_off[b+1]-1. The unknowns are
// x = (F, W/mu) (3n + 6 n_bodies values, W rows (U_b, Gamma_b)); the residual is
// R = ((V - K W)/mu, K^T F - ft) with V = M^VF F and (K W)_i = U_b + Gamma_b x r_i.
// Broyden's method starts from the Jacobian of the diagonal mobility mu I,
// J0 = [[I, -K], [K^T, 0]], whose inverse acts body by body:
//     W = (K^T K)^-1 (r2 - K^T r1),  F = r1 + K W.
// One warp per body computes the residual, its norm and -J0^-1 R in one pass; the
// Broyden update itself is a Gram-matrix expansion of the product form
// H_k = prod_j (I + s_{j+1} s_j^T / |s_j|^2) H0: per iteration one multi-dot
// (z0 . s_j for every stored step), one warp of scalar recursion for the
// coefficients, one multi-axpy writing the next step (and x += step), and one
// multi-dot for the new row of the Gram matrix s_i . s_j.
#include "fcm_internal.cuh"

namespace fcm {

namespace {

constexpr int kBodyWarps = 8;   // bodies per 256-thread block
constexpr int kCoefSmemMax = 45 * 1024;   // Gram triangle staged up to this size (with the static 2 KB, under 48 KB)

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum (blockDim.x == 256) of one value per thread, added atomically to *out by thread 0.
__device__ inline void block_atomic_add(double v, double* out) {
  __shared__ double part[8];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t);
  }
}

// Lever arms r_i = Y_i - X_b (minimum image, FP64) and (K^T K)^-1 of every body, one warp per body:
// K^T K = [[n I, -[S]x], [[S]x, sum(|r|^2 I - r r^T)]] with S = sum r. Every lane factors the 6 x 6
// matrix (Cholesky, FP64, registers); lanes 0..5 then solve for one column each. A pivot below
// 1e-10 of its diagonal entry marks the body singular (fewer than 3 particles off one line).
// flags[0] <- 1 + first body with invalid offsets, flags[1] <- 1 + a singular body, flags[3] <- the
// largest body's particle count.
template <typename R>
__global__ void __launch_bounds__(256) rigid_setup_kernel(const R* __restrict__ pos, const int* __restrict__ body_off,
                                                          const R* __restrict__ X, int n, int nb, double Lx,
                                                          double Ly, double Lz, R* __restrict__ arm,
                                                          R* __restrict__ ginv, int* flags) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * kBodyWarps + (threadIdx.x >> 5);
  if (b >= nb) return;   // whole warps leave together
  const int o0 = body_off[b], o1 = body_off[b + 1];
  if (o0 < 0 || o1 > n || o1 <= o0 || (b == 0 && o0 != 0) || (b == nb - 1 && o1 != n)) {
    if (lane == 0) atomicCAS(&flags[0], 0, b + 1);
    return;
  }
  if (lane == 0) atomicMax(&flags[3], o1 - o0);   // largest body (the body preconditioner's limit)
  const double xb = (double)X[3 * (size_t)b], yb = (double)X[3 * (size_t)b + 1], zb = (double)X[3 * (size_t)b + 2];
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // Sx Sy Sz, then xx yy zz xy xz yz
  for (int i = o0 + lane; i < o1; i += 32) {
    double rx = (double)pos[3 * (size_t)i] - xb;
    double ry = (double)pos[3 * (size_t)i + 1] - yb;
    double rz = (double)pos[3 * (size_t)i + 2] - zb;
    rx -= Lx * rint(rx / Lx);
    ry -= Ly * rint(ry / Ly);
    rz -= Lz * rint(rz / Lz);
    arm[3 * (size_t)i] = (R)rx;
    arm[3 * (size_t)i + 1] = (R)ry;
    arm[3 * (size_t)i + 2] = (R)rz;
    // the sums use the stored (rounded) arms, which every later kernel reads
    rx = (double)(R)rx; ry = (double)(R)ry; rz = (double)(R)rz;
    s[0] += rx; s[1] += ry; s[2] += rz;
    s[3] += rx * rx; s[4] += ry * ry; s[5] += rz * rz;
    s[6] += rx * ry; s[7] += rx * rz; s[8] += ry * rz;
  }
  if (ginv == nullptr) return;   // the body preconditioner does not use (K^T K)^-1
#pragma unroll
  for (int k = 0; k < 9; ++k) s[k] = warp_sum(s[k]);
  const double cnt = (double)(o1 - o0), tr = s[3] + s[4] + s[5];
  const double Sx = s[0], Sy = s[1], Sz = s[2];
  // G row-major; top right -[S]x, bottom left [S]x, [S]x = [[0, -Sz, Sy], [Sz, 0, -Sx], [-Sy, Sx, 0]]
  const double G[36] = {cnt, 0.0, 0.0, 0.0,  Sz,  -Sy,
                        0.0, cnt, 0.0, -Sz, 0.0,  Sx,
                        0.0, 0.0, cnt,  Sy, -Sx, 0.0,
                        0.0, -Sz,  Sy, tr - s[3], -s[6], -s[7],
                         Sz, 0.0, -Sx, -s[6], tr - s[4], -s[8],
                        -Sy,  Sx, 0.0, -s[7], -s[8], tr - s[5]};
  double Lc[6][6];
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double dgl = G[j * 6 + j];
#pragma unroll
    for (int k = 0; k < j; ++k) dgl -= Lc[j][k] * Lc[j][k];
    ok = ok && (dgl > 1e-10 * G[j * 6 + j]);
    Lc[j][j] = sqrt(fmax(dgl, 1e-300));
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      double v = G[i * 6 + j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= Lc[i][k] * Lc[j][k];
      Lc[i][j] = v / Lc[j][j];
    }
  }
  if (!ok) {
    if (lane == 0) atomicCAS(&flags[1], 0, b + 1);
    for (int k = lane; k < 36; k += 32) ginv[36 * (size_t)b + k] = R(0);
    return;
  }
  if (lane < 6) {   // column c = lane of G^-1: L y = e_c, then L^T x = y
    double y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double v = (i == lane) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < i; ++k) v -= Lc[i][k] * y[k];
      y[i] = v / Lc[i][i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
      double v = y[i];
#pragma unroll
      for (int k = i + 1; k < 6; ++k) v -= Lc[k][i] * y[k];
      y[i] = v / Lc[i][i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) ginv[36 * (size_t)b + i * 6 + lane] = (R)y[i];
  }
}

// One warp per body, in the handle's precision R: R1_i = V_i / mu - (W^_U + W^_G x r_i),
// R2 = (sum F - f, sum r x F - tau), ||R||^2 added to *norm2 (FP64 across warps), and z = -J0^-1 R
// written for the body's particles and its 6 values.
template <typename R>
__global__ void __launch_bounds__(256) rigid_residual_kernel(const R* __restrict__ V, const R* __restrict__ x,
                                                             const R* __restrict__ ft, const R* __restrict__ arm,
                                                             const R* __restrict__ ginv,
                                                             const int* __restrict__ body_off, int n, int nb,
                                                             R inv_mu, R* __restrict__ z,
                                                             double* __restrict__ norm2) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * kBodyWarps + (threadIdx.x >> 5);
  double nr = 0.0;
  if (b < nb) {
    const int o0 = body_off[b], o1 = body_off[b + 1];
    const R* wh = x + 3 * (size_t)n + 6 * (size_t)b;
    R w[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = wh[k];
    R acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = R(0);
    for (int i = o0 + lane; i < o1; i += 32) {
      const size_t q = 3 * (size_t)i;
      const R rx = arm[q], ry = arm[q + 1], rz = arm[q + 2];
      const R e0 = V[q] * inv_mu - (w[0] + (w[4] * rz - w[5] * ry));
      const R e1 = V[q + 1] * inv_mu - (w[1] + (w[5] * rx - w[3] * rz));
      const R e2 = V[q + 2] * inv_mu - (w[2] + (w[3] * ry - w[4] * rx));
      const R f0 = x[q], f1 = x[q + 1], f2 = x[q + 2];
      acc[0] += e0; acc[1] += e1; acc[2] += e2;
      acc[3] += ry * e2 - rz * e1; acc[4] += rz * e0 - rx * e2; acc[5] += rx * e1 - ry * e0;
      acc[6] += f0; acc[7] += f1; acc[8] += f2;
      acc[9] += ry * f2 - rz * f1; acc[10] += rz * f0 - rx * f2; acc[11] += rx * f1 - ry * f0;
      acc[12] += e0 * e0 + e1 * e1 + e2 * e2;
    }
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = warp_sum(acc[k]);
    R r2[6], g[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      r2[k] = acc[6 + k] - ft[6 * (size_t)b + k];
      g[k] = r2[k] - acc[k];               // r2 - K^T r1
    }
    // y = (K^T K)^-1 g: lane i < 6 forms row i, then every lane takes the six values
    R yi = R(0);
    if (lane < 6) {
      const R* gi = ginv + 36 * (size_t)b + 6 * lane;
#pragma unroll
      for (int k = 0; k < 6; ++k) yi += gi[k] * g[k];
    }
    R y[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = __shfl_sync(0xffffffffu, yi, k);
    if (lane < 6) z[3 * (size_t)n + 6 * (size_t)b + lane] = -yi;
    if (lane == 0) {
      R t = acc[12];
#pragma unroll
      for (int k = 0; k < 6; ++k) t += r2[k] * r2[k];
      nr = (double)t;
    }
    for (int i = o0 + lane; i < o1; i += 32) {
      const size_t q = 3 * (size_t)i;
      const R rx = arm[q], ry = arm[q + 1], rz = arm[q + 2];
      const R e0 = V[q] * inv_mu - (w[0] + (w[4] * rz - w[5] * ry));
      const R e1 = V[q + 1] * inv_mu - (w[1] + (w[5] * rx - w[3] * rz));
      const R e2 = V[q + 2] * inv_mu - (w[2] + (w[3] * ry - w[4] * rx));
      z[q] = -(e0 + y[0] + (y[4] * rz - y[5] * ry));
      z[q + 1] = -(e1 + y[1] + (y[5] * rx - y[3] * rz));
      z[q + 2] = -(e2 + y[2] + (y[3] * ry - y[4] * rx));
    }
  }
  block_atomic_add(nr, norm2);
}

// ---------------------------------------------------------------- body preconditioner
//
// J0 with each body's own free-space FCM mobility (not the paper's choice, which is mu I): per body b
// with k particles the (3k + 6) x (3k + 6) matrix
//     A_b = [[M_bb / mu, -K_b], [K_b^T, 0]],
// M_bb's blocks the FCM pair mobility S(x; sigma sqrt 2) = A(r) I + B(r) x^ x^ of the minimum-image
// separation (from the Gaussian-regularised Stokeslet terms S1, S2, S3 of Section 2.2) and 1/(6 pi
// eta a) I on the diagonal. One CTA per body builds A_b in shared memory (entries in FP64, stored in
// R) and inverts it in place by Gauss-Jordan elimination (no row exchanges needed, see below); the inverse is
// written transposed (column j of A_b^-1 contiguous), stride ms x ms per body, for the residual
// kernel's coalesced matrix-vector product. flags[1] <- 1 + a body whose pivot vanished.

// S(x; sigma sqrt 2) = A I + B x x^T for r > 0, in the arithmetic type T. c8 = 1/(8 pi eta),
// s2 = 2 sigma^2, dn = (2 pi s2)^(-3/2) (the Gaussian's normalisation), e2 = 1/(2 s2), inv2sg = 1/(2 sigma).
template <typename T>
__device__ inline void fcm_pair_vf(T dx, T dy, T dz, T c8, T s2, T dn, T e2, T inv2sg, T eta, T* A, T* B) {
  const T r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
  const T E = erf(r * inv2sg);
  const T D = dn * exp(-r2 * e2);
  const T t1 = c8 * E / r, t2 = c8 * s2 * E / (r2 * r), t3 = (s2 * s2 / (T(2) * eta * r2)) * D;
  *A = t1 + t2 - t3;
  *B = (t1 - T(3) * t2 + T(3) * t3) / r2;
}

template <typename R>
__global__ void __launch_bounds__(256) body_precond_kernel(const R* __restrict__ arm, const int* __restrict__ body_off,
                                                           int nb, double Lx, double Ly, double Lz, double a,
                                                           double eta, int ms, R* __restrict__ aT, int* flags) {
  extern __shared__ unsigned char smraw[];
  const int b = blockIdx.x;
  if (b >= nb) return;
  const int o0 = body_off[b], o1 = body_off[b + 1];
  const int k = o1 - o0, m = 3 * k + 6, w2 = m;
  R* aug = reinterpret_cast<R*>(smraw);            // m x m, inverted in place
  R* fac = aug + (size_t)m * w2;                    // m factors of the current column
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  // A_b: the K blocks and zeros element by element, then the mobility blocks pair by
  // pair (one closed form per pair, in the handle's precision)
  for (int e = threadIdx.x; e < m * w2; e += blockDim.x) {
    const int r = e / w2, c = e - r * w2;
    R v = R(0);
    if (r < 3 * k && c >= 3 * k) {   // -K_i: [-I, [r_i]x], [r]x = [[0, -rz, ry], [rz, 0, -rx], [-ry, rx, 0]]
      const int i = r / 3, p = r - 3 * i, q = c - 3 * k;
      const size_t ai = 3 * (size_t)(o0 + i);
      const R rx = arm[ai], ry = arm[ai + 1], rz = arm[ai + 2];
      if (q < 3) v = (p == q) ? R(-1) : R(0);
      else {
        const int t = q - 3;
        v = p == 0 ? (t == 1 ? -rz : (t == 2 ? ry : R(0)))
                   : (p == 1 ? (t == 0 ? rz : (t == 2 ? -rx : R(0))) : (t == 0 ? -ry : (t == 1 ? rx : R(0))));
      }
    } else if (r >= 3 * k && c < 3 * k) {   // K^T: (K^T)_{r', (j, q)} = K_{(j, q), r'}, K_j = [I, -[r_j]x]
      const int rp = r - 3 * k, j = c / 3, q = c - 3 * j;
      const size_t aj = 3 * (size_t)(o0 + j);
      const R rx = arm[aj], ry = arm[aj + 1], rz = arm[aj + 2];
      if (rp < 3) v = (q == rp) ? R(1) : R(0);
      else {
        const int t = rp - 3;
        const R cxqt = q == 0 ? (t == 1 ? -rz : (t == 2 ? ry : R(0)))
                              : (q == 1 ? (t == 0 ? rz : (t == 2 ? -rx : R(0))) : (t == 0 ? -ry : (t == 1 ? rx : R(0))));
        v = -cxqt;
      }
    }
    aug[e] = v;   // the mobility blocks are written below
  }
  __syncthreads();
  {
    const R sg = (R)(a / sqrt(kPi));
    const R s2 = R(2) * sg * sg;
    const R c8 = (R)(1.0 / (8.0 * kPi * eta));
    const R dn = (R)pow(2.0 * kPi * 2.0 * (a * a / kPi), -1.5);
    const R e2 = R(1) / (R(2) * s2);
    const R inv2sg = R(1) / (R(2) * sg);
    const R inv_mu = (R)(6.0 * kPi * eta * a);
    for (int pq = threadIdx.x; pq < k * k; pq += blockDim.x) {
      const int i = pq / k, j = pq - i * k;
      R blk[9];
      if (i == j) {   // (1/(6 pi eta a)) I / mu
#pragma unroll
        for (int t = 0; t < 9; ++t) blk[t] = (t % 4 == 0) ? R(1) : R(0);
      } else {
        const size_t ai = 3 * (size_t)(o0 + i), aj = 3 * (size_t)(o0 + j);
        R d0 = arm[ai] - arm[aj], d1 = arm[ai + 1] - arm[aj + 1], d2 = arm[ai + 2] - arm[aj + 2];
        d0 -= (R)Lx * rint(d0 / (R)Lx);
        d1 -= (R)Ly * rint(d1 / (R)Ly);
        d2 -= (R)Lz * rint(d2 / (R)Lz);
        R A, B;
        fcm_pair_vf<R>(d0, d1, d2, c8, s2, dn, e2, inv2sg, (R)eta, &A, &B);
        const R d[3] = {d0, d1, d2};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < 3; ++q) blk[3 * p + q] = ((p == q ? A : R(0)) + B * d[p] * d[q]) * inv_mu;
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) aug[(size_t)(3 * i + p) * w2 + 3 * j + q] = blk[3 * p + q];
    }
  }
  __syncthreads();
  // Gauss-Jordan without row exchanges: M_bb / mu is symmetric positive definite, so the first 3k
  // pivots are positive, and the last 6 are those of the Schur complement -K^T (M_bb / mu)^-1 K,
  // negative definite when K has full column rank (3 particles off one line); a vanishing pivot
  // flags the body.
  const R tiny = sizeof(R) == 4 ? R(1e-6) : R(1e-12);
  for (int col = 0; col < m; ++col) {   // in-place Gauss-Jordan: after step col, column col holds A^-1's
    const R pv = aug[(size_t)col * w2 + col];
    if (!(fabs((double)pv) > (double)tiny)) {
      if (threadIdx.x == 0) bad = 1;
      break;   // every thread reads the same pivot, so all leave together
    }
    const R inv_p = R(1) / pv;
    __syncthreads();   // everyone has read the pivot before row col changes
    for (int c = threadIdx.x; c < w2; c += blockDim.x)
      aug[(size_t)col * w2 + c] = (c == col ? R(1) : aug[(size_t)col * w2 + c]) * inv_p;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {   // the factors; column col of the other rows set to 0,
      if (r == col) { fac[r] = R(0); continue; }           // so that the update below is the same everywhere
      fac[r] = aug[(size_t)r * w2 + col];
      aug[(size_t)r * w2 + col] = R(0);
    }
    __syncthreads();
    {   // warps over rows, lanes over columns (at most 4 per lane: m <= 3 kRigidBodyMax + 6 = 102 < 128)
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      const R* rowc = aug + (size_t)col * w2;
      R cv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) cv[t] = (lane + 32 * t < w2) ? rowc[lane + 32 * t] : R(0);
      for (int r = wid; r < m; r += nw) {
        const R f = fac[r];
        if (f == R(0)) continue;
        R* rowr = aug + (size_t)r * w2;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (lane + 32 * t < w2) rowr[lane + 32 * t] -= f * cv[t];
      }
    }
    __syncthreads();
  }
  __syncthreads();
  R* out = aT + (size_t)b * ms * ms;
  if (bad) {
    if (threadIdx.x == 0) atomicCAS(&flags[1], 0, b + 1);
    for (int e = threadIdx.x; e < ms * ms; e += blockDim.x) out[e] = R(0);
    return;
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {   // out[j][i] = (A^-1)[i][j]
    const int j = e / m, i = e - j * m;
    out[(size_t)j * ms + i] = aug[(size_t)i * w2 + j];
  }
}

// The residual kernel with the body preconditioner: R1 and R2 of the body go to a per-warp vector
// v (3k + 6 values, up to kRigidBodyMax particles), then z = -A_b^-1 v with lanes over rows.
template <typename R>
__global__ void __launch_bounds__(256) rigid_residual_body_kernel(const R* __restrict__ V, const R* __restrict__ x,
                                                                  const R* __restrict__ ft, const R* __restrict__ arm,
                                                                  const R* __restrict__ aT, int ms,
                                                                  const int* __restrict__ body_off, int n, int nb,
                                                                  R inv_mu, R* __restrict__ z,
                                                                  double* __restrict__ norm2) {
  __shared__ R vbuf[kBodyWarps][3 * kRigidBodyMax + 6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int b = blockIdx.x * kBodyWarps + wid;
  double nr = 0.0;
  if (b < nb) {
    const int o0 = body_off[b], o1 = body_off[b + 1];
    const int k = o1 - o0, m = 3 * k + 6;
    R* v = vbuf[wid];
    const R* wh = x + 3 * (size_t)n + 6 * (size_t)b;
    R w[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) w[t] = wh[t];
    R acc[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) acc[t] = R(0);
    for (int i = o0 + lane; i < o1; i += 32) {
      const size_t q = 3 * (size_t)i;
      const R rx = arm[q], ry = arm[q + 1], rz = arm[q + 2];
      const R e0 = V[q] * inv_mu - (w[0] + (w[4] * rz - w[5] * ry));
      const R e1 = V[q + 1] * inv_mu - (w[1] + (w[5] * rx - w[3] * rz));
      const R e2 = V[q + 2] * inv_mu - (w[2] + (w[3] * ry - w[4] * rx));
      const R f0 = x[q], f1 = x[q + 1], f2 = x[q + 2];
      v[3 * (i - o0)] = e0;
      v[3 * (i - o0) + 1] = e1;
      v[3 * (i - o0) + 2] = e2;
      acc[0] += f0; acc[1] += f1; acc[2] += f2;
      acc[3] += ry * f2 - rz * f1; acc[4] += rz * f0 - rx * f2; acc[5] += rx * f1 - ry * f0;
      acc[6] += e0 * e0 + e1 * e1 + e2 * e2;
    }
#pragma unroll
    for (int t = 0; t < 7; ++t) acc[t] = warp_sum(acc[t]);
    if (lane < 6) v[3 * k + lane] = acc[lane] - ft[6 * (size_t)b + lane];   // R2
    if (lane == 0) {
      R t = acc[6];
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const R r2 = acc[u] - ft[6 * (size_t)b + u];
        t += r2 * r2;
      }
      nr = (double)t;
    }
    __syncwarp();
    const R* A = aT + (size_t)b * ms * ms;
    for (int i = lane; i < m; i += 32) {
      R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);   // four independent chains: loads in flight
      int j = 0;
      for (; j + 3 < m; j += 4) {
        s0 += A[(size_t)j * ms + i] * v[j];
        s1 += A[(size_t)(j + 1) * ms + i] * v[j + 1];
        s2 += A[(size_t)(j + 2) * ms + i] * v[j + 2];
        s3 += A[(size_t)(j + 3) * ms + i] * v[j + 3];
      }
      for (; j < m; ++j) s0 += A[(size_t)j * ms + i] * v[j];
      const R sum = (s0 + s1) + (s2 + s3);
      if (i < 3 * k) z[3 * (size_t)o0 + i] = -sum;
      else z[3 * (size_t)n + 6 * (size_t)b + (i - 3 * k)] = -sum;
    }
  }
  block_atomic_add(nr, norm2);
}

// out[j] += a . S_j for the k vectors S_j = S + j * stride (blockIdx.y = j); each thread sums its
// elements in R with four independent partial sums, blocks combine in FP64.
template <typename R>
__global__ void __launch_bounds__(256) multi_dot_kernel(const R* __restrict__ a, const R* __restrict__ S, size_t m,
                                                        size_t stride, double* __restrict__ out) {
  const R* sj = S + (size_t)blockIdx.y * stride;
  const size_t step = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  R v0 = R(0), v1 = R(0), v2 = R(0), v3 = R(0);
  for (; e + 3 * step < m; e += 4 * step) {
    v0 += a[e] * sj[e];
    v1 += a[e + step] * sj[e + step];
    v2 += a[e + 2 * step] * sj[e + 2 * step];
    v3 += a[e + 3 * step] * sj[e + 3 * step];
  }
  for (; e < m; e += step) v0 += a[e] * sj[e];
  block_atomic_add((double)((v0 + v1) + (v2 + v3)), out + blockIdx.y);
}

// Coefficients of the next step from d_j = s_j . z0 (j <= n) and the Gram rows G[j][i] = s_j . s_i
// (i <= j, row stride ld): with z_j = z0 + sum_{i<j} c_i s_{i+1},
//     c_j = s_j . z_j / |s_j|^2 = (d_j + sum_{i<j} c_i G[j][i+1]) / G[j][j]       (j < n)
//     s_{n+1} = z_n / (1 - s_n . z_n / |s_n|^2)
// coef[0] multiplies z0 and coef[1 + j] multiplies s_{j+1}. One warp; the lower triangle of G
// (rows 0..n) and d are first copied to shared memory with independent loads when they fit in the
// default 48 KB (gsm), so the sequential recursion reads shared memory. flags[2] <- 1 on breakdown.
__global__ void __launch_bounds__(32) broyden_coef_kernel(const double* __restrict__ d, const double* __restrict__ G,
                                                          int ld, int n, double* __restrict__ coef, int* flags,
                                                          int gsm) {
  extern __shared__ double blk[];   // triangle rows 0..n (row j: j + 1 values from offset j(j+1)/2), then d
  __shared__ double c[kBroydenMax + 1];
  const int lane = threadIdx.x;
  const int tot = (n + 1) * (n + 2) / 2;
  double* dsm = blk + tot;
  if (gsm) {
    for (int e = lane; e < tot; e += 32) {
      int j = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);   // row of triangle entry e, then exact
      while (j * (j + 1) / 2 > e) --j;
      while ((j + 1) * (j + 2) / 2 <= e) ++j;
      blk[e] = G[(size_t)j * ld + (e - j * (j + 1) / 2)];
    }
    for (int j = lane; j <= n; j += 32) dsm[j] = d[j];
    __syncwarp();
  }
  const double* dr = gsm ? dsm : d;
  double denom = 1.0;
  for (int j = 0; j <= n; ++j) {
    const double* row = gsm ? blk + (size_t)j * (j + 1) / 2 : G + (size_t)j * ld;
    double t = 0.0;
    for (int i = lane; i < j; i += 32) t += c[i] * row[i + 1];
    t = warp_sum(t) + dr[j];
    const double gjj = row[j];
    if (j < n) {
      if (lane == 0) c[j] = t / gjj;
      __syncwarp();
    } else {
      denom = 1.0 - t / gjj;
    }
  }
  const bool ok = fabs(denom) > 1e-12 && isfinite(denom);
  if (!ok && lane == 0) atomicCAS(&flags[2], 0, 1);
  const double inv = ok ? 1.0 / denom : 0.0;
  if (lane == 0) coef[0] = inv;
  for (int j = lane; j < n; j += 32) coef[1 + j] = c[j] * inv;
}

// s_out = coef[0] z + sum_{j<n} coef[1+j] s_{j+1}, and x += s_out (arithmetic in R).
template <typename R>
__global__ void __launch_bounds__(256) broyden_step_kernel(const R* __restrict__ z, const R* __restrict__ S, size_t m,
                                                           size_t stride, int n, const double* __restrict__ coef,
                                                           R* __restrict__ s_out, R* __restrict__ x) {
  __shared__ R c[kBroydenMax + 1];
  for (int k = threadIdx.x; k <= n; k += blockDim.x) c[k] = (R)coef[k];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < m; e += (size_t)gridDim.x * blockDim.x) {
    R v = c[0] * z[e];
    for (int j = 0; j < n; ++j) v += c[1 + j] * S[(size_t)(j + 1) * stride + e];
    s_out[e] = v;
    x[e] = x[e] + v;
  }
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int vec_blocks(size_t m) {
  const size_t want = (m + 255) / 256;
  const size_t cap = (size_t)sm_count() * 8;
  return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

template <typename R>
void launch_rigid_setup(const R* pos, const int* body_off, const R* X, int n, int nb, const double L[3], R* arm,
                        R* ginv, int* flags, cudaStream_t s, long long* launches) {
  const int blocks = (nb + kBodyWarps - 1) / kBodyWarps;
  rigid_setup_kernel<R><<<blocks, 256, 0, s>>>(pos, body_off, X, n, nb, L[0], L[1], L[2], arm, ginv, flags);
  *launches += 1;
}

template <typename R>
void launch_rigid_residual(const R* V, const R* x, const R* ft, const R* arm, const R* ginv, const int* body_off,
                           int n, int nb, double inv_mu, R* z, double* norm2, cudaStream_t s, long long* launches) {
  const int blocks = (nb + kBodyWarps - 1) / kBodyWarps;
  rigid_residual_kernel<R><<<blocks, 256, 0, s>>>(V, x, ft, arm, ginv, body_off, n, nb, (R)inv_mu, z, norm2);
  *launches += 1;
}

template <typename R>
void launch_body_precond(const R* arm, const int* body_off, int nb, int kmax, const double L[3], double a, double eta,
                         R* aT, int* flags, cudaStream_t s, long long* launches) {
  const int m = 3 * kmax + 6;
  const size_t smem = sizeof(R) * ((size_t)m * m + m);
  cudaFuncSetAttribute(body_precond_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  body_precond_kernel<R><<<nb, 256, smem, s>>>(arm, body_off, nb, L[0], L[1], L[2], a, eta, m, aT, flags);
  *launches += 1;
}

template <typename R>
void launch_rigid_residual_body(const R* V, const R* x, const R* ft, const R* arm, const R* aT, int ms,
                                const int* body_off, int n, int nb, double inv_mu, R* z, double* norm2, cudaStream_t s,
                                long long* launches) {
  const int blocks = (nb + kBodyWarps - 1) / kBodyWarps;
  rigid_residual_body_kernel<R><<<blocks, 256, 0, s>>>(V, x, ft, arm, aT, ms, body_off, n, nb, (R)inv_mu, z, norm2);
  *launches += 1;
}

template <typename R>
void launch_multi_dot(const R* a, const R* S, size_t m, size_t stride, int k, double* out, cudaStream_t s,
                      long long* launches) {
  // about 8 blocks per SM in total, at least one per vector
  const int per = std::max(1, std::min(vec_blocks(m), (8 * sm_count() + k - 1) / k));
  multi_dot_kernel<R><<<dim3(per, k), 256, 0, s>>>(a, S, m, stride, out);
  *launches += 1;
}

void launch_broyden_coef(const double* d, const double* G, int ld, int n, double* coef, int* flags, cudaStream_t s,
                         long long* launches) {
  const size_t bytes = sizeof(double) * ((size_t)(n + 1) * (n + 2) / 2 + (size_t)(n + 1));
  const bool fits = bytes <= (size_t)kCoefSmemMax;
  broyden_coef_kernel<<<1, 32, fits ? bytes : 0, s>>>(d, G, ld, n, coef, flags, fits ? 1 : 0);
  *launches += 1;
}

template <typename R>
void launch_broyden_step(const R* z, const R* S, size_t m, size_t stride, int n, const double* coef, R* s_out, R* x,
                         cudaStream_t s, long long* launches) {
  broyden_step_kernel<R><<<vec_blocks(m), 256, 0, s>>>(z, S, m, stride, n, coef, s_out, x);
  *launches += 1;
}

#define FCM_RIGID_INSTANTIATE(R)                                                                                    \
  template void launch_rigid_setup<R>(const R*, const int*, const R*, int, int, const double[3], R*, R*, int*,      \
                                      cudaStream_t, long long*);                                                    \
  template void launch_rigid_residual<R>(const R*, const R*, const R*, const R*, const R*, const int*, int, int,    \
                                         double, R*, double*, cudaStream_t, long long*);                            \
  template void launch_multi_dot<R>(const R*, const R*, size_t, size_t, int, double*, cudaStream_t, long long*);    \
  template void launch_body_precond<R>(const R*, const int*, int, int, const double[3], double, double, R*, int*,    \
                                       cudaStream_t, long long*);                                                   \
  template void launch_rigid_residual_body<R>(const R*, const R*, const R*, const R*, const R*, int, const int*, int, \
                                              int, double, R*, double*, cudaStream_t, long long*);                  \
  template void launch_broyden_step<R>(const R*, const R*, size_t, size_t, int, const double*, R*, R*, cudaStream_t, \
                                       long long*);
FCM_RIGID_INSTANTIATE(float)
FCM_RIGID_INSTANTIATE(double)
#undef FCM_RIGID_INSTANTIATE

}  // namespace fcm
