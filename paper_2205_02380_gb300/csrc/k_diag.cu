// Phase-space diagnostics of Sec. 5, in FP64 with a fixed summation order (bitwise reproducible):
//
//   W_j(x, k)  = integral of f over the other two x and the other two k coordinates
//   P(x1, x2)  = integral of f over x3 and k
//   <x_d>, <k_d> = sum x_d f / sum f, sum k_d f / sum f   (averaged position and momentum)
//
// Stage 1 (k_diag_kpart, one launch per k-dimension d): S_d[x][q] = sum of f[x] over the two k
// indices other than k_d = q, one thread per (x point, q), the other indices in row-major order.
// Stage 2: W_j sums S_j over the other two x indices (thread per (x_j, q)); P sums S_0 over x3
// and q (thread per (x1, x2)); the averages come from one block that reduces S_0, S_1, S_2 in a
// fixed tree.  The grid factors (cell volumes, x and k node positions) are applied in FP64.
#include "internal.hpp"

namespace chasm {
namespace {

constexpr int kDiagThreads = 256;

template <typename T, int N>
__global__ void k_diag_kpart(const T* __restrict__ f, int64_t nxp, int d, double* __restrict__ S) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxp * N) return;
  const int64_t xp = t / N;
  const int q = (int)(t % N);
  const T* fx = f + xp * (N * N * N);
  double s = 0.0;
  for (int a = 0; a < N; ++a) {
#pragma unroll 8
    for (int b = 0; b < N; ++b) {
      const int off = d == 0 ? (q * N + a) * N + b : (d == 1 ? (a * N + q) * N + b : (a * N + b) * N + q);
      s += (double)fx[off];
    }
  }
  S[t] = s;
}

// Single precision: each row of N elements is summed in compensated FP32 (two-sum) and added to
// the FP64 total (the FP64 pipe runs at 1/64 of the FP32 rate here); rows along k3 read 16 bytes
// at a time.
template <int N>
__global__ void k_diag_kpart_f(const float* __restrict__ f, int64_t nxp, int d, double* __restrict__ S) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxp * N) return;
  const int64_t xp = t / N;
  const int q = (int)(t % N);
  const float* fx = f + xp * (N * N * N);
  double s = 0.0;
  for (int a = 0; a < N; ++a) {
    float hi = 0.f, lo = 0.f;
    if (d == 2) {
#pragma unroll 8
      for (int b = 0; b < N; ++b) two_sum_f(hi, lo, fx[(a * N + b) * N + q]);
    } else {
      const float4* row = reinterpret_cast<const float4*>(fx + (d == 0 ? (q * N + a) * N : (a * N + q) * N));
#pragma unroll
      for (int b4 = 0; b4 < N / 4; ++b4) {
        const float4 v = row[b4];
        two_sum_f(hi, lo, v.x);
        two_sum_f(hi, lo, v.y);
        two_sum_f(hi, lo, v.z);
        two_sum_f(hi, lo, v.w);
      }
    }
    s += (double)hi + (double)lo;
  }
  S[t] = s;
}

// W_j[i][q] = vol * sum over the other two x indices (ascending) of S_j[x][q]
__global__ void k_diag_wigner(const double* __restrict__ S, int j, int nx0, int nx1, int nx2, int N,
                              double vol, double* __restrict__ W) {
  const int nx[3] = {nx0, nx1, nx2};
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx[j] * N) return;
  const int i = t / N, q = t % N;
  const int oa = j == 0 ? 1 : 0, ob = j == 2 ? 1 : 2;
  double s = 0.0;
  for (int a = 0; a < nx[oa]; ++a)
    for (int b = 0; b < nx[ob]; ++b) {
      int ix[3];
      ix[j] = i;
      ix[oa] = a;
      ix[ob] = b;
      const int64_t xp = ((int64_t)ix[0] * nx1 + ix[1]) * nx2 + ix[2];
      s += S[xp * N + q];
    }
  W[t] = s * vol;
}

// P[i1][i2] = vol * sum over i3 and q of S_0[x][q]
__global__ void k_diag_marginal(const double* __restrict__ S0, int nx0, int nx1, int nx2, int N,
                                double vol, double* __restrict__ P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx0 * nx1) return;
  double s = 0.0;
  for (int i3 = 0; i3 < nx2; ++i3) {
    const double* r = S0 + ((int64_t)t * nx2 + i3) * N;
    for (int q = 0; q < N; ++q) s += r[q];
  }
  P[t] = s * vol;
}

// One block: m = sum S_0, x_d = sum_x x_d sum_q S_0, k_d = sum_x sum_q k_q S_d; out = (x, k) / m
__global__ void __launch_bounds__(kDiagThreads) k_diag_expect(const double* __restrict__ S, int64_t nxp,
                                                              int nx1, int nx2, int N, double3 xlo,
                                                              double3 h, double dk,
                                                              double* __restrict__ out) {
  __shared__ double red[7][kDiagThreads];
  const int tid = threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t xp = tid; xp < nxp; xp += kDiagThreads) {
    const int i3 = (int)(xp % nx2), i2 = (int)((xp / nx2) % nx1), i1 = (int)(xp / ((int64_t)nx1 * nx2));
    double m = 0.0, k[3] = {0, 0, 0};
    for (int q = 0; q < N; ++q) {
      const double kq = (q - N / 2) * dk;
      m += S[xp * N + q];
      for (int d = 0; d < 3; ++d) k[d] += kq * S[((int64_t)d * nxp + xp) * N + q];
    }
    acc[0] += m;
    acc[1] += (xlo.x + i1 * h.x) * m;
    acc[2] += (xlo.y + i2 * h.y) * m;
    acc[3] += (xlo.z + i3 * h.z) * m;
    for (int d = 0; d < 3; ++d) acc[4 + d] += k[d];
  }
  for (int c = 0; c < 7; ++c) red[c][tid] = acc[c];
  __syncthreads();
  for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
    if (tid < s)
      for (int c = 0; c < 7; ++c) red[c][tid] += red[c][tid + s];
    __syncthreads();
  }
  if (tid == 0)
    for (int c = 0; c < 6; ++c) out[c] = red[1 + c][0] / red[0][0];
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int N>
cudaError_t kpart_tn(const Handle& H, const void* f, int d, double* S, cudaStream_t s) {
  if constexpr (sizeof(T) == 4)
    k_diag_kpart_f<N><<<nblk(H.g.nxp * N, kDiagThreads), kDiagThreads, 0, s>>>(
        static_cast<const float*>(f), H.g.nxp, d, S + (size_t)d * H.g.nxp * N);
  else
    k_diag_kpart<T, N><<<nblk(H.g.nxp * N, kDiagThreads), kDiagThreads, 0, s>>>(
        static_cast<const T*>(f), H.g.nxp, d, S + (size_t)d * H.g.nxp * N);
  return cudaGetLastError();
}

cudaError_t kpart(const Handle& H, const void* f, int d, double* S, cudaStream_t s) {
  switch (H.g.nk) {
    case 8: return H.fp64 ? kpart_tn<double, 8>(H, f, d, S, s) : kpart_tn<float, 8>(H, f, d, S, s);
    case 16: return H.fp64 ? kpart_tn<double, 16>(H, f, d, S, s) : kpart_tn<float, 16>(H, f, d, S, s);
    case 32: return H.fp64 ? kpart_tn<double, 32>(H, f, d, S, s) : kpart_tn<float, 32>(H, f, d, S, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t diag_bytes(const int nx[3], int nk) {
  const size_t nxp = (size_t)nx[0] * nx[1] * nx[2];
  const size_t outn = std::max<size_t>({(size_t)nx[0] * nk, (size_t)nx[1] * nk, (size_t)nx[2] * nk,
                                        (size_t)nx[0] * nx[1], 8});
  return (3 * nxp * nk + outn) * sizeof(double);
}

cudaError_t launch_diag(const Handle& H, const void* f, int what, int j, double* buf, double* out_dev,
                        cudaStream_t s) {
  const int N = H.g.nk;
  const int* nx = H.g.nx;
  cudaError_t e = cudaSuccess;
  if (what == 0) {   // reduced Wigner function W_j
    e = kpart(H, f, j, buf, s);
    if (e != cudaSuccess) return e;
    const int oa = j == 0 ? 1 : 0, ob = j == 2 ? 1 : 2;
    const double vol = H.g.h[oa] * H.g.h[ob] * H.g.dk * H.g.dk;
    k_diag_wigner<<<nblk((int64_t)nx[j] * N, kDiagThreads), kDiagThreads, 0, s>>>(
        buf + (size_t)j * H.g.nxp * N, j, nx[0], nx[1], nx[2], N, vol, out_dev);
  } else if (what == 1) {   // marginal P(x1, x2)
    e = kpart(H, f, 0, buf, s);
    if (e != cudaSuccess) return e;
    const double vol = H.g.h[2] * H.g.dk * H.g.dk * H.g.dk;
    k_diag_marginal<<<nblk((int64_t)nx[0] * nx[1], kDiagThreads), kDiagThreads, 0, s>>>(
        buf, nx[0], nx[1], nx[2], N, vol, out_dev);
  } else {   // averages
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = kpart(H, f, d, buf, s);
    if (e != cudaSuccess) return e;
    k_diag_expect<<<1, kDiagThreads, 0, s>>>(buf, H.g.nxp, nx[1], nx[2], N,
                                             make_double3(H.g.x_lo[0], H.g.x_lo[1], H.g.x_lo[2]),
                                             make_double3(H.g.h[0], H.g.h[1], H.g.h[2]), H.g.dk, out_dev);
  }
  return cudaGetLastError();
}

}  // namespace chasm
