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

// Single precision: one warp per (x point, q) for d = 0, 1 and one warp per x point for d = 2,
// every lane summing its 16-byte loads in compensated FP32 (two-sum; the FP64 pipe runs at 1/64
// of the FP32 rate here), then a compensated butterfly across the lanes and one rounding to FP64.
// The lanes of a warp read consecutive 16-byte pieces: d = 0, the k1 = q slab (N^2 contiguous
// values); d = 1, the rows (a, q) of N contiguous values, N/4 lanes per row; d = 2, the rows
// (a, b), one k3 quad per lane, so that each lane owns four bins.
__device__ __forceinline__ void warp_two_sum(float& hi, float& lo, unsigned mask, int o) {
  const float oh = __shfl_xor_sync(mask, hi, o), ol = __shfl_xor_sync(mask, lo, o);
  two_sum_f(hi, lo, oh);
  lo += ol;
}

template <int N, int D>
__global__ void __launch_bounds__(kDiagThreads) k_diag_kpart_w(const float* __restrict__ f, int64_t nxp,
                                                               double* __restrict__ S) {
  constexpr int Q = N / 4;   // float4 per row of N
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if constexpr (D < 2) {
    if (w >= nxp * N) return;
    const int64_t xp = w / N;
    const int q = (int)(w % N);
    const float4* base = reinterpret_cast<const float4*>(f + xp * (N * N * N));
    float hi = 0.f, lo = 0.f;
#pragma unroll 8
    for (int g = lane; g < N * Q; g += 32) {
      const int a = g / Q, b4 = g % Q;
      const float4 v = __ldcs(base + (D == 0 ? q * N * Q + g : (a * N + q) * Q + b4));
      two_sum_f(hi, lo, v.x);
      two_sum_f(hi, lo, v.y);
      two_sum_f(hi, lo, v.z);
      two_sum_f(hi, lo, v.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) warp_two_sum(hi, lo, 0xffffffffu, o);
    if (lane == 0) S[w] = (double)hi + (double)lo;
  } else {
    if (w >= nxp) return;
    const float4* base = reinterpret_cast<const float4*>(f + w * (N * N * N));
    constexpr int RPI = 32 / Q;   // rows read per iteration by the warp
    const int p = lane % Q, r0 = lane / Q;
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int row = r0; row < N * N; row += RPI) {
      const float4 v = __ldcs(base + row * Q + p);
      two_sum_f(hi[0], lo[0], v.x);
      two_sum_f(hi[1], lo[1], v.y);
      two_sum_f(hi[2], lo[2], v.z);
      two_sum_f(hi[3], lo[3], v.w);
    }
#pragma unroll
    for (int o = Q; o < 32; o <<= 1)
#pragma unroll
      for (int c = 0; c < 4; ++c) warp_two_sum(hi[c], lo[c], 0xffffffffu, o);
    if (lane < Q)
#pragma unroll
      for (int c = 0; c < 4; ++c) S[w * N + 4 * p + c] = (double)hi[c] + (double)lo[c];
  }
}

// W_j[i][q] = vol * sum over the other two x indices of S_j[x][q]: one block per i, thread t adds
// q = t mod N over the (a, b) pairs t / N, t / N + G, ... (G = threads / N), then the G partials
// of each q in ascending order (a fixed order: bitwise reproducible)
__global__ void __launch_bounds__(kDiagThreads) k_diag_wigner(const double* __restrict__ S, int j, int nx0,
                                                              int nx1, int nx2, int N, double vol,
                                                              double* __restrict__ W) {
  __shared__ double part[kDiagThreads];
  const int nx[3] = {nx0, nx1, nx2};
  const int i = blockIdx.x, t = threadIdx.x;
  const int q = t % N, G = kDiagThreads / N;
  const int oa = j == 0 ? 1 : 0, ob = j == 2 ? 1 : 2;
  double s = 0.0;
  for (int ab = t / N; ab < nx[oa] * nx[ob]; ab += G) {
    int ix[3];
    ix[j] = i;
    ix[oa] = ab / nx[ob];
    ix[ob] = ab % nx[ob];
    const int64_t xp = ((int64_t)ix[0] * nx1 + ix[1]) * nx2 + ix[2];
    s += S[xp * N + q];
  }
  part[t] = s;
  __syncthreads();
  if (t < N) {
    double r = 0.0;
    for (int g = 0; g < G; ++g) r += part[g * N + t];
    W[(int64_t)i * N + t] = r * vol;
  }
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

// Averages, stage 1 (kExpBlocks blocks, each a fixed range of x points): m = sum S_0,
// x_d m, k_d = sum_q k_q S_d; the 7 block partials go to part[7 * block + c]
constexpr int kExpBlocks = 256;
__global__ void __launch_bounds__(kDiagThreads) k_diag_expect(const double* __restrict__ S, int64_t nxp,
                                                              int nx1, int nx2, int N, double3 xlo,
                                                              double3 h, double dk,
                                                              double* __restrict__ part) {
  __shared__ double red[7][kDiagThreads];
  const int tid = threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t per = (nxp + gridDim.x - 1) / gridDim.x;
  const int64_t x0 = (int64_t)blockIdx.x * per, x1 = min(nxp, x0 + per);
  for (int64_t xp = x0 + tid; xp < x1; xp += kDiagThreads) {
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
    for (int c = 0; c < 7; ++c) part[7 * blockIdx.x + c] = red[c][0];
}

// Averages, stage 2 (one thread per average): the block partials in ascending order
__global__ void k_diag_expect_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= 6) return;
  double m = 0.0, v = 0.0;
  for (int b = 0; b < nb; ++b) {
    m += part[7 * b];
    v += part[7 * b + 1 + c];
  }
  out[c] = v / m;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int N>
cudaError_t kpart_tn(const Handle& H, const void* f, int d, double* S, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const float* ff = static_cast<const float*>(f);
    double* Sd = S + (size_t)d * H.g.nxp * N;
    const int64_t warps = d == 2 ? H.g.nxp : H.g.nxp * N;
    const unsigned nb = nblk(warps * 32, kDiagThreads);
    if (d == 0) k_diag_kpart_w<N, 0><<<nb, kDiagThreads, 0, s>>>(ff, H.g.nxp, Sd);
    else if (d == 1) k_diag_kpart_w<N, 1><<<nb, kDiagThreads, 0, s>>>(ff, H.g.nxp, Sd);
    else k_diag_kpart_w<N, 2><<<nb, kDiagThreads, 0, s>>>(ff, H.g.nxp, Sd);
  } else
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
  return (3 * nxp * nk + std::max<size_t>(outn, 8 + 7 * (size_t)kExpBlocks)) * sizeof(double);
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
    k_diag_wigner<<<nx[j], kDiagThreads, 0, s>>>(buf + (size_t)j * H.g.nxp * N, j, nx[0], nx[1],
                                                 nx[2], N, vol, out_dev);
  } else if (what == 1) {   // marginal P(x1, x2)
    e = kpart(H, f, 0, buf, s);
    if (e != cudaSuccess) return e;
    const double vol = H.g.h[2] * H.g.dk * H.g.dk * H.g.dk;
    k_diag_marginal<<<nblk((int64_t)nx[0] * nx[1], kDiagThreads), kDiagThreads, 0, s>>>(
        buf, nx[0], nx[1], nx[2], N, vol, out_dev);
  } else {   // averages
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = kpart(H, f, d, buf, s);
    if (e != cudaSuccess) return e;
    // the block partials go behind the six results (diag_bytes reserves them)
    double* part = out_dev + 8;
    k_diag_expect<<<kExpBlocks, kDiagThreads, 0, s>>>(buf, H.g.nxp, nx[1], nx[2], N,
                                                      make_double3(H.g.x_lo[0], H.g.x_lo[1], H.g.x_lo[2]),
                                                      make_double3(H.g.h[0], H.g.h[1], H.g.h[2]), H.g.dk, part);
    k_diag_expect_final<<<1, 32, 0, s>>>(part, kExpBlocks, out_dev);
  }
  return cudaGetLastError();
}

}  // namespace chasm
