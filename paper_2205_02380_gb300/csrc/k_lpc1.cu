// Kernels of the LPC1 integrator (Sec. 2.2) that the Strang step does not have:
//
//   k_kderiv        Theta for V = kappa/2 |x - c|^2 (Eq. 5.1), one k-dimension per launch:
//                   out = (base or out) + coef kappa (x_d - c_d)/hbar D u along k_d, where D is the
//                   spectral derivative on the periodic k-grid (i xi_m, xi_m = pi m / L_k, the
//                   Nyquist mode dropped), applied as its circulant: (D u)_p = sum_j d_j u_{p-j},
//                   d_j = -(2/N) sum_{m=1}^{N/2-1} xi_m sin(2 pi m j / N).  One thread per k-line
//                   (two k-adjacent lines in FP32), the N taps in the kernel's parameter block
//                   (constant-bank operands); the k3 pass (k_kderiv3) stages its contiguous
//                   lines in shared memory.
//   k_lpc1_combine  predictor and corrector base from the advected fields g = f(A_dt) and
//                   h = Theta[f](A_dt): v = g + dt h (the predictor f~), f = g + dt/2 h.
#include "internal.hpp"

namespace chasm {
namespace {

template <typename T, int N>
struct KDerivParams {
  const T* in;
  const T* base;     // first dimension: out = base + ...; null: out = ...
  T* out;
  int64_t nxp;
  int nx1, nx2, nx3;
  int dim;
  bool accumulate;   // out += ...
  double x_lo, h, center, rate_scale;   // rate(x_d) = rate_scale (x_lo + i h - center)
  T coef;
  T d[N];
};

// FP64: one line per thread.  FP32: two lines per thread, k-adjacent in memory (r even and r + 1,
// the same x point), moved with 8-byte accesses.
template <typename T, int N>
__global__ void __launch_bounds__(128) k_kderiv(const KDerivParams<T, N> p) {
  constexpr int LPT = sizeof(T) == 4 ? 2 : 1;
  const int64_t line = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * LPT;
  if (line >= p.nxp * N * N) return;
  const int64_t xp = line / (N * N);
  const int r = (int)(line % (N * N));
  int64_t base, stride;
  int id;
  if (p.dim == 0) {
    base = xp * N * N * N + r;
    stride = N * N;
    id = (int)(xp / ((int64_t)p.nx2 * p.nx3));
  } else if (p.dim == 1) {
    base = xp * N * N * N + (r / N) * N * N + (r % N);
    stride = N;
    id = (int)((xp / p.nx3) % p.nx2);
  } else {
    base = xp * N * N * N + (int64_t)r * N;
    stride = 1;
    id = (int)(xp % p.nx3);
  }
  const T scale = (T)(p.rate_scale * (p.x_lo + id * p.h - p.center)) * p.coef;
  if constexpr (LPT == 1) {
    T v[N];
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = p.in[base + l * stride];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T acc = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) acc = fma(p.d[(q - l + N) & (N - 1)], v[l], acc);
      const int64_t o = base + q * stride;
      T b = (T)0;
      if (p.accumulate)
        b = p.out[o];
      else if (p.base)
        b = p.base[o];
      p.out[o] = fma(scale, acc, b);
    }
  } else {
    // the lines and the terms they are added to, all loads in flight before the arithmetic
    T v0[N], v1[N];
    float2 b[N];
    const T* add = p.accumulate ? p.out : p.base;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const float2 u = *reinterpret_cast<const float2*>(p.in + base + l * stride);
      v0[l] = u.x;
      v1[l] = u.y;
      b[l] = add ? *reinterpret_cast<const float2*>(add + base + l * stride) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T a0 = (T)0, a1 = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        a0 = fma(p.d[(q - l + N) & (N - 1)], v0[l], a0);
        a1 = fma(p.d[(q - l + N) & (N - 1)], v1[l], a1);
      }
      *reinterpret_cast<float2*>(p.out + base + q * stride) =
          make_float2(fma(scale, a0, b[q].x), fma(scale, a1, b[q].y));
    }
  }
}

// The k3 pass (contiguous lines): a block stages LB consecutive lines of in and of the term it
// adds to (out or base) in shared memory with coalesced loads (row stride N + 1), each thread
// forms its line in registers, and the block stores the tile coalesced.
template <typename T, int N>
struct KDeriv3 {
  static constexpr int LB = (sizeof(T) == 8 && N == 32) ? 64 : 128;   // lines per block
};

// FP32 with N = 32: the tiles move as 16-byte quads (coalesced 512-byte warp accesses), quad q of
// line r stored at quad position q ^ (r & 7) of its row (32 distinct banks for every quad access).
__device__ __forceinline__ int kd_quad(int r, int q) { return r * 32 + ((q ^ (r & 7)) << 2); }

template <typename T, int N>
__global__ void __launch_bounds__(KDeriv3<T, N>::LB) k_kderiv3(const KDerivParams<T, N> p) {
  constexpr int LB = KDeriv3<T, N>::LB;
  const int tid = threadIdx.x;
  const int64_t lines = p.nxp * N * N;
  const int64_t l0 = (int64_t)blockIdx.x * LB;
  const int nl = lines - l0 < LB ? (int)(lines - l0) : LB;
  const T* b = p.accumulate ? p.out : p.base;   // the term added to (null: none)
  if constexpr (sizeof(T) == 4 && N == 32) {
    __shared__ __align__(16) float qin[LB * N];
    __shared__ __align__(16) float qb[LB * N];
    const float4* gin = reinterpret_cast<const float4*>(p.in + l0 * N);
    const float4* gb = b ? reinterpret_cast<const float4*>(b + l0 * N) : nullptr;
    for (int i4 = tid; i4 < nl * (N / 4); i4 += LB) {
      const int o = kd_quad(i4 / (N / 4), i4 % (N / 4));
      *reinterpret_cast<float4*>(qin + o) = gin[i4];
      *reinterpret_cast<float4*>(qb + o) = gb ? gb[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (tid < nl) {
      const int64_t xp = (l0 + tid) / (N * N);
      const int id = (int)(xp % p.nx3);
      const float scale = (float)(p.rate_scale * (p.x_lo + id * p.h - p.center)) * p.coef;
      float v[N];
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        const float4 u = *reinterpret_cast<const float4*>(qin + kd_quad(tid, q));
        v[4 * q] = u.x;
        v[4 * q + 1] = u.y;
        v[4 * q + 2] = u.z;
        v[4 * q + 3] = u.w;
      }
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        float4* dst = reinterpret_cast<float4*>(qb + kd_quad(tid, q));
        const float4 t = *dst;
        const float tb4[4] = {t.x, t.y, t.z, t.w};
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * q + e;
          float acc = 0.f;
#pragma unroll
          for (int l = 0; l < N; ++l) acc = fmaf(p.d[(j - l + N) & (N - 1)], v[l], acc);
          o[e] = fmaf(scale, acc, tb4[e]);
        }
        *dst = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
    __syncthreads();
    float4* gout = reinterpret_cast<float4*>(p.out + l0 * N);
    for (int i4 = tid; i4 < nl * (N / 4); i4 += LB)
      gout[i4] = *reinterpret_cast<const float4*>(qb + kd_quad(i4 / (N / 4), i4 % (N / 4)));
    return;
  }
  __shared__ T tin[LB][N + 1];
  __shared__ T tb[LB][N + 1];
  for (int i = tid; i < nl * N; i += LB) {
    tin[i / N][i % N] = p.in[l0 * N + i];
    tb[i / N][i % N] = b ? b[l0 * N + i] : (T)0;
  }
  __syncthreads();
  if (tid < nl) {
    const int64_t xp = (l0 + tid) / (N * N);
    const int id = (int)(xp % p.nx3);
    const T scale = (T)(p.rate_scale * (p.x_lo + id * p.h - p.center)) * p.coef;
    T v[N];
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = tin[tid][l];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T acc = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) acc = fma(p.d[(q - l + N) & (N - 1)], v[l], acc);
      tb[tid][q] = fma(scale, acc, tb[tid][q]);
    }
  }
  __syncthreads();
  for (int i = tid; i < nl * N; i += LB) p.out[l0 * N + i] = tb[i / N][i % N];
}

template <typename T>
__global__ void k_lpc1_combine(T* __restrict__ f, const T* __restrict__ h, T* __restrict__ v, int64_t n,
                               T dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const T half = dt * (T)0.5;
  if constexpr (sizeof(T) == 4) {
    if (4 * i >= n) return;   // n is a multiple of 4 (N_k^3 per x point)
    const float4 g4 = reinterpret_cast<const float4*>(f)[i];
    const float4 h4 = reinterpret_cast<const float4*>(h)[i];
    reinterpret_cast<float4*>(v)[i] = make_float4(fmaf(dt, h4.x, g4.x), fmaf(dt, h4.y, g4.y),
                                                  fmaf(dt, h4.z, g4.z), fmaf(dt, h4.w, g4.w));
    reinterpret_cast<float4*>(f)[i] = make_float4(fmaf(half, h4.x, g4.x), fmaf(half, h4.y, g4.y),
                                                  fmaf(half, h4.z, g4.z), fmaf(half, h4.w, g4.w));
  } else {
    if (2 * i >= n) return;
    const double2 g2 = reinterpret_cast<const double2*>(f)[i];
    const double2 h2 = reinterpret_cast<const double2*>(h)[i];
    reinterpret_cast<double2*>(v)[i] = make_double2(fma(dt, h2.x, g2.x), fma(dt, h2.y, g2.y));
    reinterpret_cast<double2*>(f)[i] = make_double2(fma(half, h2.x, g2.x), fma(half, h2.y, g2.y));
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int N>
cudaError_t kderiv_tn(const Handle& H, const void* in, const void* base, void* out, double coef,
                      cudaStream_t s) {
  KDerivParams<T, N> p;
  p.in = static_cast<const T*>(in);
  p.base = static_cast<const T*>(base);
  p.out = static_cast<T*>(out);
  p.nxp = H.g.nxp;
  p.nx1 = H.g.nx[0];
  p.nx2 = H.g.nx[1];
  p.nx3 = H.g.nx[2];
  p.coef = (T)coef;
  p.rate_scale = H.kappa / H.hbar;
  for (int j = 0; j < N; ++j) {
    double acc = 0.0;
    for (int m = 1; m < N / 2; ++m)
      acc += (M_PI * m / H.g.lk) * std::sin(2.0 * M_PI * m * j / N);
    p.d[j] = (T)(-2.0 * acc / N);
  }
  const unsigned nb = nblk(H.g.nxp * N * N / (sizeof(T) == 4 ? 2 : 1), 128);   // lines per thread
  for (int d = 0; d < 3; ++d) {
    p.dim = d;
    p.accumulate = d > 0;
    p.x_lo = H.g.x_lo[d];
    p.h = H.g.h[d];
    p.center = H.center[d];
    if (d == 2)
      k_kderiv3<T, N><<<nblk(H.g.nxp * N * N, KDeriv3<T, N>::LB), KDeriv3<T, N>::LB, 0, s>>>(p);
    else
      k_kderiv<T, N><<<nb, 128, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_theta_harm(const Handle& H, const void* in, const void* base, void* out,
                              double coef, cudaStream_t s) {
  switch (H.g.nk) {
    case 8:
      return H.fp64 ? kderiv_tn<double, 8>(H, in, base, out, coef, s)
                    : kderiv_tn<float, 8>(H, in, base, out, coef, s);
    case 16:
      return H.fp64 ? kderiv_tn<double, 16>(H, in, base, out, coef, s)
                    : kderiv_tn<float, 16>(H, in, base, out, coef, s);
    case 32:
      return H.fp64 ? kderiv_tn<double, 32>(H, in, base, out, coef, s)
                    : kderiv_tn<float, 32>(H, in, base, out, coef, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_lpc1_combine(const Handle& H, void* f, const void* h, void* v, double dt,
                                cudaStream_t s) {
  const int64_t n = H.g.ncell;
  if (H.fp64) {
    k_lpc1_combine<double><<<nblk(n / 2, 256), 256, 0, s>>>((double*)f, (const double*)h, (double*)v, n, dt);
  } else {
    k_lpc1_combine<float><<<nblk(n / 4, 256), 256, 0, s>>>((float*)f, (const float*)h, (float*)v, n,
                                                             (float)dt);
  }
  return cudaGetLastError();
}

}  // namespace chasm
