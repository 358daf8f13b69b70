// Reductions (mass, energy), the quadratic-potential P-flow and the initial-data kernels.
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace chasm {
namespace {

constexpr int kMomBlocks = 1024;   // fixed: the reduction tree does not depend on the device
constexpr int kMomThreads = 256;

// ---------------------------------------------------------------------------------------------
// Mass and energy (diagnostics of Sec. 5): per x point, S0 = sum_k f and S2 = sum_k |k|^2 f;
// mass += S0, energy += (hbar^2/2m) dk^2 S2' + V(x) S0 where S2' uses integer |j - N/2|^2.
// Every thread accumulates its own elements of the block's x points (V(x) S0 is linear in the
// thread's partial of S0, so no per-x-point reduction is needed); one block reduction at the end
// and a second kernel that adds the block partials in a fixed order make the result bitwise
// reproducible (the grid size is fixed).
// ---------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double red[NV][kMomThreads / 32];
  const int tid = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NV; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  if ((tid & 31) == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) red[c][tid >> 5] = v[c];
  __syncthreads();
  if (tid == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double a = 0.0;
      for (int w = 0; w < kMomThreads / 32; ++w) a += red[c][w];
      out[(int64_t)NV * blockIdx.x + c] = a;
    }
}

template <typename T>
__global__ void __launch_bounds__(kMomThreads) k_moments(const T* __restrict__ f, int64_t nxp,
                                                         int nk, const double* __restrict__ vx,
                                                         double* __restrict__ partials) {
  const int kvol = nk * nk * nk;
  double acc[3] = {0.0, 0.0, 0.0};   // sum f, sum |j - N/2|^2 f, sum V(x) f
  for (int64_t xp = blockIdx.x; xp < nxp; xp += gridDim.x) {
    const T* fx = f + xp * kvol;
    double s0 = 0.0, s2 = 0.0;
    for (int e = threadIdx.x; e < kvol; e += kMomThreads) {
      const double v = (double)fx[e];
      const int k3 = e % nk - nk / 2, k2 = (e / nk) % nk - nk / 2, k1 = e / (nk * nk) - nk / 2;
      s0 += v;
      s2 += v * (double)(k1 * k1 + k2 * k2 + k3 * k3);
    }
    acc[0] += s0;
    acc[1] += s2;
    acc[2] += vx[xp] * s0;
  }
  block_sum_store<3>(acc, partials);
}

// Single precision: the FP64 pipe (1/64 of the FP32 rate on this part) cannot keep up with one
// FP64 add per element at HBM speed, so each thread sums its elements of an x point in compensated
// FP32 pairs (Knuth's error-free two-sum; the products v |k|^2 with their exact FMA residual; about
// 2^-44 relative) and adds the pairs to FP64 accumulators once per x point; float4 loads, eight in
// flight per thread.
template <>
__global__ void __launch_bounds__(kMomThreads) k_moments<float>(const float* __restrict__ f, int64_t nxp,
                                                                int nk, const double* __restrict__ vx,
                                                                double* __restrict__ partials) {
  const int tid = threadIdx.x;
  const int lg = __ffs(nk) - 1;              // nk is a power of two
  const int kvol4 = (nk * nk * nk) >> 2;     // float4 per x point
  const int half = nk >> 1;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t xp = blockIdx.x; xp < nxp; xp += gridDim.x) {
    const float4* fx = reinterpret_cast<const float4*>(f + xp * (int64_t)(kvol4 << 2));
    float h0 = 0.f, l0 = 0.f, h2 = 0.f, l2 = 0.f;
#pragma unroll 8
    for (int e4 = tid; e4 < kvol4; e4 += kMomThreads) {
      const float4 q = __ldcs(fx + e4);
      const float v[4] = {q.x, q.y, q.z, q.w};
      const int e = e4 << 2;
      const int k1 = (e >> (2 * lg)) - half, k2 = ((e >> lg) & (nk - 1)) - half;
      const int k3b = (e & (nk - 1)) - half;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k3 = k3b + c;
        const float w = (float)(k1 * k1 + k2 * k2 + k3 * k3);   // exact: at most 3 (nk/2)^2
        two_sum_f(h0, l0, v[c]);
        const float pr = v[c] * w;
        l2 += fmaf(v[c], w, -pr);                                 // exact product residual
        two_sum_f(h2, l2, pr);
      }
    }
    const double s0 = (double)h0 + (double)l0;
    acc[0] += s0;
    acc[1] += (double)h2 + (double)l2;
    acc[2] += vx[xp] * s0;
  }
  block_sum_store<3>(acc, partials);
}

__global__ void k_moments_final(const double* __restrict__ partials, int nblocks, double cell,
                                double kin_fac, double* __restrict__ out) {
  __shared__ double red[3][kMomThreads];
  const int tid = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = tid; i < nblocks; i += kMomThreads) {
    a += partials[3 * i];
    b += partials[3 * i + 1];
    c += partials[3 * i + 2];
  }
  red[0][tid] = a;
  red[1][tid] = b;
  red[2][tid] = c;
  __syncthreads();
  for (int s = kMomThreads / 2; s > 0; s >>= 1) {
    if (tid < s) {
      red[0][tid] += red[0][tid + s];
      red[1][tid] += red[1][tid + s];
      red[2][tid] += red[2][tid + s];
    }
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = red[0][0] * cell;
    out[1] = (red[1][0] * kin_fac + red[2][0]) * cell;
  }
}

// ---------------------------------------------------------------------------------------------
// Quadratic potential: P(dt) is the exact shift f(x, k + s(x)), s_d = dt kappa (x_d - c_d)/hbar
// (Eq. 5.1).  Per k-dimension it is the band-limited (periodic, spectral) shift, i.e. a circulant
// matrix whose first column c[q] = (1/N) sum_m phi_m e^{2 pi i m q / N} is tabulated per x_d on
// the host; one thread applies it to one k-line in registers.
// ---------------------------------------------------------------------------------------------
// FP64: one line per thread.  FP32: two lines per thread, k-adjacent in memory (r even and r + 1,
// the same x point), moved with 8-byte accesses, at three 128-thread CTAs per SM (a register bound
// that spills a few coefficients but keeps 12 warps per SM: 6.25 -> 5.40 ms for the three passes
// at 32^3 x 32^3).
template <typename T, int N>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 1) k_kshift(T* __restrict__ f, int64_t nxp, int nx1, int nx2, int nx3, int dim,
                         const T* __restrict__ rows) {
  constexpr int LPT = sizeof(T) == 4 ? 2 : 1;
  const int64_t line = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * LPT;
  if (line >= nxp * N * N) return;
  const int64_t xp = line / (N * N);
  const int r = (int)(line % (N * N));
  int64_t base, stride;
  int id;
  if (dim == 0) {
    base = xp * N * N * N + r;
    stride = N * N;
    id = (int)(xp / ((int64_t)nx2 * nx3));
  } else if (dim == 1) {
    base = xp * N * N * N + (r / N) * N * N + (r % N);
    stride = N;
    id = nx1 + (int)((xp / nx3) % nx2);
  } else {
    base = xp * N * N * N + (int64_t)r * N;
    stride = 1;
    id = nx1 + nx2 + (int)(xp % nx3);
  }
  const T* crow = rows + (int64_t)id * N;
  T c[N];
#pragma unroll
  for (int q = 0; q < N; ++q) c[q] = __ldg(crow + q);
  if constexpr (LPT == 1) {
    T v[N];
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = f[base + l * stride];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T acc = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) acc += c[(j - l + N) & (N - 1)] * v[l];
      f[base + j * stride] = acc;
    }
  } else {
    T v0[N], v1[N];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const float2 q = *reinterpret_cast<const float2*>(f + base + l * stride);
      v0[l] = q.x;
      v1[l] = q.y;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T a0 = (T)0, a1 = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) {
        a0 += c[(j - l + N) & (N - 1)] * v0[l];
        a1 += c[(j - l + N) & (N - 1)] * v1[l];
      }
      *reinterpret_cast<float2*>(f + base + j * stride) = make_float2(a0, a1);
    }
  }
}

// The k3 pass: the lines are contiguous, so a thread walking its own line would touch a new cache
// line with every load of its warp.  A block stages its kKsLines consecutive lines in shared memory
// with coalesced loads (row stride N + 1: conflict-free line reads), each thread applies the
// circulant to its line in registers, and the block writes the tile back coalesced.
constexpr int kKsLines = 128;

// FP32 with N = 32: the tile moves as 16-byte quads (coalesced 512-byte warp accesses), quad q
// of line r stored at quad position q ^ (r & 7) of its row, so the quad accesses of both the
// copies and the per-line reads and writes touch 32 distinct banks.
__device__ __forceinline__ int ks_quad(int r, int q) { return r * 32 + ((q ^ (r & 7)) << 2); }

template <int N>
__device__ __forceinline__ void tile_load4(float* tile, const float* g, int nl, int tid) {
  for (int i4 = tid; i4 < nl * (N / 4); i4 += kKsLines)
    *reinterpret_cast<float4*>(tile + ks_quad(i4 / (N / 4), i4 % (N / 4))) = reinterpret_cast<const float4*>(g)[i4];
}
template <int N>
__device__ __forceinline__ void tile_store4(const float* tile, float* g, int nl, int tid) {
  for (int i4 = tid; i4 < nl * (N / 4); i4 += kKsLines)
    reinterpret_cast<float4*>(g)[i4] = *reinterpret_cast<const float4*>(tile + ks_quad(i4 / (N / 4), i4 % (N / 4)));
}

template <typename T, int N>
__global__ void __launch_bounds__(kKsLines) k_kshift3(T* __restrict__ f, int64_t nxp, int nx1, int nx2,
                                                      int nx3, const T* __restrict__ rows) {
  const int tid = threadIdx.x;
  const int64_t lines = nxp * N * N;
  const int64_t l0 = (int64_t)blockIdx.x * kKsLines;   // first line of the block
  const int nl = lines - l0 < kKsLines ? (int)(lines - l0) : kKsLines;
  T* g = f + l0 * N;
  if constexpr (sizeof(T) == 4 && N == 32) {
    __shared__ __align__(16) float tq[kKsLines * N];
    tile_load4<N>(tq, g, nl, tid);
    __syncthreads();
    if (tid < nl) {
      const int64_t xp = (l0 + tid) / (N * N);
      const float* crow = rows + (int64_t)(nx1 + nx2 + (int)(xp % nx3)) * N;
      float c[N], v[N];
#pragma unroll
      for (int q = 0; q < N; ++q) c[q] = __ldg(crow + q);
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        const float4 u = *reinterpret_cast<const float4*>(tq + ks_quad(tid, q));
        v[4 * q] = u.x;
        v[4 * q + 1] = u.y;
        v[4 * q + 2] = u.z;
        v[4 * q + 3] = u.w;
      }
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * q + e;
          float acc = 0.f;
#pragma unroll
          for (int l = 0; l < N; ++l) acc += c[(j - l + N) & (N - 1)] * v[l];
          o[e] = acc;
        }
        *reinterpret_cast<float4*>(tq + ks_quad(tid, q)) = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
    __syncthreads();
    tile_store4<N>(tq, g, nl, tid);
    return;
  }
  __shared__ T tile[kKsLines][N + 1];
  for (int i = tid; i < nl * N; i += kKsLines) tile[i / N][i % N] = g[i];
  __syncthreads();
  if (tid < nl) {
    const int64_t xp = (l0 + tid) / (N * N);
    const T* crow = rows + (int64_t)(nx1 + nx2 + (int)(xp % nx3)) * N;
    T c[N], v[N];
#pragma unroll
    for (int q = 0; q < N; ++q) c[q] = __ldg(crow + q);
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = tile[tid][l];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T acc = (T)0;
#pragma unroll
      for (int l = 0; l < N; ++l) acc += c[(j - l + N) & (N - 1)] * v[l];
      tile[tid][j] = acc;
    }
  }
  __syncthreads();
  for (int i = tid; i < nl * N; i += kKsLines) g[i] = tile[i / N][i % N];
}

// ---------------------------------------------------------------------------------------------
// Initial data
// ---------------------------------------------------------------------------------------------
struct Packets {
  int n;
  chasm_gaussian g[16];
};

// Each packet factorises, w exp(-ax |x - x0|^2) exp(-ak |k - k0|^2) = w prod_d gx_d(x_d) prod_d
// gk_d(k_d), so one block per x point forms w prod_d gx_d once per packet and the 1-D k factors
// gk_d (3 N_k per packet) in shared memory; every cell is then three FP64 products per packet,
// summed in FP64 and rounded once to T.  The threads write four consecutive k3 values each.
constexpr int kInitThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kInitThreads) k_init_gauss(T* __restrict__ f, GridDesc gd, Packets P) {
  __shared__ double gk[16][3][32];   // gk[p][d][j] = exp(-ak (k_j - k0_d)^2)
  __shared__ double wx[16];          // w prod_d exp(-ax (x_d - x0_d)^2)
  const int nk = gd.nk, tid = threadIdx.x;
  int lg = 0;
  while ((1 << lg) < nk) ++lg;   // nk = 2^lg
  for (int i = tid; i < P.n * 3 * nk; i += blockDim.x) {
    const int p = i / (3 * nk), d = (i / nk) % 3, j = i % nk;
    const double k = (j - nk / 2) * gd.dk - P.g[p].k0[d];
    gk[p][d][j] = exp(-P.g[p].ak * k * k);
  }
  for (int64_t xp = blockIdx.x; xp < gd.nxp; xp += gridDim.x) {
    __syncthreads();   // gk written; the previous x point's wx read
    if (tid < P.n) {
      const int i3 = (int)(xp % gd.nx[2]), i2 = (int)((xp / gd.nx[2]) % gd.nx[1]);
      const int i1 = (int)(xp / ((int64_t)gd.nx[2] * gd.nx[1]));
      const chasm_gaussian& g = P.g[tid];
      const double dx[3] = {gd.x_lo[0] + i1 * gd.h[0] - g.x0[0], gd.x_lo[1] + i2 * gd.h[1] - g.x0[1],
                            gd.x_lo[2] + i3 * gd.h[2] - g.x0[2]};
      wx[tid] = g.w * (exp(-g.ax * dx[0] * dx[0]) * exp(-g.ax * dx[1] * dx[1]) * exp(-g.ax * dx[2] * dx[2]));
    }
    __syncthreads();
    T* fx = f + xp * gd.kvol;
    for (int e0 = 4 * tid; e0 < gd.kvol; e0 += 4 * blockDim.x) {   // kvol = nk^3 is a multiple of 4
      const int k1 = e0 >> (2 * lg), k2 = (e0 >> lg) & (nk - 1), k3 = e0 & (nk - 1);
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      for (int p = 0; p < P.n; ++p) {
        const double a = wx[p] * (gk[p][0][k1] * gk[p][1][k2]);
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = fma(a, gk[p][2][k3 + c], s[c]);
      }
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(fx + e0) = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
      } else {
        reinterpret_cast<double2*>(fx + e0)[0] = make_double2(s[0], s[1]);
        reinterpret_cast<double2*>(fx + e0)[1] = make_double2(s[2], s[3]);
      }
    }
  }
}

// Hydrogen 1s Wigner function, discrete Fourier sum of Sec. 5.2.  Because dk dy = 2 pi / N the
// phase is N-periodic in the sample index, so the N_y^3 samples fold into N^3 bins (this
// kernel), followed by an N^3 DFT (three separable passes) and the dy^3 factor.
struct OneS {
  double x_lo[3], h[3];
  double c[3];
  double dy;
  int nx[3];
  int nk, ny;
  int64_t xp0, nxl;   // first x point of the chunk and its length
};

// Folded sample sums.  The FP32-mixed form accumulates the samples in FP32 (the result is stored
// in FP32), the FP64 form in FP64.
template <typename R>
__global__ void k_1s_fold(double2* __restrict__ P, OneS o) {
  const int N = o.nk;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= o.nxl * N * N * N) return;
  const int64_t xp = o.xp0 + t / (N * N * N);
  const int r = (int)(t % (N * N * N));
  const int r3 = r % N, r2 = (r / N) % N, r1 = r / (N * N);
  const int i3 = (int)(xp % o.nx[2]), i2 = (int)((xp / o.nx[2]) % o.nx[1]);
  const int i1 = (int)(xp / ((int64_t)o.nx[2] * o.nx[1]));
  const R a1 = (R)(o.x_lo[0] + i1 * o.h[0] - o.c[0]);
  const R a2 = (R)(o.x_lo[1] + i2 * o.h[1] - o.c[1]);
  const R a3 = (R)(o.x_lo[2] + i3 * o.h[2] - o.c[2]);
  const int rep = o.ny / N;
  const R hdy = (R)(0.5 * o.dy);
  R s = 0;
  for (int b1 = 0; b1 < rep; ++b1) {
    const R y1 = (R)(r1 + b1 * N - o.ny / 2) * hdy;
    const R m1 = (a1 - y1) * (a1 - y1), p1 = (a1 + y1) * (a1 + y1);
    for (int b2 = 0; b2 < rep; ++b2) {
      const R y2 = (R)(r2 + b2 * N - o.ny / 2) * hdy;
      const R m2 = m1 + (a2 - y2) * (a2 - y2), p2 = p1 + (a2 + y2) * (a2 + y2);
      for (int b3 = 0; b3 < rep; ++b3) {
        const R y3 = (R)(r3 + b3 * N - o.ny / 2) * hdy;
        const R rm = sqrt(m2 + (a3 - y3) * (a3 - y3));
        const R rp = sqrt(p2 + (a3 + y3) * (a3 + y3));
        s += exp(-(rm + rp));
      }
    }
  }
  const double norm = 1.0 / (8.0 * 3.141592653589793 * 3.141592653589793 * 3.141592653589793 *
                             3.141592653589793);   // (2 sqrt 2 pi^2)^-2
  P[t] = make_double2((double)s * norm, 0.0);
}

// out[.., j, ..] = sum_r in[.., r, ..] e^{-2 pi i (j - N/2) r / N} along one k axis; the N roots
// of unity sit in shared memory.
__global__ void k_1s_dft(const double2* __restrict__ in, double2* __restrict__ out, int64_t nxl,
                         int N, int axis) {
  __shared__ double2 w[64];
  if (threadIdx.x < N) {
    double sn, cs;
    sincospi(-2.0 * (double)threadIdx.x / N, &sn, &cs);
    w[threadIdx.x] = make_double2(cs, sn);
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxl * N * N * N) return;
  const int64_t cell0 = t - t % ((int64_t)N * N * N);
  const int e = (int)(t % (N * N * N));
  const int stride = axis == 0 ? N * N : (axis == 1 ? N : 1);
  const int j = (e / stride) % N;
  const int64_t lb = cell0 + (e - j * stride);
  const int js = ((j - N / 2) % N + N) % N;
  double re = 0.0, im = 0.0;
  int q = 0;
  for (int r = 0; r < N; ++r) {
    const double2 c = w[q];
    const double2 v = in[lb + (int64_t)r * stride];
    re = fma(v.x, c.x, fma(-v.y, c.y, re));
    im = fma(v.x, c.y, fma(v.y, c.x, im));
    q += js;
    if (q >= N) q -= N;
  }
  out[t] = make_double2(re, im);
}

template <typename T>
__global__ void k_1s_store(const double2* __restrict__ P, T* __restrict__ f, int64_t off,
                           int64_t n, double scale) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  f[off + t] = (T)(P[t].x * scale);
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

int moments_blocks() { return kMomBlocks; }

cudaError_t launch_moments(const Handle& H, const void* f, double* partials, double* result_dev,
                           cudaStream_t s) {
  const int nb = (int)std::min<int64_t>(kMomBlocks, H.g.nxp);
  if (H.fp64)
    k_moments<double><<<nb, kMomThreads, 0, s>>>((const double*)f, H.g.nxp, H.g.nk, H.d_vx, partials);
  else
    k_moments<float><<<nb, kMomThreads, 0, s>>>((const float*)f, H.g.nxp, H.g.nk, H.d_vx, partials);
  const double cell = H.g.h[0] * H.g.h[1] * H.g.h[2] * H.g.dk * H.g.dk * H.g.dk;
  const double kin = H.hbar * H.hbar / (2.0 * H.m) * H.g.dk * H.g.dk;
  k_moments_final<<<1, kMomThreads, 0, s>>>(partials, nb, cell, kin, result_dev);
  return cudaGetLastError();
}

cudaError_t launch_kshift(const Handle& H, void* f, int dim, const void* rows, cudaStream_t s) {
  const int64_t lines = H.g.nxp * H.g.nk * H.g.nk;
  const unsigned nb = nblk(lines, 128), nb2 = nblk(lines / 2, 128);   // lines = nxp N^2 is even
  const int* nx = H.g.nx;
#define CHASM_KS(TT, NN)                                                                           \
  do {                                                                                             \
    if (dim == 2)                                                                                  \
      k_kshift3<TT, NN><<<nblk(lines, kKsLines), kKsLines, 0, s>>>((TT*)f, H.g.nxp, nx[0], nx[1],  \
                                                                   nx[2], (const TT*)rows);        \
    else                                                                                           \
      k_kshift<TT, NN><<<sizeof(TT) == 4 ? nb2 : nb, 128, 0, s>>>((TT*)f, H.g.nxp, nx[0], nx[1],   \
                                                                  nx[2], dim, (const TT*)rows);    \
  } while (0)
  switch (H.g.nk) {
    case 8:
      if (H.fp64) CHASM_KS(double, 8); else CHASM_KS(float, 8);
      break;
    case 16:
      if (H.fp64) CHASM_KS(double, 16); else CHASM_KS(float, 16);
      break;
    case 32:
      if (H.fp64) CHASM_KS(double, 32); else CHASM_KS(float, 32);
      break;
    default:
      return cudaErrorInvalidValue;
  }
#undef CHASM_KS
  return cudaGetLastError();
}

cudaError_t launch_init_gaussians(const Handle& H, void* f, const chasm_gaussian* g, int n,
                                  cudaStream_t s) {
  Packets P;
  P.n = n;
  for (int i = 0; i < n; ++i) P.g[i] = g[i];
  const unsigned nb = (unsigned)std::min<int64_t>(H.g.nxp, (int64_t)H.num_sms * 8);
  if (H.fp64)
    k_init_gauss<double><<<nb, kInitThreads, 0, s>>>((double*)f, H.g, P);
  else
    k_init_gauss<float><<<nb, kInitThreads, 0, s>>>((float*)f, H.g, P);
  return cudaGetLastError();
}

cudaError_t launch_init_1s(const Handle& H, void* f, int n_y, const double c[3], cudaStream_t s,
                           std::string* err) {
  const int N = H.g.nk;
  const int64_t kvol = H.g.kvol;
  const size_t per_x = (size_t)kvol * sizeof(double2) * 2;
  int64_t chunk = std::max<int64_t>(1, (int64_t)((size_t)2 << 30) / (int64_t)per_x);
  chunk = std::min<int64_t>(chunk, H.g.nxp);
  double2 *A = nullptr, *B = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&A, (size_t)chunk * kvol * sizeof(double2), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&B, (size_t)chunk * kvol * sizeof(double2), s);
  if (e != cudaSuccess) {
    if (err) *err = "init_hydrogen_1s: temporary allocation failed";
    if (A) cudaFreeAsync(A, s);
    return e;
  }
  OneS o;
  for (int d = 0; d < 3; ++d) {
    o.x_lo[d] = H.g.x_lo[d];
    o.h[d] = H.g.h[d];
    o.c[d] = c ? c[d] : 0.0;
    o.nx[d] = H.g.nx[d];
  }
  o.nk = N;
  o.ny = n_y;
  o.dy = 2.0 * M_PI / (N * H.g.dk);
  const double scale = o.dy * o.dy * o.dy;
  for (int64_t x0 = 0; x0 < H.g.nxp && e == cudaSuccess; x0 += chunk) {
    o.xp0 = x0;
    o.nxl = std::min<int64_t>(chunk, H.g.nxp - x0);
    const int64_t n = o.nxl * kvol;
    if (H.fp64)
      k_1s_fold<double><<<nblk(n, 128), 128, 0, s>>>(A, o);
    else
      k_1s_fold<float><<<nblk(n, 128), 128, 0, s>>>(A, o);
    k_1s_dft<<<nblk(n, 256), 256, 0, s>>>(A, B, o.nxl, N, 2);
    k_1s_dft<<<nblk(n, 256), 256, 0, s>>>(B, A, o.nxl, N, 1);
    k_1s_dft<<<nblk(n, 256), 256, 0, s>>>(A, B, o.nxl, N, 0);
    if (H.fp64)
      k_1s_store<double><<<nblk(n, 256), 256, 0, s>>>(B, (double*)f, x0 * kvol, n, scale);
    else
      k_1s_store<float><<<nblk(n, 256), 256, 0, s>>>(B, (float*)f, x0 * kvol, n, scale);
    e = cudaGetLastError();
  }
  cudaFreeAsync(A, s);
  cudaFreeAsync(B, s);
  return e;
}

}  // namespace chasm
