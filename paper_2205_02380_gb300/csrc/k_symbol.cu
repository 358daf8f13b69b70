// Symbol precompute for the truncated kernel method (Sec. 4.1), FP64 throughout.
//
//   U_D-hat(xi) = 4 pi Si(|xi| D) / |xi|,  U_D-hat(0) = 4 pi D,  D = diam [-L,L]^3 = 2 sqrt(3) L
//                                                                               (Eqs. 4.2-4.3)
//   T_m = (3N)^-3 sum_{n in I} U_D-hat(2 pi n / (6L)) e^{2 pi i m.n / (3N)},
//         I = {-3N/2 .. 3N/2-1}^3, m in [-(N-1), N-1]^3                          (Eqs. 4.7-4.8)
//   T-hat_xi = sum_m T_m e^{-2 pi i xi.m / (2N)},  xi in [0, 2N)^3  (twofold-padded circulant)
//
// U_D-hat depends on |n|^2 only, so it is tabulated over the integer q = |n|^2 (one Si per q, by
// composite 16-point Gauss-Legendre on panels of width at most pi/2; the nodes come from Newton's
// iteration on the Legendre recurrence, computed on the host).  Because U_D-hat is even in each
// n_d and the unpaired index -3N/2 contributes (-1)^m, T is real and even in each m_d:
// T_m = (3N)^-3 sum_n U prod_d cos(2 pi m_d n_d / 3N), evaluated as three separable passes.
// T-hat is real and even likewise: T-hat_xi = sum_{m_d >= 0} T_m prod_d w(m_d) cos(pi xi_d m_d/N)
// with w(0) = 1, w(m > 0) = 2, again three separable passes.  The result is written in the
// parity-major order of the Theta kernel (s = (xi mod 2) N + xi / 2 per dimension), as
// [s3][s1][s2], scaled by 1/(2N)^3, in the storage precision.
#include <cmath>
#include <vector>

#include "internal.hpp"

namespace chasm {
namespace {

constexpr int kGL = 16;
struct GLRule {
  double x[kGL];
  double w[kGL];
};

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's iteration on P_n (three-term recurrence).
GLRule gauss_legendre() {
  GLRule r{};
  const int n = kGL;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    r.x[i] = z;
    r.w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return r;
}

// Si(x) = int_0^x sin(t)/t dt, composite Gauss-Legendre
__device__ double sine_integral(double x, const GLRule& gl) {
  if (x == 0.0) return 0.0;
  const double panel = 1.5707963267948966;  // pi / 2
  const int np = (int)ceil(x / panel);
  const double wdt = x / np;
  double s = 0.0;
  for (int k = 0; k < np; ++k) {
    const double a = k * wdt;
    double ps = 0.0;
#pragma unroll
    for (int i = 0; i < kGL; ++i) {
      const double t = a + 0.5 * wdt * (gl.x[i] + 1.0);
      ps += gl.w[i] * sin(t) / t;
    }
    s += 0.5 * wdt * ps;
  }
  return s;
}

__global__ void k_uhat_table(double* __restrict__ U, int qmax, double c, double D, GLRule gl) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > qmax) return;
  if (q == 0) {
    U[0] = 4.0 * 3.141592653589793 * D;
    return;
  }
  const double xi = sqrt((double)q) * c;
  U[q] = 4.0 * 3.141592653589793 * sine_integral(xi * D, gl) / xi;
}

// cos(2 pi r / M) with the integer product reduced modulo M first
__device__ __forceinline__ double cos2pi_frac(long long num, int M) {
  long long r = num % M;
  if (r < 0) r += M;
  return cospi(2.0 * (double)r / (double)M);
}

// pass 1: A1[n1][n2][m3] = sum_{n3} U(|n|^2) cos(2 pi m3 n3 / M), n in [-M/2, M/2)
__global__ void k_t_pass1(const double* __restrict__ U, double* __restrict__ A1, int M, int N) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * M * N) return;
  const int m3 = (int)(t % N);
  const int n2 = (int)((t / N) % M) - M / 2;
  const int n1 = (int)(t / ((int64_t)N * M)) - M / 2;
  double s = 0.0;
  for (int n3 = -M / 2; n3 < M / 2; ++n3)
    s += U[n1 * n1 + n2 * n2 + n3 * n3] * cos2pi_frac((long long)m3 * n3, M);
  A1[t] = s;
}
// pass 2: A2[n1][m2][m3] = sum_{n2} A1[n1][n2][m3] cos(2 pi m2 n2 / M)
__global__ void k_t_pass2(const double* __restrict__ A1, double* __restrict__ A2, int M, int N) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)M * N * N) return;
  const int m3 = (int)(t % N);
  const int m2 = (int)((t / N) % N);
  const int i1 = (int)(t / ((int64_t)N * N));
  double s = 0.0;
  for (int i2 = 0; i2 < M; ++i2)
    s += A1[((int64_t)i1 * M + i2) * N + m3] * cos2pi_frac((long long)m2 * (i2 - M / 2), M);
  A2[t] = s;
}
// pass 3: T[m1][m2][m3] = M^-3 sum_{n1} A2[n1][m2][m3] cos(2 pi m1 n1 / M); also the full
// (2N-1)^3 export array by evenness
__global__ void k_t_pass3(const double* __restrict__ A2, double* __restrict__ Th,
                          double* __restrict__ Tfull, int M, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N * N) return;
  const int m3 = t % N, m2 = (t / N) % N, m1 = t / (N * N);
  double s = 0.0;
  for (int i1 = 0; i1 < M; ++i1)
    s += A2[((int64_t)i1 * N + m2) * N + m3] * cos2pi_frac((long long)m1 * (i1 - M / 2), M);
  s /= (double)M * M * M;
  Th[t] = s;
  const int W = 2 * N - 1;
  for (int sg = 0; sg < 8; ++sg) {
    const int p1 = (sg & 4) ? -m1 : m1, p2 = (sg & 2) ? -m2 : m2, p3 = (sg & 1) ? -m3 : m3;
    Tfull[((int64_t)(p1 + N - 1) * W + (p2 + N - 1)) * W + (p3 + N - 1)] = s;
  }
}

// T-hat passes over m_d >= 0 with weights w(0) = 1, w(m>0) = 2, xi in [0, 2N)
__global__ void k_th_pass(const double* __restrict__ in, double* __restrict__ out, int N,
                          int64_t outer, int inner_in, int inner_out) {
  // generic: out[o][xi][i] = sum_m w(m) in[o][m][i] cos(pi xi m / N); in has extent N along m,
  // out has extent 2N along xi; i runs over inner_in == inner_out elements
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int L = 2 * N;
  if (t >= outer * L * inner_out) return;
  const int i = (int)(t % inner_out);
  const int xi = (int)((t / inner_out) % L);
  const int64_t o = t / ((int64_t)inner_out * L);
  double s = 0.0;
  for (int m = 0; m < N; ++m)
    s += (m == 0 ? 1.0 : 2.0) * in[(o * N + m) * inner_in + i] * cos2pi_frac((long long)xi * m, L);
  out[t] = s;
}

template <typename T>
__global__ void k_that_store(const double* __restrict__ TH, T* __restrict__ that, int N) {
  // TH[xi1][xi2][xi3] natural order -> that[s3][s1][s2] parity-major, / (2N)^3
  const int L = 2 * N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L * L * L) return;
  const int x3 = t % L, x2 = (t / L) % L, x1 = t / (L * L);
  const int s1 = (x1 & 1) * N + x1 / 2, s2 = (x2 & 1) * N + x2 / 2, s3 = (x3 & 1) * N + x3 / 2;
  that[((int64_t)s3 * L + s1) * L + s2] = (T)(TH[t] / ((double)L * L * L));
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t compute_symbol(int N, double lk, double* T_dev, void* that_dev, bool fp64,
                           double* that_absmax_host, cudaStream_t s) {
  const int M = 3 * N;
  const double D = 2.0 * std::sqrt(3.0) * lk;
  const double c = 2.0 * M_PI / (6.0 * lk);
  const int qmax = 3 * (M / 2) * (M / 2);
  const int L = 2 * N;
  const GLRule gl = gauss_legendre();

  double *U = nullptr, *A1 = nullptr, *A2 = nullptr, *Th = nullptr, *B1 = nullptr, *B2 = nullptr,
         *TH = nullptr;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** p, size_t n) {
    if (e == cudaSuccess) e = cudaMallocAsync((void**)p, n * sizeof(double), s);
  };
  alloc(&U, qmax + 1);
  alloc(&A1, (size_t)M * M * N);
  alloc(&A2, (size_t)M * N * N);
  alloc(&Th, (size_t)N * N * N);
  alloc(&B1, (size_t)N * N * L);
  alloc(&B2, (size_t)N * L * L);
  alloc(&TH, (size_t)L * L * L);
  if (e == cudaSuccess) {
    k_uhat_table<<<nblk(qmax + 1, 128), 128, 0, s>>>(U, qmax, c, D, gl);
    k_t_pass1<<<nblk((int64_t)M * M * N, 256), 256, 0, s>>>(U, A1, M, N);
    k_t_pass2<<<nblk((int64_t)M * N * N, 256), 256, 0, s>>>(A1, A2, M, N);
    k_t_pass3<<<nblk((int64_t)N * N * N, 256), 256, 0, s>>>(A2, Th, T_dev, M, N);
    // T-hat: along m3 -> xi3, then m2 -> xi2, then m1 -> xi1
    k_th_pass<<<nblk((int64_t)N * N * L, 256), 256, 0, s>>>(Th, B1, N, (int64_t)N * N, 1, 1);
    k_th_pass<<<nblk((int64_t)N * L * L, 256), 256, 0, s>>>(B1, B2, N, N, L, L);
    k_th_pass<<<nblk((int64_t)L * L * L, 256), 256, 0, s>>>(B2, TH, N, 1, L * L, L * L);
    if (fp64)
      k_that_store<double><<<nblk((int64_t)L * L * L, 256), 256, 0, s>>>(TH, (double*)that_dev, N);
    else
      k_that_store<float><<<nblk((int64_t)L * L * L, 256), 256, 0, s>>>(TH, (float*)that_dev, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && that_absmax_host) {
    std::vector<double> h((size_t)L * L * L);
    e = cudaMemcpyAsync(h.data(), TH, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    double mx = 0.0;
    for (double v : h) mx = std::fmax(mx, std::fabs(v));
    *that_absmax_host = mx;
  }
  for (double* p : {U, A1, A2, Th, B1, B2, TH})
    if (p) cudaFreeAsync(p, s);
  return e;
}

}  // namespace chasm
