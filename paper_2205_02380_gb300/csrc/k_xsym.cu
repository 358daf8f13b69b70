// Per-x symbol table of the real form of Theta^T (k_theta_xs.cu).
//
// For the x point x the convolution kernel is S_m(x) = sum_A c_A T_m sin(a_A . m), with
// a_A = 2 (x - x_A) dk and c_A = -2 Z_A / (pi^2 hbar) (Eqs. 4.1, 4.6, sign of Eq. 2.3).  Its
// spectrum on the frequencies omega = (2 pi xi1 / 2N, 2 pi xi2 / 2N, pi (4j + 1) / (2N)) of the
// mixed circular/negacyclic embedding is i Im(S-hat), and with sin(a.m) sin(omega.m) =
// [cos((omega - a).m) - cos((omega + a).m)] / 2 and T even in every m_d (Eq. 4.7):
//   sigma(x)[j][xi1][xi2] = (2 / (2N)^3) Im S-hat = sum_A g_A [Tt(omega - a_A) - Tt(omega + a_A)],
//   Tt(theta) = sum_{m in [0, N)^3} T_m prod_d w(m_d) cos(theta_d m_d),  w(0) = 1, w(m > 0) = 2,
//   g_A = 2 Z_A / (pi^2 hbar (2N)^3).
// The product of cosines makes Tt separable: three contractions, over m3 for each (x3, sign)
// [R3], over m2 for each (x2, x3, sign) [R2], over m1 for each x point [the table].  The cosine
// tables and the first two contractions are FP64; the last runs in the storage precision (FP32
// for the mixed form: its rounding adds about 1e-7 relative to Theta) with FP64 inputs rounded
// once.  The table is written as [x][j][s1][s2], s = (xi mod 2) N + xi / 2 per dimension (the
// parity-major order of the slab phase of k_theta_xs.cu), or, for the packed single-precision
// kernel (xs_packed: k_theta_pk.cu), as [x][j][xi1 / 4][xi2][xi1 % 4] in natural frequency order
// (a lane of its column pass reads the four values of one 16-byte quad).
#include <cmath>

#include "internal.hpp"

namespace chasm {
namespace {

struct XsGeom {
  int N, L;
  int nx[3];
  double x_lo[3], h[3];
  double dk;
  int n_nuc;
  double pos[kMaxNuclei][3];
  double g[kMaxNuclei];
  int plain;   // 1: the sg = 1 terms are dropped (the spectrum of T itself, build_tkm_table)
};

// C[A][i][sg][xi][m] = scale w(m) cos(omega(xi) m - s a m), s = +1 (sg = 0) or -1 (sg = 1),
// a = 2 (x_{d,i} - x_{A,d}) dk; d < 2: xi in [0, 2N), omega = 2 pi xi / 2N; d = 2: xi = j in
// [0, N), omega = pi (4j + 1) / (2N).  scale = s g_A for d = 0, 1 otherwise.  The omega m part is
// reduced exactly (integer arithmetic) before sincospi.
__global__ void k_xs_costab(double* __restrict__ C, XsGeom G, int d, int nxi) {
  const int N = G.N;
  const int64_t total = (int64_t)G.n_nuc * G.nx[d] * 2 * nxi * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int m = (int)(t % N);
  int64_t r = t / N;
  const int xi = (int)(r % nxi);
  r /= nxi;
  const int sg = (int)(r % 2);
  r /= 2;
  const int i = (int)(r % G.nx[d]);
  const int A = (int)(r / G.nx[d]);
  const double s = sg == 0 ? 1.0 : -1.0;
  const double a = 2.0 * (G.x_lo[d] + i * G.h[d] - G.pos[A][d]) * G.dk;
  double sa, ca;
  if (d < 2) {
    const int rr = (xi * m) % G.L;
    sincospi(2.0 * rr / G.L, &sa, &ca);
  } else {
    const int M4 = 4 * N;
    const int rr = ((4 * xi + 1) * m) % M4;
    sincospi(2.0 * rr / M4, &sa, &ca);
  }
  double sb, cb;
  sincos(a * m, &sb, &cb);
  double v = (m == 0 ? 1.0 : 2.0) * (ca * cb + s * sa * sb);
  if (d == 0) v *= s * G.g[A];
  if (G.plain && sg == 1) v = 0.0;
  C[t] = v;
}

// R3[A][sg][i3][j][m1][m2] = sum_{m3} C3[A][i3][sg][j][m3] T[m1][m2][m3]  (T from the full
// (2N-1)^3 array, index m + N - 1)
__global__ void k_xs_r3(const double* __restrict__ C3, const double* __restrict__ Tfull,
                        double* __restrict__ R3, XsGeom G) {
  const int N = G.N, W = 2 * N - 1;
  const int64_t total = (int64_t)G.n_nuc * 2 * G.nx[2] * N * N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int m2 = (int)(t % N);
  const int m1 = (int)((t / N) % N);
  const int j = (int)((t / ((int64_t)N * N)) % N);
  const int64_t r = t / ((int64_t)N * N * N);   // (A, sg, i3)
  const int i3 = (int)(r % G.nx[2]);
  const int sg = (int)((r / G.nx[2]) % 2);
  const int A = (int)(r / (2 * G.nx[2]));
  const double* c = C3 + ((((int64_t)A * G.nx[2] + i3) * 2 + sg) * N + j) * N;
  const double* tq = Tfull + ((int64_t)(m1 + N - 1) * W + (m2 + N - 1)) * W + (N - 1);
  double acc = 0.0;
  for (int m3 = 0; m3 < N; ++m3) acc = fma(c[m3], tq[m3], acc);
  R3[t] = acc;
}

// R2[A][sg][ic][i3][m1][j][s2] = sum_{m2} C2[A][i2][sg][xi2(s2)][m2] R3[A][sg][i3][j][m1][m2],
// i2 = i2_0 + ic, ic in [0, c2)
__global__ void k_xs_r2(const double* __restrict__ C2, const double* __restrict__ R3,
                        double* __restrict__ R2, XsGeom G, int i2_0, int c2) {
  const int N = G.N, L = G.L;
  const int64_t per = (int64_t)N * N * L;   // (m1, j, s2)
  const int64_t total = (int64_t)G.n_nuc * 2 * c2 * G.nx[2] * per;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int s2 = (int)(t % L);
  const int j = (int)((t / L) % N);
  const int m1 = (int)((t / ((int64_t)L * N)) % N);
  int64_t r = t / per;
  const int i3 = (int)(r % G.nx[2]);
  r /= G.nx[2];
  const int ic = (int)(r % c2);
  r /= c2;
  const int sg = (int)(r % 2);
  const int A = (int)(r / 2);
  const int xi2 = 2 * (s2 % N) + s2 / N;
  const double* c = C2 + ((((int64_t)A * G.nx[1] + i2_0 + ic) * 2 + sg) * L + xi2) * N;
  const double* q = R3 + (((((int64_t)A * 2 + sg) * G.nx[2] + i3) * N + j) * N + m1) * N;
  double acc = 0.0;
  for (int m2 = 0; m2 < N; ++m2) acc = fma(c[m2], q[m2], acc);
  R2[t] = acc;
}

// One CTA per x point of the i2 chunk: sigma[x][j][s1][s2] = sum_{A, sg, m1} C1 R2, the last
// contraction in the accumulate type AT.  Thread = column (j, s2); the C1 rows of the CTA's x1
// sit in shared memory (read by all threads at once).
template <typename T, typename AT, int N>
__global__ void __launch_bounds__(256) k_xs_table(const double* __restrict__ C1,
                                                  const double* __restrict__ R2, T* __restrict__ sig,
                                                  XsGeom G, int i2_0, int c2) {
  constexpr int L = 2 * N;
  __shared__ AT c1s[2][L][N];
  const int nx3 = G.nx[2];
  const int blk = blockIdx.x;
  const int i3 = blk % nx3;
  const int ic = (blk / nx3) % c2;
  const int i1 = blk / (nx3 * c2);
  const int64_t xp = ((int64_t)i1 * G.nx[1] + (i2_0 + ic)) * nx3 + i3;
  T* out = sig + xp * (int64_t)(N * L * L);
  for (int A = 0; A < G.n_nuc; ++A) {
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * L * N; e += blockDim.x)
      (&c1s[0][0][0])[e] = (AT)C1[((int64_t)A * G.nx[0] + i1) * 2 * L * N + e];
    __syncthreads();
    const double* r2 = R2 + (((int64_t)A * 2 * c2 + ic) * nx3 + i3) * (int64_t)N * N * L;
    const int64_t sg_stride = (int64_t)c2 * nx3 * N * N * L;
    for (int col = threadIdx.x; col < N * L; col += blockDim.x) {
      AT r[2][N];
#pragma unroll
      for (int m = 0; m < N; ++m) {
        r[0][m] = (AT)r2[(int64_t)m * N * L + col];
        r[1][m] = (AT)r2[sg_stride + (int64_t)m * N * L + col];
      }
      const int j = col / L, s2 = col % L;
      for (int xi1 = 0; xi1 < L; ++xi1) {
        AT acc = 0;
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(c1s[0][xi1][m], r[0][m], acc);
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fma(c1s[1][xi1][m], r[1][m], acc);
        T* dst;
        if constexpr (xs_packed(sizeof(T) == 8, N)) {
          const int xi2 = 2 * (s2 % N) + s2 / N;
          dst = out + (((int64_t)j * (L / 4) + xi1 / 4) * L + xi2) * 4 + (xi1 & 3);
        } else {
          const int s1 = (xi1 & 1) * N + xi1 / 2;
          dst = out + ((int64_t)j * L + s1) * L + s2;
        }
        *dst = A == 0 ? (T)acc : (T)((AT)*dst + acc);
      }
    }
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, typename AT, int N>
cudaError_t launch_table(const double* C1, const double* R2, void* sig, const XsGeom& G, int i2_0,
                         int c2, cudaStream_t s) {
  const unsigned nb = (unsigned)(G.nx[0] * c2 * G.nx[2]);
  k_xs_table<T, AT, N><<<nb, 256, 0, s>>>(C1, R2, static_cast<T*>(sig), G, i2_0, c2);
  return cudaGetLastError();
}

cudaError_t table_chunk(bool fp64, int N, const double* C1, const double* R2, void* sig,
                        const XsGeom& G, int i2_0, int c2, cudaStream_t s) {
  switch (N) {
    case 8:
      return fp64 ? launch_table<double, double, 8>(C1, R2, sig, G, i2_0, c2, s)
                  : launch_table<float, float, 8>(C1, R2, sig, G, i2_0, c2, s);
    case 16:
      return fp64 ? launch_table<double, double, 16>(C1, R2, sig, G, i2_0, c2, s)
                  : launch_table<float, float, 16>(C1, R2, sig, G, i2_0, c2, s);
    case 32:
      return fp64 ? launch_table<double, double, 32>(C1, R2, sig, G, i2_0, c2, s)
                  : launch_table<float, float, 32>(C1, R2, sig, G, i2_0, c2, s);
  }
  return cudaErrorInvalidValue;
}

// the three cosine tables, R3, then per chunk of x2 planes R2 and the table
cudaError_t run_table(const XsGeom& G, bool fp64, const double* Tfull, void* sig, cudaStream_t s) {
  const int N = G.N, L = G.L;
  const int64_t n1 = (int64_t)G.n_nuc * G.nx[0] * 2 * L * N;
  const int64_t n2 = (int64_t)G.n_nuc * G.nx[1] * 2 * L * N;
  const int64_t n3 = (int64_t)G.n_nuc * G.nx[2] * 2 * N * N;
  const int64_t nr3 = (int64_t)G.n_nuc * 2 * G.nx[2] * N * N * N;
  const int64_t per_i2 = (int64_t)G.n_nuc * 2 * G.nx[2] * N * N * L;   // R2 doubles per x2 plane
  const int64_t cap = (int64_t)32 << 20;                                  // 256 MB of R2 per chunk
  const int c2 = (int)std::max<int64_t>(1, std::min<int64_t>(G.nx[1], cap / per_i2));

  double *C1 = nullptr, *C2 = nullptr, *C3 = nullptr, *R3 = nullptr, *R2 = nullptr;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** p, int64_t n) {
    if (e == cudaSuccess) e = cudaMallocAsync((void**)p, (size_t)n * sizeof(double), s);
  };
  alloc(&C1, n1);
  alloc(&C2, n2);
  alloc(&C3, n3);
  alloc(&R3, nr3);
  alloc(&R2, per_i2 * c2);
  if (e == cudaSuccess) {
    k_xs_costab<<<nblk(n1, 256), 256, 0, s>>>(C1, G, 0, L);
    k_xs_costab<<<nblk(n2, 256), 256, 0, s>>>(C2, G, 1, L);
    k_xs_costab<<<nblk(n3, 256), 256, 0, s>>>(C3, G, 2, N);
    k_xs_r3<<<nblk(nr3, 256), 256, 0, s>>>(C3, Tfull, R3, G);
    e = cudaGetLastError();
  }
  for (int i2 = 0; e == cudaSuccess && i2 < G.nx[1]; i2 += c2) {
    const int cc = std::min(c2, G.nx[1] - i2);
    k_xs_r2<<<nblk(per_i2 * cc, 256), 256, 0, s>>>(C2, R3, R2, G, i2, cc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = table_chunk(fp64, N, C1, R2, sig, G, i2, cc, s);
  }
  for (double* p : {C1, C2, C3, R3, R2})
    if (p) cudaFreeAsync(p, s);
  return e;
}

}  // namespace

size_t xs_table_bytes(int nk, int64_t nxp, size_t elt) { return (size_t)nxp * 4 * nk * nk * nk * elt; }

cudaError_t build_xs_table(const Handle& H, void* sig, cudaStream_t s) {
  XsGeom G{};
  const int N = H.g.nk, L = 2 * N;
  G.N = N;
  G.L = L;
  for (int d = 0; d < 3; ++d) {
    G.nx[d] = H.g.nx[d];
    G.x_lo[d] = H.g.x_lo[d];
    G.h[d] = H.g.h[d];
  }
  G.dk = H.g.dk;
  G.n_nuc = (int)H.nuclei.size();
  if (G.n_nuc < 1 || G.n_nuc > kMaxNuclei || !H.d_T) return cudaErrorInvalidValue;
  for (int a = 0; a < G.n_nuc; ++a) {
    for (int d = 0; d < 3; ++d) G.pos[a][d] = H.nuclei[a].pos[d];
    G.g[a] = 2.0 * H.nuclei[a].charge / (M_PI * M_PI * H.hbar * (double)L * L * L);
  }
  return run_table(G, H.fp64, H.d_T, sig, s);
}

// One x point at the (virtual) nucleus (a = 0), only the sg = 0 terms: sum_m T_m prod_d w(m_d)
// cos(omega_d m_d) = sum over all m in (-N, N)^3 of T_m e^{-i omega . m} (T even in every m_d),
// times 2 / (2N)^3 as the per-x table carries.
cudaError_t build_tkm_table(const Handle& H, void* out, cudaStream_t s) {
  XsGeom G{};
  const int N = H.g.nk, L = 2 * N;
  G.N = N;
  G.L = L;
  for (int d = 0; d < 3; ++d) {
    G.nx[d] = 1;
    G.x_lo[d] = 0.0;
    G.h[d] = 1.0;
  }
  G.dk = H.g.dk;
  G.n_nuc = 1;
  G.g[0] = 2.0 / ((double)L * L * L);
  G.plain = 1;
  if (!H.d_T) return cudaErrorInvalidValue;
  return run_table(G, H.fp64, H.d_T, out, s);
}

}  // namespace chasm
