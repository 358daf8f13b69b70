// Spatial advection A(tau): f(x, k) <- f(x - hbar k tau / m, k)   (Eq. 2.6, Sec. 3)
//
// The tensor-product spline of Eq. 3.9 and the 64-tap evaluation of Eq. 3.10 are computed in
// sum-factorised form: the 3-D operator is (E1 S1)(E2 S2)(E3 S3), where S_d is the PMBC-closed
// 1-D spline transform along x_d (Eq. 3.5 closure + Hermite-closed tridiagonal solve, step (5) of
// Sec. 3.1.2) and E_d the 4-tap evaluation at the feet x_j - alpha_d h_d (Eqs. 3.7-3.8).  Operators
// acting on different dimensions commute, so three in-place passes, one per x-dimension, give
// exactly the 64-term sum (up to rounding order) without ever storing the (N+3)^3 coefficient
// tensor.
//
// One thread owns one line: fixed k (the contiguous index, so a warp reads 32 consecutive k and
// every load/store is a coalesced 128-byte (FP32) or 256-byte (FP64) transaction) and fixed
// other two x indices.  The thread loads its nx values, forms the PMBC closure phi_L, phi_R in
// FP64, runs the constant-LU Thomas sweep, evaluates the 4-tap stencil and writes the nx new
// values back over the old ones (no other thread touches the line, so in place is safe).
// The line lives in shared memory in a column layout (element e of thread t at e*B + t), which
// is free of bank conflicts.
#include "internal.hpp"

namespace chasm {
namespace {

template <typename T>
struct AdvParams {
  T* f;
  int64_t n_lines;
  int64_t kvol;       // nk^3
  int64_t s_d;        // stride along the advected dimension
  int64_t s_a, s_b;   // strides of the two other x dimensions
  int n;              // points along the advected dimension
  int n_b;            // extent of the second "other" dimension
  int kdiv;           // k_d = (kidx / kdiv) % nk
  int nk;
  int J;              // stencil length
  double h;
  const double* cplus;
  const double* cminus;
  const T* cprime;    // Thomas c'_i, i = 0..N
  const T* mult;      // Thomas 1/(b_i - a_i c'_{i-1}), i = 0..N
  const T* w;         // [nk][4] (b4, b3, b2, b1)
  const int* ns;      // [nk] floor(alpha)
};

template <typename T>
__global__ void __launch_bounds__(kAdvectThreads) k_advect_dim(AdvParams<T> p) {
  extern __shared__ unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
  const int B = blockDim.x;
  const int64_t line = (int64_t)blockIdx.x * B + threadIdx.x;
  if (line >= p.n_lines) return;
  const int64_t kidx = line % p.kvol;
  const int64_t outer = line / p.kvol;
  const int64_t ia = outer / p.n_b, ib = outer % p.n_b;
  T* __restrict__ src = p.f + ia * p.s_a + ib * p.s_b + kidx;
  const int kd = (int)((kidx / p.kdiv) % p.nk);
  const int n = p.n, N = p.n - 1;

  // load phi_0..phi_N into the slots of eta_0..eta_N (slot of eta_nu is nu + 1)
#pragma unroll 8
  for (int j = 0; j < n; ++j) buf[(j + 1) * B] = src[(int64_t)j * p.s_d];

  // PMBC closure of the natural-BC global spline (Eq. 3.5), FP64 in both forms
  double phiL = 0.0, phiR = 0.0;
  for (int j = 0; j < p.J; ++j) {
    phiL = fma(__ldg(p.cplus + j), (double)buf[(j + 1) * B], phiL);
    phiR = fma(__ldg(p.cminus + j), (double)buf[(N - j + 1) * B], phiR);
  }

  // Hermite-closed system with eta_{-1}, eta_{N+1} eliminated:
  //   2 eta_0 + eta_1 = 3 phi_0 + h phi_L;  eta_{i-1} + 4 eta_i + eta_{i+1} = 6 phi_i;
  //   eta_{N-1} + 2 eta_N = 3 phi_N - h phi_R.   Constant LU (Thomas) factors from the plan.
  T dp = (T)(3.0 * (double)buf[B] + p.h * phiL) * __ldg(p.mult);
  buf[B] = dp;
  for (int i = 1; i < N; ++i) {
    dp = ((T)6 * buf[(i + 1) * B] - dp) * __ldg(p.mult + i);
    buf[(i + 1) * B] = dp;
  }
  dp = ((T)(3.0 * (double)buf[(N + 1) * B] - p.h * phiR) - dp) * __ldg(p.mult + N);
  buf[(N + 1) * B] = dp;
  T e = dp;
  for (int i = N - 1; i >= 0; --i) {
    e = buf[(i + 1) * B] - __ldg(p.cprime + i) * e;
    buf[(i + 1) * B] = e;
  }
  // eta_{-1} = eta_1 - 2 h phi_L,  eta_{N+1} = eta_{N-1} + 2 h phi_R   (Eq. 2.12)
  buf[0] = (T)((double)buf[2 * B] - 2.0 * p.h * phiL);
  buf[(N + 2) * B] = (T)((double)buf[N * B] + 2.0 * p.h * phiR);

  // 4-tap evaluation at x_j - alpha h: (eta_{j-n-2}, eta_{j-n-1}, eta_{j-n}, eta_{j-n+1}) .
  // (b4, b3, b2, b1)(alpha - n), n = floor(alpha); coefficients outside [-1, N+1] are zero.
  const int sh = __ldg(p.ns + kd);
  const T w0 = __ldg(p.w + 4 * kd + 0), w1 = __ldg(p.w + 4 * kd + 1);
  const T w2 = __ldg(p.w + 4 * kd + 2), w3 = __ldg(p.w + 4 * kd + 3);
  for (int j = 0; j < n; ++j) {
    const int nu0 = j - sh - 2;   // first tap index
    T acc = (T)0;
    if (nu0 >= -1 && nu0 <= N + 1) acc = w0 * buf[(nu0 + 1) * B];
    if (nu0 + 1 >= -1 && nu0 + 1 <= N + 1) acc += w1 * buf[(nu0 + 2) * B];
    if (nu0 + 2 >= -1 && nu0 + 2 <= N + 1) acc += w2 * buf[(nu0 + 3) * B];
    if (nu0 + 3 >= -1 && nu0 + 3 <= N + 1) acc += w3 * buf[(nu0 + 4) * B];
    src[(int64_t)j * p.s_d] = acc;
  }
}

template <typename T>
cudaError_t launch_t(const Handle& H, void* f, int dim, cudaStream_t s) {
  const GridDesc& g = H.g;
  AdvParams<T> p;
  p.f = static_cast<T*>(f);
  p.kvol = g.kvol;
  const int64_t s3 = g.kvol, s2 = (int64_t)g.nx[2] * g.kvol, s1 = (int64_t)g.nx[1] * s2;
  const int64_t strides[3] = {s1, s2, s3};
  const int other[3][2] = {{1, 2}, {0, 2}, {0, 1}};
  p.s_d = strides[dim];
  p.s_a = strides[other[dim][0]];
  p.s_b = strides[other[dim][1]];
  p.n_b = g.nx[other[dim][1]];
  p.n = g.nx[dim];
  p.n_lines = (int64_t)g.nx[other[dim][0]] * g.nx[other[dim][1]] * g.kvol;
  p.nk = g.nk;
  p.kdiv = dim == 0 ? g.nk * g.nk : (dim == 1 ? g.nk : 1);
  p.J = H.J[dim];
  p.h = g.h[dim];
  p.cplus = H.d_cplus[dim];
  p.cminus = H.d_cminus[dim];
  p.cprime = static_cast<const T*>(H.d_lu[dim]);
  p.mult = static_cast<const T*>(H.d_lu[dim]) + g.nx[dim];
  const T* wbase = static_cast<const T*>(H.adv.dev);
  p.w = wbase + (size_t)dim * g.nk * 4;
  p.ns = reinterpret_cast<const int*>(wbase + (size_t)3 * g.nk * 4) + dim * g.nk;
  const int B = kAdvectThreads;
  const size_t smem = (size_t)(g.nx[dim] + 2) * B * sizeof(T);
  const int64_t blocks = (p.n_lines + B - 1) / B;
  k_advect_dim<T><<<(unsigned)blocks, B, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t advect_prepare() {
  // up to (nx + 2) * 128 * 8 bytes of dynamic shared memory (nx <= 4096 is validated; lines
  // longer than the shared-memory limit are rejected at create time)
  cudaError_t e = cudaFuncSetAttribute(k_advect_dim<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kAdvectMaxSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_advect_dim<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kAdvectMaxSmem);
}

cudaError_t launch_advect_dim(const Handle& H, void* f, int dim, cudaStream_t s) {
  return H.fp64 ? launch_t<double>(H, f, dim, s) : launch_t<float>(H, f, dim, s);
}

}  // namespace chasm
