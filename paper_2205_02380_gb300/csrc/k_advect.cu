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
// One thread owns one line: fixed k (the contiguous index, so a warp reads consecutive k and every
// load/store is a coalesced transaction) and fixed other two x indices; in the FP32 register
// kernel a thread owns the lines of two adjacent k and moves both with 8-byte accesses (each warp
// access 256 contiguous bytes, as in FP64).  The thread loads its nx values, forms the PMBC
// closure phi_L, phi_R, runs the constant-LU Thomas sweep, evaluates the 4-tap stencil and writes
// the nx new values back over the old ones (no other thread touches the line, so in place is
// safe).
//
// Closure precision.  FP64 form: native FP64.  FP32-mixed form: the closure dot products are
// accumulated in compensated FP32-pair arithmetic (error-free products by FMA, Knuth's two-sum;
// about 48 significant bits), i.e. at FP64-class precision without the FP64 pipe, which on GB300
// delivers 1/64 of the FP32 rate and otherwise bounds this pass.  Everything else is FP32.
//
// Two kernels: k_advect_reg keeps the line in registers (line length a compile-time constant
// from {16, 24, 32, 48, 64} and integer shift in [-2, 1], the usual case since |alpha| < 1);
// k_advect_smem is the general fallback with the line in shared memory (column layout, element
// e of thread t at e*B + t, conflict-free).
#include <cstring>

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
  int J;              // stencil length (<= n); the coefficient arrays are zero-padded to n
  double h;
  float hf, h2f;      // h and 2h rounded to FP32 (FP32-mixed closure terms)
  const T* clos;      // closure coefficients (see ClosureFmt)
  const T* cprime;    // Thomas c'_i, i = 0..N
  const T* mult;      // Thomas 1/(b_i - a_i c'_{i-1}), i = 0..N
  const T* w;         // [nk][4] (b4, b3, b2, b1)
  const int* ns;      // [nk] floor(alpha)
};

// ---- closure accumulators ----
// FP64: c+ at clos[j], c- at clos[n + j].
// FP32: c+ hi/lo at clos[j], clos[n + j]; c- hi/lo at clos[2n + j], clos[3n + j].
struct DF {           // unevaluated sum hi + lo
  float hi, lo;
};
__device__ __forceinline__ void df_acc(DF& s, float x, float chi, float clo) {
  const float p = x * chi;
  float e = fmaf(x, chi, -p);          // x * chi = p + e exactly
  e = fmaf(x, clo, e);
  const float t = s.hi + p;            // two-sum s.hi + p = t + err
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + e;
}

template <typename T>
struct Closure;

template <>
struct Closure<double> {
  double L = 0.0, R = 0.0;
  __device__ __forceinline__ void add(const double* c, int n, int j, double phiL, double phiR) {
    L = fma(__ldg(c + j), phiL, L);
    R = fma(__ldg(c + n + j), phiR, R);
  }
  // 3 phi_0 + h phi_L, 3 phi_N - h phi_R, and the ghost offsets 2 h phi_L, 2 h phi_R
  __device__ __forceinline__ double d0(double phi0, double h) const { return 3.0 * phi0 + h * L; }
  __device__ __forceinline__ double dN(double phiN, double h) const { return 3.0 * phiN - h * R; }
  __device__ __forceinline__ double gl(double eta1, double h) const { return eta1 - 2.0 * h * L; }
  __device__ __forceinline__ double gr(double etaNm1, double h) const { return etaNm1 + 2.0 * h * R; }
};

template <>
struct Closure<float> {
  DF L{0.f, 0.f}, R{0.f, 0.f};
  __device__ __forceinline__ void add(const float* c, int n, int j, float phiL, float phiR) {
    df_acc(L, phiL, __ldg(c + j), __ldg(c + n + j));
    df_acc(R, phiR, __ldg(c + 2 * n + j), __ldg(c + 3 * n + j));
  }
  __device__ __forceinline__ float d0(float phi0, float hf) const {
    return fmaf(hf, L.hi, fmaf(hf, L.lo, 3.0f * phi0));
  }
  __device__ __forceinline__ float dN(float phiN, float hf) const {
    return fmaf(-hf, R.hi, fmaf(-hf, R.lo, 3.0f * phiN));
  }
  __device__ __forceinline__ float gl(float eta1, float h2f) const {
    return fmaf(-h2f, L.hi, fmaf(-h2f, L.lo, eta1));
  }
  __device__ __forceinline__ float gr(float etaNm1, float h2f) const {
    return fmaf(h2f, R.hi, fmaf(h2f, R.lo, etaNm1));
  }
};

// Closure stencils and Thomas factors of the register kernel, passed by value in the kernel's
// parameter block: every index is a compile-time constant there, so each coefficient is a
// constant-bank operand of its FMA instead of a load per line.
constexpr int kRegMaxNx = 64;
template <typename T>
struct AdvTabs;
template <>
struct AdvTabs<float> {
  float c[4][kRegMaxNx];     // c+ hi, c+ lo, c- hi, c- lo (zero-padded)
  float lu[2][kRegMaxNx];    // c'_i, 1 / pivot_i
};
template <>
struct AdvTabs<double> {
  double c[2][kRegMaxNx];    // c+, c-
  double lu[2][kRegMaxNx];
};

// The closure stencils decay like |sqrt(3) - 2|^j (about 0.27^j): from tap kClosHead on the
// coefficients are below 1e-5 of the leading ones, so the FP32 rounding of each tail product
// (added to the low part) is below about 1e-12 of the data's scale over h; the leading taps are
// accumulated error-free.
constexpr int kClosHead = 10;
template <int NX>
__device__ __forceinline__ void closure_tab(Closure<float>& cl, const AdvTabs<float>& tb, int j,
                                            float phiL, float phiR) {
  if (j < kClosHead) {
    df_acc(cl.L, phiL, tb.c[0][j], tb.c[1][j]);
    df_acc(cl.R, phiR, tb.c[2][j], tb.c[3][j]);
  } else {
    cl.L.lo = fmaf(phiL, tb.c[0][j], cl.L.lo);
    cl.R.lo = fmaf(phiR, tb.c[2][j], cl.R.lo);
  }
}
template <int NX>
__device__ __forceinline__ void closure_tab(Closure<double>& cl, const AdvTabs<double>& tb, int j,
                                            double phiL, double phiR) {
  cl.L = fma(tb.c[0][j], phiL, cl.L);
  cl.R = fma(tb.c[1][j], phiR, cl.R);
}

// the h arguments of the closure terms in the storage precision
template <typename T>
__device__ __forceinline__ T hval(const AdvParams<T>& p);
template <>
__device__ __forceinline__ double hval<double>(const AdvParams<double>& p) { return p.h; }
template <>
__device__ __forceinline__ float hval<float>(const AdvParams<float>& p) { return p.hf; }
template <typename T>
__device__ __forceinline__ T h2val(const AdvParams<T>& p);
template <>
__device__ __forceinline__ double h2val<double>(const AdvParams<double>& p) { return p.h; }
template <>
__device__ __forceinline__ float h2val<float>(const AdvParams<float>& p) { return p.h2f; }

template <typename T>
__device__ __forceinline__ void line_setup(const AdvParams<T>& p, int64_t line, T*& src, int& kd) {
  const int64_t kidx = line % p.kvol;
  const int64_t outer = line / p.kvol;
  const int64_t ia = outer / p.n_b, ib = outer % p.n_b;
  src = p.f + ia * p.s_a + ib * p.s_b + kidx;
  kd = (int)((kidx / p.kdiv) % p.nk);
}

// ---- register kernel ----
// out_j = w0 eta_{j-S-2} + w1 eta_{j-S-1} + w2 eta_{j-S} + w3 eta_{j-S+1}; slot of eta_nu = nu+1.
// st(j, out_j) writes the result (global memory or a shared-memory tile).
template <typename T, int NX, int S, class St>
__device__ __forceinline__ void eval_line(const T (&v)[NX + 2], T w0, T w1, T w2, T w3, St&& st) {
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T acc = (T)0;
    const int s0 = j - S - 1;   // slot of eta_{j-S-2}
    if (s0 >= 0 && s0 <= NX + 1) acc = w0 * v[s0];
    if (s0 + 1 >= 0 && s0 + 1 <= NX + 1) acc = fma(w1, v[s0 + 1], acc);
    if (s0 + 2 >= 0 && s0 + 2 <= NX + 1) acc = fma(w2, v[s0 + 2], acc);
    if (s0 + 3 >= 0 && s0 + 3 <= NX + 1) acc = fma(w3, v[s0 + 3], acc);
    st(j, acc);
  }
}

// One line in registers: closure, Thomas sweep and ghosts; v holds the spline coefficients
// eta_{-1..N+1} afterwards.  JC: the number of closure taps evaluated (the stencil is zero beyond
// the launch's J <= JC).
template <typename T, int NX, int JC>
__device__ __forceinline__ void solve_line(const AdvParams<T>& p, const AdvTabs<T>& tb, T (&v)[NX + 2]) {
  constexpr int N = NX - 1;
  Closure<T> cl;
#pragma unroll
  for (int j = 0; j < JC; ++j) closure_tab<NX>(cl, tb, j, v[j + 1], v[N - j + 1]);

  T dp = (T)cl.d0(v[1], hval(p)) * tb.lu[1][0];
  v[1] = dp;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    dp = ((T)6 * v[i + 1] - dp) * tb.lu[1][i];
    v[i + 1] = dp;
  }
  dp = ((T)cl.dN(v[N + 1], hval(p)) - dp) * tb.lu[1][N];
  v[N + 1] = dp;
#pragma unroll
  for (int i = N - 1; i >= 0; --i) v[i + 1] = v[i + 1] - tb.lu[0][i] * v[i + 2];
  v[0] = (T)cl.gl(v[2], h2val(p));
  v[N + 2] = (T)cl.gr(v[N], h2val(p));
}

// the 4-tap evaluation of two lines with the same integer shift S (weights wa, wb), written
// together by st(j, out_a, out_b)
template <typename T, int NX, int S, class St>
__device__ __forceinline__ void eval_line2(const T (&va)[NX + 2], const T (&vb)[NX + 2], const T (&wa)[4],
                                           const T (&wb)[4], St&& st) {
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T a = (T)0, b = (T)0;
    const int s0 = j - S - 1;
    if (s0 >= 0 && s0 <= NX + 1) {
      a = wa[0] * va[s0];
      b = wb[0] * vb[s0];
    }
    if (s0 + 1 >= 0 && s0 + 1 <= NX + 1) {
      a = fma(wa[1], va[s0 + 1], a);
      b = fma(wb[1], vb[s0 + 1], b);
    }
    if (s0 + 2 >= 0 && s0 + 2 <= NX + 1) {
      a = fma(wa[2], va[s0 + 2], a);
      b = fma(wb[2], vb[s0 + 2], b);
    }
    if (s0 + 3 >= 0 && s0 + 3 <= NX + 1) {
      a = fma(wa[3], va[s0 + 3], a);
      b = fma(wb[3], vb[s0 + 3], b);
    }
    st(j, a, b);
  }
}

// solve_line, then the 4-tap evaluation at the feet of line k index kd, written by st
template <typename T, int NX, int JC, class St>
__device__ __forceinline__ void solve_eval_line(const AdvParams<T>& p, const AdvTabs<T>& tb,
                                                T (&v)[NX + 2], int kd, St&& st) {
  solve_line<T, NX, JC>(p, tb, v);
  const int sh = __ldg(p.ns + kd);
  const T w0 = __ldg(p.w + 4 * kd + 0), w1 = __ldg(p.w + 4 * kd + 1);
  const T w2 = __ldg(p.w + 4 * kd + 2), w3 = __ldg(p.w + 4 * kd + 3);
  switch (sh) {
    case -2: eval_line<T, NX, -2>(v, w0, w1, w2, w3, st); break;
    case -1: eval_line<T, NX, -1>(v, w0, w1, w2, w3, st); break;
    case 0: eval_line<T, NX, 0>(v, w0, w1, w2, w3, st); break;
    default: eval_line<T, NX, 1>(v, w0, w1, w2, w3, st); break;
  }
}

// FP64 form: one line per thread.  FP32-mixed form: two adjacent k (lines l and l + 1 share the
// x indices) per thread, loaded with 8-byte accesses so each thread keeps twice the bytes in
// flight, and stored with 8-byte accesses when both lines have the same integer shift (always
// for the x1 and x2 passes, whose shift depends on k1 or k2 only).
template <typename T, int NX, int JC>
__global__ void __launch_bounds__(kAdvectThreads) k_advect_reg(AdvParams<T> p, const AdvTabs<T> tb) {
  constexpr int LPT = sizeof(T) == 4 ? 2 : 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t * LPT >= p.n_lines) return;
  T* src;
  int kd;
  line_setup(p, t * LPT, src, kd);
  if constexpr (LPT == 1) {
    T v[NX + 2];   // slot nu + 1 holds eta_nu (phi_j before the solve)
#pragma unroll
    for (int j = 0; j < NX; ++j) v[j + 1] = src[(int64_t)j * p.s_d];
    solve_eval_line<T, NX, JC>(p, tb, v, kd, [&](int j, T o) { src[(int64_t)j * p.s_d] = o; });
  } else {
    T v0[NX + 2], v1[NX + 2];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      const float2 q = *reinterpret_cast<const float2*>(src + (int64_t)j * p.s_d);
      v0[j + 1] = q.x;
      v1[j + 1] = q.y;
    }
    int kd1;
    T* src1;
    line_setup(p, t * LPT + 1, src1, kd1);
    const int sh0 = __ldg(p.ns + kd), sh1 = __ldg(p.ns + kd1);
    if (sh0 != sh1) {   // rare: the two k straddle an integer shift
      solve_eval_line<T, NX, JC>(p, tb, v0, kd, [&](int j, T o) { src[(int64_t)j * p.s_d] = o; });
      solve_eval_line<T, NX, JC>(p, tb, v1, kd1, [&](int j, T o) { src1[(int64_t)j * p.s_d] = o; });
      return;
    }
    solve_line<T, NX, JC>(p, tb, v0);
    solve_line<T, NX, JC>(p, tb, v1);
    T wa[4], wb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      wa[c] = __ldg(p.w + 4 * kd + c);
      wb[c] = __ldg(p.w + 4 * kd1 + c);
    }
    auto st = [&](int j, T a, T b) { *reinterpret_cast<float2*>(src + (int64_t)j * p.s_d) = make_float2(a, b); };
    switch (sh0) {
      case -2: eval_line2<T, NX, -2>(v0, v1, wa, wb, st); break;
      case -1: eval_line2<T, NX, -1>(v0, v1, wa, wb, st); break;
      case 0: eval_line2<T, NX, 0>(v0, v1, wa, wb, st); break;
      default: eval_line2<T, NX, 1>(v0, v1, wa, wb, st); break;
    }
  }
}

// ---- shared-memory kernel (any line length, any shift) ----
template <typename T>
__global__ void __launch_bounds__(kAdvectThreads) k_advect_smem(AdvParams<T> p) {
  extern __shared__ unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
  const int B = blockDim.x;
  const int64_t line = (int64_t)blockIdx.x * B + threadIdx.x;
  if (line >= p.n_lines) return;
  T* src;
  int kd;
  line_setup(p, line, src, kd);
  const int n = p.n, N = p.n - 1;

#pragma unroll 8
  for (int j = 0; j < n; ++j) buf[(j + 1) * B] = src[(int64_t)j * p.s_d];

  Closure<T> cl;
  for (int j = 0; j < p.J; ++j) cl.add(p.clos, n, j, buf[(j + 1) * B], buf[(N - j + 1) * B]);

  T dp = (T)cl.d0(buf[B], hval(p)) * __ldg(p.mult);
  buf[B] = dp;
  for (int i = 1; i < N; ++i) {
    dp = ((T)6 * buf[(i + 1) * B] - dp) * __ldg(p.mult + i);
    buf[(i + 1) * B] = dp;
  }
  dp = ((T)cl.dN(buf[(N + 1) * B], hval(p)) - dp) * __ldg(p.mult + N);
  buf[(N + 1) * B] = dp;
  T e = dp;
  for (int i = N - 1; i >= 0; --i) {
    e = buf[(i + 1) * B] - __ldg(p.cprime + i) * e;
    buf[(i + 1) * B] = e;
  }
  buf[0] = (T)cl.gl(buf[2 * B], h2val(p));
  buf[(N + 2) * B] = (T)cl.gr(buf[N * B], h2val(p));

  const int sh = __ldg(p.ns + kd);
  const T w0 = __ldg(p.w + 4 * kd + 0), w1 = __ldg(p.w + 4 * kd + 1);
  const T w2 = __ldg(p.w + 4 * kd + 2), w3 = __ldg(p.w + 4 * kd + 3);
  for (int j = 0; j < n; ++j) {
    const int nu0 = j - sh - 2;   // first tap index
    T acc = (T)0;
    if (nu0 >= -1 && nu0 <= N + 1) acc = w0 * buf[(nu0 + 1) * B];
    if (nu0 + 1 >= -1 && nu0 + 1 <= N + 1) acc = fma(w1, buf[(nu0 + 2) * B], acc);
    if (nu0 + 2 >= -1 && nu0 + 2 <= N + 1) acc = fma(w2, buf[(nu0 + 3) * B], acc);
    if (nu0 + 3 >= -1 && nu0 + 3 <= N + 1) acc = fma(w3, buf[(nu0 + 4) * B], acc);
    src[(int64_t)j * p.s_d] = acc;
  }
}

// ---- patches (p > 1): Sec. 3.1.2 steps (1)-(5) and the interpolation with correction of
// Sec. 3.1.3, one line per thread in shared memory (column layout) ----
template <typename T>
struct PatchArgs {
  int P, M, nb, W;
  const T* win;   // closure windows: FP64 [(P+1)][W]; FP32 [(P+1)][2][W] (hi, lo)
  const T* lu;    // [c' (M+1) | 1/pivot (M+1)] of the (M+1)-node patch system
};

// closure value of boundary b = sum over its window of coefficient * phi, hi/lo parts
__device__ __forceinline__ void patch_closure(const PatchArgs<double>& q, const double* buf, int B, int N,
                                              int b, double& hi, double& lo) {
  double acc = 0.0;
  for (int i = 0; i < q.W; ++i) {
    const int node = b * q.M - q.nb + i;
    if (node >= 0 && node <= N) acc = fma(__ldg(q.win + (size_t)b * q.W + i), buf[(size_t)node * B], acc);
  }
  hi = acc;
  lo = 0.0;
}
__device__ __forceinline__ void patch_closure(const PatchArgs<float>& q, const float* buf, int B, int N,
                                              int b, float& hi, float& lo) {
  DF acc{0.f, 0.f};
  const float* w = q.win + (size_t)b * 2 * q.W;
  for (int i = 0; i < q.W; ++i) {
    const int node = b * q.M - q.nb + i;
    if (node >= 0 && node <= N) df_acc(acc, buf[(size_t)node * B], __ldg(w + i), __ldg(w + q.W + i));
  }
  hi = acc.hi;
  lo = acc.lo;
}

template <typename T>
__global__ void __launch_bounds__(kAdvectThreads) k_advect_patches(AdvParams<T> p, PatchArgs<T> q) {
  extern __shared__ unsigned char smem_raw[];
  const int B = blockDim.x;
  const int n = p.n, N = n - 1, P = q.P, M = q.M;
  T* buf = reinterpret_cast<T*>(smem_raw) + threadIdx.x;   // phi_j at buf[j B]
  T* cvh = buf + (size_t)n * B;                             // closure b: cvh[b B], cvl[b B]
  T* cvl = cvh + (size_t)(P + 1) * B;
  T* eta = cvl + (size_t)(P + 1) * B;                       // eta^(l)_nu at eta[(l (M+3) + nu + 1) B]
  const int64_t line = (int64_t)blockIdx.x * B + threadIdx.x;
  if (line >= p.n_lines) return;
  T* src;
  int kd;
  line_setup(p, line, src, kd);
  for (int j = 0; j < n; ++j) buf[(size_t)j * B] = src[(int64_t)j * p.s_d];
  for (int b = 0; b <= P; ++b) {
    T hi, lo;
    patch_closure(q, buf, B, N, b, hi, lo);
    cvh[(size_t)b * B] = hi;
    cvl[(size_t)b * B] = lo;
  }
  const T* cprime = q.lu;
  const T* mult = q.lu + (M + 1);
  for (int l = 0; l < P; ++l) {
    const T* ph = buf + (size_t)l * M * B;
    T* e = eta + (size_t)l * (M + 3) * B;
    Closure<T> cl;   // phi_L of patch l in cl.L, phi_R in cl.R
    if constexpr (sizeof(T) == 4) {
      cl.L = DF{cvh[(size_t)l * B], cvl[(size_t)l * B]};
      cl.R = DF{cvh[(size_t)(l + 1) * B], cvl[(size_t)(l + 1) * B]};
    } else {
      cl.L = cvh[(size_t)l * B];
      cl.R = cvh[(size_t)(l + 1) * B];
    }
    T dp = (T)cl.d0(ph[0], hval(p)) * __ldg(mult);
    e[B] = dp;
    for (int i = 1; i < M; ++i) {
      dp = ((T)6 * ph[(size_t)i * B] - dp) * __ldg(mult + i);
      e[(size_t)(i + 1) * B] = dp;
    }
    dp = ((T)cl.dN(ph[(size_t)M * B], hval(p)) - dp) * __ldg(mult + M);
    e[(size_t)(M + 1) * B] = dp;
    T nx = dp;
    for (int i = M - 1; i >= 0; --i) {
      nx = e[(size_t)(i + 1) * B] - __ldg(cprime + i) * nx;
      e[(size_t)(i + 1) * B] = nx;
    }
    e[0] = (T)cl.gl(e[2 * (size_t)B], h2val(p));
    e[(size_t)(M + 2) * B] = (T)cl.gr(e[(size_t)M * B], h2val(p));
  }
  const int sh = __ldg(p.ns + kd);
  const T w[4] = {__ldg(p.w + 4 * kd + 0), __ldg(p.w + 4 * kd + 1), __ldg(p.w + 4 * kd + 2),
                  __ldg(p.w + 4 * kd + 3)};
  for (int j = 0; j < n; ++j) {
    // patch of the foot x_j - (sh + a) h: floor((j - sh - 1) / M), clamped (left patch at a node)
    const int t = j - sh - 1;
    int l = t >= 0 ? t / M : -((-t + M - 1) / M);
    l = l < 0 ? 0 : (l > P - 1 ? P - 1 : l);
    const int nu0 = j - l * M - sh - 2;   // first tap, local index
    const T* e = eta + (size_t)l * (M + 3) * B;
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int nu = nu0 + c;
      if (nu >= -1 && nu <= M + 1) acc = fma(w[c], e[(size_t)(nu + 1) * B], acc);
    }
    src[(int64_t)j * p.s_d] = acc;
  }
}

template <typename T>
AdvParams<T> make_params(const Handle& H, void* f, int dim) {
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
  p.hf = (float)g.h[dim];
  p.h2f = (float)(2.0 * g.h[dim]);
  p.clos = static_cast<const T*>(H.d_clos[dim]);
  p.cprime = static_cast<const T*>(H.d_lu[dim]);
  p.mult = static_cast<const T*>(H.d_lu[dim]) + g.nx[dim];
  const T* wbase = static_cast<const T*>(H.adv.dev);
  p.w = wbase + (size_t)dim * g.nk * 4;
  p.ns = reinterpret_cast<const int*>(wbase + (size_t)3 * g.nk * 4) + dim * g.nk;
  return p;
}

// closure stencils and Thomas factors of dimension dim for the register kernels
template <typename T>
AdvTabs<T> make_tabs(const Handle& H, int dim) {
  const int n = H.g.nx[dim];
  AdvTabs<T> tb;
  std::memset(&tb, 0, sizeof(tb));
  const std::vector<double>& hc = H.h_clos[dim];
  const std::vector<double>& hl = H.h_lu[dim];
  for (int j = 0; j < n; ++j) {
    if constexpr (sizeof(T) == 4) {   // unevaluated float pairs hi + lo of the FP64 stencils
      tb.c[0][j] = (float)hc[j];
      tb.c[1][j] = (float)(hc[j] - (double)tb.c[0][j]);
      tb.c[2][j] = (float)hc[n + j];
      tb.c[3][j] = (float)(hc[n + j] - (double)tb.c[2][j]);
    } else {
      tb.c[0][j] = hc[j];
      tb.c[1][j] = hc[n + j];
    }
    tb.lu[0][j] = (T)hl[j];
    tb.lu[1][j] = (T)hl[n + j];
  }
  return tb;
}

// the register kernels apply: integer shifts in [-2, 1] and a compiled line length
bool reg_applies(const Handle& H, int dim) {
  return H.adv.ns_min[dim] >= -2 && H.adv.ns_max[dim] <= 1 && H.opt.patches[dim] <= 1 &&
         H.g.nx[dim] <= kRegMaxNx;
}

template <typename T>
cudaError_t launch_t(const Handle& H, void* f, int dim, cudaStream_t s) {
  const GridDesc& g = H.g;
  AdvParams<T> p = make_params<T>(H, f, dim);
  const int B = kAdvectThreads;
  const int P = H.opt.patches[dim];
  if (P > 1) {
    PatchArgs<T> q;
    q.P = P;
    q.M = (p.n - 1) / P;
    q.nb = H.opt.n_nb;
    q.W = 2 * q.nb + 1;
    q.win = static_cast<const T*>(H.d_pclos[dim]);
    q.lu = static_cast<const T*>(H.d_plu[dim]);
    const size_t elems = advect_smem_elems(p.n, P);
    const int Bp = advect_smem_threads(elems, sizeof(T));
    if (Bp == 0) return cudaErrorInvalidValue;
    k_advect_patches<T><<<(unsigned)((p.n_lines + Bp - 1) / Bp), Bp, elems * Bp * sizeof(T), s>>>(p, q);
    return cudaGetLastError();
  }
  if (reg_applies(H, dim)) {
    const int64_t lpt = sizeof(T) == 4 ? 2 : 1;   // kvol = nk^3 is even
    const unsigned rblocks = (unsigned)((p.n_lines / lpt + B - 1) / B);
    const AdvTabs<T> tb = make_tabs<T>(H, dim);
    // closure taps: the launch's J rounded up to a compiled bucket (the stencil is zero beyond J)
    const bool short_j = p.J <= 24 && p.n > 24;
#define CHASM_REG(NX)                                                                   \
  case NX:                                                                              \
    if (short_j && NX > 24)                                                             \
      k_advect_reg<T, NX, (NX > 24 ? 24 : NX)><<<rblocks, B, 0, s>>>(p, tb);            \
    else                                                                                \
      k_advect_reg<T, NX, NX><<<rblocks, B, 0, s>>>(p, tb);                             \
    return cudaGetLastError();
    switch (p.n) {
      CHASM_REG(16)
      CHASM_REG(24)
      CHASM_REG(32)
      CHASM_REG(48)
      CHASM_REG(64)
      default: break;
    }
#undef CHASM_REG
  }
  const size_t elems = advect_smem_elems(g.nx[dim], 1);
  const int Bs = advect_smem_threads(elems, sizeof(T));
  if (Bs == 0) return cudaErrorInvalidValue;
  k_advect_smem<T><<<(unsigned)((p.n_lines + Bs - 1) / Bs), Bs, elems * Bs * sizeof(T), s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t advect_prepare() {
  // up to kAdvectMaxSmem bytes of dynamic shared memory (fewer threads per block for long lines;
  // lines too long even for 32 threads are rejected at create time)
  cudaError_t e = cudaFuncSetAttribute(k_advect_smem<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kAdvectMaxSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_advect_smem<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kAdvectMaxSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_advect_patches<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdvectMaxSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_advect_patches<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdvectMaxSmem);
  return e;
}

cudaError_t launch_advect_dim(const Handle& H, void* f, int dim, cudaStream_t s) {
  return H.fp64 ? launch_t<double>(H, f, dim, s) : launch_t<float>(H, f, dim, s);
}

}  // namespace chasm
