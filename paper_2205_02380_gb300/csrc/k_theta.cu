// Coulomb pseudodifferential operator by the truncated kernel method (Sec. 4).
//
//   Theta^T[u](x, k_p) = sum_A coef_A Im[ e^{2i(x-x_A).k_p} Phi_p ],
//   Phi_p = sum_q T_{p-q} u_q e^{-2i(x-x_A).k_q}                      (Eqs. 4.1, 4.5, 4.6)
//   coef_A = -(2 Z_A / (pi^2 hbar)) * c   (the Eq. 2.3 sign; c = Horner factor or 1)
//
// The linear convolution with T ((2N-1)^3 taps) is a circular convolution of length 2N per
// dimension (twofold zero padding, Sec. 4.1), diagonalised by the DFT: Phi = IDFT(T-hat DFT(g)).
// Each padded length-2N transform is split by frequency parity xi = 2j + r into two length-N
// transforms of the input twisted by tw_r[n] = e^{-i pi r n / N} (forward) and the same split
// on the inverse side with the conjugate twist, keeping only the N unpadded outputs.  All
// transforms are therefore length-N FFTs held entirely in registers (one line per thread,
// fully unrolled radix-2, no shared-memory traffic inside a transform).
//
// One CTA processes one x point at a time (persistent loop over x points), per nucleus:
//   Phase A  2N^2 jobs (k1, k2, r3): load the u line along k3, modulate, twist, FFT_N
//            -> G[s3][k1][k2] in the CTA's global scratch (s3 = r3 N + j3, parity-major).
//   Phase B  for each of the 2N slabs s3 (NG slabs in parallel, one group of 4N threads each):
//            B1 FFT along k2 (2N jobs), B2 along k1: FFT, multiply by T-hat, inverse FFT (4N
//            jobs), B3 inverse along k2 (2N jobs) and parity combine; in shared memory.
//   Phase C  2N^2 jobs: inverse FFT along k3, demodulate, Im, scale, accumulate per parity.
//   Phase D  out = base + acc_0 + acc_1 (coalesced).
// T-hat is stored in parity-major order [s3][s1][s2] with the 1/(2N)^3 normalisation folded in.
#include <cooperative_groups.h>

#include <cstdlib>
#include <cstring>

#include "internal.hpp"

namespace chasm {
namespace {

namespace cg = cooperative_groups;

template <typename T>
struct cpx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cpx<T> conjg(cpx<T> a) {
  return {a.re, -a.im};
}

// ---- twiddle tables: cos(2 pi k / 64), sin(2 pi k / 64), k = 0..63, evaluated at compile time
// by Taylor series after exact octant reduction (own implementation, no libm). ----
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double ce_sin_series(double x) {
  double t = x, s = x;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    s += t;
  }
  return s;
}
constexpr double ce_cos_series(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    s += t;
  }
  return s;
}
// cos(2 pi k / n) for n divisible by 8
constexpr double ce_cos2pi(int k, int n) {
  k %= n;
  if (k < 0) k += n;
  if (2 * k > n) k = n - k;          // cos is even: k in [0, n/2]
  double sg = 1.0;
  if (4 * k > n) {                    // cos(pi - a) = -cos(a)
    k = n / 2 - k;
    sg = -1.0;
  }
  // k in [0, n/4]
  return (8 * k > n) ? sg * ce_sin_series(2.0 * kPi * (n / 4 - k) / n)
                     : sg * ce_cos_series(2.0 * kPi * k / n);
}
constexpr double ce_sin2pi(int k, int n) { return ce_cos2pi(k - n / 4, n); }

#define CHASM_C4(f, b) f(b, 64), f(b + 1, 64), f(b + 2, 64), f(b + 3, 64)
#define CHASM_C16(f, b) CHASM_C4(f, b), CHASM_C4(f, b + 4), CHASM_C4(f, b + 8), CHASM_C4(f, b + 12)
#define CHASM_C64(f) CHASM_C16(f, 0), CHASM_C16(f, 16), CHASM_C16(f, 32), CHASM_C16(f, 48)
__constant__ double c_cos64d[64] = {CHASM_C64(ce_cos2pi)};
__constant__ double c_sin64d[64] = {CHASM_C64(ce_sin2pi)};
__constant__ float c_cos64f[64] = {CHASM_C64((float)ce_cos2pi)};
__constant__ float c_sin64f[64] = {CHASM_C64((float)ce_sin2pi)};

// FMA-form butterfly constants (Linzer and Feig, "Modified FFTs for fused multiply-add
// architectures", Math. Comp. 1993): the twiddle w = cos + i sin is written as m (1 + i r) or
// m (r + i) with |r| <= 1, so that a +- w x costs six FMAs.  big(k): |cos| >= |sin|.
__host__ __device__ constexpr bool lf_big(int k) { return (k % 32) <= 8 || (k % 32) >= 24; }
constexpr double lf_ratio(int k, int n) {
  return lf_big(k) ? ce_sin2pi(k, n) / ce_cos2pi(k, n) : ce_cos2pi(k, n) / ce_sin2pi(k, n);
}
constexpr double lf_scale(int k, int n) { return lf_big(k) ? ce_cos2pi(k, n) : ce_sin2pi(k, n); }
__constant__ double c_lfr64d[64] = {CHASM_C64(lf_ratio)};
__constant__ double c_lfm64d[64] = {CHASM_C64(lf_scale)};
__constant__ float c_lfr64f[64] = {CHASM_C64((float)lf_ratio)};
__constant__ float c_lfm64f[64] = {CHASM_C64((float)lf_scale)};
template <typename T>
__device__ __forceinline__ T lf_r(int k) {
  if constexpr (sizeof(T) == 4) return c_lfr64f[k];
  else return c_lfr64d[k];
}
template <typename T>
__device__ __forceinline__ T lf_m(int k) {
  if constexpr (sizeof(T) == 4) return c_lfm64f[k];
  else return c_lfm64d[k];
}

template <typename T>
__device__ __forceinline__ T tw_cos(int k);
template <typename T>
__device__ __forceinline__ T tw_sin(int k);
template <>
__device__ __forceinline__ float tw_cos<float>(int k) { return c_cos64f[k]; }
template <>
__device__ __forceinline__ float tw_sin<float>(int k) { return c_sin64f[k]; }
template <>
__device__ __forceinline__ double tw_cos<double>(int k) { return c_cos64d[k]; }
template <>
__device__ __forceinline__ double tw_sin<double>(int k) { return c_sin64d[k]; }

template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// In-register radix-2 DIT FFT of length N (N | 32).  Forward: X_j = sum_n x_n e^{-2 pi i jn/N};
// inverse (INV): unnormalised, e^{+2 pi i jn/N}.  Natural order in and out.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft(T (&re)[N], T (&im)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int j = bitrev<N>(i);
    if (j > i) {
      T t = re[i];
      re[i] = re[j];
      re[j] = t;
      t = im[i];
      im[i] = im[j];
      im[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < N; half <<= 1) {
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const int k64 = j * (32 / half);  // twiddle e^{-+2 pi i j / (2 half)} = entry k64 of 64
#pragma unroll
      for (int i = j; i < N; i += 2 * half) {
        const T xr = re[i + half], xi = im[i + half];
        if (k64 == 0 || k64 == 16) {
          T tr, ti;   // w = 1, or w = -i (forward) / +i (inverse)
          if (k64 == 0) {
            tr = xr;
            ti = xi;
          } else if (!INV) {
            tr = xi;
            ti = -xr;
          } else {
            tr = -xi;
            ti = xr;
          }
          re[i + half] = re[i] - tr;
          im[i + half] = im[i] - ti;
          re[i] += tr;
          im[i] += ti;
        } else {
          // w = cos -+ i sin = m (1 + i r) (big) or m (r + i); w x = m (p + i q)
          const T r = INV ? lf_r<T>(k64) : -lf_r<T>(k64);
          const T m = (lf_big(k64) || INV) ? lf_m<T>(k64) : -lf_m<T>(k64);
          T pr, qi;
          if (lf_big(k64)) {
            pr = fma(-xi, r, xr);
            qi = fma(xr, r, xi);
          } else {
            pr = fma(xr, r, -xi);
            qi = fma(xi, r, xr);
          }
          re[i + half] = fma(-m, pr, re[i]);
          re[i] = fma(m, pr, re[i]);
          im[i + half] = fma(-m, qi, im[i]);
          im[i] = fma(m, qi, im[i]);
        }
      }
    }
  }
}

// Twist by tw_1[n] = e^{-i pi n / N} = entry n*32/N of the 64-table (CONJ: e^{+i pi n/N}).
template <typename T, int N, bool CONJ>
__device__ __forceinline__ void twist(T (&re)[N], T (&im)[N]) {
#pragma unroll
  for (int n = 1; n < N; ++n) {
    const int k64 = n * (32 / N);
    const T c = tw_cos<T>(k64), s = CONJ ? tw_sin<T>(k64) : -tw_sin<T>(k64);
    const T a = re[n], b = im[n];
    re[n] = a * c - b * s;
    im[n] = a * s + b * c;
  }
}


// ---- scratch accesses with an L2 evict-last policy (the per-CTA spectrum of the global-scratch
// kernel is rewritten and reread within microseconds; u, f and out stream with evict-first) ----
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
template <typename T>
__device__ __forceinline__ cpx<T> ld_keep(const cpx<T>* p, uint64_t pol);
template <>
__device__ __forceinline__ cpx<float> ld_keep<float>(const cpx<float>* p, uint64_t pol) {
  cpx<float> v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.re), "=f"(v.im)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}
template <>
__device__ __forceinline__ cpx<double> ld_keep<double>(const cpx<double>* p, uint64_t pol) {
  cpx<double> v;
  asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.re), "=d"(v.im)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_keep(cpx<float>* p, cpx<float> v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.re), "f"(v.im),
               "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_keep(cpx<double>* p, cpx<double> v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.re), "d"(v.im),
               "l"(pol)
               : "memory");
}
// two adjacent single-precision complex values per access (16-byte aligned)
__device__ __forceinline__ void ld2_keep(const cpx<float>* p, uint64_t pol, cpx<float>& a, cpx<float>& b) {
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(a.re), "=f"(a.im), "=f"(b.re), "=f"(b.im)
               : "l"(p), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st2_keep(cpx<float>* p, cpx<float> a, cpx<float> b, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a.re),
               "f"(a.im), "f"(b.re), "f"(b.im), "l"(pol)
               : "memory");
}

// ---- Phase B building blocks shared by both kernels ----
// A slab group has GS = 2N threads: lane pair (2 row, 2 row + 1) holds the two frequency
// parities h = 0, 1 of one padded transform and combines them with warp shuffles, so no thread
// idles and no parity buffer is needed.  Groups synchronise among themselves only.
template <int GS>
__device__ __forceinline__ void group_sync(int grp) {
  if constexpr (GS <= 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(GS) : "memory");
}

// Layout of the group's slab buffer V (N rows of the two parity halves of a padded transform):
// element (row, h, j) at row * VR + h * VH + j with VH = 8 (mod 16) and VR odd, so that the lanes
// of a half-warp (8 rows x 2 parities) hit 16 different 8-byte banks in every sub-phase.
template <int N>
struct VLayout {
  static constexpr int VH = N >= 16 ? N + 8 : N;
  static constexpr int VR = VH + N + 1;
  static constexpr int D = N >= 16 ? 8 : N / 2;   // lane h keeps the elements m with (m / D) % 2 == h
  __device__ static constexpr int col(int c) { return (c / N) * VH + (c % N); }
};

// r = mine + partner's (parity partials of the same output vector); lane h stores the elements m
// with (m / D) % 2 == h of r at dst[m * stride], so the two lanes of a pair write rows D apart.
template <typename T, int N, bool GLOBAL = false>
__device__ __forceinline__ void pair_combine_store(const T (&re)[N], const T (&im)[N], int h,
                                                   cpx<T>* dst, int stride, uint64_t pol = 0) {
  constexpr int D = VLayout<N>::D;
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const int m0 = (i / D) * 2 * D + (i % D);   // kept by lane 0
    const int m1 = m0 + D;                      // kept by lane 1
    const T sre = h ? re[m0] : re[m1];
    const T sim = h ? im[m0] : im[m1];
    const T rre = __shfl_xor_sync(0xffffffffu, sre, 1);
    const T rim = __shfl_xor_sync(0xffffffffu, sim, 1);
    const T kre = h ? re[m1] : re[m0];
    const T kim = h ? im[m1] : im[m0];
    if constexpr (GLOBAL)
      st_keep(dst + (h ? m1 : m0) * stride, {kre + rre, kim + rim}, pol);
    else
      dst[(h ? m1 : m0) * stride] = {kre + rre, kim + rim};
  }
}

// The same into a contiguous single-precision global row (stride 1): the two elements m, m + 1 a
// lane keeps are written by one 16-byte store.
template <int N>
__device__ __forceinline__ void pair_combine_store_row(const float (&re)[N], const float (&im)[N],
                                                       int h, cpx<float>* dst, uint64_t pol) {
  constexpr int D = VLayout<N>::D;
  static_assert(D % 2 == 0, "element pairs stay within a lane's run");
#pragma unroll
  for (int i = 0; i < N / 2; i += 2) {
    const int m0 = (i / D) * 2 * D + (i % D);
    const int m1 = m0 + D;
    cpx<float> r[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float sre = h ? re[m0 + e] : re[m1 + e];
      const float sim = h ? im[m0 + e] : im[m1 + e];
      const float rre = __shfl_xor_sync(0xffffffffu, sre, 1);
      const float rim = __shfl_xor_sync(0xffffffffu, sim, 1);
      const float kre = h ? re[m1 + e] : re[m0 + e];
      const float kim = h ? im[m1 + e] : im[m0 + e];
      r[e] = {kre + rre, kim + rim};
    }
    st2_keep(dst + (h ? m1 : m0), r[0], r[1], pol);
  }
}

// The 2-D padded convolution of one slab s3 (fixed k3-frequency) in place: Gs holds the N x N
// complex k3-spectrum (row stride SR) on entry and Phi's k3-spectrum on exit.  V is the group's
// N x (2N + 1) complex buffer.  th is T-hat[s3] (parity-major [s1][s2], row length 2N).
template <typename T, int N, int GS, int SR, bool GLOBAL>
__device__ __forceinline__ void slab_conv(cpx<T>* Gs, cpx<T>* V, const T* __restrict__ th, int tg,
                                          int grp, uint64_t pol) {
  constexpr int L = 2 * N;
  using VL = VLayout<N>;
  const int h = tg & 1, row = tg >> 1;
  {  // B1: forward along k2 of row k1 = row, parity h
    T re[N], im[N];
#pragma unroll
    for (int n = 0; n < N; n += 2) {
      cpx<T> a, b;
      if constexpr (GLOBAL && sizeof(T) == 4) {
        ld2_keep(Gs + row * SR + n, pol, a, b);
      } else if constexpr (GLOBAL) {
        a = ld_keep<T>(Gs + row * SR + n, pol);
        b = ld_keep<T>(Gs + row * SR + n + 1, pol);
      } else {
        a = Gs[row * SR + n];
        b = Gs[row * SR + n + 1];
      }
      re[n] = a.re;
      im[n] = a.im;
      re[n + 1] = b.re;
      im[n + 1] = b.im;
    }
    if (h) twist<T, N, false>(re, im);
    fft<T, N, false>(re, im);
#pragma unroll
    for (int j = 0; j < N; ++j) V[row * VL::VR + h * VL::VH + j] = {re[j], im[j]};
  }
  group_sync<GS>(grp);
#pragma unroll 1
  for (int rho = 0; rho < 2; ++rho) {  // B2: column c along k1: forward, x T-hat, inverse
    const int c = row + N * rho;
    const int vc = rho * VL::VH + row;
    T re[N], im[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const cpx<T> v = V[n * VL::VR + vc];
      re[n] = v.re;
      im[n] = v.im;
    }
    if (h) twist<T, N, false>(re, im);
    fft<T, N, false>(re, im);
    const T* t = th + (size_t)(h * N) * L + c;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T w = __ldg(t + (size_t)j * L);
      re[j] *= w;
      im[j] *= w;
    }
    fft<T, N, true>(re, im);
    if (h) twist<T, N, true>(re, im);
    pair_combine_store<T, N>(re, im, h, V + vc, VL::VR);   // column c is read by this pair only
  }
  group_sync<GS>(grp);
  {  // B3: inverse along k2 of row n1 = row, parity h; result back into the slab
    T re[N], im[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const cpx<T> v = V[row * VL::VR + h * VL::VH + j];
      re[j] = v.re;
      im[j] = v.im;
    }
    fft<T, N, true>(re, im);
    if (h) twist<T, N, true>(re, im);
    if constexpr (GLOBAL && sizeof(T) == 4)
      pair_combine_store_row<N>(re, im, h, Gs + row * SR, pol);
    else
      pair_combine_store<T, N, GLOBAL>(re, im, h, Gs + row * SR, 1, pol);
  }
  group_sync<GS>(grp);
}

// Lines of u, f and the output are touched once per launch: streaming (evict-first) accesses
// keep them from displacing the per-CTA spectrum scratch and T-hat in L2.
template <typename T, int N>
__device__ __forceinline__ void load_line(const T* __restrict__ src, T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 t = __ldcs(s4 + q);
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 t = __ldcs(s2 + q);
      v[2 * q] = (T)t.x;
      v[2 * q + 1] = (T)t.y;
    }
  }
}

template <typename T, int N>
__device__ __forceinline__ void store_line(T* __restrict__ dst, const T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) d2[q] = make_double2(v[2 * q], v[2 * q + 1]);
  }
}

// o[n] = b[n] + coef * v[n] (b may be null: o[n] = coef * v[n]), vectorised, 4 or 2 at a time
template <typename T, int N>
__device__ __forceinline__ void finish_line(T* __restrict__ o, const T* b, T coef, const T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    float4* o4 = reinterpret_cast<float4*>(o);
    const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      float4 r = b ? __ldcs(b4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      r.x += coef * v[4 * q];
      r.y += coef * v[4 * q + 1];
      r.z += coef * v[4 * q + 2];
      r.w += coef * v[4 * q + 3];
      __stcs(o4 + q, r);
    }
  } else {
    double2* o2 = reinterpret_cast<double2*>(o);
    const double2* b2 = reinterpret_cast<const double2*>(b);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      double2 r = b ? __ldcs(b2 + q) : make_double2(0.0, 0.0);
      r.x += coef * v[2 * q];
      r.y += coef * v[2 * q + 1];
      __stcs(o2 + q, r);
    }
  }
}

template <typename T>
struct ThetaParams {
  const T* in;
  const T* base;        // may be null: out = Theta[in]
  T* out;
  int64_t nxp;
  int nx1, nx2, nx3;
  const T* that;        // [2N][2N][2N] parity-major [s3][s1][s2], scaled by 1/(2N)^3
  const cpx<T>* ph;     // per nucleus: E1[nx1][N], E2[nx2][N], E3[nx3][4][N] (M0, M1, D0, D1)
  int64_t ph_stride;
  int n_nuc;
  T coef[kMaxNuclei];
  cpx<T>* G;            // per CTA: 2N^3 complex
};

template <int N, int NT_>
struct ThetaCfg {
  static constexpr int NT = NT_;
  static constexpr int L = 2 * N;
  static constexpr int GS = 2 * N;         // threads per slab group
  static constexpr int NG = NT / GS;       // slab groups per CTA
  static_assert(NT % GS == 0 && (GS <= 32 || NG <= 15), "slab groups must tile the CTA");
  static constexpr int smem_cpx = NG * N * VLayout<N>::VR;
};

// Global-scratch kernel: the CTA's 2N^3 complex k3-spectrum lives in a private global scratch
// region (L2-resident when one CTA runs per SM); phases A/B/C as described at the top.
template <typename T, int N, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_theta(const ThetaParams<T> p) {
  using C = ThetaCfg<N, NT>;
  constexpr int L = C::L, GS = C::GS, NG = C::NG;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cpx<T>* smem = reinterpret_cast<cpx<T>*>(sm_raw);
  const int tid = threadIdx.x;
  const int grp = tid / GS, tg = tid % GS;
  cpx<T>* V = smem + grp * (N * VLayout<N>::VR);
  cpx<T>* G = p.G + (size_t)blockIdx.x * (2 * N3);
  const uint64_t pol = l2_keep_policy();

  for (int64_t xp = blockIdx.x; xp < p.nxp; xp += gridDim.x) {
    const int i3 = (int)(xp % p.nx3);
    const int i2 = (int)((xp / p.nx3) % p.nx2);
    const int i1 = (int)(xp / ((int64_t)p.nx3 * p.nx2));
    const T* __restrict__ u = p.in + xp * N3;

    for (int a = 0; a < p.n_nuc; ++a) {
      const cpx<T>* E1 = p.ph + a * p.ph_stride + (int64_t)i1 * N;
      const cpx<T>* E2 = p.ph + a * p.ph_stride + (int64_t)(p.nx1 + i2) * N;
      const cpx<T>* E3 = p.ph + a * p.ph_stride + (int64_t)(p.nx1 + p.nx2) * N + (int64_t)i3 * 4 * N;
      T coef = p.coef[0];   // static indexing keeps the parameter block out of local memory
#pragma unroll
      for (int q = 1; q < kMaxNuclei; ++q)
        if (q == a) coef = p.coef[q];

      // ---- Phase A: modulate + twist + FFT along k3 -> G[s3][k1][k2] ----
      for (int job = tid; job < 2 * N2; job += NT) {
        const int r3 = job / N2, line = job % N2;
        const int k1 = line / N, k2 = line % N;
        const cpx<T> e12 = conjg(cmul(E1[k1], E2[k2]));
        T re[N], im[N];
        load_line<T, N>(u + (size_t)line * N, re);
#pragma unroll
        for (int n = 0; n < N; ++n) {
          const cpx<T> mm = cmul(e12, E3[r3 * N + n]);
          im[n] = re[n] * mm.im;
          re[n] = re[n] * mm.re;
        }
        fft<T, N, false>(re, im);
        cpx<T>* g = G + (size_t)(r3 * N) * N2 + line;
#pragma unroll
        for (int j = 0; j < N; ++j) st_keep(g + (size_t)j * N2, cpx<T>{re[j], im[j]}, pol);
      }
      __syncthreads();

      // ---- Phase B: per slab s3, the 2-D padded convolution in (k1, k2) ----
      for (int s = grp; s < L; s += NG)
        slab_conv<T, N, GS, N, true>(G + (size_t)s * N2, V, p.that + (size_t)s * L * L, tg, grp, pol);
      __syncthreads();

      // ---- Phase C: inverse along k3 (both parities), demodulate, Im, write the line ----
      T* P = reinterpret_cast<T*>(smem);   // parity-0 partials, column layout (idle slab buffers)
      for (int line = tid; line < N2; line += NT) {
        const int k1 = line / N, k2 = line % N;
        const cpx<T> e12 = cmul(E1[k1], E2[k2]);
        T re[N], im[N];
#pragma unroll
        for (int r3 = 0; r3 < 2; ++r3) {
          const cpx<T>* g = G + (size_t)(r3 * N) * N2 + line;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const cpx<T> v = ld_keep<T>(g + (size_t)j * N2, pol);
            re[j] = v.re;
            im[j] = v.im;
          }
          fft<T, N, true>(re, im);
#pragma unroll
          for (int n = 0; n < N; ++n) {
            const cpx<T> z = cmul(e12, E3[(2 + r3) * N + n]);
            const T t = z.re * im[n] + z.im * re[n];
            if (r3 == 0)
              P[n * NT + tid] = t;
            else
              re[n] = P[n * NT + tid] + t;
          }
        }
        finish_line<T, N>(p.out + xp * N3 + (size_t)line * N,
                          a > 0 ? p.out + xp * N3 + (size_t)line * N
                                : (p.base ? p.base + xp * N3 + (size_t)line * N : nullptr),
                          coef, re);
      }
      __syncthreads();   // G and the slab buffers are reused by the next nucleus / x point
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Cluster variant: the padded spectrum of one x point lives in distributed shared memory.
//
// A cluster of C CTAs owns one x point at a time.  CTA rank c keeps the slabs
// s in [c SPC, (c+1) SPC), SPC = 2N / C, each N x (N+1) complex (padded rows), in its own shared
// memory.  Phase A jobs of CTA c cover k1 in [c N/C, (c+1) N/C) and store their k3-spectra
// straight into the owning CTA's slab (DSMEM stores, coalesced along k2); Phase B works on the
// local slabs only; Phase C jobs read their k3-spectra back from the owners (DSMEM loads), do the
// inverse transform, demodulate and write the output line.  Three cluster barriers per x point
// and nucleus order the phases.  No global scratch is used.  For N <= 16 the whole spectrum fits
// one CTA and C = 1.
// ------------------------------------------------------------------------------------------------
template <typename T, int N, int C>
struct ClCfg {
  static constexpr int NT = 256;
  static constexpr int L = 2 * N;
  static constexpr int GS = 2 * N;
  static constexpr int NG = NT / GS;
  static constexpr int SPC = L / C;          // slabs per CTA
  static constexpr int SLAB = N * (N + 1);   // padded slab, complex entries
  static constexpr int KPC = N / C;          // k1 rows per CTA in phases A and C
  static_assert(NT % GS == 0 && N % C == 0 && (GS <= 32 || NG <= 15), "cluster tiling");
  // slab buffers; the group buffers also hold the Phase C partials (NT x N reals)
  static constexpr size_t grp_cpx = (size_t)NG * N * VLayout<N>::VR;
  static constexpr size_t smem_cpx =
      (size_t)SPC * SLAB + (grp_cpx * 2 >= (size_t)NT * N ? grp_cpx : ((size_t)NT * N + 1) / 2);
  static constexpr size_t smem_bytes = smem_cpx * sizeof(cpx<T>);
};

template <typename T>
struct ThetaClParams {
  const T* in;
  const T* base;
  T* out;
  int64_t nxp;
  int nx1, nx2, nx3;
  const T* that;
  const cpx<T>* ph;
  int64_t ph_stride;
  int n_nuc;
  T coef[kMaxNuclei];
};

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C == 1)
    __syncthreads();
  else
    cg::this_cluster().sync();
}

template <typename T, int N, int C, int MINB>
__global__ void __launch_bounds__(256, MINB) k_theta_cl(const ThetaClParams<T> p) {
  using K = ClCfg<T, N, C>;
  constexpr int L = K::L, GS = K::GS, NG = K::NG, NT = K::NT;
  constexpr int SPC = K::SPC, SLAB = K::SLAB, KPC = K::KPC;
  (void)NG;
  constexpr int N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cpx<T>* Gl = reinterpret_cast<cpx<T>*>(sm_raw);
  const int tid = threadIdx.x;
  const int grp = tid / GS, tg = tid % GS;
  cpx<T>* V = Gl + SPC * SLAB + grp * (N * VLayout<N>::VR);
  int rank = 0;
  cpx<T>* Gr[C];
  if constexpr (C == 1) {
    Gr[0] = Gl;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    // launched without the matching cluster shape: touch no remote memory (uniform exit)
    if (cl.num_blocks() != (unsigned)C || gridDim.x % C != 0) return;
    rank = (int)cl.block_rank();
#pragma unroll
    for (int o = 0; o < C; ++o) Gr[o] = cl.map_shared_rank(Gl, o);
    cl.sync();   // every CTA of the cluster is running before any remote shared-memory access
  }
  const int64_t cl_id = blockIdx.x / C, ncl = gridDim.x / C;

  for (int64_t xp = cl_id; xp < p.nxp; xp += ncl) {
    const int i3 = (int)(xp % p.nx3);
    const int i2 = (int)((xp / p.nx3) % p.nx2);
    const int i1 = (int)(xp / ((int64_t)p.nx3 * p.nx2));
    const T* __restrict__ u = p.in + xp * N3;
    for (int a = 0; a < p.n_nuc; ++a) {
      const cpx<T>* E1 = p.ph + a * p.ph_stride + (int64_t)i1 * N;
      const cpx<T>* E2 = p.ph + a * p.ph_stride + (int64_t)(p.nx1 + i2) * N;
      const cpx<T>* E3 = p.ph + a * p.ph_stride + (int64_t)(p.nx1 + p.nx2) * N + (int64_t)i3 * 4 * N;
      T coef = p.coef[0];
#pragma unroll
      for (int q = 1; q < kMaxNuclei; ++q)
        if (q == a) coef = p.coef[q];

      // ---- Phase A: modulate + twist + FFT along k3, scattered to the owners' slabs ----
#pragma unroll
      for (int r3 = 0; r3 < 2; ++r3) {
        for (int job = tid; job < KPC * N; job += NT) {
          const int k1 = rank * KPC + job / N, k2 = job % N;
          const int line = k1 * N + k2;
          const cpx<T> e12 = conjg(cmul(E1[k1], E2[k2]));
          T re[N], im[N];
          load_line<T, N>(u + (size_t)line * N, re);
#pragma unroll
          for (int n = 0; n < N; ++n) {
            const cpx<T> mm = cmul(e12, E3[r3 * N + n]);
            im[n] = re[n] * mm.im;
            re[n] = re[n] * mm.re;
          }
          fft<T, N, false>(re, im);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int sg = r3 * N + j;        // global slab index (compile-time per j, r3)
            Gr[sg / SPC][(sg % SPC) * SLAB + k1 * (N + 1) + k2] = {re[j], im[j]};
          }
        }
      }
      cluster_barrier<C>();

      // ---- Phase B: the local slabs, 2-D padded convolution in (k1, k2) ----
      for (int sl = grp; sl < SPC; sl += NG) {
        const int sg = rank * SPC + sl;
        slab_conv<T, N, GS, N + 1, false>(Gl + sl * SLAB, V, p.that + (size_t)sg * L * L, tg, grp, 0);
      }
      cluster_barrier<C>();

      // ---- Phase C: inverse along k3 (both parities), demodulate, Im, write the line ----
      for (int job = tid; job < KPC * N; job += NT) {
        const int k1 = rank * KPC + job / N, k2 = job % N;
        const int line = k1 * N + k2;
        const cpx<T> e12 = cmul(E1[k1], E2[k2]);
        T* P = reinterpret_cast<T*>(Gl + SPC * SLAB);   // parity-0 partials (idle group buffers)
        T re[N], im[N];
#pragma unroll
        for (int r3 = 0; r3 < 2; ++r3) {
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int sg = r3 * N + j;
            const cpx<T> v = Gr[sg / SPC][(sg % SPC) * SLAB + k1 * (N + 1) + k2];
            re[j] = v.re;
            im[j] = v.im;
          }
          fft<T, N, true>(re, im);
#pragma unroll
          for (int n = 0; n < N; ++n) {
            const cpx<T> z = cmul(e12, E3[(2 + r3) * N + n]);
            const T t = z.re * im[n] + z.im * re[n];
            if (r3 == 0)
              P[n * NT + tid] = t;
            else
              re[n] = P[n * NT + tid] + t;
          }
        }
        finish_line<T, N>(p.out + xp * N3 + (size_t)line * N,
                          a > 0 ? p.out + xp * N3 + (size_t)line * N
                                : (p.base ? p.base + xp * N3 + (size_t)line * N : nullptr),
                          coef, re);
      }
      cluster_barrier<C>();
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Launch plans
// ------------------------------------------------------------------------------------------------
// global-scratch kernel configuration: one 512-thread CTA per SM for FP32 at N = 32 (the
// per-CTA scratch then totals 152 x 512 KB, L2-resident); 256 threads otherwise
template <typename T, int N>
constexpr int gs_threads() {
  return (sizeof(T) == 4 && N == 32) ? 512 : 256;
}
template <typename T, int N>
constexpr int minb() {
  return (sizeof(T) == 4 && N < 32) ? 2 : 1;
}
template <typename T, int N>
size_t smem_bytes() {
  return (size_t)ThetaCfg<N, gs_threads<T, N>()>::smem_cpx * sizeof(cpx<T>);
}

// CTAs per SM the cluster kernel is compiled for (registers capped at 128 when 2)
template <typename T, int N>
constexpr int cl_minb() {
  return (sizeof(T) == 4 && N <= 16) ? 2 : 1;
}

// cluster size used for (T, N), 0 = global-scratch kernel
template <typename T, int N>
constexpr int cluster_size() {
  if constexpr (N <= 16) return 1;
  if constexpr (sizeof(T) == 4) return 4;
  return 0;
}

template <typename T, int N>
int gs_occupancy() {
  auto kern = k_theta<T, N, gs_threads<T, N>(), minb<T, N>()>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<T, N>()) !=
      cudaSuccess)
    return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, gs_threads<T, N>(), smem_bytes<T, N>()) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

template <typename T, int N, int C>
int cl_max_clusters(int num_sms) {
  using K = ClCfg<T, N, C>;
  auto kern = k_theta_cl<T, N, C, cl_minb<T, N>()>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes) !=
      cudaSuccess)
    return 0;
  if constexpr (C == 1) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 256, K::smem_bytes) != cudaSuccess)
      return 0;
    return nb * num_sms;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * num_sms, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = K::smem_bytes;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) return 0;
    return n;
  }
}

// CHASM_THETA_VARIANT=global|cluster overrides the choice (both are parity-tested).
template <typename T, int N>
void plan_tn(int64_t nxp, int num_sms, ThetaPlan* pl) {
  constexpr int C = cluster_size<T, N>();
  const char* env = std::getenv("CHASM_THETA_VARIANT");
  const bool want_global = env ? std::strcmp(env, "global") == 0 : (C > 1);
  if constexpr (C > 0) {
   if (!want_global) {
    const int ncl = cl_max_clusters<T, N, C>(num_sms);
    if (ncl > 0) {
      pl->cluster = C;
      pl->blocks = (int)std::min<int64_t>(nxp, ncl) * C;
      pl->scratch_bytes = 0;
      return;
    }
   }
  }
  pl->cluster = 0;
  pl->blocks = (int)std::min<int64_t>(nxp, (int64_t)gs_occupancy<T, N>() * num_sms);
  pl->scratch_bytes = (size_t)pl->blocks * 2 * N * N * N * 2 * sizeof(T);
}

template <typename T, int N>
cudaError_t launch_tn(const Handle& H, const void* in, const void* base, void* out,
                      const double* coef, cudaStream_t s) {
  const int n_nuc = (int)H.nuclei.size();
  if constexpr (cluster_size<T, N>() > 0) {
   if (H.theta.cluster > 0) {
    constexpr int C = cluster_size<T, N>();
    ThetaClParams<T> p;
    p.in = static_cast<const T*>(in);
    p.base = static_cast<const T*>(base);
    p.out = static_cast<T*>(out);
    p.nxp = H.g.nxp;
    p.nx1 = H.g.nx[0];
    p.nx2 = H.g.nx[1];
    p.nx3 = H.g.nx[2];
    p.that = static_cast<const T*>(H.d_that);
    p.ph = static_cast<const cpx<T>*>(H.d_phase);
    p.ph_stride = (int64_t)(H.g.nx[0] + H.g.nx[1] + 4 * H.g.nx[2]) * N;
    p.n_nuc = n_nuc;
    for (int a = 0; a < kMaxNuclei; ++a) p.coef[a] = a < n_nuc ? (T)coef[a] : (T)0;
    if constexpr (C == 1) {
      k_theta_cl<T, N, C, cl_minb<T, N>()><<<H.theta.blocks, 256, ClCfg<T, N, C>::smem_bytes, s>>>(p);
      return cudaGetLastError();
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)H.theta.blocks, 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = ClCfg<T, N, C>::smem_bytes;
      cfg.stream = s;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = C;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_theta_cl<T, N, C, cl_minb<T, N>()>, p);
    }
   }
  }
  ThetaParams<T> p;
  p.in = static_cast<const T*>(in);
  p.base = static_cast<const T*>(base);
  p.out = static_cast<T*>(out);
  p.nxp = H.g.nxp;
  p.nx1 = H.g.nx[0];
  p.nx2 = H.g.nx[1];
  p.nx3 = H.g.nx[2];
  p.that = static_cast<const T*>(H.d_that);
  p.ph = static_cast<const cpx<T>*>(H.d_phase);
  p.ph_stride = (int64_t)(H.g.nx[0] + H.g.nx[1] + 4 * H.g.nx[2]) * N;
  p.n_nuc = n_nuc;
  for (int a = 0; a < kMaxNuclei; ++a) p.coef[a] = a < p.n_nuc ? (T)coef[a] : (T)0;
  p.G = static_cast<cpx<T>*>(H.d_scratch);
  k_theta<T, N, gs_threads<T, N>(), minb<T, N>()><<<H.theta.blocks, gs_threads<T, N>(), smem_bytes<T, N>(), s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_theta(const Handle& H, const void* in, const void* base, void* out,
                         const double* coef, cudaStream_t s) {
  switch (H.g.nk) {
    case 8:
      return H.fp64 ? launch_tn<double, 8>(H, in, base, out, coef, s)
                    : launch_tn<float, 8>(H, in, base, out, coef, s);
    case 16:
      return H.fp64 ? launch_tn<double, 16>(H, in, base, out, coef, s)
                    : launch_tn<float, 16>(H, in, base, out, coef, s);
    case 32:
      return H.fp64 ? launch_tn<double, 32>(H, in, base, out, coef, s)
                    : launch_tn<float, 32>(H, in, base, out, coef, s);
  }
  return cudaErrorInvalidValue;
}

void theta_plan(int nk, bool fp64, int64_t nxp, int num_sms, ThetaPlan* pl) {
  switch (nk) {
    case 8:
      fp64 ? plan_tn<double, 8>(nxp, num_sms, pl) : plan_tn<float, 8>(nxp, num_sms, pl);
      return;
    case 16:
      fp64 ? plan_tn<double, 16>(nxp, num_sms, pl) : plan_tn<float, 16>(nxp, num_sms, pl);
      return;
    case 32:
      fp64 ? plan_tn<double, 32>(nxp, num_sms, pl) : plan_tn<float, 32>(nxp, num_sms, pl);
      return;
  }
  pl->cluster = 0;
  pl->blocks = 1;
  pl->scratch_bytes = 0;
}

}  // namespace chasm
