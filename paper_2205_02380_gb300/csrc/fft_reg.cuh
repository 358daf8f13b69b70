// Register-resident FFT building blocks shared by the Coulomb-operator kernels (k_theta.cu and
// k_theta_xs.cu): complex arithmetic, compile-time twiddle tables, the in-register radix-2 FFT
// with fused-multiply-add butterflies, the parity twists of the twofold-padded transform, L2
// cache-policy accesses, and the per-slab 2-D padded convolution of the slab phase.
#pragma once

#include <cstdint>

namespace chasm {
namespace {

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

// Quarter-turn twist table of the negacyclic (half-shifted) transform: cos and sin of
// 2 pi k / 128, k = 0..31 (angles in [0, pi/2)); for length N the twist e^{-i pi n / (2N)} is
// entry n * 32 / N.
#define CHASM_H4(f, b) f(b, 128), f(b + 1, 128), f(b + 2, 128), f(b + 3, 128)
#define CHASM_H16(f, b) CHASM_H4(f, b), CHASM_H4(f, b + 4), CHASM_H4(f, b + 8), CHASM_H4(f, b + 12)
#define CHASM_H32(f) CHASM_H16(f, 0), CHASM_H16(f, 16)
__constant__ double c_hcos32d[32] = {CHASM_H32(ce_cos2pi)};
__constant__ double c_hsin32d[32] = {CHASM_H32(ce_sin2pi)};
__constant__ float c_hcos32f[32] = {CHASM_H32((float)ce_cos2pi)};
__constant__ float c_hsin32f[32] = {CHASM_H32((float)ce_sin2pi)};
template <typename T>
__device__ __forceinline__ T ht_cos(int k) {
  if constexpr (sizeof(T) == 4) return c_hcos32f[k];
  else return c_hcos32d[k];
}
template <typename T>
__device__ __forceinline__ T ht_sin(int k) {
  if constexpr (sizeof(T) == 4) return c_hsin32f[k];
  else return c_hsin32d[k];
}

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
// streamed read-only data (the per-x symbol table) with an L2 evict-first policy, so that it does
// not displace the spectrum scratch
__device__ __forceinline__ uint64_t l2_stream_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
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
};

// Rows of the group's slab buffer V: N rows of stride VR.
template <typename T, int N>
struct VRows {
  static constexpr int SIZE = N * VLayout<N>::VR;   // elements per group buffer
  __host__ __device__ static constexpr int off(int r) { return r * VLayout<N>::VR; }
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
// N x (2N + 1) complex buffer.  th is the slab of the symbol (parity-major [s1][s2], row length
// 2N): real (the spectrum is multiplied by th) or, with IMAG, the imaginary part of a purely
// imaginary symbol (the spectrum is multiplied by i th).
template <typename T, int N, int GS, int SR, bool GLOBAL, bool IMAG = false>
__device__ __forceinline__ void slab_conv(cpx<T>* Gs, cpx<T>* V, const T* __restrict__ th, int tg,
                                          int grp, uint64_t pol) {
  constexpr int L = 2 * N;
  using VL = VLayout<N>;
  using VW = VRows<T, N>;
  const int h = tg & 1, row = tg >> 1;
  const int vrow = VW::off(row);
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
    for (int j = 0; j < N; ++j) V[vrow + h * VL::VH + j] = {re[j], im[j]};
  }
  group_sync<GS>(grp);
#pragma unroll 1
  for (int rho = 0; rho < 2; ++rho) {  // B2: column c along k1: forward, x T-hat, inverse
    const int c = row + N * rho;
    const int vc = rho * VL::VH + row;
    T re[N], im[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
      const cpx<T> v = V[VW::off(n) + vc];
      re[n] = v.re;
      im[n] = v.im;
    }
    if (h) twist<T, N, false>(re, im);
    fft<T, N, false>(re, im);
    const T* t = th + (size_t)(h * N) * L + c;
    uint64_t spol = 0;
    if constexpr (IMAG) spol = l2_stream_policy();
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T w = IMAG ? ld_stream(t + (size_t)j * L, spol) : __ldg(t + (size_t)j * L);
      if constexpr (IMAG) {
        const T a = re[j];
        re[j] = -w * im[j];
        im[j] = w * a;
      } else {
        re[j] *= w;
        im[j] *= w;
      }
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
      const cpx<T> v = V[vrow + h * VL::VH + j];
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

}  // namespace
}  // namespace chasm
