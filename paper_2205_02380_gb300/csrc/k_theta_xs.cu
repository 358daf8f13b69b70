// Coulomb operator and P-flow in the real form with a per-x symbol table (Sec. 4): FP64 and
// N_k = 8 (single precision with N_k = 16 or 32 runs the packed kernel of k_theta_pk.cu).
//
// For one x point, Theta^T is a real linear convolution over the k-grid:
//   Theta^T[u]_p = sum_q S_{p-q}(x) u_q,
//   S_m(x) = sum_A c_A T_m sin(2 (x - x_A) . m dk),  c_A = -2 Z_A / (pi^2 hbar),
// because k_p - k_q = (p - q) dk, so e^{2i(x-x_A).k_p} e^{-2i(x-x_A).k_q} depends on p - q only
// and Im[e^{i th_p} sum_q T_{p-q} u_q e^{-i th_q}] = sum_q T_{p-q} sin(th_p - th_q) u_q for real u
// (Eqs. 4.1, 4.5, 4.6 with the sign of Eq. 2.3).  All nuclei fold into the one kernel S.
//
// The convolution is embedded circularly with length 2N along k1 and k2 (twofold zero padding,
// Sec. 4.1) and negacyclically with length 2N along k3 (frequencies nu3 = xi3 + 1/2; for inputs
// on [0, N) and taps on (-N, N) the wrap-around terms fall outside the taps, so the result is
// the linear convolution).  u and S are real, so the product spectrum is conjugate-symmetric
// under (xi1, xi2, xi3) -> (-xi1, -xi2, 2N-1-xi3), which pairs every even xi3 = 2j with an odd
// one: only nu3 = 2j + 1/2, j = 0..N-1, is kept and Theta = 2 Re[...] / (2N)^3.  Along k3 this is
// one N-point FFT of the input twisted by e^{-i pi n/(2N)} (forward) and one inverse FFT
// followed by the conjugate twist and the real part (inverse).  S is real and odd, so its
// spectrum is i sigma with sigma real; the table (k_xsym.cu) holds sigma(x)[j][s1][s2] with the
// factor 2 / (2N)^3 folded in, in the parity-major order of the slab phase.
//
// Per x point (one CTA, persistent loop over x points):
//   Phase A   N^2 lines along k3: twist, FFT_N -> G[j][k1][k2]
//   Phase B   N slabs j: the 2-D padded convolution in (k1, k2) (slab_conv), spectrum times i sigma
//   Phase CA  N^2 lines: inverse FFT_N along k3, conjugate twist, real part = Theta line;
//             v = base + c_s Theta.  After the last stage v is written out; otherwise the same
//             thread twists and transforms v in place of the next stage's Phase A (same lines,
//             same spectrum locations), so the stages chain without a round trip through HBM.
// P(dt) = four Horner stages u <- f + (dt/s) Theta^T[u], s = 4, 3, 2, 1, on one x point in a
// row: f is read once and written once per step.  Work per stage and x point: 14 N^2 FFTs of
// length N (the modulated complex form needs 28 N^2 per nucleus).
#include "internal.hpp"
#include "fft_reg.cuh"

namespace chasm {
namespace {

template <typename T>
struct XsParams {
  const T* in;     // stage-0 input u_0 = in + cin2 in2 (in2 may be null)
  const T* base;   // Horner base base + cbase2 base2 (base2 may be null), or null (out = c Theta)
  const T* in2;
  const T* base2;
  T cin2, cbase2;
  T* out;          // result of the last stage; may alias in, in2, base and base2
  int64_t nxp;
  const T* sig;    // [nxp][N][2N][2N] symbol table
  int64_t sig_xs;  // elements per x point of sig (0: one table for every x point)
  int nst;         // stages, 1..4
  T coef[4];       // c_s per stage
  cpx<T>* G;       // per-CTA spectrum scratch (N^3 complex) when it is not in shared memory
};

// launch shape per (precision, N): threads, spectrum in shared memory, CTAs per SM compiled for
template <typename T, int N>
struct XsCfg {
  static constexpr int NT = N == 32 ? (sizeof(T) == 4 ? 512 : 256) : (N == 16 ? 256 : 128);
  static constexpr bool GSM = N <= 16;
  static constexpr int MINB = (sizeof(T) == 4 && N == 16) ? 2 : 1;
  static constexpr int L = 2 * N;
  static constexpr int GS = 2 * N;
  static constexpr int NG = NT / GS;
  static constexpr int SR = GSM ? N + 1 : N;   // spectrum row stride (padded in shared memory)
  static constexpr int SLAB = N * SR;
  static_assert(NT % GS == 0 && (GS <= 32 || NG <= 15), "slab groups must tile the CTA");
  static constexpr int VSIZE = VRows<T, N>::SIZE;   // group slab buffer, elements
  static constexpr size_t smem_cpx = (size_t)NG * VSIZE + (GSM ? (size_t)N * SLAB : 0);
  static constexpr size_t smem_bytes = smem_cpx * sizeof(cpx<T>);
};

// quarter-turn twist e^{-i pi n/(2N)} applied to a real line: re = v cos, im = -v sin
template <typename T, int N>
__device__ __forceinline__ void twist_real(T (&re)[N], T (&im)[N]) {
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const T v = re[n];
    re[n] = v * ht_cos<T>(n * (32 / N));
    im[n] = -v * ht_sin<T>(n * (32 / N));
  }
}

template <typename T, int N, bool GSM>
__device__ __forceinline__ void store_col(cpx<T>* g, int stride, const T (&re)[N], const T (&im)[N],
                                          uint64_t pol) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if constexpr (GSM)
      g[(size_t)j * stride] = {re[j], im[j]};
    else
      st_keep(g + (size_t)j * stride, cpx<T>{re[j], im[j]}, pol);
  }
}

template <typename T, int N, bool GSM>
__device__ __forceinline__ void load_col(const cpx<T>* g, int stride, T (&re)[N], T (&im)[N],
                                         uint64_t pol) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    cpx<T> v;
    if constexpr (GSM)
      v = g[(size_t)j * stride];
    else
      v = ld_keep<T>(g + (size_t)j * stride, pol);
    re[j] = v.re;
    im[j] = v.im;
  }
}

// re[n] <- (b[n] + cb2 b2[n]) + c Re[e^{+i pi n/(2N)} (re[n] + i im[n])]   (b null: 0; b2 null: b)
template <typename T, int N>
__device__ __forceinline__ void horner_line(T (&re)[N], const T (&im)[N], const T* b, const T* b2,
                                            T cb2, T c) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4* c4 = reinterpret_cast<const float4*>(b2);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      float4 bb = b ? b4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (b2) {
        const float4 cc = c4[q];
        bb = make_float4(fmaf(cb2, cc.x, bb.x), fmaf(cb2, cc.y, bb.y), fmaf(cb2, cc.z, bb.z),
                         fmaf(cb2, cc.w, bb.w));
      }
      const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n = 4 * q + e;
        const T th = re[n] * ht_cos<T>(n * (32 / N)) - im[n] * ht_sin<T>(n * (32 / N));
        re[n] = fma(c, th, (T)bv[e]);
      }
    }
  } else {
    const double2* bd = reinterpret_cast<const double2*>(b);
    const double2* cd = reinterpret_cast<const double2*>(b2);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      double2 bb = b ? bd[q] : make_double2(0.0, 0.0);
      if (b2) {
        const double2 cc = cd[q];
        bb = make_double2(fma((double)cb2, cc.x, bb.x), fma((double)cb2, cc.y, bb.y));
      }
      const T bv[2] = {(T)bb.x, (T)bb.y};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = 2 * q + e;
        const T th = re[n] * ht_cos<T>(n * (32 / N)) - im[n] * ht_sin<T>(n * (32 / N));
        re[n] = fma(c, th, bv[e]);
      }
    }
  }
}

template <typename T, int N>
__device__ __forceinline__ void store_line_cs(T* __restrict__ dst, const T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) __stcs(d4 + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
  } else {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) __stcs(d2 + q, make_double2(v[2 * q], v[2 * q + 1]));
  }
}

template <typename T, int N>
__device__ __forceinline__ void load_line_plain(const T* src, T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 t = s4[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 t = s2[q];
      v[2 * q] = (T)t.x;
      v[2 * q + 1] = (T)t.y;
    }
  }
}

// bytes (a multiple of 16, 16-byte aligned source) towards L2, asynchronously, no completion
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// X2: the second input and base terms (in2, base2) are read (the LPC1 corrector); without it
// they are compiled out.  IMAG: the table is the imaginary part sigma of the symbol i sigma (the
// Coulomb operator); without it the real spectrum of an even kernel (the plain TKM convolution).
template <typename T, int N, int NT, bool GSM, int MINB, bool X2, bool IMAG = true>
__global__ void __launch_bounds__(NT, MINB) k_theta_xs(const XsParams<T> p) {
  using C = XsCfg<T, N>;
  constexpr int L = C::L, GS = C::GS, NG = C::NG, SR = C::SR, SLAB = C::SLAB;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cpx<T>* smem = reinterpret_cast<cpx<T>*>(sm_raw);
  const int tid = threadIdx.x;
  const int grp = tid / GS, tg = tid % GS;
  cpx<T>* V = smem + grp * C::VSIZE;
  cpx<T>* G = GSM ? smem + NG * C::VSIZE : p.G + (size_t)blockIdx.x * (N * SLAB);
  const uint64_t pol = l2_keep_policy();

  for (int64_t xp = blockIdx.x; xp < p.nxp; xp += gridDim.x) {
    // ---- Phase A: twist + FFT along k3 of the stage-0 input ----
    for (int line = tid; line < N2; line += NT) {
      const int off = (line / N) * SR + (line % N);
      T re[N], im[N];
      load_line_plain<T, N>(p.in + xp * N3 + (size_t)line * N, re);
      if (X2 && p.in2) {   // u_0 = in + cin2 in2 (the LPC1 predictor)
        load_line_plain<T, N>(p.in2 + xp * N3 + (size_t)line * N, im);
#pragma unroll
        for (int n = 0; n < N; ++n) re[n] = fma(p.cin2, im[n], re[n]);
      }
      twist_real<T, N>(re, im);
      fft<T, N, false>(re, im);
      store_col<T, N, GSM>(G + off, SLAB, re, im, pol);
    }
    __syncthreads();

    for (int st = 0; st < p.nst; ++st) {
      // ---- Phase B: per slab j, the 2-D padded convolution with i sigma_j ----
      for (int s = grp; s < N; s += NG) {
        if (tg == 0) {   // the symbol slab this group needs next, into L2 (one bulk prefetch)
          const int sn = s + NG < N ? s + NG : grp;
          const int64_t xn = s + NG < N || st + 1 < p.nst ? xp : xp + gridDim.x;
          if (xn < p.nxp) bulk_prefetch_l2(p.sig + xn * p.sig_xs + sn * (int64_t)(L * L), L * L * sizeof(T));
        }
        slab_conv<T, N, GS, SR, !GSM, IMAG>(G + (size_t)s * SLAB, V,
                                            p.sig + xp * p.sig_xs + s * (int64_t)(L * L), tg, grp, pol);
      }
      __syncthreads();

      T c = p.coef[0];   // static indexing keeps the parameter block out of local memory
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (q == st) c = p.coef[q];
      const bool last = st == p.nst - 1;

      // ---- Phase CA: inverse along k3, Theta line, Horner update; next stage's Phase A ----
      for (int line = tid; line < N2; line += NT) {
        const int off = (line / N) * SR + (line % N);
        T re[N], im[N];
        load_col<T, N, GSM>(G + off, SLAB, re, im, pol);
        fft<T, N, true>(re, im);
        horner_line<T, N>(re, im, p.base ? p.base + xp * N3 + (size_t)line * N : nullptr,
                          X2 && p.base2 ? p.base2 + xp * N3 + (size_t)line * N : nullptr, p.cbase2, c);
        if (last) {
          store_line_cs<T, N>(p.out + xp * N3 + (size_t)line * N, re);
        } else {
          twist_real<T, N>(re, im);
          fft<T, N, false>(re, im);
          store_col<T, N, GSM>(G + off, SLAB, re, im, pol);
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, int N, bool X2 = false, bool IMAG = true>
auto xs_kernel() {
  using C = XsCfg<T, N>;
  return k_theta_xs<T, N, C::NT, C::GSM, C::MINB, X2, IMAG>;
}

template <typename T, int N>
void plan_xs_tn(int64_t nxp, int num_sms, ThetaPlan* pl) {
  using C = XsCfg<T, N>;
  auto kern = xs_kernel<T, N>();
  int nb = 0;
  cudaFuncSetAttribute(xs_kernel<T, N, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)C::smem_bytes);
  cudaFuncSetAttribute(xs_kernel<T, N, false, false>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)C::smem_bytes);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::NT, C::smem_bytes) != cudaSuccess ||
      nb < 1)
    nb = 1;
  pl->cluster = 0;
  pl->blocks = (int)std::min<int64_t>(nxp, (int64_t)nb * num_sms);
  pl->scratch_bytes = C::GSM ? 0 : (size_t)pl->blocks * N * C::SLAB * sizeof(cpx<T>);
}

template <typename T, int N>
cudaError_t launch_xs_tn(const Handle& H, const void* in, const void* base, void* out, int nst,
                         const double* coef, const XsExtra& x, cudaStream_t s) {
  using C = XsCfg<T, N>;
  XsParams<T> p;
  p.in = static_cast<const T*>(in);
  p.base = static_cast<const T*>(base);
  p.in2 = static_cast<const T*>(x.in2);
  p.base2 = static_cast<const T*>(x.base2);
  p.cin2 = (T)x.cin2;
  p.cbase2 = (T)x.cbase2;
  p.out = static_cast<T*>(out);
  p.nxp = H.g.nxp;
  p.sig = static_cast<const T*>(x.sig ? x.sig : H.d_sig);
  p.sig_xs = x.sig ? 0 : (int64_t)N * C::L * C::L;
  p.nst = nst;
  for (int q = 0; q < 4; ++q) p.coef[q] = q < nst ? (T)coef[q] : (T)0;
  p.G = static_cast<cpx<T>*>(H.d_scratch);
  if (x.real_symbol) {
    if (x.in2 || x.base2) return cudaErrorInvalidValue;
    k_theta_xs<T, N, C::NT, C::GSM, C::MINB, false, false><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  } else if (x.in2 || x.base2) {
    k_theta_xs<T, N, C::NT, C::GSM, C::MINB, true><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  } else {
    k_theta_xs<T, N, C::NT, C::GSM, C::MINB, false><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_theta_xs(const Handle& H, const void* in, const void* base, void* out, int nst,
                            const double* coef, cudaStream_t s, const XsExtra& x) {
  if (nst < 1 || nst > 4 || !H.d_sig) return cudaErrorInvalidValue;
  if (xs_packed(H.fp64, H.g.nk)) return launch_theta_pk(H, in, base, out, nst, coef, s, x);
  switch (H.g.nk) {
    case 8:
      return H.fp64 ? launch_xs_tn<double, 8>(H, in, base, out, nst, coef, x, s)
                    : launch_xs_tn<float, 8>(H, in, base, out, nst, coef, x, s);
    case 16:
      return H.fp64 ? launch_xs_tn<double, 16>(H, in, base, out, nst, coef, x, s) : cudaErrorInvalidValue;
    case 32:
      return H.fp64 ? launch_xs_tn<double, 32>(H, in, base, out, nst, coef, x, s) : cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

void theta_xs_plan(int nk, bool fp64, int64_t nxp, int num_sms, ThetaPlan* pl) {
  if (xs_packed(fp64, nk)) {
    theta_pk_plan(nk, nxp, num_sms, pl);
    return;
  }
  switch (nk) {
    case 8:
      fp64 ? plan_xs_tn<double, 8>(nxp, num_sms, pl) : plan_xs_tn<float, 8>(nxp, num_sms, pl);
      return;
    case 16:
      if (fp64) plan_xs_tn<double, 16>(nxp, num_sms, pl);
      return;
    case 32:
      if (fp64) plan_xs_tn<double, 32>(nxp, num_sms, pl);
      return;
  }
  pl->cluster = 0;
  pl->blocks = 1;
  pl->scratch_bytes = 0;
}

}  // namespace chasm
