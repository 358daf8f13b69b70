// P-flow of the Coulomb operator in the real form, single precision, N_k = 16 and 32: the packed
// (two-lane) variant of the table-form kernel (Sec. 4; the FP64 form and N_k = 8 run
// k_theta_xs.cu).
//
// It evaluates the same real linear convolution per x point,
//   Theta^T[u]_p = sum_q S_{p-q}(x) u_q,  S_m(x) = sum_A c_A T_m sin(2 (x - x_A) . m dk),
// embedded circularly with length 2N along k1 and k2 (twofold zero padding, Sec. 4.1) and
// negacyclically with length 2N along k3 (only the k3 frequencies nu3 = 2j + 1/2 are kept; the
// others follow by conjugate symmetry), with the spectrum of S equal to i sigma, sigma real and
// tabulated per x point (k_xsym.cu).  What differs from k_theta_xs.cu is the mapping onto
// threads, chosen so that the arithmetic runs as packed FP32 instructions:
//   * a zero-padded transform of length 2N along k1 or k2 is held by ONE thread as the pair
//     (E, O) = (x, x e^{-i pi n/N}): its even and odd output frequencies are the N-point FFTs of
//     E and O, computed in lockstep by fft_pk; the inverse transform of a padded spectrum,
//     cropped to N outputs, is y_n = IFFT(E)_n + e^{+i pi n/N} IFFT(O)_n (no cross-lane combine);
//   * along k3 one thread transforms two neighbouring lines (k2 = 2m, 2m + 1) in lockstep;
//   * the factor i of the symbol is carried through the linear inverse transforms and applied at
//     the end: Re[e^{i phi} i y] = -(sin phi Re y + cos phi Im y), the sign folded into the
//     Horner coefficient.
// Data layouts (floats):
//   spectrum G[j][m][k1] (float4) = (Re z_{2m}, Re z_{2m+1}, Im z_{2m}, Im z_{2m+1}), z the k3
//     spectrum of the line pair (k1, k2 = 2m, 2m + 1) at frequency j: row k1 of slab j holds the
//     N values along k2 as the N/2 quads m, N quads apart (the lanes of a row pass, one row each,
//     touch N consecutive quads per access);
//   slab buffer V[row][jj] (float4, one buffer of N rows per slab, row stride 4N + 4 floats) =
//     (Re E_jj, Re O_jj, Im E_jj, Im O_jj) for the frequency pair (2 jj, 2 jj + 1), halves
//     swapped when jj & 8 (so the column accesses of the second pass are free of bank conflicts);
//   symbol sig[x][j][q][c][e] = sigma at (xi1 = 4q + e, xi2 = c) of slab j (k_xsym.cu).
// Per x point (one CTA, persistent loop over x points), per Horner stage:
//   Phase B  one warp per slab (two slabs for N = 16): rows forward along k2 (B1), columns
//            forward along k1, times sigma, inverse (B2, two columns per lane), rows inverse (B3);
//   Phase CA line pairs: inverse along k3, Theta, Horner update v = base + c_s Theta, and for
//            all but the last stage the next stage's forward k3 transform of v (Phase A of
//            stage 0 reads the input instead).
#include "internal.hpp"
#include "fft_pk.cuh"

namespace chasm {
namespace {

struct PkParams {
  const float* in;     // stage-0 input u_0 = in + cin2 in2 (in2 may be null)
  const float* base;   // Horner base base + cbase2 base2 (base2 may be null), or null (0)
  const float* in2;
  const float* base2;
  float cin2, cbase2;
  float* out;          // result of the last stage; may alias in, in2, base and base2
  int64_t nxp;
  const float* sig;    // [nxp][N][L/4][L][4] symbol table
  int64_t sig_xs;      // floats per x point of sig (0: one table for every x point)
  int nst;             // stages, 1..4
  float ncoef[4];      // -c_s per stage (the sign of the deferred factor i); +c_s when REAL
  float4* G;           // per-CTA spectrum scratch [N][N/2][N] when it is not in shared memory
};

template <int N>
struct PkCfg {
  static constexpr int L = 2 * N;
  static constexpr int NT = 256;
  static constexpr int NW = NT / 32;
  static constexpr int SPW = 32 / N;                 // slabs per warp
  static constexpr int MINB = N == 32 ? 1 : 2;
  static constexpr bool GSM = N <= 16;               // spectrum in shared memory
  static constexpr int RS = 4 * N + 4;               // slab-buffer row stride (floats)
  static constexpr int VW = SPW * N * RS;            // slab-buffer floats per warp
  static constexpr int GQ = N * N * N / 2;           // spectrum quads per CTA
  static constexpr size_t smem_bytes = (size_t)NW * VW * 4 + (GSM ? (size_t)GQ * 16 : 0);
  static_assert(N == 16 || N == 32, "packed kernel: N = 16 or 32");
};

// ---- memory accesses ----
__device__ __forceinline__ float4 ldg_keep4(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void stg_keep4(float4* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ float4 ldg_stream4(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
// spectrum quads: shared memory (GSM) or the CTA's global scratch with an L2 evict-last policy
template <bool GSM>
__device__ __forceinline__ float4 g_load(const float4* p, uint64_t pol) {
  if constexpr (GSM) return *p;
  else return ldg_keep4(p, pol);
}
template <bool GSM>
__device__ __forceinline__ void g_store(float4* p, float4 v, uint64_t pol) {
  if constexpr (GSM) *p = v;
  else stg_keep4(p, v, pol);
}

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// two neighbouring lines of N reals (2N contiguous floats) -> a[n], b[n]
template <int N>
__device__ __forceinline__ void load_pair(const float* src, float (&a)[N], float (&b)[N]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 u = __ldcs(s4 + q), v = __ldcs(s4 + N / 4 + q);
    a[4 * q] = u.x;
    a[4 * q + 1] = u.y;
    a[4 * q + 2] = u.z;
    a[4 * q + 3] = u.w;
    b[4 * q] = v.x;
    b[4 * q + 1] = v.y;
    b[4 * q + 2] = v.z;
    b[4 * q + 3] = v.w;
  }
}
template <int N>
__device__ __forceinline__ void store_pair(float* dst, const float (&a)[N], const float (&b)[N]) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    __stcs(d4 + q, make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]));
    __stcs(d4 + N / 4 + q, make_float4(b[4 * q], b[4 * q + 1], b[4 * q + 2], b[4 * q + 3]));
  }
}

// The line pairs of one warp in a k3 pass (N = 32): lane k1 owns the pair (k1, k2 = 2m, 2m + 1)
// with m common to the warp, i.e. 2N contiguous floats at src_m + k1 N^2.  Read through the warp's
// slab buffer so that every global access of the warp covers two whole pairs (512 contiguous
// bytes) instead of one 16-byte piece of 32 pairs: the loads no longer depend on L1 to merge.
template <int N>
__device__ __forceinline__ void warp_load_pairs(const float* src_m, float* T, float (&a)[N], float (&b)[N]) {
  constexpr int Q = N / 2, RW = 2 * N + 4;   // quads per pair, buffer row (floats)
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = 2 * q + (lane >> 4), e = lane & 15;
    const float4 v = __ldcs(reinterpret_cast<const float4*>(src_m + (size_t)t * N * N) + e);
    *reinterpret_cast<float4*>(T + t * RW + 4 * e) = v;
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float4 v = *reinterpret_cast<const float4*>(T + lane * RW + 4 * q);
    float* d = q < Q / 2 ? a + 4 * q : b + 4 * (q - Q / 2);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
  __syncwarp();
}
template <int N>
__device__ __forceinline__ void warp_store_pairs(float* dst_m, float* T, const float (&a)[N], const float (&b)[N]) {
  constexpr int Q = N / 2, RW = 2 * N + 4;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float* d = q < Q / 2 ? a + 4 * q : b + 4 * (q - Q / 2);
    *reinterpret_cast<float4*>(T + lane * RW + 4 * q) = make_float4(d[0], d[1], d[2], d[3]);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = 2 * q + (lane >> 4), e = lane & 15;
    __stcs(reinterpret_cast<float4*>(dst_m + (size_t)t * N * N) + e,
           *reinterpret_cast<const float4*>(T + t * RW + 4 * e));
  }
  __syncwarp();
}

// k3 forward of a real line pair: twist by e^{-i pi n/(2N)}, FFT_N, spectrum quads out
template <int N, bool GSM>
__device__ __forceinline__ void k3_forward(const float (&a)[N], const float (&b)[N], float4* g,
                                           uint64_t pol) {
  pc z[N];
  sfor<0, N>([&](auto I) {
    constexpr int n = decltype(I)::value;
    constexpr float c = CS<n, 4 * N>::c, s = CS<n, 4 * N>::s;
    z[n].re = f2(a[n] * c, b[n] * c);
    z[n].im = f2(-a[n] * s, -b[n] * s);
  });
  fft_pk<N, false>(z);
#pragma unroll
  for (int j = 0; j < N; ++j)
    g_store<GSM>(g + (size_t)j * (N * N / 2), make_float4(z[j].re.x, z[j].re.y, z[j].im.x, z[j].im.y), pol);
}

// (E, O) = (x, x e^{-i pi n/N}) from the complex value x at index n
template <int N, int n>
__device__ __forceinline__ pc split_pair(float re, float im) {
  constexpr float c = CS<n, 2 * N>::c, s = CS<n, 2 * N>::s;
  return {f2(re, fmaf(im, s, re * c)), f2(im, fmaf(-re, s, im * c))};
}
// y_n = E_n + e^{+i pi n/N} O_n (the cropped inverse of a padded spectrum)
template <int N, int n>
__device__ __forceinline__ float2 join_pair(const pc& y) {
  constexpr float c = CS<n, 2 * N>::c, s = CS<n, 2 * N>::s;
  return make_float2(fmaf(-s, y.im.y, fmaf(c, y.re.y, y.re.x)), fmaf(s, y.re.y, fmaf(c, y.im.y, y.im.x)));
}

// slab-buffer quad jj of a row: (E.re, O.re, E.im, O.im), halves swapped when jj & 8
template <int jj>
__device__ __forceinline__ void v_store(float* row, const pc& x) {
  float4 v = (jj & 8) ? make_float4(x.im.x, x.im.y, x.re.x, x.re.y) : make_float4(x.re.x, x.re.y, x.im.x, x.im.y);
  *reinterpret_cast<float4*>(row + 4 * jj) = v;
}
template <int jj>
__device__ __forceinline__ pc v_load(const float* row) {
  const float4 v = *reinterpret_cast<const float4*>(row + 4 * jj);
  if constexpr (jj & 8) return {f2(v.z, v.w), f2(v.x, v.y)};
  else return {f2(v.x, v.y), f2(v.z, v.w)};
}

// The 2-D padded convolution of one slab in place.  g: the slab's N x N/2 spectrum quads; Vs: its
// buffer (N rows of stride RS); sg: the slab's symbol (L/4 x L quads).  Lanes r < N (row r) do
// the row passes; the column pass takes columns cc = lane + 32 rnd over all slabs of the warp.
template <int N, bool GSM>
__device__ __forceinline__ void slab_rows_forward(const float4* g, float* vrow, uint64_t pol) {
  using C = PkCfg<N>;
  pc x[N];
#pragma unroll
  for (int mm = 0; mm < N / 2; ++mm) {
    const float4 v = g_load<GSM>(g + mm * N, pol);
    x[2 * mm] = {f2(v.x, 0.f), f2(v.z, 0.f)};
    x[2 * mm + 1] = {f2(v.y, 0.f), f2(v.w, 0.f)};
  }
  sfor<0, N>([&](auto I) {
    constexpr int n = decltype(I)::value;
    x[n] = split_pair<N, n>(x[n].re.x, x[n].im.x);
  });
  fft_pk<N, false>(x);
  sfor<0, N>([&](auto J) { v_store<decltype(J)::value>(vrow, x[decltype(J)::value]); });
  (void)C::RS;
}

template <int N>
__device__ __forceinline__ void slab_column(float* Vc, int c, const float4* sg, uint64_t spol) {
  using C = PkCfg<N>;
  constexpr int RS = C::RS, L = C::L;
  const int jc = c >> 1, h = c & 1;
  const int ore = 4 * jc + ((jc & 8) ? 2 : 0) + h, oim = ore ^ 2;
  pc y[N];
  sfor<0, N>([&](auto I) {
    constexpr int n = decltype(I)::value;
    y[n] = split_pair<N, n>(Vc[n * RS + ore], Vc[n * RS + oim]);
  });
  fft_pk<N, false>(y);
#pragma unroll
  for (int q = 0; q < L / 4; ++q) {
    const float4 w = ldg_stream4(sg + (size_t)q * L + c, spol);
    const float2 w0 = f2(w.x, w.y), w1 = f2(w.z, w.w);
    y[2 * q].re = mul2(y[2 * q].re, w0);
    y[2 * q].im = mul2(y[2 * q].im, w0);
    y[2 * q + 1].re = mul2(y[2 * q + 1].re, w1);
    y[2 * q + 1].im = mul2(y[2 * q + 1].im, w1);
  }
  fft_pk<N, true>(y);
  sfor<0, N>([&](auto I) {
    constexpr int n = decltype(I)::value;
    const float2 o = join_pair<N, n>(y[n]);
    Vc[n * RS + ore] = o.x;
    Vc[n * RS + oim] = o.y;
  });
}

template <int N, bool GSM>
__device__ __forceinline__ void slab_rows_inverse(float4* g, const float* vrow, uint64_t pol) {
  pc x[N];
  sfor<0, N>([&](auto J) { x[decltype(J)::value] = v_load<decltype(J)::value>(vrow); });
  fft_pk<N, true>(x);
  sfor<0, N / 2>([&](auto M) {
    constexpr int mm = decltype(M)::value;
    const float2 a = join_pair<N, 2 * mm>(x[2 * mm]);
    const float2 b = join_pair<N, 2 * mm + 1>(x[2 * mm + 1]);
    g_store<GSM>(g + mm * N, make_float4(a.x, b.x, a.y, b.y), pol);
  });
}

// X2: the second input and base terms (in2, base2) are read (the LPC1 corrector).  REAL: the
// table holds the real spectrum of an even kernel (the plain TKM convolution with T): no deferred
// factor i, the result is Re[e^{i phi} y].
template <int N, bool X2, bool REAL = false>
__global__ void __launch_bounds__(PkCfg<N>::NT, PkCfg<N>::MINB) k_theta_pk(const PkParams p) {
  using C = PkCfg<N>;
  constexpr int NT = C::NT, NW = C::NW, SPW = C::SPW, L = C::L, RS = C::RS;
  constexpr int N3 = N * N * N, NP = N * N / 2, SQ = N * N / 2;   // line pairs, quads per slab
  constexpr bool GSM = C::GSM;
  extern __shared__ __align__(16) float smf[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* Vw = smf + warp * C::VW;
  float4* G = GSM ? reinterpret_cast<float4*>(smf + NW * C::VW) : p.G + (size_t)blockIdx.x * C::GQ;
  const uint64_t pol = l2_keep_policy();
  const uint64_t spol = l2_stream_policy();
  const int sub = lane / N, r = lane % N;

  // Phase A for line pair pr of x point xq: k3 forward of the stage-0 input
  auto phase_a = [&](int64_t xq, int pr) {
    const int k1 = pr % N, m = pr / N;
    const size_t off = (size_t)xq * N3 + ((size_t)k1 * N + 2 * m) * N;
    const size_t offm = (size_t)xq * N3 + (size_t)2 * m * N;   // the warp's common part (N = 32)
    float a[N], b[N];
    if constexpr (!GSM) warp_load_pairs<N>(p.in + offm, Vw, a, b);
    else load_pair<N>(p.in + off, a, b);
    if (X2 && p.in2) {   // u_0 = in + cin2 in2 (the LPC1 predictor)
      float a2[N], b2[N];
      if constexpr (!GSM) warp_load_pairs<N>(p.in2 + offm, Vw, a2, b2);
      else load_pair<N>(p.in2 + off, a2, b2);
#pragma unroll
      for (int n = 0; n < N; ++n) {
        a[n] = fmaf(p.cin2, a2[n], a[n]);
        b[n] = fmaf(p.cin2, b2[n], b[n]);
      }
    }
    k3_forward<N, GSM>(a, b, G + (size_t)m * N + k1, pol);
  };
  if (blockIdx.x < p.nxp) {
    for (int pr = tid; pr < NP; pr += NT) phase_a(blockIdx.x, pr);
  }
  __syncthreads();

  for (int64_t xp = blockIdx.x; xp < p.nxp; xp += gridDim.x) {
    for (int st = 0; st < p.nst; ++st) {
      // ---- Phase B: one warp per slab group ----
      for (int s0 = warp * SPW; s0 < N; s0 += NW * SPW) {
        if (lane == 0) {   // the symbol slabs this warp needs next, into L2
          const int sn = s0 + NW * SPW < N ? s0 + NW * SPW : warp * SPW;
          const int64_t xn = s0 + NW * SPW < N || st + 1 < p.nst ? xp : xp + gridDim.x;
          if (xn < p.nxp)
            bulk_prefetch_l2(p.sig + xn * p.sig_xs + sn * (int64_t)(L * L), SPW * L * L * sizeof(float));
        }
        float* Vs = Vw + sub * N * RS;
        float4* gs = G + (size_t)(s0 + sub) * SQ;
        slab_rows_forward<N, GSM>(gs + r, Vs + r * RS, pol);
        __syncwarp();
#pragma unroll 1
        for (int rnd = 0; rnd < 2; ++rnd) {
          const int cc = lane + 32 * rnd, sc = cc / L, c = cc % L;
          const float4* sg = reinterpret_cast<const float4*>(p.sig + xp * p.sig_xs) + (s0 + sc) * (int64_t)(L * L / 4);
          slab_column<N>(Vw + sc * N * RS, c, sg, spol);
        }
        __syncwarp();
        slab_rows_inverse<N, GSM>(gs + r, Vs + r * RS, pol);
        __syncwarp();
      }
      __syncthreads();

      float nc = p.ncoef[0];   // static indexing keeps the parameter block out of local memory
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (q == st) nc = p.ncoef[q];
      const bool last = st == p.nst - 1;

      // ---- Phase CA: k3 inverse, Theta, Horner update; the next stage's k3 forward ----
      for (int pr = tid; pr < NP; pr += NT) {
        const int k1 = pr % N, m = pr / N;
        const size_t off = (size_t)xp * N3 + ((size_t)k1 * N + 2 * m) * N;
        const size_t offm = (size_t)xp * N3 + (size_t)2 * m * N;
        float4* g = G + (size_t)m * N + k1;
        pc y[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float4 v = g_load<GSM>(g + (size_t)j * SQ, pol);
          y[j] = {f2(v.x, v.y), f2(v.z, v.w)};
        }
        fft_pk<N, true>(y);
        float a[N], b[N];   // Horner base of the two lines
        if (p.base) {
          if constexpr (!GSM) warp_load_pairs<N>(p.base + offm, Vw, a, b);
          else load_pair<N>(p.base + off, a, b);
          if (X2 && p.base2) {
            float a2[N], b2[N];
            if constexpr (!GSM) warp_load_pairs<N>(p.base2 + offm, Vw, a2, b2);
            else load_pair<N>(p.base2 + off, a2, b2);
#pragma unroll
            for (int n = 0; n < N; ++n) {
              a[n] = fmaf(p.cbase2, a2[n], a[n]);
              b[n] = fmaf(p.cbase2, b2[n], b[n]);
            }
          }
        } else {
#pragma unroll
          for (int n = 0; n < N; ++n) a[n] = b[n] = 0.f;
        }
        sfor<0, N>([&](auto I) {   // v = base - c_s (sin phi Re y + cos phi Im y), phi = pi n/(2N)
          constexpr int n = decltype(I)::value;
          constexpr float c = CS<n, 4 * N>::c, s = CS<n, 4 * N>::s;
          const float2 th = REAL ? fma2(y[n].re, f2(c, c), mul2(y[n].im, f2(-s, -s)))   // Re[e^{i phi} y]
                                 : fma2(y[n].im, f2(c, c), mul2(y[n].re, f2(s, s)));
          a[n] = fmaf(nc, th.x, a[n]);
          b[n] = fmaf(nc, th.y, b[n]);
        });
        if (last) {
          if constexpr (!GSM) warp_store_pairs<N>(p.out + offm, Vw, a, b);
          else store_pair<N>(p.out + off, a, b);
          // this thread alone used these spectrum columns: the next x point's Phase A for the
          // same line pair writes them without a barrier
          if (xp + gridDim.x < p.nxp) phase_a(xp + gridDim.x, pr);
        } else
          k3_forward<N, GSM>(a, b, g, pol);
      }
      __syncthreads();
    }
  }
}

template <int N>
void plan_pk_n(int64_t nxp, int num_sms, ThetaPlan* pl) {
  using C = PkCfg<N>;
  int nb = 0;
  cudaFuncSetAttribute(k_theta_pk<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes);
  cudaFuncSetAttribute(k_theta_pk<N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)C::smem_bytes);
  if (cudaFuncSetAttribute(k_theta_pk<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::smem_bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_theta_pk<N, false>, C::NT, C::smem_bytes) !=
          cudaSuccess ||
      nb < 1)
    nb = 1;
  pl->cluster = 0;
  pl->blocks = (int)std::min<int64_t>(nxp, (int64_t)nb * num_sms);
  pl->scratch_bytes = C::GSM ? 0 : (size_t)pl->blocks * C::GQ * sizeof(float4);
}

template <int N>
cudaError_t launch_pk_n(const Handle& H, const void* in, const void* base, void* out, int nst,
                        const double* coef, const XsExtra& x, cudaStream_t s) {
  using C = PkCfg<N>;
  PkParams p;
  p.in = static_cast<const float*>(in);
  p.base = static_cast<const float*>(base);
  p.in2 = static_cast<const float*>(x.in2);
  p.base2 = static_cast<const float*>(x.base2);
  p.cin2 = (float)x.cin2;
  p.cbase2 = (float)x.cbase2;
  p.out = static_cast<float*>(out);
  p.nxp = H.g.nxp;
  p.sig = static_cast<const float*>(x.sig ? x.sig : H.d_sig);
  p.sig_xs = x.sig ? 0 : (int64_t)N * C::L * C::L;
  p.nst = nst;
  for (int q = 0; q < 4; ++q) p.ncoef[q] = q < nst ? (float)(x.real_symbol ? coef[q] : -coef[q]) : 0.f;
  p.G = static_cast<float4*>(H.d_scratch);
  if (x.real_symbol) {
    if (x.in2 || x.base2) return cudaErrorInvalidValue;
    k_theta_pk<N, false, true><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  } else if (x.in2 || x.base2) {
    k_theta_pk<N, true><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  } else {
    k_theta_pk<N, false><<<H.theta.blocks, C::NT, C::smem_bytes, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace

bool theta_pk_applies(int nk, bool fp64) { return !fp64 && (nk == 16 || nk == 32); }

void theta_pk_plan(int nk, int64_t nxp, int num_sms, ThetaPlan* pl) {
  if (nk == 16) plan_pk_n<16>(nxp, num_sms, pl);
  else plan_pk_n<32>(nxp, num_sms, pl);
}

cudaError_t launch_theta_pk(const Handle& H, const void* in, const void* base, void* out, int nst,
                            const double* coef, cudaStream_t s, const XsExtra& x) {
  if (nst < 1 || nst > 4 || !H.d_sig) return cudaErrorInvalidValue;
  if (H.g.nk == 16) return launch_pk_n<16>(H, in, base, out, nst, coef, x, s);
  if (H.g.nk == 32) return launch_pk_n<32>(H, in, base, out, nst, coef, x, s);
  return cudaErrorInvalidValue;
}

}  // namespace chasm
