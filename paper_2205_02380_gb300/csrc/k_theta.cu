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
#include "fft_reg.cuh"

namespace chasm {
namespace {

namespace cg = cooperative_groups;


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
