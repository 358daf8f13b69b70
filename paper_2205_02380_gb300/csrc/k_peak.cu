// SIMT fused-multiply-add throughput of the current device, FP32 and FP64, for the ALU roofline
// of the Coulomb kernels (which are bound by plain FMA/add arithmetic, not by HBM or tensor cores).
// Every thread runs K independent FMA chains (enough independent work to hide the pipeline
// latency) for `iters` rounds; the grid covers every SM several times over.  Counted flops: two
// per FMA (four per packed FP32 FMA, which works on a register pair).  The chains' final values are
// written out so the compiler keeps the work.
#include "internal.hpp"
#include "fft_pk.cuh"

namespace chasm {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ out, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed single precision: each chain is a pair, one instruction does two FMAs
__global__ void __launch_bounds__(256) k_fma2_peak(float* __restrict__ out, int iters, float a, float b) {
  float2 v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x + 2 * c) * 1e-3f);
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], A, B);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// times one launch of `kern` (after a warm-up launch of a quarter of the iterations) over
// num_sms x 8 CTAs of 256 threads; flops_per_iter = flops one thread does per outer iteration
template <typename T, typename K>
cudaError_t time_peak(K kern, int num_sms, int iters, double flops_per_iter, T a, T b, double* tflops) {
  const int blocks = num_sms * 8, threads = 256;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&out, (size_t)blocks * threads * sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    kern<<<blocks, threads>>>(out, iters / 4, a, b);   // warm-up
    e = cudaEventRecord(e0);
    kern<<<blocks, threads>>>(out, iters, a, b);
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && ms > 0.f)
      *tflops = flops_per_iter * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return e;
}

// a = 1 - 2^-20, b = 2^-20: the chains stay bounded
template <typename T>
cudaError_t measure(int num_sms, int iters, double* tflops) {
  return time_peak<T>(k_fma_peak<T>, num_sms, iters, 2.0 * kChains * 16.0, (T)(1.0 - 1.0 / 1048576.0),
                      (T)(1.0 / 1048576.0), tflops);
}

// The register FFT of the packed P(dt) kernel alone, with that kernel's CTA shape (256 threads,
// one CTA per SM): every thread runs a forward and an inverse packed 32-point FFT (two
// transforms in lockstep) per round on register data and rescales by 1/32.  Counted flops: the
// 5 n log2 n per complex length-n FFT of the kernel's algorithmic count, 4 x 800 per round.
__global__ void __launch_bounds__(256, 1) k_fft_pk_rate(float* __restrict__ out, int rounds) {
  pc x[32];
#pragma unroll
  for (int n = 0; n < 32; ++n) {
    const float t = (float)(threadIdx.x + n) * 1e-3f;
    x[n] = {f2(t, t + 1.f), f2(t - 1.f, 0.5f * t)};
  }
  const float2 sc = f2(1.f / 32, 1.f / 32);
  for (int r = 0; r < rounds; ++r) {
    fft_pk<32, false>(x);
    fft_pk<32, true>(x);
#pragma unroll
    for (int n = 0; n < 32; ++n) {
      x[n].re = mul2(x[n].re, sc);
      x[n].im = mul2(x[n].im, sc);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int n = 0; n < 32; ++n) s += x[n].re.x + x[n].re.y + x[n].im.x + x[n].im.y;
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_fft_pk_rate(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int threads = 256, rounds = 400;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc((void**)&out, (size_t)sms * threads * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fft_pk_rate<<<sms, threads>>>(out, rounds / 4);   // warm-up
    e = cudaEventRecord(e0);
    k_fft_pk_rate<<<sms, threads>>>(out, rounds);
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    const double flops_per_round = 4.0 * 5.0 * 32.0 * 5.0;   // four length-32 transforms
    if (e == cudaSuccess && ms > 0.f)
      *tflops = flops_per_round * rounds * (double)sms * threads / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return e;
}

cudaError_t measure_fma_peaks(double* fp32_tflops, double* fp64_tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && fp32_tflops) e = measure<float>(sms, 256, fp32_tflops);
  if (e == cudaSuccess && fp64_tflops) e = measure<double>(sms, 8, fp64_tflops);
  return e;
}

cudaError_t measure_fma_peak_f32x2(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = time_peak<float>(k_fma2_peak, sms, 256, 4.0 * kChains * 16.0, 1.0f - 1.0f / 1048576.0f,
                         1.0f / 1048576.0f, tflops);
  return e;
}

}  // namespace chasm
