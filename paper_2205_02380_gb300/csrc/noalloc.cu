// chasm_moments_noalloc: mass and energy of a caller's f without allocating any memory.
//
// Some callers cannot allocate device memory at the moment they need these diagnostics:
// services that hand their whole device-memory budget to solves up front (the serving loop of
// this library admits requests against such a budget, so a check that allocated could push the
// device past it or fail with out-of-memory), and plug-ins that only receive a device pointer from
// a host framework that owns all device memory and its allocator.  chasm_moments needs a handle,
// and a handle allocates its tables and work buffers; this variant needs neither.  Its scratch
// (one partial-sum triple per x point and the two results) is a fixed file-scope device array, so
// the library reserves that memory on every GPU that loads it, for as long as the process lives.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.hpp"

namespace chasm {
namespace {

constexpr int64_t kNoallocMaxXPoints = 64 * 64 * 64;   // 262144 x points: 6 MiB of scratch
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// [3 * x point]: sum f, sum |j - N/2|^2 f, V(x) sum f;  [3 * kNoallocMaxXPoints + 0/1]: results
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoallocMaxXPoints + 2];

struct NoallocArgs {
  int nx[3];
  int nk;
  double x_lo[3], h[3];
  int n_nuc;
  double pos[kMaxNuclei][3];
  double charge[kMaxNuclei];
  double kappa;
  double center[3];
};

// One block per x point: the two k-sums in a fixed tree order, and V(x) from its definition.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_moments_per_x(const T* __restrict__ f, NoallocArgs a,
                                                            double* __restrict__ part) {
  __shared__ double red[2][kThreads / 32];
  const int64_t xp = blockIdx.x;
  const int nk = a.nk, kvol = nk * nk * nk;
  const T* fx = f + xp * kvol;
  double s0 = 0.0, s2 = 0.0;
  for (int e = threadIdx.x; e < kvol; e += kThreads) {
    const double v = (double)fx[e];
    const int k3 = e % nk - nk / 2, k2 = (e / nk) % nk - nk / 2, k1 = e / (nk * nk) - nk / 2;
    s0 += v;
    s2 += v * (double)(k1 * k1 + k2 * k2 + k3 * k3);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t2 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t0 += red[0][w];
      t2 += red[1][w];
    }
    const int i3 = (int)(xp % a.nx[2]), i2 = (int)((xp / a.nx[2]) % a.nx[1]);
    const int i1 = (int)(xp / ((int64_t)a.nx[2] * a.nx[1]));
    const double x[3] = {a.x_lo[0] + i1 * a.h[0], a.x_lo[1] + i2 * a.h[1], a.x_lo[2] + i3 * a.h[2]};
    double V = 0.0;
    if (a.n_nuc > 0) {
      for (int n = 0; n < a.n_nuc; ++n) {
        const double d0 = x[0] - a.pos[n][0], d1 = x[1] - a.pos[n][1], d2 = x[2] - a.pos[n][2];
        V -= a.charge[n] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      }
    } else {
      for (int d = 0; d < 3; ++d) V += 0.5 * a.kappa * (x[d] - a.center[d]) * (x[d] - a.center[d]);
    }
    part[3 * xp + 0] = t0;
    part[3 * xp + 1] = t2;
    part[3 * xp + 2] = V * t0;
  }
}

// One block adds the per-x-point triples in a fixed order and writes mass and energy.
__global__ void __launch_bounds__(kThreads) k_moments_total(const double* __restrict__ part,
                                                            int64_t nxp, double cell, double kin,
                                                            double* __restrict__ out) {
  __shared__ double red[3][kThreads];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < nxp; i += kThreads) {
    a += part[3 * i];
    b += part[3 * i + 1];
    c += part[3 * i + 2];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0] * cell;
    out[1] = (red[1][0] * kin + red[2][0]) * cell;
  }
}

// Per-device set-up, done once with that device current: the device address of the scratch
// array (in host code the array's name is only a host-side stand-in) and the loading of the three
// kernels (with lazy module loading a kernel's first launch would otherwise load its code then,
// which needs device memory).  The cached address belongs to the device's primary context, the
// one the CUDA runtime uses.
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_moments_per_x<float>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_moments_per_x<double>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_moments_total);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace chasm

extern "C" int chasm_moments_noalloc(const void* f_dev, const chasm_grid* grid, const chasm_box* box,
                                     const chasm_potential* pot, double hbar, double m,
                                     int32_t precision, void* cuda_stream, double* mass,
                                     double* energy) {
  using namespace chasm;
  if (!f_dev || !grid || !box || !pot || (!mass && !energy)) {
    set_thread_error("moments_noalloc: f, grid, box, potential and an output are required");
    return CHASM_EINVAL;
  }
  if (precision != CHASM_FP32_MIXED && precision != CHASM_FP64) {
    set_thread_error("moments_noalloc: precision must be CHASM_FP32_MIXED or CHASM_FP64");
    return CHASM_EINVAL;
  }
  const std::string bad = validate_problem(grid, box, pot, hbar, m);
  if (!bad.empty()) {
    set_thread_error("moments_noalloc: " + bad);
    return CHASM_EINVAL;
  }
  const int nk = grid->nk[0];
  const int64_t nxp = (int64_t)grid->nx[0] * grid->nx[1] * grid->nx[2];
  if (nxp > kNoallocMaxXPoints) {
    set_thread_error("moments_noalloc: at most " + std::to_string(kNoallocMaxXPoints) +
                     " x points (nx1 nx2 nx3); this grid has " + std::to_string(nxp));
    return CHASM_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
  double* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &scratch);
  if (e != cudaSuccess) {
    set_thread_error(std::string("moments_noalloc: ") + cudaGetErrorString(e));
    return CHASM_ECUDA;
  }
  NoallocArgs a{};
  for (int d = 0; d < 3; ++d) {
    a.nx[d] = grid->nx[d];
    a.x_lo[d] = box->x_lo[d];
    a.h[d] = (box->x_hi[d] - box->x_lo[d]) / (grid->nx[d] - 1);
    a.center[d] = pot->harm_center[d];
  }
  a.nk = nk;
  a.n_nuc = pot->n_nuc;
  for (int n = 0; n < pot->n_nuc; ++n) {
    for (int d = 0; d < 3; ++d) a.pos[n][d] = pot->nuc[n].pos[d];
    a.charge[n] = pot->nuc[n].charge;
  }
  a.kappa = pot->harm_kappa;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // cudaLaunchKernel returns the status of this launch itself, so an earlier error of the
  // caller's own code is neither reported here nor cleared
  const void* fptr = f_dev;
  void* args1[] = {(void*)&fptr, (void*)&a, (void*)&scratch};
  e = cudaLaunchKernel(precision == CHASM_FP64 ? (const void*)k_moments_per_x<double>
                                               : (const void*)k_moments_per_x<float>,
                       dim3((unsigned)nxp), dim3(kThreads), args1, 0, s);
  const double dk = 2.0 * box->k_half[0] / nk;
  double cell = a.h[0] * a.h[1] * a.h[2] * dk * dk * dk;
  double kin = hbar * hbar / (2.0 * m) * dk * dk;
  int64_t n = nxp;
  double* res = scratch + 3 * kNoallocMaxXPoints;
  void* args2[] = {(void*)&scratch, (void*)&n, (void*)&cell, (void*)&kin, (void*)&res};
  if (e == cudaSuccess)
    e = cudaLaunchKernel((const void*)k_moments_total, dim3(1), dim3(kThreads), args2, 0, s);
  double out[2];
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_thread_error(std::string("moments_noalloc: ") + cudaGetErrorString(e));
    return CHASM_ECUDA;
  }
  if (mass) *mass = out[0];
  if (energy) *energy = out[1];
  return CHASM_OK;
}
