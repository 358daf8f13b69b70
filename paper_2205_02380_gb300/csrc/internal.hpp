// Internal host-side declarations shared by the translation units of libchasm.
// Not part of the public ABI (include/chasm.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/chasm.h"

namespace chasm {

constexpr int kMaxNuclei = 8;

// Device-side description of the grid used by every kernel.
struct GridDesc {
  int nx[3];        // x points per dimension
  int nk;           // k points per dimension
  int64_t nxp;      // nx0 * nx1 * nx2 (x points)
  int64_t kvol;     // nk^3 (cells per x point)
  int64_t ncell;    // nxp * kvol
  double h[3];      // x spacings
  double x_lo[3];
  double lk;        // k half-width
  double dk;        // 2 lk / nk
};

// Per-dimension advection tables for one tau (A(tau), Sec. 3.2): for every k index the integer
// part n = floor(alpha) and the four B-spline weights (b4, b3, b2, b1)(alpha - n) of Eq. 3.7.
struct AdvectTables {
  double tau = 0.0;
  bool valid = false;
  void* dev = nullptr;      // [3][nk] weights (T x4) followed by [3][nk] int shifts
  int ns_min[3] = {0, 0, 0}, ns_max[3] = {0, 0, 0};   // range of the integer shifts per dim
};

struct Handle;

// ---- kernel launchers (defined in the .cu files) ----
// advection (k_advect.cu)
constexpr int kAdvectThreads = 128;
constexpr int kAdvectMaxSmem = 200 * 1024;
// shared-memory elements per line of the general advection kernel: the line (n + 2), and for
// p > 1 patches the line, the p + 1 closure values (hi and lo parts) and the p (M + 3) patch
// coefficients
inline size_t advect_smem_elems(int n, int p) {
  return p > 1 ? (size_t)n + 2 * (p + 1) + (size_t)p * ((n - 1) / p + 3) : (size_t)n + 2;
}
// threads per block of the shared-memory advection kernels: kAdvectThreads, or fewer (a multiple
// of 32) for long lines so that the block's line buffers fit kAdvectMaxSmem; 0 if even 32 lines
// do not fit
inline int advect_smem_threads(size_t elems, size_t elt) {
  const size_t per = elems * elt;
  const int b = (int)std::min<size_t>(kAdvectThreads, (size_t)kAdvectMaxSmem / per / 32 * 32);
  return b >= 32 ? b : 0;
}
cudaError_t advect_prepare();
cudaError_t launch_advect_dim(const Handle& H, void* f, int dim, cudaStream_t s);
// Coulomb operator (k_theta.cu): out = (base or 0) + sum_a coef[a] * Theta_a[in]
cudaError_t launch_theta(const Handle& H, const void* in, const void* base, void* out,
                         const double* coef, cudaStream_t s);
struct ThetaPlan {
  int cluster = 0;          // CTAs per cluster of the distributed-shared-memory kernel, 0 = global
  int blocks = 0;           // grid size (a multiple of cluster)
  size_t scratch_bytes = 0; // global scratch of the fallback kernel
};
void theta_plan(int nk, bool fp64, int64_t nxp, int num_sms, ThetaPlan* plan);
// real form with the per-x symbol table (k_theta_xs.cu): u_0 = in + cin2 in2, u_{s+1} =
// (base + cbase2 base2, or 0) + coef[s] Theta^T[u_s] for s < nst (1..4), out = u_nst; out may
// alias in, in2, base and base2 (in2, base2 null: the plain forms)
struct XsExtra {
  const void* in2 = nullptr;
  const void* base2 = nullptr;
  double cin2 = 0.0, cbase2 = 0.0;
  // the plain TKM convolution (chasm_tkm_convolve): sig replaces the per-x table, one table for
  // every x point, holding the real spectrum of T (the output is then T * in, no sine kernel)
  const void* sig = nullptr;
  bool real_symbol = false;
};
cudaError_t launch_theta_xs(const Handle& H, const void* in, const void* base, void* out, int nst,
                            const double* coef, cudaStream_t s, const XsExtra& x = XsExtra());
void theta_xs_plan(int nk, bool fp64, int64_t nxp, int num_sms, ThetaPlan* plan);
// LPC1 (k_lpc1.cu): Theta of the quadratic potential, out = (base or 0) + coef Theta[in]
// (in must not alias out), and the predictor/corrector combination v = f + dt h, f = f + dt/2 h
cudaError_t launch_theta_harm(const Handle& H, const void* in, const void* base, void* out,
                              double coef, cudaStream_t s);
cudaError_t launch_lpc1_combine(const Handle& H, void* f, const void* h, void* v, double dt,
                                cudaStream_t s);
// phase-space diagnostics (k_diag.cu): what = 0 reduced Wigner W_j, 1 marginal P(x1, x2),
// 2 averages <x_d>, <k_d>; buf holds diag_bytes of FP64 scratch, out_dev the result
size_t diag_bytes(const int nx[3], int nk);
cudaError_t launch_diag(const Handle& H, const void* f, int what, int j, double* buf, double* out_dev,
                        cudaStream_t s);
// SIMT FMA throughput of the current device in TFLOP/s (k_peak.cu); either pointer may be null
cudaError_t measure_fma_peaks(double* fp32_tflops, double* fp64_tflops);
cudaError_t measure_fma_peak_f32x2(double* tflops);
cudaError_t measure_fft_pk_rate(double* tflops);
// the per-x symbol table (k_xsym.cu), [nxp][N][2N][2N] in the storage type; needs H.d_T
size_t xs_table_bytes(int nk, int64_t nxp, size_t elt);
cudaError_t build_xs_table(const Handle& H, void* sig, cudaStream_t s);
// the spectrum of T on the same frequencies, (2 / (2N)^3) sum_m T_m e^{-i omega . m} (real: T is
// even), one x point's worth of table in the layout of the per-x table; needs H.d_T
cudaError_t build_tkm_table(const Handle& H, void* out, cudaStream_t s);
// Packed single-precision variant of the table-form P(dt) kernel (k_theta_pk.cu), used for
// FP32-mixed handles with N_k = 16 or 32: its symbol table has the layout
// [x][j][xi1 / 4][xi2][xi1 % 4] (k_xsym.cu writes it), the other cases [x][j][s1][s2]
// parity-major.
__host__ __device__ constexpr bool xs_packed(bool fp64, int nk) { return !fp64 && (nk == 16 || nk == 32); }
void theta_pk_plan(int nk, int64_t nxp, int num_sms, ThetaPlan* plan);
cudaError_t launch_theta_pk(const Handle& H, const void* in, const void* base, void* out, int nst,
                            const double* coef, cudaStream_t s, const XsExtra& x);

constexpr size_t kXsAutoMaxBytes = (size_t)64 << 30;

#ifdef __CUDACC__
// hi + lo += v with Knuth's error-free two-sum (the rounding error of hi + v goes to lo): the
// compensated single-precision sums of the reductions
__device__ __forceinline__ void two_sum_f(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}
#endif   // CHASM_THETA_AUTO limit without a device
// symbol precompute (k_symbol.cu): T (FP64, (2N-1)^3) and T-hat (parity-major, scaled)
cudaError_t compute_symbol(int nk, double lk, double* T_dev, void* that_dev, bool fp64,
                           double* that_absmax_host, cudaStream_t s);
// misc (k_misc.cu)
cudaError_t launch_moments(const Handle& H, const void* f, double* partials, double* result_dev,
                           cudaStream_t s);
cudaError_t launch_kshift(const Handle& H, void* f, int dim, const void* rows, cudaStream_t s);
cudaError_t launch_init_gaussians(const Handle& H, void* f, const chasm_gaussian* g, int n,
                                  cudaStream_t s);
cudaError_t launch_init_1s(const Handle& H, void* f, int n_y, const double c[3], cudaStream_t s,
                           std::string* err);
int moments_blocks();

struct Handle {
  chasm_grid grid{};
  chasm_box box{};
  double hbar = 1.0, m = 1.0;
  chasm_options opt{};
  std::vector<chasm_nucleus> nuclei;
  double kappa = 0.0;
  double center[3] = {0, 0, 0};
  bool fp64 = false;
  size_t elt = 4;
  GridDesc g{};
  int device = 0;
  int num_sms = 0;

  cudaStream_t stream = nullptr;
  bool own_stream = false;

  // PMBC end stencils (Eq. 3.5) and LU factors of the Hermite-closed system per dimension
  int J[3] = {0, 0, 0};            // stencil lengths min(n_nb, N) + 1
  // closure coefficients, zero-padded to nx[d] per segment: FP64 [c+ | c-], FP32-mixed
  // [c+ hi | c+ lo | c- hi | c- lo] (unevaluated float pairs for the compensated dot product)
  void* d_clos[3] = {nullptr, nullptr, nullptr};
  void* d_lu[3] = {nullptr, nullptr, nullptr};   // [cprime (n) | mult (n)] in storage type
  // patches p > 1 (Sec. 3.1.2): closure windows [(p+1)][W] (FP32: [(p+1)][2][W] hi/lo) for the
  // nodes b M - n_nb + i, W = 2 n_nb + 1, and the LU factors of the (M+1)-node patch system
  void* d_pclos[3] = {nullptr, nullptr, nullptr};
  void* d_plu[3] = {nullptr, nullptr, nullptr};
  // host copies (FP64) of the closure stencils [c+ (n) | c- (n)] and LU factors [cprime | mult],
  // passed by value to the register advection kernel
  std::vector<double> h_clos[3], h_lu[3];

  AdvectTables adv;                // current tau tables
  // Coulomb
  double* d_T = nullptr;           // FP64 T_p, (2N-1)^3
  void* d_that = nullptr;          // T-hat, storage type, (2N)^3 parity-major, / (2N)^3
  double that_absmax = 0.0;
  void* d_phase = nullptr;         // modulation tables (storage type complex)
  bool xs = false;                 // table (real) form of Theta^T, else the modulated form
  void* d_sig = nullptr;           // per-x symbol table of the table form
  void* d_tkm = nullptr;           // spectrum of T in the table layout (chasm_tkm_convolve)
  ThetaPlan theta;                 // launch plan of the Theta kernel
  void* d_scratch = nullptr;       // per-CTA scratch of the global-scratch Theta kernel
  void* d_u[2] = {nullptr, nullptr};  // Horner buffers
  // harmonic
  void* d_krows = nullptr;         // circulant rows [3][nx_d][nk] for the current dt
  double krows_dt = 0.0;
  bool krows_valid = false;
  // reductions
  double* d_partials = nullptr;
  double* d_result = nullptr;
  double* d_vx = nullptr;          // V(x) per x point (FP64)
  double* d_diag = nullptr;        // diagnostics: per-x partial sums and the result
  // host-buffer entry point
  void* d_fhost = nullptr;
  // step graph cache (one Strang or LPC1 step) and the kernel launches it holds
  cudaGraphExec_t graph = nullptr;
  int64_t graph_nodes = 0;
  void* graph_f = nullptr;
  double graph_dt = 0.0;
  int64_t launches = 0;            // kernels issued by the stepping calls (chasm_launch_count)

  std::string err;
  size_t workspace = 0;
};

// Returns a message for the last error on this thread when no handle exists.
void set_thread_error(const std::string& e);

// The checks chasm_create applies to grid, box (may be NULL), potential, hbar and m; an empty
// string when they pass, else the message.
std::string validate_problem(const chasm_grid* grid, const chasm_box* box, const chasm_potential* pot,
                             double hbar, double m);

}  // namespace chasm
