/*
 * chasm.h -- C ABI of the GB300 implementation of one Strang step of the CHASM scheme
 * (Xiong, Zhang, Shao: "A characteristic-spectral-mixed scheme for six-dimensional
 * Wigner-Coulomb dynamics", arXiv 2205.02380).
 *
 * The Wigner function f(x, k) lives on a uniform 6-D grid and is stored by the CALLER in device
 * memory as a contiguous array f[x1][x2][x3][k1][k2][k3] (k3 fastest), element type float
 * (CHASM_FP32_MIXED) or double (CHASM_FP64).  The base address must be 16-byte aligned.
 *
 *   x_d grid : nx[d] points including both ends, x_{d,j} = x_lo[d] + j h_d,
 *              h_d = (x_hi[d] - x_lo[d]) / (nx[d] - 1)                 (Sec. 2.2, N+1 points)
 *   k grid   : k_j = (j - N_k/2) dk, dk = 2 L_k / N_k, j = 0..N_k-1  (Sec. 5.2, k_zeta = zeta dk)
 *
 * One step S(dt) = A(dt/2) P(dt) A(dt/2) (Strang splitting, Sec. 2.2):
 *   A(tau)  spatial advection f(x - hbar k tau / m, k) by tensor-product cubic B-splines whose
 *           coefficients are closed by the perfectly matched boundary condition (Sec. 3, Eqs.
 *           3.5 and 3.10);
 *   P(dt)   the quantum interaction d f/dt = Theta_V[f].  For V = -sum_A Z_A/|x - x_A| the
 *           Coulomb operator is applied with the truncated kernel method (Sec. 4, Eqs. 4.1,
 *           4.5-4.8) and the flow is the 4-term Taylor (Horner) polynomial of exp(dt Theta^T);
 *           for V = kappa/2 |x - c|^2 it is the exact shift f(x, k + dt kappa (x - c)/hbar)
 *           (Eq. 5.1).
 *
 * Every function returns an int status (CHASM_OK = 0, CHASM_PENDING = 1, negative = error).
 * On error the message is available from chasm_last_error(handle) (or chasm_last_error(NULL)
 * for errors raised before a handle exists).  No exception crosses this boundary.  All device
 * work is issued on the handle's CUDA stream; functions that return host values synchronise
 * that stream.  A handle must not be used from two host threads at the same time.
 */
#ifndef CHASM_H
#define CHASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CHASM_OK = 0,
  CHASM_PENDING = 1,      /* chasm_poll: the request is queued or running                    */
  CHASM_EINVAL = -1,      /* invalid argument (the message names it)                           */
  CHASM_ENOMEM = -2,      /* device or host allocation failed                                  */
  CHASM_ECUDA = -3,       /* a CUDA runtime call failed (message carries cudaGetErrorString)   */
  CHASM_EUNSTABLE = -4,   /* dt * rho(Theta^T) above the Taylor-4 stability limit 2.8          */
  CHASM_EBUSY = -5,       /* server: request larger than the whole HBM budget                  */
  CHASM_EAGAIN = -6,      /* server: submission queue full, retry later                        */
  CHASM_ETIMEOUT = -7,    /* chasm_wait: timed out                                             */
  CHASM_ENOTFOUND = -8,   /* server: unknown ticket                                            */
  CHASM_ECANCELED = -9    /* server: request cancelled before it finished                      */
};

enum { CHASM_FP32_MIXED = 0, CHASM_FP64 = 1 };

/* How the Coulomb operator Theta^T is evaluated (chasm_options.theta_form).  Both forms compute
 * the same truncated-kernel convolution (Eqs. 4.1, 4.5-4.7) and agree to rounding.
 *   CHASM_THETA_TABLE: the real form.  For each x point Theta^T[u] = sum_q S_{p-q}(x) u_q with the
 *     real, odd kernel S_m(x) = sum_A -(2 Z_A/(pi^2 hbar)) T_m sin(2 (x - x_A) . m dk); chasm_create
 *     tabulates the spectrum of S for every x point (4 N_k^3 values per x point, i.e. four copies
 *     of f) and each application then costs one real padded convolution for all nuclei together
 *     (half the FFT work of one nucleus in the modulated form).  P(dt) runs its four Horner
 *     stages per x point in one kernel and needs no Horner buffers.
 *   CHASM_THETA_MODULATED: the complex form of Eq. 4.6 per nucleus (modulate by e^{-2i(x-x_A).k},
 *     convolve with T, demodulate, imaginary part); workspace two copies of f.
 *   CHASM_THETA_AUTO (default): the table form when the table needs at most half of the current
 *     device's memory (64 GiB when no device can be queried), else the modulated form. */
enum { CHASM_THETA_AUTO = 0, CHASM_THETA_TABLE = 1, CHASM_THETA_MODULATED = 2 };

/* Time integrator of chasm_step (chasm_options.integrator).
 *   CHASM_STRANG (default): S(dt) = A(dt/2) P(dt) A(dt/2), P the Horner-Taylor-4 flow of Theta^T
 *     (Coulomb) or the exact k-shift (quadratic potential).
 *   CHASM_LPC1: the one-stage Lawson predictor-corrector of Sec. 2.2,
 *       f~  = f(A_dt) + dt Theta_V[f](A_dt),
 *       f'  = f(A_dt) + dt/2 Theta_V[f~] + dt/2 Theta_V[f](A_dt),
 *     g(A_dt(x, k)) = g(x - hbar k dt / m, k) evaluated by the advection of Sec. 3 (one
 *     advection of f and one of Theta_V[f] per step) and Theta_V applied twice per step; for the
 *     quadratic potential Theta_V f = kappa (x - c)/hbar . grad_k f with the spectral k-derivative.
 *     Needs more workspace: one copy of f in the table form (the predictor is formed inside the
 *     Theta kernel), two for the quadratic potential; the modulated Coulomb form already has them.
 *     EUNSTABLE when dt rho > 1, rho the spectral-radius bound of Theta_V (chasm_step below). */
enum { CHASM_STRANG = 0, CHASM_LPC1 = 1 };

/* Grid: points per dimension.  nx[d] >= 4; nk[0] = nk[1] = nk[2] in {8, 16, 32}.  Lines that are
 * neither 16, 24, 32, 48 nor 64 points long (or patches > 1) are advected in shared memory, which
 * bounds nx[d]: at most 798 points in FP64 and 1598 in FP32-mixed with one patch (about half that
 * with patches); chasm_create returns EINVAL beyond. */
typedef struct {
  int32_t nx[3];
  int32_t nk[3];
} chasm_grid;

/* Box: x in [x_lo, x_hi] (both ends are grid points); k in [-k_half, k_half) with
 * k_half[0] = k_half[1] = k_half[2] = L_k (the TKM of Sec. 4 is built on a cube). */
typedef struct {
  double x_lo[3];
  double x_hi[3];
  double k_half[3];
} chasm_box;

/* One nucleus of V = -sum_A charge_A / |x - pos_A| (attractive for charge > 0). */
typedef struct {
  double pos[3];
  double charge;
} chasm_nucleus;

/* Potential: n_nuc > 0 selects the Coulomb operator (at most 8 nuclei); n_nuc == 0 selects the
 * quadratic potential kappa/2 |x - center|^2 (kappa may be 0: free streaming). */
typedef struct {
  const chasm_nucleus* nuc;
  int32_t n_nuc;
  double harm_kappa;
  double harm_center[3];
} chasm_potential;

typedef struct {
  int32_t precision;    /* CHASM_FP32_MIXED (default) or CHASM_FP64                         */
  int32_t n_nb;         /* PMBC stencil length n_nb of Eq. 3.2 (default 20, >= 1)           */
  int32_t patches[3];   /* PMBC patches per x-dimension p (Sec. 3.1.3; default 1): p divides
                           nx - 1 and leaves at least 2 intervals per patch, else EINVAL     */
  int32_t use_graphs;   /* 1 (default): chasm_step replays a captured CUDA graph per step   */
  void* cuda_stream;    /* cudaStream_t to run on; NULL: the handle creates its own stream  */
  int32_t theta_form;   /* CHASM_THETA_AUTO (default), CHASM_THETA_TABLE, CHASM_THETA_MODULATED */
  int32_t integrator;   /* CHASM_STRANG (default) or CHASM_LPC1                              */
} chasm_options;

/* One initial wavepacket w exp(-ax |x - x0|^2 - ak |k - k0|^2). */
typedef struct {
  double w;
  double x0[3];
  double k0[3];
  double ax;
  double ak;
} chasm_gaussian;

typedef struct chasm_handle chasm_handle;

/* Fills *opt with the defaults listed above.  Never fails for a non-NULL pointer. */
int chasm_options_default(chasm_options* opt);

/* Creates a solver for one grid/box/potential.  Validates every argument (EINVAL), copies the
 * nuclei, builds the PMBC end stencils (Eq. 3.5) and the constant LU factors of the Hermite-
 * closed spline system (Eq. 2.14, step (5) of Sec. 3.1.2), runs the truncated-kernel symbol
 * precompute on the GPU (Eqs. 4.3, 4.7 and the DFT of the twofold-padded tensor, FP64), and
 * allocates the workspace reported by chasm_workspace_bytes.  hbar > 0, m > 0.
 * opt may be NULL (defaults).  On success *out owns all of this until chasm_destroy. */
int chasm_create(const chasm_grid* grid, const chasm_box* box, const chasm_potential* pot,
                 double hbar, double m, const chasm_options* opt, chasm_handle** out);

/* Frees everything the handle owns (waits for its stream first).  NULL is accepted. */
int chasm_destroy(chasm_handle* h);

/* Last error message of this handle (or of the calling thread when h == NULL). */
const char* chasm_last_error(const chasm_handle* h);

/* Device bytes the handle allocates besides the caller's f, for Coulomb potentials: in the table
 * form the per-x symbol table (4 N_k^3 elements per x point), in the modulated form two Horner
 * buffers; in both the per-CTA FFT scratch of the Theta kernel, the symbol T, T-hat and small
 * tables.  0 on invalid arguments. */
size_t chasm_workspace_bytes(const chasm_grid* grid, const chasm_potential* pot,
                             const chasm_options* opt);

/* Number of cells N_x1 N_x2 N_x3 N_k^3 and bytes of one copy of f for this handle. */
int64_t chasm_num_cells(const chasm_handle* h);
size_t chasm_f_bytes(const chasm_handle* h);

/* Replaces the stream the handle issues work on (cudaStream_t; NULL = legacy default stream).
 * Drops captured graphs. */
int chasm_set_stream(chasm_handle* h, void* cuda_stream);

/* Waits for all work issued on the handle's stream; reports asynchronous CUDA errors. */
int chasm_sync(chasm_handle* h);

/* nsteps steps of the handle's integrator (Strang: S(dt) = A(dt/2) P(dt) A(dt/2); LPC1: the
 * predictor-corrector above) on f_dev, in place, asynchronous on the handle's stream.  dt > 0 and
 * finite, nsteps >= 0.  EUNSTABLE: Strang/Coulomb if dt rho > 2.8 (the Taylor-4 limit on the
 * imaginary axis is 2 sqrt 2), rho = (2 sum|Z| / (pi^2 hbar)) max|T-hat|; LPC1 if dt rho > 1, rho
 * as for Strang (Coulomb) or (kappa / hbar) sum_d max_i |x_{d,i} - c_d| pi (N_k/2 - 1) / L_k
 * (quadratic potential). */
int chasm_step(chasm_handle* h, void* f_dev, double dt, int32_t nsteps);

/* Kernel launches issued on the handle's stream by chasm_step, chasm_advect and chasm_pflow
 * since chasm_create (a replayed graph counts each kernel it holds), in *out.  EINVAL when h or
 * out is NULL. */
int chasm_launch_count(const chasm_handle* h, int64_t* out);

/* The two substeps on their own (same layout, in place, asynchronous):
 *   chasm_advect: A(tau), any finite tau (tau = 0 is the identity up to rounding);
 *   chasm_pflow:  P(dt). */
int chasm_advect(chasm_handle* h, void* f_dev, double tau);
int chasm_pflow(chasm_handle* h, void* f_dev, double dt);

/* out = Theta_V[u]: Coulomb: sum_A -(2 Z_A / (pi^2 hbar)) Im[e^{2i(x-x_A).k} (T * (u e^{-2i(x-x_A).k}))]
 * (Eqs. 4.1, 4.6 with the sign of Eq. 2.3); quadratic potential: kappa (x - c)/hbar . grad_k u
 * (Eq. 5.1, spectral k-derivative without the Nyquist mode).  u and out must not alias; EINVAL for
 * kappa = 0 without nuclei. */
int chasm_theta(chasm_handle* h, const void* u_dev, void* out_dev);

/* phi = T * g: the truncated-kernel convolution of Sec. 4 without the modulation of Eq. 4.6,
 * phi(x, k_p) = sum_q T_{p-q} g(x, k_q) for every x point, with T of Eq. 4.7 (T carries dk^3, so
 * phi approximates the convolution (1/|k|^2 * g)(k) of Example 4.1).  g and phi have the layout
 * and element type of f; they must not alias.  Coulomb handles in the table form only (EINVAL
 * otherwise); the first call builds the spectrum of T on the handle's stream (one x point's worth
 * of the per-x table, FP64 precompute) and keeps it until chasm_destroy.  Asynchronous. */
int chasm_tkm_convolve(chasm_handle* h, const void* g_dev, void* phi_dev);

/* Mass h1 h2 h3 dk^3 sum f and energy h1 h2 h3 dk^3 sum (hbar^2 |k|^2 / 2m + V(x)) f, both
 * accumulated in FP64 with a fixed reduction tree (bitwise reproducible); synchronous. */
int chasm_mass(chasm_handle* h, const void* f_dev, double* out);
int chasm_energy(chasm_handle* h, const void* f_dev, double* out);
int chasm_moments(chasm_handle* h, const void* f_dev, double* mass, double* energy);

/* Phase-space diagnostics of Sec. 5, accumulated in FP64 in a fixed order (bitwise reproducible),
 * synchronous; f_dev as in chasm_step, results in host memory:
 *   chasm_reduced_wigner: W_j(x, k) = integral of f over the other two x and the other two k
 *     coordinates (grid sums times their cell volume), j in {0, 1, 2}; w_host[i][q] for the
 *     nx[j] x N_k nodes (x_{j,i}, k_q), row-major;
 *   chasm_marginal_x12: the spatial marginal P(x1, x2) = integral over x3 and k; p_host[i1][i2],
 *     nx[0] x nx[1];
 *   chasm_expectations: out_host[0..2] = <x_d> = sum x_d f / sum f and out_host[3..5] = <k_d>
 *     (the averaged position and momentum). */
int chasm_reduced_wigner(chasm_handle* h, const void* f_dev, int32_t j, double* w_host);
int chasm_marginal_x12(chasm_handle* h, const void* f_dev, double* p_host);
int chasm_expectations(chasm_handle* h, const void* f_dev, double* out_host);

/* Measures the SIMT fused-multiply-add throughput of the current device (independent FMA chains on
 * every SM, two flops per FMA), in TFLOP/s, FP32 and FP64: the ALU ceiling of the Coulomb kernels,
 * which are bound by plain FMA/add arithmetic.  Either pointer may be NULL (not both).  Allocates
 * and frees a small device buffer; synchronous, about a second.  Not part of the paper: a
 * measurement utility for roofline reports. */
int chasm_fma_peaks(double* fp32_tflops, double* fp64_tflops);

/* The same measurement with the packed single-precision FMA (two FP32 FMAs per instruction on
 * register pairs, sm_100 and later), four flops per instruction, in TFLOP/s: whether the pairs
 * raise the FP32 arithmetic ceiling or only halve the instructions issued.  Synchronous. */
int chasm_fma_peak_f32x2(double* tflops);

/* The register FFT of the FP32 table-form P(dt) kernel (N_k = 32) alone, in that kernel's CTA
 * shape (256 threads, one CTA per SM): forward and inverse packed 32-point FFTs on register data,
 * no memory traffic, flops counted as the kernel's roofline counts them (5 n log2 n per complex
 * length-n FFT), in TFLOP/s.  The ceiling of FFT arithmetic at that occupancy, beside the FMA
 * peaks above.  Synchronous. */
int chasm_fft_pk_rate(double* tflops);

/* Mass and energy exactly as chasm_moments defines them, for callers that cannot allocate
 * device memory when they need them: services that hand their whole device-memory budget to
 * solves up front (an allocation for a check could then fail or push the device past the budget)
 * and plug-ins that only receive a device pointer from a host framework that owns all device
 * memory.  The paper has no counterpart; this is a library convenience.  It needs no handle and
 * allocates nothing: its scratch is a fixed device array of 3 * 262144 + 2 doubles (6 MiB) that
 * the library reserves on every GPU that loads it until the process exits.  Hence at most 262144
 * x points (nx1 nx2 nx3, e.g. 64^3); larger grids are rejected with EINVAL and a message.  f_dev
 * has the layout and element type (precision) of chasm_step; grid, box, potential, hbar and m pass
 * the checks of chasm_create (else EINVAL); mass/energy are host pointers (either may be NULL, not
 * both).  Work runs on cuda_stream (NULL = the legacy default stream) and the call waits for it.
 * The first call on each device, with that device current, looks up the array's device address
 * and loads the entry point's kernels; the address is kept for the device's primary context (the
 * one the CUDA runtime uses), so the entry point must not be called again after cudaDeviceReset.
 * All calls share the one array and it keeps the last call's contents (every entry a call reads
 * is written by that call first), so calls whose work overlaps on the GPU race with each other:
 * serialise them. */
int chasm_moments_noalloc(const void* f_dev, const chasm_grid* grid, const chasm_box* box,
                          const chasm_potential* pot, double hbar, double m, int32_t precision,
                          void* cuda_stream, double* mass, double* energy);

/* Initial data written on the GPU (asynchronous):
 *   chasm_init_gaussians: f = sum_i w_i exp(-ax_i |x - x0_i|^2 - ak_i |k - k0_i|^2), 1 <= n <=
 *     16, evaluated in FP64 as products of the per-dimension factors and rounded to the storage
 *     type; f_dev 16-byte aligned (EINVAL otherwise);
 *   chasm_init_hydrogen_1s: the 1s Wigner function of phi = exp(-|x - c|)/(2 sqrt(2) pi^2) by
 *     the discrete Fourier sum of Sec. 5.2 with n_y samples per dimension (n_y a multiple of
 *     2 N_k, at most 256), dy = 2 pi / (N_k dk), computed in FP64 and rounded to the storage
 *     type.  It uses a temporary device buffer of at most 2 GiB. */
int chasm_init_gaussians(chasm_handle* h, void* f_dev, const chasm_gaussian* g, int32_t n);
int chasm_init_hydrogen_1s(chasm_handle* h, void* f_dev, int32_t n_y, const double center[3]);

/* Copies the FP64 convolution tensor T_p of Eq. 4.7, p in [-(N_k-1), N_k-1]^3, index
 * ((p1+N_k-1)(2N_k-1) + p2+N_k-1)(2N_k-1) + p3+N_k-1, to host memory ((2N_k-1)^3 doubles), as
 * computed by the symbol-precompute kernels of chasm_create.  Coulomb handles only. */
int chasm_tkm_tensor(chasm_handle* h, double* t_host);

/* End-to-end call with HOST buffers: copies f0_host (may be pinned or pageable) to a device
 * buffer owned by the handle, runs nsteps steps, copies the result to f_out_host (may equal
 * f0_host) and returns its mass.  Synchronous. */
int chasm_run_host(chasm_handle* h, const void* f0_host, void* f_out_host, double dt,
                   int32_t nsteps, double* mass_out);

/* ------------------------------------------------------------------------------------------
 * Continuous-batching server.  Requests (grid, potential, initial data, dt, steps, precision)
 * are admitted in arrival order whenever a slot is free and the sum of the admitted requests'
 * device bytes (f plus workspace) stays within hbm_budget_bytes.  Each admitted request owns a
 * stream, its f and its workspace; the scheduler thread issues its steps in chunks of
 * steps_per_launch (one captured CUDA graph launch per chunk), round-robin over the running
 * requests, so the work of different requests overlaps on the GPU.  A finished request's
 * resources are freed at once and the next queued request is admitted.  Results do not depend
 * on what else is running: every kernel's result is a function of its own request's data only.
 * ---------------------------------------------------------------------------------------- */

typedef struct chasm_server chasm_server;

typedef struct {
  chasm_grid grid;
  chasm_box box;
  chasm_nucleus nuclei[8];
  int32_t n_nuc;               /* 0: quadratic potential with harm_kappa, harm_center          */
  double harm_kappa;
  double harm_center[3];
  double hbar, m;
  int32_t precision;
  int32_t n_nb;
  double dt;
  int32_t nsteps;
  chasm_gaussian packets[4];   /* initial data when f0_host == NULL                            */
  int32_t n_packets;
  const void* f0_host;         /* optional initial f (copied at submission time)               */
  void* f_out_host;            /* optional destination of the final f (caller keeps it alive)  */
} chasm_request;

typedef struct {
  int32_t status;              /* CHASM_OK, or the error of this request                       */
  double mass, energy;         /* of the final f                                               */
  double queue_ms;             /* submission -> admission                                      */
  double run_ms;               /* admission -> completion                                      */
  double latency_ms;           /* submission -> completion                                     */
  int64_t cells;               /* N_x1 N_x2 N_x3 N_k^3                                         */
  int32_t nsteps;
} chasm_result;

/* max_slots in [1, 64]; steps_per_launch >= 1; hbm_budget_bytes > 0; queue_capacity >= 1. */
int chasm_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t steps_per_launch,
                        int32_t queue_capacity, chasm_server** out);
/* Queues a copy of *req.  EINVAL for an invalid request, EBUSY if it can never fit the budget,
 * EAGAIN if the queue is full. */
int chasm_submit(chasm_server* s, const chasm_request* req, uint64_t* ticket);
/* CHASM_PENDING while queued or running; CHASM_OK with *out filled once finished (the ticket is
 * then released); ENOTFOUND for an unknown or already collected ticket. */
int chasm_poll(chasm_server* s, uint64_t ticket, chasm_result* out);
/* Like chasm_poll but blocks up to timeout_s seconds (ETIMEOUT). */
int chasm_wait(chasm_server* s, uint64_t ticket, double timeout_s, chasm_result* out);
/* Cancels a queued or running request (its result reports ECANCELED). */
int chasm_cancel(chasm_server* s, uint64_t ticket);
/* Current queue length, running requests and bytes in use. */
int chasm_server_stats(chasm_server* s, int32_t* queued, int32_t* running, size_t* bytes_in_use);
/* Stops the scheduler (running requests are cancelled) and frees everything. */
int chasm_server_destroy(chasm_server* s);

#ifdef __cplusplus
}
#endif

#endif /* CHASM_H */
