// C ABI of libchasm: argument validation, the plan (PMBC stencils, LU factors, tables, symbol),
// the Strang step driver with CUDA-graph replay, diagnostics and initial data.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.hpp"

namespace chasm {

namespace {
thread_local std::string g_thread_err;

int fail(Handle* H, int code, const std::string& msg) {
  if (H)
    H->err = msg;
  else
    g_thread_err = msg;
  return code;
}

int cuda_fail(Handle* H, cudaError_t e, const char* what) {
  return fail(H, CHASM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CHASM_CUDA(H, call)                          \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_fail(H, _e, #call); \
  } while (0)
// a kernel launch of the stepping calls, counted for chasm_launch_count
#define CHASM_LAUNCH(H, call)                        \
  do {                                               \
    CHASM_CUDA(H, call);                             \
    ++(H)->launches;                                 \
  } while (0)

bool is_finite(double v) { return std::isfinite(v); }

// Validation shared by create and workspace_bytes; returns an empty string when valid.
std::string validate(const chasm_grid* grid, const chasm_box* box, const chasm_potential* pot,
                     double hbar, double m, const chasm_options* opt) {
  if (!grid) return "grid is NULL";
  for (int d = 0; d < 3; ++d)
    if (grid->nx[d] < 4 || grid->nx[d] > 4096) return "nx[d] must be in [4, 4096]";
  if (grid->nk[0] != grid->nk[1] || grid->nk[0] != grid->nk[2])
    return "nk must be equal in the three k-dimensions";
  const int nk = grid->nk[0];
  if (nk != 8 && nk != 16 && nk != 32) return "nk must be 8, 16 or 32";
  if (box) {
    for (int d = 0; d < 3; ++d) {
      if (!is_finite(box->x_lo[d]) || !is_finite(box->x_hi[d]) || !(box->x_hi[d] > box->x_lo[d]))
        return "box: x_hi must exceed x_lo (finite)";
      if (!is_finite(box->k_half[d]) || !(box->k_half[d] > 0)) return "box: k_half must be > 0";
    }
    if (box->k_half[0] != box->k_half[1] || box->k_half[0] != box->k_half[2])
      return "box: k_half must be equal in the three dimensions";
  }
  if (pot) {
    if (pot->n_nuc < 0 || pot->n_nuc > kMaxNuclei) return "potential: n_nuc must be in [0, 8]";
    if (pot->n_nuc > 0 && !pot->nuc) return "potential: nuc is NULL";
    for (int a = 0; a < pot->n_nuc; ++a) {
      const chasm_nucleus& n = pot->nuc[a];
      if (!is_finite(n.charge) || !is_finite(n.pos[0]) || !is_finite(n.pos[1]) || !is_finite(n.pos[2]))
        return "potential: nucleus not finite";
    }
    if (!is_finite(pot->harm_kappa)) return "potential: harm_kappa not finite";
  }
  if (!(hbar > 0) || !is_finite(hbar)) return "hbar must be > 0";
  if (!(m > 0) || !is_finite(m)) return "m must be > 0";
  if (opt) {
    if (opt->precision != CHASM_FP32_MIXED && opt->precision != CHASM_FP64)
      return "options: precision must be CHASM_FP32_MIXED or CHASM_FP64";
    if (opt->n_nb < 1) return "options: n_nb must be >= 1";
    for (int d = 0; d < 3; ++d) {
      if (opt->patches[d] < 1) return "options: patches must be >= 1";
      if ((grid->nx[d] - 1) % opt->patches[d] != 0)
        return "options: patches[d] must divide nx[d] - 1";
      if (opt->patches[d] > 1 && (grid->nx[d] - 1) / opt->patches[d] < 2)
        return "options: patches[d] must leave at least 2 intervals per patch";
    }
    if (opt->theta_form != CHASM_THETA_AUTO && opt->theta_form != CHASM_THETA_TABLE &&
        opt->theta_form != CHASM_THETA_MODULATED)
      return "options: theta_form must be CHASM_THETA_AUTO, _TABLE or _MODULATED";
    if (opt->integrator != CHASM_STRANG && opt->integrator != CHASM_LPC1)
      return "options: integrator must be CHASM_STRANG or CHASM_LPC1";
  }
  return std::string();
}

// CHASM_THETA_AUTO limit: half of the current device's memory (kXsAutoMaxBytes when the device
// cannot be queried), looked up once per device.
size_t auto_table_limit() {
  static std::mutex mu;
  static size_t limit[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kXsAutoMaxBytes;
  std::lock_guard<std::mutex> lk(mu);
  if (!limit[dev]) {
    cudaDeviceProp prop;
    limit[dev] = cudaGetDeviceProperties(&prop, dev) == cudaSuccess && prop.totalGlobalMem > 0
                     ? prop.totalGlobalMem / 2
                     : kXsAutoMaxBytes;
  }
  return limit[dev];
}

// Whether the Coulomb operator uses the per-x symbol table.
bool table_form(int nk, int64_t nxp, size_t elt, const chasm_options& o) {
  if (o.theta_form == CHASM_THETA_TABLE) return true;
  if (o.theta_form == CHASM_THETA_MODULATED) return false;
  return xs_table_bytes(nk, nxp, elt) <= auto_table_limit();
}

chasm_options defaults() {
  chasm_options o;
  o.precision = CHASM_FP32_MIXED;
  o.n_nb = 20;
  o.patches[0] = o.patches[1] = o.patches[2] = 1;
  o.use_graphs = 1;
  o.cuda_stream = nullptr;
  o.theta_form = CHASM_THETA_AUTO;
  o.integrator = CHASM_STRANG;
  return o;
}

// ---- PMBC plan (host, FP64) ----

// Rows nu of the inverse of the natural-BC matrix A-tilde (order N+3, unknowns eta_{-1..N+1},
// Eqs. 2.11, 2.13): solves A-tilde^T y = e_nu by Gaussian elimination with partial pivoting.
std::vector<std::vector<double>> natural_inverse_rows(int n, double h, const std::vector<int>& rows) {
  const int N = n - 1, S = N + 3;
  std::vector<double> A((size_t)S * S, 0.0);   // A-tilde, row-major
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * S + j]; };
  a(0, 0) = 1.0 / (h * h);
  a(0, 1) = -2.0 / (h * h);
  a(0, 2) = 1.0 / (h * h);
  for (int i = 0; i <= N; ++i) {
    a(i + 1, i) = 1.0 / 6.0;
    a(i + 1, i + 1) = 2.0 / 3.0;
    a(i + 1, i + 2) = 1.0 / 6.0;
  }
  a(N + 2, N) = 1.0 / (h * h);
  a(N + 2, N + 1) = -2.0 / (h * h);
  a(N + 2, N + 2) = 1.0 / (h * h);
  // M = A^T with several right-hand sides
  const int R = (int)rows.size();
  std::vector<double> M((size_t)S * (S + R), 0.0);
  const int W = S + R;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) M[(size_t)i * W + j] = a(j, i);
  for (int r = 0; r < R; ++r) M[(size_t)(rows[r] + 1) * W + S + r] = 1.0;
  for (int c = 0; c < S; ++c) {
    int piv = c;
    for (int i = c + 1; i < S; ++i)
      if (std::fabs(M[(size_t)i * W + c]) > std::fabs(M[(size_t)piv * W + c])) piv = i;
    if (piv != c)
      for (int j = 0; j < W; ++j) std::swap(M[(size_t)c * W + j], M[(size_t)piv * W + j]);
    const double d = M[(size_t)c * W + c];
    for (int i = 0; i < S; ++i) {
      if (i == c) continue;
      const double f = M[(size_t)i * W + c] / d;
      if (f == 0.0) continue;
      for (int j = c; j < W; ++j) M[(size_t)i * W + j] -= f * M[(size_t)c * W + j];
    }
  }
  std::vector<std::vector<double>> out(R, std::vector<double>(S));
  for (int r = 0; r < R; ++r)
    for (int i = 0; i < S; ++i) out[r][i] = M[(size_t)i * W + S + r] / M[(size_t)i * W + i];
  return out;
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

int upload(Handle* H, void** dst, const void* src, size_t bytes) {
  if (!*dst) CHASM_CUDA(H, cudaMallocAsync(dst, bytes, H->stream));
  CHASM_CUDA(H, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, H->stream));
  return CHASM_OK;
}

template <typename T>
int upload_typed(Handle* H, void** dst, const std::vector<double>& v) {
  std::vector<T> t = cast_vec<T>(v);
  int rc = upload(H, dst, t.data(), t.size() * sizeof(T));
  if (rc != CHASM_OK) return rc;
  // the host vector dies at return: make the copy complete first
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  return CHASM_OK;
}

int upload_real(Handle* H, void** dst, const std::vector<double>& v) {
  return H->fp64 ? upload_typed<double>(H, dst, v) : upload_typed<float>(H, dst, v);
}

int build_spline_plan(Handle* H) {
  for (int d = 0; d < 3; ++d) {
    const int n = H->g.nx[d], N = n - 1;
    const double h = H->g.h[d];
    // c+_{j,0} = (-bt_{-1,j} + bt_{1,j})/2h,  c-_{j,p} = (-bt_{N-1,N-j} + bt_{N+1,N-j})/2h (Eq. 3.5)
    auto rows = natural_inverse_rows(n, h, {-1, 1, N - 1, N + 1});
    const int J = std::min(H->opt.n_nb, N) + 1;
    std::vector<double> cp(J), cm(J);
    for (int j = 0; j < J; ++j) {
      cp[j] = (-rows[0][j + 1] + rows[1][j + 1]) / (2.0 * h);
      cm[j] = (-rows[2][N - j + 1] + rows[3][N - j + 1]) / (2.0 * h);
    }
    H->J[d] = J;
    H->h_clos[d].assign(2 * (size_t)n, 0.0);
    for (int j = 0; j < J; ++j) {
      H->h_clos[d][j] = cp[j];
      H->h_clos[d][n + j] = cm[j];
    }
    int rc;
    if (H->fp64) {
      std::vector<double> c(2 * (size_t)n, 0.0);
      for (int j = 0; j < J; ++j) {
        c[j] = cp[j];
        c[n + j] = cm[j];
      }
      rc = upload(H, &H->d_clos[d], c.data(), c.size() * sizeof(double));
    } else {
      // unevaluated float pairs hi + lo of the FP64 coefficients
      std::vector<float> c(4 * (size_t)n, 0.0f);
      for (int j = 0; j < J; ++j) {
        c[j] = (float)cp[j];
        c[n + j] = (float)(cp[j] - (double)c[j]);
        c[2 * n + j] = (float)cm[j];
        c[3 * n + j] = (float)(cm[j] - (double)c[2 * n + j]);
      }
      rc = upload(H, &H->d_clos[d], c.data(), c.size() * sizeof(float));
      if (rc) return rc;
      CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
    }
    if (rc) return rc;
    CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
    // Thomas factors of the reduced Hermite system (rows: [2 1], [1 4 1] ..., [1 2])
    std::vector<double> lu(2 * n);
    double cprev = 0.0;
    for (int i = 0; i <= N; ++i) {
      const double b = (i == 0 || i == N) ? 2.0 : 4.0;
      const double aa = (i == 0) ? 0.0 : 1.0;
      const double c = (i == N) ? 0.0 : 1.0;
      const double mlt = 1.0 / (b - aa * cprev);
      lu[i] = c * mlt;        // c'_i
      lu[n + i] = mlt;        // 1 / pivot
      cprev = lu[i];
    }
    rc = upload_real(H, &H->d_lu[d], lu);
    if (rc) return rc;
    H->h_lu[d] = lu;
    const int P = H->opt.patches[d];
    if (P > 1) {   // closure windows of the p + 1 patch boundaries and the patch LU factors
      const int M = N / P, nb = H->opt.n_nb, W = 2 * nb + 1;
      std::vector<int> need;
      for (int b = 1; b < P; ++b) {
        need.push_back(b * M - 1);
        need.push_back(b * M + 1);
      }
      auto r2 = natural_inverse_rows(n, h, need);
      std::vector<double> win((size_t)(P + 1) * W, 0.0);
      for (int j = 0; j < J; ++j) {
        win[nb + j] = cp[j];                        // b = 0: node j
        win[(size_t)P * W + nb - j] = cm[j];        // b = p: node N - j
      }
      for (int b = 1; b < P; ++b)
        for (int i = 0; i < W; ++i) {
          const int node = b * M - nb + i;
          if (node < 0 || node > N) continue;
          win[(size_t)b * W + i] = (-r2[2 * (b - 1)][node + 1] + r2[2 * (b - 1) + 1][node + 1]) / (2.0 * h);
        }
      if (H->fp64) {
        rc = upload_real(H, &H->d_pclos[d], win);
      } else {
        std::vector<double> hl((size_t)(P + 1) * 2 * W);
        for (int b = 0; b <= P; ++b)
          for (int i = 0; i < W; ++i) {
            const double v = win[(size_t)b * W + i];
            const float hi = (float)v;
            hl[((size_t)b * 2) * W + i] = hi;
            hl[((size_t)b * 2 + 1) * W + i] = (float)(v - (double)hi);
          }
        rc = upload_real(H, &H->d_pclos[d], hl);
      }
      if (rc) return rc;
      std::vector<double> plu(2 * (size_t)(M + 1));
      double cprev = 0.0;
      for (int i = 0; i <= M; ++i) {
        const double bb = (i == 0 || i == M) ? 2.0 : 4.0;
        const double aa = (i == 0) ? 0.0 : 1.0;
        const double c = (i == M) ? 0.0 : 1.0;
        const double mlt = 1.0 / (bb - aa * cprev);
        plu[i] = c * mlt;
        plu[M + 1 + i] = mlt;
        cprev = plu[i];
      }
      rc = upload_real(H, &H->d_plu[d], plu);
      if (rc) return rc;
    }
  }
  return CHASM_OK;
}

// Advection weights for A(tau): alpha = hbar k tau / (m h_d), n = floor(alpha), a = alpha - n,
// (b4, b3, b2, b1)(a) of Eq. 3.7 (reading for any sign and size of alpha: shift by n nodes).
// Rounds n weights whose exact sum is 1 to FP32 and then resets the one of smallest magnitude
// to 1 minus the (exact) sum of the others, so the stored weights still form a partition of
// unity.  Otherwise the rounding of the same weights, applied at every pass, shifts the mass by
// up to a few 1e-8 per pass in one direction (for alpha = 0: fl(1/6) + fl(2/3) + fl(1/6) =
// 1 + 3e-8).
static void round_unit_sum(const double* w, float* out, int n) {
  int jmin = 0;
  for (int i = 0; i < n; ++i) {
    out[i] = (float)w[i];
    if (std::fabs(out[i]) < std::fabs(out[jmin])) jmin = i;
  }
  double rest = 0.0;
  for (int i = 0; i < n; ++i)
    if (i != jmin) rest += (double)out[i];
  out[jmin] = (float)(1.0 - rest);
}

int ensure_advect_tables(Handle* H, double tau) {
  if (H->adv.valid && H->adv.tau == tau) return CHASM_OK;
  const int nk = H->g.nk;
  std::vector<double> w((size_t)3 * nk * 4);
  std::vector<int> ns((size_t)3 * nk);
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < nk; ++j) {
      const double k = (j - nk / 2) * H->g.dk;
      const double alpha = H->hbar * k * tau / (H->m * H->g.h[d]);
      const double fl = std::floor(alpha);
      const double a = alpha - fl, b = 1.0 - a;
      double* ww = &w[((size_t)d * nk + j) * 4];
      ww[0] = a * a * a / 6.0;                                         // b4
      ww[1] = -a * a * a / 2.0 + a * a / 2.0 + a / 2.0 + 1.0 / 6.0;    // b3
      ww[2] = -b * b * b / 2.0 + b * b / 2.0 + b / 2.0 + 1.0 / 6.0;    // b2
      ww[3] = b * b * b / 6.0;                                         // b1
      if (std::fabs(fl) > 1e6) return fail(H, CHASM_EINVAL, "advection shift too large");
      ns[(size_t)d * nk + j] = (int)fl;
    }
  for (int d = 0; d < 3; ++d) {
    H->adv.ns_min[d] = *std::min_element(ns.begin() + (size_t)d * nk, ns.begin() + (size_t)(d + 1) * nk);
    H->adv.ns_max[d] = *std::max_element(ns.begin() + (size_t)d * nk, ns.begin() + (size_t)(d + 1) * nk);
  }
  const size_t wbytes = w.size() * H->elt;
  std::vector<unsigned char> blob(wbytes + ns.size() * sizeof(int));
  if (H->fp64)
    std::memcpy(blob.data(), w.data(), wbytes);
  else {
    std::vector<float> wf(w.size());
    for (size_t q = 0; q < w.size(); q += 4) round_unit_sum(&w[q], &wf[q], 4);
    std::memcpy(blob.data(), wf.data(), wbytes);
  }
  std::memcpy(blob.data() + wbytes, ns.data(), ns.size() * sizeof(int));
  int rc = upload(H, &H->adv.dev, blob.data(), blob.size());
  if (rc) return rc;
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  H->adv.tau = tau;
  H->adv.valid = true;
  return CHASM_OK;
}

// Circulant first columns of the periodic spectral k-shift by s = dt kappa (x_d - c_d)/hbar:
// c[q] = (1/N) sum_{m=-N/2}^{N/2-1} phi_m e^{2 pi i m q / N}, phi_m = e^{i pi m s / L}, and
// phi_{-N/2} = cos(pi N s / (2L)) (Nyquist mode kept real).
int ensure_kshift_rows(Handle* H, double dt) {
  if (H->krows_valid && H->krows_dt == dt) return CHASM_OK;
  const int N = H->g.nk;
  const int tot = H->g.nx[0] + H->g.nx[1] + H->g.nx[2];
  std::vector<double> rows((size_t)tot * N);
  int id = 0;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < H->g.nx[d]; ++i, ++id) {
      const double x = H->g.x_lo[d] + i * H->g.h[d];
      const double s = dt * H->kappa * (x - H->center[d]) / H->hbar;
      for (int q = 0; q < N; ++q) {
        double acc = 0.0;
        for (int mm = -N / 2; mm < N / 2; ++mm) {
          const double xi = M_PI * mm / H->g.lk;
          const double ang = 2.0 * M_PI * mm * q / N;
          if (mm == -N / 2)
            acc += std::cos(xi * s) * std::cos(ang);
          else
            acc += std::cos(xi * s + ang);
        }
        rows[(size_t)id * N + q] = acc / N;
      }
    }
  int rc;
  if (H->fp64) {
    rc = upload_real(H, &H->d_krows, rows);
  } else {   // the columns of the circulant sum to 1: keep that in FP32 (mass of the k-shift)
    std::vector<float> rf(rows.size());
    for (int r = 0; r < tot; ++r) round_unit_sum(&rows[(size_t)r * N], &rf[(size_t)r * N], N);
    rc = upload(H, &H->d_krows, rf.data(), rf.size() * sizeof(float));
    if (rc == CHASM_OK && cudaStreamSynchronize(H->stream) != cudaSuccess)
      rc = fail(H, CHASM_ECUDA, "k-shift table upload");
  }
  if (rc) return rc;
  H->krows_dt = dt;
  H->krows_valid = true;
  return CHASM_OK;
}

// Modulation tables per nucleus (storage-type complex): E1[nx1][N], E2[nx2][N],
// E3[nx3][4][N] = (conj E3, conj E3 tw1, E3, E3 conj tw1), E_d[i][n] = e^{i theta_d k_n},
// theta_d = 2 (x_{d,i} - x_{A,d}), tw1[n] = e^{-i pi n / N}.
int build_phase_tables(Handle* H) {
  const int N = H->g.nk;
  const int* nx = H->g.nx;
  const size_t per = (size_t)(nx[0] + nx[1] + 4 * nx[2]) * N;
  std::vector<double> re(per * H->nuclei.size()), im(per * H->nuclei.size());
  for (size_t a = 0; a < H->nuclei.size(); ++a) {
    size_t o = a * per;
    for (int d = 0; d < 2; ++d)
      for (int i = 0; i < nx[d]; ++i) {
        const double th = 2.0 * (H->g.x_lo[d] + i * H->g.h[d] - H->nuclei[a].pos[d]);
        for (int n = 0; n < N; ++n, ++o) {
          const double ang = th * (n - N / 2) * H->g.dk;
          re[o] = std::cos(ang);
          im[o] = std::sin(ang);
        }
      }
    for (int i = 0; i < nx[2]; ++i, o += 4 * (size_t)N) {
      const double th = 2.0 * (H->g.x_lo[2] + i * H->g.h[2] - H->nuclei[a].pos[2]);
      for (int n = 0; n < N; ++n) {
        const double ang = th * (n - N / 2) * H->g.dk;
        const double c = std::cos(ang), s = std::sin(ang);
        const double tc = std::cos(M_PI * n / N), ts = -std::sin(M_PI * n / N);  // tw1
        re[o + n] = c;                          // conj E3
        im[o + n] = -s;
        re[o + N + n] = c * tc + s * ts;        // conj E3 * tw1 = (c - i s)(tc + i ts)
        im[o + N + n] = c * ts - s * tc;
        re[o + 2 * N + n] = c;                  // E3
        im[o + 2 * N + n] = s;
        re[o + 3 * N + n] = c * tc + s * ts;    // E3 * conj tw1 = (c + i s)(tc - i ts)
        im[o + 3 * N + n] = s * tc - c * ts;
      }
    }
  }
  const size_t n = re.size();
  if (H->fp64) {
    std::vector<double> v(2 * n);
    for (size_t i = 0; i < n; ++i) {
      v[2 * i] = re[i];
      v[2 * i + 1] = im[i];
    }
    int rc = upload(H, &H->d_phase, v.data(), v.size() * sizeof(double));
    if (rc) return rc;
    CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  } else {
    std::vector<float> v(2 * n);
    for (size_t i = 0; i < n; ++i) {
      v[2 * i] = (float)re[i];
      v[2 * i + 1] = (float)im[i];
    }
    int rc = upload(H, &H->d_phase, v.data(), v.size() * sizeof(float));
    if (rc) return rc;
    CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  }
  return CHASM_OK;
}

int build_potential_table(Handle* H) {
  const int* nx = H->g.nx;
  std::vector<double> v((size_t)H->g.nxp);
  size_t idx = 0;
  for (int i1 = 0; i1 < nx[0]; ++i1)
    for (int i2 = 0; i2 < nx[1]; ++i2)
      for (int i3 = 0; i3 < nx[2]; ++i3, ++idx) {
        const double x[3] = {H->g.x_lo[0] + i1 * H->g.h[0], H->g.x_lo[1] + i2 * H->g.h[1],
                             H->g.x_lo[2] + i3 * H->g.h[2]};
        double V = 0.0;
        if (!H->nuclei.empty()) {
          for (const auto& nu : H->nuclei) {
            const double r = std::sqrt((x[0] - nu.pos[0]) * (x[0] - nu.pos[0]) +
                                       (x[1] - nu.pos[1]) * (x[1] - nu.pos[1]) +
                                       (x[2] - nu.pos[2]) * (x[2] - nu.pos[2]));
            V -= nu.charge / r;
          }
        } else {
          for (int d = 0; d < 3; ++d) V += 0.5 * H->kappa * (x[d] - H->center[d]) * (x[d] - H->center[d]);
        }
        v[idx] = V;
      }
  int rc = upload(H, (void**)&H->d_vx, v.data(), v.size() * sizeof(double));
  if (rc) return rc;
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  return CHASM_OK;
}

void drop_graphs(Handle* H);

void free_all(Handle* H) {
  if (H->stream) cudaStreamSynchronize(H->stream);
  drop_graphs(H);
  void* ptrs[] = {H->d_clos[0], H->d_clos[1], H->d_clos[2], H->d_lu[0], H->d_lu[1], H->d_lu[2],
                  H->d_pclos[0], H->d_pclos[1], H->d_pclos[2], H->d_plu[0], H->d_plu[1], H->d_plu[2],
                  H->adv.dev, H->d_T,
                  H->d_that, H->d_phase, H->d_sig, H->d_tkm, H->d_scratch, H->d_u[0], H->d_u[1], H->d_krows,
                  H->d_partials, H->d_result, H->d_vx, H->d_diag, H->d_fhost};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, H->stream);
  if (H->stream) cudaStreamSynchronize(H->stream);
  if (H->own_stream && H->stream) cudaStreamDestroy(H->stream);
  H->stream = nullptr;
}

double coulomb_rho(const Handle* H) {
  double zs = 0.0;
  for (const auto& n : H->nuclei) zs += std::fabs(n.charge);
  return 2.0 * zs / (M_PI * M_PI * H->hbar) * H->that_absmax;
}

// ---- the substeps ----

int do_advect(Handle* H, void* f, double tau, bool tables_ready) {
  if (!tables_ready) {
    int rc = ensure_advect_tables(H, tau);
    if (rc) return rc;
  }
  for (int d = 0; d < 3; ++d) CHASM_LAUNCH(H, launch_advect_dim(*H, f, d, H->stream));
  return CHASM_OK;
}

int do_pflow(Handle* H, void* f, double dt) {
  if (H->nuclei.empty()) {
    if (H->kappa == 0.0) return CHASM_OK;
    for (int d = 0; d < 3; ++d) CHASM_LAUNCH(H, launch_kshift(*H, f, d, H->d_krows, H->stream));
    return CHASM_OK;
  }
  if (H->xs) {   // the four stages per x point in one launch, in place on f
    const double c[4] = {dt / 4, dt / 3, dt / 2, dt};
    CHASM_LAUNCH(H, launch_theta_xs(*H, f, f, f, 4, c, H->stream));
    return CHASM_OK;
  }
  // u <- f + (dt/s) Theta[u], s = 4, 3, 2, 1, u_0 = f; buffers f -> u0 -> u1 -> u0 -> f
  const void* in[4] = {f, H->d_u[0], H->d_u[1], H->d_u[0]};
  void* out[4] = {H->d_u[0], H->d_u[1], H->d_u[0], f};
  for (int st = 0; st < 4; ++st) {
    const double c = dt / (4 - st);
    double coef[kMaxNuclei];
    for (size_t a = 0; a < H->nuclei.size(); ++a)
      coef[a] = -(2.0 * H->nuclei[a].charge / (M_PI * M_PI * H->hbar)) * c;
    CHASM_LAUNCH(H, launch_theta(*H, in[st], f, out[st], coef, H->stream));
  }
  return CHASM_OK;
}

// Spectral-radius bound of Theta for the quadratic potential: the rate kappa |x_d - c_d| / hbar
// times the largest kept k-frequency pi (N/2 - 1) / L_k, summed over d.
double harmonic_rho(const Handle* H) {
  double r = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double lo = H->g.x_lo[d], hi = lo + (H->g.nx[d] - 1) * H->g.h[d];
    r += std::max(std::fabs(lo - H->center[d]), std::fabs(hi - H->center[d]));
  }
  return std::fabs(H->kappa) / H->hbar * r * M_PI * (H->g.nk / 2 - 1) / H->g.lk;
}

// out = (base or 0) + c Theta_V[in] for either potential and either Coulomb form; in != out
int theta_any(Handle* H, const void* in, const void* base, void* out, double c) {
  if (H->nuclei.empty()) {
    CHASM_LAUNCH(H, launch_theta_harm(*H, in, base, out, c, H->stream));
  } else if (H->xs) {
    CHASM_LAUNCH(H, launch_theta_xs(*H, in, base, out, 1, &c, H->stream));
  } else {
    double coef[kMaxNuclei];
    for (size_t a = 0; a < H->nuclei.size(); ++a)
      coef[a] = -(2.0 * H->nuclei[a].charge / (M_PI * M_PI * H->hbar)) * c;
    CHASM_LAUNCH(H, launch_theta(*H, in, base, out, coef, H->stream));
  }
  return CHASM_OK;
}

// One LPC1 step (Sec. 2.2): U = Theta f; advect f (= g) and U (= h) by dt; then
// f = (g + dt/2 h) + dt/2 Theta[g + dt h].  The table form forms the predictor g + dt h and the
// corrector base in the Theta kernel itself; the other forms go through V = g + dt h.
int issue_step_lpc1(Handle* H, void* f, double dt) {
  void* U = H->d_u[0];
  void* V = H->d_u[1];
  int rc = theta_any(H, f, nullptr, U, 1.0);
  if (rc) return rc;
  rc = do_advect(H, f, dt, true);
  if (rc) return rc;
  rc = do_advect(H, U, dt, true);
  if (rc) return rc;
  if (!H->nuclei.empty() && H->xs) {
    XsExtra x;
    x.in2 = U;
    x.cin2 = dt;
    x.base2 = U;
    x.cbase2 = 0.5 * dt;
    const double c = 0.5 * dt;
    CHASM_LAUNCH(H, launch_theta_xs(*H, f, f, f, 1, &c, H->stream, x));
    return CHASM_OK;
  }
  CHASM_LAUNCH(H, launch_lpc1_combine(*H, f, U, V, dt, H->stream));
  return theta_any(H, V, f, f, 0.5 * dt);
}

int prepare_step(Handle* H, double dt) {
  if (!is_finite(dt) || !(dt > 0)) return fail(H, CHASM_EINVAL, "dt must be > 0 and finite");
  if (H->opt.integrator == CHASM_LPC1) {
    const double rho = H->nuclei.empty() ? harmonic_rho(H) : coulomb_rho(H);
    if (dt * rho > 1.0)
      return fail(H, CHASM_EUNSTABLE, "dt * rho(Theta) = " + std::to_string(dt * rho) +
                                          " exceeds the LPC1 limit 1");
    return ensure_advect_tables(H, dt);
  }
  if (!H->nuclei.empty() && dt * coulomb_rho(H) > 2.8)
    return fail(H, CHASM_EUNSTABLE,
                "dt * rho(Theta^T) = " + std::to_string(dt * coulomb_rho(H)) +
                    " exceeds the Taylor-4 stability limit 2.8");
  int rc = ensure_advect_tables(H, 0.5 * dt);
  if (rc) return rc;
  if (H->nuclei.empty() && H->kappa != 0.0) {
    rc = ensure_kshift_rows(H, dt);
    if (rc) return rc;
  }
  return CHASM_OK;
}

int issue_step(Handle* H, void* f, double dt) {
  if (H->opt.integrator == CHASM_LPC1) return issue_step_lpc1(H, f, dt);
  int rc = do_advect(H, f, 0.5 * dt, true);
  if (rc) return rc;
  rc = do_pflow(H, f, dt);
  if (rc) return rc;
  return do_advect(H, f, 0.5 * dt, true);
}

void drop_graphs(Handle* H) {
  if (H->graph) cudaGraphExecDestroy(H->graph);
  H->graph = nullptr;
}

// Captures what issue() issues on the handle's stream into an executable graph; the kernels it
// holds are counted in *nodes (and not in H->launches, which counts replays).
template <class F>
int capture(Handle* H, cudaGraphExec_t* out, int64_t* nodes, F&& issue) {
  cudaGraph_t gr = nullptr;
  const int64_t before = H->launches;
  CHASM_CUDA(H, cudaStreamBeginCapture(H->stream, cudaStreamCaptureModeThreadLocal));
  int rc = issue();
  cudaError_t e = cudaStreamEndCapture(H->stream, &gr);
  *nodes = H->launches - before;
  H->launches = before;
  if (rc) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(H, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(H, e, "cudaGraphInstantiate");
  return CHASM_OK;
}

}  // namespace

void set_thread_error(const std::string& e) { g_thread_err = e; }

std::string validate_problem(const chasm_grid* grid, const chasm_box* box, const chasm_potential* pot,
                             double hbar, double m) {
  return validate(grid, box, pot, hbar, m, nullptr);
}

}  // namespace chasm

using namespace chasm;

extern "C" {

int chasm_options_default(chasm_options* opt) {
  if (!opt) return fail(nullptr, CHASM_EINVAL, "opt is NULL");
  *opt = defaults();
  return CHASM_OK;
}

const char* chasm_last_error(const chasm_handle* h) {
  const Handle* H = reinterpret_cast<const Handle*>(h);
  return H ? H->err.c_str() : g_thread_err.c_str();
}

size_t chasm_workspace_bytes(const chasm_grid* grid, const chasm_potential* pot,
                             const chasm_options* opt) {
  chasm_options o = opt ? *opt : defaults();
  if (!validate(grid, nullptr, pot, 1.0, 1.0, &o).empty()) return 0;
  const int nk = grid->nk[0];
  const bool fp64 = o.precision == CHASM_FP64;
  const size_t e = fp64 ? 8 : 4;
  const int64_t nxp = (int64_t)grid->nx[0] * grid->nx[1] * grid->nx[2];
  const size_t fbytes = (size_t)nxp * nk * nk * nk * e;
  size_t w = 0;
  const bool coulomb = pot && pot->n_nuc > 0;
  if (coulomb) {
    const bool xs = table_form(nk, nxp, e, o);
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    ThetaPlan tp;
    if (xs) {
      w += xs_table_bytes(nk, nxp, e);
      theta_xs_plan(nk, fp64, nxp, sms, &tp);
    } else {
      w += 2 * fbytes;
      theta_plan(nk, fp64, nxp, sms, &tp);
      w += (size_t)pot->n_nuc * (grid->nx[0] + grid->nx[1] + 4 * grid->nx[2]) * nk * 2 * e;
    }
    w += tp.scratch_bytes;
    w += (size_t)8 * nk * nk * nk * e + (size_t)(2 * nk - 1) * (2 * nk - 1) * (2 * nk - 1) * 8;
    if (xs && o.integrator == CHASM_LPC1) w += fbytes;   // Theta f (the predictor is formed in-kernel)
  } else if (o.integrator == CHASM_LPC1) {
    w += 2 * fbytes;
  }
  w += (size_t)nxp * 8 + 3 * (size_t)moments_blocks() * 8 + 64;
  w += diag_bytes(grid->nx, nk);
  w += (size_t)3 * (grid->nx[0] + grid->nx[1] + grid->nx[2]) * (8 + 2 * e);
  w += (size_t)(grid->nx[0] + grid->nx[1] + grid->nx[2]) * nk * e + 3 * nk * (4 * e + 4);
  return w;
}

int chasm_create(const chasm_grid* grid, const chasm_box* box, const chasm_potential* pot,
                 double hbar, double m, const chasm_options* opt, chasm_handle** out) {
  if (!out) return fail(nullptr, CHASM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!box) return fail(nullptr, CHASM_EINVAL, "box is NULL");
  if (!pot) return fail(nullptr, CHASM_EINVAL, "potential is NULL");
  chasm_options o = opt ? *opt : defaults();
  const std::string v = validate(grid, box, pot, hbar, m, &o);
  if (!v.empty()) return fail(nullptr, CHASM_EINVAL, v);

  Handle* H = new (std::nothrow) Handle();
  if (!H) return fail(nullptr, CHASM_ENOMEM, "host allocation failed");
  H->grid = *grid;
  H->box = *box;
  H->hbar = hbar;
  H->m = m;
  H->opt = o;
  for (int a = 0; a < pot->n_nuc; ++a) H->nuclei.push_back(pot->nuc[a]);
  H->kappa = pot->harm_kappa;
  for (int d = 0; d < 3; ++d) H->center[d] = pot->harm_center[d];
  H->fp64 = o.precision == CHASM_FP64;
  H->elt = H->fp64 ? 8 : 4;
  GridDesc& g = H->g;
  for (int d = 0; d < 3; ++d) {
    g.nx[d] = grid->nx[d];
    g.x_lo[d] = box->x_lo[d];
    g.h[d] = (box->x_hi[d] - box->x_lo[d]) / (grid->nx[d] - 1);
  }
  g.nk = grid->nk[0];
  g.nxp = (int64_t)g.nx[0] * g.nx[1] * g.nx[2];
  g.kvol = (int64_t)g.nk * g.nk * g.nk;
  g.ncell = g.nxp * g.kvol;
  g.lk = box->k_half[0];
  g.dk = 2.0 * g.lk / g.nk;

  auto bail = [&](int rc) {
    std::string msg = H->err;
    free_all(H);
    delete H;
    return fail(nullptr, rc, msg);
  };
  cudaError_t e = cudaGetDevice(&H->device);
  if (e != cudaSuccess) {
    delete H;
    return fail(nullptr, CHASM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, H->device);
  if (o.cuda_stream) {
    H->stream = static_cast<cudaStream_t>(o.cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete H;
      return fail(nullptr, CHASM_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    H->own_stream = true;
  }
  for (int d = 0; d < 3; ++d)
    if (advect_smem_threads(advect_smem_elems(g.nx[d], o.patches[d]), H->elt) == 0) {
      std::string m = "nx[d] too large for the advection kernel's shared-memory line buffer";
      if (H->own_stream) cudaStreamDestroy(H->stream);
      delete H;
      return fail(nullptr, CHASM_EINVAL, m);
    }
  e = advect_prepare();
  if (e != cudaSuccess) return bail(cuda_fail(H, e, "advect_prepare"));
  int rc = build_spline_plan(H);
  if (rc) return bail(rc);
  rc = build_potential_table(H);
  if (rc) return bail(rc);
  if (cudaMallocAsync((void**)&H->d_partials, sizeof(double) * 3 * moments_blocks(), H->stream) != cudaSuccess ||
      cudaMallocAsync((void**)&H->d_result, sizeof(double) * 4, H->stream) != cudaSuccess ||
      cudaMallocAsync((void**)&H->d_diag, diag_bytes(g.nx, g.nk), H->stream) != cudaSuccess)
    return bail(fail(H, CHASM_ENOMEM, "device allocation failed (reductions)"));
  const size_t fbytes = (size_t)g.ncell * H->elt;
  if (!H->nuclei.empty()) {
    const int N = g.nk;
    const size_t tfull = (size_t)(2 * N - 1) * (2 * N - 1) * (2 * N - 1);
    if (cudaMallocAsync((void**)&H->d_T, tfull * sizeof(double), H->stream) != cudaSuccess ||
        cudaMallocAsync(&H->d_that, (size_t)8 * N * N * N * H->elt, H->stream) != cudaSuccess)
      return bail(fail(H, CHASM_ENOMEM, "device allocation failed (symbol)"));
    e = compute_symbol(N, g.lk, H->d_T, H->d_that, H->fp64, &H->that_absmax, H->stream);
    if (e != cudaSuccess) return bail(cuda_fail(H, e, "symbol precompute"));
    H->xs = table_form(N, g.nxp, H->elt, o);
    if (H->xs) {
      if (cudaMallocAsync(&H->d_sig, xs_table_bytes(N, g.nxp, H->elt), H->stream) != cudaSuccess)
        return bail(fail(H, CHASM_ENOMEM, "device allocation failed (per-x symbol table)"));
      e = build_xs_table(*H, H->d_sig, H->stream);
      if (e != cudaSuccess) return bail(cuda_fail(H, e, "per-x symbol table"));
      theta_xs_plan(N, H->fp64, g.nxp, H->num_sms, &H->theta);
      const size_t sb = H->theta.scratch_bytes;
      if (sb > 0 && cudaMallocAsync(&H->d_scratch, sb, H->stream) != cudaSuccess)
        return bail(fail(H, CHASM_ENOMEM, "device allocation failed (Theta scratch)"));
    } else {
      rc = build_phase_tables(H);
      if (rc) return bail(rc);
      theta_plan(N, H->fp64, g.nxp, H->num_sms, &H->theta);
      const size_t sb = H->theta.scratch_bytes;
      if ((sb > 0 && cudaMallocAsync(&H->d_scratch, sb, H->stream) != cudaSuccess) ||
          cudaMallocAsync(&H->d_u[0], fbytes, H->stream) != cudaSuccess ||
          cudaMallocAsync(&H->d_u[1], fbytes, H->stream) != cudaSuccess)
        return bail(fail(H, CHASM_ENOMEM, "device allocation failed (Horner buffers / scratch)"));
    }
  }
  if (o.integrator == CHASM_LPC1 && !H->d_u[0]) {   // LPC1 work copies: Theta f, the predictor
    const bool fused = !H->nuclei.empty() && H->xs;  // the table form forms the predictor in-kernel
    if (cudaMallocAsync(&H->d_u[0], fbytes, H->stream) != cudaSuccess ||
        (!fused && cudaMallocAsync(&H->d_u[1], fbytes, H->stream) != cudaSuccess))
      return bail(fail(H, CHASM_ENOMEM, "device allocation failed (LPC1 buffers)"));
  }
  e = cudaStreamSynchronize(H->stream);
  if (e != cudaSuccess) return bail(cuda_fail(H, e, "create"));
  H->workspace = chasm_workspace_bytes(grid, pot, &o);
  *out = reinterpret_cast<chasm_handle*>(H);
  return CHASM_OK;
}

int chasm_destroy(chasm_handle* h) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return CHASM_OK;
  free_all(H);
  delete H;
  return CHASM_OK;
}

int64_t chasm_num_cells(const chasm_handle* h) {
  const Handle* H = reinterpret_cast<const Handle*>(h);
  return H ? H->g.ncell : 0;
}

size_t chasm_f_bytes(const chasm_handle* h) {
  const Handle* H = reinterpret_cast<const Handle*>(h);
  return H ? (size_t)H->g.ncell * H->elt : 0;
}

int chasm_set_stream(chasm_handle* h, void* stream) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  drop_graphs(H);
  cudaStreamSynchronize(H->stream);
  if (H->own_stream) cudaStreamDestroy(H->stream);
  H->own_stream = false;
  H->stream = static_cast<cudaStream_t>(stream);
  return CHASM_OK;
}

int chasm_launch_count(const chasm_handle* h, int64_t* out) {
  const Handle* H = reinterpret_cast<const Handle*>(h);
  if (!H || !out) return fail(nullptr, CHASM_EINVAL, "handle or out is NULL");
  *out = H->launches;
  return CHASM_OK;
}

int chasm_sync(chasm_handle* h) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  CHASM_CUDA(H, cudaGetLastError());
  return CHASM_OK;
}

int chasm_step(chasm_handle* h, void* f, double dt, int32_t nsteps) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f) return fail(H, CHASM_EINVAL, "f is NULL");
  if ((reinterpret_cast<uintptr_t>(f) & 15) != 0) return fail(H, CHASM_EINVAL, "f must be 16-byte aligned");
  if (nsteps < 0) return fail(H, CHASM_EINVAL, "nsteps must be >= 0");
  int rc = prepare_step(H, dt);
  if (rc) return rc;
  if (nsteps == 0) return CHASM_OK;
  const bool graphs = H->opt.use_graphs && H->stream != nullptr;
  if (!graphs) {
    for (int i = 0; i < nsteps; ++i) {
      rc = issue_step(H, f, dt);
      if (rc) return rc;
    }
    return CHASM_OK;
  }
  if (!H->graph || H->graph_f != f || H->graph_dt != dt) {
    drop_graphs(H);
    rc = capture(H, &H->graph, &H->graph_nodes, [&] { return issue_step(H, f, dt); });
    if (rc) return rc;
    H->graph_f = f;
    H->graph_dt = dt;
  }
  for (int i = 0; i < nsteps; ++i) {
    CHASM_CUDA(H, cudaGraphLaunch(H->graph, H->stream));
    H->launches += H->graph_nodes;
  }
  return CHASM_OK;
}

int chasm_advect(chasm_handle* h, void* f, double tau) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f) return fail(H, CHASM_EINVAL, "f is NULL");
  if (!is_finite(tau)) return fail(H, CHASM_EINVAL, "tau must be finite");
  return do_advect(H, f, tau, false);
}

int chasm_pflow(chasm_handle* h, void* f, double dt) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f) return fail(H, CHASM_EINVAL, "f is NULL");
  if ((reinterpret_cast<uintptr_t>(f) & 15) != 0) return fail(H, CHASM_EINVAL, "f must be 16-byte aligned");
  if (!is_finite(dt) || !(dt > 0)) return fail(H, CHASM_EINVAL, "dt must be > 0 and finite");
  if (!H->nuclei.empty() && dt * coulomb_rho(H) > 2.8)
    return fail(H, CHASM_EUNSTABLE, "dt exceeds the Taylor-4 stability limit");
  if (H->nuclei.empty() && H->kappa != 0.0) {
    int rc = ensure_kshift_rows(H, dt);
    if (rc) return rc;
  }
  return do_pflow(H, f, dt);
}

int chasm_theta(chasm_handle* h, const void* u, void* out) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (H->nuclei.empty() && H->kappa == 0.0)
    return fail(H, CHASM_EINVAL, "chasm_theta needs a Coulomb or a quadratic potential (kappa != 0)");
  if (!u || !out) return fail(H, CHASM_EINVAL, "u/out is NULL");
  if (u == out) return fail(H, CHASM_EINVAL, "u and out must not alias");
  if (((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(out)) & 15) != 0)
    return fail(H, CHASM_EINVAL, "u/out must be 16-byte aligned");
  return theta_any(H, u, nullptr, out, 1.0);
}

int chasm_tkm_convolve(chasm_handle* h, const void* g, void* phi) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (H->nuclei.empty()) return fail(H, CHASM_EINVAL, "chasm_tkm_convolve needs a Coulomb handle");
  if (!H->xs) return fail(H, CHASM_EINVAL, "chasm_tkm_convolve needs the table form of Theta (theta_form)");
  if (!g || !phi) return fail(H, CHASM_EINVAL, "g/phi is NULL");
  if (g == phi) return fail(H, CHASM_EINVAL, "g and phi must not alias");
  if (((reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(phi)) & 15) != 0)
    return fail(H, CHASM_EINVAL, "g/phi must be 16-byte aligned");
  if (!H->d_tkm) {   // the spectrum of T, built once per handle on first use
    const int N = H->g.nk;
    const size_t bytes = (size_t)4 * N * N * N * H->elt;
    if (cudaMallocAsync(&H->d_tkm, bytes, H->stream) != cudaSuccess) {
      H->d_tkm = nullptr;
      return fail(H, CHASM_ENOMEM, "chasm_tkm_convolve: table allocation failed");
    }
    const cudaError_t e = build_tkm_table(*H, H->d_tkm, H->stream);
    if (e != cudaSuccess) return cuda_fail(H, e, "build_tkm_table");
  }
  XsExtra x;
  x.sig = H->d_tkm;
  x.real_symbol = true;
  const double one = 1.0;
  CHASM_CUDA(H, launch_theta_xs(*H, g, nullptr, phi, 1, &one, H->stream, x));
  return CHASM_OK;
}

int chasm_moments(chasm_handle* h, const void* f, double* mass, double* energy) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f) return fail(H, CHASM_EINVAL, "f is NULL");
  CHASM_CUDA(H, launch_moments(*H, f, H->d_partials, H->d_result, H->stream));
  double r[2];
  CHASM_CUDA(H, cudaMemcpyAsync(r, H->d_result, sizeof(r), cudaMemcpyDeviceToHost, H->stream));
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  if (mass) *mass = r[0];
  if (energy) *energy = r[1];
  return CHASM_OK;
}

namespace {
int diag_call(chasm_handle* h, const void* f, int what, int j, double* out, size_t n) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f || !out) return fail(H, CHASM_EINVAL, "f/out is NULL");
  double* res = H->d_diag + (size_t)3 * H->g.nxp * H->g.nk;
  CHASM_CUDA(H, launch_diag(*H, f, what, j, H->d_diag, res, H->stream));
  CHASM_CUDA(H, cudaMemcpyAsync(out, res, n * sizeof(double), cudaMemcpyDeviceToHost, H->stream));
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  return CHASM_OK;
}
}  // namespace

int chasm_reduced_wigner(chasm_handle* h, const void* f, int32_t j, double* w_host) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (H && (j < 0 || j > 2)) return fail(H, CHASM_EINVAL, "j must be 0, 1 or 2");
  return diag_call(h, f, 0, j, w_host, H ? (size_t)H->g.nx[j < 0 || j > 2 ? 0 : j] * H->g.nk : 0);
}

int chasm_marginal_x12(chasm_handle* h, const void* f, double* p_host) {
  Handle* H = reinterpret_cast<Handle*>(h);
  return diag_call(h, f, 1, 0, p_host, H ? (size_t)H->g.nx[0] * H->g.nx[1] : 0);
}

int chasm_expectations(chasm_handle* h, const void* f, double* out_host) {
  return diag_call(h, f, 2, 0, out_host, 6);
}

int chasm_fma_peaks(double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops && !fp64_tflops) return fail(nullptr, CHASM_EINVAL, "both outputs are NULL");
  const cudaError_t e = measure_fma_peaks(fp32_tflops, fp64_tflops);
  if (e != cudaSuccess)
    return fail(nullptr, CHASM_ECUDA, std::string("chasm_fma_peaks: ") + cudaGetErrorString(e));
  return CHASM_OK;
}

int chasm_fma_peak_f32x2(double* tflops) {
  if (!tflops) return fail(nullptr, CHASM_EINVAL, "output is NULL");
  const cudaError_t e = measure_fma_peak_f32x2(tflops);
  if (e != cudaSuccess)
    return fail(nullptr, CHASM_ECUDA, std::string("chasm_fma_peak_f32x2: ") + cudaGetErrorString(e));
  return CHASM_OK;
}

int chasm_fft_pk_rate(double* tflops) {
  if (!tflops) return fail(nullptr, CHASM_EINVAL, "output is NULL");
  const cudaError_t e = measure_fft_pk_rate(tflops);
  if (e != cudaSuccess)
    return fail(nullptr, CHASM_ECUDA, std::string("chasm_fft_pk_rate: ") + cudaGetErrorString(e));
  return CHASM_OK;
}

int chasm_mass(chasm_handle* h, const void* f, double* out) {
  if (!out) return fail(reinterpret_cast<Handle*>(h), CHASM_EINVAL, "out is NULL");
  return chasm_moments(h, f, out, nullptr);
}

int chasm_energy(chasm_handle* h, const void* f, double* out) {
  if (!out) return fail(reinterpret_cast<Handle*>(h), CHASM_EINVAL, "out is NULL");
  return chasm_moments(h, f, nullptr, out);
}

int chasm_init_gaussians(chasm_handle* h, void* f, const chasm_gaussian* g, int32_t n) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f || !g) return fail(H, CHASM_EINVAL, "f/g is NULL");
  if ((reinterpret_cast<uintptr_t>(f) & 15) != 0) return fail(H, CHASM_EINVAL, "f must be 16-byte aligned");
  if (n < 1 || n > 16) return fail(H, CHASM_EINVAL, "n must be in [1, 16]");
  for (int i = 0; i < n; ++i)
    if (!is_finite(g[i].w) || !is_finite(g[i].ax) || !is_finite(g[i].ak) || g[i].ax < 0 || g[i].ak < 0)
      return fail(H, CHASM_EINVAL, "gaussian: w finite, ax >= 0, ak >= 0 required");
  CHASM_CUDA(H, launch_init_gaussians(*H, f, g, n, H->stream));
  return CHASM_OK;
}

int chasm_init_hydrogen_1s(chasm_handle* h, void* f, int32_t n_y, const double center[3]) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f) return fail(H, CHASM_EINVAL, "f is NULL");
  if (n_y < 2 * H->g.nk || n_y % (2 * H->g.nk) != 0 || n_y > 256)
    return fail(H, CHASM_EINVAL, "n_y must be a multiple of 2 N_k and at most 256");
  std::string err;
  cudaError_t e = launch_init_1s(*H, f, n_y, center, H->stream, &err);
  if (e != cudaSuccess) return cuda_fail(H, e, err.empty() ? "init_hydrogen_1s" : err.c_str());
  return CHASM_OK;
}

int chasm_tkm_tensor(chasm_handle* h, double* t_host) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (H->nuclei.empty() || !H->d_T) return fail(H, CHASM_EINVAL, "no Coulomb symbol in this handle");
  if (!t_host) return fail(H, CHASM_EINVAL, "t_host is NULL");
  const int N = H->g.nk;
  const size_t n = (size_t)(2 * N - 1) * (2 * N - 1) * (2 * N - 1);
  CHASM_CUDA(H, cudaMemcpyAsync(t_host, H->d_T, n * sizeof(double), cudaMemcpyDeviceToHost, H->stream));
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  return CHASM_OK;
}

int chasm_run_host(chasm_handle* h, const void* f0, void* fout, double dt, int32_t nsteps,
                   double* mass_out) {
  Handle* H = reinterpret_cast<Handle*>(h);
  if (!H) return fail(nullptr, CHASM_EINVAL, "handle is NULL");
  if (!f0 || !fout) return fail(H, CHASM_EINVAL, "host buffers are NULL");
  const size_t fb = (size_t)H->g.ncell * H->elt;
  if (!H->d_fhost) CHASM_CUDA(H, cudaMallocAsync(&H->d_fhost, fb, H->stream));
  CHASM_CUDA(H, cudaMemcpyAsync(H->d_fhost, f0, fb, cudaMemcpyHostToDevice, H->stream));
  int rc = chasm_step(h, H->d_fhost, dt, nsteps);
  if (rc) return rc;
  double ms = 0.0;
  rc = chasm_moments(h, H->d_fhost, &ms, nullptr);
  if (rc) return rc;
  CHASM_CUDA(H, cudaMemcpyAsync(fout, H->d_fhost, fb, cudaMemcpyDeviceToHost, H->stream));
  CHASM_CUDA(H, cudaStreamSynchronize(H->stream));
  if (mass_out) *mass_out = ms;
  return CHASM_OK;
}

}  // extern "C"
