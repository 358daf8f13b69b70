/* A C11 caller of the library with no Python or PyTorch: one Coulomb solve through the host-buffer
 * entry point.  f is a Gaussian packet near a nucleus, filled on the host in the documented layout
 * f[x1][x2][x3][k1][k2][k3] (k3 fastest, FP32-mixed form: float); chasm_run_host copies it in, runs
 * the steps, measures the mass and copies f back.  Prints "mass <m0> <m1>" and exits 0; a failed
 * call prints its status and chasm_last_error and exits 3 (argument errors are checked first, so
 * the program also exercises the error path on a machine without a GPU). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "chasm.h"

int main(void) {
  const int nx = 8, nk = 8;
  const double L = 3.0, lk = 3.0, dt = 0.02;
  chasm_grid g = {{nx, nx, nx}, {nk, nk, nk}};
  chasm_box box = {{-L, -L, -L}, {L, L, L}, {lk, lk, lk}};
  chasm_nucleus nuc = {{0.1, -0.2, 0.15}, 1.0};
  chasm_potential pot = {&nuc, 1, 0.0, {0.0, 0.0, 0.0}};
  chasm_options opt;
  chasm_handle* h = NULL;
  int rc;

  if (chasm_options_default(&opt) != CHASM_OK) return 3;
  /* an invalid grid must be rejected with EINVAL before any device work */
  chasm_grid bad = g;
  bad.nk[0] = bad.nk[1] = bad.nk[2] = 12;
  rc = chasm_create(&bad, &box, &pot, 1.0, 1.0, &opt, &h);
  if (rc != CHASM_EINVAL || h != NULL) {
    printf("expected EINVAL for N_k = 12, got %d\n", rc);
    return 4;
  }

  rc = chasm_create(&g, &box, &pot, 1.0, 1.0, &opt, &h);
  if (rc != CHASM_OK) {
    printf("chasm_create: %d %s\n", rc, chasm_last_error(NULL));
    return 3;
  }
  const size_t n = (size_t)chasm_num_cells(h);
  float* f = (float*)malloc(n * sizeof(float));
  float* out = (float*)malloc(n * sizeof(float));
  if (!f || !out) return 3;
  const double h_x = 2.0 * L / (nx - 1), dk = 2.0 * lk / nk;
  double m0 = 0.0;
  size_t i = 0;
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < nx; ++b)
      for (int c = 0; c < nx; ++c)
        for (int p = 0; p < nk; ++p)
          for (int q = 0; q < nk; ++q)
            for (int r = 0; r < nk; ++r, ++i) {
              const double x1 = -L + a * h_x - 0.5, x2 = -L + b * h_x, x3 = -L + c * h_x;
              const double k1 = (p - nk / 2) * dk, k2 = (q - nk / 2) * dk - 0.3, k3 = (r - nk / 2) * dk;
              f[i] = (float)(exp(-(x1 * x1 + x2 * x2 + x3 * x3) - (k1 * k1 + k2 * k2 + k3 * k3)) /
                             pow(M_PI, 3.0));
              m0 += f[i];
            }
  m0 *= h_x * h_x * h_x * dk * dk * dk;
  double m1 = 0.0;
  rc = chasm_run_host(h, f, out, dt, 2, &m1);
  if (rc != CHASM_OK) {
    printf("chasm_run_host: %d %s\n", rc, chasm_last_error(h));
    chasm_destroy(h);
    return 3;
  }
  printf("mass %.12e %.12e\n", m0, m1);
  chasm_destroy(h);
  free(f);
  free(out);
  return 0;
}
