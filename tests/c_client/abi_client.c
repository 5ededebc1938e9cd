/* A plain C11 client of the FC library's C ABI (no C++, no CUDA headers): builds the
 * 5 MHz / 24 PRB symbol-synchronized geometry (N = 512, L = 384, 14 symbols with the
 * 40/36 CP schedule), asks the host-only validation for its sizes, and tries to create a
 * plan. Prints "sizes <grid_len> <wave_len> <nominal_len>", "status <code> <name>" per
 * call and exits 0; the test compares the numbers with the Python binding. */
#include <stdio.h>
#include <stdlib.h>

#include "fcofdm.h"

int main(void) {
  int32_t n_cp[14];
  for (int n = 0; n < 14; ++n) n_cp[n] = (n == 0 || n == 7) ? 40 : 36;
  double* weights = (double*)malloc(384 * sizeof(double));
  if (!weights) return 2;
  for (int p = 0; p < 384; ++p) weights[p] = 1.0;
  const fc_group group = {512, 256, -1, 14, n_cp};
  const fc_subband sub = {384, 384, 288, 0, 0, weights};
  const fc_geometry geo = {FC_SYMBOL_SYNC, FC_OLS, FC_OLS, 1, &group, 1, &sub, 0};

  fc_sizes sz;
  const int st = fc_geometry_check(&geo, &sz);
  printf("status %d %s\n", st, fc_status_string(st));
  if (st != FC_OK) return 1;
  printf("sizes %lld %lld %lld\n", (long long)sz.grid_len, (long long)sz.wave_len, (long long)sz.nominal_len);

  fc_plan* plan = NULL;
  const int pc = fc_plan_create(&plan, &geo, 0);
  printf("status %d %s\n", pc, fc_status_string(pc));
  if (pc == FC_OK) fc_plan_destroy(plan);
  else if (plan != NULL) return 3;                 /* on error *out must be NULL */
  free(weights);
  return 0;
}
