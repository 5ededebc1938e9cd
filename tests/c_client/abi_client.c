/* A plain C11 client of the FC library's C ABI (no C++, no CUDA headers): builds the
 * 5 MHz / 24 PRB symbol-synchronized geometry (N = 512, L = 384, 14 symbols with the
 * 40/36 CP schedule), asks the host-only validation for its sizes, and tries to create a
 * plan. Prints "status <code> <name>" and "sizes <grid_len> <wave_len> <nominal_len>"
 * and exits 0; the test compares the numbers with the Python binding.
 *
 * With a directory argument and a plan created (a GPU machine), it then runs one TX and
 * one RX of 4 streams through the host-buffer calls (fc_pipeline_create,
 * fc_tx_synthesize_host, fc_rx_analyze_host; fc_pipeline_destroy waits for the work)
 * on a QPSK grid drawn from a 32-bit linear congruential generator, RX on the TX
 * output, and writes grid.bin, wave.bin and est.bin (complex64, interleaved) there for
 * the test to compare with the oracle. */
#include <stdio.h>
#include <stdlib.h>

#include "fcofdm.h"

#define N_STREAMS 4

static int write_file(const char* dir, const char* name, const float* data, size_t n_floats) {
  char path[1024];
  snprintf(path, sizeof path, "%s/%s", dir, name);
  FILE* f = fopen(path, "wb");
  if (!f) return 1;
  const size_t w = fwrite(data, sizeof(float), n_floats, f);
  fclose(f);
  return w == n_floats ? 0 : 1;
}

static int run_tx_rx(const fc_plan* plan, const fc_sizes* sz, const char* dir) {
  const size_t g_n = (size_t)N_STREAMS * (size_t)sz->grid_len;
  const size_t w_n = (size_t)N_STREAMS * (size_t)sz->wave_len;
  float* grid = (float*)malloc(2 * g_n * sizeof(float));
  float* wave = (float*)malloc(2 * w_n * sizeof(float));
  float* est = (float*)malloc(2 * g_n * sizeof(float));
  int rc = 10;
  if (!grid || !wave || !est) goto out;
  {
    unsigned int x = 12345u;
    const float a = 0.70710678f;
    for (size_t i = 0; i < 2 * g_n; ++i) {
      x = x * 1664525u + 1013904223u;
      grid[i] = (x >> 31) ? a : -a;
    }
  }
  fc_pipeline* pipe = NULL;
  int st = fc_pipeline_create(plan, 2, 2, &pipe);
  printf("status %d %s\n", st, fc_status_string(st));
  if (st != FC_OK) { rc = 11; goto out; }
  st = fc_tx_synthesize_host(pipe, N_STREAMS, grid, wave, NULL);
  printf("status %d %s\n", st, fc_status_string(st));
  fc_pipeline_destroy(pipe);                       /* waits for the pipeline's work */
  if (st != FC_OK) { rc = 12; goto out; }
  pipe = NULL;
  st = fc_pipeline_create(plan, 2, 2, &pipe);
  if (st != FC_OK) { rc = 13; goto out; }
  st = fc_rx_analyze_host(pipe, N_STREAMS, wave, est, NULL);
  printf("status %d %s\n", st, fc_status_string(st));
  fc_pipeline_destroy(pipe);
  if (st != FC_OK) { rc = 14; goto out; }
  rc = write_file(dir, "grid.bin", grid, 2 * g_n) | write_file(dir, "wave.bin", wave, 2 * w_n) |
       write_file(dir, "est.bin", est, 2 * g_n);
  if (rc) rc = 15;
out:
  free(grid);
  free(wave);
  free(est);
  return rc;
}

int main(int argc, char** argv) {
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
  int rc = 0;
  if (pc == FC_OK) {
    if (argc > 1) rc = run_tx_rx(plan, &sz, argv[1]);
    fc_plan_destroy(plan);
  } else if (plan != NULL) {
    rc = 3;                                        /* on error *out must be NULL */
  }
  free(weights);
  return rc;
}
