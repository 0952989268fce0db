/* Solve one pose graph (the paper's PGO problem, Sec. IV-D) through
 * include/ba.h with host pointers only (no CUDA headers, no Python): read
 * the graph from a file, run the LM trials, print every trial's cost and
 * trial cost, and the final poses.  Built and run by tests/test_gpu_pgo.py,
 * which compares the output with the oracle.
 *
 * Input file: int32 N, E, iters, solver, pcg_maxiter; double pcg_tol; then
 * double poses[N][7], int32 ei[E], int32 ej[E], double meas[E][7],
 * double info[E][21], uint8 fixed[N] (native byte order). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "ba.h"

static void* read_n(FILE* f, size_t size, size_t n) {
  void* p = malloc(size * (n ? n : 1));
  if (!p || fread(p, size, n, f) != n) {
    fprintf(stderr, "short read\n");
    exit(2);
  }
  return p;
}

int main(int argc, char** argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: %s graph.bin\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t* hdr = (int32_t*)read_n(f, sizeof(int32_t), 5);
  const int N = hdr[0], E = hdr[1], iters = hdr[2];
  double* tol = (double*)read_n(f, sizeof(double), 1);
  double* poses = (double*)read_n(f, sizeof(double), 7 * (size_t)N);
  int32_t* ei = (int32_t*)read_n(f, sizeof(int32_t), (size_t)E);
  int32_t* ej = (int32_t*)read_n(f, sizeof(int32_t), (size_t)E);
  double* meas = (double*)read_n(f, sizeof(double), 7 * (size_t)E);
  double* info = (double*)read_n(f, sizeof(double), 21 * (size_t)E);
  uint8_t* fixed = (uint8_t*)read_n(f, 1, (size_t)N);
  fclose(f);

  ba_options o;
  if (ba_options_default(&o) != BA_OK) return 3;
  o.solver = hdr[3];
  o.pcg_maxiter = hdr[4];
  o.pcg_tol = *tol;
  ba_pgo* h = NULL;
  ba_status st = ba_pgo_create(&h, N, E, poses, ei, ej, meas, info, fixed, &o, NULL);
  if (st != BA_OK) {
    fprintf(stderr, "create: %d %s\n", (int)st, ba_last_error());
    return 4;
  }
  st = ba_pgo_solve(h, iters, NULL);
  ba_iter_stats* rec = (ba_iter_stats*)calloc((size_t)iters, sizeof(ba_iter_stats));
  int n = 0;
  if (st == BA_OK) st = ba_pgo_get_stats(h, rec, iters, &n);
  if (st == BA_OK) st = ba_pgo_get_poses(h, poses, NULL);
  double cost = 0.0, lambda = 0.0;
  if (st == BA_OK) st = ba_pgo_get_scalars(h, &cost, &lambda);
  if (st != BA_OK) {
    fprintf(stderr, "solve: %d %s\n", (int)st, ba_last_error());
    return 5;
  }
  for (int t = 0; t < n; ++t)
    printf("trial %d %.17g %.17g %d %d\n", t, rec[t].cost, rec[t].cost_trial, rec[t].accepted, rec[t].pcg_iters);
  printf("final %.17g\n", cost);
  for (int i = 0; i < 7 * N; ++i) printf("pose %.17g\n", poses[i]);
  ba_pgo_destroy(h);
  free(rec);
  free(fixed);
  free(info);
  free(meas);
  free(ej);
  free(ei);
  free(poses);
  free(tol);
  free(hdr);
  return 0;
}
