/* Solve one bundle-adjustment problem through include/ba.h with host
 * pointers only (no CUDA headers, no Python): read the problem from a file,
 * run the LM trials, print every trial's cost and trial cost, and the final
 * parameters.  Built and run by tests/test_gpu_c_abi.py, which compares the
 * output with the oracle.
 *
 * Input file: int32 C, P, O, iters, pcg_maxiter; double pcg_tol; then
 * double cams[C][9], double points[P][3], int32 cam_idx[O], int32 pt_idx[O],
 * double pixels[O][2] (native byte order). */
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
    fprintf(stderr, "usage: %s problem.bin\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t* hdr = (int32_t*)read_n(f, sizeof(int32_t), 5);
  const int C = hdr[0], P = hdr[1], O = hdr[2], iters = hdr[3];
  double* tol = (double*)read_n(f, sizeof(double), 1);
  double* cams = (double*)read_n(f, sizeof(double), 9 * (size_t)C);
  double* points = (double*)read_n(f, sizeof(double), 3 * (size_t)P);
  int32_t* cam_idx = (int32_t*)read_n(f, sizeof(int32_t), (size_t)O);
  int32_t* pt_idx = (int32_t*)read_n(f, sizeof(int32_t), (size_t)O);
  double* pixels = (double*)read_n(f, sizeof(double), 2 * (size_t)O);
  fclose(f);

  ba_options o;
  if (ba_options_default(&o) != BA_OK) return 3;
  o.precision = BA_PREC_F64;
  o.pcg_maxiter = hdr[4];
  o.pcg_tol = *tol;
  ba_problem* h = NULL;
  ba_status st = ba_problem_create(&h, C, P, O, cams, points, cam_idx, pt_idx, pixels, &o, NULL);
  if (st != BA_OK) {
    fprintf(stderr, "create: %d %s\n", (int)st, ba_last_error());
    return 4;
  }
  st = ba_solve(h, iters, NULL);
  ba_iter_stats* rec = (ba_iter_stats*)calloc((size_t)iters, sizeof(ba_iter_stats));
  int n = 0;
  if (st == BA_OK) st = ba_get_stats(h, rec, iters, &n);
  if (st == BA_OK) st = ba_get_params(h, cams, points, NULL);
  double cost = 0.0, lambda = 0.0;
  if (st == BA_OK) st = ba_get_scalars(h, &cost, &lambda); /* synchronises the stream */
  if (st != BA_OK) {
    fprintf(stderr, "solve: %d %s\n", (int)st, ba_last_error());
    return 5;
  }
  for (int t = 0; t < n; ++t)
    printf("trial %d %.17g %.17g %d %d\n", t, rec[t].cost, rec[t].cost_trial, rec[t].accepted, rec[t].pcg_iters);
  printf("final %.17g\n", cost);
  for (int i = 0; i < 9 * C; ++i) printf("cam %.17g\n", cams[i]);
  ba_problem_destroy(h);
  free(rec);
  free(pixels);
  free(pt_idx);
  free(cam_idx);
  free(points);
  free(cams);
  free(tol);
  free(hdr);
  return 0;
}
