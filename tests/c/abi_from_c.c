/* A C program that uses the library through include/ba.h alone: it reads
 * the defaults and checks the argument errors that need no GPU.  Built and
 * run by tests/test_abi.py. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "ba.h"

static int fails = 0;
#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "%s:%d: %s\n", __FILE__, __LINE__, #cond); \
      ++fails;                                                   \
    }                                                            \
  } while (0)

int main(void) {
  ba_options o;
  memset(&o, 0, sizeof o);
  CHECK(ba_options_default(&o) == BA_OK);
  CHECK(o.precision == BA_PREC_F64 && o.up == 2.0 && o.down == 0.0625);
  CHECK(o.pcg_maxiter == 250 && o.pcg_tol == 1e-4 && o.lambda0 == 1e-4);
  CHECK(o.jacobian_mode == BA_JAC_AUTO);

  ba_problem* h = (ba_problem*)1;
  CHECK(ba_problem_create(&h, 0, 1, 1, NULL, NULL, NULL, NULL, NULL, &o, NULL) == BA_ERR_INVALID_ARG);
  CHECK(h == NULL);
  CHECK(strlen(ba_last_error()) > 0);
  CHECK(ba_lm_step(NULL, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_solve(NULL, 1, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_csr_build(NULL, -1, 3, NULL, NULL, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_csr_build_noalloc(NULL, BA_NOALLOC_MAX_KEYS + 1, 3, NULL, NULL, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_problem_destroy(NULL) == BA_OK);
  /* pose graphs: argument errors found before any device work */
  ba_pgo* g = (ba_pgo*)1;
  CHECK(ba_pgo_create(&g, 1, 1, NULL, NULL, NULL, NULL, NULL, NULL, &o, NULL) == BA_ERR_INVALID_ARG);
  CHECK(g == NULL);
  CHECK(ba_pgo_create(NULL, 4, 3, NULL, NULL, NULL, NULL, NULL, NULL, &o, NULL) == BA_ERR_INVALID_ARG);
  ba_options o32 = o;
  o32.precision = BA_PREC_F32;
  double pose[14] = {0, 0, 0, 0, 0, 0, 1, 1, 0, 0, 0, 0, 0, 1};
  int32_t ei = 0, ej = 1;
  double info[21] = {0};
  CHECK(ba_pgo_create(&g, 2, 1, pose, &ei, &ej, pose, info, NULL, &o32, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_pgo_solve(NULL, 1, NULL) == BA_ERR_INVALID_ARG);
  CHECK(ba_pgo_destroy(NULL) == BA_OK);
  CHECK(ba_state_size(NULL) == 0);
  printf("%s\n", fails ? "FAIL" : "OK");
  return fails ? 1 : 0;
}
