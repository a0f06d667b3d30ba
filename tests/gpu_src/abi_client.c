/* A plain C client of librlb (include/rlb.h): no Python, no torch. It runs the paper's Sod tube and a
 * second tube in one handle through the C ABI, writes the fields after the run to a binary file, checks
 * a state round trip and the error reporting, and prints one line per check. Built and run by
 * tests/test_c_client_gpu.py, which compares its fields with those of the Python binding. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "rlb.h"

#define CHECK(call)                                                                  \
  do {                                                                               \
    rlb_status s_ = (call);                                                          \
    if (s_ != RLB_OK) {                                                              \
      fprintf(stderr, "%s failed: %s\n", #call, rlb_error_string(s_));               \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

int main(int argc, char **argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s nsteps out.bin\n", argv[0]);
    return 2;
  }
  const long nsteps = atol(argv[1]);
  rlb_tube t[2];
  memset(t, 0, sizeof t);
  /* the paper's Sod tube: Nx = 400, Qp = 3, Qxi = 8, Np = 2, Nv = 5, tau = 1e-3, CFL 0.5 */
  t[0].Qp = 3; t[0].Qxi = 8; t[0].Np = 2; t[0].Nv = 5; t[0].Nx = 400;
  t[0].dx = 1.0 / 400; t[0].tau = 1e-3; t[0].dt = rlb_suggest_dt(t[0].dx, t[0].tau, 0.5);
  t[0].bc = RLB_BC_OPEN; t[0].storage = RLB_STORAGE_F64;
  /* a ballistic tube with 32 polar nodes */
  t[1] = t[0];
  t[1].Qxi = 32; t[1].Nx = 257; t[1].dx = 1.0 / 257; t[1].tau = INFINITY;
  t[1].dt = rlb_suggest_dt(t[1].dx, t[1].tau, 0.5);
  const double states[12] = {1.0, 1.0, 0.0, 0.1, 0.125, 0.0, 1.0, 1.0, 0.0, 0.1, 0.125, 0.0};
  const double x_left[2] = {-0.5, -0.5};

  rlb_handle h = NULL;
  CHECK(rlb_init_riemann(&h, t, 2, states, x_left, NULL));
  const long long size = rlb_state_size(h), nx = 400 + 257;
  printf("state size %lld\n", size);

  /* a checkpoint after half the run, restored after the full run: the second half repeats exactly */
  double *ck = malloc(sizeof(double) * size), *fa = malloc(sizeof(double) * RLB_NFIELDS * nx),
         *fb = malloc(sizeof(double) * RLB_NFIELDS * nx);
  if (!ck || !fa || !fb) return 1;
  CHECK(rlb_step(h, nsteps / 2));
  CHECK(rlb_get_state(h, ck, 0));
  CHECK(rlb_step(h, nsteps - nsteps / 2));
  CHECK(rlb_moments(h, fa, 0));
  CHECK(rlb_set_state(h, ck, 0));
  CHECK(rlb_step(h, nsteps - nsteps / 2));
  CHECK(rlb_moments(h, fb, 0));
  printf("restart repeats the run: %s\n", memcmp(fa, fb, sizeof(double) * RLB_NFIELDS * nx) ? "no" : "yes");

  /* errors are returned, never aborted on */
  printf("negative nsteps: %s\n", rlb_step(h, -1) == RLB_EINVAL ? "EINVAL" : "other");
  rlb_tube bad = t[0];
  bad.Qxi = 2; /* 2 Qxi < Nv + 3 */
  rlb_handle hb = NULL;
  printf("bad orders: %s\n", rlb_init_riemann(&hb, &bad, 1, states, x_left, NULL) == RLB_EINVAL ? "EINVAL" : "other");

  FILE *f = fopen(argv[2], "wb");
  if (!f || fwrite(fa, sizeof(double), RLB_NFIELDS * nx, f) != (size_t)(RLB_NFIELDS * nx)) return 1;
  fclose(f);
  CHECK(rlb_destroy(h));
  free(ck);
  free(fa);
  free(fb);
  printf("done\n");
  return 0;
}
