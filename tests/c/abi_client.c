/* A plain C client of libsld: compiled with gcc against include/sld.h and
 * linked to the library, it checks what needs no GPU -- the defaults and the
 * argument checks, which return status codes and set sld_last_error(). */
#include <stdio.h>
#include <string.h>

#include "sld.h"
#include "sld_net.h"

static int fails = 0;
#define CHECK(c)                                        \
  do {                                                  \
    if (!(c)) {                                         \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
      ++fails;                                          \
    }                                                   \
  } while (0)

int main(void) {
  sld_options o;
  memset(&o, 0xff, sizeof o);
  sld_default_options(&o);
  CHECK(o.precision == SLD_FP64);
  CHECK(o.tol == 1e-9);
  CHECK(o.maxiter == 20000 && o.max_outer == 40 && o.ctas_per_sm == 0);
  CHECK(o.debug_skip_barrier == -1);
  CHECK(o.fwd_tol == 0.0);
  /* argument checks happen before any device work */
  double x = 0.0;
  CHECK(sld_solve(NULL, NULL, &o, &x, NULL) == SLD_ERR_INVALID_ARG);
  CHECK(strlen(sld_last_error()) > 0);
  CHECK(sld_solve_gmres(NULL, NULL, 20, 1, 1e-6, 100, &x, NULL) == SLD_ERR_INVALID_ARG);
  int d = -1;
  CHECK(sld_make_labels_cc(NULL, 1, 1, 1, NULL, 1, NULL, &d) == SLD_ERR_INVALID_ARG);
  CHECK(sld_solve_rdgmres(NULL, NULL, 30, 3, 1e-6, 100, &x, NULL) == SLD_ERR_INVALID_ARG);
  {
    /* harmonic Ritz pairs of a 2-step "Arnoldi cycle": pure host code */
    const double Hbar[3 * 2] = {2.0, 1.0, 1.0, 3.0, 0.0, 0.0}; /* h_{3,2} = 0: F = H_2 */
    double Y[2 * 2], tre[2], tim[2];
    CHECK(sld_harmonic_ritz(Hbar, 2, 2, Y, tre, tim) == SLD_OK);
    /* eigenvalues of [[2, 1], [1, 3]]: (5 -+ sqrt 5) / 2, smallest first */
    CHECK(tre[0] > 1.38 && tre[0] < 1.39 && tre[1] > 3.61 && tre[1] < 3.62 && tim[0] == 0.0);
    CHECK(sld_harmonic_ritz(Hbar, 1, 1, Y, tre, tim) == SLD_ERR_INVALID_ARG);
  }
  CHECK(sld_net_num_params() > 0);
  {
    /* the learned-deflation calls: defaults, and argument checks before any device work */
    sld_train_options t;
    memset(&t, 0xff, sizeof t);
    sld_default_train_options(&t);
    CHECK(t.epochs == 12 && t.lr > 1.99e-3f && t.lr < 2.01e-3f && t.lr_decay == 0.5f && t.decay_every == 0);
    CHECK(t.beta1 == 0.9f && t.beta2 > 0.998f && t.seed == 0);
    CHECK(sld_learned_train(NULL, 1, NULL, NULL, 8, NULL, &t, NULL) == SLD_ERR_INVALID_ARG);
    CHECK(sld_learned_infer(NULL, NULL, NULL) == SLD_ERR_INVALID_ARG);
    CHECK(strlen(sld_last_error()) > 0);
  }
  sld_destroy(NULL); /* ignored */
  printf("%s\n", fails ? "FAIL" : "OK");
  return fails ? 1 : 0;
}
