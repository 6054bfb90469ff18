/* A plain C99 caller of the library's host-only entry points (test code):
 * it includes lrdmc.h, links liblrdmc.so and calls what needs no GPU, so a
 * CPU test can check that the boundary is usable from C. It prints
 * key=value lines for the test to compare with the oracle. Helium with a
 * 1s Slater orbital, zeta = 1.6875, and a Pade electron-electron Jastrow
 * factor. */
#include <stdio.h>
#include <string.h>

#include "lrdmc.h"

int main(void)
{
  const double xyz[3] = {0.0, 0.0, 0.0};
  const double Z[1] = {2.0};
  const double C[1] = {1.0};
  lrdmc_shell sh;
  lrdmc_jastrow jas;
  lrdmc_spacing_fn sp;
  lrdmc_system_t sys = NULL;
  lrdmc_status st;
  double ratio = 0.0, rc = 0.0;
  size_t bytes = 0;

  memset(&sh, 0, sizeof sh);
  sh.center = 0;
  sh.l = 0;
  sh.kind = 0;
  sh.n_eff = 1.0;
  sh.zeta = 1.6875;
  memset(&jas, 0, sizeof jas);
  jas.b_ee = 1.0;
  jas.c_par = 0.25;
  jas.c_anti = 0.5;
  jas.en_b2 = 1.0;
  jas.ee_on = 1;

  printf("build_flags=%d\n", lrdmc_build_flags());
  st = lrdmc_create_system(1, xyz, Z, 1, 1, &sh, 1, C, 1, 1, &jas, &sys);
  printf("create=%d\n", (int)st);
  if (st != LRDMC_OK) return 1;

  memset(&sp, 0, sizeof sp);
  sp.kind = LRDMC_DOUBLE_THIS_WORK;
  sp.beta = 0.75;
  sp.kappa = 2.5;
  st = lrdmc_spacing_params(sys, 0.2, &sp, &ratio, &rc);
  printf("spacing=%d\naprime_over_a=%.17g\nrc=%.17g\n", (int)st, ratio, rc);

  st = lrdmc_workspace_bytes(sys, 256, 100, &bytes);
  printf("workspace=%d\nbytes=%lu\n", (int)st, (unsigned long)bytes);

  /* errors come back as status codes with a message, never an abort */
  st = lrdmc_workspace_bytes(sys, 0, 100, &bytes);
  printf("bad_walkers=%d\n", (int)st);
  st = lrdmc_step(sys, 1, 0.2, &sp);
  printf("step_before_init=%d\nmessage=%s\n", (int)st, lrdmc_last_error(sys));
  lrdmc_destroy(sys);

  sys = NULL;
  st = lrdmc_create_system(1, xyz, Z, 40, 1, &sh, 1, C, 1, 1, &jas, &sys);
  printf("too_many_electrons=%d\n", (int)st);
  return 0;
}
