/*
 * eos.c -- TEST INFRASTRUCTURE ONLY (see oracle.h).  Stellar EOS of the oracle.
 * (Filled in with the stellar equation of state; until then the stellar path
 * reports an error.)
 */
#include <math.h>
#include "oracle.h"

int ora_eos_invert(const ora_cfg *cfg, double rho, double eint, const double *X,
                   double *T_inout, double *P, double *ge, double *gc, int *iters) {
  (void)cfg; (void)rho; (void)eint; (void)X; (void)T_inout; (void)P; (void)ge; (void)gc;
  if (iters) *iters = 0;
  return -3;
}
