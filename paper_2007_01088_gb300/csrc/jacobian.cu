// Right Jacobian transformation (placeholder).
#include "cc3_internal.h"

extern "C" int cc3_jacobian_triples(cc3_ctx *c, cc3_prec, int, const double *,
                                    const double *, const double *, double *,
                                    double *, void *) {
  return c ? CC3_ERR_UNSUPPORTED : CC3_ERR_ARG;
}
