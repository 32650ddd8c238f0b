// Split-precision (BF16 slice) path of libcc3.
#pragma once
#include "cc3_internal.h"

namespace cc3 {
int split_omega(cc3_ctx *c, cudaStream_t s);
void split_invalidate(cc3_ctx *c);
void split_destroy(cc3_ctx *c);
size_t split_footprint(int no, int nv, int slices, int ntri);
// right Jacobian transformation of nvec trial vectors (device pointers)
int split_jacobian(cc3_ctx *c, int nvec, const double *w, const double *R1, const double *R2,
                   double *rho1, double *rho2, cudaStream_t s);
size_t split_jacobian_footprint(int no, int nv, int slices, int nvec);
// Algorithm 3's densities of one left state (device pointers)
int split_density(cc3_ctx *c, double w, const double *L1, const double *L2, double *Doo,
                  double *Dov, double *Dvv, cudaStream_t s);
// left (transpose) Jacobian transformation of nvec left vectors (device pointers)
int split_left_jacobian(cc3_ctx *c, int nvec, const double *w, const double *L1,
                        const double *L2, double *sigma1, double *sigma2, cudaStream_t s);
int split_autotune(cc3_ctx *c, cudaStream_t s, int *ksteps_per_tile, int *ntile_w);
int split_tuning(cc3_ctx *c, int *ksteps_per_tile, int *ntile_w);
}  // namespace cc3
