// Launchers of the split path's element-wise kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cc3_internal.h"

namespace cc3 {

enum { S_MAX_SLICES_K = 8 };

// Strided gather of an FP64 tensor as a [rows][K] matrix:
//   row = (r2, r1, r0) with r0 < n0, r1 < n1;  k = (k1, k0) with k0 < kin;
//   element = src[off + r2*s2 + r1*s1 + r0*s0 + k1*sk1 + k0*sk0] when
//   k0 < k0v and k1 < k1v, else 0 (padding).
// With zblk = 1 the K index is instead (zb, u, zz) = (k / (16 kin), (k / 16) % kin,
// k % 16) and the element is src[... + u*sk1 + (16 zb + zz)*sk0], valid when
// 16 zb + zz < k0v and u < k1v: K runs over 16-wide blocks of the inner index
// with the outer index in between (the K order of the residual contractions).
struct Gather {
  long long off, s2, s1, s0, sk1, sk0;
  int n1, n0, kin, k0v, k1v;
  int zblk;
};

// dst layout: [slice][slab][K / 16][rps rows][16] (rows = slabs * rps)
int launch_slice_gather(const double *src, __nv_bfloat16 *dst, int s, int e, const Gather &g,
                        long long nrows, int Kp, int rps, cudaStream_t st);
int launch_maxabs(const double *x, long long n, unsigned long long *out, cudaStream_t st);
// tau from the W build's three partial sums W1 + W2 + W3 (dd, [slot][c][a][b])
// over (w - eps), and tau~ (dd, [slot][a][b][c]) into tt, which may be W2;
// ev: dd virtual orbital energies, eo: dd e_i + e_j + e_k of each slot
// tau_out (optional): tau itself, [slot][a][b][c] (dd), written as well
int launch_tau_contravariant_dd(const float2 *W1, const float2 *W2, const float2 *W3,
                                float2 *tt, const float2 *ev, const float2 *eo, float w_hi,
                                float w_lo, int nv, int nslot, unsigned int *maxbits,
                                cudaStream_t st, float2 *tau_out = nullptr);
int launch_slot_exponent(const unsigned int *maxbits, int *ex, int nslot, cudaStream_t st);
// maxbits[u] = max |x.hi| over the n elements of slot u (atomic max; zero it first)
int launch_slot_maxabs_dd(const float2 *x, long long n, int nslot, unsigned int *maxbits,
                          cudaStream_t st);
// c[i] = a[i] + b[i]
int launch_add_int(const int *a, const int *b, int *c, int n, cudaStream_t st);
// one exponent (that of the largest maximum) for every active slot u (u % bj < ns)
int launch_common_exponent(const unsigned int *maxbits, int *ex, int nslot, int bj, int ns,
                           cudaStream_t st);
// y[e] = x[e] as a double-float pair
int launch_to_dd(const double *x, float2 *y, long long n, cudaStream_t st);
// the left transformation's outer products L1 (x) g_ovov + Lt2 (x) F of the L3
// numerator (six terms of P) added to W1[u][c][a][b] (dd) of the nslot slots
// u = v * bj + t of a batch of ns triples (tri: 3 ints per triple); all
// factors as dd pairs (L1[v][i][a], Lt[v][i][j][a][b], ovov, F_ov)
int launch_left_outer_dd(float2 *W1, const int *tri, int bj, int ns, int nslot, const float2 *L1,
                         const float2 *Lt, const float2 *ovov, const float2 *F, int no, int nv,
                         cudaStream_t st);
// v: device array of 3 pointers (one per cyclic layout)
int launch_slice_tt(const float2 *tt, __nv_bfloat16 *const *v, int nv, int vp, int s,
                    const int *ex, int nslot, int nslot_alloc, cudaStream_t st);

}  // namespace cc3
