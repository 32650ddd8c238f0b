// Element-wise kernels of the split path: exact digit extraction into BF16
// slices, max-abs reductions, and the per-triple double-float contravariant
// combination (paper, Algorithm 1: tau~ from tau with i, j, k fixed).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "dd.cuh"
#include "split_kernels.h"

namespace cc3 {

// Fixed-point value round(x * 2^sh) of a finite double as a signed 64-bit
// integer, from its bits (integer arithmetic only; |result| < 2^62 assumed).
__device__ __forceinline__ long long fixed_from_double(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal (below every digit used here)
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int s = ex - 1075 + sh;  // x = mant * 2^(ex-1075)
  long long v;
  if (s >= 0) {
    v = s > 9 ? (mant << 9) : (mant << s);  // |x 2^sh| < 2^62 keeps s <= 9
  } else if (s > -63) {
    v = (mant + (1ll << (-s - 1))) >> (-s);
  } else {
    v = 0;
  }
  return (b >> 63) ? -v : v;
}
__device__ __forceinline__ long long fixed_from_float(float x, int sh) {
  const unsigned int b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFF);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int s = ex - 150 + sh;  // x = mant * 2^(ex-150)
  long long v;
  if (s >= 0) {
    v = s > 38 ? (mant << 38) : (mant << s);
  } else if (s > -40) {
    v = (mant + (1ll << (-s - 1))) >> (-s);
  } else {
    v = 0;
  }
  return (b >> 31) ? -v : v;
}

// 2^(-8p): the exact scale of slice p (a multiply, not a library call)
__device__ __forceinline__ float slice_scale(int p) {
  return __int_as_float((127 - 8 * p) << 23);
}

// Balanced base-256 digits of T (|T| < 2^(7+8(s-1))): T = sum_p d_p 256^(s-1-p),
// d_p in [-128, 128]; slice p stores d_p 2^(-8p) as an exact BF16.
__device__ __forceinline__ void store_digits(long long T, int s, __nv_bfloat16 *dst,
                                             long long slice_stride) {
  float d[S_MAX_SLICES_K];
#pragma unroll
  for (int p = S_MAX_SLICES_K - 1; p >= 0; --p) {
    if (p < s) {
      if (p > 0) {
        const long long r = ((T + 128) & 255) - 128;
        d[p] = (float)(int)r;
        T = (T - r) >> 8;
      } else {
        d[0] = (float)(int)T;  // |d_0| <= 128 by the bound on T
      }
    }
  }
#pragma unroll
  for (int p = 0; p < S_MAX_SLICES_K; ++p)
    if (p < s) dst[p * slice_stride] = __float2bfloat16_rn(d[p] * slice_scale(p));
}

// Offset of slice 0 of (row r, k in 0..15) inside one 16-column K block of
// rows, in the tensor cores' canonical no-swizzle K-major order with the s
// slices interleaved per row group: each group of 8 rows holds, for slice
// 0..s-1 in turn, two 8 x 8 core matrices (the K halves, 64 elements apart);
// slice p is 128 p elements further, the next row group 128 s elements.
__device__ __forceinline__ long long cm_off(long long r, int k, int s) {
  return (r >> 3) * (128LL * s) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Slices of an FP64 tensor read through a strided gather
//   row = (r2, r1, r0), k = (k1, k0); value 0 outside (k0 < k0v, k1 < k1v),
// stored K-blocked: [slab][K/16][row groups][slice][8 x 16], row =
// slab * rps + r, rows per slab rounded up to 8.  The slices of every 16 x R
// tile the tensor cores read are one contiguous block.
__global__ void slice_gather_kernel(const double *__restrict__ src, __nv_bfloat16 *__restrict__ dst,
                                    int s, int e, Gather g, long long nrows, int Kp, int rps) {
  const long long n = nrows * Kp;
  const int sh = 7 + 8 * (s - 1) - e;
  const long long KB = Kp / 16;
  const long long rps8 = (rps + 7) / 8 * 8;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long row = idx / Kp;
    const int k = (int)(idx % Kp);
    int k1, k0;
    if (g.zblk) {
      k1 = (k / 16) % g.kin;
      k0 = 16 * (k / (16 * g.kin)) + (k % 16);
    } else {
      k1 = k / g.kin;
      k0 = k % g.kin;
    }
    long long T = 0;
    if (k0 < g.k0v && k1 < g.k1v) {
      const long long r0 = row % g.n0, r1 = (row / g.n0) % g.n1, r2 = row / ((long long)g.n0 * g.n1);
      const long long off = g.off + r2 * g.s2 + r1 * g.s1 + r0 * g.s0 + k1 * g.sk1 + k0 * g.sk0;
      T = fixed_from_double(src[off], sh);
    }
    const long long slab = row / rps, r = row % rps;
    const long long o = (slab * KB + k / 16) * rps8 * 16 * s + cm_off(r, k % 16, s);
    store_digits(T, s, dst + o, 128);
  }
}

__global__ void maxabs_kernel(const double *__restrict__ x, long long n,
                              unsigned long long *__restrict__ out) {
  unsigned long long m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull;
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// tau = (W_1 + W_2 + W_3) / (w - e_a - e_b - e_c + e_ijk) from the three
// partial sums of the W build, then
// tau~ = 4 tau^{abc} - 2 tau^{acb} - 2 tau^{cba} - 2 tau^{bac} + tau^{bca} + tau^{cab},
// all in double-float.  The partial sums are stored as W[slot][c][a][b]; tau~
// is written as TT[slot][a][b][c], together with the max |tau~| of each slot
// (float bits, atomic max).  TT may be the buffer of W_2 (see below).
//
// The six values tau^{pi(a,b,c)} over the permutations pi are the same set
// for every permutation of (a,b,c), and tau~ at each of the six points is a
// combination of that set: with E = tau^{abc} + tau^{bca} + tau^{cab} and
// O = tau^{acb} + tau^{cba} + tau^{bac},
//   tau~ at an even permutation (abc, bca, cab) = 3 tau^{itself} + E - 2 O,
//   tau~ at an odd one (acb, cba, bac)           = 3 tau^{itself} + O - 2 E.
// A block takes one triple of 8-cube indices A >= B >= C, forms tau for the
// (up to six distinct) cubes whose index triples permute it and stages them
// in shared memory (coalesced row reads), forms all six outputs of each of
// its points from the six staged values, and writes the output cubes back
// row by row: every partial sum is read once and every tau~ element written
// once.  The locations a block reads are exactly those it writes (the cubes
// of one permutation orbit, in either layout), so TT may alias W_2: each
// block reads all of its locations before it writes any.  When cube indices
// coincide, only points with a >= b (A = B) and b >= c (B = C) are formed,
// so that each output is produced by one thread.
constexpr int CV_SX = 8, CV_SZ = 65, CV_SLOT = 8 * CV_SZ;  // padded cube strides (float2)
__global__ void __launch_bounds__(256)
tau_contravariant_dd_kernel(const float2 *__restrict__ W1, const float2 *W2,
                            const float2 *__restrict__ W3, float2 *tt,
                            const float2 *__restrict__ ev, const float2 *__restrict__ eo,
                            float w_hi, float w_lo, int nv, unsigned int *__restrict__ maxbits,
                            float2 *__restrict__ tau_out) {
  __shared__ float2 sm[6][CV_SLOT];
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long sbase = blockIdx.y * nv3;
  // w - ... + e_ijk of this slot
  const float2 eos = eo[blockIdx.y];
  const dd::df wo = dd::add(dd::df{w_hi, w_lo}, dd::df{eos.x, eos.y});
  // block -> (A, B, C), A >= B >= C, in lexicographic order
  int r = blockIdx.x, A = 0;
  while (r >= (A + 1) * (A + 2) / 2) {
    r -= (A + 1) * (A + 2) / 2;
    ++A;
  }
  int B = 0;
  while (r >= B + 1) {
    r -= B + 1;
    ++B;
  }
  const int C = r;
  // cube of term q, order abc, acb, cba, bac, bca, cab (cube indices of the
  // tau superscripts); the same triple indexes the output cube of point q
  const int cx[6] = {A, A, C, B, B, C}, cy[6] = {B, C, B, A, C, A}, cz[6] = {C, B, A, C, A, B};
  int slot[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    slot[q] = q;
#pragma unroll
    for (int u = 0; u < q; ++u)
      if (slot[q] == q && cx[u] == cx[q] && cy[u] == cy[q] && cz[u] == cz[q]) slot[q] = u;
  }
  const int t = threadIdx.x;
  // The partial sums of two cubes at a time are loaded into registers before
  // any of them is used (12 loads in flight per thread); the first two cubes'
  // loads are issued before the reciprocals below are formed.
  float2 la[2][2][3];
  auto issue = [&](int q0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = q0 + k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = t + 256 * h, y = e & 7, x = (e >> 3) & 7, z = e >> 6;
        const int gx = cx[q] * 8 + x, gy = cy[q] * 8 + y, gz = cz[q] * 8 + z;
        if (slot[q] == q && gx < nv && gy < nv && gz < nv) {
          const long long i = sbase + (long long)gz * nv2 + (long long)gx * nv + gy;
          la[k][h][0] = W1[i];
          la[k][h][1] = W2[i];
          la[k][h][2] = W3[i];
        }
      }
    }
  };
  issue(0);
  // 1 / (w + e_ijk - e_a - e_b - e_c) at every point (a, b, c) of cube (A, B, C):
  // the six permuted points of the orbit share it, so each is formed once
  // (one dd division per orbit point instead of one per staged element)
  __shared__ float2 rcp[512];
  for (int u = t; u < 512; u += 256) {
    const int a = u >> 6, b = (u >> 3) & 7, c = u & 7;
    const int ga = A * 8 + a, gb = B * 8 + b, gc = C * 8 + c;
    if (ga >= nv || gb >= nv || gc >= nv) continue;
    const float2 ea = ev[ga], eb = ev[gb], ec = ev[gc];
    const dd::df d = dd::add(dd::add(dd::add(wo, dd::df{-ea.x, -ea.y}), dd::df{-eb.x, -eb.y}),
                             dd::df{-ec.x, -ec.y});
    const dd::df r = dd::div(dd::df{1.f, 0.f}, d);
    rcp[u] = make_float2(r.hi, r.lo);
  }
  __syncthreads();
  // stage tau^{xyz} of cube (X, Y, Z) at [z][x][y] (y contiguous in memory);
  // its point (x, y, z) is the point (a, b, c) of cube (A, B, C) with each
  // index moved to the slot of its cube index
  auto stage = [&](int q0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = q0 + k;
      if (slot[q] != q) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = t + 256 * h, y = e & 7, x = (e >> 3) & 7, z = e >> 6;
        const int gx = cx[q] * 8 + x, gy = cy[q] * 8 + y, gz = cz[q] * 8 + z;
        float2 v = make_float2(0.f, 0.f);
        if (gx < nv && gy < nv && gz < nv) {
          const float2 a1 = la[k][h][0], a2 = la[k][h][1], a3 = la[k][h][2];
          const dd::df sum =
              dd::add(dd::add(dd::df{a1.x, a1.y}, dd::df{a2.x, a2.y}), dd::df{a3.x, a3.y});
          // (a, b, c) of this point: abc, acb, cba, bac, bca, cab orders of q
          const int pa[6] = {x, x, z, y, z, y}, pb[6] = {y, z, y, x, x, z},
                    pc[6] = {z, y, x, z, y, x};
          const float2 r = rcp[pa[q] * 64 + pb[q] * 8 + pc[q]];
          const dd::df tau = dd::mul(sum, dd::df{r.x, r.y});
          v = make_float2(tau.hi, tau.lo);
        }
        sm[q][z * CV_SZ + x * CV_SX + y] = v;
      }
    }
  };
  stage(0);
  issue(2);
  stage(2);
  issue(4);
  stage(4);
  __syncthreads();
  if (tau_out) {  // tau itself, [slot][a][b][c] like tau~ (the densities' D_vv and D_oo)
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (slot[q] != q) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e = t + 256 * h, z = e & 7, y = (e >> 3) & 7, x = e >> 6;
        const int gx = cx[q] * 8 + x, gy = cy[q] * 8 + y, gz = cz[q] * 8 + z;
        if (gx < nv && gy < nv && gz < nv)
          tau_out[sbase + (long long)gx * nv2 + (long long)gy * nv + gz] =
              sm[q][z * CV_SZ + x * CV_SX + y];
      }
    }
  }
  dd::df v[2][6];
  bool own[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int p = t + 256 * h, a = p >> 6, b = (p >> 3) & 7, c = p & 7;
    const int ga = A * 8 + a, gb = B * 8 + b, gc = C * 8 + c;
    own[h] = ga < nv && gb < nv && gc < nv && !(A == B && ga < gb) && !(B == C && gb < gc);
    // term q's element sits at its cube's [z][x][y] with (x, y, z) the
    // permuted (a, b, c)
    const int off[6] = {c * CV_SZ + a * CV_SX + b, b * CV_SZ + a * CV_SX + c,
                        a * CV_SZ + c * CV_SX + b, c * CV_SZ + b * CV_SX + a,
                        a * CV_SZ + b * CV_SX + c, b * CV_SZ + c * CV_SX + a};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float2 w = sm[slot[q]][off[q]];
      v[h][q] = dd::df{w.x, w.y};
    }
  }
  __syncthreads();  // every staged value read: the cubes now take the outputs
  float mx = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!own[h]) continue;
    const int p = t + 256 * h, a = p >> 6, b = (p >> 3) & 7, c = p & 7;
    const dd::df E = dd::add(dd::add(v[h][0], v[h][4]), v[h][5]);
    const dd::df Od = dd::add(dd::add(v[h][1], v[h][2]), v[h][3]);
    const dd::df ke = dd::add(E, dd::scale(Od, -2.f)), ko = dd::add(Od, dd::scale(E, -2.f));
    // output point of term q in its cube, stored [i][j][k] (k contiguous)
    const int off[6] = {a * CV_SZ + b * CV_SX + c, a * CV_SZ + c * CV_SX + b,
                        c * CV_SZ + b * CV_SX + a, b * CV_SZ + a * CV_SX + c,
                        b * CV_SZ + c * CV_SX + a, c * CV_SZ + a * CV_SX + b};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const bool even = q == 0 || q == 4 || q == 5;
      const dd::df o = dd::add(dd::mul_f(v[h][q], 3.f), even ? ke : ko);
      sm[slot[q]][off[q]] = make_float2(o.hi, o.lo);
      mx = fmaxf(mx, fabsf(o.hi));
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (slot[q] != q) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = t + 256 * h, k = e & 7, j = (e >> 3) & 7, i = e >> 6;
      const int gi = cx[q] * 8 + i, gj = cy[q] * 8 + j, gk = cz[q] * 8 + k;
      if (gi < nv && gj < nv && gk < nv)
        tt[sbase + (long long)gi * nv2 + (long long)gj * nv + gk] = sm[q][i * CV_SZ + j * CV_SX + k];
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((t & 31) == 0) atomicMax(maxbits + blockIdx.y, __float_as_uint(mx));
}

// exponent e with max < 2^e (max slightly enlarged to cover the dd low part)
__global__ void slot_exponent_kernel(const unsigned int *__restrict__ maxbits, int *__restrict__ ex,
                                     int nslot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslot) return;
  const float m = __uint_as_float(maxbits[i]) * (1.0f + 1e-6f);
  int e = 0;
  if (m > 0.f) {
    frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  }
  ex[i] = e;
}

// One exponent for every active slot of a batch (slot u active when u % bj <
// ns): the largest of their maxima, so that the slices of all slots share a
// scale and contractions over several slots can run as one job.
__global__ void common_exponent_kernel(const unsigned int *__restrict__ maxbits,
                                       int *__restrict__ ex, int nslot, int bj, int ns) {
  __shared__ unsigned int red[256];
  unsigned int m = 0;
  for (int i = threadIdx.x; i < nslot; i += blockDim.x)
    if (i % bj < ns) m = max(m, maxbits[i]);  // non-negative floats order as their bits
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const float mf = __uint_as_float(red[0]) * (1.0f + 1e-6f);
  int e = 0;
  if (mf > 0.f) frexpf(mf, &e);
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) ex[i] = e;
}

// Slices of tau~ in the three cyclic layouts used by the residual
// contractions.  Layout L puts slot L outermost (rows x), then slot L+1 (y),
// then slot L+2 (z, padded to vp):
//   V_L[slot][kb = zb*nv + y][row group of x][slice][8 x 16 (zz)],  z = 16 zb + zz,
// core-matrix order inside every 16-column block.  Read as rows x with
// K = (zb, y, zz) it serves the vvov and singles contractions; read as rows
// (y, x) with K = z (the nv blocks of one zb are consecutive) it serves the
// ooov and F contractions.  One CTA converts a 16^3 cube of tau~ (read along
// its innermost index) into digits once, keeps them in shared memory, and
// writes the cube into all three layouts as whole 16-byte core rows.
// Digit cube in shared memory: element (a, b, c) of slice p at
// p * TT_PLANE + a * TT_APLANE + b * TT_PAD + c (bf16).  The a-plane stride is
// an odd number of 4-byte words, so that the 16 lanes of a layout-0 read
// (consecutive a) fall in distinct banks.
constexpr int TT_PAD = 18, TT_APLANE = 16 * TT_PAD + 2, TT_PLANE = 16 * TT_APLANE;
__global__ void __launch_bounds__(256)
slice_tt_kernel(const float2 *__restrict__ tt, __nv_bfloat16 *const *__restrict__ v, int nv,
                int vp, int s, const int *__restrict__ ex, int nslot_alloc) {
  extern __shared__ __nv_bfloat16 dig[];  // [p][a][b][c] (c padded to TT_PAD)
  (void)nslot_alloc;
  const int nx = (nv + 15) / 16, nzb = vp / 16;
  int blk = blockIdx.x;
  const int cb = blk % nx;
  blk /= nx;
  const int bb = blk % nx;
  const int ab = blk / nx;
  const int slot = blockIdx.y;
  const long long nv2 = (long long)nv * nv;
  const float2 *T = tt + (long long)slot * nv2 * nv;
  const int sh = 7 + 8 * (s - 1) - ex[slot];
  const int plane = TT_PLANE;
  // 2^sh and 2^(sh-24) as floats (the 32-bit digit path of s = 6)
  const float s0 = ldexpf(1.f, sh), s24 = ldexpf(1.f, sh - 24);
  // 16 elements per thread, loaded 8 at a time before any is converted (the
  // loads of a batch are in flight together)
#pragma unroll 1
  for (int i0 = 0; i0 < 16; i0 += 8) {
    float2 tv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + 256 * (i0 + u);
      const int c = e & 15, b = (e >> 4) & 15, a = e >> 8;
      const int ga = ab * 16 + a, gb = bb * 16 + b, gc = cb * 16 + c;
      tv[u] = make_float2(0.f, 0.f);
      if (ga < nv && gb < nv && gc < nv) tv[u] = T[(long long)ga * nv2 + (long long)gb * nv + gc];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + 256 * (i0 + u);
      const int c = e & 15, b = (e >> 4) & 15, a = e >> 8;
      // balanced base-256 digits of the fixed-point value T, slice p stores d_p 2^(-8p)
      float d[S_MAX_SLICES_K];
      if (s == 6 && sh >= 24 && sh <= 120) {  // 2^sh and 2^(sh-24) are normal floats
        // |T| < 2^47: T = th 2^24 + tl with 0 <= tl < 2^24, both in 32-bit
        // integers.  hi 2^(sh-24) = Hi + f (Hi = its floor, exact; f in [0, 1)),
        // so round(hi 2^sh) = Hi 2^24 + round(f 2^24); |lo| <= ulp(hi) / 2 keeps
        // round(lo 2^sh) below 2^23.  (Power-of-two scalings are exact.)
        const float H = tv[u].x * s24;
        const float Hi = floorf(H);
        int th = __float2int_rn(Hi);
        int tl = __float2int_rn((H - Hi) * 16777216.f) + __float2int_rn(tv[u].y * s0);
        const int cy = tl >> 24;  // floor(tl / 2^24)
        th += cy;
        tl -= cy * 16777216;
#pragma unroll
        for (int p = 5; p >= 3; --p) {  // the three low digits from tl
          const int r = ((tl + 128) & 255) - 128;
          d[p] = (float)r;
          tl = (tl - r) >> 8;
        }
        th += tl;  // the carry out of the low digits (0 or 1)
#pragma unroll
        for (int p = 2; p >= 1; --p) {
          const int r = ((th + 128) & 255) - 128;
          d[p] = (float)r;
          th = (th - r) >> 8;
        }
        d[0] = (float)th;  // |d_0| <= 128 by the bound on T
      } else {
        long long Tt = fixed_from_float(tv[u].x, sh) + fixed_from_float(tv[u].y, sh);
#pragma unroll
        for (int p = S_MAX_SLICES_K - 1; p >= 0; --p) {
          if (p < s) {
            if (p > 0) {
              const long long r = ((Tt + 128) & 255) - 128;
              d[p] = (float)(int)r;
              Tt = (Tt - r) >> 8;
            } else {
              d[0] = (float)(int)Tt;  // |d_0| <= 128 by the bound on Tt
            }
          }
        }
      }
      const int o = a * TT_APLANE + b * TT_PAD + c;
#pragma unroll
      for (int p = 0; p < S_MAX_SLICES_K; ++p)
        if (p < s) dig[p * plane + o] = __float2bfloat16_rn(d[p] * slice_scale(p));
    }
  }
  __syncthreads();
  const long long nv8 = (nv + 7) / 8 * 8;
  const long long KB = (long long)nzb * nv;
  const int x = threadIdx.x & 15, y = threadIdx.x >> 4;
#pragma unroll 1
  for (int L = 0; L < 3; ++L) {
    // block indices of this layout's (x, y, z) roles: (a,b,c), (b,c,a), (c,a,b)
    const int xb = L == 0 ? ab : (L == 1 ? bb : cb);
    const int yb = L == 0 ? bb : (L == 1 ? cb : ab);
    const int zb = L == 0 ? cb : (L == 1 ? ab : bb);
    const int gx = xb * 16 + x, gy = yb * 16 + y;
    if (gx >= nv || gy >= nv) continue;
    const long long blk0 = ((long long)slot * KB + (long long)zb * nv + gy) * nv8 * 16 * s;
    __nv_bfloat16 *dst = v[L];
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const long long o = blk0 + cm_off(gx, h * 8, s);
#pragma unroll 1
      for (int p = 0; p < s; ++p) {
        const __nv_bfloat16 *D = dig + p * plane;
        __align__(16) __nv_bfloat16 out[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int z = h * 8 + e;
          // (a, b, c) of the element with local (x, y, z) in layout L
          const int a = L == 0 ? x : (L == 1 ? z : y);
          const int b = L == 0 ? y : (L == 1 ? x : z);
          const int c = L == 0 ? z : (L == 1 ? y : x);
          out[e] = D[a * TT_APLANE + b * TT_PAD + c];
        }
        *reinterpret_cast<uint4 *>(dst + p * 128 + o) = *reinterpret_cast<const uint4 *>(out);
      }
    }
  }
}

// y = x as double-float pairs (hi = x rounded to FP32, lo = the rest)
__global__ void to_dd_kernel(const double *__restrict__ x, float2 *__restrict__ y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float h = (float)v;
    y[e] = make_float2(h, (float)(v - (double)h));
  }
}

// The outer products of the left transformation's L3 numerator, added to the
// W build's first partial sum W1[u][c][a][b] (double-float) of slot u = v * bj
// + t (vector v, triple t of the batch; slots with t >= ns are idle):
//   sum over the six terms of P of L1[o0][x] (o1 y|o2 z) + Lt2[o0][o1][x][y] F[o2][z],
// (o0,o1,o2) = (ijk[s0], ijk[s1], ijk[s2]), (x,y,z) = (v[s0], v[s1], v[s2]),
// v = (a, b, c).  All factors come as double-float pairs.  Consecutive threads
// take consecutive b; where b is y, the ovov factor is read as (o2 z|o1 y) and
// where b is x, the Lt2 factor as Lt2[o1][o0][y][x] (the integrals' pair symmetry
// and Lt2's pair symmetry), so that every factor that varies along b is read
// contiguously.
__global__ void __launch_bounds__(256)
left_outer_dd_kernel(float2 *__restrict__ W1, const int *__restrict__ tri, int bj, int ns,
                     const float2 *__restrict__ L1, const float2 *__restrict__ Lt,
                     const float2 *__restrict__ ovov, const float2 *__restrict__ F, int no,
                     int nv) {
  constexpr int P6[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0}, {0, 2, 1}, {1, 2, 0}, {2, 0, 1}};
  const int u = blockIdx.y, vec = u / bj, t = u % bj;
  if (t >= ns) return;
  const int ijk[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const long long n1 = (long long)no * nv, nt2 = n1 * no * nv;
  const float2 *l1 = L1 + vec * n1, *lt = Lt + vec * nt2;
  float2 *W = W1 + (long long)u * nv3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv3;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % nv), a = (int)((e / nv) % nv), c = (int)(e / nv2);
    const int v[3] = {a, b, c};
    dd::df sum = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int o0 = ijk[P6[q][0]], o1 = ijk[P6[q][1]], o2 = ijk[P6[q][2]];
      const int x = v[P6[q][0]], y = v[P6[q][1]], z = v[P6[q][2]];
      const float2 f1 = l1[(long long)o0 * nv + x];
      const float2 g1 = P6[q][1] == 1 ? ovov[(((long long)o2 * nv + z) * no + o1) * nv + y]
                                      : ovov[(((long long)o1 * nv + y) * no + o2) * nv + z];
      const float2 f2 = P6[q][0] == 1 ? lt[(((long long)o1 * no + o0) * nv + y) * nv + x]
                                      : lt[(((long long)o0 * no + o1) * nv + x) * nv + y];
      const float2 g2 = F[(long long)o2 * nv + z];
      sum = dd::add(sum, dd::add(dd::mul(dd::df{f1.x, f1.y}, dd::df{g1.x, g1.y}),
                                 dd::mul(dd::df{f2.x, f2.y}, dd::df{g2.x, g2.y})));
    }
    const float2 w0 = W[e];
    const dd::df r = dd::add(dd::df{w0.x, w0.y}, sum);
    W[e] = make_float2(r.hi, r.lo);
  }
}

// ---- launchers ----------------------------------------------------------------
static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 16384 ? (b > 0 ? b : 1) : 16384);
}

int launch_slice_gather(const double *src, __nv_bfloat16 *dst, int s, int e, const Gather &g,
                        long long nrows, int Kp, int rps, cudaStream_t st) {
  if (Kp % 16 != 0 || rps < 1 || nrows % rps != 0)
    return CC3_FAIL(CC3_ERR_ARG, "slice layout");
  slice_gather_kernel<<<grid_for(nrows * Kp), 256, 0, st>>>(src, dst, s, e, g, nrows, Kp, rps);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "split element-wise kernel launch");
}
int launch_maxabs(const double *x, long long n, unsigned long long *out, cudaStream_t st) {
  maxabs_kernel<<<grid_for(n), 256, 0, st>>>(x, n, out);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "split element-wise kernel launch");
}
int launch_tau_contravariant_dd(const float2 *W1, const float2 *W2, const float2 *W3,
                                float2 *tt, const float2 *ev, const float2 *eo, float w_hi,
                                float w_lo, int nv, int nslot, unsigned int *maxbits,
                                cudaStream_t st, float2 *tau_out) {
  if (nslot <= 0) return CC3_OK;
  const long long nx = (nv + 7) / 8, ncube = nx * (nx + 1) * (nx + 2) / 6;  // A >= B >= C
  if (ncube > 0x7fffffffLL || nslot > 65535)
    return CC3_FAIL(CC3_ERR_ARG, "tau_contravariant_dd grid");
  tau_contravariant_dd_kernel<<<dim3((unsigned)ncube, nslot), 256, 0, st>>>(
      W1, W2, W3, tt, ev, eo, w_hi, w_lo, nv, maxbits, tau_out);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "split element-wise kernel launch");
}
int launch_to_dd(const double *x, float2 *y, long long n, cudaStream_t st) {
  if (n <= 0) return CC3_OK;
  to_dd_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "to_dd launch");
}
int launch_left_outer_dd(float2 *W1, const int *tri, int bj, int ns, int nslot, const float2 *L1,
                         const float2 *Lt, const float2 *ovov, const float2 *F, int no, int nv,
                         cudaStream_t st) {
  if (nslot <= 0) return CC3_OK;
  if (nslot > 65535) return CC3_FAIL(CC3_ERR_ARG, "left outer products: slots");
  const long long nv3 = (long long)nv * nv * nv;
  const int blocks = (int)std::min<long long>((nv3 + 255) / 256, 2048);
  left_outer_dd_kernel<<<dim3(blocks, nslot), 256, 0, st>>>(W1, tri, bj, ns, L1, Lt, ovov, F, no,
                                                            nv);
  return cudaGetLastError() == cudaSuccess ? CC3_OK
                                           : CC3_FAIL(CC3_ERR_CUDA, "left outer products launch");
}
int launch_slot_exponent(const unsigned int *maxbits, int *ex, int nslot, cudaStream_t st) {
  slot_exponent_kernel<<<(nslot + 127) / 128, 128, 0, st>>>(maxbits, ex, nslot);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "split element-wise kernel launch");
}
// maxbits[u] = max |hi| (as float bits) over slot u's n elements of x
__global__ void slot_maxabs_dd_kernel(const float2 *__restrict__ x, long long n,
                                      unsigned int *__restrict__ maxbits) {
  const float2 *xs = x + (long long)blockIdx.y * n;
  float m = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(xs[e].x));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits + blockIdx.y, __float_as_uint(m));
}
__global__ void add_int_kernel(const int *__restrict__ a, const int *__restrict__ b,
                               int *__restrict__ c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] + b[i];
}
int launch_slot_maxabs_dd(const float2 *x, long long n, int nslot, unsigned int *maxbits,
                          cudaStream_t st) {
  if (nslot <= 0) return CC3_OK;
  if (nslot > 65535) return CC3_FAIL(CC3_ERR_ARG, "slot_maxabs: slots");
  const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
  slot_maxabs_dd_kernel<<<dim3(blocks, nslot), 256, 0, st>>>(x, n, maxbits);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "slot_maxabs launch");
}
int launch_add_int(const int *a, const int *b, int *c, int n, cudaStream_t st) {
  if (n <= 0) return CC3_OK;
  add_int_kernel<<<(n + 127) / 128, 128, 0, st>>>(a, b, c, n);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "add_int launch");
}
int launch_common_exponent(const unsigned int *maxbits, int *ex, int nslot, int bj, int ns,
                           cudaStream_t st) {
  if (nslot <= 0 || bj < 1) return CC3_OK;
  common_exponent_kernel<<<1, 256, 0, st>>>(maxbits, ex, nslot, bj, ns);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "split element-wise kernel launch");
}
int launch_slice_tt(const float2 *tt, __nv_bfloat16 *const *v, int nv, int vp, int s,
                    const int *ex, int nslot, int nslot_alloc, cudaStream_t st) {
  if (vp / 16 != (nv + 15) / 16 || s < 1 || s > S_MAX_SLICES_K)
    return CC3_FAIL(CC3_ERR_ARG, "slice_tt layout");
  const int nx = (nv + 15) / 16;
  const size_t smem = (size_t)s * TT_PLANE * sizeof(__nv_bfloat16);
  {
    static std::mutex mu;
    static bool set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && !set[dev]) {
      const size_t mx = (size_t)S_MAX_SLICES_K * TT_PLANE * sizeof(__nv_bfloat16);
      if (cudaFuncSetAttribute(slice_tt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)mx) != cudaSuccess)
        return CC3_FAIL(CC3_ERR_CUDA, "slice_tt shared memory");
      set[dev] = true;
    }
  }
  dim3 grid(nx * nx * nx, nslot);
  slice_tt_kernel<<<grid, 256, smem, st>>>(tt, v, nv, vp, s, ex, nslot_alloc);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, "slice_tt launch");
}

}  // namespace cc3
