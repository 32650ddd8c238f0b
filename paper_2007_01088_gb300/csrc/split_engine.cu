// Split-precision tensor-core contraction engine (tcgen05, sm_103a).
//
// Each FP64 operand is carried as s integer-valued BF16 slices with one
// power-of-two scale per tensor: x = 2^(e-7) sum_p d_p 2^(-8p), |d_p| <= 128,
// slice p stored as the exact BF16 value d_p 2^(-8p).  A contraction
// sum_k A[m][k] B[n][k] becomes the triangle of slice products p + q <= s-1
// (the products with p + q >= s are below the representation error).  Every
// slice product is exact in FP32, but the tensor core's FP32 accumulation
// does not round to nearest when addends of very different size meet, so
// each level L = p + q <= 3 gets its own tensor-memory accumulator, whose
// values stay exactly representable (multiples of 2^-8L below 2^(24-8L))
// because it is drained into double-float registers every 256 K (at most
// 4 products of |d d'| <= 2^14 per K); the levels >= 4 share a fifth,
// rounded accumulator (its error stays below 2^-50 of the result).
//
// Warp roles (576 threads): warp 0 issues one bulk copy per operand tile (all
// s slices of a 128 x 16 A tile, resp. an Ntile x 16 B tile, pre-tiled in
// global memory in the canonical no-swizzle order with the slices interleaved
// per row group; one copy per slab when the A rows are flattened over slabs)
// into a ring of stages; one thread of warp 1 issues tcgen05.mma (M = 128,
// N = Ntile <= 96, K = 16, FP32 accumulate, A kept in the collector buffer
// across the products of one A slice) and owns the tensor-memory allocation
// (5 x Ntile columns); warps 2-17 drain and finish the accumulators (each
// quadrant of 32 TMEM lanes is read by four warps, one per column quarter, 4
// columns per load) and write the outputs (double-float stores, FP64 atomics
// or 128-bit fixed-point atomics) through up to four output descriptors.  At
// a drain point the issuer queues the next step's level >= 4 products before
// it waits for the drain, so the drain overlaps tensor work.  Every wait is
// bounded: on timeout the CTA sets an error word that the host turns into
// CC3_ERR_TIMEOUT; before it exits, the CTA waits (bounded again) for its own
// bulk copies and tensor-core products in flight, then frees its tensor
// memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>

#include <cuda_bf16.h>

#include "dd.cuh"
#include "sm100_prims.cuh"
#include "fx128.cuh"
#include "split_engine.h"

namespace cc3 {
using namespace sm100;

size_t s_smem_bytes(int slices, int ntile) {
  return (size_t)s_stages(slices) * slices * (S_BM + ntile) * 32 + 1024;
}

__device__ __forceinline__ long long s_rowoff(int m, int m_in, long long s1, long long s0) {
  return (long long)(m / m_in) * s1 + (long long)(m % m_in) * s0;
}

// One slice product p x q into accumulator min(p + q, 4), as element `i` of
// a run of `n` products that share A slice p (the run keeps A in the
// collector buffer instead of reading it from shared memory again).
template <int S>
__device__ __forceinline__ void issue_one(uint32_t tmem, uint64_t dA, uint64_t dB, uint32_t a16,
                                          uint32_t b16, uint32_t Nt, uint32_t idesc,
                                          uint32_t &fresh, int p, int q, int i, int n) {
  const int lv = p + q;
  const int acc = lv < 4 ? lv : 4;
  const uint32_t d = tmem + (uint32_t)acc * Nt, en = ((fresh >> acc) & 1u) ^ 1u;
  const uint64_t a = dA + (uint64_t)(p * a16), b = dB + (uint64_t)(q * b16);
  if (n == 1)
    umma_f16_a<0>(d, a, b, idesc, en);
  else if (i == 0)
    umma_f16_a<1>(d, a, b, idesc, en);
  else if (i == n - 1)
    umma_f16_a<3>(d, a, b, idesc, en);
  else
    umma_f16_a<2>(d, a, b, idesc, en);
  fresh &= ~(1u << acc);
}

// Issues the slice products of one K step whose level is >= 4 (HIGH) or
// <= 3 (!HIGH), fully unrolled; bit L of `fresh` marks accumulator L as not
// yet written since its last reset (its first product overwrites it).
template <int S, bool HIGH>
__device__ __forceinline__ void issue_products(uint32_t tmem, uint64_t dA, uint64_t dB,
                                               uint32_t a16, uint32_t b16, uint32_t Nt,
                                               uint32_t idesc, uint32_t &fresh) {
#pragma unroll
  for (int p = 0; p < S; ++p) {
    // q range of this group for slice p
    const int qlo = HIGH ? (4 - p > 0 ? 4 - p : 0) : 0;
    const int qhi = HIGH ? S - 1 - p : (3 - p < S - 1 - p ? 3 - p : S - 1 - p);
#pragma unroll
    for (int q = qlo; q <= qhi; ++q)
      issue_one<S>(tmem, dA, dB, a16, b16, Nt, idesc, fresh, p, q, q - qlo, qhi - qlo + 1);
  }
}

// All slice products of one K step, A slice by A slice (the order of a step
// that does not wait for a drain): A is read from shared memory S times
// instead of once per product.
template <int S>
__device__ __forceinline__ void issue_products_all(uint32_t tmem, uint64_t dA, uint64_t dB,
                                                   uint32_t a16, uint32_t b16, uint32_t Nt,
                                                   uint32_t idesc, uint32_t &fresh) {
#pragma unroll
  for (int p = 0; p < S; ++p)
#pragma unroll
    for (int q = 0; q < S - p; ++q)
      issue_one<S>(tmem, dA, dB, a16, b16, Nt, idesc, fresh, p, q, q, S - p);
}

// The slice products of two consecutive K steps with their A-slice runs
// interleaved (run p of step 0, run p of step 1, run p + 1 of step 0, ...):
// the first products that read a newly landed stage then overlap the other
// step's products instead of waiting alone.  Each run keeps its A slice in
// the collector buffer, as in issue_products_all.
template <int S>
__device__ __forceinline__ void issue_products_pair(uint32_t tmem, uint64_t dA0, uint64_t dB0,
                                                    uint32_t id0, uint64_t dA1, uint64_t dB1,
                                                    uint32_t id1, uint32_t Nt, uint32_t &fresh) {
#pragma unroll
  for (int p = 0; p < S; ++p) {
#pragma unroll
    for (int q = 0; q < S - p; ++q)
      issue_one<S>(tmem, dA0, dB0, 16u, 16u, Nt, id0, fresh, p, q, q, S - p);
#pragma unroll
    for (int q = 0; q < S - p; ++q)
      issue_one<S>(tmem, dA1, dB1, 16u, 16u, Nt, id1, fresh, p, q, q, S - p);
  }
}

// Kept out of line: inlined into the unrolled output loop it would make the
// kernel large enough for instruction-cache misses to stall the MMA warp.
__device__ __noinline__ void fx_add_call(unsigned long long *slot, double v) { fx_add(slot, v); }

// Position of one tile within its job: batch index, K-split part, M/N tile
// and its K-step range [g0, g1) over the concatenated terms.
struct TileInfo {
  int j, bi, m0, n0, Nt, g0, g1;
};

// jhint: the job of this CTA's previous tile (tiles are taken in increasing
// order, so the search only moves forward).
__device__ __forceinline__ TileInfo decode_tile(const SJob *__restrict__ jobs, int njobs,
                                                const STerm *__restrict__ terms, long long tile,
                                                int &jhint) {
  int j = jhint;
  if (j >= njobs || jobs[j].tile_base > tile) j = 0;
  while (j + 1 < njobs && jobs[j + 1].tile_base <= tile) ++j;
  jhint = j;
  const SJob &J = jobs[j];
  TileInfo t;
  t.j = j;
  const long long local = tile - J.tile_base;
  const int per_batch = J.tiles_m * J.tiles_n * J.ksplit;
  t.bi = (int)(local / per_batch);
  int r = (int)(local % per_batch);
  const int ks = r % J.ksplit;
  r /= J.ksplit;
  const int tn = r % J.tiles_n, tm = r / J.tiles_n;
  t.m0 = tm * S_BM;
  t.Nt = J.Ntile;
  t.n0 = tn * J.Ntile;
  int total = 0;
  for (int q = 0; q < J.nterm; ++q) total += terms[J.term0 + q].ksteps;
  const int per = (total + J.ksplit - 1) / J.ksplit;
  t.g0 = min(total, ks * per);
  t.g1 = min(total, t.g0 + per);
  return t;
}

// Persistent: one CTA per SM takes tiles from a launch-wide counter (the plan
// lists long tiles first) and keeps the stage ring, the TMEM allocation and
// the barriers across tiles.  The producer fetches each tile index and hands
// it to the MMA thread and the epilogue warps through a small ring in shared
// memory; the epilogue releases the accumulators as soon as it has read them,
// so the next tile's products start while it finishes the previous outputs.
// 96 registers: the 18 warps sit 5 to a sub-partition of 16,384 registers.
template <int S>
__global__ void __maxnreg__(96)
split_engine_kernel(const SJob *__restrict__ jobs, int njobs, const STerm *__restrict__ terms,
                    const __grid_constant__ SArrTable arrs, VPtrTable P,
                    int kdrain_steps, int *status, unsigned long long *tile_ctr,
                    long long ntiles) {
  constexpr int s = S;
  constexpr int S_STAGES = s_stages(S);
  constexpr int TQ = 4;  // depth of the tile hand-off ring
  // accumulators that receive products: level L <= 3 exists iff L <= S-1,
  // the shared one (levels >= 4) iff S >= 5
  constexpr int NLOW = S < 4 ? S : 4;
  constexpr bool HAS_HIGH = S >= 5;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[S_STAGES], empty[S_STAGES];
  __shared__ __align__(8) uint64_t accfull, accempty, drainfull, drainempty, mmafin;
  __shared__ __align__(8) uint64_t tfull[TQ], tempty[TQ];
  __shared__ long long tq[TQ];
  // the producer decodes each tile once for everyone (tinfo, with tq) and
  // marks each stage with the sign of its term, so that the MMA thread and
  // the epilogue read no job or term tables
  __shared__ TileInfo tinfo[TQ];
  __shared__ int sneg[S_STAGES];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int err;
  // each epilogue warp's copy of its current tile's job: the output loop reads
  // its fields for every element, and global reads of them (L1 is small next
  // to 216 KB of shared memory) put an L2 round trip on each element's path
  __shared__ SJob ejob[S_EPI_WARPS];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < TQ; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 1 + S_EPI_WARPS);
    }
    mbar_init(&accfull, 1);
    mbar_init(&accempty, S_EPI_WARPS);
    mbar_init(&drainfull, 1);
    mbar_init(&drainempty, S_EPI_WARPS);
    mbar_init(&mmafin, 1);
    err = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base_sh, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t a_bytes = S_BM * 32;

  if (warp == 0) {
    if (lane == 0) {
      // producer: tile indices, then the operand tiles of every K step
      int issued = 0, jh = 0;
      for (int i = 0;; ++i) {
        const int q = i % TQ;
        if (!mbar_wait(&tempty[q], ((i / TQ) & 1) ^ 1, &err)) break;
        const long long tile = (long long)atomicAdd(tile_ctr, 1ull);
        TileInfo ti;
        if (tile < ntiles) {
          ti = decode_tile(jobs, njobs, terms, tile, jh);
          tinfo[q] = ti;
        }
        tq[q] = tile < ntiles ? tile : -1;
        mbar_arrive(&tfull[q]);
        if (tile >= ntiles) break;
        const int Nt = ti.Nt, bi = ti.bi, m0 = ti.m0, n0 = ti.n0;
        const int term0 = jobs[ti.j].term0, nterm = jobs[ti.j].nterm;
        // term cursor; per-term operand addresses live in registers (the
        // barrier asm below would otherwise force the term and array
        // descriptors to be reloaded from memory every K step)
        int t = 0, kbase = 0;
        while (t < nterm && kbase + terms[term0 + t].ksteps <= ti.g0) {
          kbase += terms[term0 + t].ksteps;
          ++t;
        }
        int kend = -1, neg = 0;
        const __nv_bfloat16 *ga0 = nullptr, *gb0 = nullptr, *gt0 = nullptr, *ga20 = nullptr,
                            *gt20 = nullptr;
        long long kbsA = 0, kbsB = 0, kbsT = 0, kbsA2 = 0, kbsT2 = 0;
        int kmax = 0;
        uint32_t abytes = 0, mbytes = 0, tbytes = 0, toff = 0, a2bytes = 0, a2off = 0,
                 t2bytes = 0, t2off = 0;
        // flattened A rows: rows to load (0: not flattened), rows in the first
        // slab, rows per slab, slab stride and row 0 of the first slab
        int fra = 0, fseg = 0, frows = 0;
        long long fstride = 0;
        const __nv_bfloat16 *gaf = nullptr;
        bool bad = false;
        for (int g = ti.g0; g < ti.g1; ++g) {
          if (g >= kend) {
            if (kend >= 0) {
              kbase = kend;
              ++t;
            }
            const STerm T = terms[term0 + t];
            neg = T.negA;
            kend = kbase + T.ksteps;
            const SArr XA = arrs.a[T.A.map], XB = arrs.a[T.B.map], XT = arrs.a[T.Bt.map];
            const int ar = T.A.row0 + bi * T.A.row_b + m0, as = T.A.slab0 + bi * T.A.slab_b;
            const int bs = T.B.slab0 + bi * T.B.slab_b, ts = T.Bt.slab0 + bi * T.Bt.slab_b;
            // B tile rows [n0, n0 + Nt): main rows from B, rows in [nbm, nbm2) from
            // the tail Bt, rows >= nbm2 from the second tail Bt2
            const int nbm = T.nbm > 0 ? T.nbm : (1 << 30);
            const int nbm2 = T.nbm2 > 0 ? T.nbm2 : (1 << 30);
            const int br = T.B.row0 + bi * T.B.row_b + n0;
            const int nmain = max(0, min(min(Nt, nbm - n0), XB.rows - br));
            const int tfirst = max(n0, nbm);                  // first tail row of the tile
            const int tr = T.Bt.row0 + tfirst - nbm;          // its row in Bt
            const int ntail =
                T.nbm > 0 ? max(0, min(min(n0 + Nt, nbm2) - tfirst, XT.rows - tr)) : 0;
            kmax = XA.kblocks;
            if (nmain > 0) kmax = min(kmax, XB.kblocks);
            if (ntail > 0) kmax = min(kmax, XT.kblocks);
            // A rows: [ar, ar + ra) of slab as, or flattened over slabs as, as + 1, ...
            int ra = 0, fs = as, fr = ar;
            bool abad = as < 0 || ar < 0;
            if (!abad && T.aflat > 0) {
              ra = min(S_BM, T.aflat - ar);
              fs = as + ar / XA.rows;
              fr = ar % XA.rows;
              abad = ra <= 0 || as + (ar + ra - 1) / XA.rows >= XA.slabs || T.asplit > 0;
            } else if (!abad) {
              abad = as >= XA.slabs || ar >= XA.rows;
              ra = min(S_BM, XA.rows - ar);
              if (T.asplit > 0) ra = min(ra, T.asplit);
            }
            if (abad || (nmain > 0 && (bs < 0 || bs >= XB.slabs || br < 0)) ||
                (ntail > 0 && (ts < 0 || ts >= XT.slabs || tr < 0 || ((tfirst - n0) & 7) != 0))) {
              err = 2;  // a plan addressed outside its slice array: stop, report
              bad = true;
              break;
            }
            abytes = (uint32_t)ra * 32u;
            fra = T.aflat > 0 ? ra : 0;
            fseg = min(ra, XA.rows - fr);
            frows = XA.rows;
            fstride = XA.slab_stride;
            gaf = reinterpret_cast<const __nv_bfloat16 *>(XA.base) + (long long)fs * XA.slab_stride;
            mbytes = (uint32_t)nmain * 32u;
            tbytes = (uint32_t)ntail * 32u;
            toff = (uint32_t)(tfirst - n0) * 32u * s;
            a2bytes = 0;
            t2bytes = 0;
            if (T.asplit > 0) {  // second A segment
              const SArr XA2 = arrs.a[T.A2.map];
              const int ar2 = T.A2.row0 + bi * T.A2.row_b, as2 = T.A2.slab0 + bi * T.A2.slab_b;
              const int ra2 = min(S_BM - T.asplit, XA2.rows - ar2);
              if (as2 < 0 || as2 >= XA2.slabs || ar2 < 0 || ra2 <= 0 || (T.asplit & 7) != 0) {
                err = 2;
                bad = true;
                break;
              }
              kmax = min(kmax, XA2.kblocks);
              a2bytes = (uint32_t)ra2 * 32u;
              a2off = (uint32_t)T.asplit * 32u * s;
              ga20 = reinterpret_cast<const __nv_bfloat16 *>(XA2.base) +
                     (long long)as2 * XA2.slab_stride + (long long)ar2 * 16 * s;
              kbsA2 = XA2.kb_stride;
            }
            if (T.nbm2 > 0) {  // second tail
              const SArr XT2 = arrs.a[T.Bt2.map];
              const int t2first = max(n0, nbm2), ts2 = T.Bt2.slab0 + bi * T.Bt2.slab_b;
              const int tr2 = T.Bt2.row0 + t2first - nbm2;
              const int ntail2 = max(0, min(n0 + Nt - t2first, XT2.rows - tr2));
              if (ntail2 > 0) {
                if (ts2 < 0 || ts2 >= XT2.slabs || tr2 < 0 || ((t2first - n0) & 7) != 0) {
                  err = 2;
                  bad = true;
                  break;
                }
                kmax = min(kmax, XT2.kblocks);
                t2bytes = (uint32_t)ntail2 * 32u;
                t2off = (uint32_t)(t2first - n0) * 32u * s;
                gt20 = reinterpret_cast<const __nv_bfloat16 *>(XT2.base) +
                       (long long)ts2 * XT2.slab_stride + (long long)tr2 * 16 * s;
                kbsT2 = XT2.kb_stride;
              }
            }
            // one bulk copy per operand tile: its s slices are contiguous
            ga0 = gaf + (long long)fr * 16 * s;
            gb0 = reinterpret_cast<const __nv_bfloat16 *>(XB.base) + (long long)bs * XB.slab_stride +
                  (long long)br * 16 * s;
            gt0 = reinterpret_cast<const __nv_bfloat16 *>(XT.base) + (long long)ts * XT.slab_stride +
                  (long long)tr * 16 * s;
            kbsA = XA.kb_stride;
            kbsB = XB.kb_stride;
            kbsT = XT.kb_stride;
          }
          const int kb = g - kbase;
          if (kb >= kmax) {
            err = 2;
            bad = true;
            break;
          }
          const int st = issued % S_STAGES, ph = (issued / S_STAGES) & 1;
          if (!mbar_wait(&empty[st], ph ^ 1, &err)) { bad = true; break; }
          sneg[st] = neg;
          mbar_arrive_expect_tx(&full[st],
                                (uint32_t)s * (abytes + a2bytes + mbytes + tbytes + t2bytes));
          // stage layout: s A slices (128 rows) then s B slices (S_NT_MAX rows)
          uint8_t *sa = smem + (size_t)st * ((size_t)s * (a_bytes + S_NT_MAX * 32));
          uint8_t *sb = sa + (size_t)s * a_bytes;
          if (fra > 0) {  // one copy per slab the tile's rows touch
            const __nv_bfloat16 *src = ga0 + (long long)kb * kbsA, *sp = gaf + (long long)kb * kbsA;
            int r = 0, cnt = fseg;
            for (;;) {
              bulk_load(sa + (uint32_t)r * 32u * s, src, (uint32_t)cnt * 32u * s, &full[st]);
              r += cnt;
              if (r >= fra) break;
              sp += fstride;
              src = sp;
              cnt = min(fra - r, frows);
            }
          } else {
            bulk_load(sa, ga0 + (long long)kb * kbsA, (uint32_t)s * abytes, &full[st]);
          }
          if (a2bytes)
            bulk_load(sa + a2off, ga20 + (long long)kb * kbsA2, (uint32_t)s * a2bytes, &full[st]);
          if (mbytes) bulk_load(sb, gb0 + (long long)kb * kbsB, (uint32_t)s * mbytes, &full[st]);
          if (tbytes)
            bulk_load(sb + toff, gt0 + (long long)kb * kbsT, (uint32_t)s * tbytes, &full[st]);
          if (t2bytes)
            bulk_load(sb + t2off, gt20 + (long long)kb * kbsT2, (uint32_t)s * t2bytes, &full[st]);
          ++issued;
        }
        if (bad) break;
      }
      // let every issued copy land before the CTA may exit, also after a
      // give-up (bounded; the wait ignores the error word)
      for (int i = (issued > S_STAGES ? issued - S_STAGES : 0); i < issued; ++i)
        mbar_wait_quiet(&full[i % S_STAGES], (i / S_STAGES) & 1, 500000000ull);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int it = 0, nd = 0;
      bool ok = true;
      for (int i = 0; ok; ++i) {
        const int q = i % TQ;
        if (!mbar_wait(&tfull[q], (i / TQ) & 1, &err)) break;
        const long long tile = tq[q];
        const TileInfo ti = tinfo[q];  // read before the slot is handed back
        mbar_arrive(&tempty[q]);
        if (tile < 0) break;
        const int Nt = ti.Nt;
        const uint32_t id_pos = idesc_bf16(S_BM, Nt, 0), id_neg = idesc_bf16(S_BM, Nt, 1);
        // the epilogue has read the previous tile's accumulators
        if (i > 0) {
          if (!mbar_wait(&accempty, (i - 1) & 1, &err)) break;
          tc_fence_after();
        }
        uint32_t fresh = (1u << S_NACC) - 1;
        int since = 0;
        bool pending = false;
        // K steps two at a time (drains come every kdrain_steps, an even
        // number, so a pair never straddles one); a lone last step of a tile
        // goes alone
        for (int g = ti.g0; g < ti.g1;) {
          const bool two = g + 1 < ti.g1;
          const int st0 = it % S_STAGES, ph0 = (it / S_STAGES) & 1;
          const int st1 = (it + 1) % S_STAGES, ph1 = ((it + 1) / S_STAGES) & 1;
          if (!mbar_wait(&full[st0], ph0, &err)) { ok = false; break; }
          if (two && !mbar_wait(&full[st1], ph1, &err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t id0 = sneg[st0] ? id_neg : id_pos, id1 = sneg[st1] ? id_neg : id_pos;
          const size_t stage_bytes = (size_t)s * (a_bytes + S_NT_MAX * 32);
          const uint32_t sa0 = smem_u32(smem + (size_t)st0 * stage_bytes),
                         sa1 = smem_u32(smem + (size_t)st1 * stage_bytes);
          // slice p of a tile starts 256 p bytes in; row groups are 256 s bytes apart
          const uint64_t dA0 = smem_desc_kmajor(sa0, 256u * s),
                         dB0 = smem_desc_kmajor(sa0 + (uint32_t)s * a_bytes, 256u * s),
                         dA1 = smem_desc_kmajor(sa1, 256u * s),
                         dB1 = smem_desc_kmajor(sa1 + (uint32_t)s * a_bytes, 256u * s);
          if (pending) {
            // levels >= 4 first (they never wait for a drain), then levels 0..3
            issue_products<S, true>(tmem, dA0, dB0, 16u, 16u, (uint32_t)Nt, id0, fresh);
            if (two) issue_products<S, true>(tmem, dA1, dB1, 16u, 16u, (uint32_t)Nt, id1, fresh);
            if (!mbar_wait(&drainempty, nd & 1, &err)) { ok = false; break; }
            tc_fence_after();
            ++nd;
            pending = false;
            fresh |= 0xFu;
            issue_products<S, false>(tmem, dA0, dB0, 16u, 16u, (uint32_t)Nt, id0, fresh);
            if (two) issue_products<S, false>(tmem, dA1, dB1, 16u, 16u, (uint32_t)Nt, id1, fresh);
          } else if (two) {
            issue_products_pair<S>(tmem, dA0, dB0, id0, dA1, dB1, id1, (uint32_t)Nt, fresh);
          } else {
            issue_products_all<S>(tmem, dA0, dB0, 16u, 16u, (uint32_t)Nt, id0, fresh);
          }
          umma_commit(&empty[st0]);
          if (two) umma_commit(&empty[st1]);
          const int n = two ? 2 : 1;
          g += n;
          it += n;
          since += n;
          if (since >= kdrain_steps && g < ti.g1) {
            umma_commit(&drainfull);
            pending = true;
            since = 0;
          }
        }
        if (!ok) break;
        umma_commit(&accfull);
      }
      // every product this thread issued has landed in tensor memory before
      // the CTA frees it, also after a give-up (bounded)
      umma_commit(&mmafin);
      mbar_wait_quiet(&mmafin, 0, 500000000ull);
    }
  } else {
    // epilogue: warps 2..17
    const int ew = warp - 2, quad = warp & 3, part = ew >> 2;
    const int row = quad * 32 + lane;
    int nd = 0, jh = 0;
    for (int i = 0;; ++i) {
      const int q = i % TQ;
      if (!mbar_wait_sleep(&tfull[q], (i / TQ) & 1, &err)) break;
      const long long tile = tq[q];
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[q]);
      if (tile < 0) break;
      // decoded again from the (read-only) tables: the compiler may reload
      // these values instead of holding them in registers across the asm
      const TileInfo ti = decode_tile(jobs, njobs, terms, tile, jh);
      __syncwarp();  // every lane is done with the previous tile's job
      {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(jobs + ti.j);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&ejob[ew]);
        for (int w = lane; w < (int)(sizeof(SJob) / 4); w += 32) dst[w] = src[w];
      }
      __syncwarp();
      const SJob &J = ejob[ew];
      const int Nt = ti.Nt;
      const int nsteps = ti.g1 - ti.g0;
      const int ndrains = nsteps > 0 ? (nsteps - 1) / kdrain_steps : 0;
      const int qc = Nt >> 2;   // columns per quarter (multiple of 4, <= 24)
      const int nch = qc >> 2;  // 4-column chunks (<= 6)
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(part * qc);
      dd::df acc[6][4];
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[c][k] = {0.f, 0.f};
      bool ok = true;
      for (int d = 0; d < ndrains && ok; ++d, ++nd) {
        ok = mbar_wait_sleep(&drainfull, nd & 1, &err);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          if (c < nch) {
            float v[4][4];
#pragma unroll
            for (int L = 0; L < 4; ++L) {
              if (L < NLOW) {
                tmem_ld4(tb + L * Nt + c * 4, v[L]);
              } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) v[L][k] = 0.f;
              }
            }
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              dd::df x = dd::two_sum(v[0][k], v[1][k]);
              x = dd::add_f(x, v[2][k]);
              x = dd::add_f(x, v[3][k]);
              acc[c][k] = dd::add(acc[c][k], x);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&drainempty);
      }
      if (!ok) break;
      if (!mbar_wait_sleep(&accfull, i & 1, &err)) break;
      tc_fence_after();
      // fold the final partial sums into acc, then hand the accumulators back
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (c < nch && nsteps > 0) {
          float v[5][4];
#pragma unroll
          for (int L = 0; L < 5; ++L) {
            if (L < NLOW || (L == 4 && HAS_HIGH)) {
              tmem_ld4(tb + L * Nt + c * 4, v[L]);
            } else {
#pragma unroll
              for (int k = 0; k < 4; ++k) v[L][k] = 0.f;
            }
          }
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            dd::df x = dd::two_sum(v[0][k], v[1][k]);
            x = dd::add_f(x, v[2][k]);
            x = dd::add_f(x, v[3][k]);
            x = dd::add(acc[c][k], x);
            acc[c][k] = dd::add_f(x, v[4][k]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty);
      const int bi = ti.bi, n0 = ti.n0, m = ti.m0 + row;
      const int *slot_ex = reinterpret_cast<const int *>(P.p[B_SLOTEXP]);
      const bool seg2 = J.msplit > 0 && m >= J.msplit;  // second row segment
      // the per-triple exponent table is read only by jobs that name a slot
      const int es = seg2 ? J.expo_slot2 : J.expo_slot;
      const float sc = ldexpf(J.mult, J.expo + (es >= 0 ? slot_ex[es] : 0));
      const int mo = seg2 ? m - J.msplit : m;  // row within its output
      const bool row_ok = m < J.M && !(J.m_pad > 0 && (m % J.m_pad) >= J.m_valid);
      // the thread's row is fixed for the tile: its output row offsets once.
      // Main columns n < Nm go to C (C2 for second-segment rows), tail
      // columns n in [tlo, thi) to Ct (Ct2); columns map linearly (n_in >= N,
      // checked when the plan is uploaded)
      const OutD &Cm = seg2 ? J.C2 : J.C;
      const long long rowM =
          row_ok ? Cm.off + (long long)bi * Cm.sb + s_rowoff(mo, Cm.m_in, Cm.sm1, Cm.sm0) : 0;
      const int mq = mo / Cm.m_in, mr = mo % Cm.m_in;  // route 1: shared by its outputs
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        if (c < nch) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const dd::df x = dd::scale(acc[c][k], sc);
            const int n = n0 + part * qc + c * 4 + k;
            if (!row_ok || n >= J.N) continue;
            long long off;
            int buf;
            if (J.route == 1) {  // two column segments (see SJob)
              const bool sg = n >= J.Nm2;
              const int jc = sg ? n - J.Nm2 : n;
              if (jc >= J.Nm + J.tw) continue;
              const OutD &O = jc < J.Nm ? (sg ? J.C2 : J.C) : (sg ? J.Ct2 : J.Ct);
              off = O.off + (long long)bi * O.sb + (long long)mq * O.sm1 + (long long)mr * O.sm0 +
                    (long long)(jc < J.Nm ? jc : jc - J.Nm) * O.sn0;
              buf = O.buf;
            } else if (n < J.Nm) {
              if (n >= J.n_valid) continue;
              off = rowM + (long long)n * Cm.sn0;
              buf = Cm.buf;
            } else {  // tail columns are few: their offsets on the fly
              const OutD &Ctl = seg2 ? J.Ct2 : J.Ct;
              const int tlo = seg2 ? (J.Nm2 > 0 ? J.Nm2 : J.N) : J.Nm;
              const int thi = seg2 ? J.N : (J.Nm2 > 0 ? J.Nm2 : J.N);
              if (n < tlo || n >= thi) continue;
              off = Ctl.off + (long long)bi * Ctl.sb + s_rowoff(mo, Ctl.m_in, Ctl.sm1, Ctl.sm0) +
                    (long long)(n - tlo) * Ctl.sn0;
              buf = Ctl.buf;
            }
            if (J.mode == SEPI_DD_STORE) {
              reinterpret_cast<float2 *>(P.p[buf])[off] = make_float2(x.hi, x.lo);
            } else if (P.fx[buf]) {
              fx_add_call(P.fx[buf] + 2 * off, dd::to_double(x));
            } else {
              atomicAdd(reinterpret_cast<double *>(P.p[buf]) + off, dd::to_double(x));
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (threadIdx.x == 0 && err) atomicExch(status, err);
}

int s_upload_plan(const SPlan &p, SDevPlan *d, cudaStream_t s) {
  s_free_plan(d);
  // the epilogue maps output columns linearly (n * sn0): no output may split
  // its columns (n_in >= N)
  for (const SJob &j : p.jobs) {
    const bool two = j.msplit > 0;
    const bool r1 = j.route == 1;
    const OutD *outs[4] = {&j.C, &j.Ct, two || r1 ? &j.C2 : nullptr, two || r1 ? &j.Ct2 : nullptr};
    for (const OutD *o : outs)
      if (o && (o->n_in < j.N || (r1 && o->m_in != j.C.m_in))) return CC3_ERR_ARG;
    if (r1 && (two || j.Nm2 <= 0 || j.Nm + j.tw > j.Nm2)) return CC3_ERR_ARG;
  }
  if (cudaMalloc(&d->counter, sizeof(unsigned long long)) != cudaSuccess) return CC3_ERR_OOM;
  d->njobs = (int)p.jobs.size();
  d->tiles = p.tiles;
  d->flop = p.flop;
  d->slice_flop = p.slice_flop;
  if (d->njobs == 0) return CC3_OK;
  if (cudaMalloc(&d->jobs, sizeof(SJob) * p.jobs.size()) != cudaSuccess) return CC3_ERR_OOM;
  if (cudaMalloc(&d->terms, sizeof(STerm) * (p.terms.size() + 1)) != cudaSuccess)
    return CC3_ERR_OOM;
  if (cudaMemcpyAsync(d->jobs, p.jobs.data(), sizeof(SJob) * p.jobs.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CC3_ERR_CUDA;
  if (!p.terms.empty() &&
      cudaMemcpyAsync(d->terms, p.terms.data(), sizeof(STerm) * p.terms.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CC3_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CC3_ERR_CUDA;
  return CC3_OK;
}

void s_free_plan(SDevPlan *d) {
  if (d->counter) cudaFree(d->counter);
  d->counter = nullptr;
  if (d->jobs) cudaFree(d->jobs);
  if (d->terms) cudaFree(d->terms);
  d->jobs = nullptr;
  d->terms = nullptr;
  d->njobs = 0;
  d->tiles = 0;
}

int s_launch_plan(const SDevPlan &d, const SArrTable &arrs, const VPtrTable &ptrs,
                  int slices, int kdrain_steps, int *status, cudaStream_t s,
                  long long *launches) {
  if (d.njobs == 0 || d.tiles == 0) return CC3_OK;
  if (d.tiles > 0x7fffffffLL) return CC3_ERR_ARG;
  if (slices < 3 || slices > S_MAX_SLICES) return CC3_ERR_ARG;
  // the issuer takes K steps in pairs, so the exact accumulators are drained
  // after an even number of steps: the interval must be even (and at most 16,
  // the bound that keeps them exact)
  if (kdrain_steps < 2 || kdrain_steps > 16 || (kdrain_steps & 1))
    return CC3_FAIL(CC3_ERR_ARG, "drain interval");
  // at least 120 KB so that one CTA (and one 512-column TMEM allocation) per SM
  const size_t smem = std::max<size_t>(s_smem_bytes(slices, S_NT_MAX), 120 * 1024);
  // per device, once; several host threads (serving slots) may get here at once
  static std::mutex attr_mu;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return CC3_FAIL(CC3_ERR_CUDA, "device index");
  std::lock_guard<std::mutex> attr_lk(attr_mu);
  if (!attr_set[dev]) {
    const void *fns[] = {(const void *)split_engine_kernel<3>, (const void *)split_engine_kernel<4>,
                         (const void *)split_engine_kernel<5>, (const void *)split_engine_kernel<6>,
                         (const void *)split_engine_kernel<7>};
    for (int S = 3; S <= 7; ++S) {
      const void *f = fns[S - 3];
      const int mx = (int)std::max<size_t>(s_smem_bytes(S, S_NT_MAX), 120 * 1024);
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      if (e != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e));
      int nb = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, S_THREADS, (size_t)mx);
      if (e != cudaSuccess || nb < 1)
        return CC3_FAIL(CC3_ERR_CUDA, "split engine kernel does not fit on an SM");
    }
    attr_set[dev] = true;
  }
  static int sms[64] = {0};
  if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<long long>(d.tiles, std::max(1, sms[dev]));
  const cudaError_t me = cudaMemsetAsync(d.counter, 0, sizeof(unsigned long long), s);
  if (me != cudaSuccess) return CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(me));
  switch (slices) {
#define CC3_SPLIT_LAUNCH(S_)                                                              \
  case S_:                                                                                \
    split_engine_kernel<S_><<<grid, S_THREADS, smem, s>>>(                                \
        d.jobs, d.njobs, d.terms, arrs, ptrs, kdrain_steps, status, d.counter, d.tiles);  \
    break;
    CC3_SPLIT_LAUNCH(3)
    CC3_SPLIT_LAUNCH(4)
    CC3_SPLIT_LAUNCH(5)
    CC3_SPLIT_LAUNCH(6)
    CC3_SPLIT_LAUNCH(7)
#undef CC3_SPLIT_LAUNCH
    default:
      return CC3_FAIL(CC3_ERR_ARG, "slices");
  }
  if (launches) ++*launches;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CC3_OK : CC3_FAIL(CC3_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace cc3
