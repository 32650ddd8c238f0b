// FP64 multi-term contraction engine.
//
// One launch runs a list of jobs; each job is a batched multi-term contraction
//   C[b][m][n] (op)= sum_terms sum_k A_t[b][m][k] * B_t[b][n][k]
// over strided two-level operand views (cc3::Opnd), with three epilogues:
// plain store, FP64 atomic accumulation (cross-triple sums of the residual)
// and the triples denominator tau = (C + acc) / (w - eps^{abc}_{ijk}).
//
// On this GPU the FP64 pipe retires ~2 DFMA per clock per SM (about 1 TFLOP/s
// for the chip), so an FP64 contraction is compute bound at any practical
// tile size; the tile is sized for DFMA latency hiding (16 independent
// accumulators per thread), not for bandwidth.
#include <cuda_runtime.h>

#include "cc3_internal.h"
#include "fx128.cuh"

namespace cc3 {

__device__ __forceinline__ long long rowoff(int m, int m_in, long long s1,
                                            long long s0) {
  return (long long)(m / m_in) * s1 + (long long)(m % m_in) * s0;
}

template <int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__(256)
fp64_engine_kernel(const Job *__restrict__ jobs, int njobs,
                   const Term *__restrict__ terms, PtrTable P) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  __shared__ double sA[BK][BM];
  __shared__ double sB[BK][BN];
  const long long cta = blockIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_base <= cta) lo = mid; else hi = mid - 1;
  }
  const Job &J = jobs[lo];
  long long local = cta - J.tile_base;
  const int per_batch = J.tiles_m * J.tiles_n * J.ksplit;
  const int bi = (int)(local / per_batch);
  int r = (int)(local % per_batch);
  const int ks = r % J.ksplit;
  r /= J.ksplit;
  const int tn = r % J.tiles_n, tm = r / J.tiles_n;
  const int m0 = tm * BM, n0 = tn * BN;
  const int M = J.M, N = J.N, Nm = J.Nm;

  constexpr int NTX = BN / TN;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int t = 0; t < J.nterm; ++t) {
    const Term &T = terms[J.term0 + t];
    const int K = T.K;
    int kchunk = (K + J.ksplit - 1) / J.ksplit;
    kchunk = (kchunk + BK - 1) / BK * BK;
    const int kbeg = ks * kchunk;
    const int kend = min(K, kbeg + kchunk);
    if (kbeg >= kend) continue;
    const double *Ab = P.p[T.A.buf] + T.A.off + (long long)bi * T.A.sb;
    const double *Bb = P.p[T.B.buf] + T.B.off + (long long)bi * T.B.sb;
    const double *Btb = P.p[T.Bt.buf] + T.Bt.off + (long long)bi * T.Bt.sb;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        const int mm = e / BK, kk = e % BK;
        const int m = m0 + mm, k = k0 + kk;
        double v = 0.0;
        if (m < M && k < kend)
          v = Ab[rowoff(m, T.A.m_in, T.A.sm1, T.A.sm0) +
                 rowoff(k, T.A.k_in, T.A.sk1, T.A.sk0)];
        sA[kk][mm] = T.A.neg ? -v : v;
      }
      for (int e = tid; e < BN * BK; e += 256) {
        const int nn = e / BK, kk = e % BK;
        const int n = n0 + nn, k = k0 + kk;
        double v = 0.0;
        if (n < N && k < kend) {
          if (n < Nm) {
            v = Bb[rowoff(n, T.B.m_in, T.B.sm1, T.B.sm0) +
                   rowoff(k, T.B.k_in, T.B.sk1, T.B.sk0)];
            if (T.B.neg) v = -v;
          } else {
            const int nt = n - Nm;
            v = Btb[rowoff(nt, T.Bt.m_in, T.Bt.sm1, T.Bt.sm0) +
                    rowoff(k, T.Bt.k_in, T.Bt.sk1, T.Bt.sk0)];
            if (T.Bt.neg) v = -v;
          }
        }
        sB[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = sA[kk][ty + i * (BM / TM)];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = sB[kk][tx + j * NTX];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }

  // epilogue
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + i * (BM / TM);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + j * NTX;
      if (n >= N) continue;
      const OutD &C = (n < Nm) ? J.C : J.Ct;
      const int nc = (n < Nm) ? n : n - Nm;
      double *dst = P.p[C.buf] + C.off + (long long)bi * C.sb +
                    rowoff(m, C.m_in, C.sm1, C.sm0) +
                    rowoff(nc, C.n_in, C.sn1, C.sn0);
      const double v = acc[i][j];
      if (J.mode == EPI_STORE) {
        *dst = v;
      } else if (J.mode == EPI_ATOMIC) {
        unsigned long long *fx = P.fx[C.buf];
        if (fx)
          fx_add(fx + 2 * (dst - P.p[C.buf]), v);
        else
          atomicAdd(dst, v);
      } else {  // EPI_TAU: m = c, n = a * nv + b
        const double *ev = P.p[B_EPSV];
        const int nvv = C.n_in;
        const double eps = ev[m] + ev[nc / nvv] + ev[nc % nvv] - J.eo;
        *dst = (*dst + v) / (J.w - eps);
      }
    }
  }
}

int upload_plan(const Plan &p, DevPlan *d, cudaStream_t s) {
  free_plan(d);
  d->njobs = (int)p.jobs.size();
  d->tiles = p.tiles;
  if (d->njobs == 0) return CC3_OK;
  if (cudaMalloc(&d->jobs, sizeof(Job) * p.jobs.size()) != cudaSuccess)
    return CC3_ERR_OOM;
  if (cudaMalloc(&d->terms, sizeof(Term) * (p.terms.size() + 1)) != cudaSuccess)
    return CC3_ERR_OOM;
  if (cudaMemcpyAsync(d->jobs, p.jobs.data(), sizeof(Job) * p.jobs.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CC3_ERR_CUDA;
  if (!p.terms.empty() &&
      cudaMemcpyAsync(d->terms, p.terms.data(), sizeof(Term) * p.terms.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CC3_ERR_CUDA;
  // the host vectors may die after return: make the copies complete
  if (cudaStreamSynchronize(s) != cudaSuccess) return CC3_ERR_CUDA;
  return CC3_OK;
}

void free_plan(DevPlan *d) {
  if (d->jobs) cudaFree(d->jobs);
  if (d->terms) cudaFree(d->terms);
  d->jobs = nullptr;
  d->terms = nullptr;
  d->njobs = 0;
  d->tiles = 0;
}

int launch_plan(const DevPlan &d, const PtrTable &ptrs, cudaStream_t s,
                long long *launches) {
  if (d.njobs == 0 || d.tiles == 0) return CC3_OK;
  if (d.tiles > 0x7fffffffLL) return CC3_ERR_ARG;
  dim3 grid((unsigned)d.tiles);
  if (d.tile_kind == 0)
    fp64_engine_kernel<64, 64, 4, 4, 16><<<grid, 256, 0, s>>>(d.jobs, d.njobs,
                                                               d.terms, ptrs);
  else
    fp64_engine_kernel<256, 4, 4, 1, 16><<<grid, 256, 0, s>>>(d.jobs, d.njobs,
                                                              d.terms, ptrs);
  if (launches) ++*launches;
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

}  // namespace cc3
