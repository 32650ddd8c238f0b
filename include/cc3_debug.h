/*
 * cc3_debug.h -- diagnostic entry points of libcc3 (not part of the hot path).
 *
 * cc3_debug_split_gemm runs ONE plain contraction C[m][n] = sum_k A[m][k] B[n][k]
 * (row-major float64 host arrays A[M][K], B[N][K], C[M][N]) through the split
 * precision tensor-core engine that the CC3 triples kernels use: both operands
 * are cut into `slices` integer-valued BF16 slices with one power-of-two scale
 * each, the slice-product triangle runs on tcgen05 tensor cores with exact
 * FP32 accumulation of the leading levels, and the result is recombined in
 * double-float and accumulated in FP64.  It exists to test the engine in
 * isolation against a plain FP64 product.  Allocates and frees its own device
 * memory; synchronous; returns a cc3 status (CC3_ERR_ARG for sizes < 1 or
 * slices outside 3..7).
 */
#ifndef CC3_DEBUG_H
#define CC3_DEBUG_H
#ifdef __cplusplus
extern "C" {
#endif
int cc3_debug_split_gemm(int M, int N, int K, const double *A, const double *B, double *C,
                         int slices);

/* Runs one bounded device wait that cannot succeed (one thread of one CTA
 * waits on an mbarrier nothing arrives on, nothing else in flight) with a
 * limit of limit_s seconds (1e-6 <= limit_s <= 1), the same bounded-wait
 * primitive every spin of the library's kernels uses.  Returns
 * CC3_ERR_TIMEOUT once the kernel has recorded the give-up in its status word
 * and returned (the CUDA context stays usable), CC3_ERR_ARG for a limit out
 * of range.  Synchronous, on the legacy default stream of the current device.
 * Exists to test the failure path without a GPU fault. */
int cc3_debug_wait_timeout(double limit_s);
#ifdef __cplusplus
}
#endif
#endif
