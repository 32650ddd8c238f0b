// Element-wise and reduction kernels of the FP64 path.
#include <cuda_runtime.h>

#include <algorithm>

#include "cc3_internal.h"

namespace cc3 {

// tau~^{abc} = 4 tau^{abc} - 2 tau^{acb} - 2 tau^{cba} - 2 tau^{bac}
//              + tau^{bca} + tau^{cab}        (Algorithm 1, i,j,k fixed)
// input tau stored as T[c][a][b], output tau~ as TT[a][b][c]; one slot per
// triple in the batch (blockIdx.y).
__global__ void contravariant_kernel(const double *__restrict__ tau,
                                     double *__restrict__ tt, int nv) {
  const long long nv2 = (long long)nv * nv, nv3 = nv2 * nv;
  const double *T = tau + blockIdx.y * nv3;
  double *O = tt + blockIdx.y * nv3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv3;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % nv);
    const int b = (int)((e / nv) % nv);
    const int a = (int)(e / nv2);
    // tau(x,y,z) = T[z][x][y]
#define TAU(x, y, z) T[(long long)(z) * nv2 + (long long)(x) * nv + (y)]
    O[e] = 4.0 * TAU(a, b, c) - 2.0 * TAU(a, c, b) - 2.0 * TAU(c, b, a) -
           2.0 * TAU(b, a, c) + TAU(b, c, a) + TAU(c, a, b);
#undef TAU
  }
}

int launch_contravariant(const double *tau_cab, double *tt_abc, int nv,
                         int nslot, cudaStream_t s) {
  if (nslot <= 0) return CC3_OK;
  const long long nv3 = (long long)nv * nv * nv;
  int blocks = (int)std::min<long long>((nv3 + 255) / 256, 4096);
  dim3 grid(blocks, nslot);
  contravariant_kernel<<<grid, 256, 0, s>>>(tau_cab, tt_abc, nv);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

// Omega2^{ab}_{ij} = (1/3) P^{ab}_{ij} (2 X^{ab}_{ij} + X^{ba}_{ij}),
// P^{ab}_{ij} Y^{ab}_{ij} = Y^{ab}_{ij} + Y^{ba}_{ji}   (Algorithm 1, the back-transform)
__global__ void back_transform_kernel(const double *__restrict__ X,
                                      double *__restrict__ Om, int no, int nv) {
  const long long nv2 = (long long)nv * nv, n = (long long)no * no * nv2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % nv);
    const int a = (int)((e / nv) % nv);
    const int j = (int)((e / nv2) % no);
    const int i = (int)(e / (nv2 * no));
    auto at = [&](int p, int q, int x, int y) {
      return X[((long long)p * no + q) * nv2 + (long long)x * nv + y];
    };
    Om[e] = (2.0 * at(i, j, a, b) + at(i, j, b, a) + 2.0 * at(j, i, b, a) +
             at(j, i, a, b)) / 3.0;
  }
}

int launch_back_transform(const double *omt, double *om2, int no, int nv,
                          cudaStream_t s) {
  const long long n = (long long)no * no * nv * nv;
  if (n == 0) return CC3_OK;
  int blocks = (int)std::min<long long>((n + 255) / 256, 8192);
  back_transform_kernel<<<blocks, 256, 0, s>>>(omt, om2, no, nv);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

// E = sum t2 * Omega~ in a fixed order: 256 block partials, then one block.
__global__ void dot_partial_kernel(const double *__restrict__ x,
                                   const double *__restrict__ y, long long n,
                                   double *__restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s = fma(x[e], y[e], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void sum_kernel(const double *__restrict__ part, int n,
                           double *__restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += part[e];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

int launch_energy(const double *t2, const double *omt, double *E, int no,
                  int nv, cudaStream_t s) {
  // E[0] result, E[1..256] partials (caller provides 257 doubles)
  const long long n = (long long)no * no * nv * nv;
  dot_partial_kernel<<<256, 256, 0, s>>>(t2, omt, n, E + 1);
  sum_kernel<<<1, 256, 0, s>>>(E + 1, 256, E);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

// oovo[l][q][z][r] = ooov[l][q][r][z]
__global__ void ooov_to_oovo_kernel(const double *__restrict__ in,
                                    double *__restrict__ out, int no, int nv) {
  const long long n = (long long)no * no * no * nv;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % no);
    const int z = (int)((e / no) % nv);
    const long long lq = e / ((long long)no * nv);
    out[e] = in[(lq * no + r) * nv + z];
  }
}

int launch_transpose_ooov_to_oovo(const double *ooov, double *oovo, int no,
                                  int nv, cudaStream_t s) {
  const long long n = (long long)no * no * no * nv;
  if (n == 0) return CC3_OK;
  int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  ooov_to_oovo_kernel<<<blocks, 256, 0, s>>>(ooov, oovo, no, nv);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

__global__ void zero_kernel(double *p, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    p[e] = 0.0;
}

int launch_zero(double *p, size_t n, cudaStream_t s) {
  if (n == 0) return CC3_OK;
  int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
  zero_kernel<<<blocks, 256, 0, s>>>(p, n);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

__global__ void fx_to_double_kernel(const unsigned long long *__restrict__ fx,
                                    double *__restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long lo = fx[2 * i];
    const long long hi = (long long)fx[2 * i + 1];
    // value = hi + lo 2^-64 (lo unsigned)
    out[i] = (double)hi + ldexp((double)lo, -64);
  }
}

int launch_fx_to_double(const unsigned long long *fx, double *out, size_t n, cudaStream_t s) {
  if (n == 0) return CC3_OK;
  const size_t b = std::min<size_t>((n + 255) / 256, 8192);
  fx_to_double_kernel<<<(unsigned)b, 256, 0, s>>>(fx, out, n);
  return cudaGetLastError() == cudaSuccess ? CC3_OK : CC3_ERR_CUDA;
}

}  // namespace cc3
