// Vector kernels of the stationary (O)RAS solver (Eq. algRAS):
//     u <- u + M^{-1} r ,   r = f - A u ,   stop when ||r||_2 <= tol ||f||_2.
// The preconditioner and the residual reuse the solve and operator kernels; what is left is
// the update u += z and a deterministic 2-norm (fixed block partition, block partials
// added in block order by one block).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int ST_THREADS = 256;

__global__ void __launch_bounds__(ST_THREADS) axpy_kernel(double* __restrict__ u, const double* __restrict__ z,
                                                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)ST_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * ST_THREADS)
    u[i] += z[i];
}

// Block b sums x[i]^2 over its contiguous chunk; partial[b] = that sum.
__global__ void __launch_bounds__(ST_THREADS) sq_partial_kernel(const double* __restrict__ x, int64_t n,
                                                                double* __restrict__ partial) {
  __shared__ double ws[ST_THREADS / 32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  double s = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += ST_THREADS) s += x[i] * x[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < ST_THREADS / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// One thread adds the block partials in order: out = sqrt(sum).
__global__ void norm_finish_kernel(const double* __restrict__ partial, int nblk, double* out) {
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += partial[b];
  *out = sqrt(t);
}

// y = a x + b y (b == 0: y = a x, without reading y)
__global__ void __launch_bounds__(ST_THREADS) axpby_kernel(int64_t n, double a, const double* __restrict__ x,
                                                           double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)ST_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * ST_THREADS)
    y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, int nblk, cudaStream_t s) {
  axpby_kernel<<<nblk, ST_THREADS, 0, s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* u, const double* z, int64_t n, int nblk, cudaStream_t s) {
  axpy_kernel<<<nblk, ST_THREADS, 0, s>>>(u, z, n);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const double* x, int64_t n, double* partial, int nblk, double* out, cudaStream_t s) {
  sq_partial_kernel<<<nblk, ST_THREADS, 0, s>>>(x, n, partial);
  norm_finish_kernel<<<1, 1, 0, s>>>(partial, nblk, out);
  return cudaGetLastError();
}

}  // namespace cpmdev
