// FP64 fused multiply-add probes: the denominator of the FP64-ALU rooflines this library
// reports, and the latency of a dependent FP64 chain (what a serial reduction pays per step).
//   throughput: every thread advances `chains` independent chains x <- x a + b for `iters`
//               steps; FLOP = 2 x threads x chains x iters over the kernel's event time.
//   latency   : one thread advances one chain; clock cycles per step from clock64().
// a = 1 - 2^-30 and b = 2^-40 keep every chain bounded and free of subnormals.
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

template <int CH>
__global__ void fma_throughput_kernel(double* out, int iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = 1.0 + 1e-9 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == 12345.678) out[blockIdx.x] = s;      // never true: keeps the chains alive
}

__global__ void fma_latency_kernel(double* out, long long* cycles, int iters, double a, double b) {
  double x = 1.0 + 1e-9 * threadIdx.x;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) x = fma(x, a, b);
  const long long t1 = clock64();
  out[0] = x;
  cycles[0] = t1 - t0;
}

cudaError_t launch_fma_throughput(int blocks, int threads, int chains, int iters, double* out, cudaStream_t s) {
  const double a = 1.0 - 0x1p-30, b = 0x1p-40;
  switch (chains) {
    case 1: fma_throughput_kernel<1><<<blocks, threads, 0, s>>>(out, iters, a, b); break;
    case 2: fma_throughput_kernel<2><<<blocks, threads, 0, s>>>(out, iters, a, b); break;
    case 4: fma_throughput_kernel<4><<<blocks, threads, 0, s>>>(out, iters, a, b); break;
    case 8: fma_throughput_kernel<8><<<blocks, threads, 0, s>>>(out, iters, a, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fma_latency(int iters, double* out, long long* cycles, cudaStream_t s) {
  fma_latency_kernel<<<1, 1, 0, s>>>(out, cycles, iters, 1.0 - 0x1p-30, 0x1p-40);
  return cudaGetLastError();
}

}  // namespace cpmdev
