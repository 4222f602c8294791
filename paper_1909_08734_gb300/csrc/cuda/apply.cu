// Matrix-free stabilised CPM operator y = A x (Eq. impLapBel), FP64.
//
//   v_k = sum_{a,b} wx_a wy_b ( sum_c wz_c x[pencil_k(a,b) + c] )   for every band node k
//   y_i = (c + 6/h^2) x_i - (1/h^2) sum_{m=0..5} v_{nbr(i,m)}       for every active i
//
// The (p+1)^3 interpolation stencil of node k is stored as (p+1)^2 z-pencils: the canonical
// (i,j,k)-lexicographic order puts the p+1 nodes of a pencil at consecutive indices, so a
// pencil is one start index.  16 lanes cooperate on one row (one lane per pencil).
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

__device__ __forceinline__ bool skip_iteration(const int* done) { return done && *done; }

template <int P>
__global__ void __launch_bounds__(256) ext_values_kernel(const int32_t* __restrict__ pencil,
                                                         const double* __restrict__ wts,
                                                         IndirectVec x, double* __restrict__ v,
                                                         int64_t n_nodes, int64_t n_active,
                                                         const int* done) {
  if (skip_iteration(done)) return;
  const double* xv = x.ptr(blockIdx.y);
  double* vv = v + (int64_t)blockIdx.y * n_nodes;
  const int lane = threadIdx.x & 15;
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  double part = 0.0;
  if (k < n_nodes && lane < P * P) {
    const int a = lane / P, b = lane % P;
    const double* w = wts + k * 3 * P;
    const int32_t st = __ldg(pencil + k * (P * P) + lane);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < P; ++c) s += __ldg(w + 2 * P + c) * __ldg(xv + st + c);
    part = (__ldg(w + a) * __ldg(w + P + b)) * s;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, 16);
  if (k < n_nodes && lane == 0) vv[k] = part;
}

// mode 0: y = A x;  mode 1: y = f - A x
__global__ void __launch_bounds__(256) nbr_sum_kernel(const int32_t* __restrict__ nbr,
                                                      IndirectVec x, const double* __restrict__ v,
                                                      const double* __restrict__ f, IndirectVec y,
                                                      int64_t n_active, int64_t n_nodes,
                                                      double diag, double invh2, int mode,
                                                      const int* done) {
  if (skip_iteration(done)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_active) return;
  const double* xv = x.ptr(blockIdx.y);
  const double* vv = v + (int64_t)blockIdx.y * n_nodes;
  const int32_t* nb = nbr + 6 * i;
  double s = 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) s += vv[__ldg(nb + m)];
  double ax = diag * xv[i] - invh2 * s;
  double* yv = y.ptr(blockIdx.y);
  yv[i] = mode ? f[(int64_t)blockIdx.y * n_active + i] - ax : ax;
}

cudaError_t launch_apply(const OperatorDev& op, IndirectVec x, double* v_scratch, const double* f,
                         IndirectVec y, int nrhs, int mode, const int* done, cudaStream_t s) {
  const int64_t n = op.n_nodes;
  dim3 g1((unsigned)((n * 16 + 255) / 256), nrhs);
  if (op.P == 4)
    ext_values_kernel<4><<<g1, 256, 0, s>>>(op.pencil, op.wts, x, v_scratch, n, op.n_active, done);
  else
    ext_values_kernel<3><<<g1, 256, 0, s>>>(op.pencil, op.wts, x, v_scratch, n, op.n_active, done);
  dim3 g2((unsigned)((op.n_active + 255) / 256), nrhs);
  nbr_sum_kernel<<<g2, 256, 0, s>>>(op.nbr, x, v_scratch, f, y, op.n_active, n, op.diag, op.invh2,
                                    mode, done);
  return cudaGetLastError();
}

}  // namespace cpmdev
