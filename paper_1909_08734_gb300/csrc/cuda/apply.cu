// Matrix-free stabilised CPM operator y = A x (Eq. impLapBel), FP64.
//
//   v_k = sum_{a,b} wx_a wy_b ( sum_c wz_c x[pencil_k(a,b) + c] )   for every band node k
//   y_i = (c + 6/h^2) x_i - (1/h^2) sum_{m=0..5} v_{nbr(i,m)}       for every active i
//
// The (p+1)^3 interpolation stencil of node k is stored as (p+1)^2 z-pencils: the canonical
// (i,j,k)-lexicographic order puts the p+1 nodes of a pencil at consecutive indices, so a
// pencil is one start index.
//
// Two extension kernels compute the v_k.  ext_values_kernel reads the 1-D weights only: four
// lanes per band node, lane a summing its x-slab wx_a sum_b wy_b sum_c wz_c x[...], then a
// two-step lane reduction.  ext_values_tw_kernel (used when the tensor weights wy_b wz_c are
// resident) gives each node one thread that forms sum_a wx_a sum_{b,c} (wy_b wz_c) x[...]:
// P^3 + P FP64 multiply-adds per node against P^3 + P^2 + P plus the lane reduction.  FP64
// instructions, not bytes, bound this apply on this GPU (two FP64 lanes per SM and clock).
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

__device__ __forceinline__ bool skip_iteration(const int* done) { return done && *done; }

// 4 lanes per band node; lane a < P sums its x-slab: wx_a sum_b wy_b sum_c wz_c x[...]
template <int P>
__global__ void __launch_bounds__(256) ext_values_kernel(const int32_t* __restrict__ pencil,
                                                         const double* __restrict__ wts,
                                                         IndirectVec x, double* __restrict__ v,
                                                         int64_t n_nodes, int64_t n_active,
                                                         const int* done) {
  if (skip_iteration(done)) return;
  const double* xv = x.ptr(blockIdx.y);
  double* vv = v + (int64_t)blockIdx.y * n_nodes;
  const int a = threadIdx.x & 3;
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  double part = 0.0;
  if (k < n_nodes && a < P) {
    const double* w = wts + k * 3 * P;
    const int32_t* pk = pencil + k * (P * P) + a * P;
    double wz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) wz[c] = __ldg(w + 2 * P + c);
    double t = 0.0;
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const int32_t st = __ldg(pk + b);
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < P; ++c) s += wz[c] * __ldg(xv + st + c);
      t += __ldg(w + P + b) * s;
    }
    part = __ldg(w + a) * t;
  }
  part += __shfl_xor_sync(0xffffffffu, part, 1, 4);
  part += __shfl_xor_sync(0xffffffffu, part, 2, 4);
  if (k < n_nodes && a == 0) vv[k] = part;
}

// one thread per band node; the x-slab sums use the tensor weights wy_b wz_c
template <int P>
__global__ void __launch_bounds__(256) ext_values_tw_kernel(const int32_t* __restrict__ pencil,
                                                            const double* __restrict__ wt2, IndirectVec x,
                                                            double* __restrict__ v, int64_t n_nodes,
                                                            const int* done) {
  if (skip_iteration(done)) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_nodes) return;
  const double* xv = x.ptr(blockIdx.y);
  int32_t pen[P * P];
  if constexpr (P == 4) {
    const int4* p4 = reinterpret_cast<const int4*>(pencil + k * 16);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int4 t = __ldg(p4 + j);
      pen[4 * j] = t.x;
      pen[4 * j + 1] = t.y;
      pen[4 * j + 2] = t.z;
      pen[4 * j + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < P * P; ++j) pen[j] = __ldg(pencil + k * (P * P) + j);
  }
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < P; ++a) {
    double xs[P * P];
#pragma unroll
    for (int b = 0; b < P; ++b)
#pragma unroll
      for (int c = 0; c < P; ++c) xs[b * P + c] = xv[pen[a * P + b] + c];
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < P * P; ++e) s = fma(__ldg(wt2 + (int64_t)e * n_nodes + k), xs[e], s);
    acc = fma(__ldg(wt2 + (int64_t)(P * P + a) * n_nodes + k), s, acc);
  }
  v[(int64_t)blockIdx.y * n_nodes + k] = acc;
}

template <int P>
__global__ void build_tw_kernel(const double* __restrict__ wts, double* __restrict__ wt2, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* w = wts + k * 3 * P;
#pragma unroll
  for (int b = 0; b < P; ++b)
#pragma unroll
    for (int c = 0; c < P; ++c) wt2[(int64_t)(b * P + c) * n + k] = w[P + b] * w[2 * P + c];
#pragma unroll
  for (int a = 0; a < P; ++a) wt2[(int64_t)(P * P + a) * n + k] = w[a];
}

cudaError_t launch_build_tensor_weights(const double* wts, double* wt2, int64_t n, int P, cudaStream_t s) {
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (P == 4) build_tw_kernel<4><<<nb, 256, 0, s>>>(wts, wt2, n);
  else build_tw_kernel<3><<<nb, 256, 0, s>>>(wts, wt2, n);
  return cudaGetLastError();
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

cudaError_t launch_ext_values(const OperatorDev& op, IndirectVec x, double* v_scratch, int nrhs, const int* done,
                              cudaStream_t s) {
  const int64_t n = op.n_nodes;
  if (op.wt2) {
    dim3 gt((unsigned)((n + 255) / 256), nrhs);
    if (op.P == 4)
      ext_values_tw_kernel<4><<<gt, 256, 0, s>>>(op.pencil, op.wt2, x, v_scratch, n, done);
    else
      ext_values_tw_kernel<3><<<gt, 256, 0, s>>>(op.pencil, op.wt2, x, v_scratch, n, done);
    return cudaGetLastError();
  }
  dim3 g1((unsigned)((n * 4 + 255) / 256), nrhs);
  if (op.P == 4)
    ext_values_kernel<4><<<g1, 256, 0, s>>>(op.pencil, op.wts, x, v_scratch, n, op.n_active, done);
  else
    ext_values_kernel<3><<<g1, 256, 0, s>>>(op.pencil, op.wts, x, v_scratch, n, op.n_active, done);
  return cudaGetLastError();
}

cudaError_t launch_apply(const OperatorDev& op, IndirectVec x, double* v_scratch, const double* f,
                         IndirectVec y, int nrhs, int mode, const int* done, cudaStream_t s) {
  const int64_t n = op.n_nodes;
  cudaError_t e = launch_ext_values(op, x, v_scratch, nrhs, done, s);
  if (e != cudaSuccess) return e;
  dim3 g2((unsigned)((op.n_active + 255) / 256), nrhs);
  nbr_sum_kernel<<<g2, 256, 0, s>>>(op.nbr, x, v_scratch, f, y, op.n_active, n, op.diag, op.invh2,
                                    mode, done);
  return cudaGetLastError();
}

}  // namespace cpmdev
