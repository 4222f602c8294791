// Device-resident right-preconditioned flexible GMRES(m) with CGS2 (Sec. 2.2: the (O)RAS
// preconditioner inside GMRES).  All Arnoldi arithmetic is FP64.
//
// Reductions are deterministic: every block writes its partial sums, and the last block to
// finish (ticket counter) adds the partials in block order.  The step index k, the
// cycle-done flag and the status live in device memory, so one captured CUDA graph of an
// iteration replays for every k; every kernel of an iteration returns at once when the
// cycle is already done.  One Arnoldi step after z_k = M^{-1} v_k and w = A z_k is four
// kernels:
//   dots    : h1 = V_k^T w                                   (first Gram-Schmidt pass)
//   update1 : w -= V_k h1 ;  h2 = V_k^T w                    (second pass)
//   update2 : w -= V_k h2 ;  ||w||, Hessenberg column, Givens rotation, stopping test
//   scale   : v_{k+1} = w / ||w|| ;  k += 1
#include <math.h>

#include "../../../include/cpm.h"
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int KT = 256;                 // threads per block of the vector kernels
constexpr int KW = KT / 32;
constexpr int ILP = 8;                  // basis vectors processed together

// int state
enum { I_K = 0, I_TOTAL = 1, I_DONE = 2, I_STATUS = 3, I_KDONE = 4, I_MAXIT = 5,
       I_TICKET = 8 };                  // tickets 8..11, one per reducing kernel
constexpr int RUNNING = -1;

// double state layout for restart length m
struct SL {
  int m;
  __host__ __device__ int H(int i, int k) const { return i + k * (m + 1); }
  __host__ __device__ int cs() const { return (m + 1) * m; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int y() const { return g() + m + 1; }
  __host__ __device__ int h1() const { return y() + m; }
  __host__ __device__ int h2() const { return h1() + m + 1; }
  __host__ __device__ int sc() const { return h2() + m + 1; }   // scalars
};
enum { S_NF = 0, S_TOL = 1, S_BETA = 2, S_HN = 3, S_RELRES = 4 };

__device__ __forceinline__ bool cycle_done(const GmresDev& g) {
  return *(volatile const int*)&g.ist[I_DONE] != 0;
}

__device__ __forceinline__ void block_rows(const GmresDev& g, int64_t* r0, int64_t* r1) {
  const int64_t chunk = (g.n + g.nblk - 1) / g.nblk;
  *r0 = blockIdx.x * chunk;
  *r1 = min(g.n, *r0 + chunk);
}

// Block partial sums s[i] (i < cnt, held in shared memory wp[KW][...]) -> part[b][i].
// Then the last block adds all blocks' partials in a fixed order into out[i].  Returns true
// in the last block (after out[] is written and visible to that block).
__device__ bool finish_reduction(const GmresDev& g, double (*wp)[130], int cnt, int ticket,
                                 double* out) {
  __shared__ bool last;
  __shared__ double gsum[1][130];
  for (int i = threadIdx.x; i < cnt; i += KT) {
    double s = 0.0;
    for (int w = 0; w < KW; ++w) s += wp[w][i];
    g.part[(int64_t)blockIdx.x * (g.m + 2) + i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&g.ist[ticket], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // warp w adds value i = w, w + KW, ...: lane l takes blocks l, l + 32, ... (loads issued
  // together), then a shuffle tree adds the lanes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ld = g.m + 2;
  for (int i = warp; i < cnt; i += KW) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int b = lane + 32 * u;
      v[u] = b < g.nblk ? __ldcg(g.part + (int64_t)b * ld + i) : 0.0;
    }
    double sum = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += v[u];
    for (int b = lane + 256; b < g.nblk; b += 32) sum += __ldcg(g.part + (int64_t)b * ld + i);
    sum = warp_sum(sum);
    if (lane == 0) gsum[0][i] = sum;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cnt; t += KT) out[t] = gsum[0][t];
  if (threadIdx.x == 0) g.ist[ticket] = 0;
  __syncthreads();
  return true;
}

constexpr int RU = 4;                   // rows per thread processed together (loads in flight)

// wp[warp][i] = this warp's share of sum_rows V[i][row] w[row], i <= k, own rows
__device__ __forceinline__ void block_dots(const GmresDev& g, int k, int64_t r0, int64_t r1,
                                           double (*wp)[130]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= k; i0 += ILP) {
    double acc[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) acc[u] = 0.0;
    for (int64_t base = r0 + threadIdx.x; base < r1; base += RU * KT) {
      double wv[RU], vv[RU][ILP];
#pragma unroll
      for (int q = 0; q < RU; ++q) {
        const int64_t row = base + (int64_t)q * KT;
        wv[q] = row < r1 ? g.w[row] : 0.0;
#pragma unroll
        for (int u = 0; u < ILP; ++u)
          vv[q][u] = (row < r1 && i0 + u <= k) ? g.V[(int64_t)(i0 + u) * g.n + row] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < RU; ++q)
#pragma unroll
        for (int u = 0; u < ILP; ++u) acc[u] += vv[q][u] * wv[q];
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
      const double sum = warp_sum(acc[u]);
      if (lane == 0 && i0 + u <= k) wp[warp][i0 + u] = sum;
    }
  }
}

// w = A z_k on this block's rows (the operator's second half, the same arithmetic as
// nbr_sum_kernel), then h1 = V_k^T w
__global__ void __launch_bounds__(KT) dots_kernel(GmresDev g, const int32_t* __restrict__ nbr, IndirectVec z,
                                                  const double* __restrict__ vext, double diag, double invh2) {
  if (cycle_done(g)) return;
  __shared__ double wp[KW][130];
  const int k = g.ist[I_K];
  int64_t r0, r1;
  block_rows(g, &r0, &r1);
  const double* zk = z.ptr(0);
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
    const int32_t* nb = nbr + 6 * row;
    double sn = 0.0;
#pragma unroll
    for (int m = 0; m < 6; ++m) sn += vext[__ldg(nb + m)];
    g.w[row] = diag * zk[row] - invh2 * sn;
  }
  block_dots(g, k, r0, r1, wp);
  __syncthreads();
  const SL L{g.m};
  finish_reduction(g, wp, k + 1, I_TICKET + 0, g.st + L.h1());
}

// w -= V_k h (h at st[h_off]); then either dots with the new w (into h2) or ||w||^2 with
// the Hessenberg / Givens update in the last block.
__global__ void __launch_bounds__(KT) update_kernel(GmresDev g, int h_off, int dots) {
  if (cycle_done(g)) return;
  __shared__ double hs[130];
  __shared__ double wp[KW][130];
  __shared__ double total[130];
  const int k = g.ist[I_K];
  for (int i = threadIdx.x; i <= k; i += KT) hs[i] = g.st[h_off + i];
  __syncthreads();
  int64_t r0, r1;
  block_rows(g, &r0, &r1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = r0 + threadIdx.x; base < r1; base += RU * KT) {
    double a[RU][ILP];
#pragma unroll
    for (int q = 0; q < RU; ++q)
#pragma unroll
      for (int u = 0; u < ILP; ++u) a[q][u] = 0.0;
    for (int i0 = 0; i0 <= k; i0 += ILP) {
      double vv[RU][ILP];
#pragma unroll
      for (int q = 0; q < RU; ++q) {
        const int64_t row = base + (int64_t)q * KT;
#pragma unroll
        for (int u = 0; u < ILP; ++u)
          vv[q][u] = (row < r1 && i0 + u <= k) ? g.V[(int64_t)(i0 + u) * g.n + row] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < RU; ++q)
#pragma unroll
        for (int u = 0; u < ILP; ++u) a[q][u] += vv[q][u] * hs[min(i0 + u, k)];
    }
#pragma unroll
    for (int q = 0; q < RU; ++q) {
      const int64_t row = base + (int64_t)q * KT;
      double sum = 0.0;
#pragma unroll
      for (int u = 0; u < ILP; ++u) sum += a[q][u];
      if (row < r1) g.w[row] -= sum;
    }
  }
  const SL L{g.m};
  if (dots) {
    __syncthreads();
    block_dots(g, k, r0, r1, wp);
    __syncthreads();
    finish_reduction(g, wp, k + 1, I_TICKET + 1, g.st + L.h2());
    return;
  }
  double s = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) s += g.w[row] * g.w[row];
  s = warp_sum(s);
  if (lane == 0) wp[warp][0] = s;
  __syncthreads();
  if (!finish_reduction(g, wp, 1, I_TICKET + 2, total)) return;
  if (threadIdx.x != 0) return;
  // Hessenberg column k, previous rotations, new rotation, residual estimate
  double* st = g.st;
  int* ist = g.ist;
  const double hn = sqrt(total[0]);
  for (int i = 0; i <= k; ++i) st[L.H(i, k)] = st[L.h1() + i] + st[L.h2() + i];
  st[L.H(k + 1, k)] = hn;
  for (int i = 0; i < k; ++i) {
    const double c = st[L.cs() + i], sv = st[L.sn() + i];
    const double a = st[L.H(i, k)], b = st[L.H(i + 1, k)];
    st[L.H(i, k)] = c * a + sv * b;
    st[L.H(i + 1, k)] = -sv * a + c * b;
  }
  const double a = st[L.H(k, k)], b = st[L.H(k + 1, k)];
  const double rho = sqrt(a * a + b * b);
  const double c = a / rho, sv = b / rho;
  st[L.cs() + k] = c;
  st[L.sn() + k] = sv;
  st[L.H(k, k)] = rho;
  st[L.H(k + 1, k)] = 0.0;
  const double gk = st[L.g() + k];
  st[L.g() + k + 1] = -sv * gk;
  st[L.g() + k] = c * gk;
  st[L.sc() + S_HN] = hn;
  ist[I_TOTAL] += 1;
  ist[I_KDONE] = k + 1;
  const double est = fabs(st[L.g() + k + 1]);
  const double nf = st[L.sc() + S_NF], tol = st[L.sc() + S_TOL];
  bool stop = est <= tol * nf || hn == 0.0 || k + 1 >= g.m || ist[I_TOTAL] >= ist[I_MAXIT];
  if (!isfinite(hn) || !isfinite(rho) || !isfinite(est)) {
    ist[I_STATUS] = CPM_ERR_NAN;
    stop = true;
  }
  if (stop) ist[I_DONE] = 1;
}

// v_{k+1} = w / ||w||, then the last block advances k
__global__ void __launch_bounds__(KT) scale_kernel(GmresDev g) {
  if (cycle_done(g)) return;
  __shared__ bool last;
  const SL L{g.m};
  const int k = g.ist[I_K];
  const double inv = 1.0 / g.st[L.sc() + S_HN];
  double* dst = g.V + (int64_t)(k + 1) * g.n;
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT)
    dst[row] = g.w[row] * inv;
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(&g.ist[I_TICKET + 3], 1) == (int)gridDim.x - 1;
    if (last) {
      g.ist[I_TICKET + 3] = 0;
      g.ist[I_K] = k + 1;
    }
  }
}

// ---- cycle start / restart ------------------------------------------------------------
// ||x||^2 over all blocks; the last block applies the begin (which = 0: ||f||) or the
// convergence test on beta = ||r|| (which = 1).
__global__ void __launch_bounds__(KT) norm_begin_kernel(GmresDev g, const double* x, double tol,
                                                        int max_it, int which) {
  __shared__ double wp[KW][130];
  __shared__ double total[130];
  int64_t r0, r1;
  block_rows(g, &r0, &r1);
  double s = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) s += x[row] * x[row];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5][0] = s;
  __syncthreads();
  if (!finish_reduction(g, wp, 1, I_TICKET + 3, total)) return;
  if (threadIdx.x != 0) return;
  const SL L{g.m};
  const double nrm = sqrt(total[0]);
  if (which == 0) {               // ||f||
    g.st[L.sc() + S_NF] = nrm;
    g.st[L.sc() + S_TOL] = tol;
    g.ist[I_MAXIT] = max_it;
    g.ist[I_TOTAL] = 0;
    g.ist[I_STATUS] = RUNNING;
    return;
  }
  const double beta = nrm;
  const double nf = g.st[L.sc() + S_NF];
  g.st[L.sc() + S_BETA] = beta;
  g.st[L.sc() + S_RELRES] = nf > 0.0 ? beta / nf : 0.0;
  if (g.ist[I_STATUS] != RUNNING) { g.ist[I_DONE] = 1; return; }
  if (!isfinite(beta)) {
    g.ist[I_STATUS] = CPM_ERR_NAN;
  } else if (nf == 0.0 || beta <= g.st[L.sc() + S_TOL] * nf) {
    g.ist[I_STATUS] = CPM_OK;
  } else if (g.ist[I_TOTAL] >= g.ist[I_MAXIT]) {
    g.ist[I_STATUS] = CPM_ERR_NOT_CONVERGED;
  } else if (g.ist[I_TOTAL] > 0 && g.st[L.sc() + S_HN] == 0.0) {
    g.ist[I_STATUS] = CPM_ERR_BREAKDOWN;
  }
  if (g.ist[I_STATUS] != RUNNING) { g.ist[I_DONE] = 1; return; }
  for (int i = 0; i <= g.m; ++i) g.st[L.g() + i] = 0.0;
  g.st[L.g()] = beta;
  g.ist[I_K] = 0;
  g.ist[I_KDONE] = 0;
  g.ist[I_DONE] = 0;
}

// V[0] = r / beta when a new cycle starts
__global__ void __launch_bounds__(KT) start_basis_kernel(GmresDev g) {
  if (cycle_done(g)) return;
  const SL L{g.m};
  const double inv = 1.0 / g.st[L.sc() + S_BETA];
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT)
    g.V[row] = g.r[row] * inv;
}

// y = H[:kd,:kd]^{-1} g[:kd] by one warp (back substitution), then u += Z y
__global__ void ysolve_kernel(GmresDev g) {
  const SL L{g.m};
  __shared__ double ys[129];
  const int kd = g.ist[I_KDONE];
  for (int i = threadIdx.x; i < kd; i += 32) ys[i] = g.st[L.g() + i];
  __syncwarp();
  for (int i = kd - 1; i >= 0; --i) {
    double s = 0.0;
    for (int q = i + 1 + threadIdx.x; q < kd; q += 32) s += g.st[L.H(i, q)] * ys[q];
    s = warp_sum(s);
    if (threadIdx.x == 0) ys[i] = (ys[i] - s) / g.st[L.H(i, i)];
    __syncwarp();
  }
  for (int i = threadIdx.x; i < kd; i += 32) g.st[L.y() + i] = ys[i];
}

__global__ void __launch_bounds__(KT) xupdate_kernel(GmresDev g, double* u) {
  const SL L{g.m};
  const int kd = g.ist[I_KDONE];
  __shared__ double ys[128];
  for (int i = threadIdx.x; i < kd; i += KT) ys[i] = g.st[L.y() + i];
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT) {
    double a[ILP];
#pragma unroll
    for (int u2 = 0; u2 < ILP; ++u2) a[u2] = 0.0;
    for (int i0 = 0; i0 < kd; i0 += ILP)
#pragma unroll
      for (int u2 = 0; u2 < ILP; ++u2)
        if (i0 + u2 < kd) a[u2] += g.Z[(int64_t)(i0 + u2) * g.n + row] * ys[i0 + u2];
    double s = 0.0;
#pragma unroll
    for (int u2 = 0; u2 < ILP; ++u2) s += a[u2];
    u[row] += s;
  }
}

int gmres_state_size(int m) { return SL{m}.sc() + 8; }
int gmres_scalar_offset(int m) { return SL{m}.sc(); }

static unsigned vec_blocks(int64_t n) {
  int64_t b = (n + KT - 1) / KT;
  return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

cudaError_t launch_gmres_begin(const GmresDev& g, const double* f, double tol, int max_it,
                               cudaStream_t s) {
  norm_begin_kernel<<<g.nblk, KT, 0, s>>>(g, f, tol, max_it, 0);
  return cudaGetLastError();
}

cudaError_t launch_cgs2_and_givens(const GmresDev& g, const OperatorDev& op, IndirectVec z, const double* vext,
                                   cudaStream_t s) {
  const SL L{g.m};
  dots_kernel<<<g.nblk, KT, 0, s>>>(g, op.nbr, z, vext, op.diag, op.invh2);
  update_kernel<<<g.nblk, KT, 0, s>>>(g, L.h1(), 1);
  update_kernel<<<g.nblk, KT, 0, s>>>(g, L.h2(), 0);
  scale_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_gmres_restart_update(const GmresDev& g, double* u, cudaStream_t s) {
  ysolve_kernel<<<1, 32, 0, s>>>(g);
  xupdate_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g, u);
  return cudaGetLastError();
}

// after r = f - A u: beta, convergence decision, and V[0] = r / beta for the next cycle
cudaError_t launch_gmres_residual_check(const GmresDev& g, cudaStream_t s) {
  norm_begin_kernel<<<g.nblk, KT, 0, s>>>(g, g.r, 0.0, 0, 1);
  start_basis_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace cpmdev
