// Device-resident right-preconditioned flexible GMRES(m) with CGS2 (Sec. 2.2: the (O)RAS
// preconditioner inside GMRES).  All Arnoldi arithmetic is FP64.  Reductions are two-stage
// (per-block partial sums in a fixed order, then a fixed-order sum over blocks), so results
// do not depend on scheduling.  The step index k, the cycle-done flag and the status live
// in device memory, so one captured CUDA graph of an iteration replays for every k; every
// kernel of an iteration returns at once when the cycle is already done.
#include <math.h>

#include "../../../include/cpm.h"
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int KT = 256;                 // threads per block of the vector kernels
constexpr int KW = KT / 32;

// int state
enum { I_K = 0, I_TOTAL = 1, I_DONE = 2, I_STATUS = 3, I_KDONE = 4, I_MAXIT = 5 };
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

// part[b * (m+2) + i] = sum over block b's rows of V_i[row] * w[row], i = 0..k
__global__ void __launch_bounds__(KT) mdot_kernel(GmresDev g) {
  if (cycle_done(g)) return;
  __shared__ double wp[KW][130];
  const int k = g.ist[I_K];
  const int64_t chunk = (g.n + g.nblk - 1) / g.nblk;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(g.n, r0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i <= k; ++i) {
    const double* Vi = g.V + (int64_t)i * g.n;
    double s = 0.0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) s += Vi[row] * g.w[row];
    s = warp_sum(s);
    if (lane == 0) wp[warp][i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= k; i += KT) {
    double s = 0.0;
    for (int w = 0; w < KW; ++w) s += wp[w][i];
    g.part[(int64_t)blockIdx.x * (g.m + 2) + i] = s;
  }
}

// out[i] = sum_b part[b][i] for i = 0..cnt-1 (cnt = k+1, or 1 for a norm)
__global__ void reduce_kernel(GmresDev g, int out_off, int norm_only) {
  if (cycle_done(g)) return;
  const int cnt = norm_only ? 1 : g.ist[I_K] + 1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < g.nblk; ++b) s += g.part[(int64_t)b * (g.m + 2) + i];
    g.st[out_off + i] = s;
  }
}

// w -= V h (i = 0..k); with dots: part[b][i] = sum V_i[row] * w_new[row];
// without: part[b][0] = sum w_new[row]^2
__global__ void __launch_bounds__(KT) cgs_update_kernel(GmresDev g, int h_off, int dots) {
  if (cycle_done(g)) return;
  __shared__ double hs[130];
  __shared__ double wp[KW][130];
  const int k = g.ist[I_K];
  for (int i = threadIdx.x; i <= k; i += KT) hs[i] = g.st[h_off + i];
  __syncthreads();
  const int64_t chunk = (g.n + g.nblk - 1) / g.nblk;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(g.n, r0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
    double w = g.w[row];
    for (int i = 0; i <= k; ++i) w -= g.V[(int64_t)i * g.n + row] * hs[i];
    g.w[row] = w;
  }
  __syncthreads();
  const int cnt = dots ? k + 1 : 1;
  for (int i = 0; i < cnt; ++i) {
    double s = 0.0;
    for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) {
      const double w = g.w[row];
      s += dots ? g.V[(int64_t)i * g.n + row] * w : w * w;
    }
    s = warp_sum(s);
    if (lane == 0) wp[warp][i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += KT) {
    double s = 0.0;
    for (int w = 0; w < KW; ++w) s += wp[w][i];
    g.part[(int64_t)blockIdx.x * (g.m + 2) + i] = s;
  }
}

// Hessenberg column, Givens rotations, residual estimate, stopping decision.
__global__ void givens_kernel(GmresDev g) {
  if (cycle_done(g) || threadIdx.x != 0) return;
  const SL L{g.m};
  double* st = g.st;
  int* ist = g.ist;
  const int k = ist[I_K];
  double ss = 0.0;
  for (int b = 0; b < g.nblk; ++b) ss += g.part[(int64_t)b * (g.m + 2)];
  const double hn = sqrt(ss);
  for (int i = 0; i <= k; ++i) st[L.H(i, k)] = st[L.h1() + i] + st[L.h2() + i];
  st[L.H(k + 1, k)] = hn;
  for (int i = 0; i < k; ++i) {
    const double c = st[L.cs() + i], s = st[L.sn() + i];
    const double a = st[L.H(i, k)], b = st[L.H(i + 1, k)];
    st[L.H(i, k)] = c * a + s * b;
    st[L.H(i + 1, k)] = -s * a + c * b;
  }
  const double a = st[L.H(k, k)], b = st[L.H(k + 1, k)];
  const double rho = sqrt(a * a + b * b);
  const double c = a / rho, s = b / rho;
  st[L.cs() + k] = c;
  st[L.sn() + k] = s;
  st[L.H(k, k)] = rho;
  st[L.H(k + 1, k)] = 0.0;
  const double gk = st[L.g() + k];
  st[L.g() + k + 1] = -s * gk;
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

// V[k+1] = w / ||w||
__global__ void __launch_bounds__(KT) scale_next_kernel(GmresDev g) {
  if (cycle_done(g)) return;
  const SL L{g.m};
  const int k = g.ist[I_K];
  const double inv = 1.0 / g.st[L.sc() + S_HN];
  double* dst = g.V + (int64_t)(k + 1) * g.n;
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT)
    dst[row] = g.w[row] * inv;
}

__global__ void advance_kernel(GmresDev g) {
  if (cycle_done(g)) return;
  g.ist[I_K] += 1;
}

// ---- cycle start / restart ------------------------------------------------------------
// part[b][0] = sum over block b of x[row]^2
__global__ void __launch_bounds__(KT) norm_partial_kernel(GmresDev g, const double* x) {
  __shared__ double wp[KW];
  const int64_t chunk = (g.n + g.nblk - 1) / g.nblk;
  const int64_t r0 = blockIdx.x * chunk, r1 = min(g.n, r0 + chunk);
  double s = 0.0;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += KT) s += x[row] * x[row];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < KW; ++w) t += wp[w];
    g.part[(int64_t)blockIdx.x * (g.m + 2)] = t;
  }
}

__global__ void begin_kernel(GmresDev g, double tol, int max_it, int which) {
  if (threadIdx.x != 0) return;
  const SL L{g.m};
  double ss = 0.0;
  for (int b = 0; b < g.nblk; ++b) ss += g.part[(int64_t)b * (g.m + 2)];
  if (which == 0) {               // ||f||
    g.st[L.sc() + S_NF] = sqrt(ss);
    g.st[L.sc() + S_TOL] = tol;
    g.ist[I_MAXIT] = max_it;
    g.ist[I_TOTAL] = 0;
    g.ist[I_STATUS] = RUNNING;
    return;
  }
  // which == 1: beta = ||r|| (cycle start or restart check)
  const double beta = sqrt(ss);
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

// y = H[:kd,:kd]^{-1} g[:kd] (back substitution), then u += Z y
__global__ void ysolve_kernel(GmresDev g) {
  if (threadIdx.x != 0) return;
  const SL L{g.m};
  const int kd = g.ist[I_KDONE];
  for (int i = kd - 1; i >= 0; --i) {
    double s = g.st[L.g() + i];
    for (int q = i + 1; q < kd; ++q) s -= g.st[L.H(i, q)] * g.st[L.y() + q];
    g.st[L.y() + i] = s / g.st[L.H(i, i)];
  }
}

__global__ void __launch_bounds__(KT) xupdate_kernel(GmresDev g, double* u) {
  const SL L{g.m};
  const int kd = g.ist[I_KDONE];
  __shared__ double ys[128];
  for (int i = threadIdx.x; i < kd; i += KT) ys[i] = g.st[L.y() + i];
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT) {
    double s = u[row];
    for (int i = 0; i < kd; ++i) s += g.Z[(int64_t)i * g.n + row] * ys[i];
    u[row] = s;
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
  norm_partial_kernel<<<g.nblk, KT, 0, s>>>(g, f);
  begin_kernel<<<1, 32, 0, s>>>(g, tol, max_it, 0);
  return cudaGetLastError();
}

// one Arnoldi step after z_k = M^{-1} v_k and w = A z_k
cudaError_t launch_cgs2_and_givens(const GmresDev& g, cudaStream_t s) {
  const SL L{g.m};
  mdot_kernel<<<g.nblk, KT, 0, s>>>(g);
  reduce_kernel<<<1, 128, 0, s>>>(g, L.h1(), 0);
  cgs_update_kernel<<<g.nblk, KT, 0, s>>>(g, L.h1(), 1);
  reduce_kernel<<<1, 128, 0, s>>>(g, L.h2(), 0);
  cgs_update_kernel<<<g.nblk, KT, 0, s>>>(g, L.h2(), 0);
  givens_kernel<<<1, 32, 0, s>>>(g);
  scale_next_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g);
  advance_kernel<<<1, 1, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_gmres_restart_update(const GmresDev& g, double* u, cudaStream_t s) {
  ysolve_kernel<<<1, 32, 0, s>>>(g);
  xupdate_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g, u);
  return cudaGetLastError();
}

// after r = f - A u: beta, convergence decision, and V[0] = r / beta for the next cycle
cudaError_t launch_gmres_residual_check(const GmresDev& g, cudaStream_t s) {
  norm_partial_kernel<<<g.nblk, KT, 0, s>>>(g, g.r);
  begin_kernel<<<1, 32, 0, s>>>(g, 0.0, 0, 1);
  start_basis_kernel<<<vec_blocks(g.n), KT, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace cpmdev
