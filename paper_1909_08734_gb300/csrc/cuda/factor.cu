// Batched LU with partial pivoting of all local matrices A_j (Sec. 5: the local problems
// are solved by LU factorisation).  Every A_j (unknowns in reverse Cuthill-McKee order) is
// padded to 64 T_j with an identity block and stored as 64 x 64 tiles; one blocked
// right-looking step per tile column s runs over all subdomains at once:
//   panel    : factor tile column s column by column, pivoting on max |a|, over the rows
//              that can be nonzero in it (below pend[s])
//   envelope : move (first, last) with the interchanges, take the U row's extent hiu, and
//              raise last to hiu for the rows the step updates
//   swap     : apply the panel's row interchanges to every other tile column
//   trsm     : U_sJ = L_ss^{-1} A_sJ for s < J <= hiu
//   update   : A_IJ -= L_Is U_sJ for the tiles inside the envelope (SIMT here, the
//              tensor-core versions live in lu_tc.cu)
// Tiles outside the envelope are zero and stay zero (the host-side rules are in
// host/ordering.cpp).  FP64 mode keeps double tiles; FP32 and BF16 modes keep float tiles in
// the swizzled layout of common.cuh.
#include <algorithm>
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace cpmdev {

template <typename T>
__device__ __forceinline__ T& at(T* a, const SubMeta& m, int i, int j) {
  return a[tile_base(m, i >> 6, j >> 6) + Layout<T>::off(i & 63, j & 63)];
}
template <typename T>
__device__ __forceinline__ T at(const T* a, const SubMeta& m, int i, int j) {
  return a[tile_base(m, i >> 6, j >> 6) + Layout<T>::off(i & 63, j & 63)];
}

// ---------------------------------------------------------------- assembly
template <typename T>
__global__ void scatter_kernel(T* a, const int64_t* __restrict__ off, const double* __restrict__ val,
                               int64_t nnz) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    a[off[e]] = (T)val[e];
}

template <typename T>
__global__ void pad_identity_kernel(T* a, const SubMeta* __restrict__ meta) {
  const SubMeta m = meta[blockIdx.y];
  const int np = 64 * m.T;
  for (int i = m.n + blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
    at(a, m, i, i) = (T)1;
}

// Failure-detection self-test: local column col of subdomain j becomes zero in every row, as
// if the assembled local matrix were singular (the factorisation must then report it).
template <typename T>
__global__ void zero_column_kernel(T* a, const SubMeta* __restrict__ meta, int j, int col) {
  const SubMeta m = meta[j];
  if (col < 0 || col >= m.n) return;
  for (int i = threadIdx.x; i < 64 * m.T; i += blockDim.x) at(a, m, i, col) = (T)0;
}

cudaError_t launch_zero_column(void* a, int fp64, const SubMeta* meta, int j, int col, cudaStream_t s) {
  if (fp64) zero_column_kernel<double><<<1, 256, 0, s>>>((double*)a, meta, j, col);
  else zero_column_kernel<float><<<1, 256, 0, s>>>((float*)a, meta, j, col);
  return cudaGetLastError();
}

cudaError_t launch_scatter(void* a, int fp64, const int64_t* off, const double* val, int64_t nnz,
                           cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  unsigned blocks = (unsigned)((nnz + 255) / 256);
  if (blocks > 152u * 64u) blocks = 152u * 64u;
  if (fp64) scatter_kernel<double><<<blocks, 256, 0, s>>>((double*)a, off, val, nnz);
  else scatter_kernel<float><<<blocks, 256, 0, s>>>((float*)a, off, val, nnz);
  return cudaGetLastError();
}

cudaError_t launch_pad_identity(void* a, int fp64, const SubMeta* meta, int n_sub, int t_max,
                                cudaStream_t s) {
  dim3 g(1, n_sub);
  if (fp64) pad_identity_kernel<double><<<g, 64, 0, s>>>((double*)a, meta);
  else pad_identity_kernel<float><<<g, 64, 0, s>>>((float*)a, meta);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- panel
constexpr int PANEL_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS) lu_panel_kernel(T* a, const SubMeta* __restrict__ meta,
                                                                 int32_t* ipiv, int* status, int s,
                                                                 const int32_t* __restrict__ pend, int t_max) {
  const SubMeta m = meta[blockIdx.x];
  if (s >= m.T) return;
  const int k0 = 64 * s, tid = threadIdx.x;
  // rows at or beyond np are zero in the panel's columns (tile envelope) and stay untouched
  const int np = pend ? pend[blockIdx.x * t_max + s] : 64 * m.T;
  const int lane = tid & 31, warp = tid >> 5;
  __shared__ T prow[64];
  __shared__ double wv[PANEL_THREADS / 32];
  __shared__ int wi[PANEL_THREADS / 32];
  __shared__ int piv_sh;
  for (int c = 0; c < 64; ++c) {
    const int col = k0 + c;
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = col + tid; i < np; i += PANEL_THREADS) {
      double v = fabs((double)at(a, m, i, col));
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      best = wv[0]; bi = wi[0];
      for (int w = 1; w < PANEL_THREADS / 32; ++w)
        if (wv[w] > best || (wv[w] == best && wi[w] < bi)) { best = wv[w]; bi = wi[w]; }
      if (!(best > 0.0)) {             // zero (or NaN) column: singular local matrix
        atomicOr(status, ST_SINGULAR);
        atomicMin(status + 1, (int)blockIdx.x);   // lowest singular subdomain
        bi = col;
      }
      piv_sh = bi;
      ipiv[m.row_off + col] = bi;
    }
    __syncthreads();
    const int piv = piv_sh;
    if (piv != col && tid < 64) {
      T t0 = at(a, m, col, k0 + tid);
      at(a, m, col, k0 + tid) = at(a, m, piv, k0 + tid);
      at(a, m, piv, k0 + tid) = t0;
    }
    __syncthreads();
    if (tid < 64) prow[tid] = at(a, m, col, k0 + tid);
    __syncthreads();
    const T d = prow[c];
    const T inv = d != (T)0 ? (T)1 / d : (T)0;
    for (int i = col + 1 + tid; i < np; i += PANEL_THREADS) {
      T l = at(a, m, i, col) * inv;
      at(a, m, i, col) = l;
      for (int cc = c + 1; cc < 64; ++cc) at(a, m, i, k0 + cc) -= l * prow[cc];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- panel in a cluster
// The same panel factorisation with the panel held in shared memory: a cluster of CS CTAs
// per subdomain, CTA r holding rows [k0 + r R, k0 + (r+1) R) of the panel's 64 columns.
// Rows are not moved during the panel: every row carries its logical position (the row index
// it would have after the interchanges so far).  Per column: cluster barrier -> every CTA
// reads the CS candidates (max |a|, lowest logical row on ties) and then the pivot row in
// place through distributed shared memory (a finished pivot row never changes again) ->
// every CTA relabels the pivot row and the row it displaces, updates its rows below the
// pivot and reduces the next column's candidate in the same pass.  One cluster barrier per
// column; the rows are written back to their final positions at the end.  Same pivots and
// the same arithmetic, element by element, as lu_panel_kernel.
constexpr int PC_THREADS = 256;
// Panel rows are 16-byte aligned (68 floats / 66 doubles: 128-bit accesses of a quarter warp
// to consecutive rows fall in distinct bank groups) and updated 16 bytes at a time.
template <typename T> struct PanelVec;
template <> struct PanelVec<float> {
  using V = float4;
  static constexpr int N = 4, STRIDE = 68;
};
template <> struct PanelVec<double> {
  using V = double2;
  static constexpr int N = 2, STRIDE = 66;
};
constexpr int PC_SMEM = 200 * 1024;           // dynamic shared memory for panel rows

__device__ __forceinline__ void argmax_pair(double& v, int& i, double ov, int oi) {
  if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
}

// Block-wide (max value, lowest index) of the threads' pairs into *ov, *oi (thread 0 writes).
__device__ __forceinline__ void block_argmax(double best, int bi, double* wv, int* wi, double* ov, int* oi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    argmax_pair(best, bi, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bi, o));
  if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wv[0];
    int i = wi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) argmax_pair(b, i, wv[w], wi[w]);
    *ov = b;
    *oi = i;
  }
}

template <typename T>
__global__ void __launch_bounds__(PC_THREADS) lu_panel_cluster_kernel(T* a, const SubMeta* __restrict__ meta,
                                                                      int32_t* ipiv, int* status, int s,
                                                                      int rows_per_cta,
                                                                      const int32_t* __restrict__ pend,
                                                                      int t_max) {
  constexpr int PC_STRIDE = PanelVec<T>::STRIDE;
  constexpr int VN = PanelVec<T>::N;
  using VT = typename PanelVec<T>::V;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const SubMeta m = meta[blockIdx.x / cs];
  if (s >= m.T) return;                         // the whole cluster (one subdomain) leaves together
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* panel = (T*)smem_raw;
  // logical row (index within the subdomain) of every physical slot; rows with a logical
  // index below the current column are finished pivot rows and never change again
  int* lg = (int*)(smem_raw + (size_t)rows_per_cta * PC_STRIDE * sizeof(T));
  __shared__ double cval[2], wv[PC_THREADS / 32];
  __shared__ int cidx[2], cloc[2], wi[PC_THREADS / 32], wl[PC_THREADS / 32];
  __shared__ __align__(16) T prow[64];
  __shared__ int piv_sh, piv_rank, piv_slot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k0 = 64 * s;
  // rows at or beyond np are zero in the panel's columns (tile envelope) and stay untouched
  const int np = pend ? pend[(blockIdx.x / cs) * t_max + s] : 64 * m.T;
  const int r0 = k0 + rank * rows_per_cta;
  const int nr = max(0, min(np, r0 + rows_per_cta) - r0);
  for (int e = tid; e < nr * 64; e += PC_THREADS) {
    const int i = e % nr, j = e / nr;
    panel[i * PC_STRIDE + j] = at(a, m, r0 + i, k0 + j);
  }
  for (int i = tid; i < nr; i += PC_THREADS) lg[i] = r0 + i;
  // block candidate (max |value|, lowest logical row on ties) with its slot -> slot sl
  auto block_candidate = [&](double best, int bi, int bs, int sl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o), os = __shfl_xor_sync(0xffffffffu, bs, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; bs = os; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; wl[warp] = bs; }
    __syncthreads();
    if (tid == 0) {
      double b = wv[0];
      int i = wi[0], l = wl[0];
      for (int w = 1; w < PC_THREADS / 32; ++w)
        if (wv[w] > b || (wv[w] == b && wi[w] < i)) { b = wv[w]; i = wi[w]; l = wl[w]; }
      cval[sl] = b;
      cidx[sl] = i;
      cloc[sl] = l;
    }
  };
  __syncthreads();
  {
    double best = -1.0;
    int bi = 0x7fffffff, bs = -1;
    for (int i = tid; i < nr; i += PC_THREADS) {
      const double v = fabs((double)panel[i * PC_STRIDE]);
      if (v > best) { best = v; bi = r0 + i; bs = i; }
    }
    block_candidate(best, bi, bs, 0);
  }
  for (int c = 0; c < 64; ++c) {
    const int col = k0 + c, slot = c & 1;
    cl.sync();                                  // every CTA's candidate of column c is visible
    if (warp == 0) {
      double v = -1.0;
      int ix = 0x7fffffff, loc = -1, rk = -1;
      if (lane < cs) {
        v = *cl.map_shared_rank(&cval[slot], lane);
        ix = *cl.map_shared_rank(&cidx[slot], lane);
        loc = *cl.map_shared_rank(&cloc[slot], lane);
        rk = lane;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ix, o), ol = __shfl_xor_sync(0xffffffffu, loc, o);
        const int orr = __shfl_xor_sync(0xffffffffu, rk, o);
        if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; loc = ol; rk = orr; }
      }
      if (lane == 0) {
        if (!(v > 0.0) || loc < 0) {            // zero (or NaN) column: singular local matrix
          if (rank == 0) {
            atomicOr(status, ST_SINGULAR);
            atomicMin(status + 1, (int)(blockIdx.x / cs));   // lowest singular subdomain
          }
          ix = -1;
        }
        piv_sh = ix;
        piv_rank = rk;
        piv_slot = loc;
      }
    }
    __syncthreads();
    const int p = piv_sh;                       // logical row chosen (-1: singular column)
    const int prk = piv_rank, psl = piv_slot;
    if (tid < 64) prow[tid] = p >= 0 ? cl.map_shared_rank(panel, prk)[psl * PC_STRIDE + tid] : (T)0;
    if (rank == 0 && tid == 0) ipiv[m.row_off + col] = p >= 0 ? p : col;
    __syncthreads();
    const T d = prow[c];
    const T inv = d != (T)0 ? (T)1 / d : (T)0;
    double best = -1.0;
    int bi = 0x7fffffff, bs = -1;
    for (int i = tid; i < nr; i += PC_THREADS) {
      int L = lg[i];
      if (L < col) continue;                     // finished pivot row
      if (p >= 0) {
        if (rank == prk && i == psl) { lg[i] = col; continue; }   // the pivot row: logical col
        if (L == col) { L = p; lg[i] = p; }      // the row displaced from position col
      } else if (L == col) {
        continue;                                // singular column: the row at col stays
      }
      T* row = panel + i * PC_STRIDE;
      const T l = row[c] * inv;
      row[c] = l;
      // columns c+1 .. 63, VN at a time from the group holding column c+1
      for (int g = (c + 1) / VN; g < 64 / VN; ++g) {
        VT v = ((VT*)row)[g];
        const VT pv = ((const VT*)prow)[g];
        T* ve = (T*)&v;
        const T* pe = (const T*)&pv;
#pragma unroll
        for (int u = 0; u < VN; ++u)
          if (VN * g + u > c) ve[u] -= l * pe[u];
        ((VT*)row)[g] = v;
      }
      if (c + 1 < 64) {
        const double v = fabs((double)row[c + 1]);
        if (v > best || (v == best && L < bi)) { best = v; bi = L; bs = i; }
      }
    }
    if (c + 1 < 64) block_candidate(best, bi, bs, slot ^ 1);
  }
  __syncthreads();
  for (int e = tid; e < nr * 64; e += PC_THREADS) {
    const int i = e % nr, j = e / nr;
    at(a, m, lg[i], k0 + j) = panel[i * PC_STRIDE + j];
  }
  cl.sync();                                    // no CTA leaves while its panel may be read
}

// Cluster size and rows per CTA for a panel of at most max_rows rows; 0 if it does not fit.
static int panel_cluster_size(int max_rows, size_t elem, int* rows_per_cta) {
  const int stride = elem == 8 ? PanelVec<double>::STRIDE : PanelVec<float>::STRIDE;
  const int cap = PC_SMEM / (stride * (int)elem + (int)sizeof(int));
  for (int cs = 1; cs <= 16; cs *= 2) {
    const int r = (max_rows + cs - 1) / cs;
    if (r <= cap) {
      *rows_per_cta = r;
      return cs;
    }
  }
  return 0;
}

template <typename T>
static cudaError_t launch_panel_cluster(const FactorDev& f, int step, int cs, int rpc, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(f.n_sub * cs);
  cfg.blockDim = dim3(PC_THREADS);
  cfg.dynamicSmemBytes = (size_t)rpc * PanelVec<T>::STRIDE * sizeof(T) + (size_t)rpc * sizeof(int);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<T>, (T*)f.a, f.meta, f.ipiv, f.status, step, rpc,
                            f.pend, f.t_max);
}

// ---------------------------------------------------------------- tile envelope, step s
// After the panel of step s: apply its 64 row interchanges to the rows' first / last tile
// columns, take the U row's extent hiu = max last over the pivot block, and extend last to
// hiu for every row below the block that the step updates (first <= s).  Rows [k0, pend)
// are staged in shared memory (ENV_SMEM_ROWS at most; beyond that the kernel works in
// global memory).
constexpr int ENV_THREADS = 256;
constexpr int ENV_SMEM_ROWS = 16384;
__global__ void __launch_bounds__(ENV_THREADS) lu_envelope_kernel(int32_t* first, int32_t* last,
                                                                 const SubMeta* __restrict__ meta,
                                                                 const int32_t* __restrict__ ipiv,
                                                                 const int32_t* __restrict__ pend, int t_max,
                                                                 int s, int32_t* hiu, int* status) {
  const SubMeta m = meta[blockIdx.x];
  if (s >= m.T) return;
  const int k0 = 64 * s, tid = threadIdx.x;
  const int nrow = pend[blockIdx.x * t_max + s] - k0;
  extern __shared__ int32_t env_smem[];
  const bool staged = nrow <= ENV_SMEM_ROWS;
  int32_t* F = staged ? env_smem : first + m.row_off + k0;
  int32_t* Lr = staged ? env_smem + nrow : last + m.row_off + k0;
  if (staged) {
    for (int i = tid; i < nrow; i += ENV_THREADS) {
      F[i] = first[m.row_off + k0 + i];
      Lr[i] = last[m.row_off + k0 + i];
    }
  }
  __syncthreads();
  if (tid == 0)
    for (int c = 0; c < 64; ++c) {
      const int p = ipiv[m.row_off + k0 + c] - k0;
      if (p < c || p >= nrow) {                // outside the panel's rows: cannot happen
        atomicOr(status, ST_SINGULAR);
        atomicMin(status + 1, (int)blockIdx.x);
        continue;
      }
      const int32_t tf = F[c], tl = Lr[c];
      F[c] = F[p];
      Lr[c] = Lr[p];
      F[p] = tf;
      Lr[p] = tl;
    }
  __syncthreads();
  __shared__ int32_t hmax[ENV_THREADS / 32];
  int32_t h = tid < 64 ? Lr[tid] : s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
  if ((tid & 31) == 0) hmax[tid >> 5] = h;
  __syncthreads();
  int32_t hu = s;
  for (int w = 0; w < ENV_THREADS / 32; ++w) hu = max(hu, hmax[w]);
  if (tid == 0) hiu[blockIdx.x] = hu;
  for (int i = 64 + tid; i < nrow; i += ENV_THREADS)
    if (F[i] <= s && Lr[i] < hu) Lr[i] = hu;
  __syncthreads();
  if (staged)
    for (int i = tid; i < nrow; i += ENV_THREADS) {
      first[m.row_off + k0 + i] = F[i];
      last[m.row_off + k0 + i] = Lr[i];
    }
}

// Largest cluster size each device can co-schedule with the panel kernel's shared memory
// (probed once per device, under a lock: set-ups may run in several host threads, and a reader
// must never see a half-finished probe).
constexpr int PANEL_MAX_DEVICES = 64;
static int g_panel_max_cs[PANEL_MAX_DEVICES][2] = {};
static bool g_panel_probed[PANEL_MAX_DEVICES] = {};
static std::mutex g_panel_mu;

static int panel_max_cs(int fp64) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PANEL_MAX_DEVICES) return 0;
  std::lock_guard<std::mutex> lock(g_panel_mu);
  return g_panel_probed[dev] ? g_panel_max_cs[dev][fp64] : 0;
}

cudaError_t lu_panel_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= PANEL_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_panel_mu);
  if (g_panel_probed[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(lu_envelope_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(ENV_SMEM_ROWS * 2 * sizeof(int32_t)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_panel_cluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, PC_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_panel_cluster_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, PC_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_panel_cluster_kernel<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(lu_panel_cluster_kernel<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 2; ++k) {
    int best = 0;
    for (int cs = 16; cs >= 1 && !best; cs /= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(PC_THREADS);
      cfg.dynamicSmemBytes = PC_SMEM;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cs;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      e = k ? cudaOccupancyMaxActiveClusters(&n, lu_panel_cluster_kernel<double>, &cfg)
            : cudaOccupancyMaxActiveClusters(&n, lu_panel_cluster_kernel<float>, &cfg);
      if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
      }
      if (n > 0) best = cs;
    }
    g_panel_max_cs[dev][k] = best;
  }
  g_panel_probed[dev] = true;
  return cudaSuccess;
}

// ---------------------------------------------------------------- row interchanges
template <typename T>
__global__ void lu_swap_kernel(T* a, const SubMeta* __restrict__ meta, const int32_t* __restrict__ ipiv,
                               int s) {
  const SubMeta m = meta[blockIdx.y];
  const int J = blockIdx.x;
  if (s >= m.T || J >= m.T || J == s) return;
  const int k0 = 64 * s, col = 64 * J + threadIdx.x;
  for (int c = 0; c < 64; ++c) {
    const int r = k0 + c, p = ipiv[m.row_off + r];
    if (p != r) {
      T t0 = at(a, m, r, col);
      at(a, m, r, col) = at(a, m, p, col);
      at(a, m, p, col) = t0;
    }
  }
}

// ---------------------------------------------------------------- U_sJ = L_ss^{-1} A_sJ
template <typename T>
__global__ void __launch_bounds__(64) lu_trsm_kernel(T* a, const SubMeta* __restrict__ meta, int s,
                                                     const int32_t* __restrict__ hiu) {
  const SubMeta m = meta[blockIdx.y];
  const int J = s + 1 + blockIdx.x;
  if (J >= m.T || (hiu && J > hiu[blockIdx.y])) return;   // zero tiles of the U row stay zero
  __shared__ T L[64][65];
  const T* ts = a + tile_base(m, s, s);
  for (int e = threadIdx.x; e < 4096; e += 64) {
    int i = e & 63, j = e >> 6;
    L[i][j] = ts[Layout<T>::off(i, j)];
  }
  __syncthreads();
  T* tj = a + tile_base(m, s, J);
  const int col = threadIdx.x;
  T x[64];
#pragma unroll
  for (int r = 0; r < 64; ++r) x[r] = tj[Layout<T>::off(r, col)];
#pragma unroll
  for (int r = 1; r < 64; ++r) {
    T acc = x[r];
#pragma unroll
    for (int c = 0; c < r; ++c) acc -= L[r][c] * x[c];
    x[r] = acc;
  }
#pragma unroll
  for (int r = 0; r < 64; ++r) tj[Layout<T>::off(r, col)] = x[r];
}

// ---------------------------------------------------------------- A_IJ -= L_Is U_sJ (SIMT)
template <typename T>
__global__ void __launch_bounds__(256) lu_update_simt_kernel(T* a, const SubMeta* __restrict__ meta,
                                                             int s, int t_max, const int32_t* __restrict__ pend,
                                                             const int32_t* __restrict__ hiu) {
  const SubMeta m = meta[blockIdx.y];
  const int W = t_max - 1 - s;
  const int I = s + 1 + blockIdx.x / W, J = s + 1 + blockIdx.x % W;
  if (I >= m.T || J >= m.T) return;
  // outside the envelope L_Is or U_sJ is zero: the tile does not change
  if (pend && (64 * I >= pend[blockIdx.y * t_max + s] || J > hiu[blockIdx.y])) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = (T*)smem_raw;              // As[i*65 + k]
  T* Bs = As + 64 * 65;              // Bs[k*65 + j]
  const T* ta = a + tile_base(m, I, s);
  const T* tb = a + tile_base(m, s, J);
  for (int e = threadIdx.x; e < 4096; e += 256) {
    int i = e & 63, k = e >> 6;
    As[i * 65 + k] = ta[Layout<T>::off(i, k)];
    Bs[i * 65 + k] = tb[Layout<T>::off(i, k)];   // (row i = k-index of U, col k = j)
  }
  __syncthreads();
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = (T)0;
#pragma unroll 8
  for (int k = 0; k < 64; ++k) {
    T av[4], bv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) av[p] = As[(ti + 16 * p) * 65 + k];
#pragma unroll
    for (int q = 0; q < 4; ++q) bv[q] = Bs[k * 65 + tj + 16 * q];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
  }
  T* tc = a + tile_base(m, I, J);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) tc[Layout<T>::off(ti + 16 * p, tj + 16 * q)] -= acc[p][q];
}



cudaError_t launch_lu_step(const FactorDev& f, int step, int use_tc, cudaStream_t s) {
  const int W = f.t_max - 1 - step;
  const bool env = f.pend != nullptr;
  // panel rows of this step: the largest envelope range over the subdomains
  const int max_rows = env ? f.step_rows[step] : 64 * (f.t_max - step);
  int rpc = 0;
  const int cs = panel_cluster_size(max_rows, f.fp64 ? 8 : 4, &rpc);
  const bool cluster = cs > 0 && cs <= panel_max_cs(f.fp64 ? 1 : 0);
  const size_t sm = 2 * 64 * 65 * (f.fp64 ? sizeof(double) : sizeof(float));
  const size_t env_smem = (size_t)std::min(max_rows, ENV_SMEM_ROWS) * 2 * sizeof(int32_t);
  auto envelope = [&]() {
    if (env)
      lu_envelope_kernel<<<f.n_sub, ENV_THREADS, env_smem, s>>>(f.first, f.last, f.meta, f.ipiv, f.pend,
                                                                f.t_max, step, f.hiu, f.status);
  };
  if (f.fp64) {
    double* a = (double*)f.a;
    if (cluster) {
      cudaError_t e = launch_panel_cluster<double>(f, step, cs, rpc, s);
      if (e != cudaSuccess) return e;
    } else {
      lu_panel_kernel<double><<<f.n_sub, PANEL_THREADS, 0, s>>>(a, f.meta, f.ipiv, f.status, step, f.pend,
                                                                f.t_max);
    }
    envelope();
    lu_swap_kernel<double><<<dim3(f.t_max, f.n_sub), 64, 0, s>>>(a, f.meta, f.ipiv, step);
    if (W > 0) {
      lu_trsm_kernel<double><<<dim3(W, f.n_sub), 64, 0, s>>>(a, f.meta, step, f.hiu);
      cudaFuncSetAttribute(lu_update_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      lu_update_simt_kernel<double><<<dim3(W * W, f.n_sub), 256, sm, s>>>(a, f.meta, step, f.t_max, f.pend,
                                                                          f.hiu);
    }
  } else {
    float* a = (float*)f.a;
    if (cluster) {
      cudaError_t e = launch_panel_cluster<float>(f, step, cs, rpc, s);
      if (e != cudaSuccess) return e;
    } else {
      lu_panel_kernel<float><<<f.n_sub, PANEL_THREADS, 0, s>>>(a, f.meta, f.ipiv, f.status, step, f.pend,
                                                               f.t_max);
    }
    envelope();
    lu_swap_kernel<float><<<dim3(f.t_max, f.n_sub), 64, 0, s>>>(a, f.meta, f.ipiv, step);
    if (W > 0) {
      lu_trsm_kernel<float><<<dim3(W, f.n_sub), 64, 0, s>>>(a, f.meta, step, f.hiu);
      if (use_tc) {
        cudaError_t e = launch_lu_update_tc(f, step, use_tc == 2, s);
        if (e != cudaSuccess) return e;
      } else {
        lu_update_simt_kernel<float><<<dim3(W * W, f.n_sub), 256, sm, s>>>(a, f.meta, step, f.t_max, f.pend,
                                                                           f.hiu);
      }
    }
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- after the factorisation
// perm: the row interchanges applied in order to the identity; gather[r] = global index of
// local unknown perm[r] when it carries residual (own_flag bit 2: in Sigma_j), else -1;
// scatter[r] = global index of local unknown r if r is in the disjoint set (own_flag bit 1),
// else -1;
// dinv[r] = 1 / U_rr.
template <typename T>
__global__ void lu_finish_kernel(const T* a, const SubMeta* __restrict__ meta, const int32_t* ipiv,
                                 const int32_t* __restrict__ unknowns, const int64_t* __restrict__ unk_off,
                                 const int32_t* __restrict__ own_flag, int32_t* gather,
                                 int32_t* scatter, T* dinv) {
  const SubMeta m = meta[blockIdx.x];
  const int np = 64 * m.T;
  int32_t* perm = gather + m.row_off;       // built in place, then mapped
  if (threadIdx.x == 0) {
    for (int r = 0; r < np; ++r) perm[r] = r;
    for (int r = 0; r < np; ++r) {
      int p = ipiv[m.row_off + r];
      int t = perm[r]; perm[r] = perm[p]; perm[p] = t;
    }
  }
  __syncthreads();
  const int64_t uo = unk_off[blockIdx.x];
  for (int r = threadIdx.x; r < np; r += blockDim.x) {
    int pr = perm[r];
    perm[r] = (pr < m.n && (own_flag[uo + pr] & 2)) ? unknowns[uo + pr] : -1;
    scatter[m.row_off + r] = (r < m.n && (own_flag[uo + r] & 1)) ? unknowns[uo + r] : -1;
    T d = at(a, m, r, r);
    dinv[m.row_off + r] = d != (T)0 ? (T)1 / d : (T)0;
  }
}

cudaError_t launch_lu_finish(const FactorDev& f, const int32_t* unknowns, const int64_t* unk_off,
                             const int32_t* own_flag, int32_t* gather, int32_t* scatter,
                             void* dinv, cudaStream_t s) {
  if (f.fp64)
    lu_finish_kernel<double><<<f.n_sub, 256, 0, s>>>((const double*)f.a, f.meta, f.ipiv, unknowns,
                                                     unk_off, own_flag, gather, scatter, (double*)dinv);
  else
    lu_finish_kernel<float><<<f.n_sub, 256, 0, s>>>((const float*)f.a, f.meta, f.ipiv, unknowns,
                                                    unk_off, own_flag, gather, scatter, (float*)dinv);
  return cudaGetLastError();
}

// Inverses of the diagonal blocks of every tile row: Linv = L_II^{-1} (unit lower) and
// Uinv = U_II^{-1} (upper), stored column-major in the compute precision C at
// inv + ((row_off/64 + I) * 2 + {0: L, 1: U}) * 4096.  The triangular solves then apply a
// diagonal block as one parallel matrix-vector product instead of a 64-step substitution.
template <typename T, typename C>
__global__ void __launch_bounds__(64) diag_inverse_kernel(const T* a, const SubMeta* __restrict__ meta,
                                                          C* inv) {
  const SubMeta m = meta[blockIdx.y];
  const int I = blockIdx.x;
  if (I >= m.T) return;
  __shared__ C D[64][65];
  const T* td = a + tile_base(m, I, I);
  for (int e = threadIdx.x; e < 4096; e += 64) {
    int i = e & 63, j = e >> 6;
    D[i][j] = (C)td[Layout<T>::off(i, j)];
  }
  __syncthreads();
  const int c = threadIdx.x;
  C* li = inv + (((m.row_off >> 6) + I) * 2) * (int64_t)TILE_ELEMS;
  C* ui = li + TILE_ELEMS;
  C x[64];
  // column c of L^{-1}: x_r = delta_rc - sum_{k<r} L_rk x_k (x_r = 0 for r < c)
#pragma unroll
  for (int r = 0; r < 64; ++r) {
    C s = (r == c) ? (C)1 : (C)0;
#pragma unroll
    for (int k = 0; k < r; ++k) s -= D[r][k] * x[k];
    x[r] = r < c ? (C)0 : s;
  }
#pragma unroll
  for (int r = 0; r < 64; ++r) li[off_plain(r, c)] = x[r];
  // column c of U^{-1}: x_r = (delta_rc - sum_{k>r} U_rk x_k) / U_rr (x_r = 0 for r > c)
#pragma unroll
  for (int r = 63; r >= 0; --r) {
    C s = (r == c) ? (C)1 : (C)0;
#pragma unroll
    for (int k = r + 1; k < 64; ++k) s -= D[r][k] * x[k];
    x[r] = r > c ? (C)0 : s / D[r][r];
  }
#pragma unroll
  for (int r = 0; r < 64; ++r) ui[off_plain(r, c)] = x[r];
}

cudaError_t launch_diag_inverse(const void* a, int fp64, const SubMeta* meta, int n_sub, int t_max,
                                void* inv, cudaStream_t s) {
  dim3 g(t_max, n_sub);
  if (fp64) diag_inverse_kernel<double, double><<<g, 64, 0, s>>>((const double*)a, meta, (double*)inv);
  else diag_inverse_kernel<float, float><<<g, 64, 0, s>>>((const float*)a, meta, (float*)inv);
  return cudaGetLastError();
}

// Chain tiles of the solves.  In tile row I the forward substitution computes
//     x_I = Linv_I (b_I - sum_{J < I-1} L_IJ x_J) - (Linv_I L_{I,I-1}) x_{I-1}
// and the backward one likewise with Uinv_I U_{I,I+1} x_{I+1}: the product with the inverse
// is taken before the neighbouring row's piece arrives, which leaves one matrix-vector
// product on the chain between consecutive tile rows.  This kernel replaces L_{I,I-1} by
// Linv_I L_{I,I-1} and U_{I,I+1} by Uinv_I U_{I,I+1} in place (tiles inside the envelope
// only; sums in FP64).
template <typename T, typename C>
__global__ void __launch_bounds__(64) chain_tiles_kernel(T* a, const SubMeta* __restrict__ meta, const C* inv,
                                                        const int32_t* __restrict__ tlo,
                                                        const int32_t* __restrict__ thi) {
  const SubMeta m = meta[blockIdx.y];
  const int I = blockIdx.x;
  if (I >= m.T) return;
  const int64_t trow = (m.row_off >> 6) + I;
  __shared__ C X[64][65];
  const int c = threadIdx.x;
  for (int side = 0; side < 2; ++side) {
    const int J = side == 0 ? I - 1 : I + 1;
    if (side == 0 ? tlo[trow] > J : thi[trow] < J) continue;   // outside the envelope
    const C* xi = inv + (trow * 2 + side) * (int64_t)TILE_ELEMS;
    T* tb = a + tile_base(m, I, J);
    __syncthreads();
    for (int e = threadIdx.x; e < 4096; e += 64) {
      const int i = e & 63, j = e >> 6;
      X[i][j] = xi[off_plain(i, j)];
    }
    double bc[64];                              // column c of the tile
#pragma unroll
    for (int k = 0; k < 64; ++k) bc[k] = (double)tb[Layout<T>::off(k, c)];
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < 64; ++r) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 64; ++k) acc += (double)X[r][k] * bc[k];
      tb[Layout<T>::off(r, c)] = (T)acc;
    }
  }
}

cudaError_t launch_chain_tiles(void* a, int fp64, const SubMeta* meta, int n_sub, int t_max, const void* inv,
                               const int32_t* tlo, const int32_t* thi, cudaStream_t s) {
  dim3 g(t_max, n_sub);
  if (fp64)
    chain_tiles_kernel<double, double><<<g, 64, 0, s>>>((double*)a, meta, (const double*)inv, tlo, thi);
  else
    chain_tiles_kernel<float, float><<<g, 64, 0, s>>>((float*)a, meta, (const float*)inv, tlo, thi);
  return cudaGetLastError();
}

// Packs every diagonal-block inverse into its triangle at the start of its slot (slot 2 trow:
// L^{-1}, slot 2 trow + 1: U^{-1}; INV_PACKED entries each), after the chain tiles have used
// the full tiles: the solves then stream half a tile per inverse.
template <typename C>
__global__ void __launch_bounds__(64) pack_inverse_kernel(C* inv) {
  const int64_t slot = blockIdx.x;
  const bool upper = (slot & 1) != 0;
  C* t = inv + slot * (int64_t)TILE_ELEMS;
  __shared__ C X[TILE_ELEMS];
  for (int e = threadIdx.x; e < TILE_ELEMS; e += 64) X[e] = t[e];
  __syncthreads();
  const int c = threadIdx.x;
  if (upper) {
    for (int r = 0; r <= c; ++r) t[inv_upper_index(r, c)] = X[off_plain(r, c)];
  } else {
    for (int r = c; r < TILE; ++r) t[inv_lower_index(r, c)] = X[off_plain(r, c)];
  }
}

cudaError_t launch_pack_inverse(void* inv, int fp64, int64_t n_tile_rows, cudaStream_t s) {
  const int64_t slots = 2 * n_tile_rows;
  if (slots <= 0) return cudaSuccess;
  if (slots > 2147483647) return cudaErrorInvalidValue;
  if (fp64) pack_inverse_kernel<double><<<(unsigned)slots, 64, 0, s>>>((double*)inv);
  else pack_inverse_kernel<float><<<(unsigned)slots, 64, 0, s>>>((float*)inv);
  return cudaGetLastError();
}

__global__ void pack_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ out,
                                 int64_t n_tiles) {
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const float* src = a + t * TILE_ELEMS;
    __nv_bfloat16* dst = out + t * TILE_ELEMS;
    for (int e = threadIdx.x; e < TILE_ELEMS; e += blockDim.x) {
      int i = e & 63, j = e >> 6;
      dst[off_plain(i, j)] = __float2bfloat16_rn(src[off_sw32(i, j)]);
    }
  }
}

cudaError_t launch_pack_bf16(const float* a, __nv_bfloat16* out, int64_t n_tiles, cudaStream_t s) {
  unsigned g = (unsigned)(n_tiles < 152 * 16 ? n_tiles : 152 * 16);
  if (g == 0) return cudaSuccess;
  pack_bf16_kernel<<<g, 256, 0, s>>>(a, out, n_tiles);
  return cudaGetLastError();
}

}  // namespace cpmdev
