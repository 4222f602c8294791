// Device-resident right-preconditioned flexible GMRES(m) with CGS2 (Sec. 2.2: the (O)RAS
// preconditioner inside GMRES) for 1..8 right-hand sides advanced in lock step.  All Arnoldi
// arithmetic is FP64.
//
// FP64 instructions are the scarce resource here (this GPU issues two FP64 lanes per SM and
// clock, 1/64 of its FP32 rate), so the kernels issue as few as the method needs:
//  * dot products V_k^T w: a warp owns whole basis vectors (lanes read consecutive rows) and
//    leaves 32 lane partials per vector, which one thread then adds; a shuffle tree per value
//    and warp would cost 5 x 32 lane additions per value;
//  * updates w -= V_k h: one thread per row and no reduction;
//  * block partials (stored vector-major, so that one warp reads a vector's partials of all
//    blocks in one coalesced round) are added by every block of the consuming kernel in one
//    fixed order (deterministic, no atomics); only the norm's last block finishes the step;
//  * v_{k+1} = w / ||w|| is no pass of its own: a step stores w unnormalised in V[k+1] with the
//    scale 1/||w||; the next solve multiplies while it gathers (IndirectVec::scale) and the next
//    step's first kernel normalises V[k+1] in place as it reads it.
// The kernels of a step use programmatic dependent launch: a kernel may be scheduled while its
// predecessor runs and waits (griddepcontrol.wait) before it reads anything.
//
// Right-hand side q is blockIdx.y; its state (step k, done flag, status, ...) lives in device
// memory, so one captured CUDA graph of an iteration replays for every k, and every kernel of
// an iteration returns at once for a right-hand side whose cycle has stopped.  Each right-hand
// side follows exactly the operations of a single-rhs solve (the batch only shares launches and
// the factor stream of the solves).  One Arnoldi step after z_k = M^{-1} v_k, vext = E z_k:
//   wdots : w = A z_k (operator second half);  V[k] *= s;  partial h1 = V_k^T w
//   upd1  : h1 = sum of partials;  w -= V_k h1;  partial h2 = V_k^T w
//   upd2  : h2 = sum of partials;  w -= V_k h2 -> V[k+1];  partial ||w||^2;  last block:
//           Hessenberg column, Givens rotation, stopping test, s = 1/||w||, k += 1
#include <math.h>

#include "../../../include/cpm.h"
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int KT = 256;                 // threads per block of the restart vector kernels
constexpr int KW = KT / 32;
constexpr int ST = 512;                 // threads per block of the Arnoldi step kernels
constexpr int SW = ST / 32;             // their warps (four per scheduler: latency hiding)
constexpr int MAX_UNITS = 128;          // basis vectors of one step (m + 1 <= 128)

// int state per right-hand side (GMRES_IST_STRIDE ints)
enum { I_K = 0, I_TOTAL = 1, I_DONE = 2, I_STATUS = 3, I_KDONE = 4, I_MAXIT = 5, I_SLOT = 6,
       I_TICKET = 8 };                  // tickets 8..11
constexpr int RUNNING = -1;
// batch control words
enum { C_LIVE = 0, C_ALLDONE = 1 };

// double state layout for restart length m
struct SL {
  int m;
  __host__ __device__ int H(int i, int k) const { return i + k * (m + 1); }
  __host__ __device__ int cs() const { return (m + 1) * m; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int y() const { return g() + m + 1; }
  __host__ __device__ int h1() const { return y() + m; }
  __host__ __device__ int sc() const { return h1() + m + 1; }   // scalars
};
enum { S_NF = 0, S_TOL = 1, S_BETA = 2, S_HN = 3, S_RELRES = 4, S_VSCALE = 5 };
static_assert(I_SLOT == GMRES_SLOT_INT && S_VSCALE == GMRES_VSCALE_DBL, "state layout shared with the host");

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// views of right-hand side q
struct Rhs {
  double *V, *Z, *w, *r, *st, *p1, *p2, *p3;
  int* ist;
};
__device__ __forceinline__ Rhs rhs_view(const GmresDev& g, int q) {
  Rhs v;
  v.V = g.V + (int64_t)q * (g.m + 1) * g.ld;
  v.Z = g.Z + (int64_t)q * (g.m + 1) * g.ld;
  v.w = g.w + (int64_t)q * g.ld;
  v.r = g.r + (int64_t)q * g.ld;
  v.st = g.st + (int64_t)q * g.st_stride;
  v.p1 = g.part + (int64_t)q * g.part_stride;
  v.p2 = v.p1 + (int64_t)g.nblk * (g.m + 1);
  v.p3 = v.p2 + (int64_t)g.nblk * (g.m + 1);
  v.ist = g.ist + q * GMRES_IST_STRIDE;
  return v;
}

__device__ __forceinline__ bool stopped(const Rhs& v) { return *(volatile const int*)&v.ist[I_DONE] != 0; }
// k, total, done, status of a right-hand side in one 16-byte load (state ints are 64-byte aligned)
__device__ __forceinline__ int4 load_state(const Rhs& v) { return __ldcg(reinterpret_cast<const int4*>(v.ist)); }

// this block's rows [r0, r0 + nr)
__device__ __forceinline__ int block_rows(const GmresDev& g, int64_t* r0) {
  *r0 = (int64_t)blockIdx.x * g.chunk;
  const int64_t e = min(g.n, *r0 + (int64_t)g.chunk);
  return (int)max((int64_t)0, e - *r0);
}

// ---- staged basis stream -------------------------------------------------------------
// A step kernel reads the basis rows of its block tile by tile (TR rows): for each tile one or
// two passes over the vectors, a pass being a sequence of batches of VB vectors.  Thread 0
// issues the bulk copies of batch q + 2 while the block multiplies batch q, so FP64 work never
// waits for a load; a batch is double-buffered in shared memory with one mbarrier per buffer,
// and every wait is bounded (CPM_ERR_TIMEOUT through the status word).  Only the current tile
// of w is held in shared memory, so a block may own any number of rows and the grid is one
// block per SM at every size.
constexpr int VB = 8;                   // basis vectors per batch
constexpr int TR = 1024;                // rows per tile
constexpr int RU = TR / ST;             // rows per thread in the update pass
constexpr int WPV = SW / VB;            // warps per vector in the dot pass
constexpr int TJ = TR / (32 * WPV);     // 32-row groups of a tile per warp in the dot pass
constexpr int RED_LD = 32 * WPV + 1;    // lane partials of one vector, padded
static_assert(RU * ST == TR && WPV * VB == SW && TJ % 2 == 0, "batch shape tied to the block shape");

struct StepSmem {
  double *stage, *ws, *hs, *red;
};
// Dynamic shared memory: stage[2][VB][TR] | ws[TR] | hs[MAX_UNITS] | red[MAX_UNITS * RED_LD]
__device__ __forceinline__ StepSmem step_smem() {
  extern __shared__ __align__(128) double dsm[];
  StepSmem s;
  s.stage = dsm;
  s.ws = dsm + 2 * VB * TR;
  s.hs = s.ws + TR;
  s.red = s.hs + MAX_UNITS;
  return s;
}
size_t gmres_step_smem_bytes() {
  return sizeof(double) * ((size_t)2 * VB * TR + TR + MAX_UNITS + (size_t)MAX_UNITS * RED_LD);
}

struct VStream {
  const double* Vb;   // the block's first row of V[0]
  int64_t ld;
  int nr, nv;         // rows of the block, vectors 0 .. nv-1
  int ntile, nbatch, npass, total;
  double* stage;
  uint64_t* bar;
  // batch q of the stream: tile-major, then pass, then batch of vectors
  __device__ int tile(int q) const { return q / (npass * nbatch); }
  __device__ int pass(int q) const { return (q / nbatch) % npass; }
  __device__ int batch(int q) const { return q % nbatch; }
  __device__ int rows(int q) const { return min(TR, nr - tile(q) * TR); }
  __device__ int count(int q) const { return min(VB, nv - batch(q) * VB); }
  __device__ double* buf(int q) const { return stage + (q & 1) * VB * TR; }
  // thread 0: bulk copies of batch q (each vector's tile rows, rounded up to 16 bytes: the
  // vectors are padded to a multiple of 32 doubles, so the extra double is in bounds)
  __device__ void issue(int q) const {
    if (q >= total) return;
    const uint32_t bytes = (uint32_t)((rows(q) * 8 + 15) & ~15);
    const int i0 = batch(q) * VB, cnt = count(q);
    mbar_expect_tx(&bar[q & 1], bytes * (uint32_t)cnt);
    if (bytes == 0) return;             // a block without rows: the arrival completes the phase
    const double* src = Vb + (int64_t)tile(q) * TR;
    for (int u = 0; u < cnt; ++u) bulk_g2s(buf(q) + u * TR, src + (int64_t)(i0 + u) * ld, bytes, &bar[q & 1]);
  }
  __device__ bool wait(int q) const { return mbar_wait_bounded(&bar[q & 1], (q >> 1) & 1); }
};

__device__ __forceinline__ VStream make_stream(const GmresDev& g, const double* V, int64_t r0, int nr, int nv,
                                               int npass, const StepSmem& sm, uint64_t* bar) {
  VStream v;
  v.Vb = V + r0;
  v.ld = g.ld;
  v.nr = nr;
  v.nv = nv;
  v.ntile = max(1, (nr + TR - 1) / TR);
  v.nbatch = (nv + VB - 1) / VB;
  v.npass = npass;
  v.total = v.ntile * npass * v.nbatch;
  v.stage = sm.stage;
  v.bar = bar;
  return v;
}

// Start of a step kernel's stream: barriers initialised, the first two batches in flight.  The
// block barrier between the initialisation and the copies orders every thread's first wait
// after the initialisation (a wait on an mbarrier that thread 0 has not yet initialised is
// undefined); the copies are issued after it, so the other threads go on meanwhile.
__device__ __forceinline__ void stream_begin(const VStream& vs, uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    vs.issue(0);
    vs.issue(1);
  }
}

// Bounded wait for batch q by every thread, folded into one block-wide vote.  On failure the
// status word records the timeout and thread 0 waits (bounded) for the copies still in flight
// (batches q and q + 1), so that none lands after the block has left.
__device__ __forceinline__ bool stream_wait(const GmresDev& g, const VStream& vs, int q) {
  const bool ok = __syncthreads_and(vs.wait(q));
  if (!ok && threadIdx.x == 0) {
    atomicOr(g.status, ST_TIMEOUT | ST_AT_KRYLOV);
    for (int r = q; r < min(q + 2, vs.total); ++r) vs.wait(r);
  }
  return ok;
}

// Dot pass over batch q of the stream: warps 2s and 2s+1 own vector i0 + s and take the
// even / odd 32-row groups of the tile; lane partials x[row] ws[row] accumulate in
// red[i RED_LD + 32 half + lane] (started at the block's first tile).  scale_vec >= 0: that
// vector's values are first multiplied by scale and written back to V.
__device__ __forceinline__ void dots_batch(const VStream& vs, int q, const StepSmem& sm, int scale_vec,
                                           double scale, double* Vglob_row0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = warp / WPV, half = warp % WPV;
  const int cnt = vs.count(q);
  if (slot >= cnt) return;
  const int t = vs.tile(q), rows = vs.rows(q);
  const int i = vs.batch(q) * VB + slot;
  const double* x = vs.buf(q) + slot * TR;
  const double* ws = sm.ws;
  double a0 = 0.0, a1 = 0.0;
  if (i == scale_vec) {
    double* vg = Vglob_row0 + (int64_t)i * vs.ld + (int64_t)t * TR;
    for (int row = half * 32 + lane; row < rows; row += 32 * WPV) {
      const double v = x[row] * scale;
      vg[row] = v;
      a0 = fma(v, ws[row], a0);
    }
  } else if (rows == TR) {
#pragma unroll
    for (int j = 0; j < TJ; j += 2) {
      const int row = (j * WPV + half) * 32 + lane;
      a0 = fma(x[row], ws[row], a0);
      a1 = fma(x[row + 32 * WPV], ws[row + 32 * WPV], a1);
    }
  } else {
    // a ragged tile: a loop with warp-uniform bounds (per-group predication of the unrolled
    // loop above measured slower where this pass is the block's arithmetic bound)
    for (int row = half * 32 + lane; row < rows; row += 32 * WPV) a0 = fma(x[row], ws[row], a0);
  }
  double* r = sm.red + i * RED_LD + half * 32 + lane;
  *r = (t == 0 ? 0.0 : *r) + (a0 + a1);
}

// Update pass over batch q: a[j] += sum_u x_u[row_j] hs[i0 + u] for the thread's rows
// tid + ST j of the tile (vectors in increasing order).
__device__ __forceinline__ void update_batch(const VStream& vs, int q, const StepSmem& sm, double (&a)[RU]) {
  const int cnt = vs.count(q), rows = vs.rows(q), i0 = vs.batch(q) * VB;
  const double* x = vs.buf(q);
  if (cnt == VB && rows == TR) {
#pragma unroll
    for (int u = 0; u < VB; ++u) {
      const double h = sm.hs[i0 + u];
#pragma unroll
      for (int j = 0; j < RU; ++j) a[j] = fma(x[u * TR + threadIdx.x + ST * j], h, a[j]);
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < VB; ++u) {
    if (u < cnt) {
      const double h = sm.hs[i0 + u];
#pragma unroll
      for (int j = 0; j < RU; ++j) {
        const int row = threadIdx.x + ST * j;
        if (row < rows) a[j] = fma(x[u * TR + row], h, a[j]);
      }
    }
  }
}

// out[i stride] = sum of red[i]'s 64 lane partials for i < nv: warp w takes vectors w, w + SW,
// ...; lane l adds its two halves, then a butterfly (a fixed order, no long chain of dependent
// FP64 additions, which cost tens of cycles each on this GPU).
__device__ __forceinline__ void finish_dots(int nv, const StepSmem& sm, double* __restrict__ out, int stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < nv; i += SW) {
    const double* p = sm.red + i * RED_LD;
    double s = p[lane] + p[lane + 32];
    s = warp_sum(s);
    if (lane == 0) out[(int64_t)i * stride] = s;
  }
}

// Sum over the warps of a block of one value per thread (fixed order); valid in thread 0.
template <int NW>
__device__ __forceinline__ double block_sum(double v, double* wsum) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < NW ? wsum[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum of nb values p[0 .. nb) by one warp, in a fixed order (valid in every lane): lane l
// loads p[l + 32 j] for SP_LOADS values of j at once, adds them in a tree, then a butterfly.
constexpr int SP_LOADS = 8;             // one round covers 256 blocks
__device__ __forceinline__ double warp_sum_blocks(const double* __restrict__ p, int nb) {
  static_assert(SP_LOADS == 8, "the tree below adds eight loads");
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 32 * SP_LOADS) {
    double x[SP_LOADS];
#pragma unroll
    for (int j = 0; j < SP_LOADS; ++j) {
      const int b = b0 + lane + 32 * j;
      x[j] = b < nb ? __ldcg(p + b) : 0.0;
    }
    s += ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
  }
  return warp_sum(s);
}

// hs[i] = sum over the grid's blocks of part[i nblk + b], i <= k; every block computes the
// same values in the same order.  Warp w takes vectors w, w + SW, ...  (one vector at a time:
// more in flight per warp measured slower, the registers they hold cost more than they save).
__device__ void sum_partials(const GmresDev& g, const double* __restrict__ part, int k, const StepSmem& sm) {
  const int nv = k + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < nv; i += SW) {
    const double t = warp_sum_blocks(part + (int64_t)i * g.nblk, g.nblk);
    if (lane == 0) sm.hs[i] = t;
  }
  __syncthreads();
}

// w = A z_k on this block's rows (the operator's second half, as in nbr_sum_kernel), V[k] *= s
// (the scale the previous step left), then partial h1 = V_k^T w.  The rows of w are formed tile
// by tile, just before the tile's dot pass.
__global__ void __launch_bounds__(ST) arn_wdots_kernel(GmresDev g, const int32_t* __restrict__ nbr,
                                                       const double* __restrict__ vext, int64_t n_nodes,
                                                       double diag, double invh2) {
  __shared__ __align__(8) uint64_t bar[2];
  pdl_launch_next();
  pdl_wait();
  const int q = blockIdx.y;
  const Rhs v = rhs_view(g, q);
  const SL L{g.m};
  const int4 st4 = load_state(v);
  const double s = __ldcg(v.st + L.sc() + S_VSCALE);
  if (st4.z) return;
  const StepSmem sm = step_smem();
  const int k = st4.x;
  int64_t r0;
  const int nr = block_rows(g, &r0);
  const VStream vs = make_stream(g, v.V, r0, nr, k + 1, 1, sm, bar);
  stream_begin(vs, bar);
  const double* zk = v.Z + (int64_t)k * g.ld + r0;
  const double* ve = vext + (int64_t)q * n_nodes;
  for (int qq = 0; qq < vs.total; ++qq) {
    if (vs.batch(qq) == 0) {          // a new tile (the previous tile's dot pass has finished)
      const int t = vs.tile(qq), rows = vs.rows(qq);
      for (int row = threadIdx.x; row < rows; row += ST) {
        const int64_t lr = (int64_t)t * TR + row;
        const int32_t* nb = nbr + 6 * (r0 + lr);
        const double e0 = __ldcg(ve + __ldg(nb + 0)), e1 = __ldcg(ve + __ldg(nb + 1));
        const double e2 = __ldcg(ve + __ldg(nb + 2)), e3 = __ldcg(ve + __ldg(nb + 3));
        const double e4 = __ldcg(ve + __ldg(nb + 4)), e5 = __ldcg(ve + __ldg(nb + 5));
        const double sn = ((e0 + e1) + (e2 + e3)) + (e4 + e5);
        const double wv = diag * __ldcg(zk + lr) - invh2 * sn;
        v.w[r0 + lr] = wv;
        sm.ws[row] = wv;
      }
    }
    if (!stream_wait(g, vs, qq)) return;
    dots_batch(vs, qq, sm, k > 0 ? k : -1, s, v.V + r0);
    __syncthreads();
    if (threadIdx.x == 0) vs.issue(qq + 2);
  }
  finish_dots(k + 1, sm, v.p1 + blockIdx.x, g.nblk);
}

// h1 = sum of the partials (block 0 keeps it for the Hessenberg column); w -= V_k h1; partial
// h2 = V_k^T w.  Per tile the stream passes over the basis twice (update, then dots; the second
// pass reads the rows the first one has just brought into L2).
__global__ void __launch_bounds__(ST) arn_upd1_kernel(GmresDev g) {
  __shared__ __align__(8) uint64_t bar[2];
  pdl_launch_next();
  pdl_wait();
  const int q = blockIdx.y;
  const Rhs v = rhs_view(g, q);
  const int4 st4 = load_state(v);
  if (st4.z) return;
  const StepSmem sm = step_smem();
  const int k = st4.x;
  const SL L{g.m};
  int64_t r0;
  const int nr = block_rows(g, &r0);
  const VStream vs = make_stream(g, v.V, r0, nr, k + 1, 2, sm, bar);
  stream_begin(vs, bar);
  sum_partials(g, v.p1, k, sm);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= k; i += ST) v.st[L.h1() + i] = sm.hs[i];
  double a[RU], wr[RU];
  for (int qq = 0; qq < vs.total; ++qq) {
    const int t = vs.tile(qq), rows = vs.rows(qq);
    double* wt = v.w + r0 + (int64_t)t * TR;
    if (vs.pass(qq) == 0 && vs.batch(qq) == 0) {   // a new tile: its rows of w, loaded early
#pragma unroll
      for (int j = 0; j < RU; ++j) {
        const int row = threadIdx.x + ST * j;
        a[j] = 0.0;
        wr[j] = row < rows ? __ldcg(wt + row) : 0.0;
      }
    }
    if (!stream_wait(g, vs, qq)) return;
    if (vs.pass(qq) == 0) {
      update_batch(vs, qq, sm, a);
      if (vs.batch(qq) == vs.nbatch - 1) {
#pragma unroll
        for (int j = 0; j < RU; ++j) {
          const int row = threadIdx.x + ST * j;
          if (row < rows) {
            const double wn = wr[j] - a[j];
            wt[row] = wn;
            sm.ws[row] = wn;
          }
        }
      }
    } else {
      dots_batch(vs, qq, sm, -1, 1.0, nullptr);
    }
    __syncthreads();
    if (threadIdx.x == 0) vs.issue(qq + 2);
  }
  finish_dots(k + 1, sm, v.p2 + blockIdx.x, g.nblk);
}

// h2 = sum of the partials; w -= V_k h2 into V[k+1] (unnormalised); ||w||^2; the last block
// adds the norm partials and finishes the step (Hessenberg column h1 + h2 and ||w||, the
// previous rotations, a new rotation, the residual estimate and the stopping test).
__global__ void __launch_bounds__(ST) arn_upd2_kernel(GmresDev g) {
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ bool last;
  __shared__ double wsum[SW];
  pdl_wait();
  const int q = blockIdx.y;
  const Rhs v = rhs_view(g, q);
  const int4 st4 = load_state(v);
  if (st4.z) return;
  const StepSmem sm = step_smem();
  const int k = st4.x;
  const SL L{g.m};
  int64_t r0;
  const int nr = block_rows(g, &r0);
  const VStream vs = make_stream(g, v.V, r0, nr, k + 1, 1, sm, bar);
  stream_begin(vs, bar);
  // the state the step's last block needs, loaded now (off the critical path): h1, the previous
  // rotations, g_k, ||f||, the tolerance and the iteration counters
  double* pre = sm.red + 1024;              // h1 [0, 128), cs [128, 256), sn [256, 384), scalars
  int* prei = reinterpret_cast<int*>(pre + 392);
  if (threadIdx.x >= 32 && threadIdx.x < 64) {
    const int l = threadIdx.x - 32;
    for (int i = l; i <= k; i += 32) pre[i] = __ldcg(v.st + L.h1() + i);
    for (int i = l; i < k; i += 32) {
      pre[128 + i] = __ldcg(v.st + L.cs() + i);
      pre[256 + i] = __ldcg(v.st + L.sn() + i);
    }
    if (l == 0) {
      pre[384] = __ldcg(v.st + L.g() + k);
      pre[385] = __ldcg(v.st + L.sc() + S_NF);
      pre[386] = __ldcg(v.st + L.sc() + S_TOL);
      prei[0] = st4.y;                                   // total
      prei[1] = __ldcg(v.ist + I_MAXIT);
    }
  }
  sum_partials(g, v.p2, k, sm);
  double acc[RU], wr[RU];
  double ss = 0.0;
  double* vn = v.V + (int64_t)(k + 1) * g.ld + r0;
  for (int qq = 0; qq < vs.total; ++qq) {
    const int t = vs.tile(qq), rows = vs.rows(qq);
    if (vs.batch(qq) == 0) {                      // a new tile: its rows of w, loaded early
#pragma unroll
      for (int j = 0; j < RU; ++j) {
        const int row = threadIdx.x + ST * j;
        acc[j] = 0.0;
        wr[j] = row < rows ? __ldcg(v.w + r0 + (int64_t)t * TR + row) : 0.0;
      }
    }
    if (!stream_wait(g, vs, qq)) return;
    update_batch(vs, qq, sm, acc);
    if (vs.batch(qq) == vs.nbatch - 1) {
#pragma unroll
      for (int j = 0; j < RU; ++j) {
        const int row = threadIdx.x + ST * j;
        if (row < rows) {
          const double wn = wr[j] - acc[j];
          vn[(int64_t)t * TR + row] = wn;
          ss = fma(wn, wn, ss);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) vs.issue(qq + 2);
  }
  const double bsum = block_sum<SW>(ss, wsum);
  if (threadIdx.x == 0) {
    v.p3[blockIdx.x] = bsum;
    __threadfence();
    last = atomicAdd(&v.ist[I_TICKET], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const double tot = warp_sum_blocks(v.p3, g.nblk);
  // Hessenberg column k = h1 + h2 (b) and the products of the previous rotations with it, formed
  // by the warp so that the rotation sweep below is one dependent FMA per rotation
  double* bcol = sm.red;                    // b_i, i <= k
  double* cb = sm.red + 128;                // cs_i b_{i+1}
  double* sb = sm.red + 256;                // sn_i b_{i+1}
  for (int i = lane; i <= k; i += 32) bcol[i] = pre[i] + sm.hs[i];
  __syncwarp();
  for (int i = lane; i < k; i += 32) {
    cb[i] = pre[128 + i] * bcol[i + 1];
    sb[i] = pre[256 + i] * bcol[i + 1];
  }
  __syncwarp();
  if (lane != 0) return;
  double* st = v.st;
  int* ist = v.ist;
  ist[I_TICKET] = 0;
  const double* csv = pre + 128;
  const double* snv = pre + 256;
  // previous rotations applied down the column: H(i,k) = c_i a + s_i b_{i+1}, and the rotated
  // entry i+1 = -s_i a + c_i b_{i+1} carries on in a register
  double cur = bcol[0];
#pragma unroll 4
  for (int i = 0; i < k; ++i) {
    const double a = cur;
    st[L.H(i, k)] = fma(csv[i], a, sb[i]);
    cur = fma(-snv[i], a, cb[i]);
  }
  // the new rotation zeroes ||w||: rho = sqrt(cur^2 + ||w||^2), formed from ||w||^2 directly so
  // that it does not wait for the square root of ||w||
  const double hn = sqrt(tot);
  const double rho = sqrt(fma(cur, cur, tot));
  // rho = 0 (then ||w|| = 0 too): A z_k lies in span(V_0 .. V_{k-1}) and the rotated column has
  // a zero diagonal, so the Hessenberg matrix is singular; the rotation is left as the identity
  // and column k is kept out of the least-squares solve below
  const bool singular = rho == 0.0;
  const double c = singular ? 1.0 : cur / rho, sv = singular ? 0.0 : hn / rho;
  st[L.cs() + k] = c;
  st[L.sn() + k] = sv;
  st[L.H(k, k)] = rho;
  st[L.H(k + 1, k)] = 0.0;
  const double gk = pre[384];
  st[L.g() + k + 1] = -sv * gk;
  st[L.g() + k] = c * gk;
  st[L.sc() + S_HN] = hn;
  st[L.sc() + S_VSCALE] = 1.0 / hn;
  const int total = prei[0] + 1;
  ist[I_TOTAL] = total;
  ist[I_KDONE] = k + 1;
  const double est = fabs(-sv * gk);
  const double nf = pre[385], tol = pre[386];
  bool stop = est <= tol * nf || hn == 0.0 || k + 1 >= g.m || total >= prei[1];
  // ||w|| = 0 ends the cycle (hn == 0 above); the restart test then reports CPM_ERR_BREAKDOWN
  // unless the true residual meets the tolerance.  A singular Hessenberg matrix updates u with
  // its first k columns only.
  if (singular) ist[I_KDONE] = k;
  if (!isfinite(hn) || !isfinite(rho) || !isfinite(est)) {
    ist[I_STATUS] = CPM_ERR_NAN;
    stop = true;
  }
  if (stop) {
    ist[I_DONE] = 1;
    ist[I_SLOT] = g.m;                     // later solves of the batch write the spare slot
    if (atomicSub(&g.ctl[C_LIVE], 1) == 1) g.ctl[C_ALLDONE] = 1;
  } else {
    ist[I_K] = k + 1;
    ist[I_SLOT] = k + 1;
  }
}

// ---- cycle start / restart ------------------------------------------------------------
// ||x_q||^2 over the blocks; the last block of right-hand side q applies the begin (which = 0:
// ||f||, tolerance, iteration limit) or the convergence test on beta = ||r|| (which = 1),
// which also opens the next cycle of a right-hand side that goes on.
__global__ void __launch_bounds__(KT) norm_kernel(GmresDev g, const double* __restrict__ x, int64_t x_stride,
                                                  int which, double tol, int max_it) {
  __shared__ bool last;
  __shared__ double wsum[KW];
  const int q = blockIdx.y;
  const Rhs v = rhs_view(g, q);
  const double* xq = x + (int64_t)q * x_stride;
  int64_t r0;
  const int nr = block_rows(g, &r0);
  double s = 0.0;
  for (int row = threadIdx.x; row < nr; row += KT) {
    const double a = xq[r0 + row];
    s = fma(a, a, s);
  }
  const double bsum = block_sum<KW>(s, wsum);
  if (threadIdx.x == 0) {
    v.p3[blockIdx.x] = bsum;
    __threadfence();
    last = atomicAdd(&v.ist[I_TICKET + 1], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x >= 32) return;
  double tot = 0.0;
  for (int b = threadIdx.x; b < g.nblk; b += 32) tot += __ldcg(v.p3 + b);
  tot = warp_sum(tot);
  if (threadIdx.x != 0) return;
  int* ist = v.ist;
  double* st = v.st;
  const SL L{g.m};
  ist[I_TICKET + 1] = 0;
  const double nrm = sqrt(tot);
  ist[I_KDONE] = 0;
  if (which == 0) {               // ||f||
    st[L.sc() + S_NF] = nrm;
    st[L.sc() + S_TOL] = tol;
    ist[I_MAXIT] = max_it;
    ist[I_TOTAL] = 0;
    ist[I_STATUS] = RUNNING;
    ist[I_DONE] = 1;
    ist[I_SLOT] = g.m;
    return;
  }
  const double beta = nrm;
  const double nf = st[L.sc() + S_NF];
  st[L.sc() + S_BETA] = beta;
  st[L.sc() + S_RELRES] = nf > 0.0 ? beta / nf : 0.0;
  if (ist[I_STATUS] == RUNNING) {
    if (!isfinite(beta)) {
      ist[I_STATUS] = CPM_ERR_NAN;
    } else if (nf == 0.0 || beta <= st[L.sc() + S_TOL] * nf) {
      ist[I_STATUS] = CPM_OK;
    } else if (ist[I_TOTAL] >= ist[I_MAXIT]) {
      ist[I_STATUS] = CPM_ERR_NOT_CONVERGED;
    } else if (ist[I_TOTAL] > 0 && st[L.sc() + S_HN] == 0.0) {
      ist[I_STATUS] = CPM_ERR_BREAKDOWN;
    }
  }
  if (ist[I_STATUS] != RUNNING) {
    ist[I_DONE] = 1;
    ist[I_SLOT] = g.m;
    return;
  }
  for (int i = 0; i <= g.m; ++i) st[L.g() + i] = 0.0;
  st[L.g()] = beta;
  st[L.sc() + S_VSCALE] = 1.0;
  ist[I_K] = 0;
  ist[I_SLOT] = 0;
  ist[I_DONE] = 0;
}

// V[0] = r / beta for every right-hand side that opens a cycle
__global__ void __launch_bounds__(KT) start_basis_kernel(GmresDev g) {
  const Rhs v = rhs_view(g, blockIdx.y);
  if (stopped(v)) return;
  const SL L{g.m};
  const double inv = 1.0 / v.st[L.sc() + S_BETA];
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT)
    v.V[row] = v.r[row] * inv;
}

// y = H[:kd,:kd]^{-1} g[:kd] (back substitution by one warp from a shared-memory copy of the
// triangle), one block per right-hand side
__global__ void ysolve_kernel(GmresDev g) {
  extern __shared__ __align__(16) double hsm[];          // kd x kd, column-major (ld kd)
  __shared__ double ys[129];
  const Rhs v = rhs_view(g, blockIdx.x);
  const SL L{g.m};
  const int kd = v.ist[I_KDONE];
  if (kd == 0) return;
  for (int e = threadIdx.x; e < kd * kd; e += blockDim.x) {
    const int i = e % kd, j = e / kd;
    hsm[e] = i <= j ? v.st[L.H(i, j)] : 0.0;
  }
  for (int i = threadIdx.x; i < kd; i += blockDim.x) ys[i] = v.st[L.g() + i];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  for (int j = kd - 1; j >= 0; --j) {
    const double yj = ys[j] / hsm[j + j * kd];
    __syncwarp();
    for (int i = threadIdx.x; i < j; i += 32) ys[i] = fma(-hsm[i + j * kd], yj, ys[i]);
    if (threadIdx.x == 0) ys[j] = yj;
    __syncwarp();
  }
  for (int i = threadIdx.x; i < kd; i += 32) v.st[L.y() + i] = ys[i];
}

// u += Z y (columns 0 .. kd-1), one thread per row
__global__ void __launch_bounds__(KT) xupdate_kernel(GmresDev g, double* u, int64_t u_stride) {
  const Rhs v = rhs_view(g, blockIdx.y);
  const SL L{g.m};
  const int kd = v.ist[I_KDONE];
  if (kd == 0) return;
  __shared__ double ys[128];
  for (int i = threadIdx.x; i < kd; i += KT) ys[i] = v.st[L.y() + i];
  __syncthreads();
  double* uq = u + (int64_t)blockIdx.y * u_stride;
  for (int64_t row = (int64_t)blockIdx.x * KT + threadIdx.x; row < g.n; row += (int64_t)gridDim.x * KT) {
    double a0 = 0.0, a1 = 0.0;
    int i = 0;
    for (; i + 1 < kd; i += 2) {
      a0 = fma(v.Z[(int64_t)i * g.ld + row], ys[i], a0);
      a1 = fma(v.Z[(int64_t)(i + 1) * g.ld + row], ys[i + 1], a1);
    }
    if (i < kd) a0 = fma(v.Z[(int64_t)i * g.ld + row], ys[i], a0);
    uq[row] += a0 + a1;
  }
}

int gmres_state_size(int m) { return SL{m}.sc() + 8; }
int gmres_scalar_offset(int m) { return SL{m}.sc(); }

static unsigned vec_blocks(int64_t n) {
  int64_t b = (n + KT - 1) / KT;
  return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

static size_t ysolve_smem(int m) { return sizeof(double) * (size_t)m * m; }

// The dynamic shared-memory limit is an attribute of the kernel function, shared by every
// handle in the process: it is set to the largest size any launch may ask for (the longest
// restart), never to one handle's size, which a later handle would exceed.
cudaError_t gmres_prepare(int m) {
  if (m > 128) return cudaErrorInvalidValue;
  const int step = (int)gmres_step_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(arn_wdots_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, step);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(arn_upd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, step);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(arn_upd2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, step);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ysolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysolve_smem(128));
  return e;
}

// kernel launch with programmatic stream serialisation (the kernel waits on its predecessor
// with griddepcontrol.wait)
template <typename... Args>
static cudaError_t launch_pdl(void (*kern)(Args...), dim3 grid, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(ST);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_gmres_begin(const GmresDev& g, const double* f, int64_t f_stride, double tol, int max_it,
                               int nr, cudaStream_t s) {
  norm_kernel<<<dim3(g.nblk, nr), KT, 0, s>>>(g, f, f_stride, 0, tol, max_it);
  return cudaGetLastError();
}

cudaError_t launch_arnoldi_step(const GmresDev& g, const OperatorDev& op, const double* vext, int nr,
                                cudaStream_t s) {
  const size_t smem = gmres_step_smem_bytes();
  const dim3 grid(g.nblk, nr);
  cudaError_t e = launch_pdl(arn_wdots_kernel, grid, smem, s, g, op.nbr, vext, op.n_nodes, op.diag, op.invh2);
  if (e == cudaSuccess) e = launch_pdl(arn_upd1_kernel, grid, smem, s, g);
  if (e == cudaSuccess) e = launch_pdl(arn_upd2_kernel, grid, smem, s, g);
  return e;
}

cudaError_t launch_gmres_restart_update(const GmresDev& g, double* u, int64_t u_stride, int nr, cudaStream_t s) {
  ysolve_kernel<<<nr, 128, ysolve_smem(g.m), s>>>(g);
  xupdate_kernel<<<dim3(vec_blocks(g.n), nr), KT, 0, s>>>(g, u, u_stride);
  return cudaGetLastError();
}

// after r = f - A u: beta, convergence decision, and V[0] = r / beta for the next cycle
cudaError_t launch_gmres_residual_check(const GmresDev& g, int nr, cudaStream_t s) {
  norm_kernel<<<dim3(g.nblk, nr), KT, 0, s>>>(g, g.r, g.ld, 1, 0.0, 0);
  start_basis_kernel<<<dim3(vec_blocks(g.n), nr), KT, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace cpmdev
