// z = M^{-1} r for all subdomains in one persistent launch (Eq. algRAS):
//   restrict: b_j = P_j [R_j r ; 0]            (gather through the pivoted row map)
//   forward : L_j y_j = b_j                    (unit lower)
//   backward: U_j z_j = y_j
//   prolong : z[g] = z_j[loc(g)] for g in the disjoint set of j (restricted partition of
//             unity, Eq. restCons), so every global entry is written exactly once.
//
// Work items are (subdomain j, tile row I, direction), queued forward items by increasing
// I across all subdomains, then backward items by decreasing I.  A CTA takes items from a
// global counter; the tiles of its tile row stream through a shared-memory ring by 1-D bulk
// copies (TMA engine) while the right-hand-side pieces it multiplies are published by
// other CTAs through per-tile-row flags (release/acquire).  Every dependency of an item was
// dispensed earlier to a running CTA, so the scheme cannot deadlock; every wait is bounded
// and reports CPM_ERR_TIMEOUT instead of hanging.
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int TRSV_THREADS = 128;
constexpr int NSTAGE = 4;

template <typename C> __device__ __forceinline__ C ld_cg(const C* p);
template <> __device__ __forceinline__ double ld_cg<double>(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<float>(const float* p) { return __ldcg(p); }

__device__ __forceinline__ double cvt(double v) { return v; }
__device__ __forceinline__ float cvt(float v) { return v; }
__device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S, typename C> __device__ __forceinline__ C tval(const S* t, int i, int j) {
  return (C)cvt(t[Layout<S>::off(i, j)]);
}

template <typename S, typename C>
__global__ void __launch_bounds__(TRSV_THREADS) trsv_kernel(TrsvDev t, IndirectVec r_in, IndirectVec z_out,
                                                            const int* done) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr uint32_t TB = sizeof(S) * TILE_ELEMS;
  S* ring = (S*)smem;
  __shared__ __align__(8) uint64_t bar[NSTAGE];
  __shared__ C yb[64];
  __shared__ C red[TRSV_THREADS];
  __shared__ int sh_item, sh_mb, sh_fl;   // item, copy-wait failure, flag-wait failure
  const int tid = threadIdx.x;
  const S* tiles = (const S*)t.tiles;
  const C* dinv = (const C*)t.dinv;
  C* ys = (C*)t.y;
  if (tid == 0) {
    for (int q = 0; q < NSTAGE; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t target = *(volatile uint32_t*)&t.sync[2] + 1u;
  const bool skip = done && *(volatile const int*)done;
  const double* rin = r_in.ptr(0);
  double* zout = z_out.ptr(0);
  uint32_t lc = 0, cc = 0;     // bulk copies issued / consumed by this CTA
  bool bad = false;

  while (!bad) {
    if (tid == 0) sh_item = skip ? t.n_items : (int)atomicAdd(&t.sync[0], 1u);
    __syncthreads();
    const int item = sh_item;
    if (item >= t.n_items) break;
    const int2 it = t.items[item];
    const int j = it.x, I = it.y & 0x3fffffff, bwd = (it.y >> 30) & 1;
    const SubMeta m = t.meta[j];
    const int T = m.T;
    const int nt = bwd ? (T - I) : (I + 1);          // tiles in this row, diagonal last
    uint32_t* fl_fwd = t.flags + t.flag_off[j];
    uint32_t* fl_bwd = fl_fwd + T;
    uint32_t* fl_mine = bwd ? fl_bwd : fl_fwd;
    auto col_of = [&](int q) { return q == nt - 1 ? I : (bwd ? T - 1 - q : q); };
    if (tid == 0)
      for (int q = 0; q < nt && q < NSTAGE; ++q) {
        const int st = (lc) % NSTAGE;
        mbar_expect_tx(&bar[st], TB);
        bulk_g2s(ring + st * TILE_ELEMS, tiles + tile_base(m, I, col_of(q)), TB, &bar[st]);
        ++lc;
      }
    // every thread tracks lc for the drain path
    lc = cc + (nt < NSTAGE ? nt : NSTAGE);
    C acc = (C)0;
    const int r = tid & 63, half = tid >> 6;
    for (int q = 0; q < nt; ++q) {
      const int st = cc % NSTAGE;
      // thread 0 waits (bounded) first so that every thread takes the same branch
      if (tid == 0) {
        const bool ok = mbar_wait_bounded(&bar[st], (cc / NSTAGE) & 1);
        if (!ok) { atomicOr(t.status, ST_TIMEOUT); atomicExch(&t.sync[3], 1u); }
        sh_mb = ok ? 0 : 1;
      }
      __syncthreads();
      if (sh_mb) { bad = true; break; }
      mbar_wait_bounded(&bar[st], (cc / NSTAGE) & 1);   // already complete: returns at once
      const S* tile = ring + st * TILE_ELEMS;
      if (q < nt - 1) {
        // off-diagonal tile: needs the solved piece of tile column J
        const int J = col_of(q);
        if (tid == 0) {
          uint32_t* f = fl_mine + J;
          int b = 0;
          for (uint32_t spin = 0; (int)(ld_acquire(f) - target) < 0; ++spin) {
            if (*(volatile uint32_t*)&t.sync[3]) { b = 1; break; }
            if (spin > SPIN_LIMIT) { atomicOr(t.status, ST_TIMEOUT); atomicExch(&t.sync[3], 1u); b = 1; break; }
            if (spin > 32) __nanosleep(128);
          }
          sh_fl = b;
        }
        __syncthreads();
        if (sh_fl) { bad = true; cc++; break; }
        if (tid < 64) yb[tid] = ld_cg(ys + m.row_off + 64 * J + tid);
        __syncthreads();
#pragma unroll 8
        for (int c = 32 * half; c < 32 * half + 32; ++c) acc += tval<S, C>(tile, r, c) * yb[c];
      } else {
        red[tid] = acc;
        if (bwd && tid == 0) {
          // the forward piece of this row (finished before any backward item of j began,
          // but wait on its flag anyway)
          uint32_t* f = fl_fwd + I;
          int b = 0;
          for (uint32_t spin = 0; (int)(ld_acquire(f) - target) < 0; ++spin) {
            if (*(volatile uint32_t*)&t.sync[3]) { b = 1; break; }
            if (spin > SPIN_LIMIT) { atomicOr(t.status, ST_TIMEOUT); atomicExch(&t.sync[3], 1u); b = 1; break; }
            if (spin > 32) __nanosleep(128);
          }
          sh_fl = b;
        } else if (tid == 0) {
          sh_fl = 0;
        }
        __syncthreads();
        if (sh_fl) { bad = true; cc++; break; }
        if (tid < 32) {
          const int l = tid;
          const int64_t ro = m.row_off + 64 * I;
          C b0, b1;
          if (!bwd) {
            const int g0 = t.gather[ro + l], g1 = t.gather[ro + l + 32];
            b0 = (g0 >= 0 ? (C)rin[g0] : (C)0) - (red[l] + red[l + 64]);
            b1 = (g1 >= 0 ? (C)rin[g1] : (C)0) - (red[l + 32] + red[l + 96]);
            // unit lower triangular diagonal block: forward substitution
#pragma unroll 4
            for (int c = 0; c < 63; ++c) {
              const C xc = __shfl_sync(0xffffffffu, c < 32 ? b0 : b1, c & 31);
              if (l > c) b0 -= tval<S, C>(tile, l, c) * xc;
              if (l + 32 > c) b1 -= tval<S, C>(tile, l + 32, c) * xc;
            }
          } else {
            b0 = ld_cg(ys + ro + l) - (red[l] + red[l + 64]);
            b1 = ld_cg(ys + ro + l + 32) - (red[l + 32] + red[l + 96]);
            const C d0 = dinv[ro + l], d1 = dinv[ro + l + 32];
            // upper triangular diagonal block: back substitution
#pragma unroll 4
            for (int c = 63; c >= 0; --c) {
              if (l == (c & 31)) {
                if (c >= 32) b1 = b1 * d1;
                else b0 = b0 * d0;
              }
              const C zc = __shfl_sync(0xffffffffu, c < 32 ? b0 : b1, c & 31);
              if (l < c) b0 -= tval<S, C>(tile, l, c) * zc;
              if (l + 32 < c) b1 -= tval<S, C>(tile, l + 32, c) * zc;
            }
            const int s0 = t.scatter[ro + l], s1 = t.scatter[ro + l + 32];
            if (s0 >= 0) zout[s0] = (double)b0;
            if (s1 >= 0) zout[s1] = (double)b1;
          }
          __stcg(ys + ro + l, b0);
          __stcg(ys + ro + l + 32, b1);
        }
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release(fl_mine + I, target);
        }
      }
      __syncthreads();               // stage st fully consumed
      cc++;
      if (tid == 0 && q + NSTAGE < nt) {
        const int st2 = lc % NSTAGE;
        mbar_expect_tx(&bar[st2], TB);
        bulk_g2s(ring + st2 * TILE_ELEMS, tiles + tile_base(m, I, col_of(q + NSTAGE)), TB, &bar[st2]);
      }
      if (q + NSTAGE < nt) lc++;
    }
  }
  // drain copies still in flight (only after an abort), then account for this CTA
  while (cc < lc) {
    mbar_wait_bounded(&bar[cc % NSTAGE], (cc / NSTAGE) & 1);
    cc++;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const uint32_t fin = atomicAdd(&t.sync[1], 1u);
    if (fin == gridDim.x - 1) {        // last CTA: reset the queue, advance the epoch
      t.sync[0] = 0u;
      t.sync[1] = 0u;
      t.sync[3] = 0u;
      __threadfence();
      atomicAdd(&t.sync[2], 1u);
    }
  }
}

int trsv_ctas_per_sm(int precision) {
  // 4-stage ring: fp64 128 KB, fp32 64 KB, bf16 32 KB of shared memory per CTA
  return precision == 0 ? 1 : (precision == 1 ? 3 : 6);
}

cudaError_t trsv_prepare(int precision) {
  if (precision == 0)
    return cudaFuncSetAttribute(trsv_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(NSTAGE * sizeof(double) * TILE_ELEMS));
  if (precision == 1)
    return cudaFuncSetAttribute(trsv_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(NSTAGE * sizeof(float) * TILE_ELEMS));
  return cudaFuncSetAttribute(trsv_kernel<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(NSTAGE * sizeof(__nv_bfloat16) * TILE_ELEMS));
}

cudaError_t launch_trsv(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done,
                        cudaStream_t s) {
  if (t.precision == 0)
    trsv_kernel<double, double><<<t.grid, TRSV_THREADS, NSTAGE * sizeof(double) * TILE_ELEMS, s>>>(
        t, r_in, z_out, done);
  else if (t.precision == 1)
    trsv_kernel<float, float><<<t.grid, TRSV_THREADS, NSTAGE * sizeof(float) * TILE_ELEMS, s>>>(
        t, r_in, z_out, done);
  else
    trsv_kernel<__nv_bfloat16, float><<<t.grid, TRSV_THREADS, NSTAGE * sizeof(__nv_bfloat16) * TILE_ELEMS, s>>>(
        t, r_in, z_out, done);
  return cudaGetLastError();
}

}  // namespace cpmdev
