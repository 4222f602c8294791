// z = M^{-1} r for all subdomains in one persistent launch (Eq. algRAS):
//   restrict: b_j = P_j [R_j r ; 0]            (gather through the pivoted row map)
//   forward : L_j y_j = b_j                    (unit lower)
//   backward: U_j z_j = y_j
//   prolong : z[g] = z_j[loc(g)] for g in the disjoint set of j (restricted partition of
//             unity, Eq. restCons), so every global entry is written exactly once.
//
// Work items are (subdomain j, tile row I, direction): forward items by increasing I across
// all subdomains, then backward items by decreasing I.  A CTA takes items from a global
// counter and streams the off-diagonal tiles of its tile row through a shared-memory ring
// with 1-D bulk copies (TMA engine), then the precomputed inverse of the diagonal block.
// The solved 64-value pieces are published as 64-bit words carrying the launch's epoch tag
// next to the value, so a consumer polls the data itself: no separate flag, no fence.
// Every dependency of an item was dispensed earlier to a running CTA, so the scheme cannot
// deadlock; every wait is bounded and reports CPM_ERR_TIMEOUT instead of hanging.
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int TRSV_THREADS = 128;
constexpr int NSTAGE = 4;

__device__ __forceinline__ double cvt(double v) { return v; }
__device__ __forceinline__ float cvt(float v) { return v; }
__device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tagged publication of one value of a solved piece.
template <typename C> struct Tagged;
template <> struct Tagged<float> {
  static constexpr int WORDS = 1;
  __device__ static void put(uint64_t* p, float v, uint32_t tag) {
    st_relaxed_u64(p, ((uint64_t)tag << 32) | (uint64_t)__float_as_uint(v));
  }
  // returns true once the word carries tag
  __device__ static bool get(const uint64_t* p, uint32_t tag, float* v) {
    const uint64_t w = ld_relaxed_u64(p);
    if ((uint32_t)(w >> 32) != tag) return false;
    *v = __uint_as_float((uint32_t)w);
    return true;
  }
};
template <> struct Tagged<double> {
  static constexpr int WORDS = 2;
  __device__ static void put(uint64_t* p, double v, uint32_t tag) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    st_relaxed_u64(p, ((uint64_t)tag << 32) | (b >> 32));
    st_relaxed_u64(p + 1, ((uint64_t)tag << 32) | (b & 0xffffffffull));
  }
  __device__ static bool get(const uint64_t* p, uint32_t tag, double* v) {
    const uint64_t hi = ld_relaxed_u64(p), lo = ld_relaxed_u64(p + 1);
    if ((uint32_t)(hi >> 32) != tag || (uint32_t)(lo >> 32) != tag) return false;
    *v = __longlong_as_double((long long)(((hi & 0xffffffffull) << 32) | (lo & 0xffffffffull)));
    return true;
  }
};

// Poll one tagged value until it carries tag; false on abort or after the spin limit.
template <typename C>
__device__ __forceinline__ bool poll_value(const uint64_t* p, uint32_t tag, C* v, uint32_t* sync,
                                           int* status) {
  for (uint32_t spin = 0;; ++spin) {
    if (Tagged<C>::get(p, tag, v)) return true;
    if ((spin & 63) == 63) {
      if (*(volatile uint32_t*)&sync[3]) return false;
      if (spin > SPIN_LIMIT) {
        atomicOr(status, ST_TIMEOUT);
        atomicExch(&sync[3], 1u);
        return false;
      }
      __nanosleep(64);
    }
  }
}

template <typename S, typename C>
__global__ void __launch_bounds__(TRSV_THREADS) trsv_kernel(TrsvDev t, IndirectVec r_in, IndirectVec z_out,
                                                            const int* done) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr uint32_t TB_S = sizeof(S) * TILE_ELEMS;     // off-diagonal factor tile
  constexpr uint32_t TB_C = sizeof(C) * TILE_ELEMS;     // inverse diagonal tile
  constexpr uint32_t STAGE = TB_S > TB_C ? TB_S : TB_C;
  constexpr int W = Tagged<C>::WORDS;
  __shared__ __align__(8) uint64_t bar[NSTAGE];
  __shared__ C yb[64];
  __shared__ C red[TRSV_THREADS];
  __shared__ int sh_item, sh_mb;
  const int tid = threadIdx.x;
  const S* tiles = (const S*)t.tiles;
  const C* inv = (const C*)t.inv;
  if (tid == 0) {
    for (int q = 0; q < NSTAGE; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t epoch = *(volatile uint32_t*)&t.sync[2];
  const uint32_t tag_f = 2u * epoch + 1u, tag_b = 2u * epoch + 2u;
  const bool skip = done && *(volatile const int*)done;
  const double* rin = r_in.ptr(0);
  double* zout = z_out.ptr(0);
  uint32_t lc = 0, cc = 0;     // bulk copies issued / consumed by this CTA
  bool bad = false;
  const int r = tid & 63, half = tid >> 6;

  while (!bad) {
    if (tid == 0) sh_item = skip ? t.n_items : (int)atomicAdd(&t.sync[0], 1u);
    __syncthreads();
    const int item = sh_item;
    if (item >= t.n_items) break;
    const int2 it = t.items[item];
    const int j = it.x, I = it.y & 0x3fffffff, bwd = (it.y >> 30) & 1;
    const SubMeta m = t.meta[j];
    const int T = m.T;
    const int nt = bwd ? (T - I) : (I + 1);          // off-diagonal tiles, then the inverse
    const int64_t ro = m.row_off + 64 * I;
    const C* inv_tile = inv + (((m.row_off >> 6) + I) * 2 + bwd) * (int64_t)TILE_ELEMS;
    auto issue = [&](int q) {
      const int st = lc % NSTAGE;
      unsigned char* dst = smem + (size_t)st * STAGE;
      if (q == nt - 1) {
        mbar_expect_tx(&bar[st], TB_C);
        bulk_g2s(dst, inv_tile, TB_C, &bar[st]);
      } else {
        const int J = bwd ? T - 1 - q : q;
        mbar_expect_tx(&bar[st], TB_S);
        bulk_g2s(dst, tiles + tile_base(m, I, J), TB_S, &bar[st]);
      }
    };
    const int pre = nt < NSTAGE ? nt : NSTAGE;
    if (tid == 0)
      for (int q = 0; q < pre; ++q) { issue(q); ++lc; }
    lc = cc + pre;                               // every thread tracks lc for the drain path
    // restrict: prefetch this row's right-hand side (forward items)
    C rhs = (C)0;
    if (!bwd && tid < 64) {
      const int g = t.gather[ro + tid];
      if (g >= 0) rhs = (C)rin[g];
    }
    C acc = (C)0;
    for (int q = 0; q < nt; ++q) {
      const int st = cc % NSTAGE;
      if (tid == 0) {
        const bool ok = mbar_wait_bounded(&bar[st], (cc / NSTAGE) & 1);
        if (!ok) { atomicOr(t.status, ST_TIMEOUT); atomicExch(&t.sync[3], 1u); }
        sh_mb = ok ? 0 : 1;
      }
      __syncthreads();
      if (sh_mb) { bad = true; break; }
      mbar_wait_bounded(&bar[st], (cc / NSTAGE) & 1);   // already complete: returns at once
      const unsigned char* stage = smem + (size_t)st * STAGE;
      if (q < nt - 1) {
        // off-diagonal tile (I, J): needs the solved piece J of this direction
        const int J = bwd ? T - 1 - q : q;
        bool ok = true;
        if (tid < 64) {
          C v;
          ok = poll_value<C>(t.ytag + (m.row_off + 64 * J + tid) * W, bwd ? tag_b : tag_f, &v,
                             t.sync, t.status);
          yb[tid] = ok ? v : (C)0;
        }
        if (!__syncthreads_and(ok)) { bad = true; cc++; break; }
        const S* tile = (const S*)stage;
#pragma unroll 8
        for (int c = 32 * half; c < 32 * half + 32; ++c)
          acc += (C)cvt(tile[Layout<S>::off(r, c)]) * yb[c];
      } else {
        // diagonal block through its inverse: x = Inv (b - partial sums)
        red[tid] = acc;
        bool ok = true;
        C own = (C)0;
        if (bwd && tid < 64)
          ok = poll_value<C>(t.ytag + (ro + tid) * W, tag_f, &own, t.sync, t.status);
        if (!__syncthreads_and(ok)) { bad = true; cc++; break; }
        if (tid < 64) yb[tid] = (bwd ? own : rhs) - (red[tid] + red[tid + 64]);
        __syncthreads();
        const C* iv = (const C*)stage;
        C part = (C)0;
#pragma unroll 8
        for (int c = 32 * half; c < 32 * half + 32; ++c) part += iv[off_plain(r, c)] * yb[c];
        red[tid] = part;
        __syncthreads();
        if (tid < 64) {
          const C x = red[tid] + red[tid + 64];
          Tagged<C>::put(t.ytag + (ro + tid) * W, x, bwd ? tag_b : tag_f);
          if (bwd) {
            const int s = t.scatter[ro + tid];
            if (s >= 0) zout[s] = (double)x;
          }
        }
      }
      __syncthreads();               // stage st fully consumed, yb / red free again
      cc++;
      if (tid == 0 && q + NSTAGE < nt) issue(q + NSTAGE);
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

template <typename S, typename C> constexpr size_t stage_bytes() {
  return (sizeof(S) > sizeof(C) ? sizeof(S) : sizeof(C)) * TILE_ELEMS;
}

int trsv_ctas_per_sm(int precision) {
  // 4-stage ring: fp64 128 KB, fp32 and bf16 (float inverse tiles) 64 KB per CTA
  return precision == 0 ? 1 : 3;
}

cudaError_t trsv_prepare(int precision) {
  if (precision == 0)
    return cudaFuncSetAttribute(trsv_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(NSTAGE * stage_bytes<double, double>()));
  if (precision == 1)
    return cudaFuncSetAttribute(trsv_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(NSTAGE * stage_bytes<float, float>()));
  return cudaFuncSetAttribute(trsv_kernel<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(NSTAGE * stage_bytes<__nv_bfloat16, float>()));
}

cudaError_t launch_trsv(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done,
                        cudaStream_t s) {
  if (t.precision == 0)
    trsv_kernel<double, double><<<t.grid, TRSV_THREADS, NSTAGE * stage_bytes<double, double>(), s>>>(
        t, r_in, z_out, done);
  else if (t.precision == 1)
    trsv_kernel<float, float><<<t.grid, TRSV_THREADS, NSTAGE * stage_bytes<float, float>(), s>>>(
        t, r_in, z_out, done);
  else
    trsv_kernel<__nv_bfloat16, float>
        <<<t.grid, TRSV_THREADS, NSTAGE * stage_bytes<__nv_bfloat16, float>(), s>>>(t, r_in, z_out, done);
  return cudaGetLastError();
}

}  // namespace cpmdev
