// z = M^{-1} r for all subdomains in one persistent launch (Eq. algRAS):
//   restrict: b_j = P_j [R_j r ; 0]            (gather through the pivoted row map)
//   forward : L_j y_j = b_j                    (unit lower)
//   backward: U_j z_j = y_j
//   prolong : z[g] = z_j[loc(g)] for g in the disjoint set of j (restricted partition of
//             unity, Eq. restCons), so every global entry is written exactly once.
//
// Work items.  Tile row I of subdomain j needs p = I (forward) or T-1-I (backward)
// off-diagonal 64x64 tiles.  They are split into segments of at most kseg tiles: every
// segment but the last is a "partial" item that publishes the partial product of its tiles
// with the solved pieces; the last segment is the "diagonal" item, which adds the partials,
// applies the precomputed inverse of the diagonal block and publishes the solved piece of
// row I.  Items are queued forward-then-backward, each direction sorted by the chain
// position they wait for.
//
// Streaming.  Each CTA holds its current item and the next one; thread 0 keeps a ring of
// NSTAGE shared-memory stages filled with 1-D bulk copies (TMA engine) across the item
// boundary, so the next item's tiles are already arriving while the current item waits
// for its last dependency.  Solved pieces and partial sums are published as 64-bit words
// that carry the launch epoch as a tag next to the value: consumers poll the data itself.
//
// Progress.  Every dependency of an item was dispensed earlier; the earliest unfinished
// item is always some CTA's current item and all of its dependencies are finished, so the
// scheme cannot deadlock.  Every wait is bounded and reports CPM_ERR_TIMEOUT instead.
#include <algorithm>
#include <tuple>

#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int TRSV_THREADS = 128;
constexpr int NSTAGE = 4;
constexpr int SEG_DIAG = 0x3ff;

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

// Tagged publication of one value.
template <typename C> struct Tagged;
// load() issues the word loads (their latency can overlap other work); check() accepts them
// if they carry the expected tag.
template <> struct Tagged<float> {
  static constexpr int WORDS = 1;
  struct Raw { uint64_t w; };
  __device__ static void put(uint64_t* p, float v, uint32_t tag) {
    st_relaxed_u64(p, ((uint64_t)tag << 32) | (uint64_t)__float_as_uint(v));
  }
  __device__ static Raw load(const uint64_t* p) { return Raw{ld_relaxed_u64(p)}; }
  __device__ static bool check(const Raw& r, uint32_t tag, float* v) {
    if ((uint32_t)(r.w >> 32) != tag) return false;
    *v = __uint_as_float((uint32_t)r.w);
    return true;
  }
  __device__ static bool get(const uint64_t* p, uint32_t tag, float* v) { return check(load(p), tag, v); }
};
template <> struct Tagged<double> {
  static constexpr int WORDS = 2;
  struct Raw { uint64_t hi, lo; };
  __device__ static void put(uint64_t* p, double v, uint32_t tag) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    st_relaxed_u64(p, ((uint64_t)tag << 32) | (b >> 32));
    st_relaxed_u64(p + 1, ((uint64_t)tag << 32) | (b & 0xffffffffull));
  }
  __device__ static Raw load(const uint64_t* p) { return Raw{ld_relaxed_u64(p), ld_relaxed_u64(p + 1)}; }
  __device__ static bool check(const Raw& r, uint32_t tag, double* v) {
    if ((uint32_t)(r.hi >> 32) != tag || (uint32_t)(r.lo >> 32) != tag) return false;
    *v = __longlong_as_double((long long)(((r.hi & 0xffffffffull) << 32) | (r.lo & 0xffffffffull)));
    return true;
  }
  __device__ static bool get(const uint64_t* p, uint32_t tag, double* v) { return check(load(p), tag, v); }
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

// Decoded work item.
struct Item {
  int j, I, seg, bwd;
  int T, p, nseg, q0, nq, nload;
  bool diag;
};

template <int PIECES>
__device__ __forceinline__ Item decode(const TrsvDev& t, int idx) {
  Item e;
  const int2 it = t.items[idx];
  e.j = it.x;
  e.I = it.y & 0xfffff;
  e.seg = (it.y >> 20) & 0x3ff;
  e.bwd = (it.y >> 30) & 1;
  e.diag = e.seg == SEG_DIAG;
  e.T = t.meta[e.j].T;
  e.p = e.bwd ? e.T - 1 - e.I : e.I;
  const int K = t.kseg;
  e.nseg = e.p > 0 ? (e.p + K - 1) / K : 1;
  e.q0 = e.diag ? (e.nseg - 1) * K : e.seg * K;
  e.nq = e.diag ? e.p - e.q0 : K;
  e.nload = e.nq + (e.diag ? PIECES : 0);
  return e;
}

template <typename S, typename C>
__global__ void __launch_bounds__(TRSV_THREADS) trsv_kernel(TrsvDev t, IndirectVec r_in, IndirectVec z_out,
                                                            const int* done) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr uint32_t STAGE = sizeof(S) * TILE_ELEMS;          // one factor tile per stage
  constexpr int PIECES = (int)(sizeof(C) / sizeof(S));        // stages per inverse tile
  constexpr int W = Tagged<C>::WORDS;
  constexpr int CPS = STAGE / sizeof(C);                      // C values per stage
  static_assert(PIECES >= 1 && PIECES <= 2 && NSTAGE >= PIECES, "ring too small");
  __shared__ __align__(8) uint64_t bar[NSTAGE];
  __shared__ C yb[2][64];                                     // solved pieces, double-buffered
  __shared__ C xb[64];
  __shared__ C red[TRSV_THREADS], red2[TRSV_THREADS];
  __shared__ int sh_cur, sh_mb;
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
  uint32_t cc = 0;                 // stages consumed (all threads)
  bool bad = false;
  const int r = tid & 63, half = tid >> 6;

  // ---- producer state (thread 0 only): current / next item and the issue position ----
  uint32_t lc = 0;                 // stages issued
  int p_cur = -1, p_next = -1;     // item indices held by this CTA
  Item pi_cur{}, pi_next{};
  int issue_slot = 0, issue_l = 0; // issuing load issue_l of item (0: current, 1: next)
  auto fetch = [&]() -> int {
    if (skip) return t.n_items;
    return (int)atomicAdd(&t.sync[0], 1u);
  };
  auto issue_load = [&](const Item& e, int l) {
    const int st = lc % NSTAGE;
    unsigned char* dst = smem + (size_t)st * STAGE;
    mbar_expect_tx(&bar[st], STAGE);
    const SubMeta m = t.meta[e.j];
    if (l < e.nq) {
      const int q = e.q0 + l;
      const int J = e.bwd ? e.T - 1 - q : q;
      bulk_g2s(dst, tiles + tile_base(m, e.I, J), STAGE, &bar[st]);
    } else {
      const int64_t trow = (m.row_off >> 6) + e.I;
      const unsigned char* it = (const unsigned char*)(inv + (trow * 2 + e.bwd) * (int64_t)TILE_ELEMS);
      bulk_g2s(dst, it + (size_t)(l - e.nq) * STAGE, STAGE, &bar[st]);
    }
    ++lc;
  };
  auto pump = [&]() {               // keep the ring full (across the item boundary)
    while (lc - cc < NSTAGE) {
      if (issue_slot == 0 && issue_l >= pi_cur.nload) {
        if (!t.prefetch) break;
        issue_slot = 1;
        issue_l = 0;
      }
      if (issue_slot == 0) { issue_load(pi_cur, issue_l++); continue; }
      if (p_next >= t.n_items || issue_l >= pi_next.nload) break;
      issue_load(pi_next, issue_l++);
    }
  };
  if (tid == 0) {
    p_cur = fetch();
    if (p_cur < t.n_items) {
      pi_cur = decode<PIECES>(t, p_cur);
      if (t.prefetch) {
        p_next = fetch();
        if (p_next < t.n_items) pi_next = decode<PIECES>(t, p_next);
      }
      pump();
    }
    sh_cur = p_cur;
  }
  __syncthreads();

  // every thread waits (bounded) for stage c itself; a failed wait raises the abort word and
  // is folded into the next block-wide vote
  auto stage_ready = [&](uint32_t c) -> bool {
    const bool ok = mbar_wait_bounded(&bar[c % NSTAGE], (c / NSTAGE) & 1);
    if (!ok) { atomicOr(t.status, ST_TIMEOUT); atomicExch(&t.sync[3], 1u); }
    return ok;
  };

  while (!bad) {
    const int idx = sh_cur;
    if (idx >= t.n_items) break;
    const Item e = decode<PIECES>(t, idx);
    const SubMeta m = t.meta[e.j];
    const int64_t ro = m.row_off + 64 * e.I;
    const int64_t trow = (m.row_off >> 6) + e.I;
    const uint32_t tag = e.bwd ? tag_b : tag_f;
    // restrict: prefetch this row's right-hand side (forward diagonal items)
    C rhs = (C)0;
    if (e.diag && !e.bwd && tid < 64) {
      const int g = t.gather[ro + tid];
      if (g >= 0) rhs = (C)rin[g];
    }
    // tagged words of the solved piece multiplying off-diagonal tile l of this item
    auto ywords = [&](int l) {
      const int q = e.q0 + l;
      const int J = e.bwd ? e.T - 1 - q : q;
      return t.ytag + (m.row_off + 64 * J + tid) * W;
    };
    typename Tagged<C>::Raw pre{};
    if (tid < 64 && e.nq > 0) pre = Tagged<C>::load(ywords(0));
    C acc = (C)0, psum = (C)0;
    for (int l = 0; l < e.nq; ++l) {
      const bool staged = stage_ready(cc);
      bool ok = staged;
      if (tid < 64) {
        // the last tile of a diagonal item waits for the chain; collect the partial sums
        // of the other segments first (they are normally ready by then)
        if (e.diag && l == e.nq - 1)
          for (int s = 0; s < e.nseg - 1 && ok; ++s) {
            C v;
            ok = poll_value<C>(t.ptag + ((trow * t.maxseg + s) * 64 + tid) * W, tag, &v, t.sync, t.status);
            psum += v;
          }
        // the words were loaded one tile earlier; poll only if they were not yet published
        C v = (C)0;
        if (ok && !Tagged<C>::check(pre, tag, &v)) ok = poll_value<C>(ywords(l), tag, &v, t.sync, t.status);
        yb[l & 1][tid] = v;
        if (l + 1 < e.nq) pre = Tagged<C>::load(ywords(l + 1));
      }
      if (!__syncthreads_and(ok)) {
        bad = true;
        if (tid == 0 && staged) cc++;
        break;
      }
      if (tid == 0) pump();            // every thread is past tile l-1: its stage is free
      const S* tile = (const S*)(smem + (size_t)(cc % NSTAGE) * STAGE);
      const C* y = yb[l & 1];
#pragma unroll 8
      for (int c = 32 * half; c < 32 * half + 32; ++c)
        acc += (C)cvt(tile[Layout<S>::off(r, c)]) * y[c];
      cc++;
    }
    if (bad) break;
    if (!e.diag) {
      red[tid] = acc;
      __syncthreads();
      if (tid < 64)
        Tagged<C>::put(t.ptag + ((trow * t.maxseg + e.seg) * 64 + tid) * W, red[tid] + red[tid + 64], tag);
    } else {
      // diagonal block through its inverse: x = Inv (b - off-diagonal products)
      red[tid] = acc;
      bool ok = true;
      if (e.nq == 0 && tid < 64)        // no own tile (first row of a sweep): no partials
        psum = (C)0;
      C own = rhs;
      if (e.bwd && tid < 64) ok = poll_value<C>(t.ytag + (ro + tid) * W, tag_f, &own, t.sync, t.status);
      int staged = 0;
      for (int k = 0; k < PIECES && ok; ++k) {
        const bool sk = stage_ready(cc + k);
        staged += sk;
        ok = sk;
      }
      if (!__syncthreads_and(ok)) {
        bad = true;
        if (tid == 0) cc += staged;
        break;
      }
      if (tid < 64) xb[tid] = own - ((red[tid] + red[tid + 64]) + psum);
      __syncthreads();
      C part = (C)0;
#pragma unroll 8
      for (int c = 32 * half; c < 32 * half + 32; ++c) {
        const int el = c * 64 + r;                      // column-major inverse element
        const C* piece = (const C*)(smem + (size_t)((cc + el / CPS) % NSTAGE) * STAGE);
        part += piece[el % CPS] * xb[c];
      }
      red2[tid] = part;
      __syncthreads();
      if (tid < 64) {
        const C x = red2[tid] + red2[tid + 64];
        Tagged<C>::put(t.ytag + (ro + tid) * W, x, tag);
        if (e.bwd) {
          const int s = t.scatter[ro + tid];
          if (s >= 0) zout[s] = (double)x;
        }
      }
      cc += PIECES;
    }
    // advance: the next item becomes current, fetch a new next one, keep the ring full
    if (tid == 0) {
      if (t.prefetch) {
        p_cur = p_next;
        pi_cur = pi_next;
        if (issue_slot == 1) issue_slot = 0;
        else issue_l = 0;
        if (p_cur < t.n_items) {
          p_next = fetch();
          if (p_next < t.n_items) pi_next = decode<PIECES>(t, p_next);
        }
      } else {
        p_cur = fetch();
        if (p_cur < t.n_items) pi_cur = decode<PIECES>(t, p_cur);
        issue_slot = 0;
        issue_l = 0;
      }
      if (p_cur < t.n_items) pump();
      sh_cur = p_cur;
    }
    __syncthreads();
  }
  // drain copies still in flight (only after an abort), then account for this CTA
  if (tid == 0)
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

// stagger = 0: all forward items, then all backward items, each sorted by the chain position
// they wait for.  stagger = 1: one queue for both sweeps, sorted by that position plus a
// per-subdomain offset (odd subdomains start half a sweep later, and a subdomain's backward
// positions follow its whole forward sweep), so the start and the tail of one subdomain's
// sweep overlap with bulk work of others.  Either way every dependency of an item sorts
// before it.
void trsv_build_items(const int* T, int n_sub, int kseg, int stagger, std::vector<int2>& items,
                      int* maxseg) {
  items.clear();
  int ms = 1;
  std::vector<std::tuple<int, int, int, int, int, int>> q;   // key, kind, j, I, seg, bwd
  for (int bwd = 0; bwd < 2; ++bwd)
    for (int j = 0; j < n_sub; ++j) {
      const int off = stagger ? ((j & 1) ? T[j] / 2 : 0) + (bwd ? T[j] : 0)
                              : (bwd ? 1 << 24 : 0);
      for (int I = 0; I < T[j]; ++I) {
        const int p = bwd ? T[j] - 1 - I : I;
        const int nseg = p > 0 ? (p + kseg - 1) / kseg : 1;
        ms = std::max(ms, nseg);
        for (int s = 0; s < nseg - 1; ++s) q.emplace_back(off + s * kseg + kseg - 1, 0, j, I, s, bwd);
        q.emplace_back(off + p - 1, 1, j, I, SEG_DIAG, bwd);
      }
    }
  std::sort(q.begin(), q.end());
  for (auto& e : q)
    items.push_back(make_int2(std::get<2>(e), std::get<3>(e) | (std::get<4>(e) << 20) | (std::get<5>(e) << 30)));
  *maxseg = ms;
}

template <typename S, typename C> constexpr size_t ring_bytes() { return NSTAGE * sizeof(S) * TILE_ELEMS; }

int trsv_ctas_per_sm(int precision) {
  // 4-stage ring: fp64 128 KB, fp32 64 KB, bf16 32 KB of shared memory per CTA
  return precision == 0 ? 1 : (precision == 1 ? 3 : 6);
}

cudaError_t trsv_prepare(int precision) {
  if (precision == 0)
    return cudaFuncSetAttribute(trsv_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ring_bytes<double, double>());
  if (precision == 1)
    return cudaFuncSetAttribute(trsv_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ring_bytes<float, float>());
  return cudaFuncSetAttribute(trsv_kernel<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ring_bytes<__nv_bfloat16, float>());
}

cudaError_t launch_trsv(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done,
                        cudaStream_t s) {
  if (t.precision == 0)
    trsv_kernel<double, double><<<t.grid, TRSV_THREADS, ring_bytes<double, double>(), s>>>(t, r_in, z_out, done);
  else if (t.precision == 1)
    trsv_kernel<float, float><<<t.grid, TRSV_THREADS, ring_bytes<float, float>(), s>>>(t, r_in, z_out, done);
  else
    trsv_kernel<__nv_bfloat16, float>
        <<<t.grid, TRSV_THREADS, ring_bytes<__nv_bfloat16, float>(), s>>>(t, r_in, z_out, done);
  return cudaGetLastError();
}

}  // namespace cpmdev
