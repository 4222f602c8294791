// z = M^{-1} r for all subdomains in one persistent launch (Eq. algRAS):
//   restrict: b_j = P_j [R_j r ; 0]            (gather through the pivoted row map)
//   forward : L_j y_j = b_j                    (unit lower)
//   backward: U_j z_j = y_j
//   prolong : z[g] = z_j[loc(g)] for g in the disjoint set of j (restricted partition of
//             unity, Eq. restCons), so every global entry is written exactly once.
//
// Work items.  Tile row I of subdomain j needs the off-diagonal 64x64 tiles inside the
// factors' tile envelope: L tiles tlo..I-1 (forward), U tiles I+1..thi (backward); the tiles
// outside are exactly zero and are never read.  They are split into segments of at most kseg
// tiles: every segment but the last is a "partial" item that publishes the partial product of
// its tiles with the solved pieces; the last segment is the "diagonal" item, which adds the
// partials, applies the precomputed inverse of the diagonal block and then the chain tile
// (the tile next to the diagonal, stored premultiplied by that inverse, so only one
// matrix-vector product waits for the neighbouring row), and publishes the solved piece of
// row I.  Items are queued forward-then-backward, each direction sorted by the chain
// position they wait for.
//
// Streaming.  Each CTA holds its current item and the next one; thread 0 keeps a ring of
// ring_stages shared-memory stages filled with 1-D bulk copies (TMA engine) across the item
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
// Stages of the shared-memory ring per CTA: 4 tiles (64 KB FP32, 32 KB BF16); FP64 tiles
// are 32 KB, so 2 stages keep three CTAs per SM (another CTA's arithmetic overlaps a CTA's
// waits, which matters where the FP64 pipe, not HBM, is the bound).
template <typename S> __host__ __device__ constexpr int ring_stages() { return sizeof(S) == 8 ? 2 : 4; }
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
        atomicOr(status, ST_TIMEOUT | ST_AT_SOLVE_POLL);
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
  int T, p, jb, nseg, q0, nq, nload;   // off-diagonal tile q sits in column jb + q (forward)
  bool diag;                           // or jb - q (backward)
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
  // tile envelope of the row: L tiles [tlo, I), U tiles (I, thi]; tiles outside are zero
  const int64_t trow = (t.meta[e.j].row_off >> 6) + e.I;
  if (e.bwd) {
    e.jb = t.thi ? t.thi[trow] : e.T - 1;
    e.p = e.jb - e.I;
  } else {
    e.jb = t.tlo ? t.tlo[trow] : 0;
    e.p = e.I - e.jb;
  }
  const int K = t.kseg;
  e.nseg = e.p > 0 ? (e.p + K - 1) / K : 1;
  e.q0 = e.diag ? (e.nseg - 1) * K : e.seg * K;
  e.nq = e.diag ? e.p - e.q0 : K;
  e.nload = e.nq + (e.diag ? PIECES : 0);
  return e;
}

// p4[q][u] += Inv[r][c] xb[q][c] over the thread's 32 columns c (half HALF of the row) of a
// packed triangular inverse (UPPER: U^{-1}, else L^{-1}); p0 / p1: the stages holding entries
// [0, CPS) and [CPS, INV_PACKED).  Column and direction are compile-time here, so each packed
// index is r plus a constant (an immediate offset); every such index lies inside the triangle's
// INV_PACKED entries, so the loads need no guard and the entries outside the triangle are
// replaced by zero after the load.
template <int HALF, bool UPPER, int CPS, int NR, typename C>
__device__ __forceinline__ void packed_inverse_product(const C* p0, const C* p1, int r, const C (*xb)[64],
                                                       C (&p4)[NR][4]) {
#pragma unroll
  for (int c0 = 32 * HALF; c0 < 32 * HALF + 32; c0 += 4)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int col = c0 + u;
      const int el = UPPER ? inv_upper_index(r, col) : inv_lower_index(r, col);
      const C v = (CPS >= INV_PACKED || el < CPS) ? p0[el] : p1[el - CPS];
      const C a = (UPPER ? r <= col : r >= col) ? v : (C)0;
#pragma unroll
      for (int q = 0; q < NR; ++q) p4[q][u] += a * xb[q][col];
    }
}

// NR right-hand sides share every streamed tile (columns NR of IndirectVec r_in / z_out);
// tagged words are laid out (row, rhs) with NR words per row.
template <typename S, typename C, int NR>
__global__ void __launch_bounds__(TRSV_THREADS) trsv_kernel(TrsvDev t, IndirectVec r_in, IndirectVec z_out,
                                                            const int* done) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr uint32_t STAGE = sizeof(S) * TILE_ELEMS;          // one factor tile per stage
  constexpr int PIECES = (int)(sizeof(C) / sizeof(S));        // stages per inverse tile
  constexpr int W = Tagged<C>::WORDS;
  constexpr int CPS = STAGE / sizeof(C);                      // C values per stage
  constexpr int NSTAGE = ring_stages<S>();
  static_assert(PIECES >= 1 && PIECES <= 2 && NSTAGE >= PIECES, "ring too small");
  // a packed inverse (one triangle, INV_PACKED entries) spans PIECES stages, the last one partly
  constexpr uint32_t INV_BYTES = (uint32_t)(sizeof(C) * INV_PACKED);
  static_assert(INV_BYTES > (PIECES - 1) * STAGE && INV_BYTES <= PIECES * STAGE && INV_BYTES % 16 == 0,
                "packed inverse does not fill its stages");
  __shared__ __align__(8) uint64_t bar[NSTAGE];
  __shared__ C yb[2][NR][64];                                 // solved pieces, double-buffered
  __shared__ C xb[NR][64];
  __shared__ C red[NR][TRSV_THREADS], red2[NR][TRSV_THREADS];
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
  const uint64_t l2_pol = l2_evict_first_policy();   // factor tiles are read once per launch
  auto issue_load = [&](const Item& e, int l) {
    const int st = lc % NSTAGE;
    unsigned char* dst = smem + (size_t)st * STAGE;
    const SubMeta m = t.meta[e.j];
    // load order of a diagonal item: off-diagonal tiles but the chain tile, the inverse
    // pieces, the chain tile (the neighbouring row's, premultiplied by the inverse)
    int tq = -1, piece = -1;
    if (e.diag && e.nq > 0) {
      if (l < e.nq - 1) tq = l;
      else if (l < e.nq - 1 + PIECES) piece = l - (e.nq - 1);
      else tq = e.nq - 1;
    } else if (l < e.nq) {
      tq = l;
    } else {
      piece = l - e.nq;
    }
    if (tq >= 0) {
      const int q = e.q0 + tq;
      const int J = e.bwd ? e.jb - q : e.jb + q;
      mbar_expect_tx(&bar[st], STAGE);
      bulk_g2s_hint(dst, tiles + tile_base(m, e.I, J), STAGE, &bar[st], l2_pol);
    } else {
      const int64_t trow = (m.row_off >> 6) + e.I;
      const unsigned char* it = (const unsigned char*)(inv + (trow * 2 + e.bwd) * (int64_t)TILE_ELEMS);
      const uint32_t bytes = min(STAGE, INV_BYTES - (uint32_t)piece * STAGE);   // the packed triangle only
      mbar_expect_tx(&bar[st], bytes);
      bulk_g2s_hint(dst, it + (size_t)piece * STAGE, bytes, &bar[st], l2_pol);
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
    if (!ok) { atomicOr(t.status, ST_TIMEOUT | ST_AT_SOLVE_COPY); atomicExch(&t.sync[3], 1u); }
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
    // restrict: prefetch this row's right-hand sides (forward diagonal items)
    C rhs[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) rhs[q] = (C)0;
    if (e.diag && !e.bwd && tid < 64) {
      const int g = t.gather[ro + tid];
      if (g >= 0)
#pragma unroll
        for (int q = 0; q < NR; ++q) rhs[q] = (C)r_in.load(q, g);
    }
    // tagged words of the solved piece multiplying off-diagonal tile l of this item
    auto ywords = [&](int l, int q) {
      const int qq = e.q0 + l;
      const int J = e.bwd ? e.jb - qq : e.jb + qq;
      return t.ytag + ((m.row_off + 64 * J + tid) * NR + q) * W;
    };
    auto pwords = [&](int seg, int q) { return t.ptag + (((trow * t.maxseg + seg) * 64 + tid) * NR + q) * W; };
    // a diagonal item leaves its chain tile (the last one, next to the diagonal) for after
    // the inverse product
    const int nt = (e.diag && e.nq > 0) ? e.nq - 1 : e.nq;
    typename Tagged<C>::Raw pre[NR];
    if (tid < 64 && nt > 0)
#pragma unroll
      for (int q = 0; q < NR; ++q) pre[q] = Tagged<C>::load(ywords(0, q));
    C acc[NR], psum[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = psum[q] = (C)0;
    for (int l = 0; l < nt; ++l) {
      const bool staged = stage_ready(cc);
      bool ok = staged;
      if (tid < 64) {
        // the words were loaded one tile earlier; poll only if they were not yet published
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          C v = (C)0;
          if (ok && !Tagged<C>::check(pre[q], tag, &v)) ok = poll_value<C>(ywords(l, q), tag, &v, t.sync, t.status);
          yb[l & 1][q][tid] = v;
        }
        if (l + 1 < nt)
#pragma unroll
          for (int q = 0; q < NR; ++q) pre[q] = Tagged<C>::load(ywords(l + 1, q));
      }
      if (!__syncthreads_and(ok)) {
        bad = true;
        if (tid == 0 && staged) cc++;
        break;
      }
      if (tid == 0) pump();            // every thread is past tile l-1: its stage is free
      const S* tile = (const S*)(smem + (size_t)(cc % NSTAGE) * STAGE);
      // four independent partial sums per right-hand side (hides the FMA latency)
      C a4[NR][4];
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) a4[q][u] = (C)0;
#pragma unroll
      for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const C a = (C)cvt(tile[Layout<S>::off(r, c0 + u)]);
#pragma unroll
          for (int q = 0; q < NR; ++q) a4[q][u] += a * yb[l & 1][q][c0 + u];
        }
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] += (a4[q][0] + a4[q][1]) + (a4[q][2] + a4[q][3]);
      cc++;
    }
    if (bad) break;
    if (!e.diag) {
#pragma unroll
      for (int q = 0; q < NR; ++q) red[q][tid] = acc[q];
      __syncthreads();
      if (tid < 64)
#pragma unroll
        for (int q = 0; q < NR; ++q) Tagged<C>::put(pwords(e.seg, q), red[q][tid] + red[q][tid + 64], tag);
    } else {
      // diagonal block through its inverse: c = Inv (b - products of the tiles before the
      // chain tile); then x = c - (Inv L_{I,I-1}) x_{I-1} (backward: Uinv U_{I,I+1} x_{I+1})
#pragma unroll
      for (int q = 0; q < NR; ++q) red[q][tid] = acc[q];
      bool ok = true;
      C own[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        if (e.nq == 0) psum[q] = (C)0;  // no off-diagonal tile (first row of a sweep): no partials
        own[q] = rhs[q];
        if (e.bwd && tid < 64 && ok)
          ok = poll_value<C>(t.ytag + ((ro + tid) * NR + q) * W, tag_f, &own[q], t.sync, t.status);
      }
      // partial sums of the other segments (normally ready by now), then start loading the
      // chain tile's solved piece
      if (tid < 64) {
        for (int sg = 0; sg < e.nseg - 1 && ok; ++sg)
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            C v = (C)0;
            if (ok) ok = poll_value<C>(pwords(sg, q), tag, &v, t.sync, t.status);
            psum[q] += v;
          }
        if (e.nq > 0)
#pragma unroll
          for (int q = 0; q < NR; ++q) pre[q] = Tagged<C>::load(ywords(e.nq - 1, q));
      }
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
      if (tid < 64)
#pragma unroll
        for (int q = 0; q < NR; ++q) xb[q][tid] = own[q] - ((red[q][tid] + red[q][tid + 64]) + psum[q]);
      __syncthreads();
      C p4[NR][4];
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) p4[q][u] = (C)0;
      {
        // the packed inverse: stage cc (and cc + 1 when it spans two stages)
        const C* p0 = (const C*)(smem + (size_t)(cc % NSTAGE) * STAGE);
        const C* p1 = (const C*)(smem + (size_t)((cc + 1) % NSTAGE) * STAGE);
        if (half == 0) {
          if (e.bwd) packed_inverse_product<0, true, CPS, NR>(p0, p1, r, xb, p4);
          else packed_inverse_product<0, false, CPS, NR>(p0, p1, r, xb, p4);
        } else {
          if (e.bwd) packed_inverse_product<1, true, CPS, NR>(p0, p1, r, xb, p4);
          else packed_inverse_product<1, false, CPS, NR>(p0, p1, r, xb, p4);
        }
      }
#pragma unroll
      for (int q = 0; q < NR; ++q) red2[q][tid] = (p4[q][0] + p4[q][1]) + (p4[q][2] + p4[q][3]);
      __syncthreads();
      C x[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) x[q] = red2[q][tid & 63] + red2[q][(tid & 63) + 64];
      cc += PIECES;
      if (e.nq > 0) {
        if (tid == 0) pump();          // every thread is past the inverse: its stages are free
        const bool sc = stage_ready(cc);
        ok = sc;
        if (tid < 64)
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            C v = (C)0;
            if (ok && !Tagged<C>::check(pre[q], tag, &v))
              ok = poll_value<C>(ywords(e.nq - 1, q), tag, &v, t.sync, t.status);
            yb[0][q][tid] = v;
          }
        if (!__syncthreads_and(ok)) {
          bad = true;
          if (tid == 0 && sc) cc++;
          break;
        }
        const S* tile = (const S*)(smem + (size_t)(cc % NSTAGE) * STAGE);
        C a4[NR][4];
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) a4[q][u] = (C)0;
#pragma unroll
        for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 4)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const C a = (C)cvt(tile[Layout<S>::off(r, c0 + u)]);
#pragma unroll
            for (int q = 0; q < NR; ++q) a4[q][u] += a * yb[0][q][c0 + u];
          }
#pragma unroll
        for (int q = 0; q < NR; ++q) red[q][tid] = (a4[q][0] + a4[q][1]) + (a4[q][2] + a4[q][3]);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NR; ++q) x[q] -= red[q][tid & 63] + red[q][(tid & 63) + 64];
        cc++;
      }
      if (tid < 64) {
        const int sidx = e.bwd ? t.scatter[ro + tid] : -1;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          Tagged<C>::put(t.ytag + ((ro + tid) * NR + q) * W, x[q], tag);
          if (sidx >= 0) z_out.ptr(q)[sidx] = (double)x[q];
        }
      }
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
                      int* maxseg, const int32_t* tlo, const int32_t* thi) {
  items.clear();
  int ms = 1;
  std::vector<std::tuple<int, int, int, int, int, int>> q;   // key, kind, j, I, seg, bwd
  // key = the position in the sweep (forward: tile row, backward: T-1 - tile row) of the last
  // solved piece the item waits for
  for (int bwd = 0; bwd < 2; ++bwd) {
    int64_t trow0 = 0;
    for (int j = 0; j < n_sub; ++j) {
      const int off = stagger ? ((j & 1) ? T[j] / 2 : 0) + (bwd ? T[j] : 0)
                              : (bwd ? 1 << 24 : 0);
      for (int I = 0; I < T[j]; ++I) {
        const int lo = tlo ? tlo[trow0 + I] : 0, hi = thi ? thi[trow0 + I] : T[j] - 1;
        const int p = bwd ? hi - I : I - lo;
        const int base = bwd ? T[j] - 1 - hi : lo;
        const int nseg = p > 0 ? (p + kseg - 1) / kseg : 1;
        ms = std::max(ms, nseg);
        for (int s = 0; s < nseg - 1; ++s) q.emplace_back(off + base + s * kseg + kseg - 1, 0, j, I, s, bwd);
        q.emplace_back(off + base + p - 1, 1, j, I, SEG_DIAG, bwd);
      }
      trow0 += T[j];
    }
  }
  std::sort(q.begin(), q.end());
  for (auto& e : q)
    items.push_back(make_int2(std::get<2>(e), std::get<3>(e) | (std::get<4>(e) << 20) | (std::get<5>(e) << 30)));
  *maxseg = ms;
}

template <typename S, typename C> constexpr size_t ring_bytes() { return ring_stages<S>() * sizeof(S) * TILE_ELEMS; }

int trsv_ctas_per_sm(int precision) {
  // rings: fp64 2 x 32 KB, fp32 4 x 16 KB, bf16 4 x 8 KB of shared memory per CTA
  return precision == 0 ? 3 : (precision == 1 ? 3 : 6);
}

template <typename S, typename C, int NR> static cudaError_t prepare_nr() {
  return cudaFuncSetAttribute(trsv_kernel<S, C, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ring_bytes<S, C>());
}
template <typename S, typename C> static cudaError_t prepare_all() {
  cudaError_t e = prepare_nr<S, C, 1>();
  if (e == cudaSuccess) e = prepare_nr<S, C, 2>();
  if (e == cudaSuccess) e = prepare_nr<S, C, 4>();
  if (e == cudaSuccess) e = prepare_nr<S, C, 8>();
  return e;
}

cudaError_t trsv_prepare(int precision) {
  if (precision == 0) return prepare_all<double, double>();
  if (precision == 1) return prepare_all<float, float>();
  return prepare_all<__nv_bfloat16, float>();
}

template <typename S, typename C>
static cudaError_t launch_typed(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done, int nr,
                                cudaStream_t s) {
  const size_t smem = ring_bytes<S, C>();
  switch (nr) {
    case 1: trsv_kernel<S, C, 1><<<t.grid, TRSV_THREADS, smem, s>>>(t, r_in, z_out, done); break;
    case 2: trsv_kernel<S, C, 2><<<t.grid, TRSV_THREADS, smem, s>>>(t, r_in, z_out, done); break;
    case 4: trsv_kernel<S, C, 4><<<t.grid, TRSV_THREADS, smem, s>>>(t, r_in, z_out, done); break;
    case 8: trsv_kernel<S, C, 8><<<t.grid, TRSV_THREADS, smem, s>>>(t, r_in, z_out, done); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_trsv(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done,
                        cudaStream_t s, int nr) {
  if (nr > t.nr_cap) return cudaErrorInvalidValue;
  if (t.precision == 0) return launch_typed<double, double>(t, r_in, z_out, done, nr, s);
  if (t.precision == 1) return launch_typed<float, float>(t, r_in, z_out, done, nr, s);
  return launch_typed<__nv_bfloat16, float>(t, r_in, z_out, done, nr, s);
}

}  // namespace cpmdev
