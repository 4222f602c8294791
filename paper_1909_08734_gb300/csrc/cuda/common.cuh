// Shared device helpers: tile layouts of the local factors, bounded waits, bulk copies.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cpmdev {

constexpr int TILE = 64;                 // local matrices are stored as 64 x 64 tiles
constexpr int TILE_ELEMS = TILE * TILE;

// Device status word bits (latched until oras_check_status clears them).
constexpr int ST_TIMEOUT = 1;
constexpr int ST_SINGULAR = 2;
// With ST_TIMEOUT: which kernel family's bounded wait gave up (diagnostics).
constexpr int ST_AT_LU = 16;            // tensor-core trailing update (copies / MMA completion)
constexpr int ST_AT_SOLVE_POLL = 32;    // batched solve: a published value that never came
constexpr int ST_AT_SOLVE_COPY = 64;    // batched solve: a factor-tile copy
constexpr int ST_AT_KRYLOV = 128;       // Arnoldi step: a basis-batch copy

// Spin limit of inter-CTA waits (each poll sleeps ~0.25-2 us): ~4 s, far above any
// legitimate wait, then the kernel reports CPM_ERR_TIMEOUT instead of hanging.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// Per-subdomain layout record.
struct SubMeta {
  int64_t tile_off;   // element offset of tile (0,0) in the factor buffer
  int64_t row_off;    // offset of this subdomain's padded rows in per-row arrays
  int32_t T;          // tiles per dimension (padded size = 64 T)
  int32_t n;          // real local size n_j
  int32_t n_sigma;    // the first n_sigma local unknowns carry the restricted residual
  int32_t pad;
};

// ---- element offsets inside one 64 x 64 tile ----------------------------------------
// FP64 / BF16 storage: plain column-major.
__host__ __device__ __forceinline__ int off_plain(int i, int j) { return j * TILE + i; }
// Packed diagonal-block inverses: each triangle stored column by column at the start of its
// 64 x 64 slot, INV_PACKED entries.  L^{-1} (unit lower) keeps rows r >= c of column c,
// U^{-1} (upper) rows r <= c; the index of (r, c) inside its triangle:
constexpr int INV_PACKED = TILE * (TILE + 1) / 2;
__host__ __device__ __forceinline__ int inv_lower_index(int r, int c) { return c * TILE - c * (c - 1) / 2 + (r - c); }
__host__ __device__ __forceinline__ int inv_upper_index(int r, int c) { return c * (c + 1) / 2 + r; }
// FP32 storage: sixteen 1 KB atoms of 32 rows x 8 columns (atom (i/32, j/8) at
// ((i/32)*8 + j/8) KB); inside an atom, column j%8 is a 128-byte line of 32 consecutive
// rows whose 16-byte chunks are XOR-swizzled with the line index.  This is the canonical
// 128-byte-swizzled operand layout of the tcgen05 tensor cores with the row index as the
// contiguous dimension.
__host__ __device__ __forceinline__ int off_sw32(int i, int j) {
  int ai = i >> 5, aj = j >> 3, line = j & 7, chunk = (i >> 2) & 7, e = i & 3;
  return ((ai * 8 + aj) << 8) + (line << 5) + ((chunk ^ line) << 2) + e;
}

template <typename T> struct Layout;
template <> struct Layout<double> {
  __host__ __device__ static __forceinline__ int off(int i, int j) { return off_plain(i, j); }
};
template <> struct Layout<float> {
  __host__ __device__ static __forceinline__ int off(int i, int j) { return off_sw32(i, j); }
};
template <> struct Layout<__nv_bfloat16> {
  __host__ __device__ static __forceinline__ int off(int i, int j) { return off_plain(i, j); }
};

__device__ __forceinline__ int64_t tile_base(const SubMeta& m, int I, int J) {
  return m.tile_off + ((int64_t)J * m.T + I) * TILE_ELEMS;
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- acquire / release flags ----------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- mbarrier + 1-D bulk copy (TMA engine, no tensor map) -----------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bulk copy global -> shared; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy for data read once (a streamed factor tile): evicted first, so that vectors
// reused across kernels (the Krylov basis) stay in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Device time in ns (the global timer).
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Time limit of a wait on this CTA's own copies or tensor-core work, far above any
// legitimate wait; then the kernel reports CPM_ERR_TIMEOUT instead of hanging.
constexpr uint64_t MBAR_WAIT_LIMIT_NS = 2000000000ull;
// Bounded wait for a phase of an mbarrier; returns false after the time limit.  try_wait
// suspends the thread in hardware until the phase completes or a short window passes, so
// the loop polls without sleeping (a sleep would add its granularity to every wait).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = MBAR_WAIT_LIMIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// ---- reductions -----------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace cpmdev
