// Trailing update of the batched LU on the 5th-generation tensor cores (tcgen05):
//     A_IJ -= L_Is U_sJ        for all I, J > s and all subdomains, in one launch.
//
// One CTA (4 warps) computes 128 x 64 blocks: tile rows I0 = s+1+2p and I0+1 of a chunk of
// tile columns J.  The FP32 tile storage (1 KB atoms of 32 rows x 8 columns, 128-byte XOR
// swizzle, row index contiguous) is the canonical K-major tcgen05 layout for a B operand
// (rows = K, columns = N): U tiles are used as loaded by one 16 KB bulk copy.  The L tiles
// are the A operand (rows = M, columns = K); they are rewritten K-major while they are
// converted (tf32 split or bf16).
//   FP32 mode: each operand is split into tf32 high and low parts (x = hi + lo, both
//              tf32-rounded) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi (kind::tf32), which
//              keeps FP32 accuracy.
//   BF16 mode: operands are rounded to bf16 into bf16 canonical layouts (kind::f16, FP32
//              accumulation).
// D (128 lanes x 64 FP32 columns) lives in tensor memory; the epilogue reads it with
// tcgen05.ld (warp w owns rows 32w..32w+31) and subtracts it from the FP32 tiles.
// Every wait is bounded; on expiry the CTA reports CPM_ERR_TIMEOUT, still frees its tensor
// memory, and returns.
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int TC_THREADS = 128;

// ---- tcgen05 / descriptor helpers -------------------------------------------------------
// Shared-memory matrix descriptor (tcgen05): start address, leading / stride byte offsets,
// version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B K-major, M = 128, N = 64.
// fmt: 1 = bf16 (kind::f16), 2 = tf32 (kind::tf32).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) {
  return (1u << 4)                   // D format F32
         | (fmt << 7) | (fmt << 10)  // A, B formats
         | (0u << 15)                // A K-major
         | (0u << 16)                // B K-major
         | ((64u >> 3) << 17)        // N >> 3
         | ((128u >> 4) << 24);      // M >> 4
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND == 2)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 consecutive FP32 accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// K-major 128-byte-swizzled operand layouts (byte offsets), 1 KB atoms of 8 rows x 128 B:
//   A tf32 (M = 128, K = 64): K halves of 32 at 16 KB, 8-row groups at 1 KB.
//   A bf16 (M = 128, K = 64): 8-row groups at 1 KB, one 128-byte line = 64 K values.
//   B bf16 (K = 64, N = 64):  8-column groups at 1 KB, one line = 64 K values.
__device__ __forceinline__ uint32_t tf32_a_off(int m, int k) {
  const int line = m & 7, chunk = (k >> 2) & 7;
  return (uint32_t)((k >> 5) * 16384 + (m >> 3) * 1024 + line * 128 + ((chunk ^ line) << 4) + (k & 3) * 4);
}
__device__ __forceinline__ uint32_t bf16_a_off(int m, int k) {
  const int line = m & 7, chunk = (k >> 3) & 7;
  return (uint32_t)((m >> 3) * 1024 + line * 128 + ((chunk ^ line) << 4) + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t bf16_b_off(int k, int n) {
  const int line = n & 7, chunk = (k >> 3) & 7;
  return (uint32_t)((n >> 3) * 1024 + line * 128 + ((chunk ^ line) << 4) + (k & 7) * 2);
}

// KIND 2: FP32 tiles, split tf32.  KIND 1: FP32 tiles, bf16 operands.
// Grid: x = pair of tile rows (I0 = s+1+2x, I0+1), y = chunk of JCHUNK tile columns,
// z = subdomain.  The A pair is loaded and converted once; B tiles of the chunk stream
// through two stages (bulk copies two ahead); each thread loads its C row before the
// tensor cores finish, then subtracts the accumulator read from tensor memory.
constexpr int JCHUNK = 8;
template <int KIND> struct TcSmem;
template <> struct TcSmem<2> {    // tf32 split: A raw 32 KB, A hi/lo 64 KB, B stages 2 x (hi 16 + lo 16 KB)
  static constexpr uint32_t A_RAW = 0, A_HI = 32768, A_LO = 65536, B0 = 98304, BSTAGE = 32768,
                            TOTAL = 163840;
};
template <> struct TcSmem<1> {    // bf16: A raw 32 KB + A bf16 16 KB, B stages 2 x (raw 16 KB + bf16 8 KB)
  static constexpr uint32_t A_RAW = 0, A_BF = 32768, B0 = 49152, BSTAGE = 24576, TOTAL = 98304;
};

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS) lu_update_tc_kernel(float* a, const SubMeta* __restrict__ meta,
                                                                   int s, int* status) {
  using L = TcSmem<KIND>;
  const SubMeta m = meta[blockIdx.z];
  const int I0 = s + 1 + 2 * blockIdx.x, I1 = I0 + 1;
  const int Jbeg = s + 1 + blockIdx.y * JCHUNK;
  if (I0 >= m.T || Jbeg >= m.T) return;        // before any tensor-memory allocation
  const int Jend = min(m.T, Jbeg + JCHUNK);
  const bool two = I1 < m.T;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_a, bar_b[2], bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ int sh_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int nissued[2] = {0, 0}, nwaited[2] = {0, 0};   // bulk copies per B stage (thread 0)
  bool a_done = false, mma_pending = false;
  if (tid == 0) {
    mbar_init(&bar_a, 1);
    mbar_init(&bar_b[0], 1);
    mbar_init(&bar_b[1], 1);
    mbar_init(&bar_mma, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 64);
  __syncthreads();
  fence_after_sync();
  const uint32_t taddr = tmem_slot;
  // raw FP32 destinations of the A pair and of the B stages
  float* rawA = (float*)(base + L::A_RAW);
  auto rawB = [&](int b) { return (float*)(base + L::B0 + b * L::BSTAGE); };
  if (tid == 0) {
    mbar_expect_tx(&bar_a, two ? 32768u : 16384u);
    bulk_g2s(rawA, a + tile_base(m, I0, s), 16384, &bar_a);
    if (two) bulk_g2s(rawA + TILE_ELEMS, a + tile_base(m, I1, s), 16384, &bar_a);
    for (int b = 0; b < 2 && Jbeg + b < Jend; ++b) {
      mbar_expect_tx(&bar_b[b], 16384u);
      bulk_g2s(rawB(b), a + tile_base(m, s, Jbeg + b), 16384, &bar_b[b]);
      nissued[b]++;
    }
    sh_ok = mbar_wait_bounded(&bar_a, 0) ? 1 : 0;
    if (!sh_ok) atomicOr(status, ST_TIMEOUT);
    a_done = sh_ok;
  }
  __syncthreads();
  bool ok = sh_ok != 0;
  if (ok) {
    mbar_wait_bounded(&bar_a, 0);              // completed: makes the copy visible here
    if (!two)
      for (int e = tid; e < TILE_ELEMS; e += TC_THREADS) rawA[TILE_ELEMS + e] = 0.0f;
    __syncthreads();
    if (KIND == 2) {                            // A hi / lo, rewritten K-major
      unsigned char* ahi = base + TcSmem<2>::A_HI;
      unsigned char* alo = base + TcSmem<2>::A_LO;
      for (int e = tid; e < 2 * TILE_ELEMS; e += TC_THREADS) {
        const int t = e >> 12, el = e & 4095, i = el & 63, k = el >> 6;
        const float x = rawA[t * TILE_ELEMS + off_sw32(i, k)], hi = tf32_round(x);
        const uint32_t o = tf32_a_off(64 * t + i, k);
        *(float*)(ahi + o) = hi;
        *(float*)(alo + o) = tf32_round(x - hi);
      }
    } else {
      unsigned char* abf = base + TcSmem<1>::A_BF;
      for (int e = tid; e < 2 * TILE_ELEMS; e += TC_THREADS) {
        const int t = e >> 12, el = e & 4095, i = el & 63, k = el >> 6;
        *(__nv_bfloat16*)(abf + bf16_a_off(64 * t + i, k)) =
            __float2bfloat16_rn(rawA[t * TILE_ELEMS + off_sw32(i, k)]);
      }
    }
  }
  const int row = 32 * warp + lane;
  const bool mine = row < 64 || two;
  const int lr = row & 63;
  for (int it = 0; ok && it < Jend - Jbeg; ++it) {
    const int J = Jbeg + it, b = it & 1;
    const uint32_t ph = (uint32_t)(it >> 1) & 1;
    float* ct = a + tile_base(m, row < 64 ? I0 : I1, J);
    float c[64];
    if (mine) {
#pragma unroll
      for (int q = 0; q < 64; ++q) c[q] = ct[off_sw32(lr, q)];
    }
    if (tid == 0) {
      sh_ok = mbar_wait_bounded(&bar_b[b], ph) ? 1 : 0;
      if (!sh_ok) atomicOr(status, ST_TIMEOUT);
      else nwaited[b]++;
    }
    __syncthreads();
    if (!sh_ok) { ok = false; break; }
    mbar_wait_bounded(&bar_b[b], ph);
    float* rb = rawB(b);
    if (KIND == 2) {                            // B_hi in place, B_lo in the second half
      float* blo = rb + TILE_ELEMS;
      for (int e = tid; e < TILE_ELEMS; e += TC_THREADS) {
        const float x = rb[e], hi = tf32_round(x);
        rb[e] = hi;
        blo[e] = tf32_round(x - hi);
      }
    } else {
      unsigned char* bbf = (unsigned char*)(rb + TILE_ELEMS);
      for (int e = tid; e < TILE_ELEMS; e += TC_THREADS) {
        const int k = e & 63, n = e >> 6;
        *(__nv_bfloat16*)(bbf + bf16_b_off(k, n)) = __float2bfloat16_rn(rb[off_sw32(k, n)]);
      }
    }
    fence_proxy_async();                        // generic-proxy writes -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t sb = smem_u32(base), bs = smem_u32(rb);
      if (KIND == 2) {
        constexpr uint32_t idesc = instr_desc(2);
        const uint32_t ahi = sb + TcSmem<2>::A_HI, alo = sb + TcSmem<2>::A_LO;
        const uint32_t bhi = bs, blo = bs + 16384;
        for (int k = 0; k < 8; ++k) {           // K = 8 tf32 values (32 bytes) per instruction
          const uint32_t ka = (k >> 2) * 16384 + (k & 3) * 32;
          const uint32_t kb = (k >> 2) * 8192 + (k & 3) * 32;
          mma<2>(taddr, smem_desc(ahi + ka, 16, 1024), smem_desc(bhi + kb, 16, 1024), idesc,
                 k > 0 ? 1u : 0u);
          mma<2>(taddr, smem_desc(ahi + ka, 16, 1024), smem_desc(blo + kb, 16, 1024), idesc, 1u);
          mma<2>(taddr, smem_desc(alo + ka, 16, 1024), smem_desc(bhi + kb, 16, 1024), idesc, 1u);
        }
      } else {
        constexpr uint32_t idesc = instr_desc(1);
        const uint32_t ab = sb + TcSmem<1>::A_BF, bb = bs + 16384;
        for (int k = 0; k < 4; ++k)             // K = 16 bf16 values (32 bytes) per instruction
          mma<1>(taddr, smem_desc(ab + k * 32, 16, 1024), smem_desc(bb + k * 32, 16, 1024), idesc,
                 k > 0 ? 1u : 0u);
      }
      mma_commit(&bar_mma);
      sh_ok = mbar_wait_bounded(&bar_mma, (uint32_t)it & 1) ? 1 : 0;
      if (!sh_ok) {
        atomicOr(status, ST_TIMEOUT);
        mma_pending = true;
      }
      // stage b is free again: stream the tile two columns ahead into it
      if (sh_ok && J + 2 < Jend) {
        mbar_expect_tx(&bar_b[b], 16384u);
        bulk_g2s(rb, a + tile_base(m, s, J + 2), 16384, &bar_b[b]);
        nissued[b]++;
      }
    }
    __syncthreads();
    if (!sh_ok) { ok = false; break; }
    mbar_wait_bounded(&bar_mma, (uint32_t)it & 1);
    fence_after_sync();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float d[32];
      tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + 32 * h, d);
      if (mine) {
#pragma unroll
        for (int q = 0; q < 32; ++q) ct[off_sw32(lr, 32 * h + q)] = c[32 * h + q] - d[q];
      }
    }
    fence_before_sync();
    __syncthreads();                            // accumulator read before the next MMA
  }
  // after an abort: wait (bounded) for this CTA's own copies and tensor-core work still in
  // flight before the shared and tensor memory are released
  if (tid == 0 && !ok) {
    if (!a_done) mbar_wait_bounded(&bar_a, 0);
    for (int b = 0; b < 2; ++b)
      for (; nwaited[b] < nissued[b]; ++nwaited[b]) mbar_wait_bounded(&bar_b[b], (uint32_t)nwaited[b] & 1);
    if (mma_pending) mbar_wait_bounded(&bar_mma, 0);
    if (mma_pending) mbar_wait_bounded(&bar_mma, 1);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 64);
}

cudaError_t lu_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(lu_update_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(1024 + TcSmem<2>::TOTAL));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(lu_update_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(1024 + TcSmem<1>::TOTAL));
}

cudaError_t launch_lu_update_tc(const FactorDev& f, int step, int bf16, cudaStream_t s) {
  const int W = f.t_max - 1 - step;
  if (W <= 0) return cudaSuccess;
  dim3 g((W + 1) / 2, (W + JCHUNK - 1) / JCHUNK, f.n_sub);
  if (bf16)
    lu_update_tc_kernel<1><<<g, TC_THREADS, 1024 + TcSmem<1>::TOTAL, s>>>((float*)f.a, f.meta, step, f.status);
  else
    lu_update_tc_kernel<2><<<g, TC_THREADS, 1024 + TcSmem<2>::TOTAL, s>>>((float*)f.a, f.meta, step, f.status);
  return cudaGetLastError();
}

}  // namespace cpmdev
