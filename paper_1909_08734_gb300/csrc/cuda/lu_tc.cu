// Trailing update of the batched LU on the 5th-generation tensor cores (tcgen05):
//     A_IJ -= L_Is U_sJ        for all I, J > s and all subdomains, in one launch.
//
// A CTA computes 128 x 64 blocks: tile rows I0 = s+1+2p and I0+1 of a chunk of tile columns
// J.  The L tiles are the A operand (rows = M, columns = K), rewritten K-major once per CTA
// while they are converted; the U row of step s is split once per step by lu_split_u_kernel
// into the B operand's K-major layout (the FP32 tile storage, 1 KB atoms of 32 rows x 8
// columns with a 128-byte XOR swizzle, is already the canonical K-major B layout), so U tiles
// reach the MMAs by one bulk copy each.  C tile pairs stream through shared memory by bulk
// copies; D (128 lanes x 64 FP32 columns, two buffers) lives in tensor memory and the
// epilogue reads it with tcgen05.ld while the next column's MMAs run.
//   FP32 mode: each operand is split into tf32 high and low parts (x = hi + lo, both
//              tf32-rounded) and D = A_hi B_hi + A_hi B_lo + A_lo B_hi (kind::tf32), which
//              keeps FP32 accuracy.  Warp-specialised kernel: one thread streams U and C
//              tiles, one issues the MMAs, eight warps run the epilogue; the roles hand over
//              through mbarriers only.
//   BF16 mode: operands are rounded to bf16 (kind::f16, FP32 accumulation); 8 warps in
//              lock step per column, two CTAs per SM, results leave by bulk copies.
// Every wait is bounded; on expiry the CTA reports CPM_ERR_TIMEOUT, waits (bounded) for its
// own copies and MMAs in flight, frees its tensor memory, and returns.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

constexpr int TC_LS_THREADS = 256;       // lock-step bf16 kernel: 8 warps, two CTAs per SM
constexpr int TC_TMEM_COLS = 64;         // FP32 accumulator columns per buffer (two buffers)

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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// Bulk copy shared -> global in a bulk async-group; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed group have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
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
// Grid: x = pair of tile rows (I0 = s+1+2x, I0+1), y = chunk of jchunk tile columns,
// z = subdomain.  The A pair is loaded and converted once.  The U tiles (B) and the C tile
// pairs of the chunk stream through two shared-memory stages each, by bulk copies issued
// two columns ahead, so that HBM traffic overlaps the conversion, the MMAs and the epilogue
// (C = C - D with D read from tensor memory, written straight back to the tiles).
constexpr int TC_JCHUNK = 32;           // tile columns per CTA (default of launch_lu_update_tc)
template <int KIND> struct TcSmem;
template <> struct TcSmem<2> {    // A hi / lo 64 KB, B stages NB x (hi 16 + lo 16 KB), C stages NC x 32 KB
  static constexpr uint32_t A_HI = 0, A_LO = 32768, B0 = 65536, BSTAGE = 32768, BBYTES = 32768, NB = 2,
                            C0 = B0 + NB * BSTAGE, CSTAGE = 32768, NC = 2, A_RAW = C0 + CSTAGE,
                            TOTAL = C0 + NC * CSTAGE;
};
template <> struct TcSmem<1> {    // A bf16 16 KB, B stages NB x bf16 8 KB, C stages NC x 32 KB (2 CTAs per SM)
  static constexpr uint32_t A_BF = 0, B0 = 16384, BSTAGE = 8192, BBYTES = 8192, NB = 2, C0 = B0 + NB * BSTAGE,
                            CSTAGE = 32768, NC = 2, A_RAW = C0 + CSTAGE, TOTAL = C0 + NC * CSTAGE;
};
// (the raw A pair is staged in C stage 1, which is refilled once A has been converted)

// The U row of step s, split once per step into the B-operand form the MMAs read (tf32 hi
// then lo, 16 KB each, in the tile's own K-major layout; or bf16, 8 KB, K-major): slot
// row_off/64 + J of the buffer holds tile (s, J) of that subdomain.
template <int KIND>
__global__ void __launch_bounds__(256) lu_split_u_kernel(const float* __restrict__ a, const SubMeta* __restrict__ meta,
                                                         int s, unsigned char* __restrict__ ubuf,
                                                         const int32_t* __restrict__ hiu) {
  const SubMeta m = meta[blockIdx.y];
  const int J = s + 1 + blockIdx.x;
  if (J >= m.T || (hiu && J > hiu[blockIdx.y])) return;
  const float* t = a + tile_base(m, s, J);
  unsigned char* dst = ubuf + (size_t)((m.row_off >> 6) + J) * TcSmem<KIND>::BBYTES;
  if (KIND == 2) {
    const float4* src4 = (const float4*)t;
    float4* hi4 = (float4*)dst;
    float4* lo4 = (float4*)(dst + 16384);
    for (int e = threadIdx.x; e < TILE_ELEMS / 4; e += 256) {
      const float4 x = src4[e];
      float4 hi, lo;
      hi.x = tf32_round(x.x); lo.x = tf32_round(x.x - hi.x);
      hi.y = tf32_round(x.y); lo.y = tf32_round(x.y - hi.y);
      hi.z = tf32_round(x.z); lo.z = tf32_round(x.z - hi.z);
      hi.w = tf32_round(x.w); lo.w = tf32_round(x.w - hi.w);
      hi4[e] = hi;
      lo4[e] = lo;
    }
  } else {
    for (int e = threadIdx.x; e < TILE_ELEMS; e += 256) {
      const int k = e & 63, n = e >> 6;
      *(__nv_bfloat16*)(dst + bf16_b_off(k, n)) = __float2bfloat16_rn(t[off_sw32(k, n)]);
    }
  }
}

// Lock-step bf16 update (KIND 1): every column passes two CTA barriers; thread 0 waits for
// the U tile and issues the MMAs, all threads run the epilogue.  (The split-tf32 update runs
// in the warp-specialised kernel further down.)
template <int KIND>
__global__ void __launch_bounds__(TC_LS_THREADS) lu_update_tc_kernel(float* a, const SubMeta* __restrict__ meta,
                                                                   const unsigned char* __restrict__ ubuf, int s,
                                                                   int jchunk, int* status,
                                                                   const int32_t* __restrict__ pend,
                                                                   const int32_t* __restrict__ hiu, int t_max) {
  static_assert(KIND == 1, "the lock-step kernel is the bf16 update");
  using L = TcSmem<KIND>;
  constexpr int TC_THREADS = TC_LS_THREADS;
  constexpr int TC_CG = TC_THREADS / 128;      // epilogue column groups (warps per lane quarter)
  constexpr int TC_CW = 64 / TC_CG;            // accumulator columns per warp in the epilogue
  const SubMeta m = meta[blockIdx.z];
  const int I0 = s + 1 + 2 * blockIdx.x, I1 = I0 + 1;
  const int Jbeg = s + 1 + blockIdx.y * jchunk;
  // tile envelope: L_Is is zero for tile rows past pend, U_sJ for columns past hiu
  int Tend = m.T;
  if (pend) {
    if (64 * I0 >= pend[blockIdx.z * t_max + s]) return;
    Tend = min(Tend, hiu[blockIdx.z] + 1);
  }
  if (I0 >= m.T || Jbeg >= Tend) return;       // before any tensor-memory allocation
  const int nJ = min(Tend, Jbeg + jchunk) - Jbeg;
  const bool two = I1 < m.T;
  const uint32_t pair_bytes = two ? 32768u : 16384u;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int NB = (int)L::NB, NC = (int)L::NC;   // U and C stages
  __shared__ __align__(8) uint64_t bar_a, bar_b[NB], bar_c[NC], bar_mma[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int sh_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // copies and commits issued / waited per stage (thread 0), for the drain after an abort
  int nb_iss[NB] = {}, nb_wait[NB] = {}, nc_iss[NC] = {}, nc_wait[NC] = {};
  int nm_iss[2] = {0, 0}, nm_wait[2] = {0, 0};
  bool a_done = false;
  if (tid == 0) {
    mbar_init(&bar_a, 1);
    for (int b = 0; b < 2; ++b) mbar_init(&bar_mma[b], 1);
    for (int b = 0; b < NB; ++b) mbar_init(&bar_b[b], 1);
    for (int b = 0; b < NC; ++b) mbar_init(&bar_c[b], 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 2 * TC_TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t taddr = tmem_slot;
  float* rawA = (float*)(base + L::A_RAW);
  auto stage_b = [&](int b) { return (float*)(base + L::B0 + b * L::BSTAGE); };
  auto stage_c = [&](int b) { return (float*)(base + L::C0 + b * L::CSTAGE); };
  auto issue_b = [&](int b, int J) {
    mbar_expect_tx(&bar_b[b], L::BBYTES);
    bulk_g2s(stage_b(b), ubuf + (size_t)((m.row_off >> 6) + J) * L::BBYTES, L::BBYTES, &bar_b[b]);
    nb_iss[b]++;
  };
  auto issue_c = [&](int b, int J) {
    mbar_expect_tx(&bar_c[b], pair_bytes);
    bulk_g2s(stage_c(b), a + tile_base(m, I0, J), 16384, &bar_c[b]);
    if (two) bulk_g2s(stage_c(b) + TILE_ELEMS, a + tile_base(m, I1, J), 16384, &bar_c[b]);
    nc_iss[b]++;
  };
  if (tid == 0) {
    mbar_expect_tx(&bar_a, pair_bytes);
    bulk_g2s(rawA, a + tile_base(m, I0, s), 16384, &bar_a);
    if (two) bulk_g2s(rawA + TILE_ELEMS, a + tile_base(m, I1, s), 16384, &bar_a);
    for (int b = 0; b < NB && b < nJ; ++b) issue_b(b, Jbeg + b);
    issue_c(0, Jbeg);
    for (int b = 2; b < NC && b < nJ; ++b) issue_c(b, Jbeg + b);   // stage 1 holds raw A for now
    sh_ok = mbar_wait_bounded(&bar_a, 0) ? 1 : 0;
    if (!sh_ok) atomicOr(status, ST_TIMEOUT | ST_AT_LU);
    a_done = sh_ok;
  }
  __syncthreads();
  bool ok = sh_ok != 0;
  if (ok) {
    mbar_wait_bounded(&bar_a, 0);              // completed: makes the copy visible here
    if (!two)
      for (int e = tid; e < TILE_ELEMS; e += TC_THREADS) rawA[TILE_ELEMS + e] = 0.0f;
    __syncthreads();
    {                                           // A pair to bf16, rewritten K-major
      unsigned char* abf = base + TcSmem<1>::A_BF;
      for (int e = tid; e < 2 * TILE_ELEMS; e += TC_THREADS) {
        const int t = e >> 12, el = e & 4095, i = el & 63, k = el >> 6;
        *(__nv_bfloat16*)(abf + bf16_a_off(64 * t + i, k)) =
            __float2bfloat16_rn(rawA[t * TILE_ELEMS + off_sw32(i, k)]);
      }
    }
    fence_proxy_async();                        // generic accesses before the async refill
    __syncthreads();                            // raw A consumed: C stage 1 is free
    if (tid == 0 && nJ > 1) issue_c(1, Jbeg + 1);
  }
  // epilogue assignment: warp w owns rows 32 (w & 3) + lane (tensor-memory lanes of its
  // quarter) and columns TC_CW (w >> 2) .. + TC_CW - 1
  const int row = 32 * (warp & 3) + lane, colg = warp >> 2;
  const bool mine = row < 64 || two;
  const int lr = row & 63;
  int v_line[8];                                // in-atom offset of column line l of this row
#pragma unroll
  for (int l = 0; l < 8; ++l) v_line[l] = (l << 5) + ((((lr >> 2) & 7) ^ l) << 2);
  // software pipeline: in iteration it thread 0 issues the MMAs of U tile J = Jbeg + it into
  // accumulator buffer it & 1 as soon as that tile lands (a failed wait there is broadcast by
  // the barrier of the next iteration), then all threads finish column J - 1 (epilogue from
  // buffer (it-1) & 1)
  for (int it = 0; ok && it <= nJ; ++it) {
    if (it < nJ && tid == 0 && sh_ok) {
      // thread 0 alone: the pre-split U tile lands in stage it % NB, the MMAs go into
      // accumulator buffer it & 1
      const int bs = it % NB, b = it & 1;
      const uint32_t ph = (uint32_t)(it / NB) & 1;
      if (!mbar_wait_bounded(&bar_b[bs], ph)) {
        atomicOr(status, ST_TIMEOUT | ST_AT_LU);
        sh_ok = 0;
      } else {
        nb_wait[bs]++;
        fence_after_sync();
        const uint32_t d_tmem = taddr + (uint32_t)(b * TC_TMEM_COLS);
        // a descriptor's start-address field holds addr >> 4: an offset adds (off >> 4)
        const uint64_t db = smem_desc(smem_u32(stage_b(bs)), 16, 1024);
        {
          constexpr uint32_t idesc = instr_desc(1);
          const uint64_t da = smem_desc(smem_u32(base) + TcSmem<1>::A_BF, 16, 1024);
#pragma unroll
          for (int k = 0; k < 4; ++k)           // K = 16 bf16 values (32 bytes) per instruction
            mma<1>(d_tmem, da + ((k * 32) >> 4), db + ((k * 32) >> 4), idesc, k > 0 ? 1u : 0u);
        }
        mma_commit(&bar_mma[b]);
        nm_iss[b]++;
      }
    }
    if (it > 0) {                               // finish column J - 1
      const int p = it - 1, bp = p & 1, cp = p % NC;
      const uint32_t php = (uint32_t)(p >> 1) & 1, phc = (uint32_t)(p / NC) & 1;
      if (tid == 0 && sh_ok) {
        sh_ok = mbar_wait_bounded(&bar_mma[bp], php) ? 1 : 0;
        if (!sh_ok) atomicOr(status, ST_TIMEOUT | ST_AT_LU);
        else nm_wait[bp]++;
        // U stage p % NB is free again: stream the tile NB columns ahead into it
        if (sh_ok && p + NB < nJ) {
          fence_proxy_async();
          issue_b(p % NB, Jbeg + p + NB);
        }
        if (sh_ok) {
          sh_ok = mbar_wait_bounded(&bar_c[cp], phc) ? 1 : 0;
          if (!sh_ok) atomicOr(status, ST_TIMEOUT | ST_AT_LU);
          else nc_wait[cp]++;
        }
      }
      __syncthreads();
      if (!sh_ok) { ok = false; break; }
      mbar_wait_bounded(&bar_mma[bp], php);
      mbar_wait_bounded(&bar_c[cp], phc);
      fence_after_sync();
      // element (lr, TC_CW colg + q) of a tile sits at row_base + (q >> 3) * 256 + v[q & 7]
      const int row_base = ((lr >> 5) * 8 + (TC_CW / 8) * colg) * 256 + (lr & 3);
      float* cs = stage_c(cp) + (row < 64 ? 0 : TILE_ELEMS) + row_base;
      float d[TC_CW];
      const uint32_t tcol = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(bp * TC_TMEM_COLS + TC_CW * colg);
      if constexpr (TC_CW == 32) tmem_ld32(tcol, d);
      else tmem_ld16(tcol, d);
      if (mine) {
#pragma unroll
        for (int q = 0; q < TC_CW; ++q) {
          const int o = (q >> 3) * 256 + v_line[q & 7];
          cs[o] = cs[o] - d[q];                 // in place: stored by a bulk copy
        }
      }
      fence_before_sync();
      fence_proxy_async();
      __syncthreads();                          // accumulator buffer and C stage read
      // the updated tile pair leaves by a bulk copy from the C stage, which is refilled once
      // that copy has read it (measured faster than per-thread stores here)
      if (tid == 0) {
        bulk_s2g(a + tile_base(m, I0, Jbeg + p), stage_c(cp), 16384);
        if (two) bulk_s2g(a + tile_base(m, I1, Jbeg + p), stage_c(cp) + TILE_ELEMS, 16384);
        bulk_commit();
        if (p + NC < nJ) {
          bulk_wait_read_all();
          issue_c(cp, Jbeg + p + NC);
        }
      }
    }
  }
  // after an abort: wait (bounded) for this CTA's own copies and tensor-core work still in
  // flight before the shared and tensor memory are released
  if (tid == 0 && !ok) {
    if (!a_done) mbar_wait_bounded(&bar_a, 0);
    for (int b = 0; b < 2; ++b)
      for (; nm_wait[b] < nm_iss[b]; ++nm_wait[b]) mbar_wait_bounded(&bar_mma[b], (uint32_t)nm_wait[b] & 1);
    for (int b = 0; b < NB; ++b)
      for (; nb_wait[b] < nb_iss[b]; ++nb_wait[b]) mbar_wait_bounded(&bar_b[b], (uint32_t)nb_wait[b] & 1);
    for (int b = 0; b < NC; ++b)
      for (; nc_wait[b] < nc_iss[b]; ++nc_wait[b]) mbar_wait_bounded(&bar_c[b], (uint32_t)nc_wait[b] & 1);
  }
  if (tid == 0) bulk_wait_all();                // bulk stores complete before the CTA exits
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 2 * TC_TMEM_COLS);
}

// ---- warp-specialised split-tf32 update ---------------------------------------------------
// Same blocks as lu_update_tc_kernel with split-tf32 operands, but the roles run independently and hand
// over through mbarriers only: thread 0 streams U tiles (after the MMAs that read a stage) and
// C tile pairs (after the epilogue that read a stage) by bulk copies, warp 1 issues the MMAs of
// column J into accumulator buffer J & 1 once its U tile has landed and the epilogue has drained
// that buffer, and EPI warps (4 .. 4 + EPI - 1) finish column J: tensor-memory load, subtract,
// store.  No CTA-wide barrier inside the column loop.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31) == 0 && (*abort_flag || global_ns() - t0 > MBAR_WAIT_LIMIT_NS)) return false;
  }
}

template <int EPI>
__global__ void __launch_bounds__(128 + 32 * EPI, 1)
    lu_update_ws_kernel(float* a, const SubMeta* __restrict__ meta, const unsigned char* __restrict__ ubuf, int s,
                        int jchunk, int* status, const int32_t* __restrict__ pend, const int32_t* __restrict__ hiu,
                        int t_max) {
  using L = TcSmem<2>;
  constexpr int NT = 128 + 32 * EPI, NB = (int)L::NB, NC = (int)L::NC;
  constexpr int CW = 64 / (EPI / 4);            // accumulator columns per epilogue warp
  static_assert(EPI % 4 == 0 && (CW == 32 || CW == 16), "epilogue warps: 8 or 16");
  const SubMeta m = meta[blockIdx.z];
  const int I0 = s + 1 + 2 * blockIdx.x, I1 = I0 + 1;
  const int Jbeg = s + 1 + blockIdx.y * jchunk;
  // tile envelope: L_Is is zero for tile rows past pend, U_sJ for columns past hiu
  int Tend = m.T;
  if (pend) {
    if (64 * I0 >= pend[blockIdx.z * t_max + s]) return;
    Tend = min(Tend, hiu[blockIdx.z] + 1);
  }
  if (I0 >= m.T || Jbeg >= Tend) return;       // before any tensor-memory allocation
  const int nJ = min(Tend, Jbeg + jchunk) - Jbeg;
  const bool two = I1 < m.T;
  const uint32_t pair_bytes = two ? 32768u : 16384u;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_a, b_full[NB], b_empty[NB], c_full[NC], c_empty[NC], t_full[2], t_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int sh_ok;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar_a, 1);
    for (int b = 0; b < NB; ++b) {
      mbar_init(&b_full[b], 1);
      mbar_init(&b_empty[b], 1);
    }
    for (int b = 0; b < NC; ++b) {
      mbar_init(&c_full[b], 1);
      mbar_init(&c_empty[b], EPI);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t_full[b], 1);
      mbar_init(&t_empty[b], EPI);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 2 * TC_TMEM_COLS);
  __syncthreads();
  fence_after_sync();
  const uint32_t taddr = tmem_slot;
  float* rawA = (float*)(base + L::A_RAW);     // C stage 1 until A has been converted
  auto stage_b = [&](int b) { return base + L::B0 + b * L::BSTAGE; };
  auto stage_c = [&](int b) { return (float*)(base + L::C0 + b * L::CSTAGE); };
  // producer bookkeeping (thread 0): copies issued per stage, for the drain
  int nb_iss[NB] = {}, nc_iss[NC] = {};
  auto issue_b = [&](int b, int J) {
    mbar_expect_tx(&b_full[b], L::BBYTES);
    bulk_g2s(stage_b(b), ubuf + (size_t)((m.row_off >> 6) + J) * L::BBYTES, L::BBYTES, &b_full[b]);
    nb_iss[b]++;
  };
  auto issue_c = [&](int b, int J) {
    mbar_expect_tx(&c_full[b], pair_bytes);
    bulk_g2s(stage_c(b), a + tile_base(m, I0, J), 16384, &c_full[b]);
    if (two) bulk_g2s(stage_c(b) + TILE_ELEMS, a + tile_base(m, I1, J), 16384, &c_full[b]);
    nc_iss[b]++;
  };
  bool a_done = false;
  if (tid == 0) {
    mbar_expect_tx(&bar_a, pair_bytes);
    bulk_g2s(rawA, a + tile_base(m, I0, s), 16384, &bar_a);
    if (two) bulk_g2s(rawA + TILE_ELEMS, a + tile_base(m, I1, s), 16384, &bar_a);
    for (int b = 0; b < NB && b < nJ; ++b) issue_b(b, Jbeg + b);
    issue_c(0, Jbeg);
    for (int b = 2; b < NC && b < nJ; ++b) issue_c(b, Jbeg + b);
    sh_ok = mbar_wait_bounded(&bar_a, 0) ? 1 : 0;
    if (!sh_ok) atomicOr(status, ST_TIMEOUT | ST_AT_LU);
    a_done = sh_ok;
  }
  __syncthreads();
  const bool ok = sh_ok != 0;
  if (ok) {
    mbar_wait_bounded(&bar_a, 0);              // completed: makes the copy visible here
    if (!two)
      for (int e = tid; e < TILE_ELEMS; e += NT) rawA[TILE_ELEMS + e] = 0.0f;
    __syncthreads();
    unsigned char* ahi = base + L::A_HI;
    unsigned char* alo = base + L::A_LO;
    for (int e = tid; e < 2 * TILE_ELEMS; e += NT) {
      const int t = e >> 12, el = e & 4095, i = el & 63, k = el >> 6;
      const float x = rawA[t * TILE_ELEMS + off_sw32(i, k)], hi = tf32_round(x);
      const uint32_t o = tf32_a_off(64 * t + i, k);
      *(float*)(ahi + o) = hi;
      *(float*)(alo + o) = tf32_round(x - hi);
    }
    fence_proxy_async();                        // generic writes -> tensor-core reads, bulk refill
    __syncthreads();                            // raw A consumed: C stage 1 is free
  }
  int nt_iss[2] = {0, 0}, ne_iss[NB] = {};    // MMA thread: commits per buffer and per U stage
  bool failed = false;                          // this role gave up a wait
  if (ok && tid == 0) {
    // ---- producer ----
    if (nJ > 1) issue_c(1, Jbeg + 1);
    for (int it = 0; it < nJ; ++it) {
      if (it + NB < nJ) {                      // U stage it % NB: free once the MMAs of column it ran
        if (!ws_wait(&b_empty[it % NB], (uint32_t)(it / NB) & 1, &abort_flag)) { failed = true; break; }
        issue_b(it % NB, Jbeg + it + NB);
      }
      if (it + NC < nJ) {                      // C stage it % NC: free once column it is finished
        if (!ws_wait(&c_empty[it % NC], (uint32_t)(it / NC) & 1, &abort_flag)) { failed = true; break; }
        issue_c(it % NC, Jbeg + it + NC);
      }
    }
  } else if (ok && warp == 1 && lane == 0) {
    // ---- MMA issue ----
    constexpr uint32_t idesc = instr_desc(2);
    const uint64_t dhi = smem_desc(smem_u32(base) + L::A_HI, 16, 1024);
    const uint64_t dlo = smem_desc(smem_u32(base) + L::A_LO, 16, 1024);
    for (int it = 0; it < nJ; ++it) {
      const int bs = it % NB, b = it & 1;
      if (!ws_wait(&b_full[bs], (uint32_t)(it / NB) & 1, &abort_flag) ||
          (it >= 2 && !ws_wait(&t_empty[b], (uint32_t)((it >> 1) - 1) & 1, &abort_flag))) {
        failed = true;
        break;
      }
      fence_after_sync();
      const uint32_t d_tmem = taddr + (uint32_t)(b * TC_TMEM_COLS);
      // a descriptor's start-address field holds addr >> 4: an offset adds (off >> 4)
      const uint64_t db = smem_desc(smem_u32(stage_b(bs)), 16, 1024);
#pragma unroll
      for (int k = 0; k < 8; ++k) {             // K = 8 tf32 values (32 bytes) per instruction
        const uint64_t ka = ((k >> 2) * 16384 + (k & 3) * 32) >> 4;
        const uint64_t kb = ((k >> 2) * 8192 + (k & 3) * 32) >> 4;
        mma<2>(d_tmem, dhi + ka, db + kb, idesc, k > 0 ? 1u : 0u);
        mma<2>(d_tmem, dhi + ka, db + (16384 >> 4) + kb, idesc, 1u);
        mma<2>(d_tmem, dlo + ka, db + kb, idesc, 1u);
      }
      mma_commit(&b_empty[bs]);
      mma_commit(&t_full[b]);
      ne_iss[bs]++;
      nt_iss[b]++;
    }
  } else if (ok && warp >= 4) {
    // ---- epilogue: warp owns rows 32 (warp & 3) + lane and CW columns ----
    const int e = warp - 4, colg = e >> 2;
    const int row = 32 * (warp & 3) + lane;
    const bool mine = row < 64 || two;
    const int lr = row & 63;
    int v_line[8];                              // in-atom offset of column line l of this row
#pragma unroll
    for (int l = 0; l < 8; ++l) v_line[l] = (l << 5) + ((((lr >> 2) & 7) ^ l) << 2);
    // element (lr, CW colg + q) of a tile sits at row_base + (q >> 3) * 256 + v[q & 7]
    const int row_base = ((lr >> 5) * 8 + (CW / 8) * colg) * 256 + (lr & 3);
    for (int p = 0; p < nJ; ++p) {
      const int b = p & 1, cp = p % NC;
      int good = 1;
      if (lane == 0)
        good = ws_wait(&t_full[b], (uint32_t)(p >> 1) & 1, &abort_flag) &&
               ws_wait(&c_full[cp], (uint32_t)(p / NC) & 1, &abort_flag);
      good = __shfl_sync(0xffffffffu, good, 0);
      if (!good) {
        failed = lane == 0;
        break;
      }
      mbar_try_wait(&t_full[b], (uint32_t)(p >> 1) & 1);    // completed: visibility in every lane
      mbar_try_wait(&c_full[cp], (uint32_t)(p / NC) & 1);
      __syncwarp();
      fence_after_sync();
      float d[CW];
      const uint32_t tcol = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * TC_TMEM_COLS + CW * colg);
      if constexpr (CW == 32) tmem_ld32(tcol, d);
      else tmem_ld16(tcol, d);
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&t_empty[b]);   // accumulator buffer b drained by this warp
      const float* cs = stage_c(cp) + (row < 64 ? 0 : TILE_ELEMS) + row_base;
      float* ct = a + tile_base(m, row < 64 ? I0 : I1, Jbeg + p) + row_base;
      if (mine) {
#pragma unroll
        for (int q = 0; q < CW; ++q) {
          const int o = (q >> 3) * 256 + v_line[q & 7];
          ct[o] = cs[o] - d[q];
        }
      }
      fence_proxy_async();                      // generic reads of the stage before its refill
      __syncwarp();
      if (lane == 0) mbar_arrive(&c_empty[cp]);
    }
  }
  if (failed) {                                 // the other roles give up their waits too
    atomicOr(status, ST_TIMEOUT | ST_AT_LU);
    abort_flag = 1;
  }
  // ---- drain: copies and tensor-core work still in flight complete before release ----
  if (tid == 0) {
    if (!a_done) mbar_wait_bounded(&bar_a, 0);
    for (int b = 0; b < NB; ++b)
      if (nb_iss[b] > 0) mbar_wait_bounded(&b_full[b], (uint32_t)(nb_iss[b] - 1) & 1);
    for (int b = 0; b < NC; ++b)
      if (nc_iss[b] > 0) mbar_wait_bounded(&c_full[b], (uint32_t)(nc_iss[b] - 1) & 1);
  }
  if (warp == 1 && lane == 0) {
    for (int b = 0; b < 2; ++b)
      if (nt_iss[b] > 0) mbar_wait_bounded(&t_full[b], (uint32_t)(nt_iss[b] - 1) & 1);
    for (int b = 0; b < NB; ++b)
      if (ne_iss[b] > 0) mbar_wait_bounded(&b_empty[b], (uint32_t)(ne_iss[b] - 1) & 1);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, 2 * TC_TMEM_COLS);
}

constexpr int TC_WS_EPI = 8;             // epilogue warps of the warp-specialised kernel

cudaError_t lu_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(lu_update_ws_kernel<TC_WS_EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(1024 + TcSmem<2>::TOTAL));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(lu_update_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(1024 + TcSmem<1>::TOTAL));
}

cudaError_t launch_lu_update_tc(const FactorDev& f, int step, int bf16, cudaStream_t s, int jchunk) {
  const int W = f.t_max - 1 - step;
  if (W <= 0) return cudaSuccess;
  if (!f.ubuf) return cudaErrorInvalidValue;
  if (jchunk < 1) jchunk = TC_JCHUNK;
  // tile rows below the pivot block that the step can update (tile envelope)
  const int WR = f.pend ? std::min(W, (f.step_rows[step] + 63) / 64 - 1) : W;
  if (WR <= 0) return cudaSuccess;
  dim3 gs(W, f.n_sub);
  dim3 g((WR + 1) / 2, (W + jchunk - 1) / jchunk, f.n_sub);
  unsigned char* ub = (unsigned char*)f.ubuf;
  if (bf16) {
    lu_split_u_kernel<1><<<gs, 256, 0, s>>>((const float*)f.a, f.meta, step, ub, f.hiu);
    lu_update_tc_kernel<1><<<g, TC_LS_THREADS, 1024 + TcSmem<1>::TOTAL, s>>>(
        (float*)f.a, f.meta, ub, step, jchunk, f.status, f.pend, f.hiu, f.t_max);
  } else {
    lu_split_u_kernel<2><<<gs, 256, 0, s>>>((const float*)f.a, f.meta, step, ub, f.hiu);
    lu_update_ws_kernel<TC_WS_EPI><<<g, 128 + 32 * TC_WS_EPI, 1024 + TcSmem<2>::TOTAL, s>>>(
        (float*)f.a, f.meta, ub, step, jchunk, f.status, f.pend, f.hiu, f.t_max);
  }
  return cudaGetLastError();
}

size_t lu_tc_ubuf_bytes(int64_t tile_rows_total, int bf16) {
  return (size_t)tile_rows_total * (bf16 ? TcSmem<1>::BBYTES : TcSmem<2>::BBYTES);
}

}  // namespace cpmdev
