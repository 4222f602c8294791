// Launchers of the device kernels (host-callable), shared by the C ABI implementation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace cpmdev {

// A vector whose address may depend on a device-resident index (so that one captured CUDA
// graph serves every Krylov step): column r is
//   base + r*rhs_stride + (k[r*k_rhs_stride] + k_add)*k_stride      (k null: base + r*rhs_stride)
// and load() multiplies by scale[r*scale_rhs_stride] when scale is set (a basis vector stored
// unnormalised together with its scale).
struct IndirectVec {
  double* base;
  int64_t rhs_stride;
  const int* k;
  int64_t k_stride;
  int k_add;
  int k_rhs_stride = 0;
  const double* scale = nullptr;
  int scale_rhs_stride = 0;
  __device__ __forceinline__ double* ptr(int r) const {
    int kk = k ? (k[r * k_rhs_stride] + k_add) : 0;
    return base + (int64_t)r * rhs_stride + (int64_t)kk * k_stride;
  }
  __device__ __forceinline__ double load(int r, int64_t i) const {
    const double v = ptr(r)[i];
    return scale ? v * scale[r * scale_rhs_stride] : v;
  }
};
inline IndirectVec direct(double* p, int64_t rhs_stride) { return IndirectVec{p, rhs_stride, nullptr, 0, 0}; }

struct OperatorDev {
  const int32_t* pencil;   // N x P^2
  const double* wts;       // N x 3 x P
  const int32_t* nbr;      // N_A x 6
  int64_t n_active, n_nodes;
  int P;
  double diag, invh2;
  const double* wt2 = nullptr;   // (P^2 + P) x N tensor weights (build_tensor_weights), or null
};
// wt2[(b P + c) N + k] = wy_b(k) wz_c(k) and wt2[(P^2 + a) N + k] = wx_a(k) for every band node
// k, from the 1-D weights (N x 3 x P); the extension kernel then needs P^3 + P multiply-adds
// per node instead of P^3 + P^2 + P plus a lane reduction.
cudaError_t launch_build_tensor_weights(const double* wts, double* wt2, int64_t n_nodes, int P, cudaStream_t s);

// kernels issued by each launcher (for the handle's launch counter)
constexpr int KERNELS_APPLY = 2;
constexpr int KERNELS_TRSV = 1;
constexpr int KERNELS_EXT_VALUES = 1;
constexpr int KERNELS_CGS2_GIVENS = 3;   // operator second half fused into the first of them
constexpr int KERNELS_PER_ITERATION = KERNELS_TRSV + KERNELS_EXT_VALUES + KERNELS_CGS2_GIVENS;
constexpr int KERNELS_BEGIN = 1;
constexpr int KERNELS_RESTART_UPDATE = 2;
constexpr int KERNELS_RESIDUAL_CHECK = 2;

// ---- expiry of the bounded waits (test entry point) ----
cudaError_t launch_bounded_wait_selftest(uint64_t limit_ns, const uint32_t* never, int* status, int* out,
                                         cudaStream_t s);

// ---- FP64 FMA probes ----
cudaError_t launch_fma_throughput(int blocks, int threads, int chains, int iters, double* out, cudaStream_t s);
cudaError_t launch_fma_latency(int iters, double* out, long long* cycles, cudaStream_t s);

// ---- stationary (O)RAS solver vectors ----
constexpr int KERNELS_AXPY = 1;
constexpr int KERNELS_NORM2 = 2;
cudaError_t launch_axpy(double* u, const double* z, int64_t n, int nblk, cudaStream_t s);
cudaError_t launch_norm2(const double* x, int64_t n, double* partial, int nblk, double* out, cudaStream_t s);
cudaError_t launch_axpby(int64_t n, double a, const double* x, double b, double* y, int nblk, cudaStream_t s);

cudaError_t launch_apply(const OperatorDev& op, IndirectVec x, double* v_scratch, const double* f,
                         IndirectVec y, int nrhs, int mode, const int* done, cudaStream_t s);
// first half of the operator only: v_scratch[k] = (E x)_k for every band node
cudaError_t launch_ext_values(const OperatorDev& op, IndirectVec x, double* v_scratch, int nrhs, const int* done,
                              cudaStream_t s);

// ---- local factorisation ----
struct FactorDev {
  void* a;                 // working tiles (double for FP64, float otherwise)
  const SubMeta* meta;     // n_sub records
  int32_t* ipiv;           // per padded row: pivot row chosen at that step (local index)
  int* status;             // device status word
  int n_sub;
  int t_max;
  int fp64;                // 1: double tiles, 0: float (swizzled) tiles
  void* ubuf = nullptr;    // tensor-core update: the step's U row split into MMA operands
                           // (lu_tc_ubuf_bytes(rows_total / 64, bf16) bytes)
  // tile envelope of the factors (rows in the order the factorisation leaves them):
  int32_t* first = nullptr;        // per padded row: first nonzero tile column (moves with the row)
  int32_t* last = nullptr;         // per padded row: last tile column that can be nonzero
  const int32_t* pend = nullptr;   // [subdomain * t_max + s]: rows with first <= s lie below this
  int32_t* hiu = nullptr;          // per subdomain: last nonzero tile column of the step's U row
  const int32_t* step_rows = nullptr;   // host, per step: max over subdomains of pend - 64 s
};
cudaError_t launch_scatter(void* a, int fp64, const int64_t* off, const double* val, int64_t nnz,
                           cudaStream_t s);
cudaError_t launch_zero_column(void* a, int fp64, const SubMeta* meta, int j, int col, cudaStream_t s);
cudaError_t launch_pad_identity(void* a, int fp64, const SubMeta* meta, int n_sub, int t_max,
                                cudaStream_t s);
// use_tc: 0 SIMT update, 1 tensor cores with split-tf32 operands, 2 tensor cores with bf16
cudaError_t launch_lu_step(const FactorDev& f, int step, int use_tc, cudaStream_t s);
// jchunk: tile columns per CTA (0 = default)
cudaError_t launch_lu_update_tc(const FactorDev& f, int step, int bf16, cudaStream_t s, int jchunk = 0);
cudaError_t lu_tc_prepare();
size_t lu_tc_ubuf_bytes(int64_t tile_rows_total, int bf16);
// Panel factorisation in a thread-block cluster (shared-memory panel); call once per device
// before launch_lu_step.  Without it the panel runs on one CTA per subdomain from global memory.
cudaError_t lu_panel_prepare();
cudaError_t launch_lu_finish(const FactorDev& f, const int32_t* unknowns, const int64_t* unk_off,
                             const int32_t* own_flag, int32_t* gather, int32_t* scatter,
                             void* dinv, cudaStream_t s);
cudaError_t launch_pack_bf16(const float* a, __nv_bfloat16* out, int64_t n_tiles, cudaStream_t s);
// Replaces L_{I,I-1} by L_II^{-1} L_{I,I-1} and U_{I,I+1} by U_II^{-1} U_{I,I+1} in every tile
// row whose envelope holds them (the solves' chain tiles); inv as from launch_diag_inverse.
cudaError_t launch_chain_tiles(void* a, int fp64, const SubMeta* meta, int n_sub, int t_max, const void* inv,
                               const int32_t* tlo, const int32_t* thi, cudaStream_t s);
// Packs the diagonal-block inverses into their triangles (after launch_chain_tiles)
cudaError_t launch_pack_inverse(void* inv, int fp64, int64_t n_tile_rows, cudaStream_t s);
cudaError_t launch_diag_inverse(const void* a, int fp64, const SubMeta* meta, int n_sub, int t_max,
                                void* inv, cudaStream_t s);

// ---- batched local solves ----
struct TrsvDev {
  const void* tiles;       // factor tiles (double / float swizzled / bf16)
  const void* inv;         // per tile row: L_II^{-1}, U_II^{-1} (compute precision, column-major)
  const SubMeta* meta;
  const int32_t* gather;   // per padded row: global active index of the permuted local row or -1
  const int32_t* scatter;  // per padded row: global index if the unknown is owned, else -1
  const int2* items;       // (subdomain, tile row | segment << 20 | direction << 30)
  int n_items;
  uint64_t* ytag;          // per padded row: published value(s) tagged with the launch epoch
                           // (1 word for FP32: tag<<32 | bits; 2 words for FP64: hi, lo)
  uint64_t* ptag;          // tagged partial sums: per tile row, maxseg segments x 64 rows
  int kseg;                // off-diagonal tiles per work item (long rows are split)
  int maxseg;
  int prefetch;            // 1: a CTA holds its next item and streams it early
  int stagger;             // 1: one queue for both sweeps with staggered subdomains
  uint32_t* sync;          // [0] item counter, [1] finished CTAs, [2] epoch, [3] abort
  int* status;
  int precision;           // 0 fp64, 1 fp32, 2 bf16
  int grid;
  int nr_cap;              // right-hand sides the tagged-word buffers hold per row
  // Tile envelope per tile row (row_off / 64 + I): L tiles [tlo, I), U tiles (I, thi].  It
  // always holds the chain tiles L_{I,I-1} and U_{I,I+1} (zero tiles where the factors have
  // none), so each sweep is one chain: every backward item then follows the subdomain's last
  // forward item, and a row's backward value never overwrites its forward value (the same
  // word) while a forward item still reads it.
  const int32_t* tlo;      // first L tile column (or null: 0)
  const int32_t* thi;      // last U tile column (or null: T - 1)
};
constexpr int TRSV_MAX_NR = 8;
// nr in {1, 2, 4, 8} right-hand sides (r_in / z_out columns) per launch, nr <= t.nr_cap
cudaError_t launch_trsv(const TrsvDev& t, IndirectVec r_in, IndirectVec z_out, const int* done,
                        cudaStream_t s, int nr = 1);
int trsv_ctas_per_sm(int precision);
cudaError_t trsv_prepare(int precision);
// Queue of work items for the batched solve: forward items, then backward items, each
// sorted by the chain position they wait for (partial segments of a row before its
// diagonal item).  T[j] = tiles per dimension of subdomain j; tlo / thi (per tile row, in
// subdomain order) bound each row's nonzero L and U tiles (null: the dense triangle).
void trsv_build_items(const int* T, int n_sub, int kseg, int stagger, std::vector<int2>& items,
                      int* maxseg, const int32_t* tlo = nullptr, const int32_t* thi = nullptr);

// ---- Krylov kernels ----
// FGMRES(m) state of up to nrhs right-hand sides advanced in lock step (right-hand side q at
// offset q times the per-rhs size of every array).
constexpr int GMRES_IST_STRIDE = 16;   // state ints per right-hand side
constexpr int GMRES_SLOT_INT = 6;      // state int: basis / direction slot the solve reads and writes
constexpr int GMRES_VSCALE_DBL = 5;    // scalar: scale of the stored basis vector V[k]
struct GmresDev {
  double* V;        // nrhs x (m+1) x ld: basis; V[k+1] holds w unnormalised until step k+1 scales it
  double* Z;        // nrhs x (m+1) x ld: preconditioned directions (slot m: the solves of a finished rhs)
  double* w;        // nrhs x ld
  double* r;        // nrhs x ld
  double* part;     // nrhs x part_stride: block partial sums of h1, h2 (vector-major: entry i of
                    // block b at i nblk + b) and ||w||^2
  double* st;       // nrhs x st_stride: H, cs, sn, g, y, h1, scalars
  int* ist;         // nrhs x GMRES_IST_STRIDE: [0] k, [1] total, [2] done, [3] status, [4] kdone,
                    // [5] max_it, [6] slot (k, or m once the cycle stopped), [8..11] tickets
  int* ctl;         // [0] right-hand sides whose cycle runs, [1] 1 once none does
  int* status;      // device status word (bounded waits that gave up: ST_TIMEOUT)
  int64_t n;        // rows (N_A)
  int64_t ld;       // leading dimension of the vectors (n rounded up)
  int m;
  int nblk;         // blocks per right-hand side of the vector kernels
  int chunk;        // rows per block
  int nrhs;         // right-hand sides the arrays hold
  int st_stride;
  int64_t part_stride;
};
int gmres_state_size(int m);       // doubles of state for restart length m
int gmres_scalar_offset(int m);     // offset of the scalars (||f||, tol, beta, ||w||, relres, scale)
size_t gmres_step_smem_bytes();    // dynamic shared memory of a step kernel (any rows per block)
cudaError_t gmres_prepare(int m);  // once per device and shape, before the launches
// begin: ||f_q|| (f_q = f + q f_stride), tolerance, iteration limit, for nr right-hand sides
cudaError_t launch_gmres_begin(const GmresDev& g, const double* f, int64_t f_stride, double tol, int max_it,
                               int nr, cudaStream_t s);
// After launch_ext_values(z_k) into vext: w = A z_k, CGS2, Givens (three kernels).
cudaError_t launch_arnoldi_step(const GmresDev& g, const OperatorDev& op, const double* vext, int nr,
                                cudaStream_t s);
cudaError_t launch_gmres_restart_update(const GmresDev& g, double* u, int64_t u_stride, int nr, cudaStream_t s);
cudaError_t launch_gmres_residual_check(const GmresDev& g, int nr, cudaStream_t s);

}  // namespace cpmdev
