// C ABI: entry points that run on the GPU (preconditioner setup, operator apply,
// preconditioner apply, FGMRES).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <memory>
#include <vector>

#include "cuda/kernels.h"
#include "host/cpm_internal.h"

using namespace cpmdev;


namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

cpm_status cuda_fail(cudaError_t e, const char* where) {
  cpm::set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CPM_ERR_OOM : CPM_ERR_CUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

template <typename T>
cudaError_t upload(const std::vector<T>& v, void** d) {
  *d = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(d, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

void cpm::band_release_device(cpm::Band& b) {
  if (b.d_device < 0) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(b.d_device);
  cudaFree(b.d_pencil);
  cudaFree(b.d_wts);
  cudaFree(b.d_nbr);
  cudaFree(b.d_wt2);
  cudaSetDevice(cur);
  b.d_pencil = b.d_wts = b.d_nbr = b.d_wt2 = nullptr;
  b.d_device = -1;
}

struct oras_precond {
  const cpm::Band* band = nullptr;
  int device = -1;
  int n_sub = 0, precision = 0, transmission = 0, t_max = 0;
  double c = 0;
  int64_t n_active = 0, n_nodes = 0;
  std::vector<int64_t> n_local, n_sigma;
  std::vector<SubMeta> meta;
  int64_t sum_n = 0, sum_n2 = 0, sum_sigma = 0, rows_total = 0, tiles_total = 0;
  std::vector<int32_t> tlo, thi;   // per tile row: nonzero L tiles [tlo, I), U tiles (I, thi]
  int64_t solve_offdiag_tiles = 0;
  double ms_assemble = 0, ms_factor = 0;
  int64_t launches = 0;       // kernels launched after setup (graph nodes included)
  int solve_ctas = 0;         // current CTAs per SM of the batched solve
  std::vector<DevBuf> bufs;
  size_t device_bytes = 0, factor_bytes = 0, peak_bytes = 0;
  // device pointers
  void* tiles = nullptr;      // factors used by the solves
  void* dinv = nullptr;
  SubMeta* d_meta = nullptr;
  int32_t* gather = nullptr;
  int32_t* scatter = nullptr;
  int* status = nullptr;
  TrsvDev trsv{};
  OperatorDev op{};
  double* v_scratch = nullptr;     // extension values for cpm_op_apply (nrhs x N)
  int64_t v_scratch_rhs = 0;
  double* g_vext = nullptr;        // extension values owned by the FGMRES path (g_vext_rhs x N)
  int g_vext_rhs = 0;
  // FGMRES workspace
  int g_m = 0;
  GmresDev gm{};
  double* g_state_host = nullptr;  // pinned: TRSV_MAX_NR x 8 scalars
  int* g_istate_host = nullptr;    // pinned: TRSV_MAX_NR x GMRES_IST_STRIDE state ints, then 4 control ints
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t iter_graph[4] = {nullptr, nullptr, nullptr, nullptr};   // one per batch width 1, 2, 4, 8
  void drop_graphs() {
    for (auto& gx : iter_graph)
      if (gx) {
        cudaGraphExecDestroy(gx);
        gx = nullptr;
      }
  }
  // stationary solver workspace
  double *st_z = nullptr, *st_r = nullptr, *st_part = nullptr, *st_norm = nullptr;
  double* st_norm_host = nullptr;
  int st_nblk = 0;

  void* alloc(size_t bytes, cudaError_t* err) {
    void* p = nullptr;
    *err = cudaMalloc(&p, bytes ? bytes : 16);
    if (*err == cudaSuccess) {
      bufs.push_back({p, bytes});
      device_bytes += bytes;
      peak_bytes = std::max(peak_bytes, device_bytes);
    }
    return p;
  }
  void release(void* p) {
    for (size_t i = 0; i < bufs.size(); ++i)
      if (bufs[i].p == p) {
        cudaFree(p);
        device_bytes -= bufs[i].bytes;
        bufs.erase(bufs.begin() + i);
        return;
      }
  }
  ~oras_precond() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0) cudaSetDevice(device);
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto& b : bufs) cudaFree(b.p);
    if (g_state_host) cudaFreeHost(g_state_host);
    if (g_istate_host) cudaFreeHost(g_istate_host);
    if (st_norm_host) cudaFreeHost(st_norm_host);
    if (cur >= 0) cudaSetDevice(cur);
  }
};

#define ALLOC(ptr, type, count)                                            \
  do {                                                                     \
    cudaError_t e__;                                                       \
    ptr = (type*)pc->alloc(sizeof(type) * (size_t)(count), &e__);          \
    if (e__ != cudaSuccess) return cuda_fail(e__, "cudaMalloc " #ptr);     \
  } while (0)

namespace {

// Operators of one band may be set up from several host threads (serving slots); the band's
// device copy is made once, under this lock.
std::mutex g_band_upload_mu;

cpm_status ensure_band_on_device(const cpm::Band& B, int dev) {
  std::lock_guard<std::mutex> lock(g_band_upload_mu);
  if (B.d_device == dev) return CPM_OK;
  if (B.d_device >= 0) cpm::band_release_device(const_cast<cpm::Band&>(B));
  CK(upload(B.pencil, &B.d_pencil));
  CK(upload(B.wts, &B.d_wts));
  CK(upload(B.nbr, &B.d_nbr));
  const int P = B.P();
  const int64_t nn = B.n_nodes();
  CK(cudaMalloc(&B.d_wt2, sizeof(double) * (size_t)(P * P + P) * nn));
  CK(launch_build_tensor_weights((const double*)B.d_wts, (double*)B.d_wt2, nn, P, 0));
  CK(cudaDeviceSynchronize());
  B.d_device = dev;
  return CPM_OK;
}

// Buffers initialised with cudaMemset / cudaMemcpy (the legacy default stream; a pageable
// cudaMemcpy may return before its DMA lands) are read by kernels on the caller's stream, which
// may be a non-blocking stream that does not wait for the legacy stream: fence the legacy
// stream before such buffers are first used.
cudaError_t legacy_fence() { return cudaStreamSynchronize(cudaStreamLegacy); }

// Which bounded device waits gave up, from the status word's diagnostic bits.
std::string timeout_where(int h) {
  std::string w;
  if (h & ST_AT_LU) w += " tensor-core LU update;";
  if (h & ST_AT_SOLVE_POLL) w += " batched solve (published value);";
  if (h & ST_AT_SOLVE_COPY) w += " batched solve (factor copy);";
  if (h & ST_AT_KRYLOV) w += " Arnoldi step (basis copy);";
  return w.empty() ? std::string(" unknown") : w;
}

int sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Work-item queue and partial-sum slots of the batched solve for a split length kseg,
// and its grid.  Drops the captured iteration graph (it holds the old schedule).
cpm_status set_schedule(oras_precond* pc, int ctas_per_sm, int kseg, int prefetch, int stagger) {
  TrsvDev& t = pc->trsv;
  if (kseg != t.kseg || stagger != t.stagger || !t.items) {
    std::vector<int2> items;
    std::vector<int> Ts(pc->n_sub);
    for (int j = 0; j < pc->n_sub; ++j) Ts[j] = pc->meta[j].T;
    int maxseg = 1;
    trsv_build_items(Ts.data(), pc->n_sub, kseg, stagger, items, &maxseg,
                     pc->tlo.empty() ? nullptr : pc->tlo.data(), pc->thi.empty() ? nullptr : pc->thi.data());
    if (t.items) pc->release(const_cast<int2*>(t.items));
    if (t.ptag) pc->release(t.ptag);
    t.items = nullptr;
    t.ptag = nullptr;
    const int words = pc->precision == CPM_FP64 ? 2 : 1;
    const int64_t nslot = (int64_t)words * (pc->rows_total / TILE) * maxseg * TILE * std::max(1, t.nr_cap);
    int2* d_items;
    uint64_t* d_ptag;
    ALLOC(d_items, int2, items.size());
    ALLOC(d_ptag, uint64_t, nslot);
    CK(cudaMemcpy(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(d_ptag, 0, 8 * (size_t)nslot));
    CK(legacy_fence());
    t.items = d_items;
    t.n_items = (int)items.size();
    t.ptag = d_ptag;
    t.kseg = kseg;
    t.stagger = stagger;
    t.maxseg = maxseg;
  }
  t.prefetch = prefetch;
  t.grid = sm_count(pc->device) * ctas_per_sm;
  pc->solve_ctas = ctas_per_sm;
  pc->drop_graphs();
  return CPM_OK;
}

cpm_status setup_impl(oras_precond* pc, const cpm::Band& B, const cpm::Partition& P, double c,
                      int transmission, double alpha, double alpha_x, int precision, bool simt_lu,
                      cudaStream_t s, int zero_column_of = -1) {
  const int ns = P.n_sub;
  pc->band = &B;
  pc->n_sub = ns;
  pc->c = c;
  pc->precision = precision;
  pc->transmission = transmission;
  pc->n_active = B.n_active;
  pc->n_nodes = B.n_nodes();
  CK(cudaGetDevice(&pc->device));
  cpm_status st = ensure_band_on_device(B, pc->device);
  if (st != CPM_OK) return st;

  // ---- host, per subdomain in one parallel loop: the local operator in coordinate form, its
  // fill-reducing order (reverse Cuthill-McKee) and the tile envelope of its factors ----
  std::vector<cpm::LocalCOO> coo(ns);
  std::vector<cpm_status> sts(ns, CPM_OK);
  std::vector<std::string> errs(ns);
  std::vector<std::vector<int32_t>> inv_order(ns), env_first(ns), env_last(ns), env_pend(ns);
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < ns; ++j) {
    try {
      sts[j] = cpm::build_local_coo(B, P, c, transmission, alpha, alpha_x, j, coo[j], false);
      if (sts[j] != CPM_OK) {
        errs[j] = cpm_last_error();
        continue;
      }
      std::vector<int32_t> perm;
      cpm::rcm_order(coo[j], perm);
      std::vector<int32_t>& inv = inv_order[j];
      inv.resize(coo[j].n);
      for (int64_t k = 0; k < coo[j].n; ++k) inv[perm[k]] = (int32_t)k;
      for (auto& r : coo[j].row) r = inv[r];
      for (auto& cc : coo[j].col) cc = inv[cc];
      cpm::envelope(coo[j], (int)((coo[j].n + TILE - 1) / TILE), env_first[j], env_last[j], env_pend[j]);
    } catch (const std::bad_alloc&) {
      sts[j] = CPM_ERR_OOM;
      errs[j] = "out of host memory building local operators";
    }
  }
  for (int j = 0; j < ns; ++j)
    if (sts[j] != CPM_OK) {
      cpm::set_error(errs[j]);
      return sts[j];
    }
  pc->meta.resize(ns);
  pc->n_local.resize(ns);
  pc->n_sigma.resize(ns);
  int64_t tile_off = 0, row_off = 0, nnz = 0;
  int t_max = 0;
  for (int j = 0; j < ns; ++j) {
    const int64_t n = coo[j].n;
    const int T = (int)((n + TILE - 1) / TILE);
    SubMeta m{};
    m.tile_off = tile_off;
    m.row_off = row_off;
    m.T = T;
    m.n = (int32_t)n;
    m.n_sigma = (int32_t)coo[j].n_sigma;
    pc->meta[j] = m;
    pc->n_local[j] = n;
    pc->n_sigma[j] = coo[j].n_sigma;
    tile_off += (int64_t)T * T * TILE_ELEMS;
    row_off += (int64_t)T * TILE;
    nnz += (int64_t)coo[j].val.size();
    t_max = std::max(t_max, T);
    pc->sum_n += n;
    pc->sum_n2 += n * n;
    pc->sum_sigma += coo[j].n_sigma;
  }
  pc->t_max = t_max;
  pc->rows_total = row_off;
  pc->tiles_total = tile_off / TILE_ELEMS;
  // tile envelope of the factors: per row first / last tile column, per step the panel's rows
  std::vector<int32_t> h_first(row_off), h_last(row_off), h_pend((size_t)ns * t_max, 0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < ns; ++j) {
    const SubMeta& m = pc->meta[j];
    std::copy(env_first[j].begin(), env_first[j].end(), h_first.begin() + m.row_off);
    std::copy(env_last[j].begin(), env_last[j].end(), h_last.begin() + m.row_off);
    std::copy(env_pend[j].begin(), env_pend[j].end(), h_pend.begin() + (size_t)j * t_max);
    std::vector<int32_t>().swap(env_first[j]);
    std::vector<int32_t>().swap(env_last[j]);
    std::vector<int32_t>().swap(env_pend[j]);
  }
  std::vector<int32_t> step_rows(t_max, 64);
  for (int j = 0; j < ns; ++j)
    for (int st2 = 0; st2 < pc->meta[j].T; ++st2)
      step_rows[st2] = std::max(step_rows[st2], h_pend[(size_t)j * t_max + st2] - 64 * st2);
  const bool fp64 = precision == CPM_FP64;
  const size_t wbytes = fp64 ? 8 : 4;

  // element offsets of every entry in the tiled layout
  // not value-initialised: the parallel loop below writes (and first-touches) every entry
  std::unique_ptr<int64_t[]> h_off(new int64_t[nnz > 0 ? nnz : 1]);
  std::unique_ptr<double[]> h_val(new double[nnz > 0 ? nnz : 1]);
  {
    std::vector<int64_t> start(ns + 1, 0);
    for (int j = 0; j < ns; ++j) start[j + 1] = start[j] + (int64_t)coo[j].val.size();
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < ns; ++j) {
      const SubMeta& m = pc->meta[j];
      const cpm::LocalCOO& L = coo[j];
      for (size_t e = 0; e < L.val.size(); ++e) {
        const int i = L.row[e], k = L.col[e];
        const int64_t tb = m.tile_off + ((int64_t)(k >> 6) * m.T + (i >> 6)) * TILE_ELEMS;
        h_off[start[j] + e] = tb + (fp64 ? off_plain(i & 63, k & 63) : off_sw32(i & 63, k & 63));
        h_val[start[j] + e] = L.val[e];
      }
    }
  }
  // unknown -> global index, ownership flags
  std::vector<int32_t> unknowns(pc->sum_n), own(pc->sum_n, 0);
  std::vector<int64_t> unk_off(ns);
  {
    int64_t o = 0;
    std::vector<uint8_t> mine(B.n_active, 0);
    for (int j = 0; j < ns; ++j) {
      const cpm::SubSets& S = P.subs[j];
      unk_off[j] = o;
      for (int32_t g : S.own) mine[g] = 1;
      // local unknown t (Sigma_j, then Sigma_j^{BC,A}) sits at position inv[t] of the order;
      // flags: 1 = in the disjoint set (prolonged), 2 = in Sigma_j (carries the residual)
      const std::vector<int32_t>& inv = inv_order[j];
      int64_t t = 0;
      for (int32_t g : S.sigma) { unknowns[o + inv[t]] = g; own[o + inv[t]] = mine[g] | 2; ++t; }
      if (transmission != CPM_RAS)
        for (int32_t g : S.bc_a) { unknowns[o + inv[t]] = g; own[o + inv[t]] = 0; ++t; }
      for (int32_t g : S.own) mine[g] = 0;
      o += pc->n_local[j];
    }
  }
  coo.clear();
  coo.shrink_to_fit();

  // ---- device buffers ----
  void* work;
  {
    cudaError_t e;
    work = pc->alloc(wbytes * (size_t)tile_off, &e);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc factor tiles");
  }
  int32_t* ipiv;
  ALLOC(pc->d_meta, SubMeta, ns);
  ALLOC(ipiv, int32_t, row_off);
  ALLOC(pc->gather, int32_t, row_off);
  ALLOC(pc->scatter, int32_t, row_off);
  ALLOC(pc->status, int, 2);                  // [0] status bits, [1] lowest singular subdomain
  void* dinv;
  {
    cudaError_t e;
    dinv = pc->alloc(wbytes * (size_t)row_off, &e);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc dinv");
  }
  pc->dinv = dinv;
  int32_t *d_unk, *d_own;
  int64_t *d_unk_off, *d_off;
  double* d_val;
  ALLOC(d_unk, int32_t, pc->sum_n);
  ALLOC(d_own, int32_t, pc->sum_n);
  ALLOC(d_unk_off, int64_t, ns);
  ALLOC(d_off, int64_t, nnz);
  ALLOC(d_val, double, nnz);
  CK(cudaMemcpyAsync(pc->d_meta, pc->meta.data(), sizeof(SubMeta) * ns, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_unk, unknowns.data(), 4 * pc->sum_n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_own, own.data(), 4 * pc->sum_n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_unk_off, unk_off.data(), 8 * ns, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_off, h_off.get(), 8 * nnz, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_val, h_val.get(), 8 * nnz, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(pc->status, 0, sizeof(int), s));
  CK(cudaMemsetAsync(pc->status + 1, 0x7f, sizeof(int), s));

  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  CK(cudaEventRecord(e0, s));
  CK(cudaMemsetAsync(work, 0, wbytes * (size_t)tile_off, s));
  CK(launch_pad_identity(work, fp64, pc->d_meta, ns, t_max, s));
  CK(launch_scatter(work, fp64, d_off, d_val, nnz, s));
  if (zero_column_of >= 0 && zero_column_of < ns) CK(launch_zero_column(work, fp64, pc->d_meta, zero_column_of, 0, s));
  CK(cudaEventRecord(e1, s));
  FactorDev f{work, pc->d_meta, ipiv, pc->status, ns, t_max, fp64 ? 1 : 0};
  int32_t *d_first, *d_last, *d_pend, *d_hiu;
  ALLOC(d_first, int32_t, row_off);
  ALLOC(d_last, int32_t, row_off);
  ALLOC(d_pend, int32_t, (int64_t)ns * t_max);
  ALLOC(d_hiu, int32_t, ns);
  CK(cudaMemcpyAsync(d_first, h_first.data(), 4 * (size_t)row_off, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_last, h_last.data(), 4 * (size_t)row_off, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_pend, h_pend.data(), 4 * h_pend.size(), cudaMemcpyHostToDevice, s));
  f.first = d_first;
  f.last = d_last;
  f.pend = d_pend;
  f.hiu = d_hiu;
  f.step_rows = step_rows.data();
  // FP32: split-tf32 tensor-core update (FP32 accuracy); BF16: bf16 inputs, FP32 accumulate
  const int use_tc = (precision == CPM_FP64 || simt_lu) ? 0 : (precision == CPM_BF16 ? 2 : 1);
  void* ubuf = nullptr;
  if (use_tc) {
    CK(lu_tc_prepare());
    cudaError_t e;
    ubuf = pc->alloc(lu_tc_ubuf_bytes(row_off / TILE, use_tc == 2), &e);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc split U operands");
    f.ubuf = ubuf;
  }
  CK(lu_panel_prepare());
  for (int step = 0; step < t_max; ++step) CK(launch_lu_step(f, step, use_tc, s));
  CK(launch_lu_finish(f, d_unk, d_unk_off, d_own, pc->gather, pc->scatter, dinv, s));
  void* inv;
  {
    cudaError_t e;
    inv = pc->alloc(2 * wbytes * (size_t)row_off * TILE, &e);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc diagonal-block inverses");
  }
  CK(launch_diag_inverse(work, fp64, pc->d_meta, ns, t_max, inv, s));
  CK(cudaEventRecord(e2, s));
  CK(cudaStreamSynchronize(s));
  float ms1 = 0, ms2 = 0;
  cudaEventElapsedTime(&ms1, e0, e1);
  cudaEventElapsedTime(&ms2, e1, e2);
  pc->ms_assemble = ms1;
  pc->ms_factor = ms2;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  pc->release(d_off);
  pc->release(d_val);
  pc->release(d_unk);
  pc->release(d_own);
  pc->release(d_unk_off);
  pc->release(ipiv);
  if (ubuf) pc->release(ubuf);
  // final envelope: per tile row the first nonzero L tile and the last nonzero U tile
  CK(cudaMemcpy(h_first.data(), d_first, 4 * (size_t)row_off, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(h_last.data(), d_last, 4 * (size_t)row_off, cudaMemcpyDeviceToHost));
  pc->release(d_first);
  pc->release(d_last);
  pc->release(d_pend);
  pc->release(d_hiu);
  const int64_t n_trow = row_off / TILE;
  pc->tlo.assign(n_trow, 0);
  pc->thi.assign(n_trow, 0);
  pc->solve_offdiag_tiles = 0;
  for (int j = 0; j < ns; ++j) {
    const SubMeta& m = pc->meta[j];
    for (int I = 0; I < m.T; ++I) {
      const int64_t tr = (m.row_off >> 6) + I;
      int32_t lo = I, hi = I;
      for (int r = 0; r < TILE; ++r) {
        lo = std::min(lo, h_first[m.row_off + 64 * I + r]);
        hi = std::max(hi, h_last[m.row_off + 64 * I + r]);
      }
      // the chain tiles L_{I,I-1} and U_{I,I+1} are always in the envelope (zero where the
      // factors have none): each sweep is then one chain of dependencies
      pc->tlo[tr] = I > 0 ? std::min(lo, I - 1) : lo;
      pc->thi[tr] = I < m.T - 1 ? std::max(std::min(hi, m.T - 1), I + 1) : m.T - 1;
      pc->solve_offdiag_tiles += (I - lo) + (pc->thi[tr] - I);
    }
  }
  int32_t *d_tlo, *d_thi;
  ALLOC(d_tlo, int32_t, n_trow);
  ALLOC(d_thi, int32_t, n_trow);
  CK(cudaMemcpy(d_tlo, pc->tlo.data(), 4 * (size_t)n_trow, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_thi, pc->thi.data(), 4 * (size_t)n_trow, cudaMemcpyHostToDevice));
  CK(legacy_fence());
  // chain tiles of the solves: L_{I,I-1} and U_{I,I+1} premultiplied by the diagonal inverses
  CK(launch_chain_tiles(work, fp64, pc->d_meta, ns, t_max, inv, d_tlo, d_thi, s));
  CK(launch_pack_inverse(inv, fp64, n_trow, s));       // the solves stream the triangles only
  CK(cudaStreamSynchronize(s));
  int hst2[2] = {0, 0};
  CK(cudaMemcpy(hst2, pc->status, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  const int hst = hst2[0];
  if (hst & ST_SINGULAR) {
    cpm::set_error("oras_setup: zero pivot in the local LU factorisation of subdomain " +
                   std::to_string(hst2[1]) + " (singular local matrix)");
    return CPM_ERR_SINGULAR;
  }
  if (hst & ST_TIMEOUT) {
    CK(cudaMemsetAsync(pc->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    cpm::set_error("oras_setup: a bounded device-side wait of the factorisation gave up:" + timeout_where(hst));
    return CPM_ERR_TIMEOUT;
  }
  if (precision == CPM_BF16) {
    cudaError_t e;
    void* lp = pc->alloc(2 * (size_t)tile_off, &e);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc bf16 factors");
    CK(launch_pack_bf16((const float*)work, (__nv_bfloat16*)lp, pc->tiles_total, s));
    CK(cudaStreamSynchronize(s));
    pc->release(work);
    pc->tiles = lp;
    pc->factor_bytes = 2 * (size_t)tile_off;
  } else {
    pc->tiles = work;
    pc->factor_bytes = wbytes * (size_t)tile_off;
  }

  // ---- persistent triangular-solve schedule ----
  uint32_t* d_sync;
  uint64_t* d_ytag;
  const int words = fp64 ? 2 : 1;             // tagged 64-bit words per published value
  ALLOC(d_sync, uint32_t, 4);
  ALLOC(d_ytag, uint64_t, (int64_t)words * row_off);
  CK(cudaMemset(d_ytag, 0, 8 * (size_t)words * row_off));
  CK(cudaMemset(d_sync, 0, 16));
  CK(legacy_fence());
  pc->release(dinv);
  pc->dinv = nullptr;
  TrsvDev& t = pc->trsv;
  t.tiles = pc->tiles;
  t.inv = inv;
  t.meta = pc->d_meta;
  t.gather = pc->gather;
  t.scatter = pc->scatter;
  t.ytag = d_ytag;
  t.sync = d_sync;
  t.status = pc->status;
  t.precision = precision;
  t.nr_cap = 1;
  t.tlo = d_tlo;
  t.thi = d_thi;
  CK(trsv_prepare(precision));
  st = set_schedule(pc, trsv_ctas_per_sm(precision), 1023, 0, 0);
  if (st != CPM_OK) return st;

  // ---- operator ----
  OperatorDev& op = pc->op;
  op.pencil = (const int32_t*)B.d_pencil;
  op.wts = (const double*)B.d_wts;
  op.nbr = (const int32_t*)B.d_nbr;
  op.n_active = B.n_active;
  op.n_nodes = B.n_nodes();
  op.P = B.P();
  op.diag = c + 6.0 / (B.h * B.h);
  op.invh2 = 1.0 / (B.h * B.h);
  op.wt2 = (const double*)B.d_wt2;
  return CPM_OK;
}

cpm_status ensure_v_scratch(oras_precond* pc, int nrhs) {
  if (pc->v_scratch_rhs >= nrhs) return CPM_OK;
  if (pc->v_scratch) pc->release(pc->v_scratch);
  pc->v_scratch = nullptr;
  pc->v_scratch_rhs = 0;
  ALLOC(pc->v_scratch, double, (int64_t)nrhs * pc->n_nodes);
  pc->v_scratch_rhs = nrhs;
  return CPM_OK;
}

int width_index(int nr) { return nr >= 8 ? 3 : (nr >= 4 ? 2 : (nr >= 2 ? 1 : 0)); }

// FGMRES workspace for restart length m and batches of up to nr right-hand sides (1, or
// TRSV_MAX_NR once a batch is asked for).  Rows are split into blocks of a multiple of 32
// rows, one block per SM (more for very long vectors, so that a block's rows fit in shared
// memory); vectors have a leading dimension rounded up to 32 doubles.
cpm_status ensure_gmres(oras_precond* pc, int m, int nr) {
  const int cap = nr > 1 ? TRSV_MAX_NR : 1;
  GmresDev& g = pc->gm;
  if (pc->g_m == m && g.nrhs >= cap) return CPM_OK;
  for (void* p : {(void*)g.V, (void*)g.Z, (void*)g.w, (void*)g.r, (void*)g.part, (void*)g.st, (void*)g.ist,
                  (void*)g.ctl})
    if (p) pc->release(p);
  pc->drop_graphs();
  g = GmresDev{};
  pc->g_m = 0;
  const int64_t n = pc->n_active;
  g.n = n;
  g.ld = (n + 31) / 32 * 32;
  g.m = m;
  g.nrhs = cap;
  g.status = pc->status;
  const int64_t sms = sm_count(pc->device);
  // one block per SM (a single wave at any size): the step kernels stream a block's rows in
  // tiles, so the rows per block are not limited by shared memory
  int64_t nblk = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms));
  const int64_t chunk = ((n + nblk - 1) / nblk + 31) / 32 * 32;
  nblk = (n + chunk - 1) / chunk;
  g.nblk = (int)std::max<int64_t>(1, nblk);
  g.chunk = (int)chunk;
  g.st_stride = (gmres_state_size(m) + 7) / 8 * 8;
  g.part_stride = (int64_t)g.nblk * (2 * (m + 1) + 1);
  ALLOC(g.V, double, (int64_t)cap * (m + 1) * g.ld);
  ALLOC(g.Z, double, (int64_t)cap * (m + 1) * g.ld);
  ALLOC(g.w, double, (int64_t)cap * g.ld);
  ALLOC(g.r, double, (int64_t)cap * g.ld);
  ALLOC(g.part, double, (int64_t)cap * g.part_stride);
  ALLOC(g.st, double, (int64_t)cap * g.st_stride);
  ALLOC(g.ist, int, cap * GMRES_IST_STRIDE);
  ALLOC(g.ctl, int, 4);
  CK(cudaMemset(g.V, 0, sizeof(double) * (size_t)cap * (m + 1) * g.ld));
  CK(cudaMemset(g.Z, 0, sizeof(double) * (size_t)cap * (m + 1) * g.ld));
  CK(cudaMemset(g.st, 0, sizeof(double) * (size_t)cap * g.st_stride));
  CK(cudaMemset(g.ist, 0, sizeof(int) * cap * GMRES_IST_STRIDE));
  CK(cudaMemset(g.ctl, 0, 4 * sizeof(int)));
  CK(legacy_fence());
  CK(gmres_prepare(m));
  if (!pc->g_istate_host)
    CK(cudaMallocHost(&pc->g_istate_host, (TRSV_MAX_NR * GMRES_IST_STRIDE + 4) * sizeof(int)));
  if (!pc->g_state_host) CK(cudaMallocHost(&pc->g_state_host, TRSV_MAX_NR * 8 * sizeof(double)));
  if (pc->g_vext_rhs < cap) {
    if (pc->g_vext) pc->release(pc->g_vext);
    pc->g_vext = nullptr;
    pc->g_vext_rhs = 0;
    ALLOC(pc->g_vext, double, (int64_t)cap * pc->n_nodes);
    pc->g_vext_rhs = cap;
  }
  pc->g_m = m;
  return CPM_OK;
}

// One FGMRES iteration of nr right-hand sides: z_k = M^{-1} v_k (one solve launch for all of
// them), vext = E z_k, then w = A z_k, CGS2 and Givens.  A right-hand side whose cycle has
// stopped points its solve at the spare slot m and skips the Arnoldi kernels; once none runs,
// every kernel returns at once.
cpm_status launch_iteration(oras_precond* pc, int nr, cudaStream_t s) {
  GmresDev& g = pc->gm;
  const int* alldone = g.ctl + 1;
  const int64_t rs = (int64_t)(g.m + 1) * g.ld;
  IndirectVec vk{g.V, rs, g.ist + GMRES_SLOT_INT, g.ld, 0, GMRES_IST_STRIDE,
                 g.st + gmres_scalar_offset(g.m) + GMRES_VSCALE_DBL, g.st_stride};
  IndirectVec zk{g.Z, rs, g.ist + GMRES_SLOT_INT, g.ld, 0, GMRES_IST_STRIDE};
  CK(launch_trsv(pc->trsv, vk, zk, alldone, s, nr));
  CK(launch_ext_values(pc->op, zk, pc->g_vext, nr, alldone, s));
  CK(launch_arnoldi_step(g, pc->op, pc->g_vext, nr, s));
  pc->launches += KERNELS_PER_ITERATION;
  return CPM_OK;
}

cpm_status capture_graph(oras_precond* pc, int nr) {
  if (!pc->cap_stream) CK(cudaStreamCreateWithFlags(&pc->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(pc->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = pc->launches;
  cpm_status st = launch_iteration(pc, nr, pc->cap_stream);
  pc->launches = before;
  cudaError_t e = cudaStreamEndCapture(pc->cap_stream, &graph);
  if (st != CPM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&pc->iter_graph[width_index(nr)], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return CPM_OK;
}

// nr (1, 2, 4 or 8) right-hand sides solved in lock step.  Every right-hand side runs the
// operations of a single-rhs solve; the batch shares launches and the factor stream.
cpm_status solve_batch(oras_precond* pc, const double* f, double* u, int nr, const cpm_gmres_opts& o,
                       bool use_graph, cpm_gmres_result* res, cudaStream_t s) {
  GmresDev& g = pc->gm;
  const int64_t n = pc->n_active;
  int* ih = pc->g_istate_host;
  int* ctl_h = ih + TRSV_MAX_NR * GMRES_IST_STRIDE;
  if (o.zero_guess) CK(cudaMemsetAsync(u, 0, sizeof(double) * n * nr, s));
  CK(launch_gmres_begin(g, f, n, o.tol, o.max_it, nr, s));
  CK(launch_apply(pc->op, direct(u, n), pc->g_vext, f, direct(g.r, g.ld), nr, 1, nullptr, s));
  CK(launch_gmres_residual_check(g, nr, s));
  pc->launches += KERNELS_BEGIN + KERNELS_APPLY + KERNELS_RESIDUAL_CHECK;
  cudaGraphExec_t gx = use_graph ? pc->iter_graph[width_index(nr)] : nullptr;
  for (;;) {
    CK(cudaMemcpyAsync(ih, g.ist, sizeof(int) * nr * GMRES_IST_STRIDE, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int live = 0;
    for (int q = 0; q < nr; ++q) live += ih[q * GMRES_IST_STRIDE + 3] == -1;   // status RUNNING
    if (live == 0) break;
    ctl_h[0] = live;
    ctl_h[1] = 0;
    CK(cudaMemcpyAsync(g.ctl, ctl_h, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int it = 0; it < g.m; ++it) {
      if (gx) {
        CK(cudaGraphLaunch(gx, s));
        pc->launches += KERNELS_PER_ITERATION;
      } else {
        cpm_status st = launch_iteration(pc, nr, s);
        if (st != CPM_OK) return st;
      }
    }
    CK(launch_gmres_restart_update(g, u, n, nr, s));
    CK(launch_apply(pc->op, direct(u, n), pc->g_vext, f, direct(g.r, g.ld), nr, 1, nullptr, s));
    CK(launch_gmres_residual_check(g, nr, s));
    pc->launches += KERNELS_RESTART_UPDATE + KERNELS_APPLY + KERNELS_RESIDUAL_CHECK;
  }
  CK(cudaMemcpy2DAsync(pc->g_state_host, 8 * sizeof(double), g.st + gmres_scalar_offset(g.m),
                       sizeof(double) * g.st_stride, 8 * sizeof(double), nr, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int dst = 0;
  CK(cudaMemcpy(&dst, pc->status, sizeof(int), cudaMemcpyDeviceToHost));
  for (int q = 0; q < nr; ++q) {
    res[q].iterations = ih[q * GMRES_IST_STRIDE + 1];
    res[q].relres = pc->g_state_host[q * 8 + 4];
    res[q].status = ih[q * GMRES_IST_STRIDE + 3];
  }
  if (dst & ST_TIMEOUT) {
    CK(cudaMemsetAsync(pc->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < nr; ++q) res[q].status = CPM_ERR_TIMEOUT;
  }
  return CPM_OK;
}

cpm_status ensure_stationary(oras_precond* pc) {
  if (pc->st_z) return CPM_OK;
  const int64_t n = pc->n_active;
  pc->st_nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count(pc->device)));
  ALLOC(pc->st_z, double, n * TRSV_MAX_NR);
  ALLOC(pc->st_r, double, n * TRSV_MAX_NR);
  ALLOC(pc->st_part, double, pc->st_nblk);
  ALLOC(pc->st_norm, double, TRSV_MAX_NR);
  if (!pc->st_norm_host) CK(cudaMallocHost(&pc->st_norm_host, TRSV_MAX_NR * sizeof(double)));
  if (!pc->g_vext) {
    ALLOC(pc->g_vext, double, pc->n_nodes);
    pc->g_vext_rhs = 1;
  }
  return CPM_OK;
}

// ||x_q||_2 for the listed columns (device), returned to the host with one synchronisation.
cpm_status norms_to_host(oras_precond* pc, const double* x, int64_t ld, const int* cols, int ncols, double* out,
                         cudaStream_t s) {
  for (int c = 0; c < ncols; ++c)
    CK(launch_norm2(x + (int64_t)cols[c] * ld, pc->n_active, pc->st_part, pc->st_nblk, pc->st_norm + cols[c], s));
  CK(cudaMemcpyAsync(pc->st_norm_host, pc->st_norm, TRSV_MAX_NR * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  pc->launches += (int64_t)KERNELS_NORM2 * ncols;
  for (int c = 0; c < ncols; ++c) out[cols[c]] = pc->st_norm_host[cols[c]];
  return CPM_OK;
}

// nr (<= TRSV_MAX_NR) right-hand sides iterated together: one batched solve launch per
// iteration for all of them; a right-hand side that has converged (or failed) is no longer
// updated, so each one follows exactly the single right-hand-side sequence of operations.
cpm_status stationary_batch(oras_precond* pc, const double* f, double* u, int nr, double tol, int max_it,
                            cpm_gmres_result* res, cudaStream_t s) {
  const int64_t n = pc->n_active;
  double nf[TRSV_MAX_NR] = {0}, nrm[TRSV_MAX_NR] = {0};
  int act[TRSV_MAX_NR], nact = 0, all[TRSV_MAX_NR];
  for (int q = 0; q < nr; ++q) all[q] = q;
  CK(cudaMemsetAsync(u, 0, sizeof(double) * n * nr, s));
  cpm_status st = norms_to_host(pc, f, n, all, nr, nf, s);
  if (st != CPM_OK) return st;
  for (int q = 0; q < nr; ++q) {
    res[q].iterations = 0;
    res[q].relres = 0.0;
    res[q].status = CPM_OK;
    if (!std::isfinite(nf[q])) res[q].status = CPM_ERR_NAN;
    else if (nf[q] > 0.0) {
      res[q].status = CPM_ERR_NOT_CONVERGED;
      act[nact++] = q;
    }
  }
  CK(cudaMemcpyAsync(pc->st_r, f, sizeof(double) * n * nr, cudaMemcpyDeviceToDevice, s));
  for (int it = 1; it <= max_it && nact > 0; ++it) {
    CK(launch_trsv(pc->trsv, direct(pc->st_r, n), direct(pc->st_z, n), nullptr, s, nr));
    pc->launches += KERNELS_TRSV;
    for (int c = 0; c < nact; ++c) {
      const int q = act[c];
      CK(launch_axpy(u + (int64_t)q * n, pc->st_z + (int64_t)q * n, n, pc->st_nblk, s));
      CK(launch_apply(pc->op, direct(u + (int64_t)q * n, 0), pc->g_vext, f + (int64_t)q * n,
                      direct(pc->st_r + (int64_t)q * n, 0), 1, 1, nullptr, s));
      pc->launches += KERNELS_AXPY + KERNELS_APPLY;
    }
    st = norms_to_host(pc, pc->st_r, n, act, nact, nrm, s);
    if (st != CPM_OK) return st;
    int keep = 0;
    for (int c = 0; c < nact; ++c) {
      const int q = act[c];
      res[q].iterations = it;
      res[q].relres = nrm[q] / nf[q];
      if (!std::isfinite(nrm[q])) res[q].status = CPM_ERR_NAN;
      else if (nrm[q] <= tol * nf[q]) res[q].status = CPM_OK;
      else act[keep++] = q;
    }
    nact = keep;
  }
  int dst = 0;
  CK(cudaMemcpy(&dst, pc->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (dst & ST_TIMEOUT) {
    CK(cudaMemsetAsync(pc->status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < nr; ++q) res[q].status = CPM_ERR_TIMEOUT;
  }
  return CPM_OK;
}

// Tagged-word buffers of the batched solve for TRSV_MAX_NR right-hand sides per launch
// (grown once; drops the captured iteration graph, which holds the old buffers).
cpm_status ensure_multi_rhs(oras_precond* pc) {
  TrsvDev& t = pc->trsv;
  if (t.nr_cap >= TRSV_MAX_NR) return CPM_OK;
  const int words = pc->precision == CPM_FP64 ? 2 : 1;
  uint64_t *y = nullptr, *pt = nullptr;
  const int64_t ny = (int64_t)words * pc->rows_total * TRSV_MAX_NR;
  const int64_t np = (int64_t)words * (pc->rows_total / TILE) * t.maxseg * TILE * TRSV_MAX_NR;
  ALLOC(y, uint64_t, ny);
  ALLOC(pt, uint64_t, np);
  CK(cudaMemset(y, 0, 8 * (size_t)ny));
  CK(cudaMemset(pt, 0, 8 * (size_t)np));
  CK(cudaDeviceSynchronize());
  pc->release(t.ytag);
  pc->release(t.ptag);
  t.ytag = y;
  t.ptag = pt;
  t.nr_cap = TRSV_MAX_NR;
  pc->drop_graphs();
  return CPM_OK;
}

// Largest launch width in {8, 4, 2, 1} not above the right-hand sides left.
int nr_chunk(int left) { return left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1)); }

}  // namespace

extern "C" {

cpm_status oras_setup(const cpm_band* band, const cpm_part* part, double c, int transmission,
                      double alpha, double alpha_x, int precision, void* stream, oras_precond** out) {
  if (!band || !part || !out || part->p.band != &band->b) {
    cpm::set_error("oras_setup: NULL argument or partition built from another band");
    return CPM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const bool simt_lu = (precision & CPM_SETUP_SIMT_LU) != 0;
  precision &= ~CPM_SETUP_SIMT_LU;
  if (!(c > 0.0) || (precision != CPM_FP64 && precision != CPM_FP32 && precision != CPM_BF16) ||
      (transmission != CPM_RAS && transmission != CPM_ORAS && transmission != CPM_ORAS_R3) ||
      (transmission != CPM_RAS && !(alpha >= 0.0 && alpha_x >= 0.0))) {
    cpm::set_error("oras_setup: need c > 0, a known precision / transmission, alpha >= 0");
    return CPM_ERR_INVALID_ARG;
  }
  oras_precond* pc = nullptr;
  try {
    pc = new oras_precond();
    cpm_status st = setup_impl(pc, band->b, part->p, c, transmission, alpha, alpha_x, precision,
                               simt_lu, (cudaStream_t)stream);
    if (st != CPM_OK) {
      delete pc;
      return st;
    }
  } catch (const std::bad_alloc&) {
    delete pc;
    cpm::set_error("oras_setup: out of host memory");
    return CPM_ERR_OOM;
  }
  *out = pc;
  return CPM_OK;
}

cpm_status oras_info_get(const oras_precond* pc, oras_info* o) {
  if (!pc || !o) {
    cpm::set_error("oras_info_get: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  o->n_sub = pc->n_sub;
  o->n_active = pc->n_active;
  o->n_nodes = pc->n_nodes;
  o->precision = pc->precision;
  o->transmission = pc->transmission;
  o->max_n = pc->n_local.empty() ? 0 : *std::max_element(pc->n_local.begin(), pc->n_local.end());
  o->sum_n = pc->sum_n;
  o->sum_n2 = pc->sum_n2;
  o->sum_sigma = pc->sum_sigma;
  o->factor_bytes = (int64_t)pc->factor_bytes;
  o->device_bytes = (int64_t)pc->device_bytes;
  o->setup_ms_assemble = pc->ms_assemble;
  o->setup_ms_factor = pc->ms_factor;
  o->kernel_launches = pc->launches;
  o->solve_ctas_per_sm = pc->solve_ctas;
  o->solve_kseg = pc->trsv.kseg;
  o->solve_prefetch = pc->trsv.prefetch;
  o->solve_stagger = pc->trsv.stagger;
  o->peak_device_bytes = (int64_t)pc->peak_bytes;
  o->tile_rows = pc->rows_total / TILE;
  o->solve_offdiag_tiles = pc->solve_offdiag_tiles;
  return CPM_OK;
}

cpm_status oras_setup_selftest_singular(const cpm_band* band, const cpm_part* part, double c, int transmission,
                                        double alpha, double alpha_x, int precision, int subdomain, void* stream) {
  if (!band || !part || part->p.band != &band->b || subdomain < 0 || subdomain >= part->p.n_sub || !(c > 0.0) ||
      (precision != CPM_FP64 && precision != CPM_FP32 && precision != CPM_BF16) ||
      (transmission != CPM_RAS && transmission != CPM_ORAS && transmission != CPM_ORAS_R3) ||
      (transmission != CPM_RAS && !(alpha >= 0.0 && alpha_x >= 0.0))) {
    cpm::set_error("oras_setup_selftest_singular: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  oras_precond* pc = nullptr;
  try {
    pc = new oras_precond();
    cpm_status st = setup_impl(pc, band->b, part->p, c, transmission, alpha, alpha_x, precision, false,
                               (cudaStream_t)stream, subdomain);
    delete pc;
    return st;
  } catch (const std::bad_alloc&) {
    delete pc;
    cpm::set_error("oras_setup_selftest_singular: out of host memory");
    return CPM_ERR_OOM;
  }
}

cpm_status oras_plan(const cpm_band* band, const cpm_part* part, int transmission, int precision,
                     int restart, int nrhs, oras_plan_info* out) {
  if (!band || !part || !out || restart < 1 || nrhs < 1 ||
      (precision != CPM_FP64 && precision != CPM_FP32 && precision != CPM_BF16) ||
      (transmission != CPM_RAS && transmission != CPM_ORAS && transmission != CPM_ORAS_R3)) {
    cpm::set_error("oras_plan: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  const cpm::Band& B = band->b;
  const cpm::Partition& P = part->p;
  if (P.band != &B) {
    cpm::set_error("oras_plan: partition of another band");
    return CPM_ERR_INVALID_ARG;
  }
  const int ns = P.n_sub;
  const int64_t N = B.n_active, NN = B.n_nodes();
  const int64_t P3 = (int64_t)B.P() * B.P() * B.P();
  const int64_t wb = precision == CPM_FP64 ? 8 : 4;
  int64_t tile_elems = 0, rows = 0, sum_n = 0, sum_n2 = 0, nnz_bound = 0;
  int t_max = 0;
  std::vector<int> Ts(ns);
  for (int j = 0; j < ns; ++j) {
    const cpm::SubSets& S = P.subs[j];
    const int64_t n = (int64_t)S.sigma.size() + (transmission != CPM_RAS ? (int64_t)S.bc_a.size() : 0);
    const int T = (int)((n + TILE - 1) / TILE);
    Ts[j] = T;
    t_max = std::max(t_max, T);
    tile_elems += (int64_t)T * T * TILE_ELEMS;
    rows += (int64_t)T * TILE;
    sum_n += n;
    sum_n2 += n * n;
    nnz_bound += n * (1 + 6 * P3);
  }
  // every allocation may be rounded up to a 2 MiB page
  const int64_t page = 2 << 20;
  auto rnd = [&](int64_t b) { return ((b + page - 1) / page) * page; };
  const int64_t band_dev = rnd(4 * NN * B.P() * B.P()) + rnd(8 * NN * 3 * B.P()) + rnd(4 * N * 6) +
                         rnd(8 * NN * (B.P() * B.P() + B.P())) /* tensor weights */;
  const int64_t work = rnd(wb * tile_elems);
  const int64_t inv = rnd(2 * wb * rows * TILE);
  const int64_t small = rnd(sizeof(SubMeta) * ns) + 2 * rnd(4 * rows) + rnd(4) + rnd(16);
  const int64_t assembly = rnd(4 * rows) /* pivots */ + rnd(wb * rows) /* dinv */ + 2 * rnd(4 * sum_n) +
                           rnd(8 * ns) + rnd(8 * nnz_bound) + rnd(8 * nnz_bound);
  const int64_t factor = precision == CPM_BF16 ? 2 * tile_elems : wb * tile_elems;
  // batched-solve schedule: the autotuner's smallest split (8 tiles) needs the most slots
  std::vector<int2> items;
  int maxseg = 1;
  trsv_build_items(Ts.data(), ns, 8, 0, items, &maxseg);
  const int words = precision == CPM_FP64 ? 2 : 1;
  const int64_t nrc = nrhs > 1 ? TRSV_MAX_NR : 1;       // tagged words per row and rhs slot
  const int64_t sched = rnd(8 * (int64_t)items.size()) + rnd(8 * words * (rows / TILE) * maxseg * TILE * nrc) +
                        rnd(8 * words * rows * nrc) + rnd(16);
  // FGMRES workspace of the lock-step batch (1 right-hand side, or TRSV_MAX_NR for batches)
  const int64_t cap = nrhs > 1 ? TRSV_MAX_NR : 1;
  const int64_t ld = (N + 31) / 32 * 32;
  const int64_t nblk = std::max<int64_t>(152, (N + 16383) / 16384);
  const int64_t gmres = 2 * rnd(8 * cap * (restart + 1) * ld) + 2 * rnd(8 * cap * ld) +
                        rnd(8 * cap * nblk * (2 * (restart + 1) + 1)) +
                        rnd(8 * cap * ((int64_t)(restart + 2) * (restart + 8) + 64)) + rnd(4 * cap * 16) + rnd(16) +
                        rnd(8 * cap * NN) /* extension values */ + rnd(8 * nrhs * NN) /* apply scratch */;
  const int64_t ubuf = precision == CPM_FP64 ? 0 : rnd((int64_t)lu_tc_ubuf_bytes(rows / TILE, precision == CPM_BF16));
  const int64_t envelope = 2 * rnd(4 * rows) + rnd(4 * (int64_t)ns * t_max) + rnd(4 * ns);
  const int64_t setup_peak = band_dev + work + inv + small + assembly + ubuf + envelope +
                             (precision == CPM_BF16 ? rnd(2 * tile_elems) : 0);
  const int64_t resident = band_dev + rnd(factor) + inv + small + sched + gmres + 2 * rnd(4 * (rows / TILE));
  out->setup_peak_bytes = setup_peak + (setup_peak >> 6);
  out->resident_bytes = resident + (resident >> 6);
  out->factor_bytes = factor;
  out->vector_bytes = 2 * 8 * (int64_t)nrhs * N;
  out->sum_n2 = sum_n2;
  out->max_tiles = t_max;
  return CPM_OK;
}

cpm_status oras_local_sizes(const oras_precond* pc, int64_t* n_out) {
  if (!pc || !n_out) {
    cpm::set_error("oras_local_sizes: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  for (int j = 0; j < pc->n_sub; ++j) n_out[j] = pc->n_local[j];
  return CPM_OK;
}

cpm_status cpm_op_apply(const oras_precond* cpc, const double* x_dev, double* y_dev, int nrhs,
                        void* stream) {
  oras_precond* pc = const_cast<oras_precond*>(cpc);
  if (!pc || !x_dev || !y_dev || nrhs < 1) {
    cpm::set_error("cpm_op_apply: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  cpm_status st = ensure_v_scratch(pc, nrhs);
  if (st != CPM_OK) return st;
  pc->launches += KERNELS_APPLY;
  CK(launch_apply(pc->op, direct(const_cast<double*>(x_dev), pc->n_active), pc->v_scratch, nullptr,
                  direct(y_dev, pc->n_active), nrhs, 0, nullptr, (cudaStream_t)stream));
  return CPM_OK;
}

cpm_status oras_apply(const oras_precond* pc, const double* r_dev, double* z_dev, int nrhs,
                      void* stream) {
  if (!pc || !r_dev || !z_dev || nrhs < 1) {
    cpm::set_error("oras_apply: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  oras_precond* mpc = const_cast<oras_precond*>(pc);
  if (nrhs > 1) {
    cpm_status st = ensure_multi_rhs(mpc);
    if (st != CPM_OK) return st;
  }
  const int64_t n = pc->n_active;
  for (int i = 0; i < nrhs;) {
    const int nr = nr_chunk(nrhs - i);
    CK(launch_trsv(pc->trsv, direct(const_cast<double*>(r_dev) + (int64_t)i * n, n), direct(z_dev + (int64_t)i * n, n),
                   nullptr, (cudaStream_t)stream, nr));
    mpc->launches += KERNELS_TRSV;
    i += nr;
  }
  return CPM_OK;
}

cpm_status oras_tune(oras_precond* pc, int knob, int value) {
  if (!pc) {
    cpm::set_error("oras_tune: NULL handle");
    return CPM_ERR_INVALID_ARG;
  }
  int ctas = pc->solve_ctas, kseg = pc->trsv.kseg, pf = pc->trsv.prefetch, sg = pc->trsv.stagger;
  const int max_ctas = trsv_ctas_per_sm(pc->precision);
  if (knob == CPM_TUNE_SOLVE_CTAS_PER_SM && value >= 1 && value <= max_ctas) ctas = value;
  else if (knob == CPM_TUNE_SOLVE_KSEG && value >= 1 && value <= 1023) kseg = value;
  else if (knob == CPM_TUNE_SOLVE_PREFETCH && (value == 0 || value == 1)) pf = value;
  else if (knob == CPM_TUNE_SOLVE_STAGGER && (value == 0 || value == 1)) sg = value;
  else {
    cpm::set_error("oras_tune: unknown knob or value out of range (CTAs per SM 1.." +
                   std::to_string(max_ctas) + ", kseg 1..1023, prefetch 0/1, stagger 0/1)");
    return CPM_ERR_INVALID_ARG;
  }
  return set_schedule(pc, ctas, kseg, pf, sg);
}

cpm_status oras_autotune(oras_precond* pc, void* stream) {
  if (!pc) {
    cpm::set_error("oras_autotune: NULL handle");
    return CPM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *r = nullptr, *z = nullptr;
  CK(cudaMalloc(&r, 8 * pc->n_active));
  CK(cudaMalloc(&z, 8 * pc->n_active));
  CK(cudaMemsetAsync(r, 0, 8 * pc->n_active, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int max_ctas = trsv_ctas_per_sm(pc->precision);
  const int ksegs[] = {8, 16, 32, 1023};
  float best = 1e30f;
  int bc = max_ctas, bk = 1023, bp = 0, bs = 0;
  cpm_status st = CPM_OK;
  for (int c = 1; c <= max_ctas && st == CPM_OK; ++c)
    for (int k : ksegs)
      for (int cand = 0; cand < 4 && st == CPM_OK; ++cand) {
        const int pf = cand & 1, sg = cand >> 1;
        st = set_schedule(pc, c, k, pf, sg);
        if (st != CPM_OK) break;
        for (int w = 0; w < 2; ++w) launch_trsv(pc->trsv, direct(r, 0), direct(z, 0), nullptr, s);
        cudaEventRecord(e0, s);
        for (int w = 0; w < 3; ++w) launch_trsv(pc->trsv, direct(r, 0), direct(z, 0), nullptr, s);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(e, "oras_autotune"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bc = c; bk = k; bp = pf; bs = sg; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(r);
  cudaFree(z);
  if (st != CPM_OK) return st;
  st = set_schedule(pc, bc, bk, bp, bs);
  if (st != CPM_OK) return st;
  return oras_check_status(pc, stream);
}

cpm_status oras_check_status(const oras_precond* pc, void* stream) {
  if (!pc) {
    cpm::set_error("oras_check_status: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  CK(cudaMemcpy(&h, pc->status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemsetAsync(pc->status, 0, sizeof(int), (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (h & ST_TIMEOUT) {
    cpm::set_error("a bounded device-side wait gave up:" + timeout_where(h));
    return CPM_ERR_TIMEOUT;
  }
  return CPM_OK;
}

cpm_status cpm_gmres_solve(const oras_precond* cpc, const double* f_dev, double* u_dev, int nrhs,
                           const cpm_gmres_opts* opts, cpm_gmres_result* results, void* stream) {
  oras_precond* pc = const_cast<oras_precond*>(cpc);
  if (!pc || !f_dev || !u_dev || nrhs < 1 || !results) {
    cpm::set_error("cpm_gmres_solve: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  cpm_gmres_opts o{50, 1e-8, 1000, 1, 1};
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 128 || !(o.tol > 0.0) || o.max_it < 1) {
    cpm::set_error("cpm_gmres_solve: need 1 <= restart <= 128, tol > 0, max_it >= 1");
    return CPM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = pc->n_active;
  const int widest = nr_chunk(nrhs);
  cpm_status st = ensure_gmres(pc, o.restart, widest);
  if (st != CPM_OK) return st;
  if (widest > 1) {
    st = ensure_multi_rhs(pc);
    if (st != CPM_OK) return st;
  }
  cpm_status first = CPM_OK;
  for (int i = 0; i < nrhs;) {
    const int nr = nr_chunk(nrhs - i);
    if (o.use_graph && !pc->iter_graph[width_index(nr)]) {
      st = capture_graph(pc, nr);
      if (st != CPM_OK) return st;
    }
    st = solve_batch(pc, f_dev + (int64_t)i * n, u_dev + (int64_t)i * n, nr, o, o.use_graph != 0, &results[i], s);
    if (st != CPM_OK) return st;
    for (int q = 0; q < nr; ++q)
      if (first == CPM_OK && results[i + q].status != CPM_OK) first = (cpm_status)results[i + q].status;
    i += nr;
  }
  if (first != CPM_OK) cpm::set_error(std::string("cpm_gmres_solve: ") + cpm_status_string(first));
  return first;
}

cpm_status oras_stationary_solve(const oras_precond* cpc, const double* f_dev, double* u_dev, int nrhs,
                                 double tol, int max_it, cpm_gmres_result* results, void* stream) {
  oras_precond* pc = const_cast<oras_precond*>(cpc);
  if (!pc || !f_dev || !u_dev || nrhs < 1 || !results || !(tol > 0.0) || max_it < 1) {
    cpm::set_error("oras_stationary_solve: bad argument (need tol > 0, max_it >= 1)");
    return CPM_ERR_INVALID_ARG;
  }
  cpm_status st = ensure_stationary(pc);
  if (st != CPM_OK) return st;
  if (nrhs > 1) {
    st = ensure_multi_rhs(pc);
    if (st != CPM_OK) return st;
  }
  cpm_status first = CPM_OK;
  const int64_t n = pc->n_active;
  for (int i = 0; i < nrhs;) {
    const int nr = nr_chunk(nrhs - i);
    st = stationary_batch(pc, f_dev + (int64_t)i * n, u_dev + (int64_t)i * n, nr, tol, max_it, &results[i],
                          (cudaStream_t)stream);
    if (st != CPM_OK) return st;
    for (int q = 0; q < nr; ++q)
      if (first == CPM_OK && results[i + q].status != CPM_OK) first = (cpm_status)results[i + q].status;
    i += nr;
  }
  if (first != CPM_OK) cpm::set_error(std::string("oras_stationary_solve: ") + cpm_status_string(first));
  return first;
}

cpm_status cpm_vec_axpby(int64_t n, double a, const double* x_dev, double b, double* y_dev, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !y_dev))) {
    cpm::set_error("cpm_vec_axpby: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  if (n == 0) return CPM_OK;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * (int64_t)sm_count(dev)));
  CK(launch_axpby(n, a, x_dev, b, y_dev, nblk, (cudaStream_t)stream));
  return CPM_OK;
}

cpm_status cpm_selftest_bounded_wait(oras_precond* pc, double limit_s, void* stream) {
  if (!pc || !(limit_s > 0.0) || limit_s > 10.0) {
    cpm::set_error("cpm_selftest_bounded_wait: need a handle and 0 < limit_s <= 10");
    return CPM_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* never = nullptr;
  int* out = nullptr;
  CK(cudaMalloc(&never, 16));
  cudaError_t e = cudaMalloc(&out, 16);
  if (e != cudaSuccess) {
    cudaFree(never);
    return cuda_fail(e, "cudaMalloc");
  }
  int h[2] = {1, 1};
  e = cudaMemsetAsync(never, 0, 16, s);
  if (e == cudaSuccess) e = launch_bounded_wait_selftest((uint64_t)(limit_s * 1e9), never, pc->status, out, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(never);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "cpm_selftest_bounded_wait");
  if (h[0] == 0 && h[1] == 0) {
    cpm::set_error("cpm_selftest_bounded_wait: both bounded waits expired (expected)");
    return CPM_ERR_TIMEOUT;
  }
  return CPM_OK;
}

cpm_status cpm_selftest_zero_operator(oras_precond* pc) {
  if (!pc) {
    cpm::set_error("cpm_selftest_zero_operator: null handle");
    return CPM_ERR_INVALID_ARG;
  }
  CK(cudaDeviceSynchronize());
  // A x = diag x - invh2 (neighbour sum of E x): both coefficients zero give A x = 0 exactly
  // for finite x; the captured iteration graphs hold the old coefficients and are dropped
  pc->op.diag = 0.0;
  pc->op.invh2 = 0.0;
  pc->drop_graphs();
  return CPM_OK;
}

cpm_status cpm_probe_fp64(int blocks, int threads, int chains, int iters, double* tflop_s, double* cycles_per_fma) {
  if (blocks < 1 || threads < 1 || threads > 1024 || iters < 1 ||
      (chains != 1 && chains != 2 && chains != 4 && chains != 8)) {
    cpm::set_error("cpm_probe_fp64: need blocks, iters >= 1, 1 <= threads <= 1024, chains in {1, 2, 4, 8}");
    return CPM_ERR_INVALID_ARG;
  }
  double* buf = nullptr;
  CK(cudaMalloc(&buf, 65536));
  long long* cyc = (long long*)(buf + 4096);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int nb = std::min(blocks, 4096);
  if (e == cudaSuccess && tflop_s) {
    e = launch_fma_throughput(nb, threads, chains, iters, buf, 0);          // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch_fma_throughput(nb, threads, chains, iters, buf, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) *tflop_s = 2.0 * nb * (double)threads * chains * iters / (ms * 1e-3) / 1e12;
  }
  if (e == cudaSuccess && cycles_per_fma) {
    e = launch_fma_latency(iters, buf, cyc, 0);
    long long c = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) *cycles_per_fma = (double)c / iters;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "cpm_probe_fp64");
  return CPM_OK;
}

void oras_destroy(oras_precond* pc) { delete pc; }

}  // extern "C"
