// C ABI: host-only entry points (band, partition, local operators, status strings).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "host/cpm_internal.h"


namespace cpm {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace cpm

extern "C" {

const char* cpm_last_error(void) { return cpm::g_err.c_str(); }

const char* cpm_status_string(cpm_status s) {
  switch (s) {
    case CPM_OK: return "CPM_OK";
    case CPM_ERR_INVALID_ARG: return "CPM_ERR_INVALID_ARG";
    case CPM_ERR_OOM: return "CPM_ERR_OOM";
    case CPM_ERR_CUDA: return "CPM_ERR_CUDA";
    case CPM_ERR_SINGULAR: return "CPM_ERR_SINGULAR";
    case CPM_ERR_NOT_CONVERGED: return "CPM_ERR_NOT_CONVERGED";
    case CPM_ERR_BREAKDOWN: return "CPM_ERR_BREAKDOWN";
    case CPM_ERR_NAN: return "CPM_ERR_NAN";
    case CPM_ERR_TIMEOUT: return "CPM_ERR_TIMEOUT";
    case CPM_ERR_BUDGET: return "CPM_ERR_BUDGET";
    case CPM_ERR_STENCIL: return "CPM_ERR_STENCIL";
  }
  return "CPM_ERR_UNKNOWN";
}

// Surface of the C ABI -> internal surface (mesh arrays copied).
static cpm_status read_surface(const cpm_surface* surface, cpm::Surface& s) {
  s = cpm::Surface{surface->kind, surface->R, surface->r, {}};
  if (s.kind == CPM_TRIMESH) {
    if (!surface->verts || !surface->tris || surface->n_verts < 3 || surface->n_tris < 1) {
      cpm::set_error("cpm_build_band: a triangulated surface needs vertices and triangles");
      return CPM_ERR_INVALID_ARG;
    }
    s.mesh.V.assign(surface->verts, surface->verts + 3 * surface->n_verts);
    s.mesh.T.assign(surface->tris, surface->tris + 3 * surface->n_tris);
    for (int32_t v : s.mesh.T)
      if (v < 0 || v >= surface->n_verts) {
        cpm::set_error("cpm_build_band: triangle vertex index out of range");
        return CPM_ERR_INVALID_ARG;
      }
  }
  return CPM_OK;
}

static cpm_status build_band_common(const cpm_surface* surface, double h, int p, double lambda_over_h,
                                    bool algorithmic, cpm_band** out, bool device = false,
                                    void* stream = nullptr) {
  if (!surface || !out) {
    cpm::set_error("cpm_build_band: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    cpm::Surface s;
    cpm_status st = read_surface(surface, s);
    if (st != CPM_OK) return st;
    cpm_band* b = new cpm_band();
    st = algorithmic ? cpm::build_band_algorithmic(s, h, p, b->b)
                     : (device ? cpm::build_band_device(s, h, p, lambda_over_h, stream, b->b)
                               : cpm::build_band(s, h, p, lambda_over_h, b->b));
    if (st != CPM_OK) {
      delete b;
      return st;
    }
    *out = b;
    return CPM_OK;
  } catch (const std::bad_alloc&) {
    cpm::set_error("cpm_build_band: out of host memory");
    return CPM_ERR_OOM;
  }
}

cpm_status cpm_build_band(const cpm_surface* surface, double h, int p, double lambda_over_h,
                          cpm_band** out) {
  return build_band_common(surface, h, p, lambda_over_h, false, out);
}

cpm_status cpm_build_band_device(const cpm_surface* surface, double h, int p, double lambda_over_h,
                                 void* stream, cpm_band** out) {
  return build_band_common(surface, h, p, lambda_over_h, false, out, true, stream);
}

cpm_status cpm_build_band_algorithmic(const cpm_surface* surface, double h, int p, cpm_band** out) {
  return build_band_common(surface, h, p, 0.0, true, out);
}

cpm_status cpm_band_info_get(const cpm_band* band, cpm_band_info* out) {
  if (!band || !out) {
    cpm::set_error("cpm_band_info_get: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  const cpm::Band& B = band->b;
  out->n_active = B.n_active;
  out->n_ghost = B.n_ghost;
  out->p = B.p;
  out->h = B.h;
  out->lambda = B.lam;
  out->ijk = B.ijk.data();
  out->cp = B.cp.data();
  out->nbr = B.nbr.data();
  out->base = B.base.data();
  out->pencil = B.pencil.data();
  out->weights = B.wts.data();
  out->tri = B.tri.empty() ? nullptr : B.tri.data();
  return CPM_OK;
}

void cpm_band_destroy(cpm_band* band) {
  if (!band) return;
  cpm::band_release_device(band->b);
  delete band;
}

static cpm_status partition_impl(const cpm_band* band, int n_sub, const int64_t* leaf_weights, int n_overlap,
                                 int align_passes, cpm_part** out, int split, const char* name) {
  if (!band || !out) {
    cpm::set_error(std::string(name) + ": NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (align_passes < 0 || align_passes > 64) {
    cpm::set_error(std::string(name) + ": need 0 <= align_passes <= 64");
    return CPM_ERR_INVALID_ARG;
  }
  try {
    cpm_part* p = new cpm_part();
    cpm_status st = cpm::build_partition(band->b, n_sub, leaf_weights, n_overlap, align_passes, p->p, split);
    if (st != CPM_OK) {
      delete p;
      return st;
    }
    *out = p;
    return CPM_OK;
  } catch (const std::bad_alloc&) {
    cpm::set_error(std::string(name) + ": out of host memory");
    return CPM_ERR_OOM;
  }
}

cpm_status cpm_partition(const cpm_band* band, int n_sub, const int64_t* leaf_weights,
                         int n_overlap, int align_passes, cpm_part** out) {
  return partition_impl(band, n_sub, leaf_weights, n_overlap, align_passes, out, 0, "cpm_partition");
}

cpm_status cpm_partition_graph(const cpm_band* band, int n_sub, const int64_t* leaf_weights,
                               int n_overlap, int align_passes, cpm_part** out) {
  return partition_impl(band, n_sub, leaf_weights, n_overlap, align_passes, out, 1, "cpm_partition_graph");
}

cpm_status cpm_partition_from_labels(const cpm_band* band, int n_sub, const int32_t* labels,
                                     int n_overlap, cpm_part** out) {
  if (!band || !labels || !out) {
    cpm::set_error("cpm_partition_from_labels: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    cpm_part* p = new cpm_part();
    cpm_status st = cpm::build_partition_from_labels(band->b, n_sub, labels, n_overlap, p->p);
    if (st != CPM_OK) {
      delete p;
      return st;
    }
    *out = p;
    return CPM_OK;
  } catch (const std::bad_alloc&) {
    cpm::set_error("cpm_partition_from_labels: out of host memory");
    return CPM_ERR_OOM;
  }
}

namespace {

// partition file: header, then N_A int32 labels
struct PartFileHeader {
  char magic[8];              // "CPMPART1"
  uint32_t version;           // 2
  int32_t n_sub, n_overlap, p;
  int64_t n_active, n_nodes;
  double h;
  uint64_t band_hash;         // FNV-1a over the grid coordinates and closest points of every node
};

uint64_t fnv1a(uint64_t x, const void* data, size_t n) {
  const unsigned char* b = (const unsigned char*)data;
  for (size_t k = 0; k < n; ++k) {
    x ^= b[k];
    x *= 1099511628211ull;
  }
  return x;
}

// The sets of Sec. 4 depend on the grid nodes and on their closest points (the generators
// of CP_{S_j} and the cross marks), so both enter the fingerprint.
uint64_t band_hash(const cpm::Band& B) {
  uint64_t x = fnv1a(1469598103934665603ull, B.ijk.data(), B.ijk.size() * sizeof(B.ijk[0]));
  return fnv1a(x, B.cp.data(), B.cp.size() * sizeof(B.cp[0]));
}

PartFileHeader header_of(const cpm::Band& B, int n_sub, int n_overlap) {
  PartFileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "CPMPART1", 8);
  h.version = 2;
  h.n_sub = n_sub;
  h.n_overlap = n_overlap;
  h.p = B.p;
  h.n_active = B.n_active;
  h.n_nodes = B.n_nodes();
  h.h = B.h;
  h.band_hash = band_hash(B);
  return h;
}

}  // namespace

cpm_status cpm_partition_save(const cpm_part* part, const char* path) {
  if (!part || !path || !part->p.band) {
    cpm::set_error("cpm_partition_save: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  const cpm::Partition& P = part->p;
  const PartFileHeader h = header_of(*P.band, P.n_sub, P.n_overlap);
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    cpm::set_error(std::string("cpm_partition_save: cannot open ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
            std::fwrite(P.labels.data(), sizeof(int32_t), P.labels.size(), f) == P.labels.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    cpm::set_error(std::string("cpm_partition_save: write failed: ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  return CPM_OK;
}

cpm_status cpm_partition_load(const cpm_band* band, const char* path, cpm_part** out) {
  if (!band || !path || !out) {
    cpm::set_error("cpm_partition_load: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    cpm::set_error(std::string("cpm_partition_load: cannot open ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  PartFileHeader h;
  const bool got = std::fread(&h, sizeof(h), 1, f) == 1;
  if (!got || std::memcmp(h.magic, "CPMPART1", 8) != 0 || h.version != 2) {
    std::fclose(f);
    cpm::set_error(std::string("cpm_partition_load: not a partition file: ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  const PartFileHeader mine = header_of(band->b, h.n_sub, h.n_overlap);
  if (h.p != mine.p || h.n_active != mine.n_active || h.n_nodes != mine.n_nodes || h.h != mine.h ||
      h.band_hash != mine.band_hash) {
    std::fclose(f);
    cpm::set_error("cpm_partition_load: the file belongs to another band");
    return CPM_ERR_INVALID_ARG;
  }
  std::vector<int32_t> labels;
  try {
    labels.resize((size_t)h.n_active);
  } catch (const std::bad_alloc&) {
    std::fclose(f);
    cpm::set_error("cpm_partition_load: out of host memory");
    return CPM_ERR_OOM;
  }
  const bool full = std::fread(labels.data(), sizeof(int32_t), labels.size(), f) == labels.size();
  unsigned char extra = 0;
  const bool trailing = full && std::fread(&extra, 1, 1, f) == 1;
  std::fclose(f);
  if (!full) {
    cpm::set_error(std::string("cpm_partition_load: truncated file: ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  if (trailing) {
    cpm::set_error(std::string("cpm_partition_load: unexpected data after the labels: ") + path);
    return CPM_ERR_INVALID_ARG;
  }
  return cpm_partition_from_labels(band, h.n_sub, labels.data(), h.n_overlap, out);
}

cpm_status cpm_partition_labels(const cpm_part* part, const int32_t** labels) {
  if (!part || !labels) {
    cpm::set_error("cpm_partition_labels: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *labels = part->p.labels.data();
  return CPM_OK;
}

cpm_status cpm_partition_set(const cpm_part* part, int j, int which, const int32_t** data,
                             int64_t* len) {
  if (!part || !data || !len || j < 0 || j >= part->p.n_sub) {
    cpm::set_error("cpm_partition_set: bad argument");
    return CPM_ERR_INVALID_ARG;
  }
  const cpm::SubSets& S = part->p.subs[j];
  const std::vector<int32_t>* v = nullptr;
  switch (which) {
    case CPM_SET_OWN: v = &S.own; break;
    case CPM_SET_SIGMA: v = &S.sigma; break;
    case CPM_SET_LAST: v = &S.last; break;
    case CPM_SET_GHOST: v = &S.ghost; break;
    case CPM_SET_BC_A: v = &S.bc_a; break;
    case CPM_SET_BC_G: v = &S.bc_g; break;
    case CPM_SET_BC_GEN: v = &S.bc_gen; break;
    case CPM_SET_BC_NEARX: v = &S.bc_nearx; break;
    default:
      cpm::set_error("cpm_partition_set: unknown set selector");
      return CPM_ERR_INVALID_ARG;
  }
  *data = v->data();
  *len = (int64_t)v->size();
  return CPM_OK;
}

cpm_status cpm_partition_cross_points(const cpm_part* part, const int32_t** data,
                                      int64_t* len) {
  if (!part || !data || !len) {
    cpm::set_error("cpm_partition_cross_points: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  *data = part->p.cross.data();
  *len = (int64_t)part->p.cross.size();
  return CPM_OK;
}

void cpm_partition_destroy(cpm_part* part) { delete part; }

cpm_status cpm_local_coo(const cpm_band* band, const cpm_part* part, double c,
                         int transmission, double alpha, double alpha_x, int j, int64_t* n,
                         int64_t* nnz, int32_t* rows, int32_t* cols, double* vals) {
  if (!band || !part || !n || !nnz) {
    cpm::set_error("cpm_local_coo: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  try {
    cpm::LocalCOO L;
    cpm_status st = cpm::build_local_coo(band->b, part->p, c, transmission, alpha, alpha_x, j, L);
    if (st != CPM_OK) return st;
    *n = L.n;
    if (rows && cols && vals) {
      if (*nnz < (int64_t)L.val.size()) {
        cpm::set_error("cpm_local_coo: output arrays too small");
        return CPM_ERR_INVALID_ARG;
      }
      for (size_t t = 0; t < L.val.size(); ++t) {
        rows[t] = L.row[t];
        cols[t] = L.col[t];
        vals[t] = L.val[t];
      }
    }
    *nnz = (int64_t)L.val.size();
    return CPM_OK;
  } catch (const std::bad_alloc&) {
    cpm::set_error("cpm_local_coo: out of host memory");
    return CPM_ERR_OOM;
  }
}

cpm_status cpm_local_order(const cpm_band* band, const cpm_part* part, double c, int transmission,
                           double alpha, double alpha_x, int j, int64_t* n, int* T, int32_t* perm,
                           int32_t* first, int32_t* last, int32_t* pend) {
  if (!band || !part || !n || !T) {
    cpm::set_error("cpm_local_order: NULL argument");
    return CPM_ERR_INVALID_ARG;
  }
  try {
    cpm::LocalCOO L;
    cpm_status st = cpm::build_local_coo(band->b, part->p, c, transmission, alpha, alpha_x, j, L);
    if (st != CPM_OK) return st;
    *n = L.n;
    *T = (int)((L.n + 63) / 64);
    if (!perm) return CPM_OK;
    if (!first || !last || !pend) {
      cpm::set_error("cpm_local_order: NULL output array");
      return CPM_ERR_INVALID_ARG;
    }
    std::vector<int32_t> p, inv(L.n), f, l, pe;
    cpm::rcm_order(L, p);
    for (int64_t k = 0; k < L.n; ++k) inv[p[k]] = (int32_t)k;
    for (auto& r : L.row) r = inv[r];
    for (auto& cc : L.col) cc = inv[cc];
    cpm::envelope(L, *T, f, l, pe);
    std::copy(p.begin(), p.end(), perm);
    std::copy(f.begin(), f.end(), first);
    std::copy(l.begin(), l.end(), last);
    std::copy(pe.begin(), pe.end(), pend);
    return CPM_OK;
  } catch (const std::bad_alloc&) {
    cpm::set_error("cpm_local_order: out of host memory");
    return CPM_ERR_OOM;
  }
}

}  // extern "C"
