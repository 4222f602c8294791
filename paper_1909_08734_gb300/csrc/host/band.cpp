// Band construction: closest points, tube-radius active set, ghost set, canonical order,
// neighbour table and interpolation stencils (Sec. 2.1).
#include <algorithm>
#include <array>
#include <cmath>
#include <limits>
#include <new>

#include "cpm_internal.h"

namespace cpm {

bool closest_point(const Surface& s, const double x[3], double y[3]) {
  if (s.kind == CPM_SPHERE) {
    // CP(x) = R x / |x|
    double r = std::sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    if (r == 0.0) return false;
    for (int a = 0; a < 3; ++a) y[a] = (x[a] / r) * s.R;
    return true;
  }
  // torus about z: ring point C = R (x, y, 0)/rho, CP = C + r (x - C)/|x - C|
  double rho = std::sqrt(x[0] * x[0] + x[1] * x[1]);
  if (rho == 0.0) return false;
  double C[3] = {(x[0] / rho) * s.R, (x[1] / rho) * s.R, 0.0};
  double v[3] = {x[0] - C[0], x[1] - C[1], x[2] - C[2]};
  double sn = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  if (sn == 0.0) return false;
  for (int a = 0; a < 3; ++a) y[a] = C[a] + (v[a] / sn) * s.r;
  return true;
}

void surface_normal(const Surface& s, const double y[3], double n[3]) {
  if (s.kind == CPM_SPHERE) {
    double r = std::sqrt((y[0] * y[0] + y[1] * y[1]) + y[2] * y[2]);
    for (int a = 0; a < 3; ++a) n[a] = y[a] / r;
    return;
  }
  double rho = std::sqrt(y[0] * y[0] + y[1] * y[1]);
  double C[3] = {(y[0] / rho) * s.R, (y[1] / rho) * s.R, 0.0};
  double v[3] = {y[0] - C[0], y[1] - C[1], y[2] - C[2]};
  double sn = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  for (int a = 0; a < 3; ++a) n[a] = v[a] / sn;
}

// ---- triangulated surfaces -------------------------------------------------------------
static inline double dot3(const double* u, const double* v) { return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2]; }

// Closest point of triangle (a, b, c) to p by Voronoi-region tests (Ericson, Real-Time
// Collision Detection, Sec. 5.1.5): vertex a, vertex b, edge ab, vertex c, edge ac, edge bc,
// face, the first region whose dot-product test holds.
static void closest_on_triangle(const double* p, const double* a, const double* b, const double* c,
                                double* y) {
  double ab[3], ac[3], ap[3], bp[3], cp[3];
  for (int e = 0; e < 3; ++e) {
    ab[e] = b[e] - a[e];
    ac[e] = c[e] - a[e];
    ap[e] = p[e] - a[e];
    bp[e] = p[e] - b[e];
    cp[e] = p[e] - c[e];
  }
  const double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
  const double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
  const double vc = d1 * d4 - d3 * d2;
  const double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
  const double vb = d5 * d2 - d1 * d6;
  const double va = d3 * d6 - d5 * d4;
  if (d1 <= 0.0 && d2 <= 0.0) {
    for (int e = 0; e < 3; ++e) y[e] = a[e];
  } else if (d3 >= 0.0 && d4 <= d3) {
    for (int e = 0; e < 3; ++e) y[e] = b[e];
  } else if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double t = d1 / (d1 - d3);
    for (int e = 0; e < 3; ++e) y[e] = a[e] + ab[e] * t;
  } else if (d6 >= 0.0 && d5 <= d6) {
    for (int e = 0; e < 3; ++e) y[e] = c[e];
  } else if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double t = d2 / (d2 - d6);
    for (int e = 0; e < 3; ++e) y[e] = a[e] + ac[e] * t;
  } else if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
    const double q = d4 - d3;
    const double t = q / (q + (d5 - d6));
    for (int e = 0; e < 3; ++e) y[e] = b[e] + (c[e] - b[e]) * t;
  } else {
    const double den = (va + vb) + vc;
    const double v = vb / den, w = vc / den;
    for (int e = 0; e < 3; ++e) y[e] = (a[e] + ab[e] * v) + ac[e] * w;
  }
}

cpm_status mesh_prepare(Mesh& m, double cell) {
  const int64_t nt = m.n_tris(), nv = (int64_t)m.V.size() / 3;
  if (nt < 1 || nv < 3 || !(cell > 0.0)) {
    set_error("mesh: empty mesh");
    return CPM_ERR_INVALID_ARG;
  }
  m.fn.resize(3 * nt);
  double lo[3] = {m.V[0], m.V[1], m.V[2]}, hi[3] = {m.V[0], m.V[1], m.V[2]};
  for (int64_t v = 0; v < nv; ++v)
    for (int e = 0; e < 3; ++e) {
      lo[e] = std::min(lo[e], m.V[3 * v + e]);
      hi[e] = std::max(hi[e], m.V[3 * v + e]);
    }
  for (int64_t t = 0; t < nt; ++t) {
    const double* a = &m.V[3 * (int64_t)m.T[3 * t]];
    const double* b = &m.V[3 * (int64_t)m.T[3 * t + 1]];
    const double* c = &m.V[3 * (int64_t)m.T[3 * t + 2]];
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]};
    double len = std::sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
    if (!(len > 0.0)) {
      set_error("mesh: degenerate triangle " + std::to_string(t));
      return CPM_ERR_INVALID_ARG;
    }
    for (int e = 0; e < 3; ++e) m.fn[3 * t + e] = n[e] / len;
  }
  // bucket grid: a margin of cells around the bounding box
  m.cell = cell;
  for (int e = 0; e < 3; ++e) {
    m.org[e] = lo[e] - 2.0 * cell;
    m.nc[e] = (int32_t)std::floor((hi[e] - m.org[e]) / cell) + 3;
  }
  const int64_t ncell = (int64_t)m.nc[0] * m.nc[1] * m.nc[2];
  if (ncell > (int64_t)400000000) {
    set_error("mesh: bucket grid too large for this grid spacing");
    return CPM_ERR_INVALID_ARG;
  }
  auto range = [&](int64_t t, int32_t c0[3], int32_t c1[3]) {
    for (int e = 0; e < 3; ++e) {
      double mn = m.V[3 * (int64_t)m.T[3 * t] + e], mx = mn;
      for (int q = 1; q < 3; ++q) {
        mn = std::min(mn, m.V[3 * (int64_t)m.T[3 * t + q] + e]);
        mx = std::max(mx, m.V[3 * (int64_t)m.T[3 * t + q] + e]);
      }
      c0[e] = std::max(0, std::min(m.nc[e] - 1, (int32_t)std::floor((mn - m.org[e]) / cell)));
      c1[e] = std::max(0, std::min(m.nc[e] - 1, (int32_t)std::floor((mx - m.org[e]) / cell)));
    }
  };
  m.cell_start.assign(ncell + 1, 0);
  for (int64_t t = 0; t < nt; ++t) {
    int32_t c0[3], c1[3];
    range(t, c0, c1);
    for (int32_t i = c0[0]; i <= c1[0]; ++i)
      for (int32_t j = c0[1]; j <= c1[1]; ++j)
        for (int32_t k = c0[2]; k <= c1[2]; ++k) m.cell_start[((int64_t)i * m.nc[1] + j) * m.nc[2] + k + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) m.cell_start[c + 1] += m.cell_start[c];
  m.cell_tris.resize(m.cell_start[ncell]);
  std::vector<int64_t> fill(m.cell_start.begin(), m.cell_start.end() - 1);
  for (int64_t t = 0; t < nt; ++t) {            // ascending triangle index inside each cell
    int32_t c0[3], c1[3];
    range(t, c0, c1);
    for (int32_t i = c0[0]; i <= c1[0]; ++i)
      for (int32_t j = c0[1]; j <= c1[1]; ++j)
        for (int32_t k = c0[2]; k <= c1[2]; ++k)
          m.cell_tris[fill[((int64_t)i * m.nc[1] + j) * m.nc[2] + k]++] = (int32_t)t;
  }
  return CPM_OK;
}

// Ring search over the bucket grid: rings of cells at Chebyshev distance K = 0, 1, ... from
// the cell of x.  A triangle not met in rings < K lies outside the box of those rings, at
// distance >= lb(K) from x (the distance from x to that box's faces); the search stops once
// lb(K) exceeds both the best distance found and dmax, so every triangle at the minimum
// distance has been compared (ties: lowest index).
int32_t mesh_closest_point(const Mesh& m, const double x[3], double dmax, double y[3],
                           std::vector<int32_t>& stamp, int32_t& qid) {
  if (++qid == std::numeric_limits<int32_t>::max()) {
    std::fill(stamp.begin(), stamp.end(), -1);
    qid = 0;
  }
  int64_t c0[3];
  for (int e = 0; e < 3; ++e) c0[e] = (int64_t)std::floor((x[e] - m.org[e]) / m.cell);
  double best = std::numeric_limits<double>::infinity();
  int32_t bt = -1;
  double ty[3];
  for (int64_t K = 0;; ++K) {
    if (K > 0) {
      double lb = std::numeric_limits<double>::infinity();
      bool covers = true;
      for (int e = 0; e < 3; ++e) {
        const double f0 = m.org[e] + (double)(c0[e] - (K - 1)) * m.cell;
        const double f1 = m.org[e] + (double)(c0[e] + K) * m.cell;
        lb = std::min(lb, std::min(x[e] - f0, f1 - x[e]));
        covers = covers && c0[e] - (K - 1) <= 0 && c0[e] + (K - 1) >= m.nc[e] - 1;
      }
      const double lim = std::min(std::sqrt(best), dmax);
      if (covers || lb > lim * (1.0 + 1e-9) + 1e-12) break;
    }
    const int64_t i0 = std::max<int64_t>(0, c0[0] - K), i1 = std::min<int64_t>(m.nc[0] - 1, c0[0] + K);
    const int64_t j0 = std::max<int64_t>(0, c0[1] - K), j1 = std::min<int64_t>(m.nc[1] - 1, c0[1] + K);
    for (int64_t i = i0; i <= i1; ++i)
      for (int64_t j = j0; j <= j1; ++j) {
        const bool shell = std::llabs(i - c0[0]) == K || std::llabs(j - c0[1]) == K;
        for (int64_t kk = 0; kk < (shell ? 2 * K + 1 : 2); ++kk) {
          const int64_t k = shell ? c0[2] - K + kk : (kk == 0 ? c0[2] - K : c0[2] + K);
          if (k < 0 || k >= m.nc[2] || (!shell && K == 0 && kk == 1)) continue;
          const int64_t c = (i * m.nc[1] + j) * m.nc[2] + k;
          for (int64_t q = m.cell_start[c]; q < m.cell_start[c + 1]; ++q) {
            const int32_t t = m.cell_tris[q];
            if (stamp[t] == qid) continue;
            stamp[t] = qid;
            closest_on_triangle(x, &m.V[3 * (int64_t)m.T[3 * (int64_t)t]], &m.V[3 * (int64_t)m.T[3 * (int64_t)t + 1]],
                                &m.V[3 * (int64_t)m.T[3 * (int64_t)t + 2]], ty);
            const double d[3] = {x[0] - ty[0], x[1] - ty[1], x[2] - ty[2]};
            const double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (d2 < best || (d2 == best && t < bt)) {
              best = d2;
              bt = t;
              y[0] = ty[0];
              y[1] = ty[1];
              y[2] = ty[2];
            }
          }
        }
      }
  }
  if (bt < 0 || std::sqrt(best) > dmax * (1.0 + 1e-9) + 1e-12) return -1;
  return bt;
}

void node_normal(const Band& B, int64_t g, double n[3]) {
  if (B.surf.kind == CPM_TRIMESH) {
    const double* f = &B.surf.mesh.fn[3 * (int64_t)B.tri[g]];
    n[0] = f[0];
    n[1] = f[1];
    n[2] = f[2];
    return;
  }
  surface_normal(B.surf, &B.cp[3 * g], n);
}

void bary_weights(double t, int p, double* w) {
  // beta_m = (-1)^m C(p, m); l_m(t) = (beta_m/(t-m)) / sum_n beta_n/(t-n); delta at nodes
  double q[8];
  double binom = 1.0;
  int exact = -1;
  for (int m = 0; m <= p; ++m) {
    double beta = (m % 2 == 0) ? binom : -binom;
    double diff = t - (double)m;
    if (diff == 0.0) exact = m;
    q[m] = beta / diff;
    binom = binom * (double)(p - m) / (double)(m + 1);
  }
  if (exact >= 0) {
    for (int m = 0; m <= p; ++m) w[m] = (m == exact) ? 1.0 : 0.0;
    return;
  }
  double s = q[0];
  for (int m = 1; m <= p; ++m) s = s + q[m];
  for (int m = 0; m <= p; ++m) w[m] = q[m] / s;
}

void point_weights(const double y[3], double h, int p, int32_t base[3], double* wx, double* wy,
                   double* wz) {
  double* W[3] = {wx, wy, wz};
  for (int a = 0; a < 3; ++a) {
    double s = y[a] / h;
    double b = std::floor(s - (double)(p - 1) / 2.0);
    double t = s - b;
    base[a] = (int32_t)b;
    bary_weights(t, p, W[a]);
  }
}

static const int NBR_OFF[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                                  {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};

cpm_status validate_surface(const Surface& s, double h, int p) {
  if (!(h > 0.0) || (p != 2 && p != 3) ||
      (s.kind != CPM_SPHERE && s.kind != CPM_TORUS && s.kind != CPM_TRIMESH) ||
      (s.kind != CPM_TRIMESH && !(s.R > 0.0)) || (s.kind == CPM_TORUS && !(s.r > 0.0 && s.r < s.R))) {
    set_error("cpm_build_band: invalid surface, h or p (p must be 2 or 3)");
    return CPM_ERR_INVALID_ARG;
  }
  return CPM_OK;
}

// Working copy of the surface (mesh bucket grid built) and its bounding box.
cpm_status prepare_surface(const Surface& s, double h, Surface& S, double lo[3], double hi[3]) {
  S = Surface{s.kind, s.R, s.r, {}};
  if (s.kind == CPM_SPHERE) {
    for (int a = 0; a < 3; ++a) { lo[a] = -s.R; hi[a] = s.R; }
  } else if (s.kind == CPM_TORUS) {
    double e = s.R + s.r;
    lo[0] = lo[1] = -e; hi[0] = hi[1] = e; lo[2] = -s.r; hi[2] = s.r;
  } else {
    S.mesh.V = s.mesh.V;
    S.mesh.T = s.mesh.T;
    cpm_status st = mesh_prepare(S.mesh, 2.0 * h);
    if (st != CPM_OK) return st;
    for (int a = 0; a < 3; ++a) { lo[a] = S.mesh.V[a]; hi[a] = S.mesh.V[a]; }
    for (size_t v = 0; v < S.mesh.V.size() / 3; ++v)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], S.mesh.V[3 * v + a]);
        hi[a] = std::max(hi[a], S.mesh.V[3 * v + a]);
      }
  }
  return CPM_OK;
}

// Mesh bucket cells with a triangle within Chebyshev distance ceil(lam/cell)+1 (separable
// dilation of the occupied cells along k, then j, then i): a grid node in any other cell is
// farther than lam from every triangle.
void mesh_near_cells(const Mesh& M, double lam, std::vector<uint8_t>& near) {
  const int64_t n0 = M.nc[0], n1 = M.nc[1], n2 = M.nc[2];
  const int R = (int)std::ceil(lam / M.cell) + 1;
  std::vector<uint8_t> a((size_t)(n0 * n1 * n2)), b(a.size());
  for (int64_t c = 0; c < n0 * n1 * n2; ++c) a[c] = M.cell_start[c + 1] > M.cell_start[c];
  auto dilate = [&](std::vector<uint8_t>& src, std::vector<uint8_t>& dst, int axis) {
    const int64_t st = axis == 2 ? 1 : (axis == 1 ? n2 : n1 * n2);
    const int64_t len = axis == 2 ? n2 : (axis == 1 ? n1 : n0);
#pragma omp parallel for
    for (int64_t c = 0; c < n0 * n1 * n2; ++c) {
      const int64_t pos = (c / st) % len;
      uint8_t v = 0;
      for (int64_t d = std::max<int64_t>(0, pos - R); d <= std::min<int64_t>(len - 1, pos + R) && !v; ++d)
        v = src[c + (d - pos) * st];
      dst[c] = v;
    }
  };
  dilate(a, b, 2);
  dilate(b, a, 1);
  dilate(a, b, 0);
  near.swap(b);
}

// Grid nodes x with ||x - CP(x)|| <= lam over the bounding box grown by lam, in
// lexicographic order (slab by slab, i slowest), with their closest points (and triangles).
static cpm_status enumerate_tube(const Surface& S, const double lo[3], const double hi[3], double h, double lam,
                                 std::vector<int32_t>& ijk, std::vector<double>& cp, std::vector<int32_t>& tri) {
  const bool mesh = S.kind == CPM_TRIMESH;
  int64_t imin[3], imax[3];
  for (int a = 0; a < 3; ++a) {
    imin[a] = (int64_t)std::floor((lo[a] - lam) / h) - 1;
    imax[a] = (int64_t)std::ceil((hi[a] + lam) / h) + 1;
  }
  const int64_t ni = imax[0] - imin[0] + 1;
  const int64_t nj = imax[1] - imin[1] + 1, nk = imax[2] - imin[2] + 1;
  if (ni * nj * nk > (int64_t)2000000000) {
    set_error("cpm_build_band: bounding grid too large");
    return CPM_ERR_INVALID_ARG;
  }
  // mesh: only nodes in cells near a triangle can be within lam of the surface
  std::vector<uint8_t> near;
  const Mesh& M = S.mesh;
  if (mesh) mesh_near_cells(M, lam, near);
  std::vector<std::vector<int32_t>> slab_ijk(ni), slab_tri(ni);
  std::vector<std::vector<double>> slab_cp(ni);
#pragma omp parallel
  {
    std::vector<int32_t> stamp(mesh ? (size_t)M.n_tris() : 0, -1);
    int32_t qid = 0;
#pragma omp for schedule(dynamic, 1)
    for (int64_t si = 0; si < ni; ++si) {
      const int64_t i = imin[0] + si;
      for (int64_t j = imin[1]; j <= imax[1]; ++j)
        for (int64_t k = imin[2]; k <= imax[2]; ++k) {
          double x[3] = {(double)i * h, (double)j * h, (double)k * h}, y[3];
          int32_t t = -1;
          if (mesh) {
            int64_t c[3];
            for (int e = 0; e < 3; ++e) c[e] = (int64_t)std::floor((x[e] - M.org[e]) / M.cell);
            if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= M.nc[0] || c[1] >= M.nc[1] || c[2] >= M.nc[2] ||
                !near[(c[0] * M.nc[1] + c[1]) * M.nc[2] + c[2]])
              continue;
            t = mesh_closest_point(M, x, lam, y, stamp, qid);
            if (t < 0) continue;
          } else if (!closest_point(S, x, y)) {
            continue;
          }
          double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
          double dist = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
          if (dist <= lam) {
            slab_ijk[si].insert(slab_ijk[si].end(), {(int32_t)i, (int32_t)j, (int32_t)k});
            slab_cp[si].insert(slab_cp[si].end(), {y[0], y[1], y[2]});
            if (mesh) slab_tri[si].push_back(t);
          }
        }
    }
  }
  ijk.clear();
  cp.clear();
  tri.clear();
  for (int64_t si = 0; si < ni; ++si) {
    ijk.insert(ijk.end(), slab_ijk[si].begin(), slab_ijk[si].end());
    cp.insert(cp.end(), slab_cp[si].begin(), slab_cp[si].end());
    tri.insert(tri.end(), slab_tri[si].begin(), slab_tri[si].end());
  }
  return CPM_OK;
}

// Ghosts, neighbour table and interpolation data of a band whose actives (ijk, cp, tri) are
// set in canonical order.
static cpm_status finish_band(Band& B) {
  const double h = B.h;
  const int p = B.p;
  const bool mesh = B.surf.kind == CPM_TRIMESH;
  const int64_t na = (int64_t)B.ijk.size() / 3;
  if (na == 0) {
    set_error("cpm_build_band: empty band");
    return CPM_ERR_INVALID_ARG;
  }
  B.n_active = na;
  int32_t amin[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, amax[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int64_t g = 0; g < na; ++g)
    for (int a = 0; a < 3; ++a) {
      amin[a] = std::min(amin[a], B.ijk[3 * g + a]);
      amax[a] = std::max(amax[a], B.ijk[3 * g + a]);
    }
  for (int a = 0; a < 3; ++a) {
    B.lo[a] = amin[a] - 2;
    B.dims[a] = amax[a] - amin[a] + 5;
  }
  B.grid.assign((size_t)B.dims[0] * B.dims[1] * B.dims[2], -1);
  auto gidx = [&](int64_t i, int64_t j, int64_t k) -> int32_t& {
    return B.grid[((i - B.lo[0]) * B.dims[1] + (j - B.lo[1])) * B.dims[2] + (k - B.lo[2])];
  };
  for (int64_t g = 0; g < na; ++g) gidx(B.ijk[3 * g], B.ijk[3 * g + 1], B.ijk[3 * g + 2]) = (int32_t)g;
  // ghosts: non-active 6-neighbours, lexicographic
  std::vector<std::array<int32_t, 3>> gh;
  for (int64_t g = 0; g < na; ++g)
    for (int m = 0; m < 6; ++m) {
      int32_t q[3] = {B.ijk[3 * g] + NBR_OFF[m][0], B.ijk[3 * g + 1] + NBR_OFF[m][1],
                      B.ijk[3 * g + 2] + NBR_OFF[m][2]};
      if (gidx(q[0], q[1], q[2]) < 0) gh.push_back({q[0], q[1], q[2]});
    }
  std::sort(gh.begin(), gh.end());
  gh.erase(std::unique(gh.begin(), gh.end()), gh.end());
  B.n_ghost = (int64_t)gh.size();
  B.ijk.resize(3 * (na + B.n_ghost));
  B.cp.resize(3 * (na + B.n_ghost));
  if (mesh) B.tri.resize(na + B.n_ghost);
  int bad_ghost = 0;
#pragma omp parallel reduction(+ : bad_ghost)
  {
    std::vector<int32_t> stamp(mesh ? (size_t)B.surf.mesh.n_tris() : 0, -1);
    int32_t qid = 0;
#pragma omp for
    for (int64_t t = 0; t < B.n_ghost; ++t) {
      const int64_t g = na + t;
      double x[3] = {(double)gh[t][0] * h, (double)gh[t][1] * h, (double)gh[t][2] * h}, y[3];
      bool ok;
      if (mesh) {
        int32_t tr = mesh_closest_point(B.surf.mesh, x, std::numeric_limits<double>::infinity(), y, stamp, qid);
        ok = tr >= 0;
        B.tri[g] = tr;
      } else {
        ok = closest_point(B.surf, x, y);
      }
      if (!ok) bad_ghost++;
      for (int a = 0; a < 3; ++a) {
        B.ijk[3 * g + a] = gh[t][a];
        B.cp[3 * g + a] = y[a];
      }
    }
  }
  for (int64_t t = 0; t < B.n_ghost; ++t) gidx(gh[t][0], gh[t][1], gh[t][2]) = (int32_t)(na + t);
  if (bad_ghost) {
    set_error("cpm_build_band: ghost node without closest point");
    return CPM_ERR_STENCIL;
  }
  B.nbr.resize(na * 6);
  for (int64_t g = 0; g < na; ++g)
    for (int m = 0; m < 6; ++m)
      B.nbr[6 * g + m] = gidx(B.ijk[3 * g] + NBR_OFF[m][0], B.ijk[3 * g + 1] + NBR_OFF[m][1],
                              B.ijk[3 * g + 2] + NBR_OFF[m][2]);
  // interpolation data for every node: base, 1-D weights, z-pencil starts
  const int64_t N = B.n_nodes();
  const int P = p + 1;
  B.base.resize(N * 3);
  B.wts.resize(N * 3 * P);
  B.pencil.resize(N * P * P);
  int bad = 0;
#pragma omp parallel for reduction(+ : bad)
  for (int64_t g = 0; g < N; ++g) {
    double* w = &B.wts[g * 3 * P];
    int32_t* b = &B.base[3 * g];
    point_weights(&B.cp[3 * g], h, p, b, w, w + P, w + 2 * P);
    for (int a = 0; a < P; ++a)
      for (int c = 0; c < P; ++c) {
        int32_t st = B.lookup((int64_t)b[0] + a, (int64_t)b[1] + c, b[2]);
        bool ok = st >= 0 && st < na;
        for (int e = 1; ok && e < P; ++e) ok = B.lookup((int64_t)b[0] + a, (int64_t)b[1] + c, (int64_t)b[2] + e) == st + e;
        if (!ok) bad += 1;
        B.pencil[g * P * P + a * P + c] = ok ? st : -1;
      }
  }
  if (bad) {
    set_error("cpm_build_band: an interpolation stencil leaves the active set (tube radius too small)");
    return CPM_ERR_STENCIL;
  }
  return CPM_OK;
}

cpm_status build_band(const Surface& s, double h, int p, double lam_over_h, Band& B) {
  cpm_status st = validate_surface(s, h, p);
  if (st != CPM_OK) return st;
  if (!(lam_over_h > 0.0)) lam_over_h = ((1.0033 * std::sqrt(3.0)) * (p + 1)) / 2.0;
  const double lam = lam_over_h * h;
  Surface S;
  double lo[3], hi[3];
  st = prepare_surface(s, h, S, lo, hi);
  if (st != CPM_OK) return st;
  std::vector<int32_t> ijk, tri;
  std::vector<double> cp;
  st = enumerate_tube(S, lo, hi, h, lam, ijk, cp, tri);
  if (st != CPM_OK) return st;
  B = Band();
  B.surf = std::move(S);
  B.h = h;
  B.lam = lam;
  B.p = p;
  B.ijk = std::move(ijk);
  B.cp = std::move(cp);
  B.tri = std::move(tri);
  return finish_band(B);
}

cpm_status build_band_algorithmic(const Surface& s, double h, int p, Band& B) {
  cpm_status st = validate_surface(s, h, p);
  if (st != CPM_OK) return st;
  Surface S;
  double lo[3], hi[3];
  st = prepare_surface(s, h, S, lo, hi);
  if (st != CPM_OK) return st;
  const bool mesh = S.kind == CPM_TRIMESH;
  // seed: grid nodes within h of the surface
  std::vector<int32_t> seed, seed_tri;
  std::vector<double> seed_cp;
  st = enumerate_tube(S, lo, hi, h, h, seed, seed_cp, seed_tri);
  if (st != CPM_OK) return st;
  // membership bitmaps over the bounding box grown by a margin wider than any stencil reach
  const int margin = 2 * (p + 1) + 4;
  int64_t gmin[3], gdim[3];
  for (int a = 0; a < 3; ++a) {
    gmin[a] = (int64_t)std::floor(lo[a] / h) - margin;
    gdim[a] = (int64_t)std::ceil(hi[a] / h) + margin - gmin[a] + 1;
  }
  if (gdim[0] * gdim[1] * gdim[2] > (int64_t)4000000000) {
    set_error("cpm_build_band: bounding grid too large");
    return CPM_ERR_INVALID_ARG;
  }
  std::vector<uint8_t> member((size_t)(gdim[0] * gdim[1] * gdim[2]), 0), done(member.size(), 0);
  auto cell = [&](int64_t i, int64_t j, int64_t k) -> int64_t {
    const int64_t a = i - gmin[0], b = j - gmin[1], c = k - gmin[2];
    if (a < 0 || b < 0 || c < 0 || a >= gdim[0] || b >= gdim[1] || c >= gdim[2]) return -1;
    return (a * gdim[1] + b) * gdim[2] + c;
  };
  std::vector<int64_t> frontier;
  for (size_t t = 0; t < seed.size() / 3; ++t) {
    const int64_t c = cell(seed[3 * t], seed[3 * t + 1], seed[3 * t + 2]);
    if (c < 0) { set_error("cpm_build_band: algorithmic band leaves its grid"); return CPM_ERR_STENCIL; }
    if (!member[c]) { member[c] = 1; frontier.push_back(c); }
  }
  const int P = p + 1;
  int bad = 0;
  while (!frontier.empty() && !bad) {
    // the new members and their 6-neighbours not processed yet
    std::vector<int64_t> cand;
    for (int64_t c : frontier) {
      const int64_t k = c % gdim[2], j = (c / gdim[2]) % gdim[1], i = c / (gdim[2] * gdim[1]);
      for (int m = -1; m < 6; ++m) {
        const int64_t q = m < 0 ? c : cell(i + gmin[0] + NBR_OFF[m][0], j + gmin[1] + NBR_OFF[m][1],
                                           k + gmin[2] + NBR_OFF[m][2]);
        if (q < 0) { bad = 1; break; }
        if (!done[q]) { done[q] = 1; cand.push_back(q); }
      }
    }
    // their interpolation stencils
    std::vector<std::vector<int64_t>> found(cand.size());
#pragma omp parallel reduction(+ : bad)
    {
      std::vector<int32_t> stamp(mesh ? (size_t)S.mesh.n_tris() : 0, -1);
      int32_t qid = 0;
#pragma omp for schedule(dynamic, 256)
      for (int64_t t = 0; t < (int64_t)cand.size(); ++t) {
        const int64_t c = cand[t];
        const int64_t k = c % gdim[2], j = (c / gdim[2]) % gdim[1], i = c / (gdim[2] * gdim[1]);
        double x[3] = {(double)(i + gmin[0]) * h, (double)(j + gmin[1]) * h, (double)(k + gmin[2]) * h}, y[3];
        bool ok = mesh ? mesh_closest_point(S.mesh, x, std::numeric_limits<double>::infinity(), y, stamp, qid) >= 0
                       : closest_point(S, x, y);
        if (!ok) { bad++; continue; }
        int32_t b[3];
        double w[24];
        point_weights(y, h, p, b, w, w + P, w + 2 * P);
        for (int a = 0; a < P; ++a)
          for (int bb = 0; bb < P; ++bb)
            for (int e = 0; e < P; ++e) {
              const int64_t q = cell((int64_t)b[0] + a, (int64_t)b[1] + bb, (int64_t)b[2] + e);
              if (q < 0) { bad++; continue; }
              found[t].push_back(q);
            }
      }
    }
    frontier.clear();
    for (auto& f : found)
      for (int64_t q : f)
        if (!member[q]) { member[q] = 1; frontier.push_back(q); }
  }
  if (bad) {
    set_error("cpm_build_band: algorithmic band reaches a point without a closest point or leaves its grid");
    return CPM_ERR_STENCIL;
  }
  // actives in lexicographic order, their closest points
  B = Band();
  for (int64_t c = 0; c < (int64_t)member.size(); ++c)
    if (member[c]) {
      const int64_t k = c % gdim[2], j = (c / gdim[2]) % gdim[1], i = c / (gdim[2] * gdim[1]);
      B.ijk.insert(B.ijk.end(), {(int32_t)(i + gmin[0]), (int32_t)(j + gmin[1]), (int32_t)(k + gmin[2])});
    }
  const int64_t na = (int64_t)B.ijk.size() / 3;
  B.cp.resize(3 * na);
  if (mesh) B.tri.resize(na);
  int nocp = 0;
#pragma omp parallel reduction(+ : nocp)
  {
    std::vector<int32_t> stamp(mesh ? (size_t)S.mesh.n_tris() : 0, -1);
    int32_t qid = 0;
#pragma omp for
    for (int64_t g = 0; g < na; ++g) {
      double x[3] = {(double)B.ijk[3 * g] * h, (double)B.ijk[3 * g + 1] * h, (double)B.ijk[3 * g + 2] * h};
      if (mesh) {
        const int32_t t = mesh_closest_point(S.mesh, x, std::numeric_limits<double>::infinity(), &B.cp[3 * g],
                                             stamp, qid);
        B.tri[g] = t;
        if (t < 0) nocp++;
      } else if (!closest_point(S, x, &B.cp[3 * g])) {
        nocp++;
      }
    }
  }
  if (nocp) {
    set_error("cpm_build_band: an active node without a closest point");
    return CPM_ERR_STENCIL;
  }
  B.surf = std::move(S);
  B.h = h;
  B.lam = 0.0;
  B.p = p;
  return finish_band(B);
}

}  // namespace cpm
