// Band construction: closest points, tube-radius active set, ghost set, canonical order,
// neighbour table and interpolation stencils (Sec. 2.1).
#include <algorithm>
#include <array>
#include <cmath>
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

cpm_status build_band(const Surface& s, double h, int p, double lam_over_h, Band& B) {
  if (!(h > 0.0) || (p != 2 && p != 3) || (s.kind != CPM_SPHERE && s.kind != CPM_TORUS) ||
      !(s.R > 0.0) || (s.kind == CPM_TORUS && !(s.r > 0.0 && s.r < s.R))) {
    set_error("cpm_build_band: invalid surface, h or p (p must be 2 or 3)");
    return CPM_ERR_INVALID_ARG;
  }
  if (!(lam_over_h > 0.0)) lam_over_h = ((1.0033 * std::sqrt(3.0)) * (p + 1)) / 2.0;
  const double lam = lam_over_h * h;
  double lo[3], hi[3];
  if (s.kind == CPM_SPHERE) {
    for (int a = 0; a < 3; ++a) { lo[a] = -s.R; hi[a] = s.R; }
  } else {
    double e = s.R + s.r;
    lo[0] = lo[1] = -e; hi[0] = hi[1] = e; lo[2] = -s.r; hi[2] = s.r;
  }
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
  // enumerate slab by slab (i slowest): actives come out in lexicographic order
  std::vector<std::vector<int32_t>> slab_ijk(ni);
  std::vector<std::vector<double>> slab_cp(ni);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t si = 0; si < ni; ++si) {
    const int64_t i = imin[0] + si;
    for (int64_t j = imin[1]; j <= imax[1]; ++j)
      for (int64_t k = imin[2]; k <= imax[2]; ++k) {
        double x[3] = {(double)i * h, (double)j * h, (double)k * h}, y[3];
        if (!closest_point(s, x, y)) continue;
        double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
        double dist = std::sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        if (dist <= lam) {
          slab_ijk[si].insert(slab_ijk[si].end(), {(int32_t)i, (int32_t)j, (int32_t)k});
          slab_cp[si].insert(slab_cp[si].end(), {y[0], y[1], y[2]});
        }
      }
  }
  B = Band();
  B.surf = s;
  B.h = h;
  B.lam = lam;
  B.p = p;
  for (int64_t si = 0; si < ni; ++si) {
    B.ijk.insert(B.ijk.end(), slab_ijk[si].begin(), slab_ijk[si].end());
    B.cp.insert(B.cp.end(), slab_cp[si].begin(), slab_cp[si].end());
  }
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
  for (int64_t t = 0; t < B.n_ghost; ++t) {
    gidx(gh[t][0], gh[t][1], gh[t][2]) = (int32_t)(na + t);
    double x[3] = {(double)gh[t][0] * h, (double)gh[t][1] * h, (double)gh[t][2] * h}, y[3];
    if (!closest_point(s, x, y)) {
      set_error("cpm_build_band: ghost node without closest point");
      return CPM_ERR_STENCIL;
    }
    B.ijk.insert(B.ijk.end(), {gh[t][0], gh[t][1], gh[t][2]});
    B.cp.insert(B.cp.end(), {y[0], y[1], y[2]});
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

}  // namespace cpm
