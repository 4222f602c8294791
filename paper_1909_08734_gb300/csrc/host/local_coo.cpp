// Local subdomain operators in coordinate form (Sec. 2.2 Eq. simpleRAS; Sec. 5 Eq. localOP,
// Sec. 4.2 Eq. locCP / Eq. naConorm, Sec. 5.2 Eq. robfo, Sec. 5.2.2 cross points).
//
// RAS:  A_j = R_j A R_j^T, rows/cols Sigma_j, with (A x)_i = (c+6/h^2) x_i
//       - (1/h^2) sum_{k in N6(i)} (E x)_k.
// ORAS: unknowns Sigma_j then Sigma_j^{BC,A}.  The extension v_k of the local vector to a
//       node k is the E-row of k for k in Sigma_j u Sigma_j^G and the Robin T-row
//       (interpolation at CP_{S_j}(x_k) scaled by 1/(1 + alpha_k d_k.q_k)) for boundary
//       nodes.  Reading R1: every unknown gets (c+6/h^2) w_i - (1/h^2) sum_{N6(i)} v_k.
//       Reading R3: boundary unknowns get (c+6/h^2) w_i - (6/h^2) v_i.
#include <algorithm>
#include <cmath>

#include "cpm_internal.h"

namespace cpm {

namespace {

struct Row {
  int n = 0;                 // (p+1)^3 entries
  int32_t col[64];           // local unknown index of each stencil node
  double w[64];
};

// Extension row at a point y: global stencil nodes mapped to local unknowns, weights
// (wx_a * wy_b) * wz_c times scale.  Returns false if a stencil node is not local.
bool ext_row(const Band& B, const double y[3], double scale, const std::vector<int32_t>& loc,
             Row& r) {
  const int p = B.p, P = p + 1;
  int32_t base[3];
  double wx[4], wy[4], wz[4];
  point_weights(y, B.h, p, base, wx, wy, wz);
  r.n = 0;
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < P; ++b)
      for (int c = 0; c < P; ++c) {
        int32_t g = B.lookup((int64_t)base[0] + a, (int64_t)base[1] + b, (int64_t)base[2] + c);
        if (g < 0 || g >= B.n_active || loc[g] < 0) return false;
        r.col[r.n] = loc[g];
        double w = (wx[a] * wy[b]) * wz[c];
        r.w[r.n] = (scale == 1.0) ? w : w * scale;
        r.n++;
      }
  return true;
}

}  // namespace

cpm_status build_local_coo(const Band& B, const Partition& part, double c, int transmission,
                           double alpha, double alpha_x, int j, LocalCOO& out, bool sorted_rows) {
  if (j < 0 || j >= part.n_sub || part.band != &B) {
    set_error("local operator: bad subdomain index or band/partition mismatch");
    return CPM_ERR_INVALID_ARG;
  }
  if (transmission != CPM_RAS && transmission != CPM_ORAS && transmission != CPM_ORAS_R3) {
    set_error("local operator: unknown transmission condition");
    return CPM_ERR_INVALID_ARG;
  }
  const SubSets& S = part.subs[j];
  const double h = B.h;
  const double diag = c + 6.0 / (h * h);
  const double invh2 = 1.0 / (h * h);
  const int64_t na = B.n_active, N = B.n_nodes();
  const bool ras = transmission == CPM_RAS;
  const bool r1 = transmission == CPM_ORAS;

  std::vector<int32_t> U(S.sigma);
  if (!ras) U.insert(U.end(), S.bc_a.begin(), S.bc_a.end());
  const int64_t n = (int64_t)U.size();
  std::vector<int32_t> loc(na, -1);
  for (int64_t i = 0; i < n; ++i) loc[U[i]] = (int32_t)i;

  // extension rows of every node whose value a local row uses
  std::vector<int32_t> pos(N, -1);
  std::vector<Row> rows;
  auto add_node_row = [&](int32_t g, const double* y, double scale) -> bool {
    Row r;
    if (!ext_row(B, y, scale, loc, r)) return false;
    pos[g] = (int32_t)rows.size();
    rows.push_back(r);
    return true;
  };
  std::vector<int32_t> interior(S.sigma);
  interior.insert(interior.end(), S.ghost.begin(), S.ghost.end());
  if (ras) {
    // RAS uses the global E-rows of every neighbour, restricted to Sigma_j columns
    for (int32_t g : S.sigma)
      for (int m = 0; m < 6; ++m) {
        int32_t k = B.nbr[6 * (size_t)g + m];
        if (pos[k] >= 0) continue;
        const int P = B.P(), P2 = P * P;
        Row r;
        r.n = 0;
        for (int s = 0; s < P2; ++s) {
          int32_t st = B.pencil[(size_t)k * P2 + s];
          for (int e = 0; e < P; ++e) {
            int a = s / P, b = s % P;
            const double* w = &B.wts[(size_t)k * 3 * P];
            r.col[r.n] = loc[st + e];                 // -1 outside Sigma_j: dropped
            r.w[r.n] = (w[a] * w[P + b]) * w[2 * P + e];
            r.n++;
          }
        }
        pos[k] = (int32_t)rows.size();
        rows.push_back(r);
      }
  } else {
    for (int32_t g : interior)
      if (!add_node_row(g, &B.cp[3 * (size_t)g], 1.0)) {
        set_error("local operator: an interior extension stencil leaves the local unknowns");
        return CPM_ERR_STENCIL;
      }
    const size_t nbc_a = S.bc_a.size();
    const size_t nbc = r1 ? nbc_a + S.bc_g.size() : nbc_a;
    for (size_t t = 0; t < nbc; ++t) {
      int32_t g = t < nbc_a ? S.bc_a[t] : S.bc_g[t - nbc_a];
      const double* y = &B.cp[3 * (size_t)S.bc_gen[t]];
      double x[3] = {(double)B.ijk[3 * (size_t)g] * h, (double)B.ijk[3 * (size_t)g + 1] * h,
                     (double)B.ijk[3 * (size_t)g + 2] * h};
      double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]}, nv[3];
      node_normal(B, S.bc_gen[t], nv);          // normal at CP_{S_j} = CP(generator)
      double dn = (d[0] * nv[0] + d[1] * nv[1]) + d[2] * nv[2];
      double dp[3] = {d[0] - dn * nv[0], d[1] - dn * nv[1], d[2] - dn * nv[2]};
      double dq = std::sqrt((dp[0] * dp[0] + dp[1] * dp[1]) + dp[2] * dp[2]);
      double a = S.bc_nearx[t] ? alpha_x : alpha;
      double scale = 1.0 / (1.0 + a * dq);
      Row r;
      if (!ext_row(B, y, 1.0, loc, r)) {
        set_error("local operator: a Robin extension stencil leaves the local unknowns");
        return CPM_ERR_STENCIL;
      }
      for (int e = 0; e < r.n; ++e) r.w[e] = r.w[e] * scale;
      pos[g] = (int32_t)rows.size();
      rows.push_back(r);
    }
  }

  // assemble row by row into a dense accumulator
  out = LocalCOO();
  out.n = n;
  out.n_sigma = (int64_t)S.sigma.size();
  std::vector<double> acc(n, 0.0);
  std::vector<uint8_t> hit(n, 0);
  std::vector<int32_t> touched;
  {
    // entries per row: about (p+1)^3 distinct columns from 6 overlapping stencils
    const size_t guess = (size_t)n * (size_t)(3 * B.P() * B.P() * B.P() / 2);
    out.row.reserve(guess);
    out.col.reserve(guess);
    out.val.reserve(guess);
  }
  const int64_t n_pde = (ras || r1) ? n : (int64_t)S.sigma.size();
  for (int64_t i = 0; i < n; ++i) {
    touched.clear();
    const int32_t g = U[i];
    auto put = [&](int32_t col, double v) {
      if (!hit[col]) { hit[col] = 1; touched.push_back(col); acc[col] = v; }
      else acc[col] += v;
    };
    if (ras) {
      for (int m = 0; m < 6; ++m) {
        const Row& r = rows[pos[B.nbr[6 * (size_t)g + m]]];
        for (int e = 0; e < r.n; ++e)
          if (r.col[e] >= 0) put(r.col[e], r.w[e]);
      }
      for (int32_t col : touched) acc[col] = -(acc[col] * invh2);
      put((int32_t)i, 0.0);
      acc[i] = diag + acc[i];
    } else if (i < n_pde) {
      for (int m = 0; m < 6; ++m) {
        int32_t k = B.nbr[6 * (size_t)g + m];
        if (pos[k] < 0) {
          set_error("local operator: a 7-point stencil leaves the local nodes");
          return CPM_ERR_STENCIL;
        }
        const Row& r = rows[pos[k]];
        for (int e = 0; e < r.n; ++e) put(r.col[e], -invh2 * r.w[e]);
      }
      put((int32_t)i, diag);
    } else {
      put((int32_t)i, diag);
      const Row& r = rows[pos[g]];
      for (int e = 0; e < r.n; ++e) put(r.col[e], -(6.0 * invh2) * r.w[e]);
    }
    // the value of every entry is summed in a fixed order either way; sorting only orders
    // the output (set-up consumes the entries in any order)
    if (sorted_rows) std::sort(touched.begin(), touched.end());
    for (int32_t col : touched) {
      out.row.push_back((int32_t)i);
      out.col.push_back(col);
      out.val.push_back(acc[col]);
      hit[col] = 0;
    }
  }
  return CPM_OK;
}

}  // namespace cpm
