// Disjoint split, overlap growth and node sets (Sec. 3.1, Sec. 4.1, Sec. 4.2, Sec. 5.2.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "cpm_internal.h"

namespace cpm {

namespace {

// Recursive coordinate bisection on CP of the actives (stands in for the graph partitioner
// of Sec. 3.1).  Axis of largest extent (ties x<y<z), order (CP[axis], index), left half
// gets floor(n * W_left / W) points and leaves [l0, l0 + P/2).
void rcb(const Band& B, const std::vector<int64_t>& w, std::vector<int32_t>& labels) {
  struct Job {
    std::vector<int32_t> idx;
    int l0, l1;
  };
  std::vector<Job> stack;
  Job root;
  root.idx.resize(B.n_active);
  std::iota(root.idx.begin(), root.idx.end(), 0);
  root.l0 = 0;
  root.l1 = (int)w.size();
  stack.push_back(std::move(root));
  while (!stack.empty()) {
    Job job = std::move(stack.back());
    stack.pop_back();
    const int P = job.l1 - job.l0;
    if (P == 1) {
      for (int32_t g : job.idx) labels[g] = job.l0;
      continue;
    }
    if (job.idx.empty()) continue;     // leaves left empty: reported when the sets are built
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) { mn[a] = mx[a] = B.cp[3 * (size_t)job.idx[0] + a]; }
    for (int32_t g : job.idx)
      for (int a = 0; a < 3; ++a) {
        double v = B.cp[3 * (size_t)g + a];
        mn[a] = std::min(mn[a], v);
        mx[a] = std::max(mx[a], v);
      }
    double ext[3] = {mx[0] - mn[0], mx[1] - mn[1], mx[2] - mn[2]};
    int axis = 0;
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    const int PL = P / 2;
    int64_t WL = 0, W = 0;
    for (int l = job.l0; l < job.l1; ++l) {
      W += w[l];
      if (l < job.l0 + PL) WL += w[l];
    }
    const int64_t n = (int64_t)job.idx.size();
    const int64_t nL = (n * WL) / W;
    // the first nL points in the order (CP[axis], index), a total order: a selection gives the
    // same halves as a full sort (each half is ordered again by its own split)
    if (nL > 0 && nL < n)
      std::nth_element(job.idx.begin(), job.idx.begin() + nL, job.idx.end(), [&](int32_t a, int32_t b) {
        double va = B.cp[3 * (size_t)a + axis], vb = B.cp[3 * (size_t)b + axis];
        return va < vb || (va == vb && a < b);
      });
    Job L, R;
    L.idx.assign(job.idx.begin(), job.idx.begin() + nL);
    R.idx.assign(job.idx.begin() + nL, job.idx.end());
    L.l0 = job.l0; L.l1 = job.l0 + PL;
    R.l0 = job.l0 + PL; R.l1 = job.l1;
    stack.push_back(std::move(R));
    stack.push_back(std::move(L));
  }
}

// Recursive graph bisection on the active 6-neighbour graph (standing in for the graph
// partitioner of Sec. 3.1).  At a tree node: a = the node a breadth-first search from the
// part's lowest index reaches last, b = the node a search from a reaches last (searches stay in
// the part and take neighbours in neighbour-table order); the nodes are ordered by
// (d(a, g) - d(b, g), index), nodes that a does not reach last, and the left half gets the
// first floor(n * W_left / W) of them and leaves [l0, l0 + P/2), as in rcb; swap passes then
// lower the cut without changing the sizes.
void rgb(const Band& B, const std::vector<int64_t>& w, std::vector<int32_t>& labels) {
  const int64_t na = B.n_active;
  std::vector<int32_t> part_of(na, 0), seen(na, -1);
  int32_t stamp = 0, next_tag = 1;
  std::vector<int32_t> order;
  // order := breadth-first search from root within the part (tag), then the other components
  // (each from its lowest index); dist[g] = distance from root for the nodes the first search
  // reaches, -1 for the others.  Returns the number of nodes the first search reached.
  std::vector<int32_t> da(na, -1), db(na, -1);
  auto search = [&](const std::vector<int32_t>& idx, int32_t tag, int32_t root, std::vector<int32_t>& dist) {
    ++stamp;
    order.clear();
    for (int32_t g : idx) dist[g] = -1;
    auto run = [&](int32_t s, bool first) {
      seen[s] = stamp;
      if (first) dist[s] = 0;
      order.push_back(s);
      for (size_t q = order.size() - 1; q < order.size(); ++q) {
        const int32_t u = order[q];
        for (int d = 0; d < 6; ++d) {
          const int32_t v = B.nbr[6 * (size_t)u + d];
          if (v >= 0 && v < na && part_of[v] == tag && seen[v] != stamp) {
            seen[v] = stamp;
            if (first) dist[v] = dist[u] + 1;
            order.push_back(v);
          }
        }
      }
    };
    run(root, true);
    const size_t first = order.size();
    for (int32_t g : idx)
      if (seen[g] != stamp) run(g, false);
    return first;
  };
  // Swap refinement of a bisection (Kernighan-Lin style, sizes kept): gain(g) = neighbours
  // in the part on the other side - neighbours on g's side.  A pass lists each side's boundary
  // nodes with gain >= 0 by (gain descending, index ascending) and walks the two lists in
  // step: the i-th pair (u, v) swaps sides if, with the gains as they are at that moment,
  // gain(u) + gain(v) - 2 [u, v neighbours] > 0.  At most 8 passes; stops at a pass without
  // a swap.
  std::vector<int8_t> side(na, 0);
  auto gain = [&](int32_t g, int32_t tag, int* ext) {
    int e = 0, i = 0;
    for (int d = 0; d < 6; ++d) {
      const int32_t v = B.nbr[6 * (size_t)g + d];
      if (v >= 0 && v < na && part_of[v] == tag) (side[v] != side[g] ? e : i)++;
    }
    if (ext) *ext = e;
    return e - i;
  };
  auto refine = [&](const std::vector<int32_t>& idx, int32_t tag) {
    std::vector<std::pair<int, int32_t>> cl, cr;
    for (int pass = 0; pass < 8; ++pass) {
      cl.clear();
      cr.clear();
      for (int32_t g : idx) {
        int e = 0;
        const int gn = gain(g, tag, &e);
        if (e > 0 && gn >= 0) (side[g] == 0 ? cl : cr).emplace_back(-gn, g);
      }
      std::sort(cl.begin(), cl.end());
      std::sort(cr.begin(), cr.end());
      int swaps = 0;
      for (size_t q = 0; q < std::min(cl.size(), cr.size()); ++q) {
        const int32_t u = cl[q].second, v = cr[q].second;
        bool adj = false;
        for (int d = 0; d < 6; ++d) adj = adj || B.nbr[6 * (size_t)u + d] == v;
        if (gain(u, tag, nullptr) + gain(v, tag, nullptr) - 2 * (adj ? 1 : 0) > 0) {
          side[u] = 1;
          side[v] = 0;
          ++swaps;
        }
      }
      if (swaps == 0) break;
    }
  };
  struct Job {
    std::vector<int32_t> idx;   // ascending
    int l0, l1;
    int32_t tag;
  };
  std::vector<Job> stack;
  std::vector<std::pair<int64_t, int32_t>> keyed;
  Job root;
  root.idx.resize(na);
  std::iota(root.idx.begin(), root.idx.end(), 0);
  root.l0 = 0;
  root.l1 = (int)w.size();
  root.tag = 0;
  stack.push_back(std::move(root));
  while (!stack.empty()) {
    Job job = std::move(stack.back());
    stack.pop_back();
    const int P = job.l1 - job.l0;
    if (P == 1) {
      for (int32_t g : job.idx) labels[g] = job.l0;
      continue;
    }
    if (job.idx.empty()) continue;     // leaves left empty: reported when the sets are built
    // a = the last node reached from the lowest index, b = the last node reached from a;
    // order by (d(a, g) - d(b, g), index): the cut is a level set of the difference of the two
    // graph distances (nodes the search from a does not reach come last, by index)
    const size_t r0 = search(job.idx, job.tag, job.idx[0], da);
    const int32_t a = order[r0 - 1];
    const size_t ra = search(job.idx, job.tag, a, da);
    const int32_t b = order[ra - 1];
    search(job.idx, job.tag, b, db);
    keyed.clear();
    for (int32_t g : job.idx)
      keyed.emplace_back(da[g] >= 0 ? (int64_t)da[g] - db[g] : (int64_t)1 << 40, g);
    std::sort(keyed.begin(), keyed.end());
    order.clear();
    for (auto& kg : keyed) order.push_back(kg.second);
    const int PL = P / 2;
    int64_t WL = 0, W = 0;
    for (int l = job.l0; l < job.l1; ++l) {
      W += w[l];
      if (l < job.l0 + PL) WL += w[l];
    }
    const int64_t n = (int64_t)job.idx.size();
    const int64_t nL = (n * WL) / W;
    for (size_t q = 0; q < order.size(); ++q) side[order[q]] = (int64_t)q < nL ? 0 : 1;
    refine(job.idx, job.tag);
    Job L, R;
    for (int32_t g : job.idx) (side[g] == 0 ? L.idx : R.idx).push_back(g);
    L.l0 = job.l0; L.l1 = job.l0 + PL; L.tag = next_tag++;
    R.l0 = job.l0 + PL; R.l1 = job.l1; R.tag = next_tag++;
    for (int32_t g : L.idx) part_of[g] = L.tag;
    for (int32_t g : R.idx) part_of[g] = R.tag;
    stack.push_back(std::move(R));
    stack.push_back(std::move(L));
  }
}

void sort_unique(std::vector<int32_t>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

}  // namespace

// Interface alignment (Sec. 3.2): an active node with an active 6-neighbour of another
// label moves to the label of the grid node nearest to its closest point,
// floor(CP/h + 0.5) per axis; every move of a pass is decided on the labels before it.
static void align_interfaces(const Band& B, int passes, std::vector<int32_t>& lab) {
  const int64_t na = B.n_active;
  std::vector<int32_t> target(na), next(na);
#pragma omp parallel for
  for (int64_t g = 0; g < na; ++g) {
    int64_t q[3];
    for (int a = 0; a < 3; ++a) q[a] = (int64_t)std::floor(B.cp[3 * g + a] / B.h + 0.5);
    const int32_t t = B.lookup(q[0], q[1], q[2]);
    target[g] = (t >= 0 && t < na) ? t : -1;
  }
  for (int pass = 0; pass < passes; ++pass) {
#pragma omp parallel for
    for (int64_t g = 0; g < na; ++g) {
      const int32_t l = lab[g];
      bool iface = false;
      for (int m = 0; m < 6; ++m) {
        const int32_t nb = B.nbr[6 * g + m];
        if (nb < na && lab[nb] != l) iface = true;
      }
      next[g] = (iface && target[g] >= 0) ? lab[target[g]] : l;
    }
    lab.swap(next);
  }
}

static cpm_status finish_partition(const Band& B, Partition& part);

cpm_status build_partition(const Band& B, int n_sub, const int64_t* weights, int n_overlap,
                           int align_passes, Partition& part, int split) {
  if (n_sub < 1 || n_overlap < 0 || n_sub > B.n_active) {
    set_error("cpm_partition: need 1 <= n_sub <= N_A and n_overlap >= 0");
    return CPM_ERR_INVALID_ARG;
  }
  std::vector<int64_t> w(n_sub, 1);
  if (weights)
    for (int l = 0; l < n_sub; ++l) {
      if (weights[l] <= 0) {
        set_error("cpm_partition: leaf weights must be positive");
        return CPM_ERR_INVALID_ARG;
      }
      w[l] = weights[l];
    }
  const int64_t na = B.n_active;
  part = Partition();
  part.band = &B;
  part.n_sub = n_sub;
  part.n_overlap = n_overlap;
  part.labels.assign(na, -1);
  if (split == 1) rgb(B, w, part.labels);
  else rcb(B, w, part.labels);
  if (align_passes > 0) align_interfaces(B, align_passes, part.labels);
  return finish_partition(B, part);
}

cpm_status build_partition_from_labels(const Band& B, int n_sub, const int32_t* labels, int n_overlap,
                                       Partition& part) {
  if (n_sub < 1 || n_overlap < 0 || n_sub > B.n_active || !labels) {
    set_error("cpm_partition_from_labels: need 1 <= n_sub <= N_A, n_overlap >= 0 and labels");
    return CPM_ERR_INVALID_ARG;
  }
  const int64_t na = B.n_active;
  for (int64_t g = 0; g < na; ++g)
    if (labels[g] < 0 || labels[g] >= n_sub) {
      set_error("cpm_partition_from_labels: a label is outside [0, n_sub)");
      return CPM_ERR_INVALID_ARG;
    }
  part = Partition();
  part.band = &B;
  part.n_sub = n_sub;
  part.n_overlap = n_overlap;
  part.labels.assign(labels, labels + na);
  return finish_partition(B, part);
}

// Everything after the split (Sec. 4.1 overlap and boundary sets, Sec. 4.2 Lambda_j and
// CP_{S_j} generators, Sec. 5.2.2 cross points): a function of the labels, n_sub and N_O.
static cpm_status finish_partition(const Band& B, Partition& part) {
  const int n_sub = part.n_sub, n_overlap = part.n_overlap;
  const int64_t na = B.n_active, N = B.n_nodes();
  std::vector<int64_t> count(n_sub, 0);
  for (int64_t g = 0; g < na; ++g) count[part.labels[g]]++;
  for (int l = 0; l < n_sub; ++l)
    if (count[l] == 0) {
      set_error("cpm_partition: a subdomain is empty");
      return CPM_ERR_INVALID_ARG;
    }
  // cross-point nodes: active neighbours in >= 2 subdomains other than the own one
  for (int64_t g = 0; g < na; ++g) {
    int32_t seen[6];
    int ns = 0;
    for (int m = 0; m < 6; ++m) {
      int32_t q = B.nbr[6 * g + m];
      if (q >= na) continue;
      int32_t l = part.labels[q];
      if (l == part.labels[g]) continue;
      bool dup = false;
      for (int t = 0; t < ns; ++t) dup |= seen[t] == l;
      if (!dup) seen[ns++] = l;
    }
    if (ns >= 2) part.cross.push_back((int32_t)g);
  }
  // grid marks within 2 N_O grid steps (inclusive, Euclidean) of any cross-point node
  const int rad = 2 * n_overlap;
  int32_t mlo[3], mdim[3];
  for (int a = 0; a < 3; ++a) {
    mlo[a] = B.lo[a] - rad;
    mdim[a] = B.dims[a] + 2 * rad;
  }
  std::vector<uint8_t> mark((size_t)mdim[0] * mdim[1] * mdim[2], 0);
  for (int32_t g : part.cross) {
    const int32_t* q = &B.ijk[3 * (size_t)g];
    for (int a = -rad; a <= rad; ++a)
      for (int b = -rad; b <= rad; ++b)
        for (int c = -rad; c <= rad; ++c) {
          if (a * a + b * b + c * c > rad * rad) continue;
          size_t o = ((size_t)(q[0] + a - mlo[0]) * mdim[1] + (q[1] + b - mlo[1])) * mdim[2] + (q[2] + c - mlo[2]);
          mark[o] = 1;
        }
  }
  auto near_cross = [&](int32_t g) {
    const int32_t* q = &B.ijk[3 * (size_t)g];
    return mark[((size_t)(q[0] - mlo[0]) * mdim[1] + (q[1] - mlo[1])) * mdim[2] + (q[2] - mlo[2])];
  };

  part.subs.resize(n_sub);
  for (int64_t g = 0; g < na; ++g) part.subs[part.labels[g]].own.push_back((int32_t)g);
  const int P = B.P(), P2 = P * P;
  int failed = 0;
#pragma omp parallel
  {
    std::vector<int32_t> dist(na, -1), tag(N, -1);
    std::vector<int32_t> touched;
#pragma omp for schedule(dynamic, 1)
    for (int j = 0; j < n_sub; ++j) {
      SubSets& S = part.subs[j];
      touched.clear();
      for (int32_t g : S.own) {
        dist[g] = 0;
        touched.push_back(g);
      }
      // BFS over the active 6-neighbour graph, N_O layers (Sec. 4.1)
      std::vector<int32_t> front = S.own, next;
      for (int layer = 1; layer <= n_overlap; ++layer) {
        next.clear();
        for (int32_t g : front)
          for (int m = 0; m < 6; ++m) {
            int32_t q = B.nbr[6 * (size_t)g + m];
            if (q < na && dist[q] < 0) {
              dist[q] = layer;
              next.push_back(q);
              touched.push_back(q);
            }
          }
        front.swap(next);
      }
      for (int32_t g : touched) {
        S.sigma.push_back(g);
        if (dist[g] == n_overlap) S.last.push_back(g);
      }
      sort_unique(S.sigma);
      sort_unique(S.last);
      // tags: 1 = Sigma_j, 2 = Sigma_j^G, 3 = BC active, 4 = BC ghost layer
      for (int32_t g : S.sigma) tag[g] = 1;
      for (int32_t g : S.sigma)
        for (int m = 0; m < 6; ++m) {
          int32_t q = B.nbr[6 * (size_t)g + m];
          if (q >= na) {
            if (tag[q] != 2) { tag[q] = 2; S.ghost.push_back(q); }
          } else if (tag[q] != 1 && tag[q] != 3) {
            tag[q] = 3;
            S.bc_a.push_back(q);
          }
        }
      sort_unique(S.ghost);
      auto add_stencil = [&](int32_t g) {
        for (int s = 0; s < P2; ++s) {
          int32_t st = B.pencil[(size_t)g * P2 + s];
          for (int e = 0; e < P; ++e) {
            int32_t q = st + e;
            if (tag[q] != 1 && tag[q] != 3) { tag[q] = 3; S.bc_a.push_back(q); }
          }
        }
      };
      for (int32_t g : S.sigma) add_stencil(g);
      for (int32_t g : S.ghost) add_stencil(g);
      sort_unique(S.bc_a);
      for (int32_t g : S.bc_a)
        for (int m = 0; m < 6; ++m) {
          int32_t q = B.nbr[6 * (size_t)g + m];
          if (tag[q] < 0) { tag[q] = 4; S.bc_g.push_back(q); }
        }
      sort_unique(S.bc_g);
      // nearest Lambda_j point of every BC node (Eq. locCP, exhaustive, ties: lowest tag)
      auto nearest = [&](int32_t g) -> int32_t {
        double x[3] = {(double)B.ijk[3 * (size_t)g] * B.h, (double)B.ijk[3 * (size_t)g + 1] * B.h,
                       (double)B.ijk[3 * (size_t)g + 2] * B.h};
        double best = 0;
        int32_t bi = -1;
        for (int32_t t : S.last) {
          const double* y = &B.cp[3 * (size_t)t];
          double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
          double dd = (d0 * d0 + d1 * d1) + d2 * d2;
          if (bi < 0 || dd < best) { best = dd; bi = t; }
        }
        return bi;
      };
      S.bc_gen.reserve(S.bc_a.size() + S.bc_g.size());
      for (int32_t g : S.bc_a) S.bc_gen.push_back(nearest(g));
      for (int32_t g : S.bc_g) S.bc_gen.push_back(nearest(g));
      for (int32_t g : S.bc_a) S.bc_nearx.push_back(near_cross(g));
      for (int32_t g : S.bc_g) S.bc_nearx.push_back(near_cross(g));
      if (!S.bc_a.empty() && S.last.empty()) {
#pragma omp atomic
        failed += 1;
      }
      // reset scratch
      for (int32_t g : touched) dist[g] = -1;
      for (int32_t g : S.sigma) tag[g] = -1;
      for (int32_t g : S.ghost) tag[g] = -1;
      for (int32_t g : S.bc_a) tag[g] = -1;
      for (int32_t g : S.bc_g) tag[g] = -1;
    }
  }
  if (failed) {
    set_error("cpm_partition: a subdomain has boundary nodes but no last overlap layer");
    return CPM_ERR_STENCIL;
  }
  return CPM_OK;
}

}  // namespace cpm
