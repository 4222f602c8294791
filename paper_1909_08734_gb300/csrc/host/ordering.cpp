// Fill-reducing order of a local operator and the tile envelope of its LU factors.
//
// The local solves are exact LU solves of A_j (Eq. localOP; Eq. algRAS applies them); any
// symmetric permutation of the local unknowns gives the same solution up to rounding.  A
// reverse Cuthill-McKee order of the pattern of A_j + A_j^T clusters the entries near the
// diagonal, so that whole 64 x 64 tiles of L and U stay exactly zero:
//   * a row's entries left of its first nonzero tile column never fill (an update adds a
//     multiple of a pivot row only to rows with a nonzero in the pivot column), and row
//     interchanges move whole rows, so "first" travels with the row;
//   * "last" (the last tile column that can be nonzero) grows at step s, for every row
//     still below the pivot block with first <= s, to the largest "last" of the pivot block's
//     rows after the interchanges of step s (tracked on the device with the real pivots);
//   * rows with first <= s occupy positions below max{r : first_r <= s} at every step: a row
//     moves down only into the old position of a pivot row of an earlier step.
#include <algorithm>
#include <memory>
#include <numeric>
#include <vector>

#include "cpm_internal.h"

namespace cpm {

namespace {

struct Graph {
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
  int32_t deg(int32_t v) const { return (int32_t)(ptr[v + 1] - ptr[v]); }
};

// symmetric pattern without the diagonal; built by counting (both directions of every
// off-diagonal entry) and per-row deduplication
Graph pattern(const LocalCOO& L) {
  const int64_t n = L.n;
  Graph g;
  std::vector<int64_t> cnt(n + 1, 0);
  for (size_t k = 0; k < L.row.size(); ++k)
    if (L.row[k] != L.col[k]) {
      cnt[L.row[k] + 1]++;
      cnt[L.col[k] + 1]++;
    }
  for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  std::unique_ptr<int32_t[]> raw(new int32_t[cnt[n]]);   // every slot is written below
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (size_t k = 0; k < L.row.size(); ++k)
    if (L.row[k] != L.col[k]) {
      raw[pos[L.row[k]]++] = L.col[k];
      raw[pos[L.col[k]]++] = L.row[k];
    }
  g.ptr.assign(n + 1, 0);
  g.adj.reserve(cnt[n]);
  std::vector<int32_t> stamp(n, -1);
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t k = cnt[v]; k < cnt[v + 1]; ++k) {
      const int32_t w = raw[k];
      if (stamp[w] != (int32_t)v) {
        stamp[w] = (int32_t)v;
        g.adj.push_back(w);
      }
    }
    g.ptr[v + 1] = (int64_t)g.adj.size();
  }
  return g;
}

// breadth-first levels from root inside the unvisited set; returns the last level
std::vector<int32_t> last_level(const Graph& g, int32_t root, const std::vector<uint8_t>& done,
                                std::vector<int32_t>& level, int* depth) {
  std::vector<int32_t> cur{root}, nxt;
  level[root] = 0;
  std::vector<int32_t> touched{root};
  int d = 0;
  for (;;) {
    nxt.clear();
    for (int32_t v : cur)
      for (int64_t k = g.ptr[v]; k < g.ptr[v + 1]; ++k) {
        const int32_t w = g.adj[k];
        if (!done[w] && level[w] < 0) {
          level[w] = d + 1;
          nxt.push_back(w);
          touched.push_back(w);
        }
      }
    if (nxt.empty()) break;
    cur.swap(nxt);
    ++d;
  }
  for (int32_t v : touched) level[v] = -1;
  *depth = d;
  return cur;
}

}  // namespace

void rcm_order(const LocalCOO& L, std::vector<int32_t>& perm) {
  const int64_t n = L.n;
  const Graph g = pattern(L);
  std::vector<uint8_t> done(n, 0);
  std::vector<int32_t> level(n, -1);
  perm.clear();
  perm.reserve(n);
  for (;;) {
    // start of the next component: the unvisited vertex of least degree (lowest index on ties)
    int32_t root = -1;
    for (int64_t v = 0; v < n; ++v)
      if (!done[v] && (root < 0 || g.deg((int32_t)v) < g.deg(root))) root = (int32_t)v;
    if (root < 0) break;
    // pseudo-peripheral vertex: move to a least-degree vertex of the last level while the
    // eccentricity grows
    int depth = 0;
    std::vector<int32_t> last = last_level(g, root, done, level, &depth);
    for (int guard = 0; guard < 4; ++guard) {
      int32_t cand = last[0];
      for (int32_t v : last)
        if (g.deg(v) < g.deg(cand) || (g.deg(v) == g.deg(cand) && v < cand)) cand = v;
      int d2 = 0;
      std::vector<int32_t> l2 = last_level(g, cand, done, level, &d2);
      if (d2 <= depth) break;
      root = cand;
      depth = d2;
      last.swap(l2);
    }
    // Cuthill-McKee sweep of the component: the unvisited neighbours of each vertex in the
    // order of (degree, index)
    const size_t start = perm.size();
    perm.push_back(root);
    done[root] = 1;
    for (size_t h = start; h < perm.size(); ++h) {
      const int32_t v = perm[h];
      const size_t first_new = perm.size();
      for (int64_t k = g.ptr[v]; k < g.ptr[v + 1]; ++k) {
        const int32_t w = g.adj[k];
        if (!done[w]) {
          done[w] = 1;
          perm.push_back(w);
        }
      }
      std::sort(perm.begin() + first_new, perm.end(), [&](int32_t a, int32_t b) {
        return g.deg(a) != g.deg(b) ? g.deg(a) < g.deg(b) : a < b;
      });
    }
    std::reverse(perm.begin() + start, perm.end());
  }
}

void envelope(const LocalCOO& L, int T, std::vector<int32_t>& first, std::vector<int32_t>& last,
              std::vector<int32_t>& pend) {
  const int64_t np = (int64_t)T * 64;
  first.resize(np);
  last.resize(np);
  for (int64_t r = 0; r < np; ++r) first[r] = last[r] = (int32_t)(r >> 6);   // diagonal / padding
  for (size_t k = 0; k < L.row.size(); ++k) {
    const int32_t r = L.row[k], c = L.col[k] >> 6;
    first[r] = std::min(first[r], c);
    last[r] = std::max(last[r], c);
  }
  // pend[s]: one past the last position that a row with first <= s can occupy, at least the
  // end of the pivot block
  std::vector<int64_t> maxpos(T, -1);
  for (int64_t r = 0; r < np; ++r) maxpos[first[r]] = std::max(maxpos[first[r]], r);
  pend.resize(T);
  int64_t m = -1;
  for (int s = 0; s < T; ++s) {
    m = std::max(m, maxpos[s]);
    pend[s] = (int32_t)std::min(np, std::max(m + 1, (int64_t)64 * (s + 1)));
  }
}

}  // namespace cpm
