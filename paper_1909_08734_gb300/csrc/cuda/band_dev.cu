// Band construction on the device (Sec. 2.1): the same active nodes, closest points, canonical
// order, ghosts, neighbour table and interpolation data as the host construction, bit for bit.
// This file is compiled without floating-point contraction (-fmad=false): every closest point,
// distance and weight is computed with the host code's operations in the host code's order
// (the host code is compiled with -ffp-contract=off); IEEE division and square root are
// correctly rounded on both.
//
// Steps, each a grid-wide kernel: tube test of every grid node of the bounding box (closest
// point, distance <= lambda), order-preserving compaction (linear box index = lexicographic
// (i, j, k) order), dense index grid over the actives' box grown by 2, ghost marks (non-active
// 6-neighbours) compacted in grid order, ghost closest points, neighbour table, stencil bases,
// 1-D weights and z-pencil starts.  The host arrays are then filled from the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "../host/cpm_internal.h"
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

struct DevMesh {
  const double* V;
  const int32_t* T;
  const int64_t* cell_start;
  const int32_t* cell_tris;
  const float4* sph;      // per triangle: a bounding sphere (centre, radius), rounded outward
  double org[3];
  double cell;
  int32_t nc[3];
};
struct Geo {
  int kind;
  double R, r;
  DevMesh m;
};

__device__ __forceinline__ double dmin(double a, double b) { return b < a ? b : a; }   // std::min
__device__ __forceinline__ double inf64() { return __longlong_as_double(0x7ff0000000000000ll); }

// Closest point of the sphere or torus (returns false where it is undefined).
__device__ bool cp_analytic(const Geo& s, const double x[3], double y[3]) {
  if (s.kind == CPM_SPHERE) {
    const double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
    if (r == 0.0) return false;
    for (int a = 0; a < 3; ++a) y[a] = (x[a] / r) * s.R;
    return true;
  }
  const double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (rho == 0.0) return false;
  const double C[3] = {(x[0] / rho) * s.R, (x[1] / rho) * s.R, 0.0};
  const double v[3] = {x[0] - C[0], x[1] - C[1], x[2] - C[2]};
  const double sn = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
  if (sn == 0.0) return false;
  for (int a = 0; a < 3; ++a) y[a] = C[a] + (v[a] / sn) * s.r;
  return true;
}

__device__ __forceinline__ double dot3(const double* u, const double* v) {
  return (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2];
}

// Closest point of triangle (a, b, c) to p: the Voronoi-region tests of the point-triangle
// algorithm (Ericson, Real-Time Collision Detection, Sec. 5.1.5) in the host code's order.
__device__ void tri_closest(const double* p, const double* a, const double* b, const double* c, double* y) {
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

// Exact closest point over all triangles by rings of bucket cells at Chebyshev distance
// K = 0, 1, ... (the search ends once the rings' box is farther than both the best distance
// and dmax); ties go to the lowest triangle index, so a triangle met in several cells changes
// nothing.  Returns the triangle, or -1 if none lies within dmax.
// A triangle whose bounding sphere is, in FP32 and less a margin far above FP32 rounding,
// farther than the best distance so far is skipped: its exact distance is then strictly larger
// than the best, so it could neither win nor tie, and the result is the host's.  Only the
// remaining triangles take the exact FP64 test (the FP64 pipe is the scarce one here).
__device__ int32_t mesh_cp(const DevMesh& m, const double x[3], double dmax, double y[3]) {
  int64_t c0[3];
  for (int e = 0; e < 3; ++e) c0[e] = (int64_t)floor((x[e] - m.org[e]) / m.cell);
  double best = inf64();
  int32_t bt = -1;
  double ty[3];
  const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
  const float xmag = 1.0f + fabsf(xf[0]) + fabsf(xf[1]) + fabsf(xf[2]);
  float sbest = __int_as_float(0x7f800000);          // sqrt(best) in FP32 (best = inf)
  for (int64_t K = 0;; ++K) {
    if (K > 0) {
      double lb = inf64();
      bool covers = true;
      for (int e = 0; e < 3; ++e) {
        const double f0 = m.org[e] + (double)(c0[e] - (K - 1)) * m.cell;
        const double f1 = m.org[e] + (double)(c0[e] + K) * m.cell;
        lb = dmin(lb, dmin(x[e] - f0, f1 - x[e]));
        covers = covers && c0[e] - (K - 1) <= 0 && c0[e] + (K - 1) >= m.nc[e] - 1;
      }
      const double lim = dmin(sqrt(best), dmax);
      if (covers || lb > lim * (1.0 + 1e-9) + 1e-12) break;
    }
    const int64_t i0 = max((int64_t)0, c0[0] - K), i1 = min((int64_t)m.nc[0] - 1, c0[0] + K);
    const int64_t j0 = max((int64_t)0, c0[1] - K), j1 = min((int64_t)m.nc[1] - 1, c0[1] + K);
    for (int64_t i = i0; i <= i1; ++i)
      for (int64_t j = j0; j <= j1; ++j) {
        const bool shell = llabs(i - c0[0]) == K || llabs(j - c0[1]) == K;
        for (int64_t kk = 0; kk < (shell ? 2 * K + 1 : 2); ++kk) {
          const int64_t k = shell ? c0[2] - K + kk : (kk == 0 ? c0[2] - K : c0[2] + K);
          if (k < 0 || k >= m.nc[2] || (!shell && K == 0 && kk == 1)) continue;
          const int64_t c = (i * m.nc[1] + j) * m.nc[2] + k;
          for (int64_t q = m.cell_start[c]; q < m.cell_start[c + 1]; ++q) {
            const int32_t t = m.cell_tris[q];
            const float4 sp = m.sph[t];
            const float dx = xf[0] - sp.x, dy = xf[1] - sp.y, dz = xf[2] - sp.z;
            // margin: 1e-5 of the coordinates' size, far above the FP32 rounding of |x - c|
            const float eps = 1e-5f * (xmag + fabsf(sp.x) + fabsf(sp.y) + fabsf(sp.z));
            if (sqrtf((dx * dx + dy * dy) + dz * dz) - sp.w > sbest + eps) continue;
            tri_closest(x, m.V + 3 * (int64_t)m.T[3 * (int64_t)t], m.V + 3 * (int64_t)m.T[3 * (int64_t)t + 1],
                        m.V + 3 * (int64_t)m.T[3 * (int64_t)t + 2], ty);
            const double d[3] = {x[0] - ty[0], x[1] - ty[1], x[2] - ty[2]};
            const double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (d2 < best || (d2 == best && t < bt)) {
              best = d2;
              bt = t;
              y[0] = ty[0];
              y[1] = ty[1];
              y[2] = ty[2];
              sbest = __fsqrt_ru(__double2float_ru(best));
            }
          }
        }
      }
  }
  if (bt < 0 || sqrt(best) > dmax * (1.0 + 1e-9) + 1e-12) return -1;
  return bt;
}

// 1-D barycentric Lagrange weights on nodes 0..p at offset t (second form, beta_m =
// (-1)^m C(p, m); a delta at a node).
__device__ void bary(double t, int p, double* w) {
  double q[8];
  double binom = 1.0;
  int exact = -1;
  for (int m = 0; m <= p; ++m) {
    const double beta = (m % 2 == 0) ? binom : -binom;
    const double diff = t - (double)m;
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

// ---- tube test over the bounding box --------------------------------------------------
// Node L of the box (k fastest, then j, then i) is x = (i h, j h, k h).  Meshes skip nodes in
// cells far from every triangle (near[cell] == 0), exactly as the host does.
struct BoxDim {
  int64_t i0, j0, k0, nj, nk, n;
};

__global__ void tube_kernel(Geo s, const uint8_t* __restrict__ near, BoxDim b, double h, double lam,
                            uint8_t* __restrict__ flag, double* __restrict__ cpd, int32_t* __restrict__ trid) {
  const bool mesh = s.kind == CPM_TRIMESH;
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < b.n; L += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b.i0 + L / (b.nj * b.nk), rem = L % (b.nj * b.nk);
    const int64_t j = b.j0 + rem / b.nk, k = b.k0 + rem % b.nk;
    const double x[3] = {(double)i * h, (double)j * h, (double)k * h};
    double y[3];
    int32_t t = -1;
    uint8_t on = 0;
    if (mesh) {
      int64_t c[3];
      for (int e = 0; e < 3; ++e) c[e] = (int64_t)floor((x[e] - s.m.org[e]) / s.m.cell);
      const bool inside = c[0] >= 0 && c[1] >= 0 && c[2] >= 0 && c[0] < s.m.nc[0] && c[1] < s.m.nc[1] &&
                          c[2] < s.m.nc[2];
      if (inside && near[(c[0] * s.m.nc[1] + c[1]) * s.m.nc[2] + c[2]]) {
        t = mesh_cp(s.m, x, lam, y);
        on = t >= 0;
      }
    } else {
      on = cp_analytic(s, x, y);
    }
    if (on) {
      const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
      const double dist = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      on = dist <= lam;
    }
    flag[L] = on;
    if (on) {
      cpd[3 * L] = y[0];
      cpd[3 * L + 1] = y[1];
      cpd[3 * L + 2] = y[2];
      if (mesh) trid[L] = t;          // trid holds one entry per box node for meshes only
    }
  }
}

// ---- order-preserving compaction -----------------------------------------------------------
// pos[L] = number of flagged entries before L (exclusive prefix sum), in three launches: chunk
// sums, a scan of the chunk sums (one block), and the per-element positions.
constexpr int CT = 1024;                // threads per block
constexpr int CE = 4;                   // elements per thread
constexpr int CCH = CT * CE;            // elements per chunk

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t s = lane < CT / 32 ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[32 + lane] = s;                  // inclusive warp totals
  }
  __syncthreads();
  const int64_t before = warp > 0 ? sh[32 + warp - 1] : 0;
  if (total) *total = sh[32 + CT / 32 - 1];
  const int64_t r = before + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(CT) chunk_sum_kernel(const uint8_t* __restrict__ flag, int64_t n,
                                                       int64_t* __restrict__ sums) {
  __shared__ int64_t sh[64];
  const int64_t base = (int64_t)blockIdx.x * CCH + (int64_t)threadIdx.x * CE;
  int64_t v = 0;
  for (int e = 0; e < CE; ++e)
    if (base + e < n) v += flag[base + e];
  int64_t tot = 0;
  block_excl_scan(v, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// sums[0 .. nb) -> exclusive prefix sums; sums[nb] = total (one block)
__global__ void __launch_bounds__(CT) scan_sums_kernel(int64_t* __restrict__ sums, int64_t nb) {
  __shared__ int64_t sh[64];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += CT) {
    const int64_t b = b0 + threadIdx.x;
    const int64_t v = b < nb ? sums[b] : 0;
    int64_t tot = 0;
    const int64_t ex = block_excl_scan(v, sh, &tot);
    if (b < nb) sums[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(CT) positions_kernel(const uint8_t* __restrict__ flag, int64_t n,
                                                       const int64_t* __restrict__ sums, int32_t* __restrict__ pos) {
  __shared__ int64_t sh[64];
  const int64_t base = (int64_t)blockIdx.x * CCH + (int64_t)threadIdx.x * CE;
  int64_t v = 0;
  for (int e = 0; e < CE; ++e)
    if (base + e < n) v += flag[base + e];
  int64_t run = sums[blockIdx.x] + block_excl_scan(v, sh, nullptr);
  for (int e = 0; e < CE; ++e)
    if (base + e < n) {
      pos[base + e] = (int32_t)run;
      run += flag[base + e];
    }
}

// actives in box order
__global__ void gather_actives_kernel(const uint8_t* __restrict__ flag, const int32_t* __restrict__ pos, BoxDim b,
                                      const double* __restrict__ cpd, const int32_t* __restrict__ trid,
                                      int32_t* __restrict__ ijk, double* __restrict__ cp, int32_t* __restrict__ tri) {
  for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < b.n; L += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[L]) continue;
    const int64_t g = pos[L];
    const int64_t rem = L % (b.nj * b.nk);
    ijk[3 * g] = (int32_t)(b.i0 + L / (b.nj * b.nk));
    ijk[3 * g + 1] = (int32_t)(b.j0 + rem / b.nk);
    ijk[3 * g + 2] = (int32_t)(b.k0 + rem % b.nk);
    cp[3 * g] = cpd[3 * L];
    cp[3 * g + 1] = cpd[3 * L + 1];
    cp[3 * g + 2] = cpd[3 * L + 2];
    if (tri) tri[g] = trid[L];
  }
}

// ---- index grid, ghosts, neighbours, interpolation data -------------------------------
struct GridDim {
  int32_t lo[3], dims[3];
  __device__ int64_t index(int64_t i, int64_t j, int64_t k) const {
    const int64_t a = i - lo[0], b = j - lo[1], c = k - lo[2];
    if (a < 0 || b < 0 || c < 0 || a >= dims[0] || b >= dims[1] || c >= dims[2]) return -1;
    return (a * dims[1] + b) * dims[2] + c;
  }
};
__constant__ int NBR_D[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

__global__ void bbox_kernel(const int32_t* __restrict__ ijk, int64_t na, int32_t* __restrict__ mn,
                            int32_t* __restrict__ mx) {
  int32_t a[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, z[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < na; g += (int64_t)gridDim.x * blockDim.x)
    for (int e = 0; e < 3; ++e) {
      a[e] = min(a[e], ijk[3 * g + e]);
      z[e] = max(z[e], ijk[3 * g + e]);
    }
  for (int e = 0; e < 3; ++e) {
    atomicMin(&mn[e], a[e]);
    atomicMax(&mx[e], z[e]);
  }
}

__global__ void grid_actives_kernel(const int32_t* __restrict__ ijk, int64_t na, GridDim gd, int32_t* __restrict__ grid) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < na; g += (int64_t)gridDim.x * blockDim.x)
    grid[gd.index(ijk[3 * g], ijk[3 * g + 1], ijk[3 * g + 2])] = (int32_t)g;
}

__global__ void ghost_mark_kernel(const int32_t* __restrict__ ijk, int64_t na, GridDim gd,
                                  const int32_t* __restrict__ grid, uint8_t* __restrict__ mark) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < na; g += (int64_t)gridDim.x * blockDim.x)
    for (int m = 0; m < 6; ++m) {
      const int64_t q = gd.index(ijk[3 * g] + NBR_D[m][0], ijk[3 * g + 1] + NBR_D[m][1], ijk[3 * g + 2] + NBR_D[m][2]);
      if (q >= 0 && grid[q] < 0) mark[q] = 1;
    }
}

// ghost t (grid order): its node index na + t, coordinates and closest point
__global__ void ghosts_kernel(Geo s, const uint8_t* __restrict__ mark, const int32_t* __restrict__ pos, GridDim gd,
                              int64_t ncell, int64_t na, double h, int32_t* __restrict__ grid, int32_t* __restrict__ ijk,
                              double* __restrict__ cp, int32_t* __restrict__ tri, int* __restrict__ bad) {
  const int64_t plane = (int64_t)gd.dims[1] * gd.dims[2];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ncell; q += (int64_t)gridDim.x * blockDim.x) {
    if (!mark[q]) continue;
    const int64_t g = na + pos[q];
    const int64_t rem = q % plane;
    const int32_t c[3] = {(int32_t)(gd.lo[0] + q / plane), (int32_t)(gd.lo[1] + rem / gd.dims[2]),
                          (int32_t)(gd.lo[2] + rem % gd.dims[2])};
    const double x[3] = {(double)c[0] * h, (double)c[1] * h, (double)c[2] * h};
    double y[3] = {0.0, 0.0, 0.0};
    bool ok;
    if (s.kind == CPM_TRIMESH) {
      const int32_t t = mesh_cp(s.m, x, inf64(), y);
      ok = t >= 0;
      tri[g] = t;
    } else {
      ok = cp_analytic(s, x, y);
    }
    if (!ok) atomicAdd(bad, 1);
    for (int e = 0; e < 3; ++e) {
      ijk[3 * g + e] = c[e];
      cp[3 * g + e] = y[e];
    }
    grid[q] = (int32_t)g;
  }
}

__global__ void nbr_kernel(const int32_t* __restrict__ ijk, int64_t na, GridDim gd, const int32_t* __restrict__ grid,
                           int32_t* __restrict__ nbr) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < na; g += (int64_t)gridDim.x * blockDim.x)
    for (int m = 0; m < 6; ++m) {
      const int64_t q = gd.index(ijk[3 * g] + NBR_D[m][0], ijk[3 * g + 1] + NBR_D[m][1], ijk[3 * g + 2] + NBR_D[m][2]);
      nbr[6 * g + m] = q >= 0 ? grid[q] : -1;
    }
}

// stencil base and 1-D weights of CP(x) for every node, and the z-pencil starts (first active
// index of each run of p+1 consecutive actives along z, or -1 and a count of bad stencils)
__global__ void interp_kernel(const double* __restrict__ cp, int64_t N, int64_t na, GridDim gd,
                              const int32_t* __restrict__ grid, double h, int p, int32_t* __restrict__ base,
                              double* __restrict__ wts, int32_t* __restrict__ pencil, int* __restrict__ bad) {
  const int P = p + 1;
  auto lookup = [&](int64_t i, int64_t j, int64_t k) -> int32_t {
    const int64_t q = gd.index(i, j, k);
    return q >= 0 ? grid[q] : -1;
  };
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    int32_t b[3];
    for (int a = 0; a < 3; ++a) {
      const double s = cp[3 * g + a] / h;
      const double bb = floor(s - (double)(p - 1) / 2.0);
      const double t = s - bb;
      b[a] = (int32_t)bb;
      base[3 * g + a] = b[a];
      bary(t, p, wts + g * 3 * P + a * P);
    }
    int nbad = 0;
    for (int a = 0; a < P; ++a)
      for (int c = 0; c < P; ++c) {
        const int32_t st = lookup((int64_t)b[0] + a, (int64_t)b[1] + c, b[2]);
        bool ok = st >= 0 && st < na;
        for (int e = 1; ok && e < P; ++e) ok = lookup((int64_t)b[0] + a, (int64_t)b[1] + c, (int64_t)b[2] + e) == st + e;
        nbad += !ok;
        pencil[g * P * P + a * P + c] = ok ? st : -1;
      }
    if (nbad) atomicAdd(bad, nbad);
  }
}

}  // namespace cpmdev

namespace cpm {

namespace {

// Device buffers of one construction, freed on every exit.
struct DevBufs {
  std::vector<void*> ptrs;
  ~DevBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T> cudaError_t get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = (T*)q;
    return e;
  }
  void release(void* p) {           // hand a buffer over to the caller
    for (auto& q : ptrs)
      if (q == p) q = nullptr;
  }
};

cpm_status cuda_error(cudaError_t e, const char* where) {
  set_error(std::string("cpm_build_band_device: ") + where + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CPM_ERR_OOM : CPM_ERR_CUDA;
}
#define DCK(call)                                                   \
  do {                                                              \
    cudaError_t e__ = (call);                                       \
    if (e__ != cudaSuccess) return cuda_error(e__, #call);          \
  } while (0)

unsigned grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

// pos[i] = exclusive prefix count of flag over [0, n); returns the total
cpm_status compact_positions(DevBufs& d, const uint8_t* flag, int64_t n, int32_t* pos, int64_t* total,
                             cudaStream_t s) {
  const int64_t nb = (n + cpmdev::CCH - 1) / cpmdev::CCH;
  int64_t* sums;
  DCK(d.get(&sums, nb + 1));
  cpmdev::chunk_sum_kernel<<<(unsigned)nb, cpmdev::CT, 0, s>>>(flag, n, sums);
  cpmdev::scan_sums_kernel<<<1, cpmdev::CT, 0, s>>>(sums, nb);
  cpmdev::positions_kernel<<<(unsigned)nb, cpmdev::CT, 0, s>>>(flag, n, sums, pos);
  DCK(cudaGetLastError());
  DCK(cudaMemcpyAsync(total, sums + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DCK(cudaStreamSynchronize(s));
  return CPM_OK;
}

template <typename T> cudaError_t download(std::vector<T>& h, const T* dptr, size_t count, cudaStream_t s) {
  h.resize(count);
  return count ? cudaMemcpyAsync(h.data(), dptr, sizeof(T) * count, cudaMemcpyDeviceToHost, s) : cudaSuccess;
}

}  // namespace

cpm_status build_band_device(const Surface& s, double h, int p, double lam_over_h, void* stream, Band& B) {
  cpm_status st = validate_surface(s, h, p);
  if (st != CPM_OK) return st;
  if (!(lam_over_h > 0.0)) lam_over_h = ((1.0033 * std::sqrt(3.0)) * (p + 1)) / 2.0;
  const double lam = lam_over_h * h;
  cudaStream_t cs = (cudaStream_t)stream;
  int dev = 0;
  DCK(cudaGetDevice(&dev));
  Surface S;
  double lo[3], hi[3];
  st = prepare_surface(s, h, S, lo, hi);
  if (st != CPM_OK) return st;
  const bool mesh = S.kind == CPM_TRIMESH;
  // the bounding box of the tube, as on the host
  int64_t imin[3], imax[3];
  for (int a = 0; a < 3; ++a) {
    imin[a] = (int64_t)std::floor((lo[a] - lam) / h) - 1;
    imax[a] = (int64_t)std::ceil((hi[a] + lam) / h) + 1;
  }
  cpmdev::BoxDim box{imin[0], imin[1], imin[2], imax[1] - imin[1] + 1, imax[2] - imin[2] + 1, 0};
  box.n = (imax[0] - imin[0] + 1) * box.nj * box.nk;
  if (box.n > (int64_t)2000000000) {
    set_error("cpm_build_band_device: bounding grid too large");
    return CPM_ERR_INVALID_ARG;
  }
  DevBufs d;
  cpmdev::Geo geo{};
  geo.kind = S.kind;
  geo.R = S.R;
  geo.r = S.r;
  uint8_t* near = nullptr;
  if (mesh) {
    const Mesh& M = S.mesh;
    std::vector<uint8_t> hnear;
    mesh_near_cells(M, lam, hnear);
    // bounding sphere of every triangle: FP32 centroid, radius = the largest vertex distance
    // from that centre (in FP64), rounded up to FP32 and grown by a relative 1e-6
    const int64_t nt = M.n_tris();
    std::vector<float> hsph(4 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
      const double* v[3] = {&M.V[3 * (int64_t)M.T[3 * t]], &M.V[3 * (int64_t)M.T[3 * t + 1]],
                            &M.V[3 * (int64_t)M.T[3 * t + 2]]};
      float c[3];
      for (int e = 0; e < 3; ++e) c[e] = (float)((v[0][e] + v[1][e] + v[2][e]) / 3.0);
      double r = 0.0;
      for (int q = 0; q < 3; ++q) {
        const double dx = v[q][0] - (double)c[0], dy = v[q][1] - (double)c[1], dz = v[q][2] - (double)c[2];
        r = std::max(r, std::sqrt((dx * dx + dy * dy) + dz * dz));
      }
      for (int e = 0; e < 3; ++e) hsph[4 * t + e] = c[e];
      hsph[4 * t + 3] = std::nextafter((float)(r * (1.0 + 1e-6)), std::numeric_limits<float>::infinity());
    }
    float4* sph;
    DCK(d.get(&sph, nt));
    DCK(cudaMemcpyAsync(sph, hsph.data(), 16 * (size_t)nt, cudaMemcpyHostToDevice, cs));
    double* V;
    int32_t *T, *ctri;
    int64_t* cstart;
    DCK(d.get(&V, M.V.size()));
    DCK(d.get(&T, M.T.size()));
    DCK(d.get(&cstart, M.cell_start.size()));
    DCK(d.get(&ctri, M.cell_tris.size()));
    DCK(d.get(&near, hnear.size()));
    DCK(cudaMemcpyAsync(V, M.V.data(), 8 * M.V.size(), cudaMemcpyHostToDevice, cs));
    DCK(cudaMemcpyAsync(T, M.T.data(), 4 * M.T.size(), cudaMemcpyHostToDevice, cs));
    DCK(cudaMemcpyAsync(cstart, M.cell_start.data(), 8 * M.cell_start.size(), cudaMemcpyHostToDevice, cs));
    if (!M.cell_tris.empty())
      DCK(cudaMemcpyAsync(ctri, M.cell_tris.data(), 4 * M.cell_tris.size(), cudaMemcpyHostToDevice, cs));
    DCK(cudaMemcpyAsync(near, hnear.data(), hnear.size(), cudaMemcpyHostToDevice, cs));
    DCK(cudaStreamSynchronize(cs));   // the host vectors go out of scope
    geo.m = cpmdev::DevMesh{V, T, cstart, ctri, sph, {M.org[0], M.org[1], M.org[2]}, M.cell,
                            {M.nc[0], M.nc[1], M.nc[2]}};
  }
  // tube test and compaction of the actives
  uint8_t* flag;
  double* cpd;
  int32_t *trid, *pos;
  DCK(d.get(&flag, box.n));
  DCK(d.get(&cpd, 3 * box.n));
  DCK(d.get(&trid, mesh ? box.n : 1));
  DCK(d.get(&pos, box.n));
  cpmdev::tube_kernel<<<grid_for(box.n, 256), 256, 0, cs>>>(geo, near, box, h, lam, flag, cpd, trid);
  DCK(cudaGetLastError());
  int64_t na = 0;
  st = compact_positions(d, flag, box.n, pos, &na, cs);
  if (st != CPM_OK) return st;
  if (na == 0) {
    set_error("cpm_build_band_device: empty band");
    return CPM_ERR_INVALID_ARG;
  }
  int32_t *aijk, *atri = nullptr;
  double* acp;
  DCK(d.get(&aijk, 3 * na));
  DCK(d.get(&acp, 3 * na));
  if (mesh) DCK(d.get(&atri, na));
  cpmdev::gather_actives_kernel<<<grid_for(box.n, 256), 256, 0, cs>>>(flag, pos, box, cpd, trid, aijk, acp, atri);
  DCK(cudaGetLastError());
  // index grid over the actives' box grown by 2
  int32_t* mm;
  DCK(d.get(&mm, 6));
  const int32_t init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
  DCK(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, cs));
  cpmdev::bbox_kernel<<<grid_for(na, 256), 256, 0, cs>>>(aijk, na, mm, mm + 3);
  int32_t hmm[6];
  DCK(cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, cs));
  DCK(cudaStreamSynchronize(cs));
  cpmdev::GridDim gd{};
  for (int a = 0; a < 3; ++a) {
    gd.lo[a] = hmm[a] - 2;
    gd.dims[a] = hmm[3 + a] - hmm[a] + 5;
  }
  const int64_t ncell = (int64_t)gd.dims[0] * gd.dims[1] * gd.dims[2];
  int32_t *grid, *gpos;
  uint8_t* mark;
  DCK(d.get(&grid, ncell));
  DCK(d.get(&mark, ncell));
  DCK(d.get(&gpos, ncell));
  DCK(cudaMemsetAsync(grid, 0xff, 4 * (size_t)ncell, cs));
  DCK(cudaMemsetAsync(mark, 0, (size_t)ncell, cs));
  cpmdev::grid_actives_kernel<<<grid_for(na, 256), 256, 0, cs>>>(aijk, na, gd, grid);
  cpmdev::ghost_mark_kernel<<<grid_for(na, 256), 256, 0, cs>>>(aijk, na, gd, grid, mark);
  DCK(cudaGetLastError());
  int64_t ng = 0;
  st = compact_positions(d, mark, ncell, gpos, &ng, cs);
  if (st != CPM_OK) return st;
  const int64_t N = na + ng;
  // all nodes: actives then ghosts
  int32_t *ijk, *tri = nullptr, *bad;
  double* cp;
  DCK(d.get(&ijk, 3 * N));
  DCK(d.get(&cp, 3 * N));
  if (mesh) DCK(d.get(&tri, N));
  DCK(d.get(&bad, 2));
  DCK(cudaMemsetAsync(bad, 0, 2 * sizeof(int), cs));
  DCK(cudaMemcpyAsync(ijk, aijk, 12 * (size_t)na, cudaMemcpyDeviceToDevice, cs));
  DCK(cudaMemcpyAsync(cp, acp, 24 * (size_t)na, cudaMemcpyDeviceToDevice, cs));
  if (mesh) DCK(cudaMemcpyAsync(tri, atri, 4 * (size_t)na, cudaMemcpyDeviceToDevice, cs));
  cpmdev::ghosts_kernel<<<grid_for(ncell, 256), 256, 0, cs>>>(geo, mark, gpos, gd, ncell, na, h, grid, ijk, cp, tri,
                                                              bad);
  int32_t* nbr;
  DCK(d.get(&nbr, 6 * na));
  cpmdev::nbr_kernel<<<grid_for(na, 256), 256, 0, cs>>>(ijk, na, gd, grid, nbr);
  const int P = p + 1;
  int32_t *base, *pencil;
  double* wts;
  DCK(d.get(&base, 3 * N));
  DCK(d.get(&wts, 3 * P * N));
  DCK(d.get(&pencil, (size_t)P * P * N));
  cpmdev::interp_kernel<<<grid_for(N, 128), 128, 0, cs>>>(cp, N, na, gd, grid, h, p, base, wts, pencil, bad + 1);
  DCK(cudaGetLastError());
  int hbad[2] = {0, 0};
  DCK(cudaMemcpyAsync(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, cs));
  DCK(cudaStreamSynchronize(cs));
  if (hbad[0]) {
    set_error("cpm_build_band_device: ghost node without closest point");
    return CPM_ERR_STENCIL;
  }
  if (hbad[1]) {
    set_error("cpm_build_band_device: an interpolation stencil leaves the active set (tube radius too small)");
    return CPM_ERR_STENCIL;
  }
  // the host copy of the band
  Band out;
  out.surf = std::move(S);
  out.h = h;
  out.lam = lam;
  out.p = p;
  out.n_active = na;
  out.n_ghost = ng;
  for (int a = 0; a < 3; ++a) {
    out.lo[a] = gd.lo[a];
    out.dims[a] = gd.dims[a];
  }
  DCK(download(out.ijk, ijk, 3 * (size_t)N, cs));
  DCK(download(out.cp, cp, 3 * (size_t)N, cs));
  if (mesh) DCK(download(out.tri, tri, (size_t)N, cs));
  DCK(download(out.nbr, nbr, 6 * (size_t)na, cs));
  DCK(download(out.base, base, 3 * (size_t)N, cs));
  DCK(download(out.wts, wts, 3 * (size_t)P * N, cs));
  DCK(download(out.pencil, pencil, (size_t)P * P * N, cs));
  DCK(download(out.grid, grid, (size_t)ncell, cs));
  // the operators' device copies stay resident: pencils, weights, neighbours, tensor weights
  double* wt2;
  DCK(d.get(&wt2, (size_t)(P * P + P) * N));
  DCK(cpmdev::launch_build_tensor_weights(wts, wt2, N, P, cs));
  DCK(cudaStreamSynchronize(cs));
  d.release(pencil);
  d.release(wts);
  d.release(nbr);
  d.release(wt2);
  out.d_pencil = pencil;
  out.d_wts = wts;
  out.d_nbr = nbr;
  out.d_wt2 = wt2;
  out.d_device = dev;
  B = std::move(out);
  return CPM_OK;
}

}  // namespace cpm
