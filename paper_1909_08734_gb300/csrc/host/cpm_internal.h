// Internal host-side structures of the CPM Schwarz library.
// Host code is compiled with -ffp-contract=off so that every set-membership decision
// (tube test, stencil bases, bisection order, argmins) is reproducible bit for bit.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../../include/cpm.h"

namespace cpm {

void set_error(const std::string& msg);

// Triangulated surface with a uniform bucket grid over the triangles' bounding boxes.
struct Mesh {
  std::vector<double> V;          // n_verts x 3
  std::vector<int32_t> T;         // n_tris x 3
  std::vector<double> fn;         // n_tris x 3 unit face normals
  double org[3] = {0, 0, 0}, cell = 0;
  int32_t nc[3] = {0, 0, 0};      // cells per axis
  std::vector<int64_t> cell_start;  // CSR over cells of triangle lists (ascending index)
  std::vector<int32_t> cell_tris;
  int64_t n_tris() const { return (int64_t)T.size() / 3; }
};

struct Surface {
  int kind;
  double R, r;
  Mesh mesh;                      // CPM_TRIMESH only
};

// Closest point (Sec. 2.1). Returns false where CP is undefined (sphere centre, torus axis
// or ring circle); such points are never band nodes.
bool closest_point(const Surface& s, const double x[3], double y[3]);
// Unit surface normal at a surface point y (analytic surfaces).
void surface_normal(const Surface& s, const double y[3], double n[3]);
// Mesh: validates the triangles, computes face normals and the bucket grid (cell size s).
cpm_status mesh_prepare(Mesh& m, double cell);
// Exact closest point over all triangles (ties: lowest index) if it lies within dmax of x;
// returns the triangle index, or -1 if every triangle is farther than dmax.
int32_t mesh_closest_point(const Mesh& m, const double x[3], double dmax, double y[3],
                           std::vector<int32_t>& stamp, int32_t& qid);

// 1-D barycentric Lagrange weights on nodes 0..p at offset t (Sec. 2.1, second form).
void bary_weights(double t, int p, double* w);
// Stencil base (lowest node) and the 1-D weights of interpolation at point y.
void point_weights(const double y[3], double h, int p, int32_t base[3], double* wx,
                   double* wy, double* wz);

struct Band {
  Surface surf;
  double h = 0, lam = 0;
  int p = 0;
  int64_t n_active = 0, n_ghost = 0;
  std::vector<int32_t> ijk;      // (N) x 3
  std::vector<double> cp;        // (N) x 3
  std::vector<int32_t> nbr;      // N_A x 6
  std::vector<int32_t> base;     // N x 3 stencil bases of CP(x)
  std::vector<double> wts;       // N x 3 x (p+1) 1-D weights (x, then y, then z)
  std::vector<int32_t> pencil;   // N x (p+1)^2 first active index of each z-pencil
  std::vector<int32_t> tri;      // N triangle holding CP(x) (meshes only)
  int32_t lo[3] = {0, 0, 0}, dims[3] = {0, 0, 0};
  std::vector<int32_t> grid;     // dense index grid, -1 = no node
  int64_t n_nodes() const { return n_active + n_ghost; }
  int32_t lookup(int64_t i, int64_t j, int64_t k) const {
    int64_t a = i - lo[0], b = j - lo[1], c = k - lo[2];
    if (a < 0 || b < 0 || c < 0 || a >= dims[0] || b >= dims[1] || c >= dims[2]) return -1;
    return grid[(a * dims[1] + b) * dims[2] + c];
  }
  int P() const { return p + 1; }
  // Device copies (uploaded lazily by oras_setup, freed with the band).
  mutable void* d_pencil = nullptr;
  mutable void* d_wts = nullptr;
  mutable void* d_nbr = nullptr;
  mutable void* d_wt2 = nullptr;   // (P^2 + P) x N tensor weights wy_b wz_c and wx_a (device)
  mutable int d_device = -1;
};

// Unit surface normal at CP(x) of node g (analytic, or the face normal of its triangle).
void node_normal(const Band& B, int64_t g, double n[3]);

struct SubSets {
  std::vector<int32_t> own, sigma, last, ghost, bc_a, bc_g;
  std::vector<int32_t> bc_gen;    // generator (last-layer node) of CP_{S_j} per BC node
  std::vector<int32_t> bc_nearx;  // 1 if the BC node is near a cross point
};

struct Partition {
  const Band* band = nullptr;
  int n_sub = 0, n_overlap = 0;
  std::vector<int32_t> labels;
  std::vector<int32_t> cross;
  std::vector<SubSets> subs;
};

// Local operator of one subdomain as summed COO triplets.
struct LocalCOO {
  int64_t n = 0;          // local unknowns
  int64_t n_sigma = 0;    // the first n_sigma are Sigma_j
  std::vector<int32_t> row, col;
  std::vector<double> val;
};

// Reverse Cuthill-McKee order of the pattern of A_j + A_j^T: perm[new] = old (deterministic).
void rcm_order(const LocalCOO& L, std::vector<int32_t>& perm);
// Tile envelope of the LU factors of a local operator with T tiles per dimension: per padded
// row its first and last nonzero tile columns, and per step s one past the last position a
// row with first <= s can take (the panel's row range).
void envelope(const LocalCOO& L, int T, std::vector<int32_t>& first, std::vector<int32_t>& last,
              std::vector<int32_t>& pend);

cpm_status build_band(const Surface& s, double h, int p, double lam_over_h, Band& out);
// Pieces of the band construction shared with the device build: argument checks, the working
// surface (mesh bucket grid) and its bounding box, and the mesh cells near a triangle.
cpm_status validate_surface(const Surface& s, double h, int p);
cpm_status prepare_surface(const Surface& s, double h, Surface& S, double lo[3], double hi[3]);
void mesh_near_cells(const Mesh& M, double lam, std::vector<uint8_t>& near);
// The same band as build_band, built on the current CUDA device (closest points, tube test,
// canonical order, ghosts, neighbour table and interpolation data); the host arrays are
// filled from the device and the device copies stay resident for the operators.
cpm_status build_band_device(const Surface& s, double h, int p, double lam_over_h, void* stream, Band& out);
// Algorithmic band: the smallest node set containing the grid nodes within h of the surface
// and the interpolation stencils of CP(x) for its nodes and their 6-neighbours.
cpm_status build_band_algorithmic(const Surface& s, double h, int p, Band& out);
// Frees the band's device copies (defined with the CUDA code).
void band_release_device(Band& b);
// split: 0 recursive coordinate bisection, 1 recursive graph bisection
cpm_status build_partition(const Band& band, int n_sub, const int64_t* weights, int n_overlap,
                           int align_passes, Partition& out, int split = 0);
// The same sets from caller-supplied labels (every label in [0, n_sub), no subdomain empty).
cpm_status build_partition_from_labels(const Band& band, int n_sub, const int32_t* labels, int n_overlap,
                                       Partition& out);
// Local operator of subdomain j, duplicates summed; sorted_rows: entries of a row in column
// order (otherwise in first-touch order; the values are the same either way).
cpm_status build_local_coo(const Band& band, const Partition& part, double c, int transmission,
                           double alpha, double alpha_x, int j, LocalCOO& out,
                           bool sorted_rows = true);

}  // namespace cpm

// Opaque handle types of the C ABI.
struct cpm_band {
  cpm::Band b;
};
struct cpm_part {
  cpm::Partition p;
};
