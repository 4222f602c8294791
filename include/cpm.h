/*
 * cpm.h — C ABI of the GB300 RAS/ORAS closest-point-method solver.
 *
 * Method: May, Haynes & Ruuth, "Schwarz solvers and preconditioners for the closest point
 * method" (arXiv:1909.08734).  The library solves (c - Lap_S) u = f on a surface S through
 * the stabilised CPM discretisation (Sec. 2.1, Eq. impLapBel) with right-preconditioned
 * flexible GMRES, the preconditioner being restricted additive Schwarz with Dirichlet
 * (RAS, Eq. simpleRAS / Eq. algRAS) or Robin (ORAS, Sec. 5.2, Eq. robfo) transmission
 * conditions, including the cross-point modification (Sec. 5.2.2).
 *
 * Conventions for every call:
 *  - Every call returns cpm_status; no exception, abort or exit crosses the ABI.
 *    cpm_last_error() returns a thread-local message for the last failing call.
 *  - Handles (cpm_band, cpm_partition, oras_precond) are opaque and library-owned; free
 *    them with the matching *_destroy.  A handle is not thread-safe; distinct handles are.
 *  - Vector arguments named *_dev are caller-owned DEVICE memory (FP64, contiguous, in
 *    canonical band order: active node g = 0..N_A-1, right-hand sides as the slow
 *    dimension).  The library never frees them.  Host arrays returned by *_info / getters
 *    stay valid until the owning handle is destroyed.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Setup calls (cpm_build_band, cpm_partition) are host-only and never touch a GPU
 *    (cpm_build_band_device is the device variant of cpm_build_band).
 *    oras_setup synchronises its stream before returning.  cpm_op_apply and oras_apply
 *    are asynchronous on the stream.  cpm_gmres_solve synchronises once per restart cycle.
 */
#ifndef CPM_H
#define CPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CPM_OK = 0,
  CPM_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported option            */
  CPM_ERR_OOM = 2,           /* host or device allocation failed                      */
  CPM_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in cpm_last_error) */
  CPM_ERR_SINGULAR = 4,      /* zero pivot in a local LU (subdomain in the message)   */
  CPM_ERR_NOT_CONVERGED = 5, /* GMRES hit max_it before the tolerance                 */
  CPM_ERR_BREAKDOWN = 6,     /* GMRES basis vector of norm 0 with a large residual    */
  CPM_ERR_NAN = 7,           /* NaN or Inf in a norm                                  */
  CPM_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up                    */
  CPM_ERR_BUDGET = 9,        /* request exceeds a memory budget                       */
  CPM_ERR_STENCIL = 10       /* an interpolation / FD stencil leaves its node set     */
} cpm_status;

/* surface kinds */
enum { CPM_SPHERE = 0, CPM_TORUS = 1, CPM_TRIMESH = 2 };
/* transmission conditions (oras_setup) */
enum {
  CPM_RAS = 0,      /* Dirichlet: A_j = R_j A R_j^T on Sigma_j (Eq. simpleRAS)              */
  CPM_ORAS = 1,     /* Robin, every local unknown gets a 7-point row (reading R1)           */
  CPM_ORAS_R3 = 2   /* Robin, boundary unknowns get (c+6/h^2) w - (6/h^2) T w (reading R3)  */
};
/* precision of the local factors and local solves; CPM_SETUP_SIMT_LU may be or-ed into the
 * precision argument of oras_setup to run the LU trailing updates on the CUDA cores instead
 * of the tensor cores (a reference path for validating the tensor-core update) */
enum { CPM_FP64 = 0, CPM_FP32 = 1, CPM_BF16 = 2, CPM_SETUP_SIMT_LU = 0x100 };
/* node-set selectors for cpm_partition_set */
enum { CPM_SET_OWN = 0, CPM_SET_SIGMA = 1, CPM_SET_LAST = 2, CPM_SET_GHOST = 3,
       CPM_SET_BC_A = 4, CPM_SET_BC_G = 5, CPM_SET_BC_GEN = 6, CPM_SET_BC_NEARX = 7 };

/* Surface (Sec. 2.1).  CPM_SPHERE: radius R at the origin.  CPM_TORUS: about the z axis,
 * major radius R, minor radius r.  CPM_TRIMESH: a closed triangulated surface given by
 * verts (host, n_verts x 3 doubles) and tris (host, n_tris x 3 vertex indices, any winding);
 * CP_S(x) is the exact closest point over all triangles (ties: lowest triangle index) and
 * the surface normal at a closest point is the unit face normal of its triangle.  The mesh
 * arrays are copied by cpm_build_band; R and r are ignored for meshes, the mesh fields for
 * analytic surfaces. */
typedef struct {
  int kind;
  double R;
  double r;
  const double* verts;
  int64_t n_verts;
  const int32_t* tris;
  int64_t n_tris;
} cpm_surface;

typedef struct cpm_band cpm_band;
typedef struct cpm_part cpm_part;
typedef struct oras_precond oras_precond;

typedef struct {
  int64_t n_active;       /* N_A */
  int64_t n_ghost;        /* N_G */
  int p;                  /* interpolation degree */
  double h;               /* grid spacing */
  double lambda;          /* tube radius actually used */
  const int32_t* ijk;     /* host, (N_A+N_G) x 3 integer grid coordinates, node x = ijk*h */
  const double* cp;       /* host, (N_A+N_G) x 3 closest points CP_S(x) */
  const int32_t* nbr;     /* host, N_A x 6 node indices of (-x,+x,-y,+y,-z,+z) neighbours */
  const int32_t* base;    /* host, (N_A+N_G) x 3 lowest interpolation-stencil node of CP(x) */
  const int32_t* pencil;  /* host, (N_A+N_G) x (p+1)^2 active index of the first node of each
                             z-pencil (a,b) of the stencil, a slowest; the pencil is p+1
                             consecutive actives */
  const double* weights;  /* host, (N_A+N_G) x 3 x (p+1) barycentric weights at CP(x): x axis,
                             then y, then z */
  const int32_t* tri;     /* host, (N_A+N_G) triangle holding CP(x) (CPM_TRIMESH), else NULL */
} cpm_band_info;

/* Band construction (Sec. 2.1, tube-radius construction).
 * Active nodes: grid nodes x = (i,j,k)h with ||x - CP_S(x)|| <= lambda, lambda =
 * lambda_over_h * h; lambda_over_h <= 0 selects ((1.0033*sqrt(3))*(p+1))/2.  Ghost nodes:
 * 6-neighbours of actives that are not active.  Canonical order: actives lexicographic in
 * (i,j,k), k fastest, then ghosts in the same order.  Also computes each node's
 * interpolation stencil base and 1-D barycentric weights at CP_S(x) (degree p in {2,3}).
 * Errors: INVALID_ARG (h <= 0, p not 2 or 3, unknown surface, a mesh without triangles, a
 * vertex index out of range or a degenerate triangle), STENCIL (an interpolation stencil of
 * some node leaves the active set: lambda too small), OOM.  Host only. */
cpm_status cpm_build_band(const cpm_surface* surface, double h, int p, double lambda_over_h,
                          cpm_band** out);
/* The band of cpm_build_band, built on the current CUDA device (no counterpart in the paper,
 * whose global meshing is serial, Sec. 6.6): closest points and the tube test of every grid node
 * of the bounding box, order-preserving compactions for the canonical order and the ghosts, the
 * neighbour table, stencil bases, 1-D weights and z-pencil starts, each a device kernel.  The
 * result equals cpm_build_band's bit for bit (the device arithmetic follows the host's
 * operations in the same order, without contraction); the host arrays are filled from the
 * device, and the device copies the operators use stay resident (oras_setup on the same device
 * does not upload them again).  stream: cudaStream_t as void* (NULL = legacy default stream);
 * the call synchronises it.  Errors: as cpm_build_band, and CUDA / OOM from the device. */
cpm_status cpm_build_band_device(const cpm_surface* surface, double h, int p, double lambda_over_h,
                                 void* stream, cpm_band** out);
/* Algorithmic band (Sec. 2.1: the active nodes are all nodes used for interpolation; the
 * paper takes this construction for triangulated surfaces and cites its algorithm).
 * Reading: Sigma_A is the smallest node set that contains the grid nodes within h of the
 * surface and the (p+1)^3 interpolation stencil of CP(x) for every node x of Sigma_A and
 * every 6-neighbour x of Sigma_A; ghosts, order and the per-node data are as for
 * cpm_build_band (lambda is reported as 0).  It is a subset of the default tube band.
 * Errors: as cpm_build_band; STENCIL if the closure reaches a point without a closest
 * point.  Host only. */
cpm_status cpm_build_band_algorithmic(const cpm_surface* surface, double h, int p, cpm_band** out);
cpm_status cpm_band_info_get(const cpm_band* band, cpm_band_info* out);
void cpm_band_destroy(cpm_band* band);

/* Partition and overlapping node sets (Sec. 3.1 split, Sec. 4.1 overlap and boundary sets,
 * Sec. 4.2 effective boundary, Sec. 5.2.2 cross points).
 * Disjoint labels by recursive coordinate bisection of the actives' closest points with
 * integer leaf weights (leaf_weights: n_sub host int64, NULL = equal).  Sigma_j = actives
 * within n_overlap steps in the active 6-neighbour graph.  Builds Sigma_j^G, Sigma_j^BC
 * (active part and the Robin ghost layer), Lambda_j, the nearest Lambda_j point of every
 * boundary node (ties: lowest generator index) and the cross-point marks (boundary nodes
 * within 2*n_overlap*h of a node with neighbours in >= 2 other subdomains).
 * align_passes (0..64) interface-alignment passes (Sec. 3.2) follow the split: an active
 * node with an active 6-neighbour of another label moves to the label of the grid node
 * nearest to its closest point (floor(CP/h + 0.5) per axis), all moves of a pass decided on
 * the labels before it; the paper uses p + 1 passes.
 * Errors: INVALID_ARG (n_sub < 1, n_overlap < 0, a leaf weight <= 0, a subdomain left
 * empty, align_passes outside 0..64), OOM.  Host only. */
cpm_status cpm_partition(const cpm_band* band, int n_sub, const int64_t* leaf_weights,
                         int n_overlap, int align_passes, cpm_part** out);
/* As cpm_partition, with the disjoint split by recursive graph bisection of the active
 * 6-neighbour graph (the nearest-neighbour graph the paper partitions, Sec. 3.1) instead of
 * coordinates: a part is ordered by breadth-first search (neighbours in neighbour-table
 * order) from a pseudo-peripheral node, the last node reached by a search from the part's
 * lowest index, with unreached components appended from their lowest index; the left half
 * takes the first floor(n * W_left / W) nodes.  Same leaf weights, overlap, alignment passes,
 * sets and errors as cpm_partition.  Host only. */
cpm_status cpm_partition_graph(const cpm_band* band, int n_sub, const int64_t* leaf_weights,
                               int n_overlap, int align_passes, cpm_part** out);
/* Labels of the N_A actives (host, int32, valid until destroy). */
cpm_status cpm_partition_labels(const cpm_part* part, const int32_t** labels);
/* One node set of subdomain j (CPM_SET_*), as a sorted host int32 array of global node
 * indices (BC_GEN: generator of CP_{S_j} for each BC node, BC_A then BC_G order; BC_NEARX:
 * 1 if that BC node uses alpha_x). */
cpm_status cpm_partition_set(const cpm_part* part, int j, int which, const int32_t** data,
                             int64_t* len);
cpm_status cpm_partition_cross_points(const cpm_part* part, const int32_t** data,
                                      int64_t* len);
/* Partition from caller-supplied labels (the paper partitions with a graph partitioner,
 * Sec. 3.1; any labelling can be brought in): labels[g] in [0, n_sub) for every active node g
 * (host, N_A entries, copied).  The overlap, boundary sets, generators and cross points follow
 * from the labels exactly as in cpm_partition (Sec. 4.1, Sec. 4.2, Sec. 5.2.2).
 * Errors: INVALID_ARG (label outside [0, n_sub), empty subdomain), STENCIL, OOM. */
cpm_status cpm_partition_from_labels(const cpm_band* band, int n_sub, const int32_t* labels,
                                     int n_overlap, cpm_part** out);
/* Checkpoint of a partition (no counterpart in the paper): cpm_partition_save writes the
 * labels with n_sub, N_O and a fingerprint of the band (N_A, N_A + N_G, h, p and a 64-bit
 * FNV-1a hash of every node's integer grid coordinates) to the file at path (binary,
 * little-endian); cpm_partition_load rebuilds the partition on a band with the same
 * fingerprint through cpm_partition_from_labels, so the sets come out identical.
 * Errors: INVALID_ARG (file cannot be opened, written or read, not a partition file, other
 * band), STENCIL, OOM. */
cpm_status cpm_partition_save(const cpm_part* part, const char* path);
cpm_status cpm_partition_load(const cpm_band* band, const char* path, cpm_part** out);
void cpm_partition_destroy(cpm_part* part);

/* Local operator of subdomain j in coordinate form (host only, no GPU).  Local unknowns are
 * Sigma_j (global order) and, for ORAS, Sigma_j^{BC,A} (global order).  RAS: A_j = R_j A
 * R_j^T (Eq. simpleRAS).  ORAS: Eq. localOP with Robin extension rows at the boundary nodes
 * (Eq. robfo; alpha_x near cross points).  Call with rows == NULL to get *nnz and *n; then
 * with arrays of *nnz entries (row, col, value), duplicates already summed. */
cpm_status cpm_local_coo(const cpm_band* band, const cpm_part* part, double c,
                         int transmission, double alpha, double alpha_x, int j, int64_t* n,
                         int64_t* nnz, int32_t* rows, int32_t* cols, double* vals);

/* Order and tile envelope of local operator j as oras_setup factors it (host only, no GPU).
 * Any symmetric permutation of the local unknowns leaves the local solves of Eq. algRAS
 * unchanged up to rounding; oras_setup uses perm[new] = old, the reverse Cuthill-McKee order
 * of the pattern of A_j + A_j^T (deterministic).  For the reordered matrix, padded to 64 T
 * rows (T = ceil(n / 64), identity on the padding): first[r] / last[r] = the first / last
 * nonzero 64-column tile of row r (64 T entries each); pend[s] (s < T) = one past the last row
 * position that a row with first <= s can occupy at step s of an LU with partial pivoting
 * (at least 64 (s + 1)): the rows the panel of step s must cover.  Call with perm == NULL to
 * get *n and *T; then with arrays of n, 64 T, 64 T and T entries (caller-owned host memory).
 * Errors: INVALID_ARG, STENCIL, OOM. */
cpm_status cpm_local_order(const cpm_band* band, const cpm_part* part, double c, int transmission,
                           double alpha, double alpha_x, int j, int64_t* n, int* T, int32_t* perm,
                           int32_t* first, int32_t* last, int32_t* pend);

/* Preconditioner setup (Sec. 5 local operators; "local operators" phase of Sec. 6.6):
 * uploads the band to the device, orders every local matrix's unknowns (cpm_local_order),
 * assembles it tile-major on the GPU, factors all of them with partial pivoting in batched
 * launches over the tiles of their envelope and keeps the factors resident.  CPM_FP64: FP64 throughout.  CPM_FP32: FP32 factors, trailing
 * updates on the tensor cores with split-tf32 operands (FP32 accuracy).  CPM_BF16: trailing
 * updates with bf16 operands and FP32 accumulation, factors stored in BF16 for the solves.
 * Synchronises the stream.
 * Errors: INVALID_ARG, STENCIL, SINGULAR (zero pivot), OOM, CUDA. */
cpm_status oras_setup(const cpm_band* band, const cpm_part* part, double c,
                      int transmission, double alpha, double alpha_x, int precision,
                      void* stream, oras_precond** out);

typedef struct {
  int n_sub;
  int64_t n_active;
  int64_t n_nodes;            /* N_A + N_G */
  int precision;
  int transmission;
  int64_t max_n;              /* largest local size n_j */
  int64_t sum_n;              /* sum of n_j */
  int64_t sum_n2;             /* sum of n_j^2 (entries of the dense local matrices) */
  int64_t sum_sigma;          /* sum of |Sigma_j| (restrict reads) */
  int64_t factor_bytes;       /* device bytes of the resident factors */
  int64_t device_bytes;       /* all device bytes held by the handle */
  double setup_ms_assemble;   /* device time of the assembly launch(es) */
  double setup_ms_factor;     /* device time of the batched LU launches */
  int64_t kernel_launches;    /* library kernels launched by this handle so far (setup
                                 excluded; graph replays count every kernel node) */
  int solve_ctas_per_sm;      /* current schedule of the batched solve (see oras_tune) */
  int solve_kseg;
  int solve_prefetch;
  int solve_stagger;
  int64_t peak_device_bytes;  /* largest device_bytes reached so far (setup included) */
  int64_t tile_rows;          /* 64-row tile rows over all subdomains (sum of T_j) */
  int64_t solve_offdiag_tiles;/* off-diagonal 64 x 64 factor tiles one solve streams: the
                                 tile envelope of L and U (local unknowns in reverse
                                 Cuthill-McKee order); tiles outside it are exactly zero */
} oras_info;
cpm_status oras_info_get(const oras_precond* pc, oras_info* out);
/* Device-memory plan of an oras_setup call, computed on the host without touching a GPU
 * (admission control of the serving loop).  No counterpart in the paper.
 *   setup_peak_bytes : upper bound of the device bytes held during oras_setup (band copies,
 *                      assembly buffers, factor work tiles, diagonal-block inverses);
 *   resident_bytes   : upper bound of the bytes held afterwards by the handle once it has
 *                      run cpm_gmres_solve with this restart length and cpm_op_apply /
 *                      oras_apply with up to nrhs right-hand sides (any solve schedule);
 *   factor_bytes     : exact bytes of the resident factors;
 *   vector_bytes     : bytes of nrhs right-hand sides and solutions (f, u: 2 nrhs N_A 8),
 *                      caller-owned, reported for budgeting.
 * Bounds include a per-allocation rounding allowance.  Errors: INVALID_ARG. */
typedef struct {
  int64_t setup_peak_bytes;
  int64_t resident_bytes;
  int64_t factor_bytes;
  int64_t vector_bytes;
  int64_t sum_n2;
  int max_tiles;            /* largest number of 64-row tiles per dimension */
} oras_plan_info;
cpm_status oras_plan(const cpm_band* band, const cpm_part* part, int transmission, int precision,
                     int restart, int nrhs, oras_plan_info* out);
/* Schedule knobs of the batched local solve (oras_apply and the solves inside
 * cpm_gmres_solve).  They change speed only, never results beyond rounding order:
 *   CPM_TUNE_SOLVE_CTAS_PER_SM  persistent CTAs per SM (1 .. shared-memory limit)
 *   CPM_TUNE_SOLVE_KSEG         off-diagonal 64x64 tiles per work item; longer tile rows
 *                               are split into partial items (1 .. 1023; 1023 = no split)
 *   CPM_TUNE_SOLVE_PREFETCH     1: a CTA holds its next work item and streams it early
 *   CPM_TUNE_SOLVE_STAGGER      1: both sweeps in one queue, odd subdomains offset by half
 *                               a sweep (overlaps sweep starts and tails across subdomains)
 * Not thread-safe with concurrent calls on the same handle; invalidates the handle's
 * captured iteration graph (recaptured on the next solve).  Errors: INVALID_ARG, OOM, CUDA. */
enum { CPM_TUNE_SOLVE_CTAS_PER_SM = 0, CPM_TUNE_SOLVE_KSEG = 1, CPM_TUNE_SOLVE_PREFETCH = 2,
       CPM_TUNE_SOLVE_STAGGER = 3 };
cpm_status oras_tune(oras_precond* pc, int knob, int value);
/* Project autotuner: times the batched solve on this handle's factors for a small grid of
 * (CTAs per SM, split length, prefetch, stagger) candidates with CUDA events on `stream` and keeps
 * the fastest.  Synchronises the stream.  The chosen values are in oras_info. */
cpm_status oras_autotune(oras_precond* pc, void* stream);

/* Local sizes n_j (host array of n_sub int64 written by the call). */
cpm_status oras_local_sizes(const oras_precond* pc, int64_t* n_out);

/* y = A x (Eq. impLapBel with A = cI - Lap_S^h), FP64, matrix-free over the band:
 * v_k = sum (wx_a wy_b wz_c) x[stencil(k)] for every band node k, then
 * y_i = (c + 6/h^2) x_i - (1/h^2) sum_{6 neighbours} v_k.  x_dev, y_dev: nrhs x N_A.
 * Asynchronous on stream.  Errors: INVALID_ARG, CUDA. */
cpm_status cpm_op_apply(const oras_precond* pc, const double* x_dev, double* y_dev, int nrhs,
                        void* stream);

/* Largest band (N_A + N_G nodes) that cpm_op_apply_noalloc accepts: its scratch is a fixed
 * 8 MB array (2^20 FP64 values) that every GPU loading this library reserves until exit. */
#define CPM_NOALLOC_MAX_NODES (1 << 20)

/* y = A x exactly as cpm_op_apply computes it, but without allocating any device memory.
 * The paper has no counterpart: this exists for callers that cannot call cudaMalloc —
 * code whose device memory is owned by someone else's allocator (a framework's caching
 * pool, an embedded runtime with a fixed budget), or a latency-critical loop where an
 * allocation, which may synchronise the whole device, is not acceptable.
 * The caller supplies every input and output as device memory: the band's z-pencil starts
 * (int32, N x (p+1)^2), 1-D weights (FP64, N x 3 x (p+1)) and neighbour table (int32,
 * N_A x 6) in the layouts cpm_band_info returns, x_dev and y_dev (FP64, N_A).  N = n_nodes.
 * The extension values live in a library-owned static device array; its device address is
 * looked up (cudaGetSymbolAddress) by the first call on each device, so make that first
 * call before any stream capture.  All calls share the array and each call rewrites every
 * entry it reads, so calls may follow one another freely, but calls that overlap on the GPU
 * (different streams, or different host threads) race on it.  One right-hand side per call.
 * Asynchronous on stream.  Errors: INVALID_ARG (NULL pointer, p not 2 or 3, n_nodes <
 * n_active, h <= 0), BUDGET (n_nodes > CPM_NOALLOC_MAX_NODES), CUDA.  Calls no cudaMalloc,
 * cudaFree or allocating library routine. */
cpm_status cpm_op_apply_noalloc(const int32_t* pencil_dev, const double* weights_dev,
                                const int32_t* nbr_dev, int64_t n_active, int64_t n_nodes, int p,
                                double c, double h, const double* x_dev, double* y_dev,
                                void* stream);

/* z = M^{-1} r (Eq. algRAS): restrict r to every Sigma_j (zero on boundary unknowns),
 * solve with the resident LU factors, write each disjoint set's values to z (restricted
 * partition of unity).  FP64 in and out; the solves run in the factor precision.
 * Asynchronous on stream.  Errors: INVALID_ARG, CUDA; device-side wait timeouts are
 * reported by oras_check_status / cpm_gmres_solve. */
cpm_status oras_apply(const oras_precond* pc, const double* r_dev, double* z_dev, int nrhs,
                      void* stream);
/* Synchronises the stream and reports device-side errors latched by earlier launches
 * (TIMEOUT from a bounded wait), clearing them. */
cpm_status oras_check_status(const oras_precond* pc, void* stream);

typedef struct {
  int restart;     /* m, default 50 */
  double tol;      /* relative residual target ||f - A u|| <= tol ||f|| */
  int max_it;      /* total inner iterations */
  int use_graph;   /* 1: replay one captured iteration as a CUDA graph */
  int zero_guess;  /* 1: u starts at 0; 0: u_dev holds the initial guess */
} cpm_gmres_opts;

typedef struct {
  int iterations;
  double relres;   /* true relative residual at exit */
  int status;      /* cpm_status for this right-hand side */
} cpm_gmres_result;

/* Right-preconditioned flexible GMRES(m) with classical Gram-Schmidt applied twice, Givens
 * rotations, FP64 Arnoldi (Sec. 2.2: (O)RAS embedded in GMRES).  Solves A u = f for each of
 * nrhs right-hand sides; results[] has nrhs entries.  Returns CPM_OK only if every
 * right-hand side converged, else the first failing status. */
cpm_status cpm_gmres_solve(const oras_precond* pc, const double* f_dev, double* u_dev, int nrhs,
                           const cpm_gmres_opts* opts, cpm_gmres_result* results, void* stream);

/* (O)RAS as a stationary iterative solver (Sec. 2.2, Eq. algRAS): u_0 = 0, r_0 = f, then
 *     u_{k+1} = u_k + M^{-1} r_k ,   r_{k+1} = f - A u_{k+1}
 * until ||r_{k+1}||_2 <= tol ||f||_2.  Update, residual and norms are FP64; M^{-1} uses the
 * factor precision chosen at oras_setup.  f_dev, u_dev: caller-owned device vectors of nrhs x
 * N_A doubles (canonical band order, rhs slowest); u_dev is overwritten.  results[] has nrhs
 * entries: iterations = preconditioner applications, relres = the true relative residual at
 * exit, status = CPM_OK, CPM_ERR_NOT_CONVERGED (max_it reached), CPM_ERR_NAN or
 * CPM_ERR_TIMEOUT.  A zero right-hand side returns u = 0 after 0 iterations.  Synchronises
 * the stream once per iteration to test convergence.  Returns CPM_OK only if every
 * right-hand side converged, else the first failing status. */
cpm_status oras_stationary_solve(const oras_precond* pc, const double* f_dev, double* u_dev, int nrhs,
                                 double tol, int max_it, cpm_gmres_result* results, void* stream);

/* y = a x + b y on the device (b == 0: y = a x and y is not read), n doubles, asynchronous on
 * the stream.  A utility for drivers above the solver (for example a backward-Euler chain
 * whose next right-hand side is u_n / dt); no counterpart in the paper.  Errors:
 * INVALID_ARG (n < 0, NULL pointers with n > 0), CUDA. */
cpm_status cpm_vec_axpby(int64_t n, double a, const double* x_dev, double b, double* y_dev, void* stream);

/* Failure-detection check of the bounded device waits; no counterpart in the paper.  Launches
 * one kernel in which a thread waits on an mbarrier phase that nothing completes and on a
 * device flag that nothing sets, each bounded by limit_s seconds (0 < limit_s <= 10); the
 * expired waits latch the timeout bit in pc's device status word, as an expired wait inside
 * the solve or factorisation kernels does, and the kernel returns normally (no fault, the
 * context stays usable).  Synchronises.  Returns CPM_ERR_TIMEOUT when both waits expired
 * (the expected outcome; oras_check_status then reports and clears it), CPM_OK if a wait
 * completed, INVALID_ARG or CUDA otherwise. */
cpm_status cpm_selftest_bounded_wait(oras_precond* pc, double limit_s, void* stream);

/* Failure-detection check of the FGMRES breakdown report; no counterpart in the paper.  Makes
 * pc's operator the zero matrix (both coefficients of the stabilised operator set to 0, so
 * cpm_op_apply, cpm_gmres_solve and oras_stationary_solve then apply A x = 0 exactly for
 * finite x; the preconditioner is unchanged) and drops the captured iteration graphs.  A
 * solve with a nonzero right-hand side then meets A z_0 = 0 in its first Arnoldi step: the
 * Hessenberg matrix is singular with the residual still at ||f||, and cpm_gmres_solve reports
 * CPM_ERR_BREAKDOWN with u unchanged.  Irreversible for this handle (destroy it afterwards).
 * Synchronises the current device.  Errors: INVALID_ARG (null handle), CUDA. */
cpm_status cpm_selftest_zero_operator(oras_precond* pc);

/* Failure-detection check of the zero-pivot report; no counterpart in the paper.  Runs the
 * set-up of oras_setup with the same arguments, but after the local matrices are assembled
 * on the device, local column 0 of subdomain `subdomain` is set to zero in every row (as if
 * that local matrix were singular).  The factorisation then meets a zero pivot; the call
 * returns CPM_ERR_SINGULAR with cpm_last_error naming the lowest singular subdomain (the
 * expected outcome), frees everything it allocated and returns no handle.  Synchronises.
 * Errors: INVALID_ARG (as oras_setup, or subdomain out of range), OOM, CUDA. */
cpm_status oras_setup_selftest_singular(const cpm_band* band, const cpm_part* part, double c, int transmission,
                                        double alpha, double alpha_x, int precision, int subdomain, void* stream);

/* FP64 fused multiply-add probe on the current device (the denominator of the FP64-ALU
 * roofline fractions this library reports); no counterpart in the paper.  Throughput: `blocks`
 * blocks of `threads` threads, each thread advancing `chains` (1, 2, 4 or 8) independent
 * chains x <- x a + b for `iters` steps; *tflop_s = 2 threads blocks chains iters / (kernel
 * time), timed with CUDA events after one warm-up launch.  Latency: one thread advancing one
 * chain for `iters` steps; *cycles_per_fma = clock64 cycles per dependent step.  Either
 * output pointer may be NULL to skip that probe.  Allocates and frees 64 KB of device memory;
 * synchronises.  Errors: INVALID_ARG (blocks, threads or iters < 1, threads > 1024, chains not
 * in {1, 2, 4, 8}), CUDA. */
cpm_status cpm_probe_fp64(int blocks, int threads, int chains, int iters, double* tflop_s, double* cycles_per_fma);

void oras_destroy(oras_precond* pc);

const char* cpm_status_string(cpm_status s);
const char* cpm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CPM_H */
