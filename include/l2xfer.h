/*
 * l2xfer — L2-projection transfer between a structured Q1 fluid grid and an
 * unstructured P1 solid mesh, on one GB300 GPU (sm_103a).
 *
 * The method is the variational transfer of Sec. 2.3 ("Variational Transfer:
 * the L2-Projection Approach"):
 *
 *   B_ij = ∫ psi_j N_i           mixed coupling matrix (mortar integral),
 *   S_ij = ∫ phi_j N_i           multiplier matrix,
 *   w_s  = S^{-1} B v_f = T v_f  velocity transfer, one scalar component at a time,
 *   f_f  = s T^T f               force transfer by the transpose, s = L_ref/(rho_f U_ref^2),
 *
 * where N_i spans the space of Lagrange multipliers: either the P1 hat
 * functions themselves (N_i = phi_i, S = M_s, the solid mass matrix; the
 * "standard" L2-projection), or the dual basis biorthogonal to them, Eq.
 * (biorth) (the "pseudo" L2-projection; S is then diagonal).  The dual basis
 * is built element by element: on a simplex E the function dual to the hat
 * function of vertex a is (d+2) lambda_a - 1 (lambda_a the barycentric
 * coordinate), so ∫_E N_a lambda_b = delta_ab |E|/(d+1) and S = diag(∫ phi_i).
 *
 * assembled in the current configuration of the solid mesh by the four steps
 * given after the transfer operator: (I) overlap detection, (II) quadrature
 * points in the intersections, (III) local contributions, (IV) assembly.
 * phi_i is the P1 hat function of solid node i (Sec. 2.1, "Spatial
 * Discretization"); psi_j is the Q1 function of node j of one of the velocity
 * grids of the staggered fluid grid (Sec. 2.2, "Spatial Discretization").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers on the current CUDA device unless
 *   said otherwise; they are read or written on `stream` (a cudaStream_t, NULL =
 *   legacy default stream).  The caller owns them.  The library owns the memory
 *   behind an l2x_handle and releases it in l2x_destroy().
 * - Every call returns an l2x_status; nothing traps.  Kernels report errors
 *   through a device status word that the call reads after synchronising
 *   `stream`; l2x_last_error() gives a one-line description.
 * - A handle is not thread-safe and must not be used from two streams at once.
 * - One CUDA device per process: kernel attributes (shared-memory opt-ins) are
 *   set once, on the device of the first launch.  Run one process per GPU.
 * - Velocity grids: with staggered = 0 there is one nodal Q1 grid (nodes at
 *   origin + i*h) and one scalar component; with staggered = 1 there are `dim`
 *   grids, grid g having nodes at origin_g + i*h along axis g and at cell
 *   centres along the other axes (so ncell-1 Q1 cells there).  A fluid array of
 *   grid g has prod_k nnode_g[k] entries, node (i0,i1,i2) at i0 + nnode0*(i1 +
 *   nnode1*i2).
 * - Field precision follows l2x_opts.precision: double arrays for L2X_FP64,
 *   float arrays for L2X_MIXED.
 */
#ifndef L2XFER_H
#define L2XFER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum l2x_status {
    L2X_OK = 0,
    L2X_EINVAL = 1,         /* bad argument (null pointer, dim, sizes, options) */
    L2X_ENOMEM = 2,         /* device allocation failed */
    L2X_ECAPACITY = 3,      /* a fixed-capacity buffer overflowed */
    L2X_EOUTOFGRID = 4,     /* a solid element leaves the cells of a velocity grid */
    L2X_EDEGENERATE = 5,    /* a solid element has zero volume */
    L2X_ENOTCONVERGED = 6,  /* CG did not reach cg_rtol within cg_max_iter */
    L2X_ETIMEOUT = 7,       /* a bounded device wait gave up */
    L2X_ECUDA = 8,          /* CUDA runtime error */
    L2X_ENONFINITE = 9      /* NaN or Inf in an input field or coordinate */
} l2x_status;

enum { L2X_PATH_PLAIN = 0, L2X_PATH_FUSED = 1 };
enum { L2X_FP64 = 0, L2X_MIXED = 1 };
enum { L2X_FORCE_NODAL = 0, L2X_FORCE_DUAL = 1 };
enum { L2X_MAT_B0 = 0, L2X_MAT_B1 = 1, L2X_MAT_B2 = 2, L2X_MAT_M = 3 };
enum { L2X_MULT_STANDARD = 0, L2X_MULT_DUAL = 1 };

/* Phases timed by l2x_set_timing (indices of l2x_info.phase_ms). */
enum {
    L2X_PH_PAIRS = 0,      /* step (I): candidate boxes, counts, scan, pair list */
    L2X_PH_CLIP = 1,       /* steps (II)-(III): clipping + quadrature of every pair */
    L2X_PH_ROWS = 2,       /* step (IV): CSR assembly of B_g */
    L2X_PH_TRANSPOSE = 3,  /* B_g^T for the force transfer */
    L2X_PH_MASS = 4,       /* values of M_s */
    L2X_PH_SPMV_B = 5,     /* y = B_g u_f */
    L2X_PH_PCG = 6,        /* M_s^-1 by Jacobi-PCG */
    L2X_PH_SPMV_BT = 7,    /* f_f += s B_g^T z */
    L2X_NPHASE = 8
};

/* Base (pressure) grid: ncell[k] cells of width h[k] from origin[k], k < dim,
 * or a stretched (rectilinear) grid as the fluid solvers of Sec. 4 use: when
 * axis[0] is not NULL, axis[k] (k < dim) are HOST arrays of ncell[k] + 1 finite,
 * strictly increasing base-node coordinates, read during l2x_build_coupling
 * only (origin and h are then ignored).  The velocity grids of a staggered
 * stretched grid have the base nodes along their own axis and the midpoints
 * 0.5 * (x_i + x_{i+1}) of consecutive base nodes along the others.  Cells are
 * half-open [x_i, x_{i+1}); the candidate cells of an element along axis k are
 * those with x_{i+1} > lo and x_i < hi, found by comparisons only.  Set axis to
 * NULL for a uniform grid. */
typedef struct l2x_grid {
    int32_t dim;        /* 2 or 3 */
    int32_t staggered;  /* 0: one nodal Q1 grid; 1: dim staggered velocity grids */
    int32_t ncell[3];
    double origin[3];
    double h[3];
    const double* axis[3];
} l2x_grid;

/* P1 simplex mesh in its current configuration.  coords: n_nodes x dim,
 * row-major doubles; elems: n_elems x (dim+1) row-major int32 node indices.
 * Both are device pointers, read during the call only (the handle keeps a copy). */
typedef struct l2x_mesh {
    int32_t dim;
    int32_t reserved;
    int64_t n_nodes;
    int64_t n_elems;
    const double* coords;
    const int32_t* elems;
} l2x_mesh;

typedef struct l2x_opts {
    int32_t path;         /* L2X_PATH_PLAIN (reference GPU path) or L2X_PATH_FUSED */
    int32_t precision;    /* L2X_FP64 or L2X_MIXED (fused path only) */
    double cg_rtol;       /* relative residual target of the mass-matrix solve */
    int32_t cg_max_iter;
    int32_t force_mode;   /* L2X_FORCE_DUAL: f_f += s B^T S^-1 r; NODAL: f_f += s B^T f */
    double force_scale;   /* s = L_ref / (rho_f U_ref^2); 1 by default */
    int32_t multiplier;   /* L2X_MULT_STANDARD (S = M_s, solved by Jacobi-PCG) or
                             L2X_MULT_DUAL (dual basis of Eq. (biorth), S diagonal: no solve) */
    int32_t reserved;     /* 0 */
} l2x_opts;

typedef struct l2x_info {
    int32_t dim, n_grids, path, precision;
    int64_t n_nodes, n_elems;
    int64_t n_pairs[3];        /* candidate pairs per velocity grid */
    int64_t n_pairs_total;
    int64_t nnz_B[3];
    int64_t nnz_M;
    int64_t n_fluid[3];        /* nodes per velocity grid */
    int32_t nnode[3][3];       /* nodes per axis per velocity grid */
    int32_t cg_iters;          /* iterations of the last mass-matrix solve (max over components) */
    int32_t reserved;
    double cg_residual;        /* relative residual reached by the last solve (max over components) */
    double phase_ms[8];        /* device time per phase since l2x_set_timing(h, 1) (CUDA events) */
    int64_t phase_calls[8];    /* timed intervals per phase */
    int32_t clip_block;        /* pairs per thread block of the clip kernel (l2x_autotune) */
    int32_t pcg_rows_per_block;/* rows per thread block of the cooperative PCG (l2x_autotune) */
    int32_t multiplier;        /* L2X_MULT_STANDARD or L2X_MULT_DUAL */
    int32_t pcg_cluster;       /* > 0: the solve runs in one thread-block cluster of this many CTAs */
    double tuned_clip_ms;      /* l2x_autotune: time of the chosen clip launch (0 before tuning) */
    double tuned_solve_ms;     /* l2x_autotune: time of the chosen mass-matrix solve of all components */
    int32_t pcg_rows_per_block_step; /* rows per block of a captured step's combined solve (2G right-hand sides) */
    int32_t clip_chunk;        /* blocks' worth of pairs per work-queue fetch of the persistent clip kernel */
} l2x_info;

typedef struct l2x_coupling* l2x_handle;
typedef struct l2x_step_graph* l2x_graph;

/* Fills *opts with the defaults: fused path, FP64, cg_rtol 1e-13, 200 iterations,
 * DUAL force mode, scale 1, standard multipliers (S = M_s). */
void l2x_default_opts(l2x_opts* opts);

/* Steps (I)-(IV) of Sec. 2.3 plus the mass matrix: candidate (element, cell)
 * pairs from bounding boxes, exact clipping of every simplex against its cells,
 * quadrature of lambda_a * psi_b on the clipped polytopes, CSR assembly of B_g
 * (rows: solid nodes, columns: nodes of grid g) for every velocity grid and of
 * S (M_s, or its diagonal form diag(∫ phi_i) for the dual basis; the dual rows
 * of B are (d+2) times the lambda integrals minus their sum over the element's
 * vertices).  Synchronises `stream` (pair counts decide allocation sizes).
 * Errors: EINVAL (arguments), EOUTOFGRID, EDEGENERATE, ENONFINITE, ENOMEM, ECUDA.
 * On success *out owns all device storage of the coupling. */
l2x_status l2x_build_coupling(const l2x_grid* grid, const l2x_mesh* mesh, const l2x_opts* opts,
                              void* stream, l2x_handle* out);

/* Re-assembles B_g and M_s for new node positions (same n_nodes, same elements),
 * as needed when the solid moves (T lives on the current configuration). */
l2x_status l2x_update_geometry(l2x_handle h, const double* coords, void* stream);

/* Velocity transfer (Step 1 of the FSI algorithm, Sec. 3): for every velocity
 * grid g, u_s[g] = S^{-1} B_g u_f[g], by Jacobi-preconditioned CG for S = M_s
 * and by a division fused into the product with B_g for the dual basis.
 * u_f: n_grids device arrays of n_fluid[g] entries; u_s: n_grids arrays of
 * n_nodes entries (written).  Returns ENOTCONVERGED if cg_rtol was not met. */
l2x_status l2x_transfer_velocity(l2x_handle h, const void* const* u_f, void* const* u_s,
                                 void* stream);

/* Force transfer by the transpose (Step 4 of Sec. 3): for every grid g,
 *   DUAL : f_f[g] += s * B_g^T S^{-1} f_s[g]   (= s T_g^T f_s[g])
 *   NODAL: f_f[g] += s * B_g^T f_s[g]          (f_s: multiplier coefficients)
 * f_s: n_grids arrays of n_nodes entries; f_f: n_grids fluid arrays, accumulated. */
l2x_status l2x_transfer_force(l2x_handle h, const void* const* f_s, void* const* f_f,
                              void* stream);

/* Building blocks of the two transfers (used by the autograd binding):
 * y_s[g] = B_g x_f[g];  f_f[g] += scale * B_g^T z_s[g];  w_s[g] = S^{-1} y_s[g]. */
l2x_status l2x_apply_B(l2x_handle h, const void* const* x_f, void* const* y_s, void* stream);
l2x_status l2x_apply_BT(l2x_handle h, const void* const* z_s, void* const* f_f, double scale,
                        void* stream);
l2x_status l2x_solve_mass(l2x_handle h, const void* const* y_s, void* const* w_s, void* stream);

/* Adjoint of the force transfer (the backward of a differentiable force
 * transfer): for every grid g,
 *   DUAL : g_s[g] = s * m ⊙ S^{-1} B_g g_f[g]
 *   NODAL: g_s[g] = s * m ⊙ B_g g_f[g]
 * with s = force_scale and m the interface mask of l2x_set_force_mask (all
 * ones without one), so that <g_f, F f_s> = <g_s, f_s> for the force transfer
 * f_f += F f_s of l2x_transfer_force (Step 4 of Sec. 3 is the transpose of the
 * velocity transfer, and this is the transpose of Step 4).  g_f: n_grids fluid
 * arrays; g_s: n_grids arrays of n_nodes entries (written).  Synchronises
 * `stream` in the DUAL mode with S = M_s (CG status).  Errors as
 * l2x_transfer_velocity. */
l2x_status l2x_transfer_force_adjoint(l2x_handle h, const void* const* g_f, void* const* g_s, void* stream);

/* Interface restriction of the force input (Sec. 2's interface Gamma_fsi; in
 * the plate benchmark of Sec. 4 only the reaction forces of the top and bottom
 * edges are communicated).  mask: device array of n_nodes bytes, nonzero =
 * node on the interface; the library copies it (stream-ordered).  Afterwards
 * every force transfer (per call, enqueue-only, captured steps created later)
 * uses mask_i * f_s[g][i] in place of f_s[g][i], i.e. f_f += s T^T (mask ⊙ f_s)
 * (DUAL) or s B^T (mask ⊙ f_s) (NODAL).  NULL removes the restriction. */
l2x_status l2x_set_force_mask(l2x_handle h, const uint8_t* mask, void* stream);

/* Picard iterations on one assembled T (Sec. 3, "Fluid-Structure Interaction
 * algorithm": Steps 1 and 4 are repeated within a time step while Steps 2, 3
 * and 5, the caller's solid and fluid solvers, run in between).  The
 * enqueue-only forms below do not synchronise the host, so a whole Picard
 * iteration can be captured into the caller's own CUDA graph:
 *
 * l2x_transfer_velocity_async / l2x_transfer_force_async: the same results as
 * l2x_transfer_velocity / l2x_transfer_force (fused path only).  The mass-matrix
 * solve runs a fixed schedule: the FP64 PCG stops on cg_rtol inside the kernel;
 * the mixed form runs one FP32 solve and one FP64 residual correction.  A solve
 * that misses cg_rtol is recorded in the handle's device status.
 * l2x_sync_status: waits for `stream`, returns the recorded status of the
 * enqueued calls since the last check (ENOTCONVERGED, or an assembly error) and
 * clears it; l2x_query then reports the last solve's iterations and residual. */
l2x_status l2x_transfer_velocity_async(l2x_handle h, const void* const* u_f, void* const* u_s, void* stream);
l2x_status l2x_transfer_force_async(l2x_handle h, const void* const* f_s, void* const* f_f, void* stream);
l2x_status l2x_sync_status(l2x_handle h, void* stream);

/* Step 6 of Sec. 3, the convergence test of the Picard iteration, Eqs. (AC) and
 * (RC).  l2x_picard_norms reduces over the n_grids solid arrays f_new and f_prev
 * (n_nodes entries each, the precision's type) on the device:
 *   norms[0] = max_{g,i} |f_new[g][i] - f_prev[g][i]|,  norms[1] = max_{g,i} |f_new[g][i]|
 * into `norms` (2 device doubles, 8-byte aligned, written; NaN in an input
 * makes the norm NaN).  With copy != 0 it also sets f_prev = f_new in the same
 * pass (the arrays must not overlap).  Enqueue-only.
 * l2x_picard_converged reads norms (synchronising `stream`; host_norms, 2
 * doubles, may be NULL) and sets *converged = 1 when
 *   norms[0] < eps_abs  (AC)   or   norms[0] / f0_norm < eps_rel  (RC),
 * where f0_norm is the caller's norm of the force of the first Picard
 * iteration (for example its norms[1]); f0_norm <= 0 disables (RC). */
l2x_status l2x_picard_norms(l2x_handle h, const void* const* f_new, void* const* f_prev, int32_t copy,
                            double* norms, void* stream);
l2x_status l2x_picard_converged(const double* norms, double eps_abs, double eps_rel, double f0_norm,
                                int32_t* converged, double* host_norms, void* stream);

/* One time step as a CUDA graph (the batched moving-bodies pattern): a mesh made
 * of many bodies (disjoint node sets in one l2x_mesh) is re-assembled in its
 * current configuration and both transfers run, with no host synchronisation,
 * by one cudaGraphLaunch per step.  Each replay copies the node positions from
 * coords_src (device, n_nodes x dim, read at replay time), rebuilds B_g, B_g^T
 * and S, writes u_s = S^-1 B u_f and f_f (+)= s B^T (S^-1) f_s (zeroed first
 * if zero_force != 0); all pointers are fixed at creation.  Pair and entry
 * capacities are the current sizes times capacity_margin (>= 1), and the rows of
 * B^T cover the fluid nodes the mesh touches at creation, padded on every side
 * by capacity_margin - 1 times the touched extent (at least 2 nodes); a replay
 * that needs more, or whose mesh leaves that box, sets a flag and skips its
 * work, reported by l2x_graph_sync_status as L2X_ECAPACITY (create the graph
 * again).  Fused path only; `stream` must
 * not be the legacy default stream.  While a graph exists, use the handle only
 * through it: l2x_update_geometry or another l2x_graph_create on the handle may
 * move the buffers it uses, so afterwards l2x_graph_launch of the older graph
 * returns L2X_EINVAL (on the host; nothing is launched).  Destroy the graphs of a
 * handle before the handle.  l2x_graph_sync_status waits for the stream and
 * returns the status of the last replay (capacity, degenerate or out-of-grid
 * elements, CG). */
l2x_status l2x_graph_create(l2x_handle h, const double* coords_src, const void* const* u_f, void* const* u_s,
                            const void* const* f_s, void* const* f_f, double capacity_margin, int32_t zero_force,
                            void* stream, l2x_graph* out);
/* The same step with its inputs and outputs in HOST memory, for a caller whose
 * fluid solver runs on the host.  Arrays as for l2x_graph_create, in host
 * memory: coords_host (n_nodes x dim doubles), u_f_host[g] and f_f_host[g]
 * (the fluid nodes of grid g, x fastest), u_s_host[g] and f_s_host[g]
 * (n_nodes); field elements are float in the mixed precision form and double
 * otherwise.  Every replay copies the positions, f_s and, of u_f, the box of
 * fluid nodes that the rows of B_g^T cover (fixed here: the nodes the mesh
 * touches, padded by the capacity margin; B_g reads u_f only there) in, and u_s
 * and the box of f_f (B_g^T writes f_f only there) out.  zero_force != 0:
 * f_f_host = s B^T ...; its entries outside the box are set to zero here, once,
 * and no replay writes them again (the caller keeps them zero).  zero_force ==
 * 0: f_f_host += s B^T ...; the box is copied in, added to and copied back.
 * The copies are nodes of the graph: the inputs on a branch beside the
 * assembly (which needs only the positions), u_s on that branch beside the
 * force transfer, f_f at the end (one grid per stream); host arrays are read
 * and written at replay time and complete once the stream has passed the
 * launch (for instance after l2x_graph_sync_status).  Every host array must be
 * page-locked (cudaHostAlloc / cudaHostRegister), else L2X_EINVAL, and stay
 * allocated while the graph exists.  The graph owns the device copies of the
 * fields (freed by l2x_graph_destroy); L2X_ENOMEM if they do not fit.
 * Everything else as for l2x_graph_create, whose launch, status and destroy
 * calls serve this graph.  l2x_graph_io_bytes gives the bytes a replay copies
 * in and out (0 for a graph of device arrays). */
l2x_status l2x_graph_create_host(l2x_handle h, const double* coords_host, const void* const* u_f_host,
                                 void* const* u_s_host, const void* const* f_s_host, void* const* f_f_host,
                                 double capacity_margin, int32_t zero_force, void* stream, l2x_graph* out);
l2x_status l2x_graph_io_bytes(l2x_graph g, int64_t* h2d_bytes, int64_t* d2h_bytes);
l2x_status l2x_graph_launch(l2x_graph g, void* stream);
l2x_status l2x_graph_sync_status(l2x_graph g, void* stream);
l2x_status l2x_graph_destroy(l2x_graph g);

/* Sizes and solver statistics of a coupling (host struct). */
l2x_status l2x_query(l2x_handle h, l2x_info* info);

/* Copies of internal data for tests, into caller-owned device buffers sized from
 * l2x_query().  Pairs of grid g: element index and linear cell index (cell
 * (i0,i1,i2) of grid g at i0 + ncell0*(i1 + ncell1*i2)), element-major with
 * cells in z, y, x order.  Pair blocks (fused path only): blocks[p*(d+1)*2^d +
 * a*2^d + b] = ∫_{E∩C} lambda_a psi_b, corner b = bits (x, y, z); vols[p] =
 * |E∩C| (the lambda integrals, for either multiplier space).  CSR (which =
 * L2X_MAT_B0..B2 or L2X_MAT_M for S): row_ptr (n_rows+1, int64),
 * cols (int32, ascending within a row), vals (double). */
l2x_status l2x_export_pairs(l2x_handle h, int32_t grid, int32_t* elem, int32_t* cell, void* stream);
l2x_status l2x_export_pair_blocks(l2x_handle h, int32_t grid, double* blocks, double* vols,
                                  void* stream);
/* The same for the pairs of elements [e_first, e_first + n_elems) of grid g only
 * (contiguous in the element-major list).  *first_pair and *n_pairs (host) receive
 * the range; pass NULL arrays to query the range alone. */
l2x_status l2x_export_pair_range(l2x_handle h, int32_t grid, int64_t e_first, int64_t n_elems,
                                 int64_t* first_pair, int64_t* n_pairs, int32_t* elem, int32_t* cell,
                                 double* blocks, double* vols, void* stream);
l2x_status l2x_export_csr(l2x_handle h, int32_t which, int64_t* row_ptr, int32_t* cols,
                          double* vals, void* stream);

/* Picks work-chunk sizes for this coupling by timing candidates on it (CUDA
 * events, best of two after a warm-up run): pairs per block of the clip kernel
 * (64, 128, 256) and the chunk it takes per fetch from its work queue (1, 4 or
 * 16 blocks' worth of pairs: the clip kernel is a persistent launch of the CTAs
 * that fit on the SMs, which take chunks of the class-ordered pairs from a device
 * counter until none are left), and the form of the Jacobi-PCG: the grid-wide cooperative
 * kernel with 32 to 1024 rows per block, or, when the search direction fits,
 * one thread-block cluster of 8 or 16 CTAs holding it in distributed shared
 * memory.  The combined solve of a captured step (both transfers at once) gets
 * its own rows per block.  Call after a build; later builds, solves and
 * captured steps use the choice (reported in l2x_info).  Runs the clip kernel
 * and the solves a few times on the stream and synchronises it. */
l2x_status l2x_autotune(l2x_handle h, void* stream);

/* Sets the work shape l2x_autotune would pick: clip_block in {64, 128, 256},
 * pcg_rows_per_block in [1, 4096] (grid-wide PCG), pcg_cluster 0 (grid-wide)
 * or the CTAs of the single-cluster PCG (EINVAL if the system does not fit). */
l2x_status l2x_set_work_shape(l2x_handle h, int32_t clip_block, int32_t pcg_rows_per_block, int32_t pcg_cluster);

/* Sets the chunk of the clip kernel's work queue (see l2x_autotune): clip_chunk
 * blocks' worth of pairs per fetch, in [1, 1024], else EINVAL.  Applies to
 * builds and steps captured afterwards. */
l2x_status l2x_set_clip_chunk(l2x_handle h, int32_t clip_chunk);

/* Sets the rows per thread block of the combined solve of captured steps (the
 * 2G right-hand sides of both transfers), which l2x_autotune tunes on its own
 * and l2x_set_work_shape sets to pcg_rows_per_block.  [1, 4096], else EINVAL.
 * Applies to steps captured afterwards. */
l2x_status l2x_set_step_work_shape(l2x_handle h, int32_t pcg_rows_per_block_step);

/* Enables (1, also clears the totals) or disables (0) CUDA-event timing of the
 * phases listed above, recorded on the stream of each call; l2x_query resolves
 * the events (waiting for them). */
l2x_status l2x_set_timing(l2x_handle h, int32_t enable);

/* Number of kernels this library has launched in this process (all handles). */
int64_t l2x_kernel_launch_count(void);

/* Throughput probe of the FP64 (precision = L2X_FP64) or FP32 (L2X_MIXED)
 * fused multiply-add pipe, the measured denominator of the ALU roofline of the
 * clipping kernel.  No counterpart in the paper.  Enqueues one kernel of
 * n_blocks blocks of 256 threads; every thread runs `iters` iterations of 8
 * independent FMA chains, i.e. 2 * 8 * 256 * n_blocks * iters floating-point
 * operations, and writes one value into sink (device, n_blocks * 256 doubles
 * or floats, caller-owned).  Time it with events on `stream`.  Does not
 * synchronise.  Errors: EINVAL (arguments), ECUDA (launch). */
l2x_status l2x_fma_probe(int32_t precision, int32_t n_blocks, int32_t iters, void* sink, void* stream);

/* Test hook for the arithmetic helpers of the clipping kernel (no counterpart
 * in the paper): out[i] = op(a[i], b[i]) for i < n, device arrays of doubles,
 * enqueued on `stream`.  op 0: the kernel's quotient (reciprocal by two
 * Newton-Raphson steps from an FP32 seed, then a * r: within two ulps);
 * 1: CUDA's a / b; 2: the kernel's double -> float conversion by
 * integer instructions (round half away from zero, below 2^-126 to zero); 3:
 * CUDA's __double2float_rn; 4: the low float of the kernel's double-float split
 * (a - float(a)); 5: the kernel's float -> double conversion of
 * __double2float_rn(a); 6: the mixed precision form's quotient (an FP32
 * quotient and one FP64 correction: within about 2^-45 relative).  b is read by
 * ops 0, 1 and 6 only.  Errors: EINVAL, ECUDA. */
l2x_status l2x_fp_selftest(int32_t op, int64_t n, const double* a, const double* b, double* out, void* stream);

/* Test hook of the library's single-pass prefix sum (no counterpart in the
 * paper; the scan behind the pair offsets, the CSR row pointers and the B^T
 * row lists): out[0..n) = exclusive prefix sums of in[0..n) (device int64,
 * non-negative values), out[n] = total.  Each tile waits for its predecessors'
 * prefixes with at most spin_limit polls; with missing_first != 0 the first tile
 * is left out, so the second tile's wait runs out and the call returns
 * L2X_ETIMEOUT without hanging (the device stays usable).  Allocates and frees
 * its own workspace; synchronises `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
l2x_status l2x_scan_selftest(int64_t n, const int64_t* in, int64_t* out, int32_t missing_first, int64_t spin_limit,
                             void* stream);

/* Jacobi-preconditioned CG that allocates no device memory.
 *
 * No counterpart in the paper: this is a service for callers that cannot call
 * cudaMalloc (for example a process whose device memory is owned by an outer
 * framework's memory pool, or a solver loop that must not add allocation calls).
 * It solves A w_k = y_k, k < n_rhs, for a caller-supplied CSR matrix A (n x n,
 * symmetric positive definite with a non-zero diagonal, such as M_s exported by
 * l2x_export_csr): row_ptr (n+1, int64), cols (int32), vals (double), all device
 * pointers; y and w are arrays of n_rhs device pointers to n doubles (w written).
 * Stops when ||r_k|| <= rtol ||y_k|| for every k or after max_iter iterations.
 * *iters and *residual (host pointers, may be NULL) receive the iterations and
 * the largest relative residual.
 *
 * Its work vectors live in one fixed device array of L2X_NOALLOC_MAX_DOUBLES
 * doubles (about 6.3 MB) that every GPU holds from the moment the library's
 * module is loaded on it until the process exits; n and n * n_rhs must not exceed
 * L2X_NOALLOC_MAX_ENTRIES, larger problems return L2X_ECAPACITY.  Under lazy
 * module loading (CUDA's default) the module, and with it the array, is loaded
 * by the first call on a device, so a caller whose pool will reserve the device
 * memory should make one small warm-up call on each device first.  Every call
 * looks up the array's device address with the device current.  The call reads
 * the solver status back and synchronises `stream`, so it cannot be captured
 * into a CUDA graph: on a capturing stream it returns L2X_EINVAL.  All calls
 * share the array and the kernel initialises everything it reads; two calls whose
 * kernels overlap on the GPU (different streams or threads) race on it and give
 * wrong results.
 * Errors: EINVAL, ECAPACITY, ENOTCONVERGED, ECUDA (l2x_noalloc_last_error()). */
#define L2X_NOALLOC_MAX_ENTRIES 131072
#define L2X_NOALLOC_MAX_DOUBLES (6 * L2X_NOALLOC_MAX_ENTRIES + 1024 * 9 + 16)
l2x_status l2x_solve_mass_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* cols, const double* vals,
                                  int32_t n_rhs, const double* const* y, double* const* w, double rtol,
                                  int32_t max_iter, void* stream, int32_t* iters, double* residual);
const char* l2x_noalloc_last_error(void);

/* Releases every device allocation of the handle (stream-ordered on the stream
 * of the last call).  NULL is accepted. */
l2x_status l2x_destroy(l2x_handle h);

const char* l2x_status_string(l2x_status s);
/* Description of the most recent error on this host thread ("" if none). */
const char* l2x_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* L2XFER_H */
