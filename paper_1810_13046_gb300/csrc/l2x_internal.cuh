// Internal declarations shared by the l2xfer translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "l2xfer.h"

namespace l2x {

constexpr int kMaxGrids = 3;

// Device status word, written with atomics by kernels, read by the host after
// the call's stream is synchronised.
enum : int32_t {
    FLAG_OUTOFGRID = 1,
    FLAG_DEGENERATE = 2,
    FLAG_CAPACITY = 4,
    FLAG_NONFINITE = 8,
    FLAG_NOTCONVERGED = 16,
    FLAG_TIMEOUT = 32,
};

// Flags after which the remaining kernels of a captured step skip their work
// (the step's result is reported invalid by l2x_graph_sync_status).
constexpr int32_t kAbortFlags = FLAG_OUTOFGRID | FLAG_DEGENERATE | FLAG_NONFINITE | FLAG_CAPACITY;

struct DevStatus {
    int32_t flags;
    int32_t bad_elem;     // first element that raised OUTOFGRID / DEGENERATE (min)
    int32_t cg_iters;
    int32_t pad;
    double cg_residual;
};

// One Q1 velocity grid.
struct SubGrid {
    int32_t ncell[3];   // Q1 cells per axis (1 on unused axes)
    int32_t nnode[3];   // ncell + 1 (1 on unused axes)
    double origin[3];
    double h[3];        // uniform grids; 1 on a stretched grid (gradients in physical units)
    double inv_h[3];
    // stretched (rectilinear) grid: per used axis the nnode node coordinates and
    // the ncell inverse cell widths (device arrays); null on a uniform grid
    const double* ax[3];
    const double* inv_w[3];
    // uniform axis whose h is a power of two: (x - o) / h == (x - o) * inv_h exactly,
    // so the candidate index rule multiplies instead of dividing
    int32_t pow2[3];
};

// Per-element candidate box on one grid: lowest cell index and extent per axis.
struct ElemBox {
    int32_t lo[3];
    int32_t ext;        // packed extents: ex | ey << 10 | ez << 20 (each <= 1023)
};

__host__ __device__ inline int box_ext(const ElemBox& b, int k) { return (b.ext >> (10 * k)) & 1023; }

// CSR matrix (int64 row pointers, int32 columns).
struct Csr {
    int64_t n_rows = 0;
    int64_t nnz = 0;
    int64_t* ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    float* val32 = nullptr;  // mixed-precision copy
};

// Transposed coupling matrix restricted to the box of fluid nodes the mesh touches.
// Rows are indexed by box position; `list` holds the non-empty rows (n_list[0]
// of them, a device value) so that sorting and the force gather skip the rest.
struct CsrT {
    int32_t lo[3] = {0, 0, 0};   // first node of the box per axis
    int32_t n[3] = {1, 1, 1};    // box nodes per axis
    int64_t n_rows = 0;          // n[0]*n[1]*n[2]
    int64_t* ptr = nullptr;
    int32_t* col = nullptr;      // solid node
    double* val = nullptr;
    float* val32 = nullptr;
    int32_t* list = nullptr;     // non-empty rows (capacity list_cap)
    int64_t* n_list = nullptr;   // device: number of non-empty rows
    int64_t list_cap = 0;
    int32_t* long_rows = nullptr;  // rows longer than a warp sorts (capacity long_cap)
    int32_t* n_long = nullptr;     // device: their number
    int64_t long_cap = 0;
};

// Counts kernel launches of the library (l2x_api.cu).
void count_launch();

// ---------------------------------------------------------------- launchers
// pairs (l2x_pairs.cu)
// Per element and grid: candidate box, pair count (counts) and node count of the
// box (nbox, for the element-local matrices); volume, gradients, orientation.
void launch_elem_boxes(int dim, int n_grids, const SubGrid* sg_host, int64_t m, const double* X,
                       const int32_t* E, ElemBox* boxes, int64_t* counts, int64_t* nbox, int32_t* node_box,
                       double* elem_vol, double* elem_grad, int8_t* elem_flag, DevStatus* st, cudaStream_t s);
void launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s, DevStatus* st = nullptr);
void launch_scan_i64_test(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s, DevStatus* st,
                          int missing_first, long long spin_limit);
size_t scan_tmp_bytes(int64_t n);
void launch_emit_pairs(int dim, int n_grids, const SubGrid* sg_host, int64_t m, const ElemBox* boxes,
                       const int64_t* offsets, int32_t* pair_elem, int32_t* pair_cell, int64_t cap, DevStatus* st,
                       cudaStream_t s);
void launch_reset_status(DevStatus* st, cudaStream_t s);
// FLAG_CAPACITY if *total > cap (device value); kernels after it skip their work
// Box of fluid nodes (inclusive bounds per axis) that a captured step's B^T rows cover, per grid.
struct NodeBoxSet {
    int32_t lo[kMaxGrids][3];
    int32_t hi[kMaxGrids][3];
};
// node_box (6 per grid: min x,y,z then max x,y,z) set to empty.
void launch_node_box_reset(int32_t* node_box, int n_grids, cudaStream_t s);
// FLAG_CAPACITY if a grid's touched nodes leave lim.
void launch_check_node_box(const int32_t* node_box, const NodeBoxSet& lim, int n_grids, DevStatus* st,
                           cudaStream_t s);
void launch_check_capacity(const int64_t* total, int64_t cap, DevStatus* st, cudaStream_t s);

// clipping + quadrature (l2x_clip.cu).  Pair blocks are stored pair-major:
// blocks[p * (d+1) * 2^d + a * 2^d + b].
// Fused: pairs of all grids are first bucketed by scheduling class (similar
// control flow per warp, launch_pair_classes), then clipped in bucket order.
// Sizes are read on the device from offsets[G * m] (bounded by n_cap); n_launch
// is the number of threads launched (exact pair count, or the capacity when the
// count is not known on the host).  keys: uint8 per pair; perm: int32 per pair;
// buckets: 2 * kClasses int32.
constexpr int kClasses = 129;  // scheduling classes of the pairs (pair_class)
void launch_pair_classes(int dim, int G, const SubGrid* sg, int64_t m, const int64_t* offsets, int64_t n_launch,
                         int64_t n_cap, const double* X, const int32_t* E, const int32_t* pair_elem,
                         const int32_t* pair_cell, uint8_t* keys, int32_t* perm, int32_t* buckets, cudaStream_t s);
void launch_clip_fused(int dim, int precision, int G, const SubGrid* sg, int64_t m, const int64_t* offsets,
                       int64_t n_launch, int64_t n_cap, const double* X, const int32_t* E, const double* elem_grad,
                       const int8_t* elem_flag, const int32_t* pair_elem, const int32_t* pair_cell,
                       const int32_t* perm, double* blocks, double* vols, DevStatus* st, cudaStream_t s,
                       int block, int chunk, unsigned long long* work);
void launch_clip_plain(int dim, const SubGrid& sg, const double* X, const int32_t* E, int64_t p_begin,
                       int64_t p_end, const int32_t* pair_elem, const int32_t* pair_cell, double* blocks,
                       double* vols, DevStatus* st, cudaStream_t s);
// plain assembly: atomicAdd of every pair block into the pre-built CSR of B_g
void launch_scatter_plain(int dim, const SubGrid& sg, const int32_t* E, int64_t p_begin, int64_t p_end,
                          const int32_t* pair_elem, const int32_t* pair_cell, const double* blocks,
                          const double* vols, const Csr& B, int dual, cudaStream_t s);

// assembly (l2x_assemble.cu)
// node -> (element, local vertex) adjacency, entries e*4 + a sorted per node.
// adj_ptr must hold n_nodes + 1 entries; cursor n_nodes int32 (scratch).
void launch_node_adjacency(int dim, int64_t n_nodes, int64_t m, const int32_t* E, int64_t* adj_ptr,
                           int32_t* adj, int32_t* cursor, void* scan_tmp, cudaStream_t s);
// Element-local matrices of grid g: for every element and every node of its
// candidate node box, the sums over the element's pairs of block[a][b] at that
// node (loc_val: d+1 planes of loc_cap entries, one per element vertex a) and
// whether a pair of positive volume touches it (loc_flag).  loc_off_g: offsets
// of the elements' node boxes.
void launch_elem_local(int dim, int64_t m, const ElemBox* boxes_g, const int64_t* offsets_g,
                       const int64_t* loc_off_g, int64_t loc_cap, const double* blocks, const double* vols,
                       double* loc_val, uint8_t* loc_flag, int dual, DevStatus* st, cudaStream_t s);
// A row of B_g as the counting pass of launch_b_rows leaves it for the emitting
// pass: the union box of the incident element boxes (lower corner, extents
// nx | ny << 8 | nz << 16, 0 = not kept), its touched nodes as a bit mask and
// the sums at the touched nodes (box order, x fastest).
constexpr int kRowKeep = 64;  // union-box nodes of a kept row
struct RowCache {
    int32_t lo[3];
    int32_t dims;
    uint32_t hit[kRowKeep / 32];
    double val[kRowKeep];
};
// One grid's matrix for launch_b_rows: its element boxes and local offsets (the
// slots of grid g), its row counts (pass 0) or row pointers, columns and values
// (passes 1, 2), its kept rows (n_nodes of them) and the node counts of its
// first two axes.
struct RowsGrid {
    const ElemBox* boxes = nullptr;
    const int64_t* loc_off = nullptr;
    int64_t* row_count = nullptr;
    const int64_t* row_ptr = nullptr;
    int32_t* cols = nullptr;
    double* vals = nullptr;
    RowCache* cache = nullptr;
    int32_t nnode0 = 1, nnode1 = 1;
};
// Row-wise assembly of the n_grids matrices B_g from the element-local matrices,
// in one launch.  pass 0: row_count[i] = nonzeros of row i (and the row kept in
// the grid's cache when its union box has at most kRowKeep nodes); pass 1: cols
// + vals; pass 2: cols only, vals zeroed (the plain path adds them with atomics).
// Passes 1 and 2 emit kept rows from the cache, so they follow a pass 0 of the
// same element-local matrices.
void launch_b_rows(int pass, int dim, int n_grids, const RowsGrid* grids, int64_t n_nodes, const int64_t* adj_ptr,
                   const int32_t* adj, const double* loc_val, int64_t loc_cap, const uint8_t* loc_flag,
                   DevStatus* st, cudaStream_t s);
// P1 mass matrix structure (pass 0 counts, pass 1 columns) and values.
void launch_mass_structure(int pass, int dim, int64_t n_nodes, const int32_t* E, const int64_t* adj_ptr,
                           const int32_t* adj, int64_t* row_count, const int64_t* row_ptr, int32_t* cols,
                           DevStatus* st, cudaStream_t s);
void launch_mass_values(int dim, int64_t n_nodes, const int32_t* E, const int64_t* adj_ptr,
                        const int32_t* adj, const double* elem_vol, const int64_t* row_ptr,
                        const int32_t* cols, double* vals, double* diag_inv, cudaStream_t s);
// S of the dual multiplier basis: diagonal CSR (row i holds column i) with
// S_ii = sum over the elements around i of |E|/(d+1), and its inverse.
void launch_lumped_mass(int dim, int64_t n_nodes, const int64_t* adj_ptr, const int32_t* adj,
                        const double* elem_vol, int64_t* row_ptr, int32_t* cols, double* vals, double* diag_inv,
                        cudaStream_t s);
// B_g^T over the box of touched fluid nodes.
void launch_transpose_count(const Csr& B, const SubGrid& sg, const CsrT& T, int64_t* cnt, const DevStatus* st,
                            cudaStream_t s);
void launch_transpose_fill(const Csr& B, const SubGrid& sg, const CsrT& T, int32_t* cursor, const DevStatus* st,
                           cudaStream_t s);
void launch_transpose_sort(const CsrT& T, const DevStatus* st, cudaStream_t s);
// Non-empty rows of B_g^T from the row counts (before they are scanned):
// flags (int64, n_rows + 1) is scratch; fills T.list and *T.n_list.
void launch_transpose_list(const CsrT& T, const int64_t* counts, int64_t* flags, void* scan_tmp,
                           const DevStatus* st, cudaStream_t s);
void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s);

// apply (l2x_apply.cu)
// y[g] = B_g x[g] (n_rows = solid nodes).  Fused: 8 lanes per row, all grids in
// one launch; plain: one thread per row, FP64 only.
void launch_spmv_B(int path, int precision, int n_grids, const Csr* B, const void* const* x,
                   void* const* y, const DevStatus* st, cudaStream_t s, const double* row_scale = nullptr);
// Step 6 of the FSI algorithm: norms[0] = max |f_new - f_prev|, norms[1] =
// max |f_new| over the G components of n entries (device doubles); f_prev =
// f_new in the same pass when copy != 0.
void launch_picard_norms(int precision, int64_t n, int G, const void* const* f_new, void* const* f_prev, int copy,
                         double* norms, cudaStream_t s);
// out_k = f_k where mask != 0, else 0 (k < nr).
void launch_mask_copy(int precision, int64_t n, int nr, const uint8_t* mask, const void* const* f, void* const* out,
                      const DevStatus* st, cudaStream_t s);
// w_k = y_k / S_ii for a diagonal S (dinv = 1/S_ii), k < nr; vectors in the
// precision's type, the product taken in FP64.
void launch_scale_mask(int precision, int64_t n, int nr, const uint8_t* mask, double scale, void* const* v,
                       const DevStatus* st, cudaStream_t s);
void launch_diag_solve(int precision, int64_t n, int nr, const double* dinv, const void* const* y,
                       void* const* w, const DevStatus* st, cudaStream_t s);
// f[g] += scale * B_g^T z[g].  Fused: gather over the rows of B_g^T (no atomics);
// plain: scatter with atomics from the rows of B_g.
void launch_spmv_BT(int path, int precision, int n_grids, const Csr* B, const CsrT* T,
                    const SubGrid* sg, const void* const* z, void* const* f, double scale,
                    const DevStatus* st, cudaStream_t s);
// Jacobi-preconditioned CG on M for n_rhs right-hand sides (FP64, or FP32 with
// compensated dot products and FP64 residual refinement in mixed mode).
struct PcgResult {
    int iters = 0;
    double residual = 0.0;
    bool converged = false;
};
// The same without any host synchronisation (capturable in a CUDA graph): FP64
// runs the cooperative PCG once; mixed runs the FP32 PCG and one FP64 residual
// refinement.  Convergence is reported through the device status word.
void solve_mass_pcg_async(int precision, const Csr& M, const double* diag_inv, const float* diag_inv32, int n_rhs,
                          const void* const* y, void* const* w, double rtol, int max_iter, void* ws, DevStatus* st,
                          cudaStream_t s, int rows_per_block = 64, int cluster = 0);
l2x_status solve_mass_pcg(int path, int precision, const Csr& M, const double* diag_inv,
                          const float* diag_inv32, int n_rhs, const void* const* y, void* const* w,
                          double rtol, int max_iter, void* ws, DevStatus* st, DevStatus* st_host,
                          cudaStream_t s, PcgResult* res, int rows_per_block = 64, int cluster = 0);
size_t pcg_ws_bytes(int64_t n, int n_rhs, int max_blocks);
int pcg_max_blocks();
// Single-cluster PCG (cluster > 0 in the solves above: one cluster of that many
// CTAs holds the search direction in distributed shared memory).  prepare sets
// the kernel attributes once (call outside stream capture); usable tells
// whether a system of n rows and nr right-hand sides fits and can launch.
void pcg_cluster_prepare();
bool pcg_cluster_usable(int precision, int64_t n, int nr, int cluster);

}  // namespace l2x
