// C-ABI entry points of l2xfer: handle management and the orchestration of the
// assembly (steps I-IV of Sec. 2.3) and of the two transfers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <memory>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "l2x_internal.cuh"

using namespace l2x;

namespace l2x {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace l2x

struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
};

struct l2x_coupling {
    int dim = 0, n_grids = 0;
    int64_t n_nodes = 0, n_elems = 0;
    l2x_grid grid{};
    l2x_opts opts{};
    SubGrid sg[kMaxGrids]{};
    double* grid_ax[kMaxGrids][3]{};   // stretched grids: node coordinates per velocity grid and axis
    double* grid_iw[kMaxGrids][3]{};   // and inverse cell widths
    cudaStream_t stream = nullptr;
    // own copies of the mesh
    double* X = nullptr;
    int32_t* E = nullptr;
    // topology
    int64_t* adj_ptr = nullptr;
    int32_t* adj = nullptr;
    int32_t* cursor = nullptr;
    // per element
    double* elem_vol = nullptr;
    double* elem_grad = nullptr;     // per element: barycentric gradients in cell-local coordinates
    int8_t* elem_flag = nullptr;     // 1 positive, 0 negative orientation, -1 degenerate
    ElemBox* boxes = nullptr;
    int64_t* counts = nullptr;
    int64_t* offsets = nullptr;      // n_grids*m + 1
    int64_t* nbox = nullptr;         // nodes of each element's candidate box, per grid (n_grids*m)
    int64_t* loc_off = nullptr;      // offsets of the element-local matrices (n_grids*m + 1)
    double* loc_val = nullptr;       // element-local matrices, (d+1) values per box node
    uint8_t* loc_flag = nullptr;     // box node touched by a pair of positive volume
    int64_t loc_cap = 0;
    int32_t* node_box = nullptr;     // n_grids * 6
    int64_t pair_begin[kMaxGrids + 1]{};
    // pairs
    int64_t n_pairs = 0, pair_cap = 0;
    int32_t* pair_elem = nullptr;
    int32_t* pair_cell = nullptr;
    double* blocks = nullptr;
    double* vols = nullptr;
    uint8_t* pair_key = nullptr;     // scheduling class per pair (fused path)
    int32_t* pair_perm = nullptr;    // pairs in class order (fused path)
    int32_t* buckets = nullptr;      // class counts and cursors
    // matrices
    Csr B[kMaxGrids];
    int64_t B_cap[kMaxGrids]{};
    CsrT T[kMaxGrids];
    int64_t T_cap[kMaxGrids]{}, T_rows_cap[kMaxGrids]{};
    Csr M;
    double* M_dinv = nullptr;
    float* M_dinv32 = nullptr;
    // scratch
    void* scan_tmp = nullptr;
    size_t scan_tmp_cap = 0;
    int64_t* row_count = nullptr;    // kMaxGrids * (n_nodes + 1): row counts per grid
    RowCache* row_cache = nullptr;   // n_grids * n_nodes: rows of B_g kept between the two row passes
    int32_t* tcursor = nullptr;      // fill cursors of the B^T rows
    int64_t tcursor_cap = 0;
    int64_t* tflags = nullptr;       // non-empty-row flags of B^T (scan scratch)
    int64_t tflags_cap = 0;
    void* pcg_ws = nullptr;
    void* vec_tmp = nullptr;         // n_grids * n_nodes doubles
    void* vec_tmp2 = nullptr;        // n_grids * n_nodes doubles (force side of a captured step)
    cudaStream_t aux_stream = nullptr;  // second branch of captured steps (values of S)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // bumped by every call that may move the buffers a captured step uses
    // (l2x_update_geometry, l2x_graph_create); a graph launches only while it
    // holds the current value
    uint64_t graph_gen = 0;
    // captured steps: B_g^T of grid g >= 1 is formed on a branch of its own, with
    // its own scratch (grid 0 uses the main stream and tcursor / tflags / scan_tmp)
    cudaStream_t t_stream[kMaxGrids]{};
    cudaEvent_t ev_tfork = nullptr, ev_tjoin[kMaxGrids]{};
    int32_t* t_cursor[kMaxGrids]{};
    int64_t* t_flags[kMaxGrids]{};
    void* t_scan[kMaxGrids]{};
    int64_t t_rows_cap[kMaxGrids]{};
    void* vec_mask = nullptr;        // n_grids * n_nodes doubles: the masked force input
    // captured steps with host buffers: the branch that copies the transfer inputs
    // in beside the assembly and the solid velocities out beside the force transfer
    cudaStream_t io_stream = nullptr;
    cudaEvent_t ev_io_fork = nullptr, ev_io_in = nullptr, ev_io_us = nullptr, ev_io_out = nullptr;
    uint8_t* fmask = nullptr;        // interface mask of the force input (n_nodes), when has_fmask
    bool has_fmask = false;
    DevStatus* st = nullptr;
    DevStatus* st_host = nullptr;    // pinned
    // work-chunk sizes (l2x_autotune)
    int clip_block = 128;            // threads (= pairs) per block of the clip kernel
    int clip_chunk = 4;              // blocks' worth of pairs per work-queue fetch of the clip kernel
    unsigned long long* clip_work = nullptr;  // work-queue counter of the clip kernel
    int pcg_rpb = 64;                // rows per block of the cooperative PCG
    int pcg_clu = 0;                 // > 0: single-cluster PCG with this many CTAs
    int pcg_rpb_step = 64;           // rows per block of a captured step's combined (2G right-hand sides) solve
    double tuned_clip_ms = 0.0, tuned_solve_ms = 0.0;
    // last solve
    int cg_iters = 0;
    double cg_residual = 0.0;
    // phase timing
    bool timing = false;
    std::vector<PhaseRec> pending;
    std::vector<cudaEvent_t> event_pool;
    double phase_ms[L2X_NPHASE]{};
    int64_t phase_calls[L2X_NPHASE]{};
};

namespace {

cudaEvent_t take_event(l2x_coupling* h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records CUDA events around one phase on the call's stream when timing is on.
struct PhaseScope {
    l2x_coupling* h;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(l2x_coupling* h_, int phase_, cudaStream_t s_) : h(h_), phase(phase_), s(s_) {
        if (h->timing) {
            a = take_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~PhaseScope() {
        if (a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, s);
            h->pending.push_back(PhaseRec{phase, a, b});
        }
    }
};

void resolve_timing(l2x_coupling* h) {
    for (auto& r : h->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            h->phase_ms[r.phase] += ms;
            h->phase_calls[r.phase] += 1;
        }
        h->event_pool.push_back(r.a);
        h->event_pool.push_back(r.b);
    }
    h->pending.clear();
}

}  // namespace

namespace {

thread_local std::string g_last_error;

l2x_status fail(l2x_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

l2x_status cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return L2X_ECUDA;
}

#define L2X_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

#define L2X_TRY(call)                     \
    do {                                  \
        l2x_status s_ = (call);           \
        if (s_ != L2X_OK) return s_;      \
    } while (0)

template <typename T>
l2x_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        g_last_error = "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed";
        return L2X_ENOMEM;
    }
    return L2X_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

l2x_status ensure_scan(l2x_coupling* h, int64_t n) {
    size_t need = scan_tmp_bytes(n);
    if (need <= h->scan_tmp_cap && h->scan_tmp) return L2X_OK;
    if (h->scan_tmp) cudaFree(h->scan_tmp);
    h->scan_tmp = nullptr;
    if (cudaMalloc(&h->scan_tmp, need) != cudaSuccess) return fail(L2X_ENOMEM, "scan scratch");
    // the single-pass scan expects a zeroed workspace and leaves it zeroed
    L2X_CUDA(cudaMemsetAsync(h->scan_tmp, 0, need, h->stream));
    h->scan_tmp_cap = need;
    return L2X_OK;
}

l2x_status flags_to_status(const DevStatus& s) {
    if (s.flags & FLAG_NONFINITE) return fail(L2X_ENONFINITE, "non-finite coordinate in element " + std::to_string(s.bad_elem));
    if (s.flags & FLAG_DEGENERATE) return fail(L2X_EDEGENERATE, "zero-volume element " + std::to_string(s.bad_elem));
    if (s.flags & FLAG_OUTOFGRID)
        return fail(L2X_EOUTOFGRID, "element " + std::to_string(s.bad_elem) + " leaves the cells of a velocity grid");
    if (s.flags & FLAG_CAPACITY) return fail(L2X_ECAPACITY, "fixed-capacity buffer overflow (element box > 1023 cells or node degree too high)");
    if (s.flags & FLAG_TIMEOUT) return fail(L2X_ETIMEOUT, "device wait timed out");
    return L2X_OK;
}

l2x_status read_status(l2x_coupling* h, cudaStream_t s) {
    L2X_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    L2X_CUDA(cudaGetLastError());
    return flags_to_status(*h->st_host);
}

l2x_status reset_status(l2x_coupling* h, cudaStream_t s) {
    DevStatus z{};
    z.bad_elem = INT_MAX;
    *h->st_host = z;
    L2X_CUDA(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
    return L2X_OK;
}

void make_subgrids(l2x_coupling* h) {
    const l2x_grid& G = h->grid;
    const bool stretched = G.axis[0] != nullptr;
    for (int g = 0; g < h->n_grids; ++g) {
        SubGrid& s = h->sg[g];
        for (int k = 0; k < 3; ++k) {
            if (k < G.dim) {
                bool shifted = G.staggered && k != g;
                s.ncell[k] = shifted ? G.ncell[k] - 1 : G.ncell[k];
                if (stretched) {
                    s.origin[k] = 0.0;
                    s.h[k] = 1.0;  // element gradients per unit length, scaled per cell
                    s.inv_h[k] = 1.0;
                } else {
                    s.origin[k] = shifted ? G.origin[k] + 0.5 * G.h[k] : G.origin[k];
                    s.h[k] = G.h[k];
                    s.inv_h[k] = 1.0 / G.h[k];
                }
            } else {
                s.ncell[k] = 1;
                s.origin[k] = 0.0;
                s.h[k] = 1.0;
                s.inv_h[k] = 1.0;
            }
            s.nnode[k] = k < G.dim ? s.ncell[k] + 1 : 1;
            s.ax[k] = nullptr;
            s.inv_w[k] = nullptr;
            int ex = 0;
            s.pow2[k] = !stretched && k < G.dim && std::frexp(s.h[k], &ex) == 0.5 && s.inv_h[k] * s.h[k] == 1.0;
        }
    }
}

// Device copies of the node coordinates and inverse cell widths of every
// velocity grid of a stretched grid (host arrays of the caller's l2x_grid).
l2x_status upload_axes(l2x_coupling* h, const l2x_grid* grid, cudaStream_t s) {
    if (!grid->axis[0]) return L2X_OK;
    for (int g = 0; g < h->n_grids; ++g) {
        SubGrid& sg = h->sg[g];
        for (int k = 0; k < grid->dim; ++k) {
            const double* x = grid->axis[k];
            const bool shifted = grid->staggered && k != g;
            const int nn = sg.nnode[k];
            std::vector<double> node(nn), iw(nn - 1);
            for (int i = 0; i < nn; ++i) node[i] = shifted ? 0.5 * (x[i] + x[i + 1]) : x[i];
            for (int i = 0; i + 1 < nn; ++i) iw[i] = 1.0 / (node[i + 1] - node[i]);
            L2X_TRY(dalloc(&h->grid_ax[g][k], nn));
            L2X_TRY(dalloc(&h->grid_iw[g][k], nn - 1));
            L2X_CUDA(cudaMemcpyAsync(h->grid_ax[g][k], node.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, s));
            L2X_CUDA(cudaMemcpyAsync(h->grid_iw[g][k], iw.data(), sizeof(double) * (nn - 1), cudaMemcpyHostToDevice, s));
            L2X_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
            sg.ax[k] = h->grid_ax[g][k];
            sg.inv_w[k] = h->grid_iw[g][k];
        }
    }
    return L2X_OK;
}

// Row list of B_g^T (non-empty rows) and the flag scratch, for up to `rows` rows
// and `entries` entries.
l2x_status ensure_tlist(l2x_coupling* h, CsrT& T, int64_t rows, int64_t entries) {
    const int64_t need = rows < entries ? rows : entries;
    if (need > T.list_cap || !T.list) {
        dfree(T.list);
        T.list_cap = 0;
        const int64_t c = need + need / 4 + 16;
        L2X_TRY(dalloc(&T.list, c));
        T.list_cap = c;
    }
    if (!T.n_list) L2X_TRY(dalloc(&T.n_list, 1));
    if (!T.n_long) L2X_TRY(dalloc(&T.n_long, 1));
    // rows longer than kSortMax (512) entries: at most entries / 513 of them
    const int64_t lneed = entries / 513 + 1;
    if (lneed > T.long_cap || !T.long_rows) {
        dfree(T.long_rows);
        T.long_cap = 0;
        L2X_TRY(dalloc(&T.long_rows, lneed));
        T.long_cap = lneed;
    }
    if (rows + 1 > h->tflags_cap || !h->tflags) {
        dfree(h->tflags);
        L2X_TRY(dalloc(&h->tflags, rows + 1));
        h->tflags_cap = rows + 1;
    }
    return L2X_OK;
}

// Topology-only structures: node adjacency and the sparsity of M_s.
l2x_status build_topology(l2x_coupling* h, cudaStream_t s) {
    const int64_t n = h->n_nodes, m = h->n_elems;
    const int NA = h->dim + 1;
    L2X_TRY(dalloc(&h->adj_ptr, n + 1));
    L2X_TRY(dalloc(&h->adj, (size_t)(m * NA)));
    L2X_TRY(dalloc(&h->cursor, n));
    L2X_TRY(dalloc(&h->row_count, (int64_t)kMaxGrids * (n + 1)));  // row counts of B_g, or of M_s
    L2X_TRY(dalloc(&h->row_cache, (size_t)h->n_grids * n));
    L2X_TRY(ensure_scan(h, n));
    launch_node_adjacency(h->dim, n, m, h->E, h->adj_ptr, h->adj, h->cursor, h->scan_tmp, s);
    L2X_TRY(dalloc(&h->M.ptr, n + 1));
    int64_t nnz = n;  // dual basis: S is diagonal (structure written with its values)
    if (h->opts.multiplier == L2X_MULT_STANDARD) {
        // sparsity of M_s
        launch_mass_structure(0, h->dim, n, h->E, h->adj_ptr, h->adj, h->row_count, nullptr, nullptr, h->st, s);
        launch_scan_i64(h->row_count, h->M.ptr, n, h->scan_tmp, s, h->st);
        L2X_CUDA(cudaMemcpyAsync(&nnz, h->M.ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    }
    L2X_TRY(read_status(h, s));
    h->M.n_rows = n;
    h->M.nnz = nnz;
    L2X_TRY(dalloc(&h->M.col, nnz));
    L2X_TRY(dalloc(&h->M.val, nnz));
    L2X_TRY(dalloc(&h->M.val32, nnz));
    L2X_TRY(dalloc(&h->M_dinv, n));
    L2X_TRY(dalloc(&h->M_dinv32, n));
    if (h->opts.multiplier == L2X_MULT_STANDARD)
        launch_mass_structure(1, h->dim, n, h->E, h->adj_ptr, h->adj, nullptr, h->M.ptr, h->M.col, h->st, s);
    return L2X_OK;
}

// Values of S (M_s, or diag(int phi_i) for the dual basis) and their FP32 copies.
void launch_S_values(l2x_coupling* h, cudaStream_t s) {
    const int64_t n = h->n_nodes;
    if (h->opts.multiplier == L2X_MULT_DUAL)
        launch_lumped_mass(h->dim, n, h->adj_ptr, h->adj, h->elem_vol, h->M.ptr, h->M.col, h->M.val, h->M_dinv, s);
    else
        launch_mass_values(h->dim, n, h->E, h->adj_ptr, h->adj, h->elem_vol, h->M.ptr, h->M.col, h->M.val,
                           h->M_dinv, s);
    launch_to_f32(h->M.val, h->M.val32, h->M.nnz, s);
    launch_to_f32(h->M_dinv, h->M_dinv32, n, s);
}

// Everything that depends on the node positions.
l2x_status build_geometry(l2x_coupling* h, cudaStream_t s) {
    const int64_t n = h->n_nodes, m = h->n_elems;
    const int G = h->n_grids, d = h->dim;
    const int NS = (d + 1) << d;
    L2X_TRY(reset_status(h, s));
    int32_t nb_init[kMaxGrids * 6];
    for (int g = 0; g < G; ++g)
        for (int k = 0; k < 3; ++k) {
            nb_init[g * 6 + k] = INT_MAX;
            nb_init[g * 6 + 3 + k] = INT_MIN;
        }
    L2X_CUDA(cudaMemcpyAsync(h->node_box, nb_init, sizeof(int32_t) * 6 * G, cudaMemcpyHostToDevice, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    // (I) candidate boxes, counts, offsets
    auto ph_pairs = std::make_unique<PhaseScope>(h, L2X_PH_PAIRS, s);
    launch_elem_boxes(d, G, h->sg, m, h->X, h->E, h->boxes, h->counts, h->nbox, h->node_box, h->elem_vol,
                      h->elem_grad, h->elem_flag, h->st, s);
    launch_scan_i64(h->counts, h->offsets, (int64_t)G * m, h->scan_tmp, s, h->st);
    launch_scan_i64(h->nbox, h->loc_off, (int64_t)G * m, h->scan_tmp, s, h->st);
    int64_t loc_total = 0;
    L2X_CUDA(cudaMemcpyAsync(&loc_total, h->loc_off + (int64_t)G * m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    std::vector<int64_t> gb(G + 1);
    for (int g = 0; g <= G; ++g)
        L2X_CUDA(cudaMemcpyAsync(&gb[g], h->offsets + (int64_t)g * m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int32_t nbh[kMaxGrids * 6];
    L2X_CUDA(cudaMemcpyAsync(nbh, h->node_box, sizeof(int32_t) * 6 * G, cudaMemcpyDeviceToHost, s));
    L2X_TRY(read_status(h, s));
    for (int g = 0; g <= G; ++g) h->pair_begin[g] = gb[g];
    h->n_pairs = gb[G];
    const int64_t NP = h->n_pairs;
    if (NP > h->pair_cap || !h->pair_elem) {
        dfree(h->pair_elem);
        dfree(h->pair_cell);
        dfree(h->blocks);
        dfree(h->vols);
        dfree(h->pair_key);
        dfree(h->pair_perm);
        h->pair_cap = 0;
        const int64_t cap = NP + NP / 4 + 128;
        L2X_TRY(dalloc(&h->pair_elem, cap));
        L2X_TRY(dalloc(&h->pair_cell, cap));
        L2X_TRY(dalloc(&h->blocks, (size_t)cap * NS));
        L2X_TRY(dalloc(&h->vols, cap));
        L2X_TRY(dalloc(&h->pair_key, cap));
        L2X_TRY(dalloc(&h->pair_perm, cap));
        h->pair_cap = cap;
    }
    if (loc_total > h->loc_cap || !h->loc_val) {
        dfree(h->loc_val);
        dfree(h->loc_flag);
        h->loc_cap = 0;
        const int64_t c = loc_total + loc_total / 4 + 64;
        L2X_TRY(dalloc(&h->loc_val, (size_t)c * (d + 1)));
        L2X_TRY(dalloc(&h->loc_flag, c));
        h->loc_cap = c;
    }
    launch_emit_pairs(d, G, h->sg, m, h->boxes, h->offsets, h->pair_elem, h->pair_cell, h->pair_cap, h->st, s);
    ph_pairs.reset();
    // (II)-(III) clip + quadrature
    const bool plain = h->opts.path == L2X_PATH_PLAIN;
    if (plain) {
        for (int g = 0; g < G; ++g) {
            PhaseScope ph(h, L2X_PH_CLIP, s);
            launch_clip_plain(d, h->sg[g], h->X, h->E, gb[g], gb[g + 1], h->pair_elem, h->pair_cell, h->blocks,
                              h->vols, h->st, s);
        }
    } else {
        {
            PhaseScope ph_cls(h, L2X_PH_PAIRS, s);
            launch_pair_classes(d, G, h->sg, m, h->offsets, NP, h->pair_cap, h->X, h->E, h->pair_elem, h->pair_cell,
                                h->pair_key, h->pair_perm, h->buckets, s);
        }
        PhaseScope ph(h, L2X_PH_CLIP, s);
        launch_clip_fused(d, h->opts.precision, G, h->sg, m, h->offsets, NP, h->pair_cap, h->X, h->E, h->elem_grad,
                          h->elem_flag, h->pair_elem, h->pair_cell, h->pair_perm, h->blocks, h->vols, h->st, s, h->clip_block, h->clip_chunk, h->clip_work);
    }
    // (IV) B_g by rows.  The element-local matrices of all grids in one launch:
    // boxes, pair offsets and local offsets run over the G*m (grid, element) slots
    {
        PhaseScope ph_loc(h, L2X_PH_ROWS, s);
        launch_elem_local(d, (int64_t)G * m, h->boxes, h->offsets, h->loc_off, h->loc_cap, h->blocks, h->vols,
                          h->loc_val, h->loc_flag, h->opts.multiplier == L2X_MULT_DUAL, h->st, s);
    }
    // rows of all grids per launch: pass 0 counts, one status read for the G
    // nonzero totals, then pass 1 (values) or 2 (structure of the plain path)
    RowsGrid rg[kMaxGrids];
    int64_t nnz_g[kMaxGrids] = {};
    {
        auto ph_rows = std::make_unique<PhaseScope>(h, L2X_PH_ROWS, s);
        for (int g = 0; g < G; ++g) {
            if (!h->B[g].ptr) L2X_TRY(dalloc(&h->B[g].ptr, n + 1));
            rg[g].boxes = h->boxes + (int64_t)g * m;
            rg[g].loc_off = h->loc_off + (int64_t)g * m;
            rg[g].row_count = h->row_count + (int64_t)g * (n + 1);
            rg[g].nnode0 = h->sg[g].nnode[0];
            rg[g].nnode1 = h->sg[g].nnode[1];
            rg[g].cache = h->row_cache + (int64_t)g * n;
        }
        launch_b_rows(0, d, G, rg, n, h->adj_ptr, h->adj, h->loc_val, h->loc_cap, h->loc_flag, h->st, s);
        for (int g = 0; g < G; ++g) {
            launch_scan_i64(rg[g].row_count, h->B[g].ptr, n, h->scan_tmp, s, h->st);
            L2X_CUDA(cudaMemcpyAsync(&nnz_g[g], h->B[g].ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        }
        ph_rows.reset();
        L2X_TRY(read_status(h, s));
    }
    for (int g = 0; g < G; ++g) {
        Csr& B = h->B[g];
        const int64_t nnz = nnz_g[g];
        B.n_rows = n;
        B.nnz = nnz;
        if (nnz > h->B_cap[g] || !B.col) {
            dfree(B.col);
            dfree(B.val);
            dfree(B.val32);
            int64_t c = nnz + nnz / 4 + 16;
            L2X_TRY(dalloc(&B.col, c));
            L2X_TRY(dalloc(&B.val, c));
            L2X_TRY(dalloc(&B.val32, c));
            h->B_cap[g] = c;
        }
        rg[g].row_ptr = B.ptr;
        rg[g].cols = B.col;
        rg[g].vals = B.val;
    }
    {
        PhaseScope ph_rows2(h, L2X_PH_ROWS, s);
        launch_b_rows(plain ? 2 : 1, d, G, rg, n, h->adj_ptr, h->adj, h->loc_val, h->loc_cap, h->loc_flag, h->st, s);
        for (int g = 0; g < G; ++g) {
            if (plain)
                launch_scatter_plain(d, h->sg[g], h->E, gb[g], gb[g + 1], h->pair_elem, h->pair_cell, h->blocks,
                                     h->vols, h->B[g], h->opts.multiplier == L2X_MULT_DUAL, s);
            else if (h->opts.precision == L2X_MIXED)
                launch_to_f32(h->B[g].val, h->B[g].val32, nnz_g[g], s);
        }
    }
    if (!plain) {
        for (int g = 0; g < G; ++g) {
            const Csr& B = h->B[g];
            const int64_t nnz = nnz_g[g];
            PhaseScope ph_t(h, L2X_PH_TRANSPOSE, s);
            // B_g^T over the box of touched fluid nodes
            CsrT& T = h->T[g];
            int64_t rows = 1;
            for (int k = 0; k < 3; ++k) {
                if (k < d && nbh[g * 6 + k] <= nbh[g * 6 + 3 + k]) {
                    T.lo[k] = nbh[g * 6 + k];
                    T.n[k] = nbh[g * 6 + 3 + k] - nbh[g * 6 + k] + 1;
                } else {
                    T.lo[k] = 0;
                    T.n[k] = 1;
                }
                rows *= T.n[k];
            }
            T.n_rows = rows;
            if (rows + 1 > h->T_rows_cap[g] || !T.ptr) {
                dfree(T.ptr);
                L2X_TRY(dalloc(&T.ptr, rows + 1));
                h->T_rows_cap[g] = rows + 1;
            }
            if (nnz > h->T_cap[g] || !T.col) {
                dfree(T.col);
                dfree(T.val);
                dfree(T.val32);
                int64_t c = nnz + nnz / 4 + 16;
                L2X_TRY(dalloc(&T.col, c));
                L2X_TRY(dalloc(&T.val, c));
                L2X_TRY(dalloc(&T.val32, c));
                h->T_cap[g] = c;
            }
            L2X_TRY(ensure_scan(h, rows));
            if (rows > h->tcursor_cap || !h->tcursor) {
                dfree(h->tcursor);
                L2X_TRY(dalloc(&h->tcursor, rows + rows / 4 + 16));
                h->tcursor_cap = rows + rows / 4 + 16;
            }
            L2X_TRY(ensure_tlist(h, T, rows, nnz));
            launch_transpose_count(B, h->sg[g], T, T.ptr, h->st, s);
            launch_transpose_list(T, T.ptr, h->tflags, h->scan_tmp, h->st, s);
            launch_scan_i64(T.ptr, T.ptr, rows, h->scan_tmp, s, h->st);
            launch_transpose_fill(B, h->sg[g], T, h->tcursor, h->st, s);
            launch_transpose_sort(T, h->st, s);
            if (h->opts.precision == L2X_MIXED) launch_to_f32(T.val, T.val32, nnz, s);
        }
    }
    // values of S
    PhaseScope ph_mass(h, L2X_PH_MASS, s);
    launch_S_values(h, s);
    return read_status(h, s);
}

l2x_status validate(const l2x_grid* grid, const l2x_mesh* mesh, const l2x_opts* o) {
    if (!grid || !mesh) return fail(L2X_EINVAL, "grid and mesh must not be NULL");
    if (grid->dim != 2 && grid->dim != 3) return fail(L2X_EINVAL, "grid dim must be 2 or 3");
    if (mesh->dim != grid->dim) return fail(L2X_EINVAL, "mesh dim differs from grid dim");
    if (mesh->n_nodes <= 0 || mesh->n_elems <= 0) return fail(L2X_EINVAL, "empty mesh");
    if (mesh->n_nodes >= INT_MAX || mesh->n_elems >= (INT_MAX >> 2)) return fail(L2X_EINVAL, "mesh too large for int32 indices");
    if (!mesh->coords || !mesh->elems) return fail(L2X_EINVAL, "mesh arrays must not be NULL");
    const bool stretched = grid->axis[0] != nullptr;
    for (int k = 0; k < grid->dim; ++k) {
        if (grid->ncell[k] < (grid->staggered ? 2 : 1)) return fail(L2X_EINVAL, "ncell too small");
        if (stretched) {
            const double* x = grid->axis[k];
            if (!x) return fail(L2X_EINVAL, "a stretched grid needs a node array on every axis");
            for (int i = 0; i <= grid->ncell[k]; ++i) {
                if (!std::isfinite(x[i])) return fail(L2X_EINVAL, "non-finite stretched node coordinate");
                if (i > 0 && !(x[i] > x[i - 1])) return fail(L2X_EINVAL, "stretched node coordinates must increase strictly");
            }
        } else if (!(grid->h[k] > 0.0)) {
            return fail(L2X_EINVAL, "h must be positive");
        }
    }
    int64_t nodes = 1;
    for (int k = 0; k < grid->dim; ++k) nodes *= (int64_t)grid->ncell[k] + 1;
    if (nodes >= INT_MAX) return fail(L2X_EINVAL, "grid too large for int32 node indices");
    if (o) {
        if (o->path != L2X_PATH_PLAIN && o->path != L2X_PATH_FUSED) return fail(L2X_EINVAL, "bad path");
        if (o->precision != L2X_FP64 && o->precision != L2X_MIXED) return fail(L2X_EINVAL, "bad precision");
        if (o->path == L2X_PATH_PLAIN && o->precision != L2X_FP64) return fail(L2X_EINVAL, "the plain path is FP64 only");
        if (!(o->cg_rtol > 0.0) || o->cg_max_iter <= 0) return fail(L2X_EINVAL, "bad CG settings");
        if (o->force_mode != L2X_FORCE_NODAL && o->force_mode != L2X_FORCE_DUAL) return fail(L2X_EINVAL, "bad force mode");
        if (o->multiplier != L2X_MULT_STANDARD && o->multiplier != L2X_MULT_DUAL) return fail(L2X_EINVAL, "bad multiplier space");
    }
    return L2X_OK;
}

l2x_status check_ptrs(const void* const* a, int n, const char* what) {
    if (!a) return fail(L2X_EINVAL, std::string(what) + " must not be NULL");
    for (int i = 0; i < n; ++i)
        if (!a[i]) return fail(L2X_EINVAL, std::string(what) + " has a NULL component");
    return L2X_OK;
}

int64_t fluid_nodes(const SubGrid& sg) { return (int64_t)sg.nnode[0] * sg.nnode[1] * sg.nnode[2]; }

// Velocity transfer without host synchronisation (fused path): B u_f with the
// division by a diagonal S fused in, or B u_f followed by the cooperative PCG
// (fixed schedule in the mixed form; non-convergence recorded in the status).
void enqueue_velocity(l2x_coupling* h, const void* const* u_f, void* const* u_s, cudaStream_t s) {
    const int G = h->n_grids;
    if (h->opts.multiplier == L2X_MULT_DUAL) {
        launch_spmv_B(L2X_PATH_FUSED, h->opts.precision, G, h->B, u_f, u_s, h->st, s, h->M_dinv);
        return;
    }
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    void* tmp[kMaxGrids];
    for (int g = 0; g < G; ++g) tmp[g] = (char*)h->vec_tmp + es * h->n_nodes * g;
    launch_spmv_B(L2X_PATH_FUSED, h->opts.precision, G, h->B, u_f, tmp, h->st, s);
    solve_mass_pcg_async(h->opts.precision, h->M, h->M_dinv, h->M_dinv32, G, (const void* const*)tmp, u_s,
                         h->opts.cg_rtol, h->opts.cg_max_iter, h->pcg_ws, h->st, s, h->pcg_rpb, h->pcg_clu);
}

// Force transfer without host synchronisation (fused path): f_f += s B^T S^-1 f_s
// (dual force mode) or s B^T f_s (nodal).
// The force input restricted to the interface mask (a copy in vec_mask), or f_s itself.
const void* const* masked_force(l2x_coupling* h, const void* const* f_s, const void** buf, cudaStream_t s) {
    if (!h->has_fmask) return f_s;
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    for (int g = 0; g < h->n_grids; ++g) buf[g] = (char*)h->vec_mask + es * h->n_nodes * g;
    launch_mask_copy(h->opts.precision, h->n_nodes, h->n_grids, h->fmask, f_s, (void* const*)buf, h->st, s);
    return buf;
}

void enqueue_force(l2x_coupling* h, const void* const* f_s_in, void* const* f_f, cudaStream_t s) {
    const int G = h->n_grids;
    const void* mbuf[kMaxGrids];
    const void* const* f_s = masked_force(h, f_s_in, mbuf, s);
    if (h->opts.force_mode == L2X_FORCE_DUAL) {
        const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
        void* tmp[kMaxGrids];
        for (int g = 0; g < G; ++g) tmp[g] = (char*)h->vec_tmp + es * h->n_nodes * g;
        if (h->opts.multiplier == L2X_MULT_DUAL)
            launch_diag_solve(h->opts.precision, h->n_nodes, G, h->M_dinv, f_s, tmp, h->st, s);
        else
            solve_mass_pcg_async(h->opts.precision, h->M, h->M_dinv, h->M_dinv32, G, f_s, tmp, h->opts.cg_rtol,
                                 h->opts.cg_max_iter, h->pcg_ws, h->st, s, h->pcg_rpb, h->pcg_clu);
        launch_spmv_BT(L2X_PATH_FUSED, h->opts.precision, G, h->B, h->T, h->sg, (const void* const*)tmp, f_f,
                       h->opts.force_scale, h->st, s);
    } else {
        launch_spmv_BT(L2X_PATH_FUSED, h->opts.precision, G, h->B, h->T, h->sg, f_s, f_f, h->opts.force_scale,
                       h->st, s);
    }
}

// Enqueues one whole time step without host synchronisation: copy of the new
// node positions, re-assembly with the capacities of the handle (overflow sets
// FLAG_CAPACITY and later kernels skip their work), velocity transfer and dual
// or nodal force transfer.  Used under stream capture by l2x_graph_create.
// The box of fluid nodes that the rows of B_g^T cover (fixed when a step graph
// is created) as a 3-D region of a fluid array of grid g (x fastest, es bytes an
// entry).
cudaPitchedPtr fluid_pitched(void* p, const SubGrid& sg, size_t es) {
    return make_cudaPitchedPtr(p, es * (size_t)sg.nnode[0], (size_t)sg.nnode[0], (size_t)sg.nnode[1]);
}
cudaExtent box_extent(const CsrT& T, size_t es) { return make_cudaExtent(es * (size_t)T.n[0], T.n[1], T.n[2]); }

// Copies the box of grid g's fluid array between host and device arrays of the
// same layout.
l2x_status copy_fluid_box(void* dst, const void* src, const SubGrid& sg, const CsrT& T, size_t es,
                          cudaMemcpyKind kind, cudaStream_t s) {
    cudaMemcpy3DParms p{};
    p.srcPtr = fluid_pitched(const_cast<void*>(src), sg, es);
    p.dstPtr = fluid_pitched(dst, sg, es);
    p.srcPos = make_cudaPos(es * (size_t)T.lo[0], T.lo[1], T.lo[2]);
    p.dstPos = p.srcPos;
    p.extent = box_extent(T, es);
    p.kind = kind;
    L2X_CUDA(cudaMemcpy3DAsync(&p, s));
    return L2X_OK;
}

// Host ends of a captured step with host buffers (page-locked): positions in,
// u_f and f_s in, u_s and f_f out, per grid.
struct HostIO {
    const void* u_f[kMaxGrids];
    void* u_s[kMaxGrids];
    const void* f_s[kMaxGrids];
    void* f_f[kMaxGrids];
};

// With `io`, coords_src is a host array and u_f .. f_f are the graph's device
// copies: the step copies the positions in first, u_f and f_s in on a branch
// beside the assembly (joined before the transfers), u_s out on that branch
// beside the force transfer, and f_f out at the end, one grid per stream.
l2x_status record_step(l2x_coupling* h, const double* coords_src, const void* const* u_f, void* const* u_s,
                       const void* const* f_s, void* const* f_f, bool zero_force, cudaStream_t s,
                       const HostIO* io = nullptr) {
    const int64_t n = h->n_nodes, m = h->n_elems;
    const int G = h->n_grids, d = h->dim;
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    L2X_CUDA(cudaMemcpyAsync(h->X, coords_src, sizeof(double) * n * d,
                             io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (io) {
        // forked after the positions are in: copies in one direction share a copy
        // engine, and the assembly waits for the positions only
        L2X_CUDA(cudaEventRecord(h->ev_io_fork, s));
        L2X_CUDA(cudaStreamWaitEvent(h->io_stream, h->ev_io_fork, 0));
        // B_g reads u_f only inside the box, and B_g^T writes f_f only there (a
        // replay whose mesh leaves the box is flagged and skipped)
        for (int g = 0; g < G; ++g)
            L2X_TRY(copy_fluid_box(const_cast<void*>(u_f[g]), io->u_f[g], h->sg[g], h->T[g], es,
                                   cudaMemcpyHostToDevice, h->io_stream));
        for (int g = 0; g < G; ++g)
            L2X_CUDA(cudaMemcpyAsync(const_cast<void*>(f_s[g]), io->f_s[g], es * n, cudaMemcpyHostToDevice,
                                     h->io_stream));
        if (!zero_force)  // f_f += ...: the host's values are the base
            for (int g = 0; g < G; ++g)
                L2X_TRY(copy_fluid_box(f_f[g], io->f_f[g], h->sg[g], h->T[g], es, cudaMemcpyHostToDevice,
                                       h->io_stream));
        L2X_CUDA(cudaEventRecord(h->ev_io_in, h->io_stream));
    }
    launch_reset_status(h->st, s);
    launch_node_box_reset(h->node_box, G, s);
    launch_elem_boxes(d, G, h->sg, m, h->X, h->E, h->boxes, h->counts, h->nbox, h->node_box, h->elem_vol,
                      h->elem_grad, h->elem_flag, h->st, s);
    {
        // the B^T rows of the captured step cover a fixed box: a step that leaves it
        // is flagged here, before any kernel indexes rows by the box
        NodeBoxSet lim{};
        for (int g = 0; g < G; ++g)
            for (int k = 0; k < 3; ++k) {
                lim.lo[g][k] = h->T[g].lo[k];
                lim.hi[g][k] = h->T[g].lo[k] + h->T[g].n[k] - 1;
            }
        launch_check_node_box(h->node_box, lim, G, h->st, s);
    }
    // the values of S depend only on the element volumes: a second branch of the
    // graph forms them while the main branch lists, clips and assembles
    L2X_CUDA(cudaEventRecord(h->ev_fork, s));
    L2X_CUDA(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
    launch_S_values(h, h->aux_stream);
    L2X_CUDA(cudaEventRecord(h->ev_join, h->aux_stream));
    launch_scan_i64(h->counts, h->offsets, (int64_t)G * m, h->scan_tmp, s, h->st);
    launch_scan_i64(h->nbox, h->loc_off, (int64_t)G * m, h->scan_tmp, s, h->st);
    launch_emit_pairs(d, G, h->sg, m, h->boxes, h->offsets, h->pair_elem, h->pair_cell, h->pair_cap, h->st, s);
    launch_pair_classes(d, G, h->sg, m, h->offsets, h->pair_cap, h->pair_cap, h->X, h->E, h->pair_elem, h->pair_cell,
                        h->pair_key, h->pair_perm, h->buckets, s);
    launch_clip_fused(d, h->opts.precision, G, h->sg, m, h->offsets, h->pair_cap, h->pair_cap, h->X, h->E,
                      h->elem_grad, h->elem_flag, h->pair_elem, h->pair_cell, h->pair_perm, h->blocks, h->vols, h->st,
                      s, h->clip_block, h->clip_chunk, h->clip_work);
    launch_elem_local(d, (int64_t)G * m, h->boxes, h->offsets, h->loc_off, h->loc_cap, h->blocks, h->vols,
                      h->loc_val, h->loc_flag, h->opts.multiplier == L2X_MULT_DUAL, h->st, s);
    // rows of all grids per launch (the B_g arrays are fixed by the capture)
    RowsGrid rg[kMaxGrids];
    for (int g = 0; g < G; ++g) {
        rg[g].boxes = h->boxes + (int64_t)g * m;
        rg[g].loc_off = h->loc_off + (int64_t)g * m;
        rg[g].row_count = h->row_count + (int64_t)g * (n + 1);
        rg[g].row_ptr = h->B[g].ptr;
        rg[g].cols = h->B[g].col;
        rg[g].vals = h->B[g].val;
        rg[g].nnode0 = h->sg[g].nnode[0];
        rg[g].nnode1 = h->sg[g].nnode[1];
        rg[g].cache = h->row_cache + (int64_t)g * n;
    }
    launch_b_rows(0, d, G, rg, n, h->adj_ptr, h->adj, h->loc_val, h->loc_cap, h->loc_flag, h->st, s);
    for (int g = 0; g < G; ++g) {
        launch_scan_i64(rg[g].row_count, h->B[g].ptr, n, h->scan_tmp, s, h->st);
        launch_check_capacity(h->B[g].ptr + n, h->B_cap[g], h->st, s);
    }
    launch_b_rows(1, d, G, rg, n, h->adj_ptr, h->adj, h->loc_val, h->loc_cap, h->loc_flag, h->st, s);
    // the G grids' FP32 copies and transposes are independent: one graph branch
    // per grid
    L2X_CUDA(cudaEventRecord(h->ev_tfork, s));
    for (int g = 0; g < G; ++g) {
        cudaStream_t ts = g == 0 ? s : h->t_stream[g];
        if (g > 0) L2X_CUDA(cudaStreamWaitEvent(ts, h->ev_tfork, 0));
        int32_t* cursor = g == 0 ? h->tcursor : h->t_cursor[g];
        int64_t* flags = g == 0 ? h->tflags : h->t_flags[g];
        void* scan = g == 0 ? h->scan_tmp : h->t_scan[g];
        Csr& B = h->B[g];
        B.n_rows = n;
        B.nnz = h->B_cap[g];  // an upper bound: the row pointers hold the actual count
        if (h->opts.precision == L2X_MIXED) launch_to_f32(B.val, B.val32, h->B_cap[g], ts);
        CsrT& T = h->T[g];
        launch_transpose_count(B, h->sg[g], T, T.ptr, h->st, ts);
        launch_transpose_list(T, T.ptr, flags, scan, h->st, ts);
        launch_scan_i64(T.ptr, T.ptr, T.n_rows, scan, ts, h->st);
        launch_transpose_fill(B, h->sg[g], T, cursor, h->st, ts);
        launch_transpose_sort(T, h->st, ts);
        if (h->opts.precision == L2X_MIXED) launch_to_f32(T.val, T.val32, h->T_cap[g], ts);
        if (g > 0) L2X_CUDA(cudaEventRecord(h->ev_tjoin[g], ts));
    }
    for (int g = 1; g < G; ++g) L2X_CUDA(cudaStreamWaitEvent(s, h->ev_tjoin[g], 0));
    L2X_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));  // S is formed
    if (io) L2X_CUDA(cudaStreamWaitEvent(s, h->ev_io_in, 0));  // u_f and f_s are in
    // u_s out on the copy branch once the velocity transfer is done
    auto copy_us_out = [&]() -> l2x_status {
        if (!io) return L2X_OK;
        L2X_CUDA(cudaEventRecord(h->ev_io_us, s));
        L2X_CUDA(cudaStreamWaitEvent(h->io_stream, h->ev_io_us, 0));
        for (int g = 0; g < G; ++g)
            L2X_CUDA(cudaMemcpyAsync(io->u_s[g], u_s[g], es * n, cudaMemcpyDeviceToHost, h->io_stream));
        L2X_CUDA(cudaEventRecord(h->ev_io_out, h->io_stream));
        return L2X_OK;
    };
    // f_f = 0 before the force transfer adds into it
    auto zero_forces = [&](void* const* ff) -> l2x_status {
        for (int g = 0; g < G; ++g) L2X_CUDA(cudaMemsetAsync(ff[g], 0, es * fluid_nodes(h->sg[g]), s));
        return L2X_OK;
    };
    // f_f out, grid g >= 1 on the stream of its transpose branch, then every
    // branch joins the main stream
    auto copy_ff_out = [&]() -> l2x_status {
        if (!io) return L2X_OK;
        L2X_CUDA(cudaEventRecord(h->ev_tfork, s));
        for (int g = 1; g < G; ++g) {
            L2X_CUDA(cudaStreamWaitEvent(h->t_stream[g], h->ev_tfork, 0));
            L2X_TRY(copy_fluid_box(io->f_f[g], f_f[g], h->sg[g], h->T[g], es, cudaMemcpyDeviceToHost,
                                   h->t_stream[g]));
            L2X_CUDA(cudaEventRecord(h->ev_tjoin[g], h->t_stream[g]));
        }
        L2X_TRY(copy_fluid_box(io->f_f[0], f_f[0], h->sg[0], h->T[0], es, cudaMemcpyDeviceToHost, s));
        for (int g = 1; g < G; ++g) L2X_CUDA(cudaStreamWaitEvent(s, h->ev_tjoin[g], 0));
        L2X_CUDA(cudaStreamWaitEvent(s, h->ev_io_out, 0));
        return L2X_OK;
    };
    // transfers
    if (h->opts.multiplier == L2X_MULT_STANDARD && h->opts.force_mode == L2X_FORCE_DUAL) {
        // the two solves with M_s are independent: one PCG on the 2G right-hand
        // sides [B u_f ; f_s] (its iterations are latency-bound, so this costs
        // about one solve)
        void* yv[kMaxGrids];
        void* zf[kMaxGrids];
        for (int g = 0; g < G; ++g) {
            yv[g] = (char*)h->vec_tmp + es * n * g;
            zf[g] = (char*)h->vec_tmp2 + es * n * g;
        }
        launch_spmv_B(L2X_PATH_FUSED, h->opts.precision, G, h->B, u_f, yv, h->st, s);
        const void* mbuf[kMaxGrids];
        const void* const* fs = masked_force(h, f_s, mbuf, s);
        const void* ys[2 * kMaxGrids];
        void* ws[2 * kMaxGrids];
        for (int g = 0; g < G; ++g) {
            ys[g] = yv[g];
            ws[g] = u_s[g];
            ys[G + g] = fs[g];
            ws[G + g] = zf[g];
        }
        solve_mass_pcg_async(h->opts.precision, h->M, h->M_dinv, h->M_dinv32, 2 * G, ys, ws, h->opts.cg_rtol,
                             h->opts.cg_max_iter, h->pcg_ws, h->st, s, h->pcg_rpb_step, 0);
        L2X_TRY(copy_us_out());
        if (zero_force) L2X_TRY(zero_forces(f_f));
        launch_spmv_BT(L2X_PATH_FUSED, h->opts.precision, G, h->B, h->T, h->sg, (const void* const*)zf, f_f,
                       h->opts.force_scale, h->st, s);
        return copy_ff_out();
    }
    enqueue_velocity(h, u_f, u_s, s);
    L2X_TRY(copy_us_out());
    if (zero_force) L2X_TRY(zero_forces(f_f));
    enqueue_force(h, f_s, f_f, s);
    return copy_ff_out();
}

}  // namespace

struct l2x_step_graph {
    l2x_coupling* h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t gen = 0;  // the handle's graph_gen at creation
    std::vector<void*> owned;  // device copies of the host-buffer form's arrays
    int64_t io_h2d = 0, io_d2h = 0;  // host-buffer form: bytes copied in and out per replay
    ~l2x_step_graph() {
        for (void* p : owned) cudaFree(p);
    }
};

extern "C" {

void l2x_default_opts(l2x_opts* o) {
    if (!o) return;
    o->path = L2X_PATH_FUSED;
    o->precision = L2X_FP64;
    o->cg_rtol = 1e-13;
    o->cg_max_iter = 200;
    o->force_mode = L2X_FORCE_DUAL;
    o->force_scale = 1.0;
    o->multiplier = L2X_MULT_STANDARD;
    o->reserved = 0;
}

const char* l2x_status_string(l2x_status s) {
    switch (s) {
        case L2X_OK: return "ok";
        case L2X_EINVAL: return "invalid argument";
        case L2X_ENOMEM: return "out of device memory";
        case L2X_ECAPACITY: return "capacity exceeded";
        case L2X_EOUTOFGRID: return "solid element outside the fluid grid";
        case L2X_EDEGENERATE: return "degenerate solid element";
        case L2X_ENOTCONVERGED: return "mass-matrix solve did not converge";
        case L2X_ETIMEOUT: return "device wait timed out";
        case L2X_ECUDA: return "CUDA error";
        case L2X_ENONFINITE: return "non-finite input";
    }
    return "unknown status";
}

const char* l2x_last_error(void) { return g_last_error.c_str(); }

l2x_status l2x_destroy(l2x_handle h) {
    if (!h) return L2X_OK;
    cudaStreamSynchronize(h->stream);
    resolve_timing(h);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    dfree(h->X); dfree(h->E); dfree(h->adj_ptr); dfree(h->adj); dfree(h->cursor); dfree(h->elem_vol);
    dfree(h->elem_grad); dfree(h->elem_flag); dfree(h->buckets); dfree(h->pair_key); dfree(h->pair_perm);
    dfree(h->nbox); dfree(h->loc_off); dfree(h->loc_val); dfree(h->loc_flag);
    dfree(h->boxes); dfree(h->counts); dfree(h->offsets); dfree(h->node_box); dfree(h->pair_elem);
    dfree(h->pair_cell); dfree(h->blocks); dfree(h->vols); dfree(h->clip_work);
    for (int g = 0; g < kMaxGrids; ++g) {
        dfree(h->B[g].ptr); dfree(h->B[g].col); dfree(h->B[g].val); dfree(h->B[g].val32);
        dfree(h->T[g].ptr); dfree(h->T[g].col); dfree(h->T[g].val); dfree(h->T[g].val32);
        dfree(h->T[g].list); dfree(h->T[g].n_list); dfree(h->T[g].long_rows); dfree(h->T[g].n_long);
    }
    dfree(h->M.ptr); dfree(h->M.col); dfree(h->M.val); dfree(h->M.val32); dfree(h->M_dinv); dfree(h->M_dinv32);
    for (int g = 0; g < kMaxGrids; ++g)
        for (int k = 0; k < 3; ++k) {
            dfree(h->grid_ax[g][k]);
            dfree(h->grid_iw[g][k]);
        }
    if (h->scan_tmp) cudaFree(h->scan_tmp);
    dfree(h->row_count);
    dfree(h->row_cache);
    dfree(h->tcursor);
    dfree(h->tflags);
    if (h->pcg_ws) cudaFree(h->pcg_ws);
    if (h->vec_tmp) cudaFree(h->vec_tmp);
    if (h->vec_tmp2) cudaFree(h->vec_tmp2);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
    if (h->ev_tfork) cudaEventDestroy(h->ev_tfork);
    for (int g = 0; g < kMaxGrids; ++g) {
        if (h->ev_tjoin[g]) cudaEventDestroy(h->ev_tjoin[g]);
        if (h->t_stream[g]) cudaStreamDestroy(h->t_stream[g]);
        dfree(h->t_cursor[g]);
        dfree(h->t_flags[g]);
        if (h->t_scan[g]) cudaFree(h->t_scan[g]);
    }
    if (h->vec_mask) cudaFree(h->vec_mask);
    dfree(h->fmask);
    if (h->io_stream) cudaStreamDestroy(h->io_stream);
    for (cudaEvent_t e : {h->ev_io_fork, h->ev_io_in, h->ev_io_us, h->ev_io_out})
        if (e) cudaEventDestroy(e);
    dfree(h->st);
    if (h->st_host) cudaFreeHost(h->st_host);
    delete h;
    return L2X_OK;
}

l2x_status l2x_build_coupling(const l2x_grid* grid, const l2x_mesh* mesh, const l2x_opts* opts, void* stream,
                              l2x_handle* out) {
    g_last_error.clear();
    if (!out) return fail(L2X_EINVAL, "out must not be NULL");
    *out = nullptr;
    l2x_opts o;
    l2x_default_opts(&o);
    if (opts) o = *opts;
    L2X_TRY(validate(grid, mesh, &o));
    cudaStream_t s = (cudaStream_t)stream;
    l2x_coupling* h = new l2x_coupling();
    h->dim = grid->dim;
    h->n_grids = grid->staggered ? grid->dim : 1;
    h->n_nodes = mesh->n_nodes;
    h->n_elems = mesh->n_elems;
    h->grid = *grid;
    h->opts = o;
    h->stream = s;
    make_subgrids(h);
    for (int k = 0; k < 3; ++k) h->grid.axis[k] = nullptr;  // the caller's arrays are read during the build only
    auto body = [&]() -> l2x_status {
        const int64_t n = h->n_nodes, m = h->n_elems;
        const int d = h->dim, G = h->n_grids;
        if (cudaMallocHost((void**)&h->st_host, sizeof(DevStatus)) != cudaSuccess) return fail(L2X_ENOMEM, "pinned status");
        L2X_TRY(dalloc(&h->st, 1));
        L2X_TRY(dalloc(&h->X, (size_t)(n * d)));
        L2X_TRY(dalloc(&h->E, (size_t)(m * (d + 1))));
        L2X_CUDA(cudaMemcpyAsync(h->X, mesh->coords, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, s));
        L2X_CUDA(cudaMemcpyAsync(h->E, mesh->elems, sizeof(int32_t) * m * (d + 1), cudaMemcpyDeviceToDevice, s));
        L2X_TRY(dalloc(&h->elem_vol, m));
        L2X_TRY(dalloc(&h->elem_grad, (size_t)(m * (d + 1) * d)));
        L2X_TRY(dalloc(&h->elem_flag, m));
        L2X_TRY(dalloc(&h->buckets, 2 * kClasses));
        L2X_TRY(dalloc(&h->clip_work, 1));
        L2X_TRY(dalloc(&h->boxes, (size_t)(G * m)));
        L2X_TRY(dalloc(&h->counts, (size_t)(G * m)));
        L2X_TRY(dalloc(&h->offsets, (size_t)(G * m + 1)));
        L2X_TRY(dalloc(&h->nbox, (size_t)(G * m)));
        L2X_TRY(dalloc(&h->loc_off, (size_t)(G * m + 1)));
        L2X_TRY(dalloc(&h->node_box, (size_t)(6 * G)));
        L2X_TRY(ensure_scan(h, (int64_t)G * m > n ? (int64_t)G * m : n));
        L2X_TRY(reset_status(h, s));
        // element indices must be valid node numbers: checked on the host copy-free path by the
        // adjacency kernel's atomics would fault otherwise, so verify here.
        {
            std::vector<int32_t> eh((size_t)(m * (d + 1)));
            L2X_CUDA(cudaMemcpyAsync(eh.data(), h->E, sizeof(int32_t) * eh.size(), cudaMemcpyDeviceToHost, s));
            L2X_CUDA(cudaStreamSynchronize(s));
            for (int32_t v : eh)
                if (v < 0 || v >= n) return fail(L2X_EINVAL, "element references a node outside [0, n_nodes)");
        }
        pcg_cluster_prepare();
        L2X_TRY(upload_axes(h, grid, s));
        L2X_TRY(build_topology(h, s));
        size_t ws = pcg_ws_bytes(n, 2 * G, pcg_max_blocks());  // a captured step solves both transfers at once
        if (cudaMalloc(&h->pcg_ws, ws) != cudaSuccess) return fail(L2X_ENOMEM, "CG workspace");
        if (cudaMalloc(&h->vec_tmp, sizeof(double) * n * G) != cudaSuccess) return fail(L2X_ENOMEM, "vector scratch");
        if (cudaMalloc(&h->vec_tmp2, sizeof(double) * n * G) != cudaSuccess) return fail(L2X_ENOMEM, "vector scratch");
        return build_geometry(h, s);
    };
    l2x_status st = body();
    if (st != L2X_OK) {
        std::string keep = g_last_error;
        l2x_destroy(h);
        g_last_error = keep;
        return st;
    }
    *out = h;
    return L2X_OK;
}

l2x_status l2x_update_geometry(l2x_handle h, const double* coords, void* stream) {
    g_last_error.clear();
    if (!h || !coords) return fail(L2X_EINVAL, "NULL handle or coordinates");
    cudaStream_t s = (cudaStream_t)stream;
    h->stream = s;
    ++h->graph_gen;  // a re-assembly may reallocate what existing graphs use
    L2X_CUDA(cudaMemcpyAsync(h->X, coords, sizeof(double) * h->n_nodes * h->dim, cudaMemcpyDeviceToDevice, s));
    return build_geometry(h, s);
}

l2x_status l2x_apply_B(l2x_handle h, const void* const* x_f, void* const* y_s, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(x_f, h->n_grids, "x_f"));
    L2X_TRY(check_ptrs((const void* const*)y_s, h->n_grids, "y_s"));
    cudaStream_t s = (cudaStream_t)stream;
    PhaseScope ph(h, L2X_PH_SPMV_B, s);
    launch_spmv_B(h->opts.path, h->opts.precision, h->n_grids, h->B, x_f, y_s, h->st, s);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_apply_BT(l2x_handle h, const void* const* z_s, void* const* f_f, double scale, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(z_s, h->n_grids, "z_s"));
    L2X_TRY(check_ptrs((const void* const*)f_f, h->n_grids, "f_f"));
    cudaStream_t s = (cudaStream_t)stream;
    PhaseScope ph(h, L2X_PH_SPMV_BT, s);
    launch_spmv_BT(h->opts.path, h->opts.precision, h->n_grids, h->B, h->T, h->sg, z_s, f_f, scale, h->st, s);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_solve_mass(l2x_handle h, const void* const* y_s, void* const* w_s, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(y_s, h->n_grids, "y_s"));
    L2X_TRY(check_ptrs((const void* const*)w_s, h->n_grids, "w_s"));
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opts.multiplier == L2X_MULT_DUAL) {  // diagonal S: one division per entry
        PhaseScope ph(h, L2X_PH_PCG, s);
        launch_diag_solve(h->opts.precision, h->n_nodes, h->n_grids, h->M_dinv, y_s, w_s, h->st, s);
        h->cg_iters = 0;
        h->cg_residual = 0.0;
        L2X_CUDA(cudaGetLastError());
        return L2X_OK;
    }
    PcgResult r;
    auto ph = std::make_unique<PhaseScope>(h, L2X_PH_PCG, s);
    l2x_status st = solve_mass_pcg(h->opts.path, h->opts.precision, h->M, h->M_dinv, h->M_dinv32, h->n_grids, y_s,
                                   w_s, h->opts.cg_rtol, h->opts.cg_max_iter, h->pcg_ws, h->st, h->st_host, s, &r,
                                   h->pcg_rpb, h->pcg_clu);
    ph.reset();
    h->cg_iters = r.iters;
    h->cg_residual = r.residual;
    if (st == L2X_ECUDA) return cuda_fail(cudaGetLastError(), "mass-matrix solve");
    if (st == L2X_ENOTCONVERGED)
        return fail(st, "CG reached relative residual " + std::to_string(r.residual) + " after " + std::to_string(r.iters) + " iterations");
    return st;
}

l2x_status l2x_transfer_velocity(l2x_handle h, const void* const* u_f, void* const* u_s, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(u_f, h->n_grids, "u_f"));
    L2X_TRY(check_ptrs((const void* const*)u_s, h->n_grids, "u_s"));
    if (h->opts.multiplier == L2X_MULT_DUAL) {  // S diagonal: the division is fused into B u_f
        cudaStream_t s = (cudaStream_t)stream;
        PhaseScope ph(h, L2X_PH_SPMV_B, s);
        launch_spmv_B(h->opts.path, h->opts.precision, h->n_grids, h->B, u_f, u_s, h->st, s, h->M_dinv);
        h->cg_iters = 0;
        h->cg_residual = 0.0;
        L2X_CUDA(cudaGetLastError());
        return L2X_OK;
    }
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    void* y[kMaxGrids];
    for (int g = 0; g < h->n_grids; ++g) y[g] = (char*)h->vec_tmp + es * h->n_nodes * g;
    L2X_TRY(l2x_apply_B(h, u_f, y, stream));
    return l2x_solve_mass(h, (const void* const*)y, u_s, stream);
}

l2x_status l2x_transfer_force(l2x_handle h, const void* const* f_s_in, void* const* f_f, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(f_s_in, h->n_grids, "f_s"));
    L2X_TRY(check_ptrs((const void* const*)f_f, h->n_grids, "f_f"));
    const void* mbuf[kMaxGrids];
    const void* const* f_s = masked_force(h, f_s_in, mbuf, (cudaStream_t)stream);
    if (h->opts.force_mode == L2X_FORCE_NODAL) return l2x_apply_BT(h, f_s, f_f, h->opts.force_scale, stream);
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    void* z[kMaxGrids];
    for (int g = 0; g < h->n_grids; ++g) z[g] = (char*)h->vec_tmp + es * h->n_nodes * g;
    L2X_TRY(l2x_solve_mass(h, f_s, z, stream));
    return l2x_apply_BT(h, (const void* const*)z, f_f, h->opts.force_scale, stream);
}

l2x_status l2x_transfer_force_adjoint(l2x_handle h, const void* const* g_f, void* const* g_s, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    L2X_TRY(check_ptrs(g_f, h->n_grids, "g_f"));
    L2X_TRY(check_ptrs((const void* const*)g_s, h->n_grids, "g_s"));
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opts.force_mode == L2X_FORCE_DUAL) {
        const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
        void* y[kMaxGrids];
        for (int g = 0; g < h->n_grids; ++g) y[g] = (char*)h->vec_tmp + es * h->n_nodes * g;
        L2X_TRY(l2x_apply_B(h, g_f, y, stream));
        L2X_TRY(l2x_solve_mass(h, (const void* const*)y, g_s, stream));
    } else {
        L2X_TRY(l2x_apply_B(h, g_f, g_s, stream));
    }
    launch_scale_mask(h->opts.precision, h->n_nodes, h->n_grids, h->has_fmask ? h->fmask : nullptr,
                      h->opts.force_scale, g_s, h->st, s);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_set_force_mask(l2x_handle h, const uint8_t* mask, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    if (!mask) {
        h->has_fmask = false;
        return L2X_OK;
    }
    if (!h->fmask) L2X_TRY(dalloc(&h->fmask, h->n_nodes));
    if (!h->vec_mask && cudaMalloc(&h->vec_mask, sizeof(double) * h->n_nodes * h->n_grids) != cudaSuccess)
        return fail(L2X_ENOMEM, "masked force scratch");
    L2X_CUDA(cudaMemcpyAsync(h->fmask, mask, h->n_nodes, cudaMemcpyDeviceToDevice, s));
    h->has_fmask = true;
    return L2X_OK;
}

l2x_status l2x_transfer_velocity_async(l2x_handle h, const void* const* u_f, void* const* u_s, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    if (h->opts.path != L2X_PATH_FUSED) return fail(L2X_EINVAL, "enqueue-only transfers need the fused path");
    L2X_TRY(check_ptrs(u_f, h->n_grids, "u_f"));
    L2X_TRY(check_ptrs((const void* const*)u_s, h->n_grids, "u_s"));
    enqueue_velocity(h, u_f, u_s, (cudaStream_t)stream);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_transfer_force_async(l2x_handle h, const void* const* f_s, void* const* f_f, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    if (h->opts.path != L2X_PATH_FUSED) return fail(L2X_EINVAL, "enqueue-only transfers need the fused path");
    L2X_TRY(check_ptrs(f_s, h->n_grids, "f_s"));
    L2X_TRY(check_ptrs((const void* const*)f_f, h->n_grids, "f_f"));
    enqueue_force(h, f_s, f_f, (cudaStream_t)stream);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_sync_status(l2x_handle h, void* stream) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    L2X_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    L2X_CUDA(cudaGetLastError());
    const DevStatus ds = *h->st_host;
    h->cg_iters = ds.cg_iters;
    h->cg_residual = ds.cg_residual;
    L2X_TRY(reset_status(h, s));
    L2X_TRY(flags_to_status(ds));
    if (ds.flags & FLAG_NOTCONVERGED) return fail(L2X_ENOTCONVERGED, "CG did not reach cg_rtol in an enqueued solve");
    return L2X_OK;
}

l2x_status l2x_picard_norms(l2x_handle h, const void* const* f_new, void* const* f_prev, int32_t copy,
                            double* norms, void* stream) {
    if (!h || !norms) return fail(L2X_EINVAL, "NULL handle or norms");
    L2X_TRY(check_ptrs(f_new, h->n_grids, "f_new"));
    L2X_TRY(check_ptrs((const void* const*)f_prev, h->n_grids, "f_prev"));
    if (((uintptr_t)norms & 7) != 0) return fail(L2X_EINVAL, "norms must be 8-byte aligned");
    launch_picard_norms(h->opts.precision, h->n_nodes, h->n_grids, f_new, f_prev, copy != 0, norms,
                        (cudaStream_t)stream);
    L2X_CUDA(cudaGetLastError());
    return L2X_OK;
}

l2x_status l2x_picard_converged(const double* norms, double eps_abs, double eps_rel, double f0_norm,
                                int32_t* converged, double* host_norms, void* stream) {
    if (!norms || !converged) return fail(L2X_EINVAL, "NULL norms or converged");
    cudaStream_t s = (cudaStream_t)stream;
    double hn[2] = {0.0, 0.0};
    L2X_CUDA(cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    if (host_norms) {
        host_norms[0] = hn[0];
        host_norms[1] = hn[1];
    }
    const bool abs_ok = hn[0] < eps_abs;
    const bool rel_ok = f0_norm > 0.0 && hn[0] / f0_norm < eps_rel;
    *converged = (abs_ok || rel_ok) ? 1 : 0;
    return L2X_OK;
}

}  // extern "C"

namespace {

// l2x_graph_create and l2x_graph_create_host: capacities, scratch, capture.  With
// `io`, u_f .. f_f are the graph's own device arrays (`owned`, freed with it).
l2x_status graph_create_common(l2x_handle h, const double* coords_src, const void* const* u_f, void* const* u_s,
                               const void* const* f_s, void* const* f_f, double capacity_margin,
                               int32_t zero_force, void* stream, l2x_graph* out, const HostIO* io,
                               std::vector<void*>& owned) {
    cudaStream_t s = (cudaStream_t)stream;
    h->stream = s;
    ++h->graph_gen;  // the capacities below may reallocate what earlier graphs use
    const int G = h->n_grids, d = h->dim;
    const int NS = (d + 1) << d;
    // capacities with margin (pairs and B entries), B^T over every fluid node
    const int64_t pcap = (int64_t)(capacity_margin * (double)h->n_pairs) + 1024;
    if (pcap > h->pair_cap) {
        dfree(h->pair_elem); dfree(h->pair_cell); dfree(h->blocks); dfree(h->vols); dfree(h->pair_key);
        dfree(h->pair_perm);
        h->pair_cap = 0;
        L2X_TRY(dalloc(&h->pair_elem, pcap));
        L2X_TRY(dalloc(&h->pair_cell, pcap));
        L2X_TRY(dalloc(&h->blocks, (size_t)pcap * NS));
        L2X_TRY(dalloc(&h->vols, pcap));
        L2X_TRY(dalloc(&h->pair_key, pcap));
        L2X_TRY(dalloc(&h->pair_perm, pcap));
        h->pair_cap = pcap;
    }
    int32_t nbh[kMaxGrids * 6];  // touched-node boxes of the last assembly
    L2X_CUDA(cudaMemcpyAsync(nbh, h->node_box, sizeof(int32_t) * 6 * G, cudaMemcpyDeviceToHost, s));
    {
        int64_t loc_total = 0;
        L2X_CUDA(cudaMemcpyAsync(&loc_total, h->loc_off + (int64_t)G * h->n_elems, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
        L2X_CUDA(cudaStreamSynchronize(s));
        const int64_t lcap = (int64_t)(capacity_margin * (double)loc_total) + 1024;
        if (lcap > h->loc_cap) {
            dfree(h->loc_val);
            dfree(h->loc_flag);
            h->loc_cap = 0;
            L2X_TRY(dalloc(&h->loc_val, (size_t)lcap * (d + 1)));
            L2X_TRY(dalloc(&h->loc_flag, lcap));
            h->loc_cap = lcap;
        }
    }
    int64_t max_rows = 0;
    for (int g = 0; g < G; ++g) {
        Csr& B = h->B[g];
        const int64_t bcap = (int64_t)(capacity_margin * (double)B.nnz) + 1024;
        if (bcap > h->B_cap[g]) {
            dfree(B.col); dfree(B.val); dfree(B.val32);
            L2X_TRY(dalloc(&B.col, bcap));
            L2X_TRY(dalloc(&B.val, bcap));
            L2X_TRY(dalloc(&B.val32, bcap));
            h->B_cap[g] = bcap;
        }
        CsrT& T = h->T[g];
        if (h->B_cap[g] > h->T_cap[g]) {
            dfree(T.col); dfree(T.val); dfree(T.val32);
            L2X_TRY(dalloc(&T.col, h->B_cap[g]));
            L2X_TRY(dalloc(&T.val, h->B_cap[g]));
            L2X_TRY(dalloc(&T.val32, h->B_cap[g]));
            h->T_cap[g] = h->B_cap[g];
        }
        // B^T rows over the nodes the mesh touches now, padded on every side by the
        // capacity margin (at least 2 nodes); replays that leave the box report
        // L2X_ECAPACITY
        int64_t rows = 1;
        for (int k = 0; k < 3; ++k) {
            const int nn = h->sg[g].nnode[k];
            int lo = 0, hi = nn - 1;
            if (k < d && nbh[g * 6 + k] <= nbh[g * 6 + 3 + k]) {
                const int ext = nbh[g * 6 + 3 + k] - nbh[g * 6 + k] + 1;
                const int pad = 2 + (int)std::ceil((capacity_margin - 1.0) * ext);
                lo = std::max(0, nbh[g * 6 + k] - pad);
                hi = std::min(nn - 1, nbh[g * 6 + 3 + k] + pad);
            }
            T.lo[k] = lo;
            T.n[k] = hi - lo + 1;
            rows *= T.n[k];
        }
        T.n_rows = rows;
        if (rows + 1 > h->T_rows_cap[g]) {
            dfree(T.ptr);
            L2X_TRY(dalloc(&T.ptr, rows + 1));
            h->T_rows_cap[g] = rows + 1;
        }
        L2X_TRY(ensure_tlist(h, T, rows, h->B_cap[g]));
        if (rows > max_rows) max_rows = rows;
    }
    if (max_rows > h->tcursor_cap) {
        dfree(h->tcursor);
        L2X_TRY(dalloc(&h->tcursor, max_rows));
        h->tcursor_cap = max_rows;
    }
    L2X_TRY(ensure_scan(h, max_rows));
    // scratch of the transposes on the branches of grids 1 .. G-1
    for (int g = 1; g < G; ++g) {
        const int64_t rows = h->T[g].n_rows;
        if (rows <= h->t_rows_cap[g] && h->t_cursor[g]) continue;
        dfree(h->t_cursor[g]);
        dfree(h->t_flags[g]);
        if (h->t_scan[g]) cudaFree(h->t_scan[g]);
        h->t_scan[g] = nullptr;
        h->t_rows_cap[g] = 0;
        L2X_TRY(dalloc(&h->t_cursor[g], rows));
        L2X_TRY(dalloc(&h->t_flags[g], rows + 1));
        if (cudaMalloc(&h->t_scan[g], scan_tmp_bytes(rows)) != cudaSuccess) return fail(L2X_ENOMEM, "scan scratch");
        L2X_CUDA(cudaMemsetAsync(h->t_scan[g], 0, scan_tmp_bytes(rows), s));
        h->t_rows_cap[g] = rows;
    }
    L2X_CUDA(cudaStreamSynchronize(s));
    if (!h->aux_stream) {
        L2X_CUDA(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
        L2X_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        L2X_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        L2X_CUDA(cudaEventCreateWithFlags(&h->ev_tfork, cudaEventDisableTiming));
        for (int g = 1; g < kMaxGrids; ++g) {
            L2X_CUDA(cudaStreamCreateWithFlags(&h->t_stream[g], cudaStreamNonBlocking));
            L2X_CUDA(cudaEventCreateWithFlags(&h->ev_tjoin[g], cudaEventDisableTiming));
        }
    }
    if (io && !h->io_stream) {
        L2X_CUDA(cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&h->ev_io_fork, &h->ev_io_in, &h->ev_io_us, &h->ev_io_out})
            L2X_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    // capture one step
    l2x_step_graph* gr = new l2x_step_graph();
    gr->h = h;
    gr->owned.swap(owned);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete gr;
        return cuda_fail(e, "cudaStreamBeginCapture (use a non-default stream)");
    }
    l2x_status st = record_step(h, coords_src, u_f, u_s, f_s, f_f, zero_force != 0, s, io);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (st != L2X_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete gr;
        cudaGetLastError();
        return st != L2X_OK ? st : cuda_fail(e, "cudaStreamEndCapture");
    }
    gr->graph = graph;
    gr->gen = h->graph_gen;
    e = cudaGraphInstantiate(&gr->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete gr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = gr;
    return L2X_OK;
}

// true if p is page-locked host memory (cudaHostAlloc or cudaHostRegister)
bool page_locked(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

l2x_status l2x_graph_create(l2x_handle h, const double* coords_src, const void* const* u_f, void* const* u_s,
                            const void* const* f_s, void* const* f_f, double capacity_margin, int32_t zero_force,
                            void* stream, l2x_graph* out) {
    g_last_error.clear();
    if (!h || !out || !coords_src) return fail(L2X_EINVAL, "NULL argument");
    *out = nullptr;
    if (h->opts.path != L2X_PATH_FUSED) return fail(L2X_EINVAL, "step graphs need the fused path");
    if (!(capacity_margin >= 1.0)) return fail(L2X_EINVAL, "capacity_margin must be >= 1");
    L2X_TRY(check_ptrs(u_f, h->n_grids, "u_f"));
    L2X_TRY(check_ptrs((const void* const*)u_s, h->n_grids, "u_s"));
    L2X_TRY(check_ptrs(f_s, h->n_grids, "f_s"));
    L2X_TRY(check_ptrs((const void* const*)f_f, h->n_grids, "f_f"));
    std::vector<void*> none;
    return graph_create_common(h, coords_src, u_f, u_s, f_s, f_f, capacity_margin, zero_force, stream, out, nullptr,
                               none);
}

l2x_status l2x_graph_create_host(l2x_handle h, const double* coords_host, const void* const* u_f_host,
                                 void* const* u_s_host, const void* const* f_s_host, void* const* f_f_host,
                                 double capacity_margin, int32_t zero_force, void* stream, l2x_graph* out) {
    g_last_error.clear();
    if (!h || !out || !coords_host) return fail(L2X_EINVAL, "NULL argument");
    *out = nullptr;
    if (h->opts.path != L2X_PATH_FUSED) return fail(L2X_EINVAL, "step graphs need the fused path");
    if (!(capacity_margin >= 1.0)) return fail(L2X_EINVAL, "capacity_margin must be >= 1");
    const int G = h->n_grids;
    L2X_TRY(check_ptrs(u_f_host, G, "u_f_host"));
    L2X_TRY(check_ptrs((const void* const*)u_s_host, G, "u_s_host"));
    L2X_TRY(check_ptrs(f_s_host, G, "f_s_host"));
    L2X_TRY(check_ptrs((const void* const*)f_f_host, G, "f_f_host"));
    if (!page_locked(coords_host)) return fail(L2X_EINVAL, "coords_host is not page-locked host memory");
    for (int g = 0; g < G; ++g)
        if (!page_locked(u_f_host[g]) || !page_locked(u_s_host[g]) || !page_locked(f_s_host[g]) ||
            !page_locked(f_f_host[g]))
            return fail(L2X_EINVAL, "a host array is not page-locked host memory (cudaHostAlloc / cudaHostRegister)");
    const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
    const int64_t n = h->n_nodes;
    HostIO io{};
    std::vector<void*> owned;
    void* uf[kMaxGrids];
    void* us[kMaxGrids];
    void* fs[kMaxGrids];
    void* ff[kMaxGrids];
    auto take = [&](void** p, size_t bytes) -> l2x_status {
        *p = nullptr;
        if (cudaMalloc(p, bytes ? bytes : 1) != cudaSuccess) {
            cudaGetLastError();
            for (void* q : owned) cudaFree(q);
            owned.clear();
            return fail(L2X_ENOMEM, "device copies of the host arrays");
        }
        owned.push_back(*p);
        return L2X_OK;
    };
    for (int g = 0; g < G; ++g) {
        const size_t nf = es * (size_t)fluid_nodes(h->sg[g]);
        L2X_TRY(take(&uf[g], nf));
        L2X_TRY(take(&ff[g], nf));
        L2X_TRY(take(&us[g], es * (size_t)n));
        L2X_TRY(take(&fs[g], es * (size_t)n));
        io.u_f[g] = u_f_host[g];
        io.u_s[g] = u_s_host[g];
        io.f_s[g] = f_s_host[g];
        io.f_f[g] = f_f_host[g];
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int g = 0; g < G; ++g) {  // defined values outside the boxes the replays copy
        const size_t nf = es * (size_t)fluid_nodes(h->sg[g]);
        if (cudaMemsetAsync(uf[g], 0, nf, s) != cudaSuccess || cudaMemsetAsync(ff[g], 0, nf, s) != cudaSuccess) {
            for (void* q : owned) cudaFree(q);
            return cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
        }
        // f_f = ...: only the box is written back by a replay, the rest is zeroed here
        if (zero_force) memset(f_f_host[g], 0, nf);
    }
    const l2x_status st = graph_create_common(h, coords_host, (const void* const*)uf, us, (const void* const*)fs, ff,
                                              capacity_margin, zero_force, stream, out, &io, owned);
    for (void* q : owned) cudaFree(q);  // left here only when the graph was not made
    if (st != L2X_OK) return st;
    int64_t box = 0;
    for (int g = 0; g < G; ++g) box += h->T[g].n_rows * (int64_t)es;
    (*out)->io_h2d = (int64_t)sizeof(double) * n * h->dim + box + (int64_t)es * n * G + (zero_force ? 0 : box);
    (*out)->io_d2h = (int64_t)es * n * G + box;
    return L2X_OK;
}

l2x_status l2x_graph_io_bytes(l2x_graph g, int64_t* h2d_bytes, int64_t* d2h_bytes) {
    if (!g || !h2d_bytes || !d2h_bytes) return fail(L2X_EINVAL, "NULL argument");
    *h2d_bytes = g->io_h2d;
    *d2h_bytes = g->io_d2h;
    return L2X_OK;
}

l2x_status l2x_graph_launch(l2x_graph g, void* stream) {
    if (!g) return fail(L2X_EINVAL, "NULL graph");
    if (g->gen != g->h->graph_gen)
        return fail(L2X_EINVAL, "the coupling was re-assembled (l2x_update_geometry) or captured again "
                                "(l2x_graph_create) after this graph was created; create the graph again");
    L2X_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return L2X_OK;
}

l2x_status l2x_graph_sync_status(l2x_graph g, void* stream) {
    if (!g) return fail(L2X_EINVAL, "NULL graph");
    l2x_coupling* h = g->h;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t np = 0;
    L2X_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaMemcpyAsync(&np, h->offsets + (int64_t)h->n_grids * h->n_elems, sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    h->n_pairs = np;  // candidate pairs of the last replay (l2x_query's n_pairs_total)
    const DevStatus& ds = *h->st_host;
    h->cg_iters = ds.cg_iters;
    h->cg_residual = ds.cg_residual;
    if (ds.flags & FLAG_CAPACITY)
        return fail(L2X_ECAPACITY, "the step needed more pairs or matrix entries than the graph's capacity; "
                                   "create the graph again (larger margin)");
    L2X_TRY(flags_to_status(ds));
    if (ds.flags & FLAG_NOTCONVERGED) return fail(L2X_ENOTCONVERGED, "CG did not reach cg_rtol in a captured step");
    return L2X_OK;
}

l2x_status l2x_graph_destroy(l2x_graph g) {
    if (!g) return L2X_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return L2X_OK;
}

l2x_status l2x_query(l2x_handle h, l2x_info* info) {
    if (!h || !info) return fail(L2X_EINVAL, "NULL handle or info");
    memset(info, 0, sizeof(*info));
    info->dim = h->dim;
    info->n_grids = h->n_grids;
    info->path = h->opts.path;
    info->precision = h->opts.precision;
    info->n_nodes = h->n_nodes;
    info->n_elems = h->n_elems;
    for (int g = 0; g < h->n_grids; ++g) {
        info->n_pairs[g] = h->pair_begin[g + 1] - h->pair_begin[g];
        info->nnz_B[g] = h->B[g].nnz;
        int64_t nf = 1;
        for (int k = 0; k < 3; ++k) {
            info->nnode[g][k] = h->sg[g].nnode[k];
            nf *= h->sg[g].nnode[k];
        }
        info->n_fluid[g] = nf;
    }
    info->n_pairs_total = h->n_pairs;
    info->nnz_M = h->M.nnz;
    info->cg_iters = h->cg_iters;
    info->cg_residual = h->cg_residual;
    info->clip_block = h->clip_block;
    info->pcg_rows_per_block = h->pcg_rpb;
    info->pcg_cluster = h->pcg_clu;
    info->multiplier = h->opts.multiplier;
    info->tuned_clip_ms = h->tuned_clip_ms;
    info->tuned_solve_ms = h->tuned_solve_ms;
    info->pcg_rows_per_block_step = h->pcg_rpb_step;
    info->clip_chunk = h->clip_chunk;
    resolve_timing(h);
    for (int p = 0; p < L2X_NPHASE; ++p) {
        info->phase_ms[p] = h->phase_ms[p];
        info->phase_calls[p] = h->phase_calls[p];
    }
    return L2X_OK;
}

l2x_status l2x_autotune(l2x_handle h, void* stream) {
    g_last_error.clear();
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    h->stream = s;
    const int64_t m = h->n_elems, n = h->n_nodes;
    const int G = h->n_grids, d = h->dim;
    cudaEvent_t a = nullptr, b = nullptr;
    L2X_CUDA(cudaEventCreate(&a));
    L2X_CUDA(cudaEventCreate(&b));
    auto timed = [&](auto&& fn) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a, s);
            fn();
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;  // first run warms up
        }
        return best;
    };
    l2x_status status = L2X_OK;
    if (h->opts.path == L2X_PATH_FUSED && h->n_pairs > 0) {
        // clip kernel: pairs per block and blocks' worth of pairs per work-queue
        // fetch, on the current pairs (class order of the last build)
        float best = 1e30f;
        int best_blk = h->clip_block, best_chunk = h->clip_chunk;
        for (int blk : {64, 128, 256})
            for (int chunk : {1, 4, 16}) {
                const float ms = timed([&] {
                    launch_clip_fused(d, h->opts.precision, G, h->sg, m, h->offsets, h->n_pairs, h->pair_cap, h->X,
                                      h->E, h->elem_grad, h->elem_flag, h->pair_elem, h->pair_cell, h->pair_perm,
                                      h->blocks, h->vols, h->st, s, blk, chunk, h->clip_work);
                });
                if (ms < best) {
                    best = ms;
                    best_blk = blk;
                    best_chunk = chunk;
                }
            }
        h->clip_block = best_blk;
        h->clip_chunk = best_chunk;
        h->tuned_clip_ms = best;
    }
    if (h->opts.multiplier == L2X_MULT_STANDARD) {
        // PCG: rows per block, on M applied to a vector of ones
        const size_t es = h->opts.precision == L2X_MIXED ? sizeof(float) : sizeof(double);
        void* y[kMaxGrids];
        void* w[kMaxGrids];
        char* tmp = nullptr;
        if (cudaMalloc((void**)&tmp, es * n * G * 4) != cudaSuccess) status = fail(L2X_ENOMEM, "autotune scratch");
        if (status == L2X_OK) {
            for (int g = 0; g < G; ++g) {
                y[g] = tmp + es * n * g;
                w[g] = tmp + es * n * (G + g);
            }
            // a fixed, non-smooth right-hand side (the iteration count then resembles a transfer's)
            std::vector<double> rhs(n);
            std::vector<float> rhsf(n);
            for (int64_t i = 0; i < n; ++i) {
                rhs[i] = 1.0 + 0.5 * std::sin(0.37 * (double)i);
                rhsf[i] = (float)rhs[i];
            }
            for (int g = 0; g < G; ++g)
                cudaMemcpyAsync(y[g], es == 8 ? (const void*)rhs.data() : (const void*)rhsf.data(), es * n,
                                cudaMemcpyHostToDevice, s);
            float best = 1e30f;
            int best_rpb = h->pcg_rpb, best_clu = 0;
            struct Shape { int rpb, clu; };
            std::vector<Shape> shapes;
            for (int rpb : {32, 64, 128, 256, 512, 1024}) shapes.push_back({rpb, 0});
            for (int clu : {8, 16})
                if (pcg_cluster_usable(h->opts.precision, n, G, clu)) shapes.push_back({h->pcg_rpb, clu});
            for (const Shape& sh : shapes) {
                const float ms = timed([&] {
                    solve_mass_pcg_async(h->opts.precision, h->M, h->M_dinv, h->M_dinv32, G, (const void* const*)y,
                                         w, h->opts.cg_rtol, h->opts.cg_max_iter, h->pcg_ws, h->st, s, sh.rpb, sh.clu);
                });
                if (ms < best) {
                    best = ms;
                    best_rpb = sh.rpb;
                    best_clu = sh.clu;
                }
            }
            h->pcg_rpb = best_rpb;
            h->pcg_clu = best_clu;
            h->tuned_solve_ms = best;
            if (h->opts.multiplier == L2X_MULT_STANDARD && 2 * G <= 6) {
                // the combined solve of a captured step (both transfers, 2G right-hand sides)
                const void* y2[2 * kMaxGrids];
                void* w2[2 * kMaxGrids];
                for (int g = 0; g < 2 * G; ++g) {
                    y2[g] = y[g % G];
                    w2[g] = tmp + es * n * (2 * G + g);
                }
                float best2 = 1e30f;
                int best2_rpb = h->pcg_rpb_step;
                for (int rpb : {32, 64, 128, 256, 512, 1024}) {
                    const float ms = timed([&] {
                        solve_mass_pcg_async(h->opts.precision, h->M, h->M_dinv, h->M_dinv32, 2 * G, y2, w2,
                                             h->opts.cg_rtol, h->opts.cg_max_iter, h->pcg_ws, h->st, s, rpb, 0);
                    });
                    if (ms < best2) {
                        best2 = ms;
                        best2_rpb = rpb;
                    }
                }
                h->pcg_rpb_step = best2_rpb;
            }
            cudaStreamSynchronize(s);
            cudaFree(tmp);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (status != L2X_OK) return status;
    L2X_CUDA(cudaGetLastError());
    return read_status(h, s);
}

l2x_status l2x_set_work_shape(l2x_handle h, int32_t clip_block, int32_t pcg_rows_per_block, int32_t pcg_cluster) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    if (clip_block != 64 && clip_block != 128 && clip_block != 256) return fail(L2X_EINVAL, "clip_block must be 64, 128 or 256");
    if (pcg_rows_per_block < 1 || pcg_rows_per_block > 4096) return fail(L2X_EINVAL, "pcg_rows_per_block must be in [1, 4096]");
    if (pcg_cluster != 0 && !pcg_cluster_usable(h->opts.precision, h->n_nodes, h->n_grids, pcg_cluster))
        return fail(L2X_EINVAL, "the system does not fit one cluster of that size");
    h->clip_block = clip_block;
    h->pcg_rpb = pcg_rows_per_block;
    h->pcg_rpb_step = pcg_rows_per_block;
    h->pcg_clu = pcg_cluster;
    return L2X_OK;
}

l2x_status l2x_set_clip_chunk(l2x_handle h, int32_t clip_chunk) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    if (clip_chunk < 1 || clip_chunk > 1024) return fail(L2X_EINVAL, "clip_chunk must be in [1, 1024]");
    h->clip_chunk = clip_chunk;
    return L2X_OK;
}

l2x_status l2x_set_step_work_shape(l2x_handle h, int32_t pcg_rows_per_block_step) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    if (pcg_rows_per_block_step < 1 || pcg_rows_per_block_step > 4096)
        return fail(L2X_EINVAL, "pcg_rows_per_block_step must be in [1, 4096]");
    h->pcg_rpb_step = pcg_rows_per_block_step;
    return L2X_OK;
}

l2x_status l2x_set_timing(l2x_handle h, int32_t enable) {
    if (!h) return fail(L2X_EINVAL, "NULL handle");
    resolve_timing(h);
    h->timing = enable != 0;
    if (enable)
        for (int p = 0; p < L2X_NPHASE; ++p) {
            h->phase_ms[p] = 0.0;
            h->phase_calls[p] = 0;
        }
    return L2X_OK;
}

int64_t l2x_kernel_launch_count(void) { return l2x::g_launches.load(); }

l2x_status l2x_export_pairs(l2x_handle h, int32_t grid, int32_t* elem, int32_t* cell, void* stream) {
    if (!h || !elem || !cell || grid < 0 || grid >= h->n_grids) return fail(L2X_EINVAL, "bad export_pairs arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t p0 = h->pair_begin[grid], np = h->pair_begin[grid + 1] - p0;
    L2X_CUDA(cudaMemcpyAsync(elem, h->pair_elem + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaMemcpyAsync(cell, h->pair_cell + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    return L2X_OK;
}

l2x_status l2x_export_pair_blocks(l2x_handle h, int32_t grid, double* blocks, double* vols, void* stream) {
    if (!h || !blocks || !vols || grid < 0 || grid >= h->n_grids) return fail(L2X_EINVAL, "bad export arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int NS = (h->dim + 1) << h->dim;
    int64_t p0 = h->pair_begin[grid], np = h->pair_begin[grid + 1] - p0;
    L2X_CUDA(cudaMemcpyAsync(vols, h->vols + p0, sizeof(double) * np, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaMemcpyAsync(blocks, h->blocks + p0 * NS, sizeof(double) * np * NS, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    return L2X_OK;
}

l2x_status l2x_export_pair_range(l2x_handle h, int32_t grid, int64_t e_first, int64_t n_elems,
                                 int64_t* first_pair, int64_t* n_pairs, int32_t* elem, int32_t* cell,
                                 double* blocks, double* vols, void* stream) {
    if (!h || grid < 0 || grid >= h->n_grids || e_first < 0 || n_elems < 0 || e_first + n_elems > h->n_elems)
        return fail(L2X_EINVAL, "bad export_pair_range arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = h->n_elems;
    int64_t p0 = 0, p1 = 0;
    L2X_CUDA(cudaMemcpyAsync(&p0, h->offsets + (int64_t)grid * m + e_first, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaMemcpyAsync(&p1, h->offsets + (int64_t)grid * m + e_first + n_elems, sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    const int64_t np = p1 - p0;
    if (first_pair) *first_pair = p0 - h->pair_begin[grid];
    if (n_pairs) *n_pairs = np;
    const int NS = (h->dim + 1) << h->dim;
    if (elem) L2X_CUDA(cudaMemcpyAsync(elem, h->pair_elem + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, s));
    if (cell) L2X_CUDA(cudaMemcpyAsync(cell, h->pair_cell + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, s));
    if (vols) L2X_CUDA(cudaMemcpyAsync(vols, h->vols + p0, sizeof(double) * np, cudaMemcpyDeviceToDevice, s));
    if (blocks)
        L2X_CUDA(cudaMemcpyAsync(blocks, h->blocks + p0 * NS, sizeof(double) * np * NS, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    return L2X_OK;
}

l2x_status l2x_export_csr(l2x_handle h, int32_t which, int64_t* row_ptr, int32_t* cols, double* vals, void* stream) {
    if (!h || !row_ptr || !cols || !vals) return fail(L2X_EINVAL, "bad export_csr arguments");
    const Csr* A = nullptr;
    if (which == L2X_MAT_M) A = &h->M;
    else if (which >= 0 && which < h->n_grids) A = &h->B[which];
    else return fail(L2X_EINVAL, "bad matrix id");
    cudaStream_t s = (cudaStream_t)stream;
    L2X_CUDA(cudaMemcpyAsync(row_ptr, A->ptr, sizeof(int64_t) * (A->n_rows + 1), cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaMemcpyAsync(cols, A->col, sizeof(int32_t) * A->nnz, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaMemcpyAsync(vals, A->val, sizeof(double) * A->nnz, cudaMemcpyDeviceToDevice, s));
    L2X_CUDA(cudaStreamSynchronize(s));
    return L2X_OK;
}

}  // extern "C"
