// Step (IV) of Sec. 2.3: assembly of the mortar matrices B_g (one per velocity
// grid) and S = M_s (P1 mass matrix, Sec. 2.1 "Spatial Discretization") into
// CSR, and the transpose of B_g used by the force transfer.
#include <algorithm>
#include <climits>

#include "l2x_internal.cuh"

namespace l2x {

namespace {

constexpr int kRowWarps = 4;
constexpr int kRowAdj = 64;     // incident elements staged in shared memory per warp
constexpr int kRowUnion = kRowKeep;  // nodes of a row's union box accumulated in shared memory per warp
constexpr int kMassMaxCand = 256;

__global__ void adj_count_kernel(int NA, int64_t total, const int32_t* __restrict__ E, int64_t* cnt) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    atomicAdd((unsigned long long*)(cnt + E[t]), 1ull);
}

__global__ void adj_fill_kernel(int NA, int64_t total, const int32_t* __restrict__ E,
                                const int64_t* __restrict__ ptr, int32_t* cursor, int32_t* adj) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= total) return;
    int64_t e = t / NA;
    int a = (int)(t - e * NA);
    int32_t node = E[t];
    int64_t pos = ptr[node] + atomicAdd(cursor + node, 1);
    adj[pos] = (int32_t)(e * 4 + a);
}

// insertion sort of every segment [ptr[i], ptr[i+1]) (short segments)
template <typename V>
__global__ void segment_sort_kernel(int64_t n, const int64_t* __restrict__ ptr, int32_t* key, V* val) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = ptr[i], hi = ptr[i + 1];
    for (int64_t a = lo + 1; a < hi; ++a) {
        int32_t k = key[a];
        V v = val ? val[a] : V(0);
        int64_t b = a - 1;
        while (b >= lo && key[b] > k) {
            key[b + 1] = key[b];
            if (val) val[b + 1] = val[b];
            --b;
        }
        key[b + 1] = k;
        if (val) val[b + 1] = v;
    }
}

// The node-box matrix of every (grid, element) slot (one launch covers the slots
// of all grids), stored as one plane per element vertex a (entry L of plane a at
// loc_val[a * loc_cap + L]).  Entry (a, node) sums block[a][corner] over the
// element's candidate cells around the node whose pair has a positive
// intersection volume, in ascending cell order (z, y, x): fixed order, so the
// result is reproducible.
//  * usual elements (at most 3 box nodes per axis, so at most 2^d cells): one
//    warp per element; the lanes load each pair's block as one coalesced run
//    (lane = block entry) and add it into the node box held in shared memory,
//    cell after cell (the entries of one block go to distinct (a, node));
//  * larger boxes: the warp's lanes take nodes of the box and sum over the
//    candidate cells around each.
constexpr int kLocWarps = 8;
constexpr int kLocBox = 27;  // nodes of a box with at most 3 per axis

// An element slot's header: its node box, local offsets and first pair.
struct LocHead {
    ElemBox b;
    int64_t L0, L1, q0;
};

__device__ __forceinline__ LocHead loc_head(int64_t e, const ElemBox* __restrict__ boxes,
                                            const int64_t* __restrict__ offsets, const int64_t* __restrict__ loc_off) {
    LocHead h;
    h.b = boxes[e];
    h.L0 = loc_off[e];
    h.L1 = loc_off[e + 1];
    h.q0 = offsets[e];
    return h;
}

// Persistent: warp w of the grid takes slots w, w + n_warps, ...; the next
// slot's header is loaded while the current slot is summed.
template <int D>
__global__ void __launch_bounds__(kLocWarps * 32) elem_local_kernel(
    int64_t m, const ElemBox* __restrict__ boxes, const int64_t* __restrict__ offsets,
    const int64_t* __restrict__ loc_off, int64_t loc_cap, const double* __restrict__ blocks,
    const double* __restrict__ vols, double* __restrict__ loc_val, uint8_t* __restrict__ loc_flag, int dual,
    DevStatus* st) {
    constexpr int NA = D + 1, NB = 1 << D, NS = NA * NB;
    constexpr int kCells = 1 << D;  // cells of a usual box
    __shared__ double s_acc[kLocWarps][NA][kLocBox];
    __shared__ uint8_t s_hit[kLocWarps][kLocBox];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (st->flags & kAbortFlags) return;
    const int64_t stride = (int64_t)gridDim.x * kLocWarps;
    int64_t e = blockIdx.x * (int64_t)kLocWarps + w;
    if (e >= m) return;
    LocHead cur = loc_head(e, boxes, offsets, loc_off);
    for (; e < m; e += stride) {
        const LocHead nxt = e + stride < m ? loc_head(e + stride, boxes, offsets, loc_off) : cur;
        const ElemBox b = cur.b;
        const int ex = box_ext(b, 0), ey = box_ext(b, 1), ez = D == 3 ? box_ext(b, 2) : 1;
        const int64_t L0 = cur.L0, L1 = cur.L1, q0 = cur.q0;
        cur = nxt;
        if (L1 == L0) continue;
        if (L1 > loc_cap) {
            if (lane == 0) atomicOr(&st->flags, FLAG_CAPACITY);
            return;
        }
        const int nbx = ex + 1, nby = ey + 1;
        const int64_t nbox = L1 - L0;
        if (ex <= 2 && ey <= 2 && ez <= 2) {
            for (int j = lane; j < nbox; j += 32) {
#pragma unroll
                for (int a = 0; a < NA; ++a) s_acc[w][a][j] = 0.0;
                s_hit[w][j] = 0;
            }
            __syncwarp();
            const int ncell = ex * ey * ez;
            const bool act = lane < NS;
            const int a = lane / NB, cb = lane % NB;  // this lane's block entry block[a][cb]
            const int bx = cb & 1, by = (cb >> 1) & 1, bz = D == 3 ? cb >> 2 : 0;
            // every pair's loads first (at most 2^d pairs), then the sums in cell order
            double v[kCells];
            bool live[kCells];
#pragma unroll
            for (int c = 0; c < kCells; ++c) {
                v[c] = 0.0;
                live[c] = false;
                if (c < ncell) {
                    const int64_t q = q0 + c;
                    live[c] = __double_as_longlong(vols[q]) > 0;  // volume > 0
                    if (act) v[c] = blocks[q * NS + lane];
                }
            }
#pragma unroll
            for (int c = 0; c < kCells; ++c) {
                if (c < ncell && live[c]) {
                    // cell c = cx + ex (cy + ey cz) with ex, ey in {1, 2}
                    const int cx = ex == 2 ? (c & 1) : 0, r = ex == 2 ? c >> 1 : c;
                    const int cy = ey == 2 ? (r & 1) : 0, cz = ey == 2 ? r >> 1 : r;
                    const int jj = (cx + bx) + nbx * ((cy + by) + nby * (cz + bz));
                    if (act) s_acc[w][a][jj] += v[c];
                    if (act && a == 0) s_hit[w][jj] = 1;
                }
                __syncwarp();
            }
            for (int j = lane; j < nbox; j += 32) {
                double acc[NA];
#pragma unroll
                for (int a2 = 0; a2 < NA; ++a2) acc[a2] = s_acc[w][a2][j];
                if (dual) {
                    // dual multiplier basis (d+2) lambda_a - 1: the lambda integrals sum
                    // to the integral of psi (partition of unity of the barycentrics)
                    double sum = 0.0;
#pragma unroll
                    for (int a2 = 0; a2 < NA; ++a2) sum += acc[a2];
#pragma unroll
                    for (int a2 = 0; a2 < NA; ++a2) acc[a2] = (double)(D + 2) * acc[a2] - sum;
                }
                loc_flag[L0 + j] = s_hit[w][j];
#pragma unroll
                for (int a2 = 0; a2 < NA; ++a2) loc_val[a2 * loc_cap + L0 + j] = acc[a2];
            }
            __syncwarp();  // the box is read out before the next slot clears it
            continue;
        }
        for (int64_t jj = lane; jj < nbox; jj += 32) {
            const int jx = (int)(jj % nbx);
            const int64_t r = jj / nbx;
            const int jy = (int)(r % nby), jz = (int)(r / nby);
            double acc[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] = 0.0;
            bool touched = false;
            const int cz0 = D == 3 ? max(jz - 1, 0) : 0, cz1 = D == 3 ? min(jz, ez - 1) : 0;
            for (int cz = cz0; cz <= cz1; ++cz)
                for (int cy = max(jy - 1, 0); cy <= min(jy, ey - 1); ++cy)
                    for (int cx = max(jx - 1, 0); cx <= min(jx, ex - 1); ++cx) {
                        const int64_t q = q0 + cx + (int64_t)ex * (cy + (int64_t)ey * cz);
                        if (__double_as_longlong(vols[q]) > 0) {  // volume > 0
                            touched = true;
                            const int cb = (jx - cx) | ((jy - cy) << 1) | (D == 3 ? (jz - cz) << 2 : 0);
                            const double* blk = blocks + q * NS + cb;
#pragma unroll
                            for (int a = 0; a < NA; ++a) acc[a] += blk[a * NB];
                        }
                    }
            if (dual) {
                double sum = 0.0;
#pragma unroll
                for (int a = 0; a < NA; ++a) sum += acc[a];
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[a] = (double)(D + 2) * acc[a] - sum;
            }
            loc_flag[L0 + jj] = touched ? 1 : 0;
#pragma unroll
            for (int a = 0; a < NA; ++a) loc_val[a * loc_cap + L0 + jj] = acc[a];
        }
    }
}

// One warp per solid node i of one grid g (row i of B_g); the rows of the n_grids
// matrices share one launch, warp r taking row r % n_nodes of grid r / n_nodes.
// The row's columns lie in the union of the node boxes of the incident elements.
// Entry (i, j) sums, in adjacency order, the entry (local vertex of i, node j)
// of each incident element's node-box matrix, so the result is reproducible and
// needs no atomics:
//  * usual rows (at most kRowAdj incident elements, a union box of at most
//    kRowUnion nodes, element boxes of at most 3 nodes per axis): the warp walks
//    the incident elements in adjacency order, its lanes covering the element's
//    box nodes, and adds into the union box held in shared memory (distinct
//    nodes within one element; __syncwarp between elements).  The counting pass
//    keeps the row (union box, touched mask, sums) in the cache, from which the
//    emitting pass writes it;
//  * other rows: every lane owns columns j of the union box and loops over the
//    incident elements, in both passes.
// Touched columns are emitted in ascending order.
// pass 0: row_count[i] = number of touched columns; pass 1: columns and values;
// pass 2: columns only, values zeroed (the plain path adds them with atomics).
struct RowsSet {
    RowsGrid g[kMaxGrids];
};

constexpr int kRowGroup = 8;  // incident elements whose loads are issued together

template <int D>
__global__ void __launch_bounds__(kRowWarps * 32, 8) b_rows_kernel(
    int pass, int n_grids, RowsSet rs, int64_t n_nodes, const int64_t* __restrict__ adj_ptr,
    const int32_t* __restrict__ adj, const double* __restrict__ loc_val, int64_t loc_cap,
    const uint8_t* __restrict__ loc_flag, DevStatus* st) {
    __shared__ ElemBox s_box[kRowWarps][kRowAdj];
    __shared__ int64_t s_off[kRowWarps][kRowAdj];
    __shared__ int32_t s_ea[kRowWarps][kRowAdj];
    __shared__ double s_acc[kRowWarps][kRowUnion];
    __shared__ uint8_t s_hit[kRowWarps][kRowUnion];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r_all = blockIdx.x * (int64_t)kRowWarps + w;
    if (r_all >= n_grids * n_nodes) return;
    if (st->flags & kAbortFlags) return;  // a captured step whose pairs or entries did not fit
    const int g = (int)(r_all / n_nodes);
    const int64_t i = r_all - g * n_nodes;
    const RowsGrid& rg = rs.g[g];
    RowCache* __restrict__ rc = rg.cache + i;
    int64_t cnt = 0;
    const int64_t out0 = pass >= 1 ? rg.row_ptr[i] : 0;
    if (pass >= 1) {
        const int dims = rc->dims;
        if (dims != 0) {  // kept by the counting pass
            const int nx = dims & 255, ny = (dims >> 8) & 255, nz = dims >> 16;
            const int total = nx * ny * nz;
            const int lo0 = rc->lo[0], lo1 = rc->lo[1], lo2 = rc->lo[2];
            for (int base = 0; base < total; base += 32) {
                const unsigned bal = rc->hit[base >> 5];
                if ((bal >> lane) & 1u) {
                    const int idx = base + lane;
                    const int jx = lo0 + idx % nx, r = idx / nx;
                    const int jy = lo1 + r % ny, jz = lo2 + r / ny;
                    const int pos = __popc(bal & ((1u << lane) - 1u));
                    rg.cols[out0 + cnt + pos] = jx + rg.nnode0 * (jy + rg.nnode1 * jz);
                    rg.vals[out0 + cnt + pos] = pass == 1 ? rc->val[idx] : 0.0;
                }
                cnt += __popc(bal);
            }
            return;
        }
    }
    const ElemBox* __restrict__ boxes = rg.boxes;
    const int64_t* __restrict__ loc_off = rg.loc_off;
    const int64_t a0 = adj_ptr[i], a1 = adj_ptr[i + 1];
    const bool staged = a1 - a0 <= kRowAdj;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    bool wide = false;  // an element box with more than 3 nodes on some axis
    for (int64_t t = a0 + lane; t < a1; t += 32) {
        const int32_t ea = adj[t];
        const int32_t e = ea >> 2;
        const ElemBox b = boxes[e];
        if (staged) {
            s_box[w][t - a0] = b;
            s_off[w][t - a0] = loc_off[e];
            s_ea[w][t - a0] = ea;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            lo[k] = min(lo[k], b.lo[k]);
            hi[k] = max(hi[k], b.lo[k] + box_ext(b, k));
            wide |= box_ext(b, k) > 2;
        }
    }
    wide = __any_sync(0xffffffffu, wide);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < D; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if (D == 2) {
        lo[2] = 0;
        hi[2] = 0;
    }
    bool kept = false;
    if (a0 < a1) {
        const int nx = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1, nz = hi[2] - lo[2] + 1;
        const int64_t total = (int64_t)nx * ny * nz;
        if (staged && !wide && total <= kRowUnion) {
            kept = pass == 0;
            for (int u = lane; u < total; u += 32) {
                s_acc[w][u] = 0.0;
                s_hit[w][u] = 0;
            }
            // per staged element, packed in place of its (element, vertex) word: the
            // union-box index of its box corner (< kRowUnion), its box extents (<= 2)
            // and the local vertex
            for (int64_t t = a0 + lane; t < a1; t += 32) {
                const ElemBox b = s_box[w][t - a0];
                const int u0 = (b.lo[0] - lo[0]) + nx * ((b.lo[1] - lo[1]) + ny * (D == 3 ? b.lo[2] - lo[2] : 0));
                const int ez = D == 3 ? box_ext(b, 2) : 0;
                s_ea[w][t - a0] = u0 | (box_ext(b, 0) << 8) | (box_ext(b, 1) << 10) | (ez << 12) |
                                  ((s_ea[w][t - a0] & 3) << 14);
            }
            __syncwarp();
            // this lane's node of an element box (at most 3 nodes per axis) and its
            // offset in the union box
            const int lx = lane % 3, ly = (lane / 3) % 3, lz = D == 3 ? lane / 9 : 0;
            const bool lane_ok = lane < (D == 3 ? 27 : 9);
            const int lane_u = lx + nx * (ly + ny * lz);
            for (int64_t t0 = a0; t0 < a1; t0 += kRowGroup) {
                int u[kRowGroup];
                uint8_t f[kRowGroup];
                double v[kRowGroup];
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    u[q] = -1;
                    f[q] = 0;
                    v[q] = 0.0;
                    const int64_t t = t0 + q;
                    if (t >= a1 || !lane_ok) continue;
                    const int pk = s_ea[w][t - a0];
                    const int ex = (pk >> 8) & 3, ey = (pk >> 10) & 3, ez = (pk >> 12) & 3;
                    if (lx > ex || ly > ey || lz > ez) continue;
                    const int64_t L = s_off[w][t - a0] + lx + (ex + 1) * (ly + (ey + 1) * lz);
                    u[q] = (pk & 255) + lane_u;
                    f[q] = loc_flag[L];
                    // the element-local matrices hold exact zeros at untouched nodes, so
                    // the value is read without waiting for the flag (same sums)
                    if (pass != 2) v[q] = loc_val[(int64_t)(pk >> 14) * loc_cap + L];
                }
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    if (u[q] >= 0) {
                        if (pass != 2) s_acc[w][u[q]] += v[q];
                        if (f[q]) s_hit[w][u[q]] = 1;
                    }
                    __syncwarp();
                }
            }
            for (int base = 0; base < (int)total; base += 32) {
                const int idx = base + lane;
                const bool touched = idx < total && s_hit[w][idx] != 0;
                const unsigned bal = __ballot_sync(0xffffffffu, touched);
                if (kept) {
                    if (lane == 0) rc->hit[base >> 5] = bal;
                    if (touched) rc->val[idx] = s_acc[w][idx];
                } else if (pass >= 1 && touched) {
                    const int jx = lo[0] + idx % nx, r = idx / nx;
                    const int jy = lo[1] + r % ny, jz = lo[2] + r / ny;
                    const int pos = __popc(bal & ((1u << lane) - 1u));
                    rg.cols[out0 + cnt + pos] = jx + rg.nnode0 * (jy + rg.nnode1 * jz);
                    rg.vals[out0 + cnt + pos] = pass == 1 ? s_acc[w][idx] : 0.0;
                }
                cnt += __popc(bal);
            }
            if (kept && lane == 0) {
                rc->lo[0] = lo[0];
                rc->lo[1] = lo[1];
                rc->lo[2] = lo[2];
                rc->dims = nx | (ny << 8) | (nz << 16);
            }
        } else {
            for (int64_t base = 0; base < total; base += 32) {
                const int64_t idx = base + lane;
                bool touched = false;
                double acc = 0.0;
                int jx = 0, jy = 0, jz = 0;
                if (idx < total) {
                    jx = lo[0] + (int)(idx % nx);
                    const int64_t r = idx / nx;
                    jy = lo[1] + (int)(r % ny);
                    jz = lo[2] + (int)(r / ny);
#pragma unroll 4
                    for (int64_t t = a0; t < a1; ++t) {
                        const int32_t ea = staged ? s_ea[w][t - a0] : adj[t];
                        const ElemBox b = staged ? s_box[w][t - a0] : boxes[ea >> 2];
                        const int ux = jx - b.lo[0], uy = jy - b.lo[1], uz = D == 3 ? jz - b.lo[2] : 0;
                        const int ex = box_ext(b, 0), ey = box_ext(b, 1), ez = box_ext(b, 2);
                        if (ux < 0 || ux > ex || uy < 0 || uy > ey || uz < 0 || (D == 3 && uz > ez)) continue;
                        const int64_t L0 = staged ? s_off[w][t - a0] : loc_off[ea >> 2];
                        const int64_t li = L0 + ux + (int64_t)(ex + 1) * (uy + (int64_t)(ey + 1) * uz);
                        touched |= loc_flag[li] != 0;
                        if (pass == 1) acc += loc_val[(int64_t)(ea & 3) * loc_cap + li];
                    }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, touched);
                if (pass >= 1 && touched) {
                    const int pos = __popc(bal & ((1u << lane) - 1u));
                    rg.cols[out0 + cnt + pos] = jx + rg.nnode0 * (jy + rg.nnode1 * jz);
                    rg.vals[out0 + cnt + pos] = pass == 1 ? acc : 0.0;
                }
                cnt += __popc(bal);
            }
        }
    }
    if (pass == 0 && lane == 0) {
        if (!kept) rc->dims = 0;
        rg.row_count[i] = cnt;
    }
}

template <int D>
__global__ void mass_structure_kernel(int pass, int64_t n_nodes, const int32_t* __restrict__ E,
                                      const int64_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                                      int64_t* row_count, const int64_t* __restrict__ row_ptr, int32_t* cols,
                                      DevStatus* st) {
    constexpr int NA = D + 1;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    int32_t cand[kMassMaxCand];
    int n = 0;
    bool overflow = false;
    for (int64_t t = adj_ptr[i]; t < adj_ptr[i + 1]; ++t) {
        int32_t e = adj[t] >> 2;
        for (int v = 0; v < NA; ++v) {
            int32_t j = E[(int64_t)e * NA + v];
            // insert keeping cand sorted and unique
            int p = n;
            bool dup = false;
            while (p > 0 && cand[p - 1] >= j) {
                if (cand[p - 1] == j) { dup = true; break; }
                --p;
            }
            if (dup) continue;
            if (n == kMassMaxCand) { overflow = true; continue; }
            for (int q = n; q > p; --q) cand[q] = cand[q - 1];
            cand[p] = j;
            ++n;
        }
    }
    if (overflow) atomicOr(&st->flags, FLAG_CAPACITY);
    if (pass == 0) {
        row_count[i] = n;
    } else {
        int64_t o = row_ptr[i];
        for (int q = 0; q < n; ++q) cols[o + q] = cand[q];
    }
}

template <int D>
__global__ void mass_values_kernel(int64_t n_nodes, const int32_t* __restrict__ E, const int64_t* __restrict__ adj_ptr,
                                   const int32_t* __restrict__ adj, const double* __restrict__ elem_vol,
                                   const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cols,
                                   double* vals, double* diag_inv) {
    constexpr int NA = D + 1;
    const double w = 1.0 / ((D + 1) * (D + 2));
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    const int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
    for (int64_t q = lo; q < hi; ++q) vals[q] = 0.0;
    for (int64_t t = adj_ptr[i]; t < adj_ptr[i + 1]; ++t) {
        const int32_t e = adj[t] >> 2;
        const int a = adj[t] & 3;
        const double ve = elem_vol[e] * w;
        for (int v = 0; v < NA; ++v) {
            const int32_t j = E[(int64_t)e * NA + v];
            int64_t l = lo, r = hi;
            while (l < r) {
                int64_t mid = (l + r) >> 1;
                if (cols[mid] < j) l = mid + 1; else r = mid;
            }
            if (l < hi && cols[l] == j) vals[l] += v == a ? 2.0 * ve : ve;
        }
    }
    double dgl = 0.0;
    for (int64_t q = lo; q < hi; ++q)
        if (cols[q] == (int32_t)i) dgl = vals[q];
    diag_inv[i] = dgl > 0.0 ? 1.0 / dgl : 0.0;
}

// Thread per solid node: S_ii = sum of |E|/(d+1) over the elements around i, in
// adjacency order (reproducible); the diagonal CSR structure is rewritten too.
template <int D>
__global__ void lumped_mass_kernel(int64_t n_nodes, const int64_t* __restrict__ adj_ptr,
                                   const int32_t* __restrict__ adj, const double* __restrict__ elem_vol,
                                   int64_t* row_ptr, int32_t* cols, double* vals, double* diag_inv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    double s = 0.0;
    for (int64_t t = adj_ptr[i]; t < adj_ptr[i + 1]; ++t) s += elem_vol[adj[t] >> 2];
    s = s / (double)(D + 1);
    row_ptr[i] = i;
    if (i == n_nodes - 1) row_ptr[n_nodes] = n_nodes;
    cols[i] = (int32_t)i;
    vals[i] = s;
    diag_inv[i] = s > 0.0 ? 1.0 / s : 0.0;
}

__device__ __forceinline__ int64_t tbox_index(const SubGrid& sg, const CsrT& T, int32_t j) {
    int x = j % sg.nnode[0];
    int r = j / sg.nnode[0];
    int y = r % sg.nnode[1];
    int z = r / sg.nnode[1];
    return (x - T.lo[0]) + (int64_t)T.n[0] * ((y - T.lo[1]) + (int64_t)T.n[1] * (z - T.lo[2]));
}

// Warp per row of B_g: count the entries of every B_g^T row.
__global__ void transpose_count_kernel(int64_t n_rows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                       SubGrid sg, CsrT T, int64_t* cnt, const DevStatus* st) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n_rows || (st->flags & kAbortFlags)) return;
    for (int64_t q = ptr[i] + lane; q < ptr[i + 1]; q += 32)
        atomicAdd((unsigned long long*)(cnt + tbox_index(sg, T, col[q])), 1ull);
}

// Warp per row of B_g: scatter (row, value) into the B_g^T rows (order fixed later).
__global__ void transpose_fill_kernel(int64_t n_rows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                      const double* __restrict__ val, SubGrid sg, CsrT T, int32_t* cursor,
                                      const DevStatus* st) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n_rows || (st->flags & kAbortFlags)) return;
    for (int64_t q = ptr[i] + lane; q < ptr[i + 1]; q += 32) {
        const int64_t r = tbox_index(sg, T, col[q]);
        const int64_t pos = T.ptr[r] + atomicAdd(cursor + r, 1);
        T.col[pos] = (int32_t)i;
        T.val[pos] = val[q];
    }
}

// Warp per B_g^T row: the keys (solid nodes) of a row are distinct, so every
// entry's final position is its rank, counted against the row staged in shared
// memory.  Rows longer than the staging area are sorted in place by one lane.
constexpr int kSortWarps = 4;
constexpr int kSortMax = 512;      // rows up to this length: one warp, shared memory
constexpr int kSortLong = 256;     // threads per block for longer rows
constexpr int kSortLongMax = 8192; // rows up to this length: one block, dynamic shared memory

__global__ void __launch_bounds__(kSortWarps * 32) transpose_sort_kernel(const int32_t* __restrict__ list,
                                                                        const int64_t* __restrict__ n_list,
                                                                        const int64_t* __restrict__ ptr,
                                                                        int32_t* key, double* val, const DevStatus* st,
                                                                        int32_t* long_rows, int32_t* n_long,
                                                                        int64_t long_cap) {
    __shared__ int32_t sk[kSortWarps][kSortMax];
    __shared__ double sv[kSortWarps][kSortMax];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (st->flags & kAbortFlags) return;
    const int64_t nl = *n_list;
    // grid-stride over the listed rows (the launch is sized for the SMs, not for
    // the row capacity, which inside a captured step covers the whole grid)
    for (int64_t li = blockIdx.x * (int64_t)kSortWarps + w; li < nl; li += (int64_t)gridDim.x * kSortWarps) {
        const int64_t i = list[li];
        const int64_t lo = ptr[i], hi = ptr[i + 1];
        const int len = (int)(hi - lo);
        if (len <= 1) continue;
        if (len <= kSortMax) {
            __syncwarp();
            for (int a = lane; a < len; a += 32) {
                sk[w][a] = key[lo + a];
                sv[w][a] = val[lo + a];
            }
            __syncwarp();
            for (int a = lane; a < len; a += 32) {
                const int32_t k = sk[w][a];
                int rank = 0;
                for (int b = 0; b < len; ++b) rank += sk[w][b] < k;
                key[lo + rank] = k;
                val[lo + rank] = sv[w][a];
            }
            continue;
        }
        // longer rows: sorted by transpose_sort_long_kernel, one block each
        if (lane == 0) {
            const int32_t slot = atomicAdd(n_long, 1);
            if (slot < long_cap) long_rows[slot] = (int32_t)i;
        }
    }
}

// Block per long row of B_g^T: rank sort of up to kSortLongMax entries staged in
// dynamic shared memory; still longer rows are sorted in place by one thread.
__global__ void __launch_bounds__(kSortLong) transpose_sort_long_kernel(const int32_t* __restrict__ long_rows,
                                                                       const int32_t* __restrict__ n_long,
                                                                       int64_t long_cap,
                                                                       const int64_t* __restrict__ ptr, int32_t* key,
                                                                       double* val, const DevStatus* st) {
    extern __shared__ unsigned char smem[];
    double* sv = reinterpret_cast<double*>(smem);
    int32_t* sk = reinterpret_cast<int32_t*>(smem + sizeof(double) * kSortLongMax);
    const int64_t b = blockIdx.x;
    if (b >= min((int64_t)*n_long, long_cap) || (st->flags & kAbortFlags)) return;
    const int64_t r = long_rows[b];
    const int64_t lo = ptr[r], hi = ptr[r + 1];
    const int len = (int)(hi - lo);
    if (len <= kSortLongMax) {
        for (int a = threadIdx.x; a < len; a += blockDim.x) {
            sk[a] = key[lo + a];
            sv[a] = val[lo + a];
        }
        __syncthreads();
        for (int a = threadIdx.x; a < len; a += blockDim.x) {
            const int32_t k = sk[a];
            int rank = 0;
            for (int c = 0; c < len; ++c) rank += sk[c] < k;
            key[lo + rank] = k;
            val[lo + rank] = sv[a];
        }
        return;
    }
    if (threadIdx.x != 0) return;
    for (int64_t a = lo + 1; a < hi; ++a) {
        const int32_t kk = key[a];
        const double vv = val[a];
        int64_t c = a - 1;
        while (c >= lo && key[c] > kk) {
            key[c + 1] = key[c];
            val[c + 1] = val[c];
            --c;
        }
        key[c + 1] = kk;
        val[c + 1] = vv;
    }
}

__global__ void nonempty_flags_kernel(int64_t n, const int64_t* __restrict__ counts, int64_t* flags,
                                      const DevStatus* st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (st->flags & kAbortFlags) ? 0 : (counts[i] > 0 ? 1 : 0);
}

__global__ void nonempty_list_kernel(int64_t n, const int64_t* __restrict__ counts, const int64_t* __restrict__ pos,
                                     int64_t list_cap, int32_t* list, int64_t* n_list, const DevStatus* st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *n_list = min(pos[n], list_cap);
    if (i >= n || (st->flags & kAbortFlags)) return;
    if (counts[i] > 0 && pos[i] < list_cap) list[pos[i]] = (int32_t)i;
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_node_adjacency(int dim, int64_t n_nodes, int64_t m, const int32_t* E, int64_t* adj_ptr,
                           int32_t* adj, int32_t* cursor, void* scan_tmp, cudaStream_t s) {
    const int NA = dim + 1;
    const int64_t total = m * NA;
    cudaMemsetAsync(adj_ptr, 0, sizeof(int64_t) * (n_nodes + 1), s);
    cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n_nodes, s);
    if (total > 0) { adj_count_kernel<<<nblk(total, 256), 256, 0, s>>>(NA, total, E, adj_ptr); count_launch(); }
    launch_scan_i64(adj_ptr, adj_ptr, n_nodes, scan_tmp, s);
    if (total > 0) { adj_fill_kernel<<<nblk(total, 256), 256, 0, s>>>(NA, total, E, adj_ptr, cursor, adj); count_launch(); }
    { segment_sort_kernel<double><<<nblk(n_nodes, 128), 128, 0, s>>>(n_nodes, adj_ptr, adj, nullptr); count_launch(); }
}

void launch_elem_local(int dim, int64_t m, const ElemBox* boxes_g, const int64_t* offsets_g,
                       const int64_t* loc_off_g, int64_t loc_cap, const double* blocks, const double* vols,
                       double* loc_val, uint8_t* loc_flag, int dual, DevStatus* st, cudaStream_t s) {
    if (m <= 0) return;
    // persistent grid: the blocks resident on the SMs at once (counted once per form)
    static int resident[2] = {0, 0};
    if (resident[dim == 3] == 0) {
        int dev = 0, n_sm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (dim == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, elem_local_kernel<2>, kLocWarps * 32, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, elem_local_kernel<3>, kLocWarps * 32, 0);
        resident[dim == 3] = std::max(1, n_sm) * std::max(1, per);
    }
    const unsigned nb = (unsigned)std::min<int64_t>(nblk(m, kLocWarps), resident[dim == 3]);
    if (dim == 2) { elem_local_kernel<2><<<nb, kLocWarps * 32, 0, s>>>(m, boxes_g, offsets_g, loc_off_g, loc_cap, blocks, vols, loc_val, loc_flag, dual, st); count_launch(); }
    else { elem_local_kernel<3><<<nb, kLocWarps * 32, 0, s>>>(m, boxes_g, offsets_g, loc_off_g, loc_cap, blocks, vols, loc_val, loc_flag, dual, st); count_launch(); }
}

void launch_b_rows(int pass, int dim, int n_grids, const RowsGrid* grids, int64_t n_nodes, const int64_t* adj_ptr,
                   const int32_t* adj, const double* loc_val, int64_t loc_cap, const uint8_t* loc_flag,
                   DevStatus* st, cudaStream_t s) {
    if (n_nodes <= 0 || n_grids <= 0) return;
    RowsSet rs{};
    for (int g = 0; g < n_grids; ++g) rs.g[g] = grids[g];
    const unsigned nb = nblk(n_grids * n_nodes, kRowWarps);
    if (dim == 2)
        { b_rows_kernel<2><<<nb, kRowWarps * 32, 0, s>>>(pass, n_grids, rs, n_nodes, adj_ptr, adj, loc_val, loc_cap, loc_flag, st); count_launch(); }
    else
        { b_rows_kernel<3><<<nb, kRowWarps * 32, 0, s>>>(pass, n_grids, rs, n_nodes, adj_ptr, adj, loc_val, loc_cap, loc_flag, st); count_launch(); }
}

void launch_mass_structure(int pass, int dim, int64_t n_nodes, const int32_t* E, const int64_t* adj_ptr,
                           const int32_t* adj, int64_t* row_count, const int64_t* row_ptr, int32_t* cols,
                           DevStatus* st, cudaStream_t s) {
    if (n_nodes <= 0) return;
    if (dim == 2)
        { mass_structure_kernel<2><<<nblk(n_nodes, 128), 128, 0, s>>>(pass, n_nodes, E, adj_ptr, adj, row_count, row_ptr, cols, st); count_launch(); }
    else
        { mass_structure_kernel<3><<<nblk(n_nodes, 128), 128, 0, s>>>(pass, n_nodes, E, adj_ptr, adj, row_count, row_ptr, cols, st); count_launch(); }
}

void launch_mass_values(int dim, int64_t n_nodes, const int32_t* E, const int64_t* adj_ptr,
                        const int32_t* adj, const double* elem_vol, const int64_t* row_ptr,
                        const int32_t* cols, double* vals, double* diag_inv, cudaStream_t s) {
    if (n_nodes <= 0) return;
    if (dim == 2)
        { mass_values_kernel<2><<<nblk(n_nodes, 128), 128, 0, s>>>(n_nodes, E, adj_ptr, adj, elem_vol, row_ptr, cols, vals, diag_inv); count_launch(); }
    else
        { mass_values_kernel<3><<<nblk(n_nodes, 128), 128, 0, s>>>(n_nodes, E, adj_ptr, adj, elem_vol, row_ptr, cols, vals, diag_inv); count_launch(); }
}

void launch_lumped_mass(int dim, int64_t n_nodes, const int64_t* adj_ptr, const int32_t* adj,
                        const double* elem_vol, int64_t* row_ptr, int32_t* cols, double* vals, double* diag_inv,
                        cudaStream_t s) {
    if (n_nodes <= 0) return;
    if (dim == 2)
        { lumped_mass_kernel<2><<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, adj_ptr, adj, elem_vol, row_ptr, cols, vals, diag_inv); count_launch(); }
    else
        { lumped_mass_kernel<3><<<nblk(n_nodes, 256), 256, 0, s>>>(n_nodes, adj_ptr, adj, elem_vol, row_ptr, cols, vals, diag_inv); count_launch(); }
}

void launch_transpose_count(const Csr& B, const SubGrid& sg, const CsrT& T, int64_t* cnt, const DevStatus* st,
                            cudaStream_t s) {
    cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (T.n_rows + 1), s);
    if (B.n_rows > 0) { transpose_count_kernel<<<nblk(B.n_rows * 32, 256), 256, 0, s>>>(B.n_rows, B.ptr, B.col, sg, T, cnt, st); count_launch(); }
}

void launch_transpose_fill(const Csr& B, const SubGrid& sg, const CsrT& T, int32_t* cursor, const DevStatus* st,
                           cudaStream_t s) {
    cudaMemsetAsync(cursor, 0, sizeof(int32_t) * T.n_rows, s);
    if (B.n_rows > 0)
        { transpose_fill_kernel<<<nblk(B.n_rows * 32, 256), 256, 0, s>>>(B.n_rows, B.ptr, B.col, B.val, sg, T, cursor, st); count_launch(); }
}

void launch_transpose_sort(const CsrT& T, const DevStatus* st, cudaStream_t s) {
    const int64_t n = T.list_cap < T.n_rows ? T.list_cap : T.n_rows;
    if (n <= 0) return;
    cudaMemsetAsync(T.n_long, 0, sizeof(int32_t), s);
    unsigned nb = nblk(n, kSortWarps);
    if (nb > 152 * 16) nb = 152 * 16;
    { transpose_sort_kernel<<<nb, kSortWarps * 32, 0, s>>>(T.list, T.n_list, T.ptr, T.col, T.val, st, T.long_rows, T.n_long, T.long_cap); count_launch(); }
    static bool attr_set = false;
    const int smem = (int)((sizeof(double) + sizeof(int32_t)) * kSortLongMax);
    if (!attr_set) {
        cudaFuncSetAttribute(transpose_sort_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    if (T.long_cap > 0) { transpose_sort_long_kernel<<<(unsigned)T.long_cap, kSortLong, smem, s>>>(T.long_rows, T.n_long, T.long_cap, T.ptr, T.col, T.val, st); count_launch(); }
}

void launch_transpose_list(const CsrT& T, const int64_t* counts, int64_t* flags, void* scan_tmp,
                           const DevStatus* st, cudaStream_t s) {
    if (T.n_rows <= 0) return;
    { nonempty_flags_kernel<<<nblk(T.n_rows, 256), 256, 0, s>>>(T.n_rows, counts, flags, st); count_launch(); }
    launch_scan_i64(flags, flags, T.n_rows, scan_tmp, s);
    { nonempty_list_kernel<<<nblk(T.n_rows, 256), 256, 0, s>>>(T.n_rows, counts, flags, T.list_cap, T.list, T.n_list, st); count_launch(); }
}

void launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
    if (n > 0) { to_f32_kernel<<<nblk(n, 256), 256, 0, s>>>(in, out, n); count_launch(); }
}

}  // namespace l2x
