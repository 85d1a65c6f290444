// Step (I) of the assembly (Sec. 2.3): overlap detection between solid elements
// and the cells of every velocity grid.  The uniform grid replaces the tree
// search: the candidate cells of an element are the cells of its bounding box,
//   i_lo = floor((lo - o) / h),   i_hi = ceil((hi - o) / h) - 1,
// with one IEEE-rounded subtraction and one correctly rounded division (the
// intrinsics below are never contracted into a fused multiply-add), so the pair
// list is reproducible bit for bit on any IEEE machine.
#include <climits>

#include "l2x_clip.cuh"
#include "l2x_internal.cuh"

namespace l2x {

namespace {

struct SubGridSet {
    SubGrid g[kMaxGrids];
};

__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }

// Entries of the increasing array x[0..n) that are <= v, resp. < v.
__device__ __forceinline__ int count_le(const double* __restrict__ x, int n, double v) {
    int l = 0, r = n;
    while (l < r) {
        const int m = (l + r) >> 1;
        if (__ldg(x + m) <= v) l = m + 1; else r = m;
    }
    return l;
}
__device__ __forceinline__ int count_lt(const double* __restrict__ x, int n, double v) {
    int l = 0, r = n;
    while (l < r) {
        const int m = (l + r) >> 1;
        if (__ldg(x + m) < v) l = m + 1; else r = m;
    }
    return l;
}

// floor(q) of a finite double by integer operations on its bits, and whether q
// is an integer; -1 for q < 0 (below the grid), 2^40 for q >= 2^40 (beyond it);
// NaN counts as beyond.
__device__ __forceinline__ long long floor_bits(double q, bool& integral) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(q);
    const int e = (int)((u >> 52) & 0x7ff) - 1023;
    integral = false;
    if (u >> 63) {  // negative (or -0.0: the floor of -0.0 is 0)
        integral = (u << 1) == 0;
        return integral ? 0 : -1;
    }
    if (e < 0) {
        integral = u == 0;
        return 0;
    }
    if (e >= 40) return 1ll << 40;
    const unsigned long long mant = (u & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = 52 - e;
    integral = (mant & ((1ull << sh) - 1)) == 0;
    return (long long)(mant >> sh);
}

template <int D>
__global__ void elem_boxes_kernel(int n_grids, SubGridSet sgs, int64_t m, const double* __restrict__ X,
                                  const int32_t* __restrict__ E, ElemBox* __restrict__ boxes,
                                  int64_t* __restrict__ counts, int64_t* __restrict__ nbox, int32_t* __restrict__ node_box,
                                  double* __restrict__ elem_vol, double* __restrict__ elem_grad,
                                  int8_t* __restrict__ elem_flag, DevStatus* st) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    double V[D + 1][D];
    bool finite = true;
    for (int a = 0; a <= D; ++a) {
        int32_t v = __ldg(E + e * (D + 1) + a);
        for (int k = 0; k < D; ++k) {
            V[a][k] = ldg(X + (int64_t)v * D + k);
            finite = finite && isfinite(V[a][k]);
        }
    }
    double det;
    if (D == 2) {
        det = (V[1][0] - V[0][0]) * (V[2][1] - V[0][1]) - (V[1][1] - V[0][1]) * (V[2][0] - V[0][0]);
    } else {
        double a0 = V[1][0] - V[0][0], a1 = V[1][1 % D] - V[0][1 % D], a2 = V[1][2 % D] - V[0][2 % D];
        double b0 = V[2][0] - V[0][0], b1 = V[2][1 % D] - V[0][1 % D], b2 = V[2][2 % D] - V[0][2 % D];
        double c0 = V[D][0] - V[0][0], c1 = V[D][1 % D] - V[0][1 % D], c2 = V[D][2 % D] - V[0][2 % D];
        det = a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
    }
    elem_vol[e] = fabs(det) / (D == 2 ? 2.0 : 6.0);
    if (elem_grad) {
        // barycentric gradients in cell-local coordinates (the same for every grid)
        double g[D + 1][D];
        bool pos = true;
        const bool ok = finite && elem_gradients<D>(V, sgs.g[0].inv_h, g, pos);
#pragma unroll
        for (int a = 0; a <= D; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) elem_grad[(e * (D + 1) + a) * D + k] = ok ? g[a][k] : 0.0;
        elem_flag[e] = ok ? (pos ? 1 : 0) : -1;
    }
    int32_t flags = 0;
    if (!finite) flags |= FLAG_NONFINITE;
    else if (det == 0.0) flags |= FLAG_DEGENERATE;
    double lo[D], hi[D];
    for (int k = 0; k < D; ++k) {
        lo[k] = V[0][k];
        hi[k] = V[0][k];
        for (int a = 1; a <= D; ++a) {
            lo[k] = fmin(lo[k], V[a][k]);
            hi[k] = fmax(hi[k], V[a][k]);
        }
    }
    for (int g = 0; g < n_grids; ++g) {
        const SubGrid& sg = sgs.g[g];
        ElemBox b;
        b.lo[0] = b.lo[1] = b.lo[2] = 0;
        int ext[3] = {1, 1, 1};
        int64_t count = 1;
        bool ok = finite;
        for (int k = 0; k < D; ++k) {
            int il, ih;
            if (sg.ax[0]) {
                // stretched axis: half-open cells [x_i, x_{i+1}); comparisons only
                il = count_le(sg.ax[k], sg.nnode[k], lo[k]) - 1;
                ih = count_lt(sg.ax[k], sg.nnode[k], hi[k]) - 1;
                if (il < 0 || ih >= sg.ncell[k]) { ok = false; break; }
            } else {
                // one rounded subtraction and one correctly rounded division (a
                // product by the exact 1/h when h is a power of two: the same value)
                const double dlo = __dsub_rn(lo[k], sg.origin[k]), dhi = __dsub_rn(hi[k], sg.origin[k]);
                const double qlo = sg.pow2[k] ? __dmul_rn(dlo, sg.inv_h[k]) : __ddiv_rn(dlo, sg.h[k]);
                const double qhi = sg.pow2[k] ? __dmul_rn(dhi, sg.inv_h[k]) : __ddiv_rn(dhi, sg.h[k]);
                // floor(qlo) and ceil(qhi) - 1 from the bits of the exact quotients
                bool int_lo, int_hi;
                const long long flo = floor_bits(qlo, int_lo), fhi = floor_bits(qhi, int_hi);
                const long long chi = int_hi ? fhi - 1 : fhi;
                if (flo < 0 || chi >= (long long)sg.ncell[k]) { ok = false; break; }
                il = (int)flo;
                ih = (int)chi;
            }
            if (ih < il) ih = il;
            ext[k] = ih - il + 1;
            b.lo[k] = il;
            if (ext[k] > 1023) { flags |= FLAG_CAPACITY; ok = false; break; }
            count *= ext[k];
        }
        if (!ok && finite && !(flags & FLAG_CAPACITY)) flags |= FLAG_OUTOFGRID;
        if (!ok || (flags & FLAG_DEGENERATE)) count = 0;
        b.ext = ext[0] | (ext[1] << 10) | (ext[2] << 20);
        boxes[g * m + e] = b;
        counts[g * m + e] = count;
        nbox[g * m + e] = count > 0 ? (int64_t)(ext[0] + 1) * (ext[1] + 1) * (D == 3 ? ext[2] + 1 : 1) : 0;
        // touched-node box of the grid: reduced over the warp first (every element
        // updates the same six words), then one atomic per warp
        const unsigned act = __activemask();
        const int leader = __ffs(act) - 1;
        for (int k = 0; k < D; ++k) {
            const int lo_k = __reduce_min_sync(act, count > 0 ? b.lo[k] : INT_MAX);
            const int hi_k = __reduce_max_sync(act, count > 0 ? b.lo[k] + ext[k] : INT_MIN);
            if ((int)(threadIdx.x & 31) == leader && lo_k <= hi_k) {
                atomicMin(node_box + g * 6 + k, lo_k);
                atomicMax(node_box + g * 6 + 3 + k, hi_k);
            }
        }
    }
    if (flags) {
        atomicOr(&st->flags, flags);
        atomicMin(&st->bad_elem, (int32_t)e);
    }
}

template <int D>
__global__ void emit_pairs_kernel(int n_grids, SubGridSet sgs, int64_t m, const ElemBox* __restrict__ boxes,
                                  const int64_t* __restrict__ offsets, int32_t* __restrict__ pair_elem,
                                  int32_t* __restrict__ pair_cell, int64_t cap, DevStatus* st) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= m * n_grids) return;
    int g = (int)(t / m);
    int64_t e = t - g * m;
    const SubGrid& sg = sgs.g[g];
    ElemBox b = boxes[t];
    int64_t p = offsets[t], p1 = offsets[t + 1];
    if (p == p1) return;
    if (p1 > cap) {  // the pair list does not fit the capacity fixed for a captured step
        atomicOr(&st->flags, FLAG_CAPACITY);
        return;
    }
    int ex = box_ext(b, 0), ey = box_ext(b, 1), ez = box_ext(b, 2);
    for (int kz = 0; kz < ez; ++kz)
        for (int ky = 0; ky < ey; ++ky)
            for (int kx = 0; kx < ex; ++kx) {
                int32_t cell = (b.lo[0] + kx) + sg.ncell[0] * ((b.lo[1] + ky) + sg.ncell[1] * (b.lo[2] + kz));
                pair_elem[p] = (int32_t)e;
                pair_cell[p] = cell;
                ++p;
            }
}

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t warp_prefix = wid > 0 ? warp_sums[wid - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// Single-pass exclusive scan with decoupled look-back (D. Merrill and M.
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back", NVIDIA
// technical report NVR-2016-002).  Workspace ws: [0] tile counter, [1] finished
// blocks, [2 .. 2 + nb) one word per tile: status in the top two bits (0 none,
// 1 the tile's own total, 2 the inclusive prefix through the tile), the value
// in the low 62 bits (the scanned values are non-negative counts).
// * Tiles are numbered in the order blocks start (atomic counter), so a tile
//   only waits on tiles whose blocks are already running.
// * Each wait polls at most spin_limit times; a wait that gives up sets
//   FLAG_TIMEOUT in the status word (when given) and the scan goes on with
//   what it has, so no launch can hang.
// * The last block to finish clears the workspace for the next launch (the
//   workspace is zeroed once when it is allocated), so captured steps need no
//   memset node per scan.
constexpr unsigned long long kScanVal = (1ull << 62) - 1;
constexpr long long kScanSpinLimit = 1ll << 22;

__device__ __forceinline__ void scan_publish(unsigned long long* w, unsigned long long status, int64_t v) {
    __threadfence();
    atomicExch(w, (status << 62) | ((unsigned long long)v & kScanVal));
}

__global__ void __launch_bounds__(kScanThreads) scan_onepass_kernel(const int64_t* in, int64_t n, int64_t* out,
                                                                   unsigned long long* ws, int64_t nb,
                                                                   DevStatus* st, long long spin_limit) {
    __shared__ int64_t s_tile, s_excl;
    __shared__ int s_last;
    unsigned long long* ctr = ws;
    unsigned long long* done = ws + 1;
    unsigned long long* state = ws + 2;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(ctr, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    const bool valid = tile < nb;
    int64_t v[kScanItems];
    int64_t sum = 0;
    const int64_t base = tile * (int64_t)kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t idx = base + i;
        v[i] = valid && idx < n ? in[idx] : 0;  // all inputs read before any output is written (in place allowed)
        sum += v[i];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(sum, &tot);
    if (threadIdx.x == 0) {
        int64_t excl = 0;
        if (valid) {
            if (tile == 0) {
                scan_publish(state, 2ull, tot);
            } else {
                scan_publish(state + tile, 1ull, tot);
                int64_t j = tile - 1;
                long long spins = 0;
                for (;;) {
                    const unsigned long long word = *(volatile unsigned long long*)(state + j);
                    const unsigned long long f = word >> 62;
                    if (f == 0) {
                        if (++spins > spin_limit) {
                            if (st) atomicOr(&st->flags, FLAG_TIMEOUT);
                            break;
                        }
                        continue;
                    }
                    excl += (int64_t)(word & kScanVal);
                    if (f == 2 || j == 0) break;
                    --j;
                }
                scan_publish(state + tile, 2ull, excl + tot);
            }
        }
        s_excl = excl;
        __threadfence();
        s_last = atomicAdd(done, 1ull) == (unsigned long long)nb;  // nb + 1 blocks run (see the launch)
    }
    __syncthreads();
    if (valid) {
        ex += s_excl;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int64_t idx = base + i;
            if (idx < n) out[idx] = ex;
            ex += v[i];
        }
        if (tile == nb - 1 && threadIdx.x == 0) out[n] = s_excl + tot;
    }
    if (s_last) {  // every other block has finished its look-back: reset for the next launch
        for (int64_t t = threadIdx.x; t < nb; t += kScanThreads) state[t] = 0ull;
        __syncthreads();
        if (threadIdx.x == 0) {
            *ctr = 0ull;
            *done = 0ull;
            __threadfence();
        }
    }
}

__global__ void reset_status_kernel(DevStatus* st) {
    if (threadIdx.x == 0) {
        st->flags = 0;
        st->bad_elem = INT_MAX;
        st->cg_iters = 0;
        st->cg_residual = 0.0;
    }
}

// Empty touched-node boxes (min = INT_MAX, max = INT_MIN) before the element pass.
__global__ void node_box_reset_kernel(int32_t* node_box, int n_grids) {
    const int t = threadIdx.x;
    if (t < 6 * n_grids) node_box[t] = (t % 6) < 3 ? INT_MAX : INT_MIN;
}

// A captured step's B^T rows cover a fixed box per grid: flag a step whose
// touched nodes leave it (its later kernels then skip their work).
__global__ void check_node_box_kernel(const int32_t* node_box, NodeBoxSet lim, int n_grids, DevStatus* st) {
    const int g = threadIdx.x;
    if (g >= n_grids) return;
    for (int k = 0; k < 3; ++k) {
        const int lo = node_box[g * 6 + k], hi = node_box[g * 6 + 3 + k];
        if (lo > hi) continue;  // no element on this grid
        if (lo < lim.lo[g][k] || hi > lim.hi[g][k]) atomicOr(&st->flags, FLAG_CAPACITY);
    }
}

__global__ void check_capacity_kernel(const int64_t* total, int64_t cap, DevStatus* st) {
    if (threadIdx.x == 0 && *total > cap) atomicOr(&st->flags, FLAG_CAPACITY);
}

}  // namespace

void launch_reset_status(DevStatus* st, cudaStream_t s) {
    { reset_status_kernel<<<1, 32, 0, s>>>(st); count_launch(); }
}

void launch_node_box_reset(int32_t* node_box, int n_grids, cudaStream_t s) {
    { node_box_reset_kernel<<<1, 32, 0, s>>>(node_box, n_grids); count_launch(); }
}

void launch_check_node_box(const int32_t* node_box, const NodeBoxSet& lim, int n_grids, DevStatus* st,
                           cudaStream_t s) {
    { check_node_box_kernel<<<1, 32, 0, s>>>(node_box, lim, n_grids, st); count_launch(); }
}

void launch_check_capacity(const int64_t* total, int64_t cap, DevStatus* st, cudaStream_t s) {
    { check_capacity_kernel<<<1, 32, 0, s>>>(total, cap, st); count_launch(); }
}

void launch_elem_boxes(int dim, int n_grids, const SubGrid* sg_host, int64_t m, const double* X,
                       const int32_t* E, ElemBox* boxes, int64_t* counts, int64_t* nbox, int32_t* node_box,
                       double* elem_vol, double* elem_grad, int8_t* elem_flag, DevStatus* st, cudaStream_t s) {
    SubGridSet sgs{};
    for (int g = 0; g < n_grids; ++g) sgs.g[g] = sg_host[g];
    int threads = 256;
    int64_t blocks = (m + threads - 1) / threads;
    if (blocks == 0) return;
    if (dim == 2)
        { elem_boxes_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(n_grids, sgs, m, X, E, boxes, counts, nbox, node_box, elem_vol, elem_grad, elem_flag, st); count_launch(); }
    else
        { elem_boxes_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(n_grids, sgs, m, X, E, boxes, counts, nbox, node_box, elem_vol, elem_grad, elem_flag, st); count_launch(); }
}

size_t scan_tmp_bytes(int64_t n) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    return (size_t)(nb + 2) * sizeof(int64_t);
}

// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.  n >= 1.
// tmp: scan_tmp_bytes(n) bytes, zeroed when allocated and left zeroed by every
// launch.  One block more than the tiles is launched: it finds no tile and only
// counts itself, so the block that clears the workspace is always the last.
void launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s, DevStatus* st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (n <= 0) return;
    { scan_onepass_kernel<<<(unsigned)(nb + 1), kScanThreads, 0, s>>>(in, n, out, (unsigned long long*)tmp, nb, st,
                                                                      kScanSpinLimit); count_launch(); }
}

// Test hook of the look-back's bounded wait: with `missing_first`, the tile
// counter starts at 1, so tile 0 never publishes and tile 1's wait runs out
// after spin_limit polls (FLAG_TIMEOUT); the workspace is reset as usual.
void launch_scan_i64_test(const int64_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s, DevStatus* st,
                          int missing_first, long long spin_limit) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (n <= 0) return;
    if (missing_first) {
        const unsigned long long one = 1ull;
        cudaMemcpyAsync(tmp, &one, sizeof(one), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    { scan_onepass_kernel<<<(unsigned)(nb + 1), kScanThreads, 0, s>>>(in, n, out, (unsigned long long*)tmp, nb, st,
                                                                      spin_limit); count_launch(); }
}

void launch_emit_pairs(int dim, int n_grids, const SubGrid* sg_host, int64_t m, const ElemBox* boxes,
                       const int64_t* offsets, int32_t* pair_elem, int32_t* pair_cell, int64_t cap, DevStatus* st,
                       cudaStream_t s) {
    SubGridSet sgs{};
    for (int g = 0; g < n_grids; ++g) sgs.g[g] = sg_host[g];
    int threads = 256;
    int64_t total = m * n_grids;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks == 0) return;
    if (dim == 2)
        { emit_pairs_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(n_grids, sgs, m, boxes, offsets, pair_elem, pair_cell, cap, st); count_launch(); }
    else
        { emit_pairs_kernel<3><<<(unsigned)blocks, threads, 0, s>>>(n_grids, sgs, m, boxes, offsets, pair_elem, pair_cell, cap, st); count_launch(); }
}

}  // namespace l2x
