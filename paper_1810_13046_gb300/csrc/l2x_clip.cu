// Kernels for steps (II)-(III) of Sec. 2.3 (clip + quadrature per candidate
// pair), the fused and the plain variants, and the plain path's atomic scatter
// of the local blocks into B (step IV).
#include "l2x_clip.cuh"

namespace l2x {

namespace {

constexpr int kClipThreads = 128;

// Lower corner, width and inverse width of a cell per axis: uniform grids
// origin + i h; stretched grids the cell between nodes x_i and x_{i+1}.
__device__ __forceinline__ void cell_frame(const SubGrid& sg, int dim, int32_t cell, double* clo, double* w,
                                           double* iw) {
    int ci[3];
    int c = cell;
    ci[0] = c % sg.ncell[0];
    c /= sg.ncell[0];
    ci[1] = c % sg.ncell[1];
    ci[2] = dim == 3 ? c / sg.ncell[1] : 0;
    for (int k = 0; k < dim; ++k) {
        if (sg.ax[0]) {
            clo[k] = __ldg(sg.ax[k] + ci[k]);
            w[k] = __ldg(sg.ax[k] + ci[k] + 1) - clo[k];
            iw[k] = __ldg(sg.inv_w[k] + ci[k]);
        } else {
            clo[k] = __dadd_rn(sg.origin[k], __dmul_rn((double)ci[k], sg.h[k]));
            w[k] = sg.h[k];
            iw[k] = sg.inv_h[k];
        }
    }
}

// Element vertices of pair p in cell-local coordinates; w receives the cell widths.
// Uniform grid whose spacing is a power of two on every used axis (h = 2^-e).
template <int D>
__device__ __forceinline__ bool pow2_grid(const SubGrid& sg) {
    return !sg.ax[0] && sg.pow2[0] && sg.pow2[1] && (D == 2 || sg.pow2[2]);
}

template <int D>
__device__ __forceinline__ void pair_vertices(const SubGrid& sg, const double* __restrict__ X, const int32_t* __restrict__ E,
                                              int32_t e, int32_t cell, double (&T)[D + 1][D], double* w) {
    if (pow2_grid<D>(sg)) {
        // the cell corner origin + i h and the scaling by 1/h = 2^e on the exponent
        // field: both products are exact, so the values are those of the general
        // branch, with integer instructions in place of FP64 ones
        int c = cell, ci[3];
        ci[0] = c % sg.ncell[0];
        c /= sg.ncell[0];
        ci[1] = c % sg.ncell[1];
        ci[2] = D == 3 ? c / sg.ncell[1] : 0;
        double clo[3];
        int es[3];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            es[k] = ilogb_int(sg.inv_h[k]);
            clo[k] = __dadd_rn(sg.origin[k], ldexp_normal_int(i2d_int(ci[k]), -es[k]));
            w[k] = sg.h[k];
        }
#pragma unroll
        for (int a = 0; a <= D; ++a) {
            const int32_t v = __ldg(E + (int64_t)e * (D + 1) + a);
#pragma unroll
            for (int k = 0; k < D; ++k) T[a][k] = ldexp_normal_int(__ldg(X + (int64_t)v * D + k) - clo[k], es[k]);
        }
        return;
    }
    double clo[3], iw[3];
    cell_frame(sg, D, cell, clo, w, iw);
#pragma unroll
    for (int a = 0; a <= D; ++a) {
        const int32_t v = __ldg(E + (int64_t)e * (D + 1) + a);
#pragma unroll
        for (int k = 0; k < D; ++k) T[a][k] = (__ldg(X + (int64_t)v * D + k) - clo[k]) * iw[k];
    }
}

// Cell volume of the local frame, and gradients brought into it: on a
// stretched grid the element gradients are stored per unit length and scaled by
// the widths of the pair's cell; on a uniform grid they are stored in cell units.
template <int D>
__device__ __forceinline__ double frame_scale(const SubGrid& sg, const double* w, double (&gr)[D + 1][D]) {
    if (sg.ax[0]) {
#pragma unroll
        for (int a = 0; a <= D; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) gr[a][k] *= w[k];
    }
    return w[0] * w[1] * (D == 3 ? w[2] : 1.0);
}

struct SubGridSet {
    SubGrid g[kMaxGrids];
};

// Pairs of all grids are listed grid by grid; offsets[g * m] is the first pair
// of grid g and offsets[G * m] the total (device values, so that the same
// kernels run inside a captured CUDA graph).  n_cap bounds every index.
__device__ __forceinline__ int grid_of_pair(int64_t p, int G, int64_t m, const int64_t* __restrict__ offsets) {
    int g = 0;
    while (g + 1 < G && p >= offsets[(int64_t)(g + 1) * m]) ++g;
    return g;
}

// Fused, step 1: scheduling class of every pair and per-class counts.
template <int D>
__global__ void pair_class_kernel(int G, SubGridSet sgs, int64_t m, const int64_t* __restrict__ offsets, int64_t n_cap,
                                  const double* __restrict__ X, const int32_t* __restrict__ E,
                                  const int32_t* __restrict__ pair_elem, const int32_t* __restrict__ pair_cell,
                                  uint8_t* __restrict__ keys, int32_t* counts) {
    __shared__ int hist[kClasses];
    if (threadIdx.x < kClasses) hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = min(offsets[(int64_t)G * m], n_cap);
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) {
        const int g = grid_of_pair(p, G, m, offsets);
        // the class only orders the pairs for the clip kernel, which classifies
        // every pair again in FP64: single precision suffices here
        const SubGrid& sg = sgs.g[g];
        const int32_t e = pair_elem[p];
        int c = pair_cell[p], ci[3];
        ci[0] = c % sg.ncell[0];
        c /= sg.ncell[0];
        ci[1] = c % sg.ncell[1];
        ci[2] = D == 3 ? c / sg.ncell[1] : 0;
        float clo[3], iw[3];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (sg.ax[0]) {
                clo[k] = d2f_int(__ldg(sg.ax[k] + ci[k]));
                iw[k] = d2f_int(__ldg(sg.inv_w[k] + ci[k]));
            } else {
                clo[k] = d2f_int(sg.origin[k]) + (float)ci[k] * d2f_int(sg.h[k]);
                iw[k] = d2f_int(sg.inv_h[k]);
            }
        }
        int lo = 0, up = 0, in = (1 << (D + 1)) - 1;
        bool live = true;
        float mn[D], mx[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            mn[k] = 3.0e38f;
            mx[k] = -3.0e38f;
        }
#pragma unroll
        for (int a = 0; a <= D; ++a) {
            const int32_t v = __ldg(E + (int64_t)e * (D + 1) + a);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = (d2f_int(__ldg(X + (int64_t)v * D + k)) - clo[k]) * iw[k];
                mn[k] = fminf(mn[k], t);
                mx[k] = fmaxf(mx[k], t);
                if (t < 0.0f || t > 1.0f) in &= ~(1 << a);
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (mx[k] <= 0.0f || mn[k] >= 1.0f) live = false;
            if (mn[k] < 0.0f) lo |= 1 << k;
            if (mx[k] > 1.0f) up |= 1 << k;
        }
        const int key = live ? min(1 + 2 * (lo | (up << D)) + (in ? 1 : 0), kClasses - 1) : 0;
        keys[p] = (uint8_t)key;
        atomicAdd(&hist[key], 1);
    }
    __syncthreads();
    if (threadIdx.x < kClasses && hist[threadIdx.x]) atomicAdd(counts + threadIdx.x, hist[threadIdx.x]);
}

// Fused, step 2: exclusive scan of the class counts into bucket cursors.
__global__ void class_scan_kernel(int32_t* counts, int32_t* cursors) {
    if (threadIdx.x != 0) return;
    int32_t acc = 0;
    for (int k = 0; k < kClasses; ++k) {
        cursors[k] = acc;
        acc += counts[k];
    }
}

// Fused, step 3: permutation listing the pairs class by class.  Each block
// reserves one range per class, so runs of consecutive pairs stay together.
__global__ void pair_scatter_kernel(int G, int64_t m, const int64_t* __restrict__ offsets, int64_t n_cap,
                                    const uint8_t* __restrict__ keys, int32_t* cursors, int32_t* perm) {
    __shared__ int hist[kClasses];
    __shared__ int base[kClasses];
    if (threadIdx.x < kClasses) hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = min(offsets[(int64_t)G * m], n_cap);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int key = 0, rank = 0;
    if (i < n) {
        key = keys[i];
        rank = atomicAdd(&hist[key], 1);
    }
    __syncthreads();
    if (threadIdx.x < kClasses && hist[threadIdx.x]) base[threadIdx.x] = atomicAdd(cursors + threadIdx.x, hist[threadIdx.x]);
    __syncthreads();
    if (i < n) perm[base[key] + rank] = (int32_t)i;
}

// Fused, step 4: clip + integrate pair i of the class order.  Gradients come
// from the element pass; the thread writes its pair's block as one contiguous
// run (pair-major), i.e. whole cache lines.
template <int D, typename R>
__device__ __forceinline__ void clip_pair(int64_t i, int G, const SubGridSet& sgs, int64_t m,
                                          const int64_t* __restrict__ offsets, const double* __restrict__ X,
                                          const int32_t* __restrict__ E, const double* __restrict__ elem_grad,
                                          const int8_t* __restrict__ elem_flag, const int32_t* __restrict__ perm,
                                          const int32_t* __restrict__ pair_elem, const int32_t* __restrict__ pair_cell,
                                          double* __restrict__ blocks, double* __restrict__ vols, DevStatus* st,
                                          double (*poly)[D]) {
    constexpr int NA = D + 1, NB = 1 << D;
    const int64_t p = perm[i];
    const int g = grid_of_pair(p, G, m, offsets);
    const SubGrid& sg = sgs.g[g];
    const int32_t e = pair_elem[p];
    double* blk = blocks + p * (NA * NB);  // the pair's block, written in place
    double vol = 0.0;
    const int flag = elem_flag[e];
    if (flag < 0) {
        atomicOr(&st->flags, FLAG_DEGENERATE);
        atomicMin(&st->bad_elem, e);
        store_zero_block<D>(blk);
    } else {
        double T[NA][D], gr[NA][D], w[3];
        pair_vertices<D>(sg, X, E, e, pair_cell[p], T, w);
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) gr[a][k] = __ldg(elem_grad + ((int64_t)e * NA + a) * D + k);
        double scale;
        if (pow2_grid<D>(sg)) {  // the cell volume 2^-(e0 + e1 + e2), exactly
            int es = ilogb_int(sg.inv_h[0]) + ilogb_int(sg.inv_h[1]);
            if (D == 3) es += ilogb_int(sg.inv_h[2]);
            scale = ldexp_normal_int(1.0, -es);
        } else {
            scale = frame_scale<D>(sg, w, gr);
        }
        pair_integrals<D, R>(T, gr, flag == 1, scale, blk, &vol, poly);
    }
    vols[p] = vol;
}

// Persistent launch over a work queue: the CTAs resident on the SMs take chunks
// of `chunk` x blockDim pairs (in class order) from a device counter until the
// pairs run out.  The counter only grows, so every CTA ends after at most
// n / (chunk x blockDim) + 1 fetches.  The chunk size is a work shape the
// autotuner picks: small chunks balance the uneven cost of the classes, large
// ones take fewer counter atomics.
template <int D, typename R>
__global__ void __launch_bounds__(256) clip_fused_kernel(int G, SubGridSet sgs, int64_t m,
                                                         const int64_t* __restrict__ offsets, int64_t n_cap,
                                                         const double* __restrict__ X, const int32_t* __restrict__ E,
                                                         const double* __restrict__ elem_grad,
                                                         const int8_t* __restrict__ elem_flag,
                                                         const int32_t* __restrict__ perm,
                                                         const int32_t* __restrict__ pair_elem,
                                                         const int32_t* __restrict__ pair_cell,
                                                         double* __restrict__ blocks, double* __restrict__ vols,
                                                         DevStatus* st, unsigned long long* work, int chunk) {
    // this thread's polygon buffers: on-chip shared memory instead of local
    // memory (whose lines the resident threads would evict from L1)
    extern __shared__ double s_poly[];
    __shared__ long long s_base;
    double (*poly)[D] = reinterpret_cast<double (*)[D]>(s_poly + threadIdx.x * PolySlot<D>::kDoubles);
    const int64_t n = min(offsets[(int64_t)G * m], n_cap);
    const long long per = (long long)blockDim.x * chunk;
    for (;;) {
        if (threadIdx.x == 0) s_base = (long long)atomicAdd(work, (unsigned long long)per);
        __syncthreads();
        const long long base = s_base;
        __syncthreads();  // every thread has read s_base before the next fetch writes it
        if (base >= n) break;
        for (int k = 0; k < chunk; ++k) {
            const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
            if (i < n)
                clip_pair<D, R>(i, G, sgs, m, offsets, X, E, elem_grad, elem_flag, perm, pair_elem, pair_cell, blocks,
                                vols, st, poly);
        }
    }
}

// Plain: one thread per pair, element data from global memory, FP64 throughout,
// blocks stored pair-major.
template <int D>
__global__ void clip_plain_kernel(SubGrid sg, const double* __restrict__ X, const int32_t* __restrict__ E,
                                  int64_t p_begin, int64_t p_end, const int32_t* __restrict__ pair_elem,
                                  const int32_t* __restrict__ pair_cell, double* __restrict__ blocks,
                                  double* __restrict__ vols, DevStatus* st) {
    constexpr int NA = D + 1, NB = 1 << D;
    const int64_t p = p_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= p_end) return;
    const int32_t e = pair_elem[p];
    double clo[3], w[3], iw[3];
    cell_frame(sg, D, pair_cell[p], clo, w, iw);
    double Xe[NA][D], T[NA][D], ge[NA][D];
    for (int a = 0; a < NA; ++a) {
        const int32_t v = E[(int64_t)e * NA + a];
        for (int k = 0; k < D; ++k) {
            Xe[a][k] = X[(int64_t)v * D + k];
            T[a][k] = (Xe[a][k] - clo[k]) * iw[k];
        }
    }
    double* blk = blocks + p * (NA * NB);
    double vol = 0.0;
    bool pos = true;
    if (!elem_gradients<D>(Xe, sg.inv_h, ge, pos)) {
        atomicOr(&st->flags, FLAG_DEGENERATE);
        atomicMin(&st->bad_elem, e);
        store_zero_block<D>(blk);
    } else {
        const double scale = frame_scale<D>(sg, w, ge);
        double poly[2 * kMaxPoly][D];
        pair_integrals<D, double>(T, ge, pos, scale, blk, &vol, poly);
    }
    vols[p] = vol;
}

template <int D>
__global__ void scatter_plain_kernel(SubGrid sg, const int32_t* __restrict__ E, int64_t p_begin, int64_t p_end,
                                     const int32_t* __restrict__ pair_elem, const int32_t* __restrict__ pair_cell,
                                     const double* __restrict__ blocks, const double* __restrict__ vols,
                                     const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                     double* __restrict__ val, int dual) {
    constexpr int NA = D + 1, NB = 1 << D;
    const int64_t p = p_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= p_end) return;
    if (!(vols[p] > 0.0)) return;
    const int32_t e = pair_elem[p];
    int c = pair_cell[p];
    int ci[3];
    ci[0] = c % sg.ncell[0];
    c /= sg.ncell[0];
    ci[1] = c % sg.ncell[1];
    ci[2] = D == 3 ? c / sg.ncell[1] : 0;
    for (int a = 0; a < NA; ++a) {
        int32_t row = E[(int64_t)e * NA + a];
        int64_t lo = ptr[row], hi = ptr[row + 1];
        for (int b = 0; b < NB; ++b) {
            int32_t node = (ci[0] + (b & 1)) +
                           sg.nnode[0] * ((ci[1] + ((b >> 1) & 1)) + sg.nnode[1] * (ci[2] + ((b >> 2) & 1)));
            int64_t l = lo, r = hi;  // lower_bound
            while (l < r) {
                int64_t mid = (l + r) >> 1;
                if (col[mid] < node) l = mid + 1; else r = mid;
            }
            if (l < hi && col[l] == node) {
                const double* blk = blocks + p * (NA * NB);
                double v = blk[a * NB + b];
                if (dual) {  // (d+2) lambda_a - 1: the lambda integrals sum to the integral of psi_b
                    double sum = 0.0;
                    for (int a2 = 0; a2 < NA; ++a2) sum += blk[a2 * NB + b];
                    v = (double)(D + 2) * v - sum;
                }
                atomicAdd(val + l, v);
            }
        }
    }
}

}  // namespace

void launch_pair_classes(int dim, int G, const SubGrid* sg, int64_t m, const int64_t* offsets, int64_t n_launch,
                         int64_t n_cap, const double* X, const int32_t* E, const int32_t* pair_elem,
                         const int32_t* pair_cell, uint8_t* keys, int32_t* perm, int32_t* buckets, cudaStream_t s) {
    if (n_launch <= 0) return;
    SubGridSet sgs{};
    for (int g = 0; g < G; ++g) sgs.g[g] = sg[g];
    cudaMemsetAsync(buckets, 0, sizeof(int32_t) * 2 * kClasses, s);
    const unsigned nb256 = (unsigned)((n_launch + 255) / 256);
    if (dim == 2) { pair_class_kernel<2><<<nb256, 256, 0, s>>>(G, sgs, m, offsets, n_cap, X, E, pair_elem, pair_cell, keys, buckets); count_launch(); }
    else { pair_class_kernel<3><<<nb256, 256, 0, s>>>(G, sgs, m, offsets, n_cap, X, E, pair_elem, pair_cell, keys, buckets); count_launch(); }
    { class_scan_kernel<<<1, 32, 0, s>>>(buckets, buckets + kClasses); count_launch(); }
    { pair_scatter_kernel<<<nb256, 256, 0, s>>>(G, m, offsets, n_cap, keys, buckets + kClasses, perm); count_launch(); }
}

void launch_clip_fused(int dim, int precision, int G, const SubGrid* sg, int64_t m, const int64_t* offsets,
                       int64_t n_launch, int64_t n_cap, const double* X, const int32_t* E, const double* elem_grad,
                       const int8_t* elem_flag, const int32_t* pair_elem, const int32_t* pair_cell,
                       const int32_t* perm, double* blocks, double* vols, DevStatus* st,
                       cudaStream_t s, int block, int chunk, unsigned long long* work) {
    if (n_launch <= 0) return;
    SubGridSet sgs{};
    for (int g = 0; g < G; ++g) sgs.g[g] = sg[g];
    if (block != 64 && block != 128 && block != 256) block = kClipThreads;
    if (chunk < 1) chunk = 1;
    const size_t sm2 = (size_t)block * PolySlot<2>::kDoubles * sizeof(double);
    const size_t sm3 = (size_t)block * PolySlot<3>::kDoubles * sizeof(double);
    // kernel attributes and resident CTAs per SM, set once per (form, block),
    // outside stream capture (the first launch of a shape comes from a build or
    // the autotuner)
    static bool smem_set = false;
    static int resident[2][2][3] = {};
    static int n_sm = 0;
    if (!smem_set) {
        const int mx2 = 256 * PolySlot<2>::kDoubles * (int)sizeof(double);
        const int mx3 = 256 * PolySlot<3>::kDoubles * (int)sizeof(double);
        cudaFuncSetAttribute(clip_fused_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx2);
        cudaFuncSetAttribute(clip_fused_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx2);
        cudaFuncSetAttribute(clip_fused_kernel<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx3);
        cudaFuncSetAttribute(clip_fused_kernel<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx3);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const void* fns[2][2] = {{(const void*)clip_fused_kernel<2, double>, (const void*)clip_fused_kernel<2, float>},
                                 {(const void*)clip_fused_kernel<3, double>, (const void*)clip_fused_kernel<3, float>}};
        const int blocks3[3] = {64, 128, 256};
        for (int dd = 0; dd < 2; ++dd)
            for (int pr = 0; pr < 2; ++pr)
                for (int b = 0; b < 3; ++b) {
                    int r = 0;
                    const size_t smb = (size_t)blocks3[b] * (dd ? PolySlot<3>::kDoubles : PolySlot<2>::kDoubles) * sizeof(double);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fns[dd][pr], blocks3[b], smb);
                    resident[dd][pr][b] = r > 0 ? r : 1;
                }
        smem_set = true;
    }
    const int bi = block == 64 ? 0 : block == 128 ? 1 : 2;
    const int res = resident[dim == 3][precision == L2X_MIXED][bi];
    const int64_t per = (int64_t)block * chunk;
    const int64_t want = (n_launch + per - 1) / per;
    const int64_t cap = (int64_t)res * (n_sm > 0 ? n_sm : 1);
    const unsigned nb = (unsigned)(want < cap ? want : cap);
    cudaMemsetAsync(work, 0, sizeof(unsigned long long), s);
#define L2X_CLIP_ARGS G, sgs, m, offsets, n_cap, X, E, elem_grad, elem_flag, perm, pair_elem, pair_cell, blocks, vols, st, work, chunk
    if (dim == 2) {
        if (precision == L2X_MIXED) { clip_fused_kernel<2, float><<<nb, block, sm2, s>>>(L2X_CLIP_ARGS); count_launch(); }
        else { clip_fused_kernel<2, double><<<nb, block, sm2, s>>>(L2X_CLIP_ARGS); count_launch(); }
    } else {
        if (precision == L2X_MIXED) { clip_fused_kernel<3, float><<<nb, block, sm3, s>>>(L2X_CLIP_ARGS); count_launch(); }
        else { clip_fused_kernel<3, double><<<nb, block, sm3, s>>>(L2X_CLIP_ARGS); count_launch(); }
    }
#undef L2X_CLIP_ARGS
}

void launch_clip_plain(int dim, const SubGrid& sg, const double* X, const int32_t* E, int64_t p_begin,
                       int64_t p_end, const int32_t* pair_elem, const int32_t* pair_cell, double* blocks,
                       double* vols, DevStatus* st, cudaStream_t s) {
    int64_t n = p_end - p_begin;
    if (n <= 0) return;
    unsigned nb = (unsigned)((n + 127) / 128);
    if (dim == 2)
        { clip_plain_kernel<2><<<nb, 128, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, st); count_launch(); }
    else
        { clip_plain_kernel<3><<<nb, 128, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, st); count_launch(); }
}

void launch_scatter_plain(int dim, const SubGrid& sg, const int32_t* E, int64_t p_begin, int64_t p_end,
                          const int32_t* pair_elem, const int32_t* pair_cell, const double* blocks,
                          const double* vols, const Csr& B, int dual, cudaStream_t s) {
    int64_t n = p_end - p_begin;
    if (n <= 0) return;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (dim == 2)
        { scatter_plain_kernel<2><<<nb, 256, 0, s>>>(sg, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, B.ptr, B.col, B.val, dual); count_launch(); }
    else
        { scatter_plain_kernel<3><<<nb, 256, 0, s>>>(sg, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, B.ptr, B.col, B.val, dual); count_launch(); }
}

}  // namespace l2x
