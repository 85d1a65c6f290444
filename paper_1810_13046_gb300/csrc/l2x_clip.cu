// Kernels for steps (II)-(III) of Sec. 2.3 (clip + quadrature per candidate
// pair), the fused and the plain variants, and the plain path's atomic scatter
// of the local blocks into B (step IV).
#include "l2x_clip.cuh"

namespace l2x {

namespace {

constexpr int kClipThreads = 128;

__device__ __forceinline__ void cell_lower(const SubGrid& sg, int dim, int32_t cell, double* clo, int* ci) {
    int c = cell;
    ci[0] = c % sg.ncell[0];
    c /= sg.ncell[0];
    ci[1] = c % sg.ncell[1];
    ci[2] = dim == 3 ? c / sg.ncell[1] : 0;
    for (int k = 0; k < dim; ++k) clo[k] = __dadd_rn(sg.origin[k], __dmul_rn((double)ci[k], sg.h[k]));
}

// Fused: one thread per pair; the block stages the vertex coordinates and the
// barycentric gradients of the (consecutive) elements of its 128 pairs in shared
// memory once.  Blocks are written structure-of-arrays so that every store
// instruction is coalesced.
template <int D, typename R>
__global__ void __launch_bounds__(kClipThreads) clip_fused_kernel(SubGrid sg, const double* __restrict__ X,
                                                                  const int32_t* __restrict__ E, int64_t p_begin,
                                                                  int64_t p_end, const int32_t* __restrict__ pair_elem,
                                                                  const int32_t* __restrict__ pair_cell,
                                                                  double* __restrict__ blocks, int64_t slot_stride,
                                                                  double* __restrict__ vols, DevStatus* st) {
    constexpr int NA = D + 1, NB = 1 << D;
    __shared__ double sV[kClipThreads][NA][D];
    __shared__ double sG[kClipThreads][NA][D];
    __shared__ int sPos[kClipThreads];
    const int64_t p0 = p_begin + (int64_t)blockIdx.x * kClipThreads;
    const int64_t plast = min(p0 + kClipThreads - 1, p_end - 1);
    const int32_t e_first = pair_elem[p0];
    const int n_e = min(pair_elem[plast] - e_first + 1, kClipThreads);
    if (threadIdx.x < n_e) {
        const int le = threadIdx.x;
        double Xe[NA][D];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int32_t v = __ldg(E + (int64_t)(e_first + le) * NA + a);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                Xe[a][k] = __ldg(X + (int64_t)v * D + k);
                sV[le][a][k] = Xe[a][k];
            }
        }
        double ge[NA][D];
        bool pos = true;
        const bool ok = elem_gradients<D>(Xe, sg.inv_h, ge, pos);
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) sG[le][a][k] = ok ? ge[a][k] : 0.0;
        sPos[le] = ok ? (pos ? 1 : 0) : -1;
    }
    __syncthreads();
    const int64_t p = p0 + threadIdx.x;
    if (p >= p_end) return;
    const int32_t e = pair_elem[p];
    double clo[3];
    int ci[3];
    cell_lower(sg, D, pair_cell[p], clo, ci);
    const int le = e - e_first;
    double Xe[NA][D], ge[NA][D];
    int posflag;
    if (le < kClipThreads) {
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                Xe[a][k] = sV[le][a][k];
                ge[a][k] = sG[le][a][k];
            }
        posflag = sPos[le];
    } else {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int32_t v = __ldg(E + (int64_t)e * NA + a);
#pragma unroll
            for (int k = 0; k < D; ++k) Xe[a][k] = __ldg(X + (int64_t)v * D + k);
        }
        bool pos = true;
        posflag = elem_gradients<D>(Xe, sg.inv_h, ge, pos) ? (pos ? 1 : 0) : -1;
    }
    double blk[NA * NB];
    double vol = 0.0;
    if (posflag < 0) {
        atomicOr(&st->flags, FLAG_DEGENERATE);
        atomicMin(&st->bad_elem, e);
#pragma unroll
        for (int i = 0; i < NA * NB; ++i) blk[i] = 0.0;
    } else {
        double T[NA][D];
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int k = 0; k < D; ++k) T[a][k] = (Xe[a][k] - clo[k]) * sg.inv_h[k];
        const double scale = sg.h[0] * sg.h[1] * (D == 3 ? sg.h[2] : 1.0);
        pair_integrals<D, R>(T, ge, posflag == 1, scale, blk, &vol);
    }
#pragma unroll
    for (int i = 0; i < NA * NB; ++i) blocks[i * slot_stride + p] = blk[i];
    vols[p] = vol;
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
    double clo[3];
    int ci[3];
    cell_lower(sg, D, pair_cell[p], clo, ci);
    double Xe[NA][D], T[NA][D], ge[NA][D];
    for (int a = 0; a < NA; ++a) {
        const int32_t v = E[(int64_t)e * NA + a];
        for (int k = 0; k < D; ++k) {
            Xe[a][k] = X[(int64_t)v * D + k];
            T[a][k] = (Xe[a][k] - clo[k]) * sg.inv_h[k];
        }
    }
    double blk[NA * NB];
    double vol = 0.0;
    bool pos = true;
    if (!elem_gradients<D>(Xe, sg.inv_h, ge, pos)) {
        atomicOr(&st->flags, FLAG_DEGENERATE);
        atomicMin(&st->bad_elem, e);
        for (int i = 0; i < NA * NB; ++i) blk[i] = 0.0;
    } else {
        const double scale = sg.h[0] * sg.h[1] * (D == 3 ? sg.h[2] : 1.0);
        pair_integrals<D, double>(T, ge, pos, scale, blk, &vol);
    }
    for (int i = 0; i < NA * NB; ++i) blocks[p * (NA * NB) + i] = blk[i];
    vols[p] = vol;
}

template <int D>
__global__ void scatter_plain_kernel(SubGrid sg, const int32_t* __restrict__ E, int64_t p_begin, int64_t p_end,
                                     const int32_t* __restrict__ pair_elem, const int32_t* __restrict__ pair_cell,
                                     const double* __restrict__ blocks, const double* __restrict__ vols,
                                     const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                     double* __restrict__ val) {
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
            if (l < hi && col[l] == node)
                atomicAdd(val + l, blocks[p * (NA * NB) + a * NB + b]);
        }
    }
}

}  // namespace

void launch_clip_fused(int dim, int precision, const SubGrid& sg, const double* X, const int32_t* E,
                       int64_t p_begin, int64_t p_end, const int32_t* pair_elem, const int32_t* pair_cell,
                       double* blocks, int64_t slot_stride, double* vols, DevStatus* st, cudaStream_t s) {
    int64_t n = p_end - p_begin;
    if (n <= 0) return;
    unsigned nb = (unsigned)((n + kClipThreads - 1) / kClipThreads);
    if (dim == 2) {
        if (precision == L2X_MIXED)
            { clip_fused_kernel<2, float><<<nb, kClipThreads, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, slot_stride, vols, st); count_launch(); }
        else
            { clip_fused_kernel<2, double><<<nb, kClipThreads, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, slot_stride, vols, st); count_launch(); }
    } else {
        if (precision == L2X_MIXED)
            { clip_fused_kernel<3, float><<<nb, kClipThreads, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, slot_stride, vols, st); count_launch(); }
        else
            { clip_fused_kernel<3, double><<<nb, kClipThreads, 0, s>>>(sg, X, E, p_begin, p_end, pair_elem, pair_cell, blocks, slot_stride, vols, st); count_launch(); }
    }
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
                          const double* vols, const Csr& B, cudaStream_t s) {
    int64_t n = p_end - p_begin;
    if (n <= 0) return;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (dim == 2)
        { scatter_plain_kernel<2><<<nb, 256, 0, s>>>(sg, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, B.ptr, B.col, B.val); count_launch(); }
    else
        { scatter_plain_kernel<3><<<nb, 256, 0, s>>>(sg, E, p_begin, p_end, pair_elem, pair_cell, blocks, vols, B.ptr, B.col, B.val); count_launch(); }
}

}  // namespace l2x
