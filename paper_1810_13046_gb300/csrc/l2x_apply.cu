// Velocity and force transfer (Sec. 2.3, algebraic form B v_f = S w_s,
// w_s = S^-1 B v_f = T v_f, forces by T^T; Steps 1 and 4 of the FSI algorithm,
// Sec. 3): sparse products with B_g and B_g^T and the Jacobi-preconditioned
// conjugate-gradient solve with S = M_s.
#include <cooperative_groups.h>

#include <cmath>
#include <type_traits>

#include "l2x_fp.cuh"
#include "l2x_internal.cuh"

namespace cg = cooperative_groups;

namespace l2x {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ B x
template <typename TV, typename TM>
struct SpmvPack {
    const int64_t* ptr[kMaxGrids];
    const int32_t* col[kMaxGrids];
    const TM* val[kMaxGrids];
    const TV* x[kMaxGrids];
    TV* y[kMaxGrids];
    const double* scale;  // optional row scaling (1/S_ii of a diagonal S), shared by the grids
};

// Sum of FP32 products in double-float: every product enters exactly (FMA
// two-product), the running sum by Knuth's two-sum, so the mixed form's only
// roundings are those of the FP32 inputs and of the one final result.
struct DFAcc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, pe));
    }
    __device__ __forceinline__ void reduce_xor(int o) {
        const DF r = df_add(DF{hi, lo}, df_shfl_xor(DF{hi, lo}, o));
        hi = r.hi;
        lo = r.lo;
    }
};

// 8 lanes per row; FP64 accumulation in FP64, double-float in the mixed form.
template <typename TV, typename TM>
__global__ void spmv_B_fused_kernel(int n_grids, int64_t n_rows, SpmvPack<TV, TM> P, const DevStatus* st) {
    if (st->flags & kAbortFlags) return;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t grp = tid >> 3;
    const int l8 = threadIdx.x & 7;
    const bool active = grp < n_rows * n_grids;
    const int g = !active ? 0 : grp >= 2 * n_rows ? 2 : grp >= n_rows ? 1 : 0;  // n_grids <= 3
    const int64_t row = active ? grp - g * n_rows : 0;
    if constexpr (sizeof(TV) == 4) {
        DFAcc acc;
        if (active) {
            const int64_t lo = P.ptr[g][row], hi = P.ptr[g][row + 1];
            const int32_t* __restrict__ col = P.col[g];
            const TM* __restrict__ val = P.val[g];
            const TV* __restrict__ x = P.x[g];
#pragma unroll 4
            for (int64_t q = lo + l8; q < hi; q += 8) acc.add_prod((float)__ldg(val + q), __ldg(x + __ldg(col + q)));
        }
        acc.reduce_xor(4);
        acc.reduce_xor(2);
        acc.reduce_xor(1);
        if (active && l8 == 0)
            P.y[g][row] = P.scale ? d2f_int((f2d_int(acc.hi) + f2d_int(acc.lo)) * __ldg(P.scale + row))
                                  : __fadd_rn(acc.hi, acc.lo);
    } else {
        TV acc = TV(0);
        if (active) {
            const int64_t lo = P.ptr[g][row], hi = P.ptr[g][row + 1];
            const int32_t* __restrict__ col = P.col[g];
            const TM* __restrict__ val = P.val[g];
            const TV* __restrict__ x = P.x[g];
#pragma unroll 4
            for (int64_t q = lo + l8; q < hi; q += 8) acc += (TV)__ldg(val + q) * __ldg(x + __ldg(col + q));
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (active && l8 == 0) P.y[g][row] = P.scale ? (TV)((double)acc * __ldg(P.scale + row)) : acc;
    }
}

__global__ void spmv_B_plain_kernel(int64_t n_rows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                                    const double* __restrict__ scale) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    double s = 0.0;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) s += val[q] * x[col[q]];
    y[i] = scale ? s * scale[i] : s;
}

// out_k = mask ⊙ f_k (interface restriction of the force input).
template <typename TV>
__global__ void mask_copy_kernel(int64_t n, int nr, const uint8_t* __restrict__ mask, const TV* f0, const TV* f1,
                                 const TV* f2, TV* o0, TV* o1, TV* o2, const DevStatus* st) {
    if (st->flags & kAbortFlags) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool on = mask[i] != 0;
    o0[i] = on ? f0[i] : TV(0);
    if (nr > 1) o1[i] = on ? f1[i] : TV(0);
    if (nr > 2) o2[i] = on ? f2[i] : TV(0);
}

// w_k = y_k / S_ii for a diagonal S; the product in FP64, one rounding to TV.
template <typename TV>
__global__ void diag_solve_kernel(int64_t n, int nr, const double* __restrict__ dinv, const TV* y0, const TV* y1,
                                  const TV* y2, TV* w0, TV* w1, TV* w2, const DevStatus* st) {
    if (st->flags & kAbortFlags) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double di = dinv[i];
    w0[i] = (TV)((double)y0[i] * di);
    if (nr > 1) w1[i] = (TV)((double)y1[i] * di);
    if (nr > 2) w2[i] = (TV)((double)y2[i] * di);
}

// v_k = s * m_i * v_k in place (m = 1 where no mask is given): the interface
// restriction and the force scale of the force transfer's adjoint; the product
// in FP64, one rounding to TV.
template <typename TV>
__global__ void scale_mask_kernel(int64_t n, int nr, const uint8_t* __restrict__ mask, double scale, TV* v0, TV* v1,
                                  TV* v2, const DevStatus* st) {
    if (st->flags & kAbortFlags) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = (mask && mask[i] == 0) ? 0.0 : scale;
    v0[i] = (TV)((double)v0[i] * f);
    if (nr > 1) v1[i] = (TV)((double)v1[i] * f);
    if (nr > 2) v2[i] = (TV)((double)v2[i] * f);
}

// ------------------------------------------------------------------ Picard norms
template <typename TV>
struct PicardPack {
    const TV* fn[kMaxGrids];
    TV* fp[kMaxGrids];
};

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    // |x| as its bit pattern: for non-negative doubles the unsigned order is the
    // numeric order, and NaN (any payload) sorts above +inf
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// out[0] = max |f_new - f_prev|, out[1] = max |f_new| over all grids and nodes
// (as bit patterns, combined by atomicMax); f_prev = f_new when copy != 0.
template <typename TV>
__global__ void picard_norms_kernel(int64_t n, int G, PicardPack<TV> P, int copy, unsigned long long* out) {
    __shared__ unsigned long long s_d[32], s_f[32];
    unsigned long long dmax = 0, fmax = 0;
    const int64_t total = n * G;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / n);
        const int64_t i = t - (int64_t)g * n;
        const TV a = P.fn[g][i];
        const TV b = P.fp[g][i];
        const unsigned long long d = abs_bits((double)a - (double)b), f = abs_bits((double)a);
        dmax = d > dmax ? d : dmax;
        fmax = f > fmax ? f : fmax;
        if (copy) P.fp[g][i] = a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long d = __shfl_xor_sync(0xffffffffu, dmax, o);
        const unsigned long long f = __shfl_xor_sync(0xffffffffu, fmax, o);
        dmax = d > dmax ? d : dmax;
        fmax = f > fmax ? f : fmax;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_d[w] = dmax;
        s_f[w] = fmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            dmax = s_d[k] > dmax ? s_d[k] : dmax;
            fmax = s_f[k] > fmax ? s_f[k] : fmax;
        }
        atomicMax(out, dmax);
        atomicMax(out + 1, fmax);
    }
}

// ------------------------------------------------------------------ B^T z
// One thread per non-empty row of B_g^T (a fluid node the mesh touches): gather,
// no atomics.  The row list and its length are device values.
// kBTLanes lanes per non-empty row of B_g^T (a fluid node the mesh touches),
// all grids in one launch: gather, no atomics.  The row lists and their lengths
// are device values; the launch covers their capacities.
constexpr int kBTLanes = 4;

template <typename TV, typename TM>
struct SpmvTPack {
    const int32_t* list[kMaxGrids];
    const int64_t* n_list[kMaxGrids];
    const int64_t* ptr[kMaxGrids];
    const int32_t* col[kMaxGrids];
    const TM* val[kMaxGrids];
    const TV* z[kMaxGrids];
    TV* f[kMaxGrids];
    int lo[kMaxGrids][3];
    int nb[kMaxGrids][2];       // rows of the B^T box along x, y
    int nn[kMaxGrids][2];       // fluid nodes of grid g along x, y
    int64_t start[kMaxGrids + 1];  // first row slot of every grid (capacities)
    int G;
};

// Fluid node of row r of the B_g^T box.
template <typename TV, typename TM>
__device__ __forceinline__ int64_t bt_node(const SpmvTPack<TV, TM>& P, int g, int64_t r) {
    // box rows number below 2^31 (int32 fluid-node columns): 32-bit division
    const unsigned int ru = (unsigned int)r, n0 = (unsigned int)P.nb[g][0], n1 = (unsigned int)P.nb[g][1];
    const unsigned int rr = ru / n0;
    const int x = (int)(ru - rr * n0);
    const int zz = (int)(rr / n1);
    const int y = (int)(rr - (unsigned int)zz * n1);
    return (x + P.lo[g][0]) + (int64_t)P.nn[g][0] * ((y + P.lo[g][1]) + (int64_t)P.nn[g][1] * (zz + P.lo[g][2]));
}

template <typename TV, typename TM>
__global__ void spmv_BT_fused_kernel(SpmvTPack<TV, TM> P, TV scale, const DevStatus* st) {
    if (st->flags & kAbortFlags) return;
    // slots of the listed rows of all grids, grid after grid (device counts)
    int64_t first[kMaxGrids + 1];
    first[0] = 0;
    for (int g = 0; g < P.G; ++g) {
        const int64_t cap = P.start[g + 1] - P.start[g];
        const int64_t nl = *P.n_list[g];
        first[g + 1] = first[g] + (nl < cap ? nl : cap);
    }
    const int64_t total = first[P.G];
    const int lane = threadIdx.x % kBTLanes;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x / kBTLanes;
    // every lane group runs the same number of passes (warp-uniform shuffles)
    const int64_t slot0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kBTLanes;
    const int64_t warp_slot0 = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) / kBTLanes;
    for (int64_t base = warp_slot0; base < total; base += stride) {
        const int64_t slot = slot0 + (base - warp_slot0);
        const bool active = slot < total;
        int g = 0;
        while (g + 1 < P.G && slot >= first[g + 1]) ++g;
        int64_t r = 0;
        TV acc = TV(0);
        if constexpr (sizeof(TV) == 4) {  // double-float sum, one rounding at the end
            DFAcc a2;
            if (active) {
                r = P.list[g][slot - first[g]];
                const int64_t hi = P.ptr[g][r + 1];
                const int32_t* __restrict__ col = P.col[g];
                const TM* __restrict__ val = P.val[g];
                const TV* __restrict__ z = P.z[g];
#pragma unroll 4
                for (int64_t q = P.ptr[g][r] + lane; q < hi; q += kBTLanes)
                    a2.add_prod((float)__ldg(val + q), __ldg(z + __ldg(col + q)));
            }
#pragma unroll
            for (int o = kBTLanes / 2; o > 0; o >>= 1) a2.reduce_xor(o);
            if (active && lane == 0) {
                const int64_t node = bt_node(P, g, r);
                P.f[g][node] = __fmaf_rn(scale, a2.lo, __fmaf_rn(scale, a2.hi, P.f[g][node]));
            }
            continue;
        } else {
            if (active) {
                r = P.list[g][slot - first[g]];
                const int64_t hi = P.ptr[g][r + 1];
                const int32_t* __restrict__ col = P.col[g];
                const TM* __restrict__ val = P.val[g];
                const TV* __restrict__ z = P.z[g];
#pragma unroll 4
                for (int64_t q = P.ptr[g][r] + lane; q < hi; q += kBTLanes) acc += (TV)__ldg(val + q) * __ldg(z + __ldg(col + q));
            }
#pragma unroll
            for (int o = kBTLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        if (active && lane == 0) {
            const int x = (int)(r % P.nb[g][0]);
            const int64_t rr = r / P.nb[g][0];
            const int y = (int)(rr % P.nb[g][1]);
            const int zz = (int)(rr / P.nb[g][1]);
            const int64_t node =
                (x + P.lo[g][0]) + (int64_t)P.nn[g][0] * ((y + P.lo[g][1]) + (int64_t)P.nn[g][1] * (zz + P.lo[g][2]));
            P.f[g][node] += scale * acc;
        }
    }
}

__global__ void spmv_BT_plain_kernel(int64_t n_rows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, const double* __restrict__ z, double* f,
                                     double scale) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    double zi = scale * z[i];
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) atomicAdd(f + col[q], val[q] * zi);
}

// ------------------------------------------------------------------ PCG (fused, cooperative)
// right-hand sides of one solve: the components of one transfer (<= 3), or of
// both transfers of a captured step solved together (<= 6)
constexpr int kMaxRhs = 6;

template <typename T>
struct VecPack {
    T* p[kMaxRhs];
};

// Dot-product accumulator: exact double for FP64 vectors; for FP32 vectors the
// product is split exactly (fma) and summed with an error-compensated pair of
// floats, converted to double once per thread.
template <typename TV>
struct DotAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(TV a, TV b) { s = fma((double)a, (double)b, s); }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ DF df(int e) const { return df_from_double(ldexp_d_int(s, e)); }
};
template <>
struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        float p = __fmul_rn(a, b);
        float e = __fmaf_rn(a, b, -p);
        float s = __fadd_rn(hi, p);
        float bb = __fsub_rn(s, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ DF df(int e) const { return df_scale(DF{hi, lo}, e); }
};

template <typename TV>
struct PcgArgs {
    int64_t n;
    int nrhs;
    const int64_t* ptr;
    const int32_t* col;
    const TV* val;
    const TV* dinv;
    const TV* y[kMaxRhs];
    TV* x[kMaxRhs];
    TV* r;   // n * nrhs each, component-major
    TV* u;
    TV* p;
    TV* s;
    TV* w;
    double* partial;  // gridDim.x * 3 * kMaxRhs
    double rtol;
    const double* rtol_k;  // optional per right-hand-side tolerances (device), in place of rtol
    int max_iter;
    DevStatus* st;
};

// Block-wide sums of N values at once (result valid in thread 0 and, through
// `out`, in every thread after the final barrier).
template <int N>
__device__ __forceinline__ void block_sum_n(double (&v)[N], double* sh, double* out) {
#pragma unroll
    for (int j = 0; j < N; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) sh[j * 32 + wid] = v[j];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double t = lane < nw ? sh[j * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) out[j] = t;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// Chronopoulos-Gear form of Jacobi-PCG: one global reduction and one vector
// exchange per iteration (two grid barriers), all right-hand sides together.
// Rows are split evenly over small blocks (2 warps) so that every SM takes part
// even for small systems; the product w = M u uses kRowLanes lanes per row.
// GB300 runs FP64 instructions on a narrow unit, so the per-iteration
// reductions run in double-float single-precision arithmetic (about 48 bits)
// and the scalars alpha, beta of right-hand side k are formed by thread k only.
constexpr int kRowLanes = 4;
constexpr int kPcgBlock = 256;

// Sum of NV double-float values over the kPcgBlock threads of a block: staged in
// shared memory, value j summed by warp j % NW (8 per lane, then 5 shuffle
// levels), result in out[j] after the final barrier.
template <int NV>
__device__ __forceinline__ void block_df_sum(const DF (&v)[NV], DF (*stage)[kPcgBlock], DF* out) {
    constexpr int NW = kPcgBlock / 32;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) stage[j][threadIdx.x] = v[j];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = wid; j < NV; j += NW) {
        DF t = stage[j][lane];
#pragma unroll
        for (int q = 1; q < kPcgBlock / 32; ++q) t = df_add(t, stage[j][lane + 32 * q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = df_add(t, df_shfl_xor(t, o));
        if (lane == 0) out[j] = t;
    }
    __syncthreads();
}

template <typename TV, int NR>
__global__ void __launch_bounds__(kPcgBlock) pcg_fused_kernel(PcgArgs<TV> A) {
    cg::grid_group grid = cg::this_grid();
    constexpr int NV = 3 * NR;                  // gamma, delta, rho per right-hand side
    __shared__ DF s_stage[NV][kPcgBlock];
    __shared__ DF s_dfo[NV];
    __shared__ double s_red[NV * 32];
    __shared__ double s_tot[NV];
    __shared__ double s_alpha[NR], s_beta[NR];
    __shared__ int s_conv[NR], s_all;
    __shared__ int s_exp[NV];
    const int64_t n = A.n;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(n, (int64_t)blockIdx.x * per), r1 = min(n, r0 + per);
    const int glane = threadIdx.x % kRowLanes;
    const int grow = threadIdx.x / kRowLanes;
    constexpr int kRowsPerPass = kPcgBlock / kRowLanes;
    DF* partial = reinterpret_cast<DF*>(A.partial);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kPcgBlock) {
        const TV di = A.dinv[i];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const TV yi = A.y[k][i];
            A.x[k][i] = TV(0);
            A.r[i * NR + k] = yi;
            A.u[i * NR + k] = di * yi;
        }
    }
    // per-rhs state kept by thread k of every block (identical in all blocks)
    double alpha = 0.0, gamma_old = 0.0, rho0 = 0.0, rho = 0.0;
    if (threadIdx.x < NR) s_conv[threadIdx.x] = 0;
    grid.sync();
    int it = 0, it_local = 0, restarts = 0;
    for (;;) {
        DotAcc<TV> dg[NR], dd[NR], dr[NR];
        for (int64_t base = r0; base < r1; base += kRowsPerPass) {
            const int64_t i = base + grow;
            const bool live = i < r1;
            TV acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = TV(0);
            if (live) {
                const int64_t hi = A.ptr[i + 1];
                for (int64_t q = A.ptr[i] + glane; q < hi; q += kRowLanes) {
                    const TV v = A.val[q];
                    const int32_t j = A.col[q];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += v * A.u[(int64_t)j * NR + k];
                }
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
#pragma unroll
                for (int o = kRowLanes / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            }
            if (live) {
                // the xor reduction left every lane of the row with the sums: lane
                // glane takes components glane, glane + kRowLanes, ...
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (k % kRowLanes != glane) continue;
                    const TV ri = A.r[i * NR + k], ui = A.u[i * NR + k];
                    A.w[i * NR + k] = acc[k];
                    dg[k].add(ri, ui);
                    dd[k].add(acc[k], ui);
                    dr[k].add(ri, ri);
                }
            }
        }
        // Reduction of (gamma, delta, rho) per right-hand side.  After a (re)start
        // the sums are formed once in FP64, which also fixes a power-of-two shift
        // per sum (about 2^100 at that point); later iterations sum the shifted
        // values in double-float single precision, whose exponent range then
        // covers the decrease by rtol^2.
        const bool exact = it_local == 0;
        {
            if (exact) {
                double v[NV];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    v[3 * k + 0] = dg[k].value();
                    v[3 * k + 1] = dd[k].value();
                    v[3 * k + 2] = dr[k].value();
                }
                block_sum_n<NV>(v, s_red, s_tot);
                if (threadIdx.x < NV) A.partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s_tot[threadIdx.x];
            } else {
                DF v[NV];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    v[3 * k + 0] = dg[k].df(s_exp[3 * k + 0]);
                    v[3 * k + 1] = dd[k].df(s_exp[3 * k + 1]);
                    v[3 * k + 2] = dr[k].df(s_exp[3 * k + 2]);
                }
                block_df_sum<NV>(v, s_stage, s_dfo);
                if (threadIdx.x < NV) partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s_dfo[threadIdx.x];
            }
        }
        grid.sync();
        // every block sums the partials of all blocks in the same order
        {
            if (exact) {
                double v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = 0.0;
                for (int b = threadIdx.x; b < (int)gridDim.x; b += kPcgBlock) {
#pragma unroll
                    for (int j = 0; j < NV; ++j) v[j] += A.partial[(int64_t)j * gridDim.x + b];
                }
                block_sum_n<NV>(v, s_red, s_tot);
                if (threadIdx.x < NV) {
                    const double t = s_tot[threadIdx.x];
                    s_exp[threadIdx.x] = t > 0.0 ? 100 - ilogb_int(t) : 0;
                }
                __syncthreads();
            } else {
                DF v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = DF{0.f, 0.f};
                for (int b = threadIdx.x; b < (int)gridDim.x; b += kPcgBlock) {
#pragma unroll
                    for (int j = 0; j < NV; ++j) v[j] = df_add(v[j], partial[(int64_t)j * gridDim.x + b]);
                }
                block_df_sum<NV>(v, s_stage, s_dfo);
                if (threadIdx.x < NV) s_tot[threadIdx.x] = ldexp_d_int(df_to_double(s_dfo[threadIdx.x]), -s_exp[threadIdx.x]);
                __syncthreads();
            }
            if (threadIdx.x < NR) {
                const int k = threadIdx.x;
                const double gam = s_tot[3 * k], del = s_tot[3 * k + 1];
                rho = s_tot[3 * k + 2];
                if (it == 0) rho0 = rho;
                const double tol = A.rtol_k ? A.rtol_k[k] : A.rtol;
                const bool conv = rho <= tol * tol * rho0;
                double beta = 0.0;
                if (!conv) {
                    if (it_local == 0) {
                        alpha = div_nr(gam, del);
                    } else {
                        beta = div_nr(gam, gamma_old);
                        alpha = div_nr(gam, del - beta * div_nr(gam, alpha));
                    }
                    gamma_old = gam;
                }
                s_alpha[k] = alpha;
                s_beta[k] = beta;
                s_conv[k] = conv ? 1 : 0;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
#pragma unroll
                for (int k = 0; k < NR; ++k) all &= s_conv[k];
                s_all = all;
            }
            __syncthreads();
        }
        if (s_all && sizeof(TV) == 8 && restarts < 2) {
            // FP64: check the true residual y - M x and restart from it if the
            // recurrence has drifted (Chronopoulos-Gear keeps an extra recurrence)
            grid.sync();
            DotAcc<TV> dt[NR];
            for (int64_t i = r0 + threadIdx.x; i < r1; i += kPcgBlock) {
                const int64_t hi = A.ptr[i + 1];
                TV acc[NR];
#pragma unroll
                for (int k = 0; k < NR; ++k) acc[k] = TV(0);
                for (int64_t q = A.ptr[i]; q < hi; ++q) {
                    const TV v = A.val[q];
                    const int32_t j = A.col[q];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += v * A.x[k][j];
                }
                const TV di = A.dinv[i];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const TV rt = A.y[k][i] - acc[k];
                    A.r[i * NR + k] = rt;
                    A.u[i * NR + k] = di * rt;
                    dt[k].add(rt, rt);
                }
            }
            {
                double v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = 0.0;
#pragma unroll
                for (int k = 0; k < NR; ++k) v[k] = dt[k].value();
                block_sum_n<NV>(v, s_red, s_tot);
                if (threadIdx.x < NV) A.partial[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = s_tot[threadIdx.x];
            }
            grid.sync();
            {
                double v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = 0.0;
                for (int b = threadIdx.x; b < (int)gridDim.x; b += kPcgBlock) {
#pragma unroll
                    for (int k = 0; k < NR; ++k) v[k] += A.partial[(int64_t)k * gridDim.x + b];
                }
                block_sum_n<NV>(v, s_red, s_tot);
                if (threadIdx.x < NR) {
                    const double rt = s_tot[threadIdx.x];
                    const bool ok = rt <= A.rtol * A.rtol * rho0;
                    s_conv[threadIdx.x] = ok ? 1 : 0;
                    if (!ok) rho = rt;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int all = 1;
#pragma unroll
                    for (int k = 0; k < NR; ++k) all &= s_conv[k];
                    s_all = all;
                }
                __syncthreads();
            }
            if (s_all) break;
            // restart the recurrences from the true residual (r, u already written)
            ++restarts;
            it_local = 0;
            grid.sync();
            continue;
        }
        if (s_all || it >= A.max_iter) break;
        // one thread per (row, component): the interleaved vectors are read and
        // written contiguously
        for (int64_t o = r0 * NR + threadIdx.x; o < r1 * NR; o += kPcgBlock) {
            const int64_t i = o / NR;
            const int k = (int)(o - i * NR);
            if (s_conv[k]) continue;
            const TV b = (TV)s_beta[k], a = (TV)s_alpha[k];
            const TV pn = it_local == 0 ? A.u[o] : A.u[o] + b * A.p[o];
            const TV sn = it_local == 0 ? A.w[o] : A.w[o] + b * A.s[o];
            A.p[o] = pn;
            A.s[o] = sn;
            A.x[k][i] += a * pn;
            const TV rn = A.r[o] - a * sn;
            A.r[o] = rn;
            A.u[o] = A.dinv[i] * rn;
        }
        grid.sync();
        ++it;
        ++it_local;
    }
    if (blockIdx.x == 0) {
        // residual of every rhs: thread k holds rho, rho0
        double rel = threadIdx.x < NR && rho0 > 0.0 ? sqrt(rho / rho0) : 0.0;
        for (int o = 16; o > 0; o >>= 1) rel = fmax(rel, __shfl_xor_sync(0xffffffffu, rel, o));
        if (threadIdx.x == 0) {
            A.st->cg_iters = it;
            A.st->cg_residual = rel;
            if (!s_all) atomicOr(&A.st->flags, FLAG_NOTCONVERGED);
        }
    }
}

// ------------------------------------------------------------------ PCG (one thread-block cluster)
// The same Chronopoulos-Gear Jacobi-PCG for systems whose search direction u
// fits in the distributed shared memory of one cluster of C CTAs (C <= 16).
// CTA c owns rows [c*S, min(n, (c+1)*S)); its slice of u lives in its own
// shared memory as [row][rhs], and the product w = M u reads the other slices
// through DSMEM.  The per-iteration sums are gathered through DSMEM in a fixed
// order (every CTA forms identical scalars) and the two barriers per iteration
// are hardware cluster barriers, which is what makes small systems fast: the
// grid-wide form pays two device-wide barriers and an L2 round trip for the
// partial sums in every iteration.
constexpr int kCluThreads = 512;
constexpr int kCluMax = 16;

template <typename TV, int NR>
__global__ void __launch_bounds__(kCluThreads, 1) pcg_cluster_kernel(PcgArgs<TV> A, int S) {
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int NV = 3 * NR;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    TV* su = reinterpret_cast<TV*>(dyn_smem);  // S x NR: this CTA's rows of u
    __shared__ const TV* s_base[kCluMax];       // every CTA's slice (DSMEM addresses)
    __shared__ double s_part[NV];               // this CTA's partial sums, read by all CTAs
    __shared__ double s_gather[kCluMax * NV];
    __shared__ double s_red[NV * 32];
    __shared__ double s_tot[NV];
    __shared__ double s_alpha[NR], s_beta[NR];
    __shared__ int s_conv[NR], s_all;
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int64_t n = A.n;
    const int64_t r0 = min(n, (int64_t)rank * S), r1 = min(n, r0 + S);
    const int glane = threadIdx.x % kRowLanes;
    const int grow = threadIdx.x / kRowLanes;
    constexpr int kRowsPerPass = kCluThreads / kRowLanes;
    if (threadIdx.x < C) s_base[threadIdx.x] = cluster.map_shared_rank(su, (unsigned)threadIdx.x);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += kCluThreads) {
        const TV di = A.dinv[i];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const TV yi = A.y[k][i];
            A.x[k][i] = TV(0);
            A.r[k * n + i] = yi;
            su[(i - r0) * NR + k] = di * yi;
        }
    }
    if (threadIdx.x < NR) s_conv[threadIdx.x] = 0;
    cluster.sync();
    // value of column j of the distributed vector held in the slices
    auto fetch = [&](int32_t j, int k) -> TV {
        if (j >= r0 && j < r1) return su[(j - r0) * NR + k];
        const unsigned owner = (unsigned)j / (unsigned)S;
        return s_base[owner][(j - (int64_t)owner * S) * NR + k];
    };
    double alpha = 0.0, gamma_old = 0.0, rho0 = 0.0, rho = 0.0;
    int it = 0, it_local = 0, restarts = 0;
    for (;;) {
        DotAcc<TV> dg[NR], dd[NR], dr[NR];
        for (int64_t base = r0; base < r1; base += kRowsPerPass) {
            const int64_t i = base + grow;
            const bool live = i < r1;
            TV acc[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = TV(0);
            if (live) {
                const int64_t hi = A.ptr[i + 1];
                for (int64_t q = A.ptr[i] + glane; q < hi; q += kRowLanes) {
                    const TV v = A.val[q];
                    const int32_t j = A.col[q];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += v * fetch(j, k);
                }
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
#pragma unroll
                for (int o = kRowLanes / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            }
            if (live && glane == 0) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const TV ri = A.r[k * n + i], ui = su[(i - r0) * NR + k];
                    A.w[k * n + i] = acc[k];
                    dg[k].add(ri, ui);
                    dd[k].add(acc[k], ui);
                    dr[k].add(ri, ri);
                }
            }
        }
        {
            double v[NV];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                v[3 * k + 0] = dg[k].value();
                v[3 * k + 1] = dd[k].value();
                v[3 * k + 2] = dr[k].value();
            }
            block_sum_n<NV>(v, s_red, s_part);
        }
        cluster.sync();  // partial sums published; every read of u for this product is done
        if (threadIdx.x < C * NV)
            s_gather[threadIdx.x] = *cluster.map_shared_rank(&s_part[threadIdx.x % NV], (unsigned)(threadIdx.x / NV));
        __syncthreads();
        if (threadIdx.x < NV) {
            double t = 0.0;
            for (int c = 0; c < C; ++c) t += s_gather[c * NV + threadIdx.x];
            s_tot[threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x < NR) {
            const int k = threadIdx.x;
            const double gam = s_tot[3 * k], del = s_tot[3 * k + 1];
            rho = s_tot[3 * k + 2];
            if (it == 0 && it_local == 0 && restarts == 0) rho0 = rho;
            const double tol = A.rtol_k ? A.rtol_k[k] : A.rtol;
            const bool conv = rho <= tol * tol * rho0;
            double beta = 0.0;
            if (!conv) {
                if (it_local == 0) {
                    alpha = div_nr(gam, del);
                } else {
                    beta = div_nr(gam, gamma_old);
                    alpha = div_nr(gam, del - beta * div_nr(gam, alpha));
                }
                gamma_old = gam;
            }
            s_alpha[k] = alpha;
            s_beta[k] = beta;
            s_conv[k] = conv ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
#pragma unroll
            for (int k = 0; k < NR; ++k) all &= s_conv[k];
            s_all = all;
        }
        __syncthreads();
        if (s_all && sizeof(TV) == 8 && restarts < 2) {
            // FP64: true residual y - M x; the slices of x go through the u buffers
            // (every CTA has finished its product and its gather of the sums)
            for (int64_t i = r0 + threadIdx.x; i < r1; i += kCluThreads)
#pragma unroll
                for (int k = 0; k < NR; ++k) su[(i - r0) * NR + k] = A.x[k][i];
            cluster.sync();
            DotAcc<TV> dt[NR];
            for (int64_t i = r0 + threadIdx.x; i < r1; i += kCluThreads) {
                const int64_t hi = A.ptr[i + 1];
                TV acc[NR];
#pragma unroll
                for (int k = 0; k < NR; ++k) acc[k] = TV(0);
                for (int64_t q = A.ptr[i]; q < hi; ++q) {
                    const TV v = A.val[q];
                    const int32_t j = A.col[q];
#pragma unroll
                    for (int k = 0; k < NR; ++k) acc[k] += v * fetch(j, k);
                }
                const TV di = A.dinv[i];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const TV rt = A.y[k][i] - acc[k];
                    A.r[k * n + i] = rt;
                    A.u[k * n + i] = di * rt;  // staged: the slices still hold x
                    dt[k].add(rt, rt);
                }
            }
            {
                double v[NV];
#pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = 0.0;
#pragma unroll
                for (int k = 0; k < NR; ++k) v[k] = dt[k].value();
                block_sum_n<NV>(v, s_red, s_part);
            }
            cluster.sync();  // sums published; every read of the x slices is done
            if (threadIdx.x < C * NR)
                s_gather[threadIdx.x] = *cluster.map_shared_rank(&s_part[threadIdx.x % NR], (unsigned)(threadIdx.x / NR));
            __syncthreads();
            if (threadIdx.x < NR) {
                double t = 0.0;
                for (int c = 0; c < C; ++c) t += s_gather[c * NR + threadIdx.x];
                const bool ok = t <= A.rtol * A.rtol * rho0;
                s_conv[threadIdx.x] = ok ? 1 : 0;
                if (!ok) rho = t;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
#pragma unroll
                for (int k = 0; k < NR; ++k) all &= s_conv[k];
                s_all = all;
            }
            for (int64_t i = r0 + threadIdx.x; i < r1; i += kCluThreads)
#pragma unroll
                for (int k = 0; k < NR; ++k) su[(i - r0) * NR + k] = A.u[k * n + i];
            __syncthreads();
            if (s_all) break;
            ++restarts;
            it_local = 0;
            cluster.sync();  // new u slices visible before the next product
            continue;
        }
        if (s_all || it >= A.max_iter) break;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += kCluThreads) {
            const TV di = A.dinv[i];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                if (s_conv[k]) continue;
                const int64_t o = k * n + i;
                const TV b = (TV)s_beta[k], a = (TV)s_alpha[k];
                const TV ui = su[(i - r0) * NR + k];
                const TV pn = it_local == 0 ? ui : ui + b * A.p[o];
                const TV sn = it_local == 0 ? A.w[o] : A.w[o] + b * A.s[o];
                A.p[o] = pn;
                A.s[o] = sn;
                A.x[k][i] += a * pn;
                const TV rn = A.r[o] - a * sn;
                A.r[o] = rn;
                su[(i - r0) * NR + k] = di * rn;
            }
        }
        cluster.sync();  // new u slices visible before the next product
        ++it;
        ++it_local;
    }
    if (rank == 0) {
        double rel = threadIdx.x < NR && rho0 > 0.0 ? sqrt(rho / rho0) : 0.0;
        for (int o = 16; o > 0; o >>= 1) rel = fmax(rel, __shfl_xor_sync(0xffffffffu, rel, o));
        if (threadIdx.x == 0) {
            A.st->cg_iters = it;
            A.st->cg_residual = rel;
            if (!s_all) atomicOr(&A.st->flags, FLAG_NOTCONVERGED);
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------------------ PCG (plain, unfused, FP64)
__global__ void plain_init_kernel(int64_t n, int nr, const double* y0, const double* y1, const double* y2,
                                  double* x0, double* x1, double* x2, const double* dinv, double* r, double* z,
                                  double* p) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* y[3] = {y0, y1, y2};
    double* x[3] = {x0, x1, x2};
    for (int k = 0; k < nr; ++k) {
        double yi = y[k][i];
        x[k][i] = 0.0;
        r[k * n + i] = yi;
        z[k * n + i] = dinv[i] * yi;
        p[k * n + i] = dinv[i] * yi;
    }
}

__global__ void plain_spmv_kernel(int64_t n, int nr, const int64_t* ptr, const int32_t* col, const double* val,
                                  const double* p, double* q) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nr; ++k) {
        double s = 0.0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += val[e] * p[k * n + col[e]];
        q[k * n + i] = s;
    }
}

// out[k] += sum_i a[k*n+i] * b[k*n+i]
__global__ void plain_dot_kernel(int64_t n, int nr, const double* a, const double* b, double* out) {
    __shared__ double sh[32];
    for (int k = 0; k < nr; ++k) {
        double v = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            v += a[k * n + i] * b[k * n + i];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) atomicAdd(out + k, v);
    }
}

// scal: [0..2] rz, [3..5] pq, [6..8] rz_new, [9..11] rr, [12..14] active flag
__global__ void plain_update_x_kernel(int64_t n, int nr, const double* scal, double* x0, double* x1, double* x2,
                                      double* r, double* z, const double* p, const double* q, const double* dinv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* x[3] = {x0, x1, x2};
    for (int k = 0; k < nr; ++k) {
        if (scal[12 + k] == 0.0) continue;
        double alpha = scal[k] / scal[3 + k];
        x[k][i] += alpha * p[k * n + i];
        double rn = r[k * n + i] - alpha * q[k * n + i];
        r[k * n + i] = rn;
        z[k * n + i] = dinv[i] * rn;
    }
}

__global__ void plain_update_p_kernel(int64_t n, int nr, const double* scal, const double* z, double* p) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nr; ++k) {
        if (scal[12 + k] == 0.0) continue;
        double beta = scal[6 + k] / scal[k];
        p[k * n + i] = z[k * n + i] + beta * p[k * n + i];
    }
}

// a component with a zero right-hand side has the solution 0 and takes no step
__global__ void plain_active_kernel(int nr, double* scal, const double* rr0) {
    if (threadIdx.x < nr) scal[12 + threadIdx.x] = rr0[threadIdx.x] > 0.0 ? 1.0 : 0.0;
}

__global__ void plain_scalars_kernel(int nr, double* scal, const double* rr0, double rtol) {
    // after an iteration: rz <- rz_new, clear accumulators, freeze converged components
    if (threadIdx.x != 0) return;
    for (int k = 0; k < nr; ++k) {
        if (scal[12 + k] != 0.0) scal[k] = scal[6 + k];
        if (scal[9 + k] <= rtol * rtol * rr0[k]) scal[12 + k] = 0.0;
        scal[3 + k] = 0.0;
        scal[6 + k] = 0.0;
        scal[9 + k] = 0.0;
    }
}

// ------------------------------------------------------------------ mixed-precision refinement
// r64 = y - M x64 (FP64), norms[k] += |r64|^2
// Power of two by which the FP32 correction solves see the residual of right-hand
// side k: about 2^30 over the typical entry of y_k (|y_k| / sqrt(n)), so that
// residuals down to rtol |y| and the products of their entries stay far from
// the FP32 subnormal range (where the FMA two-product of the double-float dots
// is no longer exact).  Exact scaling by a power of two; 0 for y_k = 0.
__device__ __forceinline__ int corr_exp(double ynorm2, int64_t n) {
    if (!(ynorm2 > 0.0)) return 0;
    const int lg_n = 63 - __clzll((unsigned long long)n);
    return 30 - ((ilogb_int(ynorm2) - lg_n) >> 1);
}

__global__ void residual_f64_kernel(int64_t n, int nr, const int64_t* ptr, const int32_t* col, const double* val,
                                    VecPack<const float> y, const double* x64, double* r64, float* r32,
                                    double* norms, const double* ynorm2) {
    __shared__ double sh[32];
    for (int k = 0; k < nr; ++k) {
        double acc = 0.0;
        const int ek = corr_exp(ynorm2[k], n);
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            double s = 0.0;
            for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s = fma(val[e], x64[k * n + col[e]], s);
            double ri = (double)y.p[k][i] - s;
            r64[k * n + i] = ri;
            r32[k * n + i] = (float)ldexp_d_int(ri, ek);
            acc = fma(ri, ri, acc);
        }
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) atomicAdd(norms + k, acc);
    }
}

// x += d: the first solve's result as it is, a correction scaled back by the
// power of two its right-hand side was scaled by (corr_exp).
__global__ void add_correction_kernel(int64_t n, int nr, double* x64, VecPack<const float> d, int first,
                                      const double* ynorm2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nr; ++k) {
        if (first) x64[k * n + i] = (double)d.p[k][i];
        else x64[k * n + i] += ldexp_d_int((double)d.p[k][i], -corr_exp(ynorm2[k], n));
    }
}

__global__ void norm2_f32_kernel(int64_t n, int nr, VecPack<const float> y, double* out) {
    __shared__ double sh[32];
    for (int k = 0; k < nr; ++k) {
        double acc = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            acc = fma((double)y.p[k][i], (double)y.p[k][i], acc);
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) atomicAdd(out + k, acc);
    }
}

// Tolerance of the FP32 correction solve of right-hand side k: the residual
// ||y - M x|| must end at rtol ||y||, and the correction solve M d = r reduces
// ||r|| by its relative tolerance, so tau_k = rtol ||y_k|| / ||r_k||, kept in
// [1e-7, 1] (FP32 cannot do better than about 1e-7).
__global__ void inner_tol_kernel(int nr, double rtol, const double* rr, const double* yy, double* tau) {
    const int k = threadIdx.x;
    if (k >= nr) return;
    double t = rr[k] > 0.0 ? rtol * sqrt(yy[k] / rr[k]) : 1.0;
    tau[k] = fmin(1.0, fmax(1e-7, t));
}

__global__ void store_f32_kernel(int64_t n, int nr, const double* x64, VecPack<float> w) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nr; ++k) w.p[k][i] = (float)x64[k * n + i];
}

template <typename TV, int NR>
int pcg_blocks_for(int64_t n, int rows_per_block_req) {
    static int sms = 0, per_sm = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_fused_kernel<TV, NR>, kPcgBlock, 0);
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t rows_per_block = rows_per_block_req > 0 ? rows_per_block_req : kPcgBlock / kRowLanes;
    int64_t want = (n + rows_per_block - 1) / rows_per_block;
    int64_t cap = (int64_t)sms * per_sm;
    int64_t b = want < cap ? want : cap;
    if (b > (int64_t)sms * 8) b = (int64_t)sms * 8;  // partial-sum buffer holds sms * 8 blocks
    return b < 1 ? 1 : (int)b;
}

// Dynamic shared memory of the cluster PCG: one CTA's rows of u (S x NR values).
constexpr size_t kCluSmemMax = 220 * 1024;

template <typename TV, int NR>
bool cluster_fits(int64_t n, int C, int& S, size_t& smem) {
    if (C < 2 || C > kCluMax || n <= 0) return false;
    const int64_t s_rows = (n + C - 1) / C;
    smem = (size_t)s_rows * NR * sizeof(TV);
    S = (int)s_rows;
    return smem <= kCluSmemMax;
}

template <typename TV, int NR>
cudaError_t launch_pcg_cluster(const PcgArgs<TV>& A, int C, cudaStream_t s) {
    int S = 0;
    size_t smem = 0;
    if (!cluster_fits<TV, NR>(A.n, C, S, smem)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kCluThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pcg_cluster_kernel<TV, NR>, A, S);
}

template <typename TV, int NR>
void prepare_cluster_kernel() {
    cudaFuncSetAttribute(pcg_cluster_kernel<TV, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCluSmemMax);
    cudaFuncSetAttribute(pcg_cluster_kernel<TV, NR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename TV>
cudaError_t run_pcg_fused(const int64_t* ptr, const int32_t* col, const TV* val, const TV* dinv, int64_t n,
                          int nr, const TV* const* y, TV* const* x, TV* vecs, double* partial, double rtol,
                          int max_iter, DevStatus* st, cudaStream_t s, int rpb = 64, int clu = 0,
                          const double* rtol_k = nullptr) {
    PcgArgs<TV> A{};
    A.n = n;
    A.nrhs = nr;
    A.ptr = ptr;
    A.col = col;
    A.val = val;
    A.dinv = dinv;
    for (int k = 0; k < kMaxRhs; ++k) {
        A.y[k] = k < nr ? y[k] : nullptr;
        A.x[k] = k < nr ? x[k] : nullptr;
    }
    int64_t stride = n * nr;
    A.r = vecs;
    A.u = vecs + stride;
    A.p = vecs + 2 * stride;
    A.s = vecs + 3 * stride;
    A.w = vecs + 4 * stride;
    A.partial = partial;
    A.rtol = rtol;
    A.rtol_k = rtol_k;
    A.max_iter = max_iter;
    A.st = st;
    void* args[] = {&A};
    count_launch();
    if (clu > 0 && nr <= 3) {
        int S = 0;
        size_t smem = 0;
        const bool fits = nr == 1 ? cluster_fits<TV, 1>(n, clu, S, smem)
                                  : nr == 2 ? cluster_fits<TV, 2>(n, clu, S, smem) : cluster_fits<TV, 3>(n, clu, S, smem);
        if (fits) {
            switch (nr) {
                case 1: return launch_pcg_cluster<TV, 1>(A, clu, s);
                case 2: return launch_pcg_cluster<TV, 2>(A, clu, s);
                default: return launch_pcg_cluster<TV, 3>(A, clu, s);
            }
        }
    }
    switch (nr) {
        case 1:
            return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<TV, 1>, dim3(pcg_blocks_for<TV, 1>(n, rpb)),
                                               dim3(kPcgBlock), args, 0, s);
        case 2:
            return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<TV, 2>, dim3(pcg_blocks_for<TV, 2>(n, rpb)),
                                               dim3(kPcgBlock), args, 0, s);
        case 4:
            return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<TV, 4>, dim3(pcg_blocks_for<TV, 4>(n, rpb)),
                                               dim3(kPcgBlock), args, 0, s);
        case 6:
            return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<TV, 6>, dim3(pcg_blocks_for<TV, 6>(n, rpb)),
                                               dim3(kPcgBlock), args, 0, s);
        case 3:
            return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<TV, 3>, dim3(pcg_blocks_for<TV, 3>(n, rpb)),
                                               dim3(kPcgBlock), args, 0, s);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace

void pcg_cluster_prepare() {
    static bool done = false;
    if (done) return;
    prepare_cluster_kernel<double, 1>(); prepare_cluster_kernel<double, 2>(); prepare_cluster_kernel<double, 3>();
    prepare_cluster_kernel<float, 1>(); prepare_cluster_kernel<float, 2>(); prepare_cluster_kernel<float, 3>();
    done = true;
}

bool pcg_cluster_usable(int precision, int64_t n, int nr, int C) {
    int S = 0;
    size_t smem = 0;
    bool fits;
    if (precision == L2X_MIXED)
        fits = nr == 1 ? cluster_fits<float, 1>(n, C, S, smem) : nr == 2 ? cluster_fits<float, 2>(n, C, S, smem) : cluster_fits<float, 3>(n, C, S, smem);
    else
        fits = nr == 1 ? cluster_fits<double, 1>(n, C, S, smem) : nr == 2 ? cluster_fits<double, 2>(n, C, S, smem) : cluster_fits<double, 3>(n, C, S, smem);
    if (!fits) return false;
    // the FP64 form of the solve needs both instantiations (the mixed form runs FP32 solves only)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kCluThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e = precision == L2X_MIXED
                        ? cudaOccupancyMaxActiveClusters(&clusters, pcg_cluster_kernel<float, 3>, &cfg)
                        : cudaOccupancyMaxActiveClusters(&clusters, pcg_cluster_kernel<double, 3>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters > 0;
}

int pcg_max_blocks() {
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 8;
}

size_t pcg_ws_bytes(int64_t n, int n_rhs, int max_blocks) {
    // 5 vectors (double upper bound) + mixed: x64, r64 (double), r32, d (float) + partials + plain scalars
    size_t v = (size_t)n * n_rhs;
    return 5 * v * sizeof(double) + 2 * v * sizeof(double) + 2 * v * sizeof(float) +
           (size_t)max_blocks * 3 * kMaxRhs * sizeof(double) + 64 * sizeof(double) + 16384;
}

void launch_picard_norms(int precision, int64_t n, int G, const void* const* f_new, void* const* f_prev, int copy,
                         double* norms, cudaStream_t s) {
    cudaMemsetAsync(norms, 0, 2 * sizeof(double), s);
    if (n <= 0 || G <= 0) return;
    const int64_t total = n * G;
    int64_t nb = (total + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    unsigned long long* out = reinterpret_cast<unsigned long long*>(norms);
    if (precision == L2X_MIXED) {
        PicardPack<float> P{};
        for (int g = 0; g < G; ++g) { P.fn[g] = (const float*)f_new[g]; P.fp[g] = (float*)f_prev[g]; }
        { picard_norms_kernel<float><<<(unsigned)nb, 256, 0, s>>>(n, G, P, copy, out); count_launch(); }
    } else {
        PicardPack<double> P{};
        for (int g = 0; g < G; ++g) { P.fn[g] = (const double*)f_new[g]; P.fp[g] = (double*)f_prev[g]; }
        { picard_norms_kernel<double><<<(unsigned)nb, 256, 0, s>>>(n, G, P, copy, out); count_launch(); }
    }
}

void launch_mask_copy(int precision, int64_t n, int nr, const uint8_t* mask, const void* const* f, void* const* out,
                      const DevStatus* st, cudaStream_t s) {
    if (n <= 0 || nr <= 0) return;
    if (precision == L2X_MIXED) {
        const float* ff[3] = {(const float*)f[0], nr > 1 ? (const float*)f[1] : nullptr, nr > 2 ? (const float*)f[2] : nullptr};
        float* oo[3] = {(float*)out[0], nr > 1 ? (float*)out[1] : nullptr, nr > 2 ? (float*)out[2] : nullptr};
        { mask_copy_kernel<float><<<nblk(n, 256), 256, 0, s>>>(n, nr, mask, ff[0], ff[1], ff[2], oo[0], oo[1], oo[2], st); count_launch(); }
    } else {
        const double* ff[3] = {(const double*)f[0], nr > 1 ? (const double*)f[1] : nullptr, nr > 2 ? (const double*)f[2] : nullptr};
        double* oo[3] = {(double*)out[0], nr > 1 ? (double*)out[1] : nullptr, nr > 2 ? (double*)out[2] : nullptr};
        { mask_copy_kernel<double><<<nblk(n, 256), 256, 0, s>>>(n, nr, mask, ff[0], ff[1], ff[2], oo[0], oo[1], oo[2], st); count_launch(); }
    }
}

void launch_diag_solve(int precision, int64_t n, int nr, const double* dinv, const void* const* y,
                       void* const* w, const DevStatus* st, cudaStream_t s) {
    if (n <= 0 || nr <= 0) return;
    if (precision == L2X_MIXED) {
        const float* yy[3] = {(const float*)y[0], nr > 1 ? (const float*)y[1] : nullptr, nr > 2 ? (const float*)y[2] : nullptr};
        float* ww[3] = {(float*)w[0], nr > 1 ? (float*)w[1] : nullptr, nr > 2 ? (float*)w[2] : nullptr};
        { diag_solve_kernel<float><<<nblk(n, 256), 256, 0, s>>>(n, nr, dinv, yy[0], yy[1], yy[2], ww[0], ww[1], ww[2], st); count_launch(); }
    } else {
        const double* yy[3] = {(const double*)y[0], nr > 1 ? (const double*)y[1] : nullptr, nr > 2 ? (const double*)y[2] : nullptr};
        double* ww[3] = {(double*)w[0], nr > 1 ? (double*)w[1] : nullptr, nr > 2 ? (double*)w[2] : nullptr};
        { diag_solve_kernel<double><<<nblk(n, 256), 256, 0, s>>>(n, nr, dinv, yy[0], yy[1], yy[2], ww[0], ww[1], ww[2], st); count_launch(); }
    }
}

void launch_scale_mask(int precision, int64_t n, int nr, const uint8_t* mask, double scale, void* const* v,
                       const DevStatus* st, cudaStream_t s) {
    if (n <= 0 || nr <= 0) return;
    if (precision == L2X_MIXED) {
        float* vv[3] = {(float*)v[0], nr > 1 ? (float*)v[1] : nullptr, nr > 2 ? (float*)v[2] : nullptr};
        { scale_mask_kernel<float><<<nblk(n, 256), 256, 0, s>>>(n, nr, mask, scale, vv[0], vv[1], vv[2], st); count_launch(); }
    } else {
        double* vv[3] = {(double*)v[0], nr > 1 ? (double*)v[1] : nullptr, nr > 2 ? (double*)v[2] : nullptr};
        { scale_mask_kernel<double><<<nblk(n, 256), 256, 0, s>>>(n, nr, mask, scale, vv[0], vv[1], vv[2], st); count_launch(); }
    }
}

void launch_spmv_B(int path, int precision, int n_grids, const Csr* B, const void* const* x, void* const* y,
                   const DevStatus* st, cudaStream_t s, const double* row_scale) {
    const int64_t n = B[0].n_rows;
    if (n <= 0) return;
    if (path == L2X_PATH_PLAIN) {
        for (int g = 0; g < n_grids; ++g)
            { spmv_B_plain_kernel<<<nblk(n, 256), 256, 0, s>>>(n, B[g].ptr, B[g].col, B[g].val, (const double*)x[g],
                                                             (double*)y[g], row_scale); count_launch(); }
        return;
    }
    const int64_t threads = n * n_grids * 8;
    if (precision == L2X_MIXED) {
        SpmvPack<float, float> P{};
        for (int g = 0; g < n_grids; ++g) {
            P.ptr[g] = B[g].ptr; P.col[g] = B[g].col; P.val[g] = B[g].val32;
            P.x[g] = (const float*)x[g]; P.y[g] = (float*)y[g];
        }
        P.scale = row_scale;
        { spmv_B_fused_kernel<float, float><<<nblk(threads, 256), 256, 0, s>>>(n_grids, n, P, st); count_launch(); }
    } else {
        SpmvPack<double, double> P{};
        for (int g = 0; g < n_grids; ++g) {
            P.ptr[g] = B[g].ptr; P.col[g] = B[g].col; P.val[g] = B[g].val;
            P.x[g] = (const double*)x[g]; P.y[g] = (double*)y[g];
        }
        P.scale = row_scale;
        { spmv_B_fused_kernel<double, double><<<nblk(threads, 256), 256, 0, s>>>(n_grids, n, P, st); count_launch(); }
    }
}

void launch_spmv_BT(int path, int precision, int n_grids, const Csr* B, const CsrT* Tm, const SubGrid* sg,
                    const void* const* z, void* const* f, double scale, const DevStatus* st, cudaStream_t s) {
    if (path == L2X_PATH_PLAIN) {
        for (int g = 0; g < n_grids; ++g)
            if (B[g].n_rows > 0)
                { spmv_BT_plain_kernel<<<nblk(B[g].n_rows, 256), 256, 0, s>>>(B[g].n_rows, B[g].ptr, B[g].col, B[g].val,
                                                                            (const double*)z[g], (double*)f[g], scale); count_launch(); }
        return;
    }
    auto launch = [&](auto* tag_v, auto* tag_m, const auto* const* vals) {
        using TV = std::remove_pointer_t<decltype(tag_v)>;
        using TM = std::remove_pointer_t<decltype(tag_m)>;
        SpmvTPack<TV, TM> P{};
        P.G = n_grids;
        int64_t acc = 0;
        for (int g = 0; g < n_grids; ++g) {
            const CsrT& T = Tm[g];
            const int64_t nl = T.list_cap < T.n_rows ? T.list_cap : T.n_rows;
            P.start[g] = acc;
            acc += nl > 0 ? nl : 0;
            P.list[g] = T.list;
            P.n_list[g] = T.n_list;
            P.ptr[g] = T.ptr;
            P.col[g] = T.col;
            P.val[g] = (const TM*)vals[g];
            P.z[g] = (const TV*)z[g];
            P.f[g] = (TV*)f[g];
            for (int k = 0; k < 3; ++k) P.lo[g][k] = T.lo[k];
            P.nb[g][0] = T.n[0];
            P.nb[g][1] = T.n[1];
            P.nn[g][0] = sg[g].nnode[0];
            P.nn[g][1] = sg[g].nnode[1];
        }
        P.start[n_grids] = acc;
        if (acc <= 0) return;
        unsigned nb = nblk(acc * kBTLanes, 256);
        if (nb > 152 * 8) nb = 152 * 8;  // grid-stride over the rows actually listed
        { spmv_BT_fused_kernel<TV, TM><<<nb, 256, 0, s>>>(P, (TV)scale, st); count_launch(); }
    };
    const void* vals[kMaxGrids];
    if (precision == L2X_MIXED) {
        for (int g = 0; g < n_grids; ++g) vals[g] = Tm[g].val32;
        launch((float*)nullptr, (float*)nullptr, vals);
    } else {
        for (int g = 0; g < n_grids; ++g) vals[g] = Tm[g].val;
        launch((double*)nullptr, (double*)nullptr, vals);
    }
}

void solve_mass_pcg_async(int precision, const Csr& M, const double* diag_inv, const float* diag_inv32, int nr,
                          const void* const* y, void* const* w, double rtol, int max_iter, void* ws, DevStatus* st,
                          cudaStream_t s, int rpb, int clu) {
    const int64_t n = M.n_rows;
    if (n <= 0 || nr <= 0) return;
    const int64_t v = n * nr;
    char* base = (char*)ws;
    auto take = [&](size_t bytes) {
        void* p = base;
        base += (bytes + 255) & ~(size_t)255;
        return p;
    };
    double* partial = (double*)take((size_t)pcg_max_blocks() * 3 * kMaxRhs * 8);
    if (precision == L2X_FP64) {
        double* vecs = (double*)take(5 * v * 8);
        run_pcg_fused<double>(M.ptr, M.col, M.val, diag_inv, n, nr, (const double* const*)y, (double* const*)w, vecs,
                              partial, rtol, max_iter, st, s, rpb, clu);
        return;
    }
    float* vecs = (float*)take(5 * v * 4);
    double* x64 = (double*)take(v * 8);
    double* r64 = (double*)take(v * 8);
    float* r32 = (float*)take(v * 4);
    float* d32 = (float*)take(v * 4);
    double* norms = (double*)take(2 * kMaxRhs * 8);
    VecPack<const float> yf{};
    VecPack<float> wf{};
    for (int k = 0; k < nr; ++k) {
        yf.p[k] = (const float*)y[k];
        wf.p[k] = (float*)w[k];
    }
    double* tau = (double*)take(kMaxRhs * 8);
    const unsigned nb = nblk(n, 256);
    const unsigned nbd = nb < 1024 ? nb : 1024;
    const double inner = rtol > 1e-7 ? rtol : 1e-7;
    cudaMemsetAsync(norms + kMaxRhs, 0, kMaxRhs * 8, s);
    { norm2_f32_kernel<<<nbd, 256, 0, s>>>(n, nr, yf, norms + kMaxRhs); count_launch(); }
    // one FP32 solve and one FP64 residual correction, fixed (no host decisions);
    // the correction solve stops at the tolerance that brings the residual to rtol
    for (int ref = 0; ref < 2; ++ref) {
        const float* rhs[kMaxRhs];
        float* dst[kMaxRhs];
        VecPack<const float> dp{};
        for (int k = 0; k < nr; ++k) {
            rhs[k] = ref == 0 ? yf.p[k] : r32 + k * n;
            dst[k] = d32 + k * n;
            dp.p[k] = dst[k];
        }
        run_pcg_fused<float>(M.ptr, M.col, M.val32, diag_inv32, n, nr, rhs, dst, vecs, partial, inner, max_iter, st, s,
                             rpb, clu, ref == 0 ? nullptr : tau);
        { add_correction_kernel<<<nb, 256, 0, s>>>(n, nr, x64, dp, ref == 0, norms + kMaxRhs); count_launch(); }
        if (ref == 0) {
            cudaMemsetAsync(norms, 0, kMaxRhs * 8, s);
            { residual_f64_kernel<<<nbd, 256, 0, s>>>(n, nr, M.ptr, M.col, M.val, yf, x64, r64, r32, norms, norms + kMaxRhs); count_launch(); }
            { inner_tol_kernel<<<1, 32, 0, s>>>(nr, rtol, norms, norms + kMaxRhs, tau); count_launch(); }
        }
    }
    { store_f32_kernel<<<nb, 256, 0, s>>>(n, nr, x64, wf); count_launch(); }
}

l2x_status solve_mass_pcg(int path, int precision, const Csr& M, const double* diag_inv, const float* diag_inv32,
                          int nr, const void* const* y, void* const* w, double rtol, int max_iter, void* ws,
                          DevStatus* st, DevStatus* st_host, cudaStream_t s, PcgResult* res, int rpb, int clu) {
    const int64_t n = M.n_rows;
    res->iters = 0;
    res->residual = 0.0;
    res->converged = true;
    if (n <= 0 || nr <= 0) return L2X_OK;
    const int64_t v = n * nr;
    char* base = (char*)ws;
    auto take = [&](size_t bytes) {
        void* p = base;
        base += (bytes + 255) & ~(size_t)255;
        return p;
    };
    cudaError_t ce;
    if (path == L2X_PATH_PLAIN) {
        double* r = (double*)take(v * 8);
        double* z = (double*)take(v * 8);
        double* p = (double*)take(v * 8);
        double* q = (double*)take(v * 8);
        double* scal = (double*)take(16 * 8);
        double* rr0 = (double*)take(4 * 8);
        double hs[16];
        const double* yy[3] = {(const double*)y[0], nr > 1 ? (const double*)y[1] : nullptr, nr > 2 ? (const double*)y[2] : nullptr};
        double* xx[3] = {(double*)w[0], nr > 1 ? (double*)w[1] : nullptr, nr > 2 ? (double*)w[2] : nullptr};
        unsigned nb = nblk(n, 256);
        unsigned nbd = nb < 1024 ? nb : 1024;
        { plain_init_kernel<<<nb, 256, 0, s>>>(n, nr, yy[0], yy[1], yy[2], xx[0], xx[1], xx[2], diag_inv, r, z, p); count_launch(); }
        cudaMemsetAsync(scal, 0, 16 * 8, s);
        cudaMemsetAsync(rr0, 0, 4 * 8, s);
        { plain_dot_kernel<<<nbd, 256, 0, s>>>(n, nr, r, z, scal); count_launch(); }      // rz
        { plain_dot_kernel<<<nbd, 256, 0, s>>>(n, nr, r, r, rr0); count_launch(); }       // |y|^2
        { plain_active_kernel<<<1, 32, 0, s>>>(nr, scal, rr0); count_launch(); }
        double rr0h[3] = {0, 0, 0};
        int it = 0;
        bool done = false;
        double worst = 0.0;
        for (; it < max_iter && !done; ++it) {
            { plain_spmv_kernel<<<nb, 256, 0, s>>>(n, nr, M.ptr, M.col, M.val, p, q); count_launch(); }
            { plain_dot_kernel<<<nbd, 256, 0, s>>>(n, nr, p, q, scal + 3); count_launch(); }
            { plain_update_x_kernel<<<nb, 256, 0, s>>>(n, nr, scal, xx[0], xx[1], xx[2], r, z, p, q, diag_inv); count_launch(); }
            { plain_dot_kernel<<<nbd, 256, 0, s>>>(n, nr, r, z, scal + 6); count_launch(); }
            { plain_dot_kernel<<<nbd, 256, 0, s>>>(n, nr, r, r, scal + 9); count_launch(); }
            { plain_update_p_kernel<<<nb, 256, 0, s>>>(n, nr, scal, z, p); count_launch(); }
            // host convergence check (read the residual norms every iteration)
            if ((ce = cudaMemcpyAsync(hs, scal, sizeof(double) * 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if (it == 0 && (ce = cudaMemcpyAsync(rr0h, rr0, sizeof(double) * nr, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) break;
            { plain_scalars_kernel<<<1, 32, 0, s>>>(nr, scal, rr0, rtol); count_launch(); }
            done = true;
            worst = 0.0;
            for (int k = 0; k < nr; ++k) {
                double rel = rr0h[k] > 0.0 ? sqrt(hs[9 + k] / rr0h[k]) : 0.0;
                worst = fmax(worst, rel);
                if (!(rel <= rtol)) done = false;
            }
        }
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return L2X_ECUDA;
        res->iters = it;
        res->residual = worst;
        res->converged = done;
        return done ? L2X_OK : L2X_ENOTCONVERGED;
    }
    double* partial = (double*)take((size_t)pcg_max_blocks() * 3 * kMaxRhs * 8);
    if (precision == L2X_FP64) {
        double* vecs = (double*)take(5 * v * 8);
        cudaMemsetAsync(&st->flags, 0, sizeof(int32_t), s);
        ce = run_pcg_fused<double>(M.ptr, M.col, M.val, diag_inv, n, nr, (const double* const*)y, (double* const*)w,
                                   vecs, partial, rtol, max_iter, st, s, rpb, clu);
        if (ce != cudaSuccess) return L2X_ECUDA;
        if (cudaMemcpyAsync(st_host, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) return L2X_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return L2X_ECUDA;
        res->iters = st_host->cg_iters;
        res->residual = st_host->cg_residual;
        res->converged = !(st_host->flags & FLAG_NOTCONVERGED);
        return res->converged ? L2X_OK : L2X_ENOTCONVERGED;
    }
    // mixed: FP32 PCG, then FP64 residual refinement (x accumulated in FP64,
    // residual y - M x in FP64) until rtol, at most 3 corrections
    float* vecs = (float*)take(5 * v * 4);
    double* x64 = (double*)take(v * 8);
    double* r64 = (double*)take(v * 8);
    float* r32 = (float*)take(v * 4);
    float* d32 = (float*)take(v * 4);
    double* norms = (double*)take(2 * kMaxRhs * 8);
    VecPack<const float> yf{};
    VecPack<float> wf{};
    for (int k = 0; k < nr; ++k) {
        yf.p[k] = (const float*)y[k];
        wf.p[k] = (float*)w[k];
    }
    unsigned nb = nblk(n, 256);
    unsigned nbd = nb < 1024 ? nb : 1024;
    const double inner = rtol > 1e-7 ? rtol : 1e-7;
    cudaMemsetAsync(norms, 0, 2 * kMaxRhs * 8, s);
    { norm2_f32_kernel<<<nbd, 256, 0, s>>>(n, nr, yf, norms + kMaxRhs); count_launch(); }
    int total_it = 0;
    double worst = 0.0;
    bool ok = false;
    double hn[2 * kMaxRhs];
    double* tau = (double*)take(kMaxRhs * 8);
    for (int ref = 0; ref < 4 && !ok; ++ref) {
        const float* rhs[kMaxRhs];
        float* dst[kMaxRhs];
        VecPack<const float> dp{};
        for (int k = 0; k < nr; ++k) {
            rhs[k] = ref == 0 ? yf.p[k] : r32 + k * n;
            dst[k] = d32 + k * n;
            dp.p[k] = dst[k];
        }
        cudaMemsetAsync(&st->flags, 0, sizeof(int32_t), s);
        if (ref > 0) { inner_tol_kernel<<<1, 32, 0, s>>>(nr, rtol, norms, norms + kMaxRhs, tau); count_launch(); }
        ce = run_pcg_fused<float>(M.ptr, M.col, M.val32, diag_inv32, n, nr, rhs, dst, vecs, partial, inner,
                                  max_iter, st, s, rpb, clu, ref == 0 ? nullptr : tau);
        if (ce != cudaSuccess) return L2X_ECUDA;
        { add_correction_kernel<<<nb, 256, 0, s>>>(n, nr, x64, dp, ref == 0, norms + kMaxRhs); count_launch(); }
        cudaMemsetAsync(norms, 0, kMaxRhs * 8, s);
        { residual_f64_kernel<<<nbd, 256, 0, s>>>(n, nr, M.ptr, M.col, M.val, yf, x64, r64, r32, norms, norms + kMaxRhs); count_launch(); }
        if (cudaMemcpyAsync(st_host, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) return L2X_ECUDA;
        if (cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s) != cudaSuccess) return L2X_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return L2X_ECUDA;
        total_it += st_host->cg_iters;
        worst = 0.0;
        for (int k = 0; k < nr; ++k)
            worst = fmax(worst, hn[kMaxRhs + k] > 0.0 ? sqrt(hn[k] / hn[kMaxRhs + k]) : 0.0);
        ok = worst <= rtol;
    }
    { store_f32_kernel<<<nb, 256, 0, s>>>(n, nr, x64, wf); count_launch(); }
    if (cudaGetLastError() != cudaSuccess) return L2X_ECUDA;
    res->iters = total_it;
    res->residual = worst;
    res->converged = ok;
    return ok ? L2X_OK : L2X_ENOTCONVERGED;
}

}  // namespace l2x
