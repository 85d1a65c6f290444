// Jacobi-preconditioned CG on a caller-supplied CSR matrix that allocates no
// memory: a variant of the cooperative mass-matrix solve whose work vectors live
// in one fixed device array of this file instead of memory obtained from
// cudaMalloc.  It exists for callers that cannot allocate device memory while
// they run it: a host process whose device memory is handed out by an outer
// framework or memory pool (so a private cudaMalloc would fail or fragment that
// pool), code that must not add allocation calls to a latency-critical loop, or
// a caller that already owns the matrix and the vectors and only wants the
// solve.  The caller passes the matrix, the right-hand sides and the outputs.
#include <cooperative_groups.h>

#include <string>

#include "l2x_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int64_t kMaxEntries = L2X_NOALLOC_MAX_ENTRIES;  // n * n_rhs and n
constexpr int kMaxRhs = 3;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;
// r, u, p, s, w (n * n_rhs each), inverse diagonal (n), partial sums, status
constexpr int64_t kScratchDoubles = 5 * kMaxEntries + kMaxEntries + (int64_t)kMaxBlocks * 3 * kMaxRhs + 16;

static_assert(kScratchDoubles == L2X_NOALLOC_MAX_DOUBLES, "scratch size differs from the header");

// Device-side scratch of every call.  Host code must not use this name as an
// address: its device address is looked up with cudaGetSymbolAddress below.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

struct Args {
    int64_t n;
    int nr;
    const int64_t* ptr;
    const int32_t* col;
    const double* val;
    const double* y[kMaxRhs];
    double* x[kMaxRhs];
    double* scratch;
    double rtol;
    int max_iter;
};

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
    return t;
}

// Chronopoulos-Gear PCG, all right-hand sides together; every value it reads
// from the scratch array is written earlier in the same call.
__global__ void __launch_bounds__(kThreads) pcg_noalloc_kernel(Args A) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double sh[32];
    __shared__ double tot[3 * kMaxRhs];
    const int nr = A.nr;
    const int64_t n = A.n, v = n * nr;
    double* r = A.scratch;
    double* u = r + v;
    double* p = u + v;
    double* s = p + v;
    double* w = s + v;
    double* dinv = w + v;
    double* partial = dinv + n;
    double* status = partial + (int64_t)kMaxBlocks * 3 * kMaxRhs;  // [0] iterations, [1] residual, [2] converged
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(n, (int64_t)blockIdx.x * per), r1 = min(n, r0 + per);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double d = 0.0;
        for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
            if (A.col[q] == (int32_t)i) d = A.val[q];
        const double di = d != 0.0 ? 1.0 / d : 0.0;
        dinv[i] = di;
        for (int k = 0; k < nr; ++k) {
            const double yi = A.y[k][i];
            A.x[k][i] = 0.0;
            r[k * n + i] = yi;
            u[k * n + i] = di * yi;
        }
    }
    grid.sync();
    double alpha[kMaxRhs], gamma_old[kMaxRhs], rho0[kMaxRhs], rho[kMaxRhs];
    bool conv[kMaxRhs];
    for (int k = 0; k < kMaxRhs; ++k) {
        alpha[k] = gamma_old[k] = rho0[k] = rho[k] = 0.0;
        conv[k] = true;
    }
    int it = 0;
    bool all_conv = false;
    for (;;) {
        double dg[kMaxRhs] = {0, 0, 0}, dd[kMaxRhs] = {0, 0, 0}, dr[kMaxRhs] = {0, 0, 0};
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            double acc[kMaxRhs] = {0, 0, 0};
            for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
                const double a = A.val[q];
                const int32_t j = A.col[q];
                for (int k = 0; k < nr; ++k) acc[k] = fma(a, u[k * n + j], acc[k]);
            }
            for (int k = 0; k < nr; ++k) {
                const double ri = r[k * n + i], ui = u[k * n + i];
                w[k * n + i] = acc[k];
                dg[k] = fma(ri, ui, dg[k]);
                dd[k] = fma(acc[k], ui, dd[k]);
                dr[k] = fma(ri, ri, dr[k]);
            }
        }
        for (int k = 0; k < nr; ++k) {
            const double a = block_sum(dg[k], sh), b = block_sum(dd[k], sh), c = block_sum(dr[k], sh);
            if (threadIdx.x == 0) {
                partial[(int64_t)blockIdx.x * 3 * kMaxRhs + 3 * k + 0] = a;
                partial[(int64_t)blockIdx.x * 3 * kMaxRhs + 3 * k + 1] = b;
                partial[(int64_t)blockIdx.x * 3 * kMaxRhs + 3 * k + 2] = c;
            }
        }
        grid.sync();
        for (int j = 0; j < 3 * nr; ++j) {
            double t = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += partial[(int64_t)b * 3 * kMaxRhs + j];
            t = block_sum(t, sh);
            if (threadIdx.x == 0) tot[j] = t;
        }
        __syncthreads();
        double beta[kMaxRhs] = {0, 0, 0};
        all_conv = true;
        for (int k = 0; k < nr; ++k) {
            const double gam = tot[3 * k], del = tot[3 * k + 1];
            rho[k] = tot[3 * k + 2];
            if (it == 0) rho0[k] = rho[k];
            conv[k] = rho[k] <= A.rtol * A.rtol * rho0[k];
            all_conv = all_conv && conv[k];
            if (!conv[k]) {
                if (it == 0) {
                    alpha[k] = gam / del;
                } else {
                    beta[k] = gam / gamma_old[k];
                    alpha[k] = gam / (del - beta[k] * gam / alpha[k]);
                }
                gamma_old[k] = gam;
            }
        }
        if (all_conv || it >= A.max_iter) break;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double di = dinv[i];
            for (int k = 0; k < nr; ++k) {
                if (conv[k]) continue;
                const int64_t o = k * n + i;
                const double pn = it == 0 ? u[o] : fma(beta[k], p[o], u[o]);
                const double sn = it == 0 ? w[o] : fma(beta[k], s[o], w[o]);
                p[o] = pn;
                s[o] = sn;
                A.x[k][i] = fma(alpha[k], pn, A.x[k][i]);
                const double rn = fma(-alpha[k], sn, r[o]);
                r[o] = rn;
                u[o] = di * rn;
            }
        }
        grid.sync();
        ++it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double worst = 0.0;
        for (int k = 0; k < nr; ++k) worst = fmax(worst, rho0[k] > 0.0 ? sqrt(rho[k] / rho0[k]) : 0.0);
        status[0] = (double)it;
        status[1] = worst;
        status[2] = all_conv ? 1.0 : 0.0;
    }
}

thread_local std::string g_err;

// Device address of g_scratch on the current device.  Looked up on every call:
// once the module is loaded on the device this is a table lookup, and it stays
// right after cudaDeviceReset or a new primary context (a cached pointer would
// then name the old context's memory).  Under lazy module loading the first
// lookup on a device loads the module and so creates the array.
l2x_status scratch_for_current_device(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        g_err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
        return L2X_ECUDA;
    }
    *out = (double*)p;
    return L2X_OK;
}

}  // namespace

extern "C" const char* l2x_noalloc_last_error(void) { return g_err.c_str(); }

extern "C" l2x_status l2x_solve_mass_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* cols,
                                             const double* vals, int32_t n_rhs, const double* const* y,
                                             double* const* w, double rtol, int32_t max_iter, void* stream,
                                             int32_t* iters, double* residual) {
    g_err.clear();
    if (n <= 0 || n_rhs < 1 || n_rhs > kMaxRhs || !row_ptr || !cols || !vals || !y || !w || !(rtol > 0.0) ||
        max_iter < 1) {
        g_err = "bad arguments: need n > 0, 1 <= n_rhs <= 3, non-NULL arrays, rtol > 0, max_iter >= 1";
        return L2X_EINVAL;
    }
    for (int k = 0; k < n_rhs; ++k)
        if (!y[k] || !w[k]) {
            g_err = "NULL right-hand side or output";
            return L2X_EINVAL;
        }
    if (n > kMaxEntries || n * n_rhs > kMaxEntries) {
        g_err = "n * n_rhs = " + std::to_string(n * n_rhs) + " exceeds the fixed scratch of " +
                std::to_string(kMaxEntries) + " entries (n <= " + std::to_string(kMaxEntries) + ")";
        return L2X_ECAPACITY;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the call reads the solver status back and synchronises the stream, which a
    // capturing stream does not allow
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &capturing);
    if (ce != cudaSuccess) {
        g_err = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce);
        return L2X_ECUDA;
    }
    if (capturing != cudaStreamCaptureStatusNone) {
        g_err = "the stream is capturing: this call synchronises it and cannot be captured";
        return L2X_EINVAL;
    }
    double* scratch = nullptr;
    l2x_status st = scratch_for_current_device(&scratch);
    if (st != L2X_OK) return st;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_noalloc_kernel, kThreads, 0);
    int64_t blocks = (n + 2 * kThreads - 1) / (2 * kThreads);
    int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > cap) blocks = cap;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    if (blocks < 1) blocks = 1;
    Args A{};
    A.n = n;
    A.nr = n_rhs;
    A.ptr = row_ptr;
    A.col = cols;
    A.val = vals;
    for (int k = 0; k < n_rhs; ++k) {
        A.y[k] = y[k];
        A.x[k] = w[k];
    }
    A.scratch = scratch;
    A.rtol = rtol;
    A.max_iter = max_iter;
    void* args[] = {&A};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_noalloc_kernel, dim3((unsigned)blocks),
                                                dim3(kThreads), args, 0, s);
    if (e == cudaSuccess) l2x::count_launch();
    if (e != cudaSuccess) {
        g_err = std::string("PCG launch: ") + cudaGetErrorString(e);
        return L2X_ECUDA;
    }
    // status words sit after r, u, p, s, w (n * n_rhs each), dinv (n) and the partial sums
    const int64_t status_off = 5 * n * n_rhs + n + (int64_t)kMaxBlocks * 3 * kMaxRhs;
    double hs[3] = {0, 0, 0};
    e = cudaMemcpyAsync(hs, scratch + status_off, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g_err = std::string("PCG status: ") + cudaGetErrorString(e);
        return L2X_ECUDA;
    }
    if (iters) *iters = (int32_t)hs[0];
    if (residual) *residual = hs[1];
    if (hs[2] != 1.0) {
        g_err = "CG reached relative residual " + std::to_string(hs[1]) + " after " + std::to_string((int)hs[0]) +
                " iterations";
        return L2X_ENOTCONVERGED;
    }
    return L2X_OK;
}
