// Measurement and test services, not part of the transfer (no counterpart in the
// paper): the throughput probe of the FP64 and FP32 fused multiply-add pipes (the
// measured denominator of the ALU roofline of the clipping kernel, whose geometry
// is FP64 and whose moment arithmetic is FP32 in the mixed form), and a test hook
// that runs the clipping kernel's arithmetic helpers elementwise.
#include <cuda_runtime.h>

#include "l2x_fp.cuh"
#include "l2x_internal.cuh"
#include "l2xfer.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent FMA chains per thread (hides the pipe latency)

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int32_t iters, T* __restrict__ sink) {
    T a[kProbeChains];
    const T m = T(0.9999999), b = T(1e-7) * T(threadIdx.x + 1);
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = T(c + 1) * T(1e-3) + T(blockIdx.x & 7);
#pragma unroll 4
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], m, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    sink[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;  // keeps the chains live
}

// out[i] = op(a[i], b[i]) for the device helpers of the clipping kernel and the
// CUDA operations they stand in for.
__global__ void fp_selftest_kernel(int32_t op, int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i], y = b[i];
    double r = 0.0;
    switch (op) {
        case 0: r = l2x::div_nr(x, y); break;
        case 1: r = x / y; break;
        case 2: r = (double)l2x::d2f_int(x); break;
        case 3: r = (double)__double2float_rn(x); break;
        case 4: r = (double)l2x::d2f_lo_int(x); break;
        case 5: r = l2x::f2d_int(__double2float_rn(x)); break;
        case 6: r = l2x::div_fast(x, y); break;
        default: break;
    }
    out[i] = r;
}

}  // namespace

extern "C" l2x_status l2x_fp_selftest(int32_t op, int64_t n, const double* a, const double* b, double* out,
                                      void* stream) {
    if (op < 0 || op > 6 || n < 0 || !a || !b || !out) return L2X_EINVAL;
    if (n == 0) return L2X_OK;
    fp_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(op, n, a, b, out);
    l2x::count_launch();
    return cudaGetLastError() == cudaSuccess ? L2X_OK : L2X_ECUDA;
}

extern "C" l2x_status l2x_fma_probe(int32_t precision, int32_t n_blocks, int32_t iters, void* sink, void* stream) {
    if (!sink || n_blocks <= 0 || iters <= 0 || (precision != L2X_FP64 && precision != L2X_MIXED))
        return L2X_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == L2X_FP64)
        fma_probe_kernel<double><<<n_blocks, kProbeThreads, 0, s>>>(iters, (double*)sink);
    else
        fma_probe_kernel<float><<<n_blocks, kProbeThreads, 0, s>>>(iters, (float*)sink);
    l2x::count_launch();
    return cudaGetLastError() == cudaSuccess ? L2X_OK : L2X_ECUDA;
}

extern "C" l2x_status l2x_scan_selftest(int64_t n, const int64_t* in, int64_t* out, int32_t missing_first,
                                       int64_t spin_limit, void* stream) {
    if (n <= 0 || !in || !out || spin_limit <= 0) return L2X_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ws_bytes = l2x::scan_tmp_bytes(n);
    void* ws = nullptr;
    l2x::DevStatus* st = nullptr;
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess) return L2X_ENOMEM;
    if (cudaMalloc((void**)&st, sizeof(l2x::DevStatus)) != cudaSuccess) {
        cudaFree(ws);
        return L2X_ENOMEM;
    }
    l2x::DevStatus h{};
    l2x_status r = L2X_OK;
    if (cudaMemsetAsync(ws, 0, ws_bytes, s) != cudaSuccess || cudaMemsetAsync(st, 0, sizeof(l2x::DevStatus), s) != cudaSuccess)
        r = L2X_ECUDA;
    if (r == L2X_OK) {
        l2x::launch_scan_i64_test(in, out, n, ws, s, st, missing_first, (long long)spin_limit);
        unsigned long long left[2] = {1, 1};
        if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(left, ws, sizeof(left), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            r = L2X_ECUDA;
        else if (h.flags & l2x::FLAG_TIMEOUT)
            r = L2X_ETIMEOUT;
        else if (left[0] != 0 || left[1] != 0)  // the workspace must be left zeroed
            r = L2X_ECUDA;
    }
    cudaFree(st);
    cudaFree(ws);
    return r;
}
