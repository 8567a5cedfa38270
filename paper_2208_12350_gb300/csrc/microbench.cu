// Integer issue-rate microbenchmark: the denominator of the alignment
// kernels' roofline.  Each thread runs 16 instructions of one kind per
// iteration step with 8-way instruction-level parallelism; the kernel
// reports instructions per second for the whole device.  The results are
// stored, so nothing is dropped.
#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

template <int OP>
__device__ __forceinline__ int step(int a, int b, int c) {
    if constexpr (OP == 0) return a + b;                          // IADD
    if constexpr (OP == 1) return max(a, b);                      // IMNMX
    if constexpr (OP == 2) return __viaddmax_s32(a, b, c);        // add + max
    if constexpr (OP == 3) return __vimax3_s32_relu(a, b, c);     // 3-way max with 0
    if constexpr (OP == 4) return (int)__viaddmax_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 5) return __vimax_s32_relu(a, b);         // 2-way max with 0
    if constexpr (OP == 6) return (int)__vimax3_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
    if constexpr (OP == 7) return (int)__viaddmax_s16x2_relu((unsigned)a, (unsigned)b, (unsigned)c);
    return a;
}

// Two banks of 8 values feed each other: every instruction reads three
// different values produced by the other bank, so no chain can be folded
// and every bank offers 8 independent instructions.
template <int OP>
__global__ void int_rate_kernel(int64_t iters, int b, int c, int *sink) {
    int x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (int)threadIdx.x * (k + 1) + b * k + c;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) y[k] = step<OP>(x[k], x[(k + 1) & 7], x[(k + 3) & 7]);
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = step<OP>(y[k], y[(k + 2) & 7], y[(k + 5) & 7]);
        }
    }
    int acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int OP>
cudaError_t run(int blocks, int threads, int64_t iters, int *sink, cudaStream_t s) {
    int_rate_kernel<OP><<<blocks, threads, 0, s>>>(iters, 3, -5, sink);
    return cudaGetLastError();
}

}  // namespace
}  // namespace swgb

extern "C" int sw_microbench_int(int32_t op, int32_t device, int64_t iters, double *ops_per_s,
                                 double *seconds) {
    using namespace swgb;
    if (!ops_per_s || op < 0 || op > 7 || iters < 1) return SW_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return SW_ECUDA;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    const int threads = 512;
    const int blocks = prop.multiProcessorCount * 4;  // 64 warps per SM
    int *sink = nullptr;
    cudaEvent_t e0, e1;
    int rc = SW_OK;
    if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(int)) != cudaSuccess) {
        cudaSetDevice(prev);
        return SW_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int64_t it) -> cudaError_t {
        switch (op) {
            case 0: return run<0>(blocks, threads, it, sink, 0);
            case 1: return run<1>(blocks, threads, it, sink, 0);
            case 2: return run<2>(blocks, threads, it, sink, 0);
            case 3: return run<3>(blocks, threads, it, sink, 0);
            case 4: return run<4>(blocks, threads, it, sink, 0);
            case 5: return run<5>(blocks, threads, it, sink, 0);
            case 6: return run<6>(blocks, threads, it, sink, 0);
            default: return run<7>(blocks, threads, it, sink, 0);
        }
    };
    float ms = 0.f;
    if (launch(1) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        rc = SW_ECUDA;
    } else {
        cudaEventRecord(e0, 0);
        launch(iters);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = SW_ECUDA;
        cudaEventElapsedTime(&ms, e0, e1);
    }
    const double ops = (double)blocks * threads * (double)iters * 16.0 * 8.0;
    *ops_per_s = ms > 0 ? ops / (ms * 1e-3) : 0.0;
    if (seconds) *seconds = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaSetDevice(prev);
    return rc;
}
