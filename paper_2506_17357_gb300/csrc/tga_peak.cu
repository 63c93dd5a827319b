// Measured 32-bit integer throughput of the GPU: the denominator of the
// evaluation kernels' roofline fractions (the paper has no counterpart; it
// reports speedups only).
//
// Every thread runs kChains independent chains of integer operations, so
// nothing waits on a result for long and the schedulers issue back to back.
// Two streams:
//   kind 0  x = max(x + a, b): one add and one max per link, two-input
//           operations that no instruction fuses, i.e. one lane-operation
//           per issued lane (the form of the delta expressions' min/max
//           terms);
//   kind 1  x = x + x' + a: two adds per link that the compiler may fuse
//           into one three-input add, so the count of source operations
//           can exceed the issue rate.
// The operands are runtime values derived from the thread index and a seed,
// and the chains feed one result that is stored only when it matches an
// impossible value, so no operation can be folded away or skipped.
#include <cuda_runtime.h>

#include "tga.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 8;
constexpr int kThreads = 256;

__device__ int g_sink[256];   // never written: the stored value cannot occur

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_int_stream(int iters, int seed, int *sink) {
    int x[kChains], a[kChains];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = (t * (2 * c + 3)) ^ seed;
        a[c] = seed + c * 7919 - t;
    }
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if (KIND == 0) x[c] = max(x[c] + a[c], a[(c + 1) % kChains]);
                else x[c] = x[c] + x[(c + 3) % kChains] + a[c];
            }
        }
    }
    int acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c];
    if (acc == 0x7ffffffe && seed == 0x13572468) sink[t & 255] = acc;
}

}  // namespace

extern "C" int tga_measure_int_peak(int32_t kind, tga_stream_t stream, int32_t iters, double *ops_per_s,
                                    float *ms_out) {
    if ((kind != 0 && kind != 1) || iters < 1 || !ops_per_s) return TGA_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    const void *fn = kind == 0 ? (const void *)k_int_stream<0> : (const void *)k_int_stream<1>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    const int blocks = nsm * per;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    int *sink = nullptr;
    if (cudaGetSymbolAddress((void **)&sink, g_sink) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        return TGA_ERR_CUDA;
    }
    auto launch = [&](int it) {
        if (kind == 0) k_int_stream<0><<<blocks, kThreads, 0, s>>>(it, 0x2468ace1, sink);
        else k_int_stream<1><<<blocks, kThreads, 0, s>>>(it, 0x2468ace1, sink);
    };
    launch(iters < 16 ? iters : 16);                         // warm-up: clocks up, code loaded
    float best = 1e30f;
    for (int k = 0; k < 3; ++k) {
        cudaEventRecord(e0, s);
        launch(iters);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || best >= 1e29f) return TGA_ERR_CUDA;
    // two source operations per link in both streams
    const double ops = 2.0 * kChains * kUnroll * (double)iters * (double)blocks * kThreads;
    *ops_per_s = ops / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return TGA_OK;
}
