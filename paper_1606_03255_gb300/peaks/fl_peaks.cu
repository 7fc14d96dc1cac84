// fl_peaks.cu -- measurement only (libflpeaks.so, used by bench.py): the
// issue rate of dependent-free FMA streams in FP32 and FP64 on this GPU, the
// denominators of the pipe fractions the benchmark reports for the kernels
// bound by arithmetic rather than by HBM (the direct sums, the float-pair
// passes, the Laplace kernels).  Not part of the transform's C ABI.
//
// Each thread runs kChains independent multiply-add chains for `iters`
// rounds; the chains' results are folded into one store so that nothing is
// eliminated.  The launch is a multiple of the SM count, so every SM issues.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_stream(int iters, T a, T b, T* __restrict__ out) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true for these inputs
}

template <typename T>
int measure(int blocks_per_sm, int iters, int reps, double* flops_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * blocks_per_sm;
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_stream<T><<<blocks, kThreads>>>(iters / 8 + 1, a, b, out);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        k_fma_stream<T><<<blocks, kThreads>>>(iters, a, b, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return 2;
    const double fmas = (double)blocks * kThreads * iters * 16.0 * kChains;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return 0;
}

}  // namespace

extern "C" {

// Best-of-reps FLOP/s (2 per FMA) of the FP32 (precision 0) or FP64 (1) FMA
// stream on the current device; returns 0 on success.
int fl_peak_fma(int precision, int blocks_per_sm, int iters, int reps, double* flops_per_s) {
    if (!flops_per_s || blocks_per_sm < 1 || iters < 1 || reps < 1) return 3;
    return precision == 0 ? measure<float>(blocks_per_sm, iters, reps, flops_per_s)
                          : measure<double>(blocks_per_sm, iters, reps, flops_per_s);
}

}  // extern "C"
