// Arithmetic throughput of the current GPU, for the roofline of the kernels
// that are bound by an ALU pipe rather than by memory: the FP64 residual hops
// (FP64 FMA pipe), the persistent block solver (FP32 FMA pipe) and the dense
// LU check path (FP64 FMA or FP64 tensor-core mma.sync).  The paper has no
// counterpart.
//
// Every thread runs eight independent FMA (or mma) chains for a fixed count;
// the grid is 8 thread blocks of 256 threads per SM; each launch is timed
// with CUDA events after one warm-up launch, the best of three repeats kept.
#include <cuda_runtime.h>

#include <algorithm>

#include "dd_internal.h"

namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* out, int iters, T a, T b) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// four independent chains of the warp-wide m8n8k4 FP64 mma (512 flops each)
__global__ void __launch_bounds__(256) dmma_chains_kernel(double* out, int iters) {
    double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 0.0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class F>
float best_ms(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F launch) {
    launch();
    float best = -1.f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.f || ms < best) best = ms;
    }
    return best;
}

}  // namespace

extern "C" int dd_alu_peaks(double* tflops, void* stream) {
    if (!tflops) return DD_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DD_ERR_CUDA;
    const int tpb = 256, nblk = std::max(1, sms) * 8;
    const double threads = (double)nblk * tpb;
    cudaStream_t s = (cudaStream_t)stream;
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * nblk * tpb) != cudaSuccess) return DD_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int it64 = 4096, it32 = 65536, itmma = 2048;
    float ms64 = best_ms(s, e0, e1, [&] { fma_chains_kernel<double><<<nblk, tpb, 0, s>>>(buf, it64, 0.999999, 1e-7); });
    float ms32 = best_ms(s, e0, e1, [&] {
        fma_chains_kernel<float><<<nblk, tpb, 0, s>>>((float*)buf, it32, 0.999999f, 1e-7f);
    });
    float msmma = best_ms(s, e0, e1, [&] { dmma_chains_kernel<<<nblk, tpb, 0, s>>>(buf, itmma); });
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess || ms64 <= 0.f || ms32 <= 0.f || msmma <= 0.f) return DD_ERR_CUDA;
    tflops[0] = 2.0 * kChains * it64 * threads / (ms64 * 1e-3) / 1e12;
    tflops[1] = 2.0 * kChains * it32 * threads / (ms32 * 1e-3) / 1e12;
    tflops[2] = 512.0 * 4 * itmma * (threads / 32) / (msmma * 1e-3) / 1e12;
    return DD_OK;
}
