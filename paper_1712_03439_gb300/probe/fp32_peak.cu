// FP32 FMA throughput probe: the non-tensor peak used as the roofline
// denominator of the FFT kernels.  Every thread runs kChains independent FMA
// chains (enough in flight to cover the FMA latency with the resident warps);
// the result is written so nothing is optimised away.  Not part of the
// filter-and-mix library.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_ffma(float* __restrict__ out, float a, float b, int iters) {
    float c[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) c[k] = fmaf(c[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += c[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// Runs the probe on `device` and returns the sustained FP32 rate in TFLOP/s
// (2 flops per FMA) over `reps` launches of about `iters` x 128 FMAs per
// thread, and the kernel time in ms.  0 on success, else the CUDA error code.
int fp32_peak_probe(int device, int iters, int reps, double* tflops, double* ms) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return (int)e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma, 256, 0);
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    float* out = nullptr;
    e = cudaMalloc(&out, sizeof(float) * (size_t)grid * 256);
    if (e != cudaSuccess) return (int)e;
    k_ffma<<<grid, 256>>>(out, 0.9999999f, 1e-7f, 16);     // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) k_ffma<<<grid, 256>>>(out, 0.9999999f, 1e-7f, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double fmas = (double)grid * 256 * (double)iters * kUnroll * kChains * reps;
    *ms = t;
    *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    return 0;
}

}  // extern "C"
