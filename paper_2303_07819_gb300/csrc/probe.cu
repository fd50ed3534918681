// probe.cu -- FP32 FMA throughput of this GPU, the denominator of the
// particle path's FP32-pipe roofline (the cell step's arithmetic is FP32).
// Every thread runs 8 independent chains of dependent FMAs, so each SM
// sub-partition always has independent FMAs to issue; the grid holds 8
// blocks of 256 threads per SM (all SMs full) for several milliseconds.
#include "common.cuh"

namespace msd {

namespace {

constexpr int PROBE_T = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_T) k_fma_probe(float *sink, int iters, float b, float cc)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) a[k] = 1.0e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; k++) a[k] = fmaf(a[k], b, cc);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; k++) s += a[k];
    if (s == -1.0f) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace

// Times `reps` launches after one warm-up on a stream of its own; returns
// the FP32 rate in TFLOP/s (an FMA counts as 2 flops).
cudaError_t fma_probe(int reps, double *tflops)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = nsm * 8, iters = 1 << 14;
    float *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float) * blocks)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        k_fma_probe<<<blocks, PROBE_T, 0, st>>>(sink, iters, 0.9999999f, 1.0e-7f);
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; r++) k_fma_probe<<<blocks, PROBE_T, 0, st>>>(sink, iters, 0.9999999f, 1.0e-7f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) {
            const double flops = 2.0 * PROBE_CHAINS * (double)iters * PROBE_T * blocks * reps;
            *tflops = flops / (ms * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return e;
}

}  // namespace msd
