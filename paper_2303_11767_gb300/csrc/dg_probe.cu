// dg_probe.cu -- measured FP64 arithmetic peak of the current GPU: the roof
// of the FP64 stage kernel, which on GB300 is bound by its double-precision
// FMA rate rather than by HBM.  Every thread runs 8 independent FMA chains
// (enough to cover the pipeline latency) over a fixed iteration count; the
// result is written out so the work cannot be elided.
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) fma_probe_kernel(double *out, int iters, double a, double b)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// FP64 FMA rate in GFLOP/s (2 flops per FMA), best of `reps` timed launches.
int dg_probe_fp64_gflops(int reps, double *gflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    const int threads = 256, blocks = sms * 8, iters = 1 << 14;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = 1;
    float best_ms = 0.0f;
    if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return 1;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    fma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);   // warm-up
    for (int r = 0; r < (reps > 0 ? reps : 1); ++r) {
        cudaEventRecord(e0, s);
        fma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best_ms) best_ms = ms;
    }
    if (cudaPeekAtLastError() != cudaSuccess || !(best_ms > 0.0f)) goto done;
    *gflops = 2.0 * CHAINS * (double)iters * threads * blocks / (best_ms * 1e-3) / 1e9;
    rc = 0;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return rc;
}
