// Measured ALU peaks for the rooflines of the CUDA-core kernels: FP32 and
// FP64 fused multiply-add throughput of the current device.  Every thread
// runs eight independent FMA chains; the grid fills every SM several times.
#include "common.cuh"

template <class R>
__global__ void k_fma_peak(R* out, int iters, R a, R b) {
    R x0 = (R)threadIdx.x, x1 = x0 + (R)1, x2 = x0 + (R)2, x3 = x0 + (R)3;
    R x4 = x0 + (R)4, x5 = x0 + (R)5, x6 = x0 + (R)6, x7 = x0 + (R)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    R s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (R)-12345.0) out[0] = s;   // keeps the chains alive
}

template <class R>
static fb_status measure(double* tflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    FB_CUDA(cudaGetDevice(&dev));
    FB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    R* out = nullptr;
    FB_CHECK(dalloc(&out, 1));
    const int threads = 256, blocks = sms * 8;
    const int iters = sizeof(R) == 8 ? 256 : 2048;
    cudaEvent_t e0, e1;
    FB_CUDA(cudaEventCreate(&e0));
    FB_CUDA(cudaEventCreate(&e1));
    k_fma_peak<R><<<blocks, threads, 0, s>>>(out, iters, (R)0.999999, (R)1e-7);   // warm-up
    cudaEventRecord(e0, s);
    k_fma_peak<R><<<blocks, threads, 0, s>>>(out, iters, (R)0.999999, (R)1e-7);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(out);
    if (err != cudaSuccess) return fb_fail(FB_ERR_CUDA, cudaGetErrorString(err));
    double flops = 2.0 * 8.0 * 16.0 * iters * (double)threads * blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return FB_OK;
}

fb_status fb_alu_peaks_impl(double* fp32, double* fp64, cudaStream_t s) {
    if (fp32) FB_CHECK(measure<float>(fp32, s));
    if (fp64) FB_CHECK(measure<double>(fp64, s));
    return FB_OK;
}
