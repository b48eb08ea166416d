// peak.cu -- FP64 and FP32 fused multiply-add throughput of the current GPU,
// measured with independent FMA chains on every SM.  The benchmark uses the
// result as the ALU roofline of the FP64 kernels (GB300 runs FP64 at a small
// fraction of its FP32 rate, so several kernels of the path are ALU-bound).
#include "internal.cuh"

namespace apc {
namespace {

template <class T>
__global__ void k_fma_chains(T *out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <class T>
double measure(int sms, int iters) {
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
    k_fma_chains<T><<<blocks, threads>>>(out, 64, (T)0.999, (T)0.001);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    return 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
}

}  // namespace
}  // namespace apc

extern "C" apcloud_status apcloud_measure_fma_peak(double *fp64_tflops, double *fp32_tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return APCLOUD_E_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) return APCLOUD_E_CUDA;
    double d = apc::measure<double>(sms, 1 << 13);
    double f = apc::measure<float>(sms, 1 << 15);
    if (d < 0 || f < 0) return APCLOUD_E_CUDA;
    if (fp64_tflops) *fp64_tflops = d;
    if (fp32_tflops) *fp32_tflops = f;
    return APCLOUD_OK;
}
