// probe.cu -- measured FMA throughput of the current GPU (FP64 and FP32), the
// denominator of the ALU roofline of the FP64 step. Eight independent FMA
// chains per thread, 8 blocks of 256 threads per SM, best of 5 timed launches.
#include <algorithm>

#include "internal.cuh"

namespace mfd {

template <typename T> __global__ void k_fma_chains(T* out, int iters, T a, T b) {
    T x0 = threadIdx.x * T(1e-3), x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T> static mfd_status fma_rate(int sms, int iters, double* gflops) {
    const int blocks = sms * 8, threads = 256;
    DevBuf out;
    MFD_TRY(out.alloc(sizeof(T) * blocks * threads));
    cudaEvent_t e0, e1;
    MFD_CUDA(cudaEventCreate(&e0));
    MFD_CUDA(cudaEventCreate(&e1));
    k_fma_chains<T><<<blocks, threads>>>(out.as<T>(), 16, T(0.999), T(1e-3));
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, threads>>>(out.as<T>(), iters, T(0.999), T(1e-3));
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MFD_CUDA(cudaGetLastError());
    *gflops = 2.0 * 8 * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
    return MFD_OK;
}

}  // namespace mfd

extern "C" mfd_status mfd_fma_peak(int device, double* fp64_gflops, double* fp32_gflops) {
    using namespace mfd;
    if (!fp64_gflops || !fp32_gflops) return fail(MFD_ERR_ARG, "NULL argument");
    MFD_CUDA(cudaSetDevice(device));
    int sms = 0;
    MFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    MFD_TRY(fma_rate<double>(sms, 1 << 13, fp64_gflops));
    MFD_TRY(fma_rate<float>(sms, 1 << 16, fp32_gflops));
    return MFD_OK;
}
