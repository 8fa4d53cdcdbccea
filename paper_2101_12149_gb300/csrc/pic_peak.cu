// Measured arithmetic peak of the device (FP32 or FP64 fused multiply-add
// throughput), the denominator of the ALU roofline the benchmark reports for
// the tile kernel.  Each thread runs eight independent FMA chains in
// registers (enough independent work per warp to keep the FMA pipes busy);
// the launch is timed with CUDA events.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "pic.h"

namespace pic {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 512;

template <typename T> __global__ void __launch_bounds__(kPeakBlock) k_fma_chains(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1)) out[blockIdx.x] = s;  // never true: keeps the chains alive
}

template <typename T> cudaError_t time_chains(int sms, int iters, float* ms) {
    const int grid = sms * 4;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<grid, kPeakBlock, 0, s>>>(nullptr, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0 && t < best) best = t;  // the first launch warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    *ms = best;
    return e;
}

}  // namespace

extern "C" pic_status pic_measure_fma_peak(int32_t precision, double* tflops) {
    if (!tflops || (precision != PIC_FP64 && precision != PIC_FP32_MIXED)) {
        pic::set_last_error("precision must be PIC_FP64 or PIC_FP32_MIXED and tflops non-NULL");
        return PIC_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        pic::set_last_error(std::string("device query: ") + cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    // iterations for roughly 20 ms at the nominal rates
    const int iters = precision == PIC_FP64 ? 2048 : 65536;
    float ms = 0.f;
    e = precision == PIC_FP64 ? time_chains<double>(sms, iters, &ms) : time_chains<float>(sms, iters, &ms);
    if (e != cudaSuccess) {
        pic::set_last_error(std::string("FMA peak kernel: ") + cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    const double flops = 2.0 * kChains * double(iters) * double(sms) * 4.0 * kPeakBlock;
    *tflops = flops / (double(ms) * 1e-3) / 1e12;
    return PIC_OK;
}
