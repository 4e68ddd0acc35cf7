// peak.cu -- the device's FP64 FMA rate, measured.
//
// The FP64 form of the path is bound by the FP64 pipe (GB300 has a small one),
// so its roofline needs that pipe's rate on the device it runs on.  This
// measures it with a kernel of independent FMA chains: eight chains per
// thread, enough resident warps to keep every SM's FP64 units busy, timed
// with CUDA events after a warm-up launch.
#include "mcpt.h"
#include "internal.h"

#include <cstdio>

namespace mcpt {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma(double* sink, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = s;   // never true (x stays near b / (1 - a)); keeps the chains live
}

}  // namespace
}  // namespace mcpt

using namespace mcpt;

extern "C" mcpt_status mcpt_fp64_fma_rate(int device, double* tflops, double* ms_per_launch)
{
    if (!tflops) {
        set_thread_error("mcpt_fp64_fma_rate: tflops is NULL");
        return MCPT_EINVAL;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    int nsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = nsm * 8, iters = 1 << 13, reps = 5;
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_dfma<<<blocks, kThreads, 0, s>>>(nullptr, iters, 0.999, 1e-3);   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++) k_dfma<<<blocks, kThreads, 0, s>>>(nullptr, iters, 0.999, 1e-3);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        char buf[160];
        snprintf(buf, sizeof buf, "mcpt_fp64_fma_rate: CUDA error %s", cudaGetErrorString(e));
        set_thread_error(buf);
        return MCPT_ECUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_per_launch) *ms_per_launch = ms / reps;
    set_thread_error("");
    return MCPT_OK;
}
