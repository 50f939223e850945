// FP64 fused multiply-add rate of the device (mg_fp64_fma_rate in include/mg.h).
//
// The FP64 kernels of the solver (the outer residual of the mixed modes, the plain FP64
// V-cycle, the adjoint gradient) run on GB300's FP64 pipe, whose rate is a small fraction of
// the FP32 rate.  Their roofline needs that rate as measured on the device, not a nominal
// figure: this kernel issues nothing but dependent chains of FP64 FMAs, enough independent
// chains per thread and enough warps per SM to cover the pipe's latency, and the host times it
// with CUDA events.
#include "mg_internal.cuh"

namespace mg {
namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kThreadsPeak = 256;

// a <- a * m + c on kChains chains, `iters` times.  m and c come from the kernel arguments and
// differ slightly per thread, so they sit in registers: an FMA that reads an operand straight
// from the constant bank issues at a lower rate on GB300 (measured: 1.06 against 1.20 TFLOP/s),
// and the solver's FP64 kernels take their operands from registers.  |m| < 1 keeps the values
// bounded.  The block's sum (every thread's chains through a shuffle and shared-memory
// reduction, so no thread's work is dead) goes to sink[blockIdx.x].
__global__ void __launch_bounds__(kThreadsPeak) k_fp64_fma_chain(int iters, double m0, double c0,
                                                                double *__restrict__ sink) {
    const double m = m0 + 1e-13 * (threadIdx.x & 7), c = c0 + 1e-15 * (threadIdx.x & 3);
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k) + 1e-6 * blockIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ double part[kThreadsPeak / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreadsPeak / 32; ++w) t += part[w];
        sink[blockIdx.x] = t;
    }
}

}  // namespace
}  // namespace mg

extern "C" int mg_fp64_fma_rate(void *stream, double *sink, int blocks, int iters, double *tflops,
                                double *ms) {
    if (!sink || blocks < 1 || iters < 1 || !tflops) return MG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    // one untimed launch (clocks up, code loaded), then the timed one
    mg::count_launch(2);
    mg::k_fp64_fma_chain<<<blocks, mg::kThreadsPeak, 0, s>>>(iters < 64 ? iters : 64, 0.999999, 1e-7, sink);
    cudaEventRecord(e0, s);
    mg::k_fp64_fma_chain<<<blocks, mg::kThreadsPeak, 0, s>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1, s);
    float t = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
                    cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || !(t > 0.f)) {
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    const double fmas = (double)blocks * mg::kThreadsPeak * mg::kChains * (double)iters;
    *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return MG_OK;
}
