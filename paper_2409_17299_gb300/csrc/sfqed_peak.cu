// Measured FP64 arithmetic peak of the device: the denominator of the FP64
// mode's roofline (its pass kernels run every step of Algorithm 1 in FP64,
// and GB300's FP64 pipe is far narrower than its FP32 one).
//
// Each thread runs CHAINS independent fused multiply-add chains, so the pipe
// always has independent work; one wave of resident blocks covers every SM.
// Two FLOPs per FMA.  The chains are folded into the output so the compiler
// keeps all of them.
#include <chrono>

#include "sfqed_internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int PEAK_THREADS = 256;

__device__ double g_fma64_sink;   // receives the folded chains (keeps them live)

__global__ void __launch_bounds__(PEAK_THREADS) k_fma64(int iters, double a, double b) {
    double acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    if (s == 12345.678) g_fma64_sink = s;    // a data-dependent store the compiler cannot remove
}

}  // namespace

extern "C" qed_status qed_measure_fp64_peak(int iters, double *flops_per_s, double *ms, void *cuda_stream) {
    if (!flops_per_s || iters <= 0) return QED_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    SFQ_CUDA(cudaGetDevice(&dev));
    SFQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SFQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma64, PEAK_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    cudaEvent_t e0, e1;
    SFQ_CUDA(cudaEventCreate(&e0));
    SFQ_CUDA(cudaEventCreate(&e1));
    // a = 1 - 2^-40 keeps every chain bounded and away from denormals
    const double a = 1.0 - 0x1p-40, b = 0x1p-30;
    k_fma64<<<blocks, PEAK_THREADS, 0, st>>>(iters / 8 > 0 ? iters / 8 : 1, a, b);   // warm-up
    SFQ_CUDA(cudaGetLastError());
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        SFQ_CUDA(cudaEventRecord(e0, st));
        k_fma64<<<blocks, PEAK_THREADS, 0, st>>>(iters, a, b);
        SFQ_CUDA(cudaEventRecord(e1, st));
        SFQ_CUDA(cudaEventSynchronize(e1));
        float m = 0.f;
        SFQ_CUDA(cudaEventElapsedTime(&m, e0, e1));
        if (rep == 0 || m < best) best = m;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
    *flops_per_s = flops / (best * 1e-3);
    if (ms) *ms = best;
    return QED_OK;
}
