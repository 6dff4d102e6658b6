// FMA throughput of this GPU in FP64 and FP32, measured with the library's own
// kernel: the roof against which the FP64-arithmetic kernels of the solver
// (FP64 BLAS-1, the FP64 stencil) are judged.  The paper has no counterpart.
//
// Every thread runs CHAINS independent dependency chains of x <- x * a + b
// (enough independent FMAs in flight to cover the pipeline latency), ITERS
// times; the grid fills every SM several times over.  Flops counted: 2 per FMA.
#include "internal.h"

namespace mgeig {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(int iters, R a, R b, R *out) {
    R x[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fma(x[k], a, b);
        }
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
    // a store the compiler cannot prove dead (the sum is never exactly -1 here)
    if (s == (R)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FLOP/s of the launch (best of `reps` timed launches after one warm-up)
template <typename R>
static double fma_peak(Ctx &c, int reps) {
    int sms = 0, per_sm = 0;
    MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<R>, PEAK_THREADS, 0));
    const int blocks = sms * std::max(per_sm, 1) * 4;
    const int iters = sizeof(R) == 8 ? 256 : 4096;
    TmpBuf out;
    out.alloc((size_t)blocks * PEAK_THREADS * sizeof(R));
    cudaEvent_t e0, e1;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    double best = 0;
    for (int r = 0; r <= reps; ++r) {
        MG_CUDA(cudaEventRecord(e0, c.stream));
        fma_peak_kernel<R><<<blocks, PEAK_THREADS, 0, c.stream>>>(iters, (R)0.999999, (R)1e-7, out.as<R>());
        MG_CHECK_LAUNCH();
        MG_CUDA(cudaEventRecord(e1, c.stream));
        MG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double flops = 2.0 * PEAK_CHAINS * 16.0 * iters * (double)blocks * PEAK_THREADS;
        if (r > 0) best = std::max(best, flops / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

double fma_peak_flops(Ctx &c, int prec, int reps) {
    return prec == MGEIG_PREC_F64 ? fma_peak<double>(c, reps) : fma_peak<float>(c, reps);
}

}  // namespace mgeig
