// probe.cu -- FP64 fused multiply-add throughput probe.
//
// The swept kernels are bound by FP64 issue, so the denominator of their
// roofline is the GPU's FP64 rate.  This kernel measures it: every thread
// runs kChains independent chains x <- fma(x, a, b), enough independent work
// per sub-partition to keep its FP64 pipe busy whatever the latency of one
// fma.  With a = 1 - 2^-30 and b = 2^-31 every chain converges to 1/2: no
// overflow, no subnormal.  Each fma counts as 2 flops.
#include <cuda_runtime.h>

#include <cstdint>

#include "sweep.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024) k_fp64_probe(double *out, int64_t iters, double a, double b)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = 0.25 + 1e-3 * (double)(c + (int)(t & 255));
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    out[t] = s;  // keeps every chain live
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int sweep_fp64_probe(double *d_out, int64_t iters,
                                                                        int blocks, int threads,
                                                                        CUstream_st *stream)
{
    if (!d_out || iters < 1 || blocks < 1 || threads < 32 || threads > 1024 || (threads % 32) != 0)
        return SWEEP_EINVAL;
    k_fp64_probe<<<blocks, threads, 0, stream>>>(d_out, iters, 1.0 - 0x1p-30, 0x1p-31);
    return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}
