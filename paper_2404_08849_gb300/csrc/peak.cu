// peak.cu - FP64 fused-multiply-add throughput kernel: the denominator of
// the FP64-pipe roofline of the double-precision dycore kernels (the paper
// keeps the pressure gradient, gravity, the equation of state and the
// column solve in double, Sec. 2.3, and on this GPU those kernels are bound
// by the FP64 pipe rather than by memory).
//
// Every thread runs kChains independent FMA chains x <- x * b + c for `iters`
// rounds (no chain waits on another, so the pipe is never starved by
// dependences), then stores the sum of its chains so that nothing is
// optimised away.  With |b| < 1 the chains converge to c / (1 - b) and stay
// finite.  FP64 flop per launch = 2 * kChains * iters * blocks * threads.
#include "common.cuh"

namespace grist {
namespace {

constexpr int kChains = 8;   // GRIST_BENCH_FP64_CHAINS in grist.h
static_assert(kChains == GRIST_BENCH_FP64_CHAINS, "header and kernel agree");

__global__ void k_fp64_fma_peak(long long iters, double b, double c, double *__restrict__ out) {
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) x[j] = (double)(threadIdx.x + j);
    for (long long r = 0; r < iters; r++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) x[j] = fma(x[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; j++) s += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace grist

extern "C" int grist_bench_fp64_fma(int64_t iters, int32_t blocks, int32_t threads, double *out, void *stream) {
    if (!out || iters < 1 || iters > ((int64_t)1 << 40) || blocks < 1 || blocks > (1 << 20) || threads < 32 ||
        threads > 1024 || threads % 32)
        return GRIST_EINVAL;
    grist::k_fp64_fma_peak<<<blocks, threads, 0, (cudaStream_t)stream>>>((long long)iters, 0.999999, 1.0e-3, out);
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}
