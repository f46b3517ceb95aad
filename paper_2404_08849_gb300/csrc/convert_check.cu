// convert_check.cu - self-tests of the arithmetic helpers in common.cuh:
// the integer binary32 <-> binary64 conversions (f2d, d2f) against the
// hardware conversions, the Newton-Raphson reciprocal (rcp_nr) against the
// IEEE quotient 1.0 / x, and the double-float splits (split_df,
// split_trunc) against their error bound.
// Each kernel compares both results in-register and counts disagreements,
// so the 2^32-pattern sweeps need no input or output buffers.
#include "common.cuh"

namespace grist {
namespace {

__device__ __forceinline__ bool same_d(double a, double b) {
    return (isnan(a) && isnan(b)) || __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_f(float a, float b) {
    return (isnan(a) && isnan(b)) || __float_as_uint(a) == __float_as_uint(b);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// out[0] checked, out[1] mismatches (binary32 -> binary64)
__global__ void k_check_f2d(unsigned long long *out) {
    unsigned long long bad = 0, n_ok = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long n = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; n < (1ull << 32);
         n += stride) {
        const float f = __uint_as_float((uint32_t)n);
        bad += !same_d(f2d(f), (double)f);
        n_ok++;
    }
    atomicAdd(out + 0, n_ok);
    atomicAdd(out + 1, bad);
}

__device__ __forceinline__ void check_d2f(double x, unsigned long long &bad, unsigned long long &n) {
    bad += !same_f(d2f(x), (float)x);
    n++;
}

// out[2] checked, out[3] mismatches (binary64 -> binary32)
__global__ void k_check_d2f(unsigned long long n_random, unsigned long long seed, unsigned long long *out) {
    unsigned long long bad = 0, cnt = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long n = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; n < (1ull << 32);
         n += stride) {
        const float f = __uint_as_float((uint32_t)n);
        if (isnan(f)) {
            check_d2f((double)f, bad, cnt);
            continue;
        }
        const double x = (double)f;
        check_d2f(x, bad, cnt);
        const float g = nextafterf(f, signbit(f) ? -INFINITY : INFINITY);
        // midpoint to the next binary32 away from zero (past the largest
        // finite value: the overflow threshold 2^128 - 2^103)
        const double mid = isinf(g) ? copysign(0x1.ffffffp127, x) : 0.5 * (x + (double)g);
        if (!isinf(f)) {
            check_d2f(mid, bad, cnt);
            check_d2f(nextafter(mid, 0.0), bad, cnt);
            check_d2f(nextafter(mid, copysign(INFINITY, x)), bad, cnt);
        }
    }
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_random;
         i += stride) {
        unsigned long long b = splitmix64(seed + i);
        if (i & 1ull) {
            // exponent in [860, 1160]: the binary32 range and its edges
            const unsigned long long ex = 860ull + (splitmix64(b) % 301ull);
            b = (b & 0x800fffffffffffffull) | (ex << 52);
        }
        check_d2f(__longlong_as_double((long long)b), bad, cnt);
    }
    atomicAdd(out + 2, cnt);
    atomicAdd(out + 3, bad);
}

// out[0] checked, out[1] results more than one ulp from 1.0 / x, out[2]
// the largest distance in ulps (as a count of binary64 steps)
__global__ void k_check_rcp(unsigned long long n, unsigned long long seed, unsigned long long *out) {
    unsigned long long cnt = 0, bad = 0, worst = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned long long b = splitmix64(seed + i);
        // exponent in [3, 2043] (|x| in [2^-1020, 2^1021)), any sign and fraction
        const unsigned long long ex = 3ull + (splitmix64(b ^ 0x5bd1e995ull) % 2041ull);
        b = (b & 0x800fffffffffffffull) | (ex << 52);
        const double x = __longlong_as_double((long long)b);
        const long long a = __double_as_longlong(rcp_nr(x)), r = __double_as_longlong(1.0 / x);
        const unsigned long long d = (unsigned long long)(a > r ? a - r : r - a);
        bad += d > 1ull;
        worst = d > worst ? d : worst;
        cnt++;
    }
    atomicAdd(out + 0, cnt);
    atomicAdd(out + 1, bad);
    atomicMax(out + 2, worst);
}

// out[0] checked, out[1] values whose split_df has h != RN32(x) or whose
// split_trunc has h != RZ32(x) (the hardware conversion toward zero), or
// where either gives |x - (h + l)| above 2^-47 |x| (the bound is exact
// arithmetic: h and l are floats, so x - h - l is formed in binary64
// without error for these magnitudes)
__global__ void k_check_split(unsigned long long n, unsigned long long seed, unsigned long long *out) {
    unsigned long long cnt = 0, bad = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned long long b = splitmix64(seed + i);
        // exponent in [949, 1149]: |x| in [2^-74, 2^127)
        const unsigned long long ex = 949ull + (splitmix64(b ^ 0x2545f491ull) % 201ull);
        b = (b & 0x800fffffffffffffull) | (ex << 52);
        const double x = __longlong_as_double((long long)b);
        float h, l;
        split_df(x, h, l);
        const double err = fabs((x - (double)h) - (double)l);
        float th, tl;
        split_trunc(x, th, tl);
        const double terr = fabs((x - (double)th) - (double)tl);
        bad += (__float_as_uint(h) != __float_as_uint((float)x)) || !(err <= ldexp(fabs(x), -47)) ||
               (__float_as_uint(th) != __float_as_uint(__double2float_rz(x))) || !(terr <= ldexp(fabs(x), -47));
        cnt++;
    }
    atomicAdd(out + 0, cnt);
    atomicAdd(out + 1, bad);
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_selftest_split(uint64_t n, uint64_t seed, uint64_t *out_checked, uint64_t *out_bad) {
    if (!out_checked || !out_bad) return GRIST_EINVAL;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return GRIST_ENOMEM;
    unsigned long long h[2] = {0, 0};
    int rc = GRIST_OK;
    if (cudaMemset(d, 0, sizeof(h)) != cudaSuccess) rc = GRIST_ECUDA;
    if (rc == GRIST_OK) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        k_check_split<<<(unsigned)(nsm > 0 ? nsm * 8 : 1024), 256>>>((unsigned long long)n, (unsigned long long)seed, d);
        if (cudaGetLastError() != cudaSuccess) rc = GRIST_ECUDA;
    }
    if (rc == GRIST_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = GRIST_ECUDA;
    cudaFree(d);
    if (rc != GRIST_OK) return rc;
    *out_checked = h[0];
    *out_bad = h[1];
    return GRIST_OK;
}

extern "C" int grist_selftest_reciprocal(uint64_t n, uint64_t seed, uint64_t *out_checked, uint64_t *out_over_1ulp,
                                         uint64_t *out_max_ulp) {
    if (!out_checked || !out_over_1ulp || !out_max_ulp) return GRIST_EINVAL;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 3 * sizeof(unsigned long long)) != cudaSuccess) return GRIST_ENOMEM;
    unsigned long long h[3] = {0, 0, 0};
    int rc = GRIST_OK;
    if (cudaMemset(d, 0, sizeof(h)) != cudaSuccess) rc = GRIST_ECUDA;
    if (rc == GRIST_OK) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        k_check_rcp<<<(unsigned)(nsm > 0 ? nsm * 8 : 1024), 256>>>((unsigned long long)n, (unsigned long long)seed, d);
        if (cudaGetLastError() != cudaSuccess) rc = GRIST_ECUDA;
    }
    if (rc == GRIST_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = GRIST_ECUDA;
    cudaFree(d);
    if (rc != GRIST_OK) return rc;
    *out_checked = h[0];
    *out_over_1ulp = h[1];
    *out_max_ulp = h[2];
    return GRIST_OK;
}

extern "C" int grist_selftest_conversions(uint64_t n_random, uint64_t seed, uint64_t *out_checked,
                                          uint64_t *out_mismatch) {
    if (!out_checked || !out_mismatch) return GRIST_EINVAL;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return GRIST_ENOMEM;
    unsigned long long h[4] = {0, 0, 0, 0};
    int rc = GRIST_OK;
    if (cudaMemset(d, 0, sizeof(h)) != cudaSuccess) rc = GRIST_ECUDA;
    if (rc == GRIST_OK) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const unsigned grid = (unsigned)(nsm > 0 ? nsm * 8 : 1024);
        k_check_f2d<<<grid, 256>>>(d);
        k_check_d2f<<<grid, 256>>>((unsigned long long)n_random, (unsigned long long)seed, d);
        if (cudaGetLastError() != cudaSuccess) rc = GRIST_ECUDA;
    }
    if (rc == GRIST_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = GRIST_ECUDA;
    cudaFree(d);
    if (rc != GRIST_OK) return rc;
    out_checked[0] = h[0];
    out_mismatch[0] = h[1];
    out_checked[1] = h[2];
    out_mismatch[1] = h[3];
    return GRIST_OK;
}
