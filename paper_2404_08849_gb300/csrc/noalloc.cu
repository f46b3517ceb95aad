// noalloc.cu - weighted compensated sum that allocates no memory.
//
// Variant of the global-sum kernels (sums.cu) for callers that must not
// allocate device memory: programs whose device memory is owned by another
// allocator (a host model or framework that reserves the GPU's memory in its
// own pool up front, so an extra cudaMalloc would fail or fragment it) and
// code paths that must not pay the device-wide synchronisation a
// cudaMalloc / cudaFree can imply.  Its per-block partial sums live in a
// fixed file-scope device array instead of library scratch.
//
// Limits and sharing rules
//   - at most kNoAllocBlocks blocks of kNoAllocChunk elements each, i.e.
//     n <= GRIST_NOALLOC_MAX_TERMS terms; larger n is rejected with
//     GRIST_EINVAL before anything is launched;
//   - the array is one per device and is shared by every call: calls whose
//     GPU work overlaps (different streams, host threads or devices' calls
//     racing on one device) race on it.  Serialise them;
//   - every partial a call reads is written earlier in the same call, so no
//     part of the array has to start at zero and stale contents from the
//     previous call are never used;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current and caches it for the
//     life of the process; make that first call before any stream capture.
//     The cache assumes the device is not reset (cudaDeviceReset) between
//     calls: a reset reloads the module, and the cached address would no
//     longer name the array.
//   - the summation is the compensated method of grist_global_sums
//     (Neumaier accumulation, then a TwoSum tree) in an order of its own:
//     bitwise reproducible run to run, not bitwise equal to
//     grist_global_sums.
#include <mutex>

#include "common.cuh"

namespace grist {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = GRIST_NOALLOC_MAX_TERMS / GRIST_NOALLOC_CHUNK;
constexpr int kMaxDevices = 64;

struct DDv {
    double s, c;
};

// Per-block (sum, compensation) pairs followed by the final pair.
static __device__ __align__(256) DDv g_noalloc_partials[kNoAllocBlocks + 1];

__device__ __forceinline__ void neumaier_add(DDv &a, double v) {
    const double t = a.s + v;
    if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
    else a.c += (v - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ DDv two_sum_add(DDv a, DDv b) {
    const double s = a.s + b.s;
    const double bb = s - a.s;
    const double err = (a.s - (s - bb)) + (b.s - bb);
    return DDv{s, a.c + b.c + err};
}

__device__ DDv block_reduce(DDv v) {
    __shared__ double ss[kNoAllocThreads], sc[kNoAllocThreads];
    ss[threadIdx.x] = v.s;
    sc[threadIdx.x] = v.c;
    __syncthreads();
    for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            DDv r = two_sum_add(DDv{ss[threadIdx.x], sc[threadIdx.x]}, DDv{ss[threadIdx.x + w], sc[threadIdx.x + w]});
            ss[threadIdx.x] = r.s;
            sc[threadIdx.x] = r.c;
        }
        __syncthreads();
    }
    return DDv{ss[0], sc[0]};
}

// Block b sums terms [b*chunk, min(n, (b+1)*chunk)); thread t takes every
// kNoAllocThreads-th term of that chunk in increasing order.
__global__ void k_noalloc_partial(const double *__restrict__ x, const double *__restrict__ w, long long n,
                                  DDv *__restrict__ part) {
    const long long lo = (long long)blockIdx.x * GRIST_NOALLOC_CHUNK;
    long long hi = lo + GRIST_NOALLOC_CHUNK;
    if (hi > n) hi = n;
    DDv acc{0.0, 0.0};
    for (long long r = lo + threadIdx.x; r < hi; r += kNoAllocThreads) neumaier_add(acc, (w ? w[r] : 1.0) * x[r]);
    DDv b = block_reduce(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void k_noalloc_final(DDv *__restrict__ part, int nblocks, double *__restrict__ out) {
    DDv acc{0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kNoAllocThreads) acc = two_sum_add(acc, part[b]);
    DDv r = block_reduce(acc);
    if (threadIdx.x == 0) {
        part[kNoAllocBlocks] = r;
        out[0] = r.s + r.c;
        out[1] = r.c;
    }
}

std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the partials array on the current device (looked up
// once per device, with that device current).
int partials_address(int dev, DDv **out) {
    if (dev < 0 || dev >= kMaxDevices) return GRIST_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return GRIST_ECUDA;
        g_addr[dev] = p;
    }
    *out = (DDv *)g_addr[dev];
    return GRIST_OK;
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_weighted_sum_noalloc(const double *x, const double *w, int64_t n, double *out_sum_and_err,
                                          void *stream) {
    if (!x || !out_sum_and_err || n < 0) return GRIST_EINVAL;
    if (n > (int64_t)GRIST_NOALLOC_MAX_TERMS) return GRIST_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GRIST_ECUDA;
    DDv *part = nullptr;
    int rc = partials_address(dev, &part);
    if (rc != GRIST_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = n == 0 ? 0 : (int)((n + GRIST_NOALLOC_CHUNK - 1) / GRIST_NOALLOC_CHUNK);
    if (nb > 0) {
        k_noalloc_partial<<<nb, kNoAllocThreads, 0, st>>>(x, w, (long long)n, part);
        if (cudaGetLastError() != cudaSuccess) return GRIST_ECUDA;
    }
    k_noalloc_final<<<1, kNoAllocThreads, 0, st>>>(part, nb, out_sum_and_err);
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}
