// sums.cu - deterministic compensated global sums (Sec. 2.3: global mass
// of pi_s - pi_t conserved to double-precision round-off; Sec. 4.4 local /
// global mass conservation).
//
// Pass 1: a fixed grid of kSumBlocks blocks; thread t of block b sums the
// terms t + b*kSumThreads + r*(kSumBlocks*kSumThreads) in increasing r with
// Neumaier's compensated summation, then the block combines its threads'
// (sum, compensation) pairs in a fixed tree with error-free TwoSum.
// Pass 2: one block combines the kSumBlocks partials the same way.  The
// order of every addition is fixed by the sizes alone, so the result is
// bitwise reproducible from run to run.
#include <cmath>

#include "common.cuh"

namespace grist {
namespace {

constexpr int kSumBlocks = 608;   // 4 x 152 SMs
constexpr int kSumThreads = 256;

struct DD {
    double s, c;  // value = s + c (c carries the accumulated rounding error)
};

__device__ __forceinline__ void neumaier(DD &a, double v) {
    const double t = a.s + v;
    if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
    else a.c += (v - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ DD dd_add(DD a, DD b) {
    // TwoSum of the leading parts (Knuth), compensation terms added
    const double s = a.s + b.s;
    const double bb = s - a.s;
    const double err = (a.s - (s - bb)) + (b.s - bb);
    return DD{s, a.c + b.c + err};
}

__device__ void block_combine(DD v, DD *out) {
    __shared__ double ss[kSumThreads], sc[kSumThreads];
    ss[threadIdx.x] = v.s;
    sc[threadIdx.x] = v.c;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            DD r = dd_add(DD{ss[threadIdx.x], sc[threadIdx.x]}, DD{ss[threadIdx.x + w], sc[threadIdx.x + w]});
            ss[threadIdx.x] = r.s;
            sc[threadIdx.x] = r.c;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = DD{ss[0], sc[0]};
}

// kind 0: A_i (x_i - offset); kind 1: A_i dpi_ik x_ik; kind 2: A_i x_ik.
template <typename T>
__global__ void k_sum_partial(DevMesh m, int kind, const T *__restrict__ x, const double *__restrict__ dpi, int L,
                              int ld, LevelDiv Dv, double offset, DD *__restrict__ part) {
    const long long n = kind == 0 ? (long long)m.nC : (long long)m.nC * L;
    DD acc{0.0, 0.0};
    const long long stride = (long long)kSumBlocks * kSumThreads;
    for (long long r = (long long)blockIdx.x * kSumThreads + threadIdx.x; r < n; r += stride) {
        double v;
        if (kind == 0) {
            v = ldg(m.area + r) * ((double)x[r] - offset);
        } else {
            int i, k;
            split_index((uint32_t)r, Dv, i, k);
            const size_t y = (size_t)i * ld + k;
            const double w = kind == 1 ? ldg(m.area + i) * dpi[y] : ldg(m.area + i);
            v = w * (double)x[y];
        }
        neumaier(acc, v);
    }
    block_combine(acc, part + blockIdx.x);
}

__global__ void k_sum_final(const DD *__restrict__ part, double *__restrict__ out) {
    DD acc{0.0, 0.0};
    for (int b = threadIdx.x; b < kSumBlocks; b += kSumThreads) acc = dd_add(acc, part[b]);
    __shared__ DD res;
    block_combine(acc, &res);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = res.s + res.c;
        out[1] = res.c;
    }
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_global_sums(grist_mesh h, grist_sum_kind kind, const void *field, const double *dpi,
                                 int32_t n_levels, int32_t ld, grist_precision field_prec, double offset,
                                 double *out, void *stream) {
    if (!h || !field || !out) return GRIST_EINVAL;
    if (kind != GRIST_SUM_DRY_MASS && kind != GRIST_SUM_TRACER_MASS && kind != GRIST_SUM_AREA_WEIGHTED)
        return GRIST_EINVAL;
    if (kind == GRIST_SUM_TRACER_MASS && !dpi) return GRIST_EINVAL;
    if (kind != GRIST_SUM_DRY_MASS && (n_levels < 1 || ld < n_levels)) return GRIST_EINVAL;
    if (kind == GRIST_SUM_DRY_MASS && field_prec != GRIST_FP64) return GRIST_EINVAL;
    const DevMesh &m = dev_mesh(h);
    if (kind != GRIST_SUM_DRY_MASS && (long long)m.nC * n_levels >= (1ll << 31)) return GRIST_EUNSUPPORTED;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    char *s = (char *)scratch(h, 2, sizeof(DD) * kSumBlocks + 256);
    if (!s) return GRIST_ENOMEM;
    DD *part = (DD *)s;
    double *res = (double *)(s + sizeof(DD) * kSumBlocks);
    cudaStream_t st = (cudaStream_t)stream;
    const int L = kind == GRIST_SUM_DRY_MASS ? 1 : n_levels;
    const LevelDiv D = make_div((uint32_t)L);
    if (field_prec == GRIST_FP64)
        k_sum_partial<double><<<kSumBlocks, kSumThreads, 0, st>>>(m, (int)kind, (const double *)field, dpi, L, ld, D,
                                                                  offset, part);
    else
        k_sum_partial<float><<<kSumBlocks, kSumThreads, 0, st>>>(m, (int)kind, (const float *)field, dpi, L, ld, D,
                                                                 offset, part);
    k_sum_final<<<1, kSumThreads, 0, st>>>(part, res);
    GRIST_CUDA_TRY(cudaGetLastError());
    GRIST_CUDA_TRY(cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GRIST_CUDA_TRY(cudaStreamSynchronize(st));
    return GRIST_OK;
}
