// common.cuh - device-side mesh view, index helpers and precision policies
// shared by the kernels of the GRIST hot-path library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "grist.h"

#define GRIST_MAXE 6
#define GRIST_MAXEOE 10
#define GRIST_D2P 7
#define GRIST_MAXL 256

namespace grist {

// Mesh tables on the device, in the library's (space-filling-curve)
// numbering.  Per-cell / per-edge / per-vertex lists are padded to a fixed
// width with a valid index and a zero coefficient, so every loop runs a
// fixed trip count without branches.  Geometric factors are folded into
// the coefficient arrays once at mesh creation:
//   cdiv[i][j]  = s(e,i) dv_e / A_i        (cell divergence)
//   kec2[i][j]  = dc_e dv_e / (2 A_i)      (twice the cell kinetic energy)
//   ccurl[v][j] = t(e,v) dc_e / A_v        (vertex circulation)
//   ckite[v][j] = kite(i,v) / A_v          (cell -> vertex remap)
//   wpv[e][j]   = w(e,e') dv_e' / dc_e     (TRiSK tangential flux)
//   d2c[e][s][j]= deriv-two coefficient    (normal second derivative)
// Single-precision copies (suffix _f) feed the FP32 advective kernels.
struct DevMesh {
    int nC, nE, nV;
    // cells
    const int32_t *eoc;   // [nC][6]  pad: eoc[i][0]
    const int32_t *coc;   // [nC][6]  pad: i itself
    const double *cdiv;   // [nC][6]
    const float *cdiv_f;
    // the same three lists in rows of 8 (entries 6, 7: eoc[i][0], i, 0), read
    // as 16-byte vectors by the gather kernels
    const int32_t *eoc8;  // [nC][8]
    const int32_t *coc8;  // [nC][8]
    const double *cdiv8;  // [nC][8]
    const float *cdiv8_f;
    const double *kec2;   // [nC][6] dc dv / (2 A): twice the kinetic-energy weight
    const double *area;   // [nC]
    // edges
    const int2 *coe;      // [nE] (c1, c2)
    const int2 *voe;      // [nE] (v1, v2)
    const double *rdc;    // [nE] 1/dc
    const double *hrdc;   // [nE] -1/(2 dc)
    const double *dc2;    // [nE] dc^2/12
    const float *dc2_f;
    const int32_t *d2i;   // [nE][2][7] pad: centre cell
    const double *d2c;    // [nE][2][7]
    const float *d2c_f;
    // Upwind-side edge value in one weighted sum (beta = 1):
    // q_e = sum_j d2w[e][s][j] q(d2wi[e][s][j]), d2w = -2 (dc^2/12) d2c with
    // 1/2 added on the entries of c1 and c2; d2w_ok = 0 when some stencil
    // lacks c1 or c2 (then the separate form is used).  Rows of 8 (entry 7:
    // the side's centre cell, weight 0), read as 16-byte vectors.
    const int32_t *d2wi;  // [nE][2][8]
    const double *d2w;    // [nE][2][8]
    const float *d2w_f;
    int d2w_ok;
    // 1 when every edge side's combined stencil is its cell's ring {i,
    // coc[i][0..5]} in that order (so the upwind cell can form the edge
    // value from its ring) and cdiv[i][j] > 0 exactly when i is c1
    int ring_ok;
    const int32_t *eoe;   // [nE][10] pad: e itself
    const double *wpv;    // [nE][10]
    const float *wpv_f;
    // vertices
    const int32_t *eov;   // [nV][3]
    const int32_t *cov;   // [nV][3]
    const double *ccurl;  // [nV][3]
    const float *ccurl_f;
    const double *ckite;  // [nV][3]
    const double *fv;     // [nV]
    const float *fv_f;
};

// Division of a flat (entity, level) index by the level count without a
// hardware divide: q = umulhi(n, floor((2^32-1)/d)) is floor(n/d) or one
// less for n < 2^31; one correction step makes it exact.
struct LevelDiv {
    uint32_t d, m;
};
inline LevelDiv make_div(uint32_t d) { return LevelDiv{d, 0xFFFFFFFFu / d}; }

__device__ __forceinline__ void split_index(uint32_t n, LevelDiv D, int &ent, int &k) {
    uint32_t q = __umulhi(n, D.m);
    uint32_t r = n - q * D.d;
    if (r >= D.d) { q++; r -= D.d; }
    ent = (int)q;
    k = (int)r;
}

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Precision policies (Sec. 2.2 "ns" kind parameter; Sec. 2.3 mass switch).
//   TU : storage of the edge wind u_n
//   TA : advective compute / storage (theta flux, PV flux, tracer fluxes)
//   TM : mass flux dpi*V and its divergence
//   EMU: the kernels carry the binary32 row emulation of the precision search
//        (grist_dycore_params.emulate_fp32_rows); the production policies
//        compile without it.
//   DF : the pressure-gradient, gravity and kinetic-energy-gradient terms of
//        the momentum equation in binary32 arithmetic, their differences of
//        nearly equal FP64 fields taken from double-float splits
//        (GRIST_MIX_DF).
struct PolFP64 {
    using TU = double; using TA = double; using TM = double;
    static constexpr bool EMU = false, DF = false;
};
struct PolMIX {
    using TU = float; using TA = float; using TM = float;
    static constexpr bool EMU = false, DF = false;
};
struct PolMIXDBL {
    using TU = float; using TA = float; using TM = double;
    static constexpr bool EMU = false, DF = false;
};
struct PolFP64EMU {
    using TU = double; using TA = double; using TM = double;
    static constexpr bool EMU = true, DF = false;
};
struct PolMIXDF {
    using TU = float; using TA = float; using TM = float;
    static constexpr bool EMU = false, DF = true;
};

template <typename T> struct Coef;
template <> struct Coef<double> {
    static __device__ __forceinline__ const double *cdiv(const DevMesh &m) { return m.cdiv; }
    static __device__ __forceinline__ const double *cdiv8(const DevMesh &m) { return m.cdiv8; }
    static __device__ __forceinline__ const double *d2c(const DevMesh &m) { return m.d2c; }
    static __device__ __forceinline__ const double *d2w(const DevMesh &m) { return m.d2w; }
    static __device__ __forceinline__ const double *dc2(const DevMesh &m) { return m.dc2; }
    static __device__ __forceinline__ const double *wpv(const DevMesh &m) { return m.wpv; }
    static __device__ __forceinline__ const double *ccurl(const DevMesh &m) { return m.ccurl; }
    static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }  // DBL_MIN
};
template <> struct Coef<float> {
    static __device__ __forceinline__ const float *cdiv(const DevMesh &m) { return m.cdiv_f; }
    static __device__ __forceinline__ const float *cdiv8(const DevMesh &m) { return m.cdiv8_f; }
    static __device__ __forceinline__ const float *d2c(const DevMesh &m) { return m.d2c_f; }
    static __device__ __forceinline__ const float *d2w(const DevMesh &m) { return m.d2w_f; }
    static __device__ __forceinline__ const float *dc2(const DevMesh &m) { return m.dc2_f; }
    static __device__ __forceinline__ const float *wpv(const DevMesh &m) { return m.wpv_f; }
    static __device__ __forceinline__ const float *ccurl(const DevMesh &m) { return m.ccurl_f; }
    static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }  // FLT_MIN
};

__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }

// Entries 0..5 of row i of a [n][8] table, read as 16-byte vectors.
__device__ __forceinline__ void load_row6(const int32_t *t, int i, int (&v)[6]) {
    const int4 *p = (const int4 *)(t + (size_t)i * 8);
    const int4 a = __ldg(p), b = __ldg(p + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void load_row6(const float *t, int i, float (&v)[6]) {
    const float4 *p = (const float4 *)(t + (size_t)i * 8);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void load_row6(const double *t, int i, double (&v)[6]) {
    const double2 *p = (const double2 *)(t + (size_t)i * 8);
    const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// The combined upwind stencil of edge e on side s (0: c1's, 1: c2's): its
// 7 cells and weights, read as 16-byte vectors from the rows of 8.
static_assert(GRIST_D2P == 7, "combined stencil rows of 8 hold 7 entries");
__device__ __forceinline__ void load_d2w(const DevMesh &m, int e, int s, int (&c)[GRIST_D2P],
                                         float (&w)[GRIST_D2P]) {
    const size_t r = ((size_t)e * 2 + s) * 8;
    const int4 a = __ldg((const int4 *)(m.d2wi + r)), b = __ldg((const int4 *)(m.d2wi + r) + 1);
    const float4 u = __ldg((const float4 *)(m.d2w_f + r)), v = __ldg((const float4 *)(m.d2w_f + r) + 1);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w; c[4] = b.x; c[5] = b.y; c[6] = b.z;
    w[0] = u.x; w[1] = u.y; w[2] = u.z; w[3] = u.w; w[4] = v.x; w[5] = v.y; w[6] = v.z;
}
// The weights alone of the combined stencil row of edge e, side s.
__device__ __forceinline__ void load_d2w_weights(const DevMesh &m, int e, int s, float (&w)[GRIST_D2P]) {
    const size_t r = ((size_t)e * 2 + s) * 8;
    const float4 u = __ldg((const float4 *)(m.d2w_f + r)), v = __ldg((const float4 *)(m.d2w_f + r) + 1);
    w[0] = u.x; w[1] = u.y; w[2] = u.z; w[3] = u.w; w[4] = v.x; w[5] = v.y; w[6] = v.z;
}
__device__ __forceinline__ void load_d2w_weights(const DevMesh &m, int e, int s, double (&w)[GRIST_D2P]) {
    const double2 *p = (const double2 *)(m.d2w + ((size_t)e * 2 + s) * 8);
    const double2 u0 = __ldg(p), u1 = __ldg(p + 1), u2 = __ldg(p + 2), u3 = __ldg(p + 3);
    w[0] = u0.x; w[1] = u0.y; w[2] = u1.x; w[3] = u1.y; w[4] = u2.x; w[5] = u2.y; w[6] = u3.x;
}
__device__ __forceinline__ void load_d2w(const DevMesh &m, int e, int s, int (&c)[GRIST_D2P],
                                         double (&w)[GRIST_D2P]) {
    const size_t r = ((size_t)e * 2 + s) * 8;
    const int4 a = __ldg((const int4 *)(m.d2wi + r)), b = __ldg((const int4 *)(m.d2wi + r) + 1);
    const double2 *p = (const double2 *)(m.d2w + r);
    const double2 u0 = __ldg(p), u1 = __ldg(p + 1), u2 = __ldg(p + 2), u3 = __ldg(p + 3);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w; c[4] = b.x; c[5] = b.y; c[6] = b.z;
    w[0] = u0.x; w[1] = u0.y; w[2] = u1.x; w[3] = u1.y; w[4] = u2.x; w[5] = u2.y; w[6] = u3.x;
}
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }

// Correctly rounded reciprocal (the same value as 1.0 / x, without the
// general division sequence).
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// Reciprocal within one ulp from three FMAs: the approximate reciprocal of
// PTX (rcp.approx.ftz.f64, about 20 correct bits) refined by one cubically
// convergent Newton-Raphson step, y (1 + e + e^2) with e = 1 - x y, so the
// seed's relative error e shrinks to e^3 plus the rounding of the last FMA.
// For normal x with |x| in [2^-1020, 2^1020] (checked against 1.0 / x by
// grist_selftest_reciprocal); used where an FP64 instruction count matters
// more than correct rounding.
__device__ __forceinline__ double rcp_nr(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(fma(e, e, e), y, y);
}

// Conversions between binary32 and binary64 in integer arithmetic.  On this
// GPU the hardware conversion instructions issue on the FP64 pipe, the
// scarce resource of the mixed-precision kernels, so the IEEE-754 fields are
// moved with integer operations instead.  Results equal the hardware
// conversions bit for bit (round to nearest even; zeros, subnormals,
// infinities and NaN classes kept).
//
// binary32 -> binary64 is exact: rebias the exponent (127 -> 1023) and shift
// the fraction left by 29; a subnormal input is normalised first.
__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t s = u & 0x80000000u, a = u & 0x7fffffffu;
    uint32_t hi = (a >> 3) + 0x38000000u, lo = a << 29;   // 0x38000000 = (1023 - 127) << 20
    if (a >= 0x7f800000u) hi = (a >> 3) | 0x7ff00000u;      // infinity / NaN
    if (a < 0x00800000u) {                                  // zero / subnormal
        const int sh = __clz(a | 1u) - 8;                   // leading one to bit 23
        const uint32_t mnt = (a << sh) & 0x7fffffu;
        hi = a ? (((uint32_t)(897 - sh) << 20) | (mnt >> 3)) : 0u;
        lo = a ? (mnt << 29) : 0u;
    }
    return __hiloint2double((int)(hi | s), (int)lo);
}

// binary64 -> binary32, round to nearest, ties to even: keep the top 23
// fraction bits, round on the 29 dropped ones; exponents past the binary32
// range give infinity (NaN stays NaN); results below 2^-126 are rounded to
// the subnormal grid 2^-149.
__device__ __forceinline__ float d2f(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t s = hi & 0x80000000u, ah = hi & 0x7fffffffu;
    const int e = (int)(ah >> 20);
    uint32_t mag;
    if (e >= 897 && e <= 1150) {
        mag = ((uint32_t)(e - 896) << 23) | ((ah & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;
        mag += (uint32_t)(rest > 0x10000000u) | ((uint32_t)(rest == 0x10000000u) & (mag & 1u));
    } else if (e > 1150) {
        mag = (e == 2047 && ((ah & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
    } else {
        const int sh = 926 - e;                             // value = M 2^(e - 1075), M 53 bits
        if (e == 0 || sh >= 54) {
            mag = 0u;
        } else {
            const unsigned long long M = (1ull << 52) | ((unsigned long long)(ah & 0xfffffu) << 32) | lo;
            const unsigned long long q = M >> sh, r = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
            mag = (uint32_t)q + (uint32_t)((r > half) | ((r == half) & (q & 1ull)));
        }
    }
    return __uint_as_float(mag | s);
}

// Double-float split in integer arithmetic: x ~ h + l with h = RN32(x) and
// l = the residual x - h (exact in binary64, at most 29 significant bits)
// rounded to binary32, so h + l carries about 48 bits of x.  The residual
// is the difference of the two significands aligned at x's exponent.  For
// |x| < 2^-74 (where the residual's scale leaves the binary32 range) and
// for non-finite x, l = 0.  No FP64 instruction is issued.
__device__ __forceinline__ void split_df(double x, float &h, float &l) {
    h = d2f(x);
    l = 0.f;
    const uint32_t hx = (uint32_t)__double2hiint(x), lx = (uint32_t)__double2loint(x);
    const int ex = (int)((hx >> 20) & 0x7ffu);
    if (ex < 949 || ex > 1150) return;
    const uint32_t hb = __float_as_uint(h);
    const int eh = (int)((hb >> 23) & 0xffu) + 896;   // binary64 exponent of h (h is normal here)
    const long long mx = (long long)(((unsigned long long)((hx & 0xfffffu) | 0x100000u) << 32) | lx);
    long long mh = (long long)((unsigned long long)((hb & 0x7fffffu) | 0x800000u) << 29);
    if (eh == ex + 1) mh <<= 1;                        // x rounded up across a power of two
    const long long r = mx - mh;                       // |r| <= 2^28: units of 2^(ex - 1075)
    const float scale = __uint_as_float((uint32_t)(ex - 1075 + 127) << 23);
    const float rl = __int2float_rn((int)r) * scale;
    l = (hx & 0x80000000u) ? -rl : rl;
}

// binary64 -> binary32 by truncation, for inputs that are multiplied, not
// differenced, inside a tendency rounded to binary32 anyway: error below one
// binary32 ulp, no branches; magnitudes below 2^-126 give 0; finite inputs
// below 2^128 only (the dycore's layer and edge factors).
__device__ __forceinline__ float d2f_trunc(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t a = hi & 0x7fffffffu;
    uint32_t m = ((a - 0x38000000u) << 3) | (lo >> 29);
    m = a < 0x38100000u ? 0u : m;
    return __uint_as_float(m | (hi & 0x80000000u));
}

// Truncating double-float split for differencing: h = x truncated toward
// zero to binary32 (d2f_trunc), l = the 29 dropped significand bits, an
// integer in units of 2^(e - 1075), converted to binary32 and scaled, with
// the sign of x: |x - (h + l)| <= 2^-47 |x| for 2^-74 <= |x| < 2^128
// (smaller magnitudes keep h only; 2^128 and above, infinities and NaN
// give a NaN h).  About a dozen integer / binary32 instructions and no
// branch - cheaper than split_df where only differences of the pair are
// taken.
__device__ __forceinline__ void split_trunc(double x, float &h, float &l) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    h = ex > 1150 ? __uint_as_float(0x7fc00000u) : d2f_trunc(x);
    const float scale = (ex >= 949 && ex <= 1150) ? __uint_as_float((uint32_t)(ex - 1075 + 127) << 23) : 0.f;
    const float rl = __uint2float_rn(lo & 0x1fffffffu) * scale;
    l = __uint_as_float(__float_as_uint(rl) | (hi & 0x80000000u));
}

// a - b for two binary64 values of similar size, in binary32 arithmetic
// from their double-float splits: the high parts subtract exactly
// (Sterbenz, when within a factor of two), the low parts add the rest; the
// result is the difference to about 2^-24 of itself.
__device__ __forceinline__ float diff_df(float ah, float al, float bh, float bl) { return (ah - bh) + (al - bl); }

// cv<T>(x): x in type T, through the integer conversions above.
template <typename T> struct Cvt;
template <> struct Cvt<double> {
    static __device__ __forceinline__ double from(double x) { return x; }
    static __device__ __forceinline__ double from(float x) { return f2d(x); }
};
template <> struct Cvt<float> {
    static __device__ __forceinline__ float from(double x) { return d2f(x); }
    static __device__ __forceinline__ float from(float x) { return x; }
};
template <typename T, typename S> __device__ __forceinline__ T cv(S x) { return Cvt<T>::from(x); }

inline unsigned grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace grist

// Library handle (host side), defined in mesh.cu.
struct grist_mesh_s;
namespace grist {
const DevMesh &dev_mesh(grist_mesh_s *m);
int mesh_device(grist_mesh_s *m);
// Device scratch owned by the handle; grows (synchronously) when a call
// needs more than the current size.  slot separates independent users.
void *scratch(grist_mesh_s *m, int slot, size_t bytes);
uint32_t *status_word(grist_mesh_s *m);
// True while per-kernel profiling (grist_profile_enable) is on; a step then
// launches its kernels directly rather than replaying a captured graph, so
// every launch is timed.
bool profiling(grist_mesh_s *m);

// Host copies of the packed connectivity (internal numbering), kept for
// building derived tables (tracer tiles) after creation.
struct HostTables {
    int nC, nE, nV;
    std::vector<int32_t> eoc;   // [nC][6]
    std::vector<int2> coe;      // [nE]
    std::vector<int32_t> d2i;   // [nE][2][7]
};
const HostTables &host_tables(grist_mesh_s *m);
// The dycore's vertical-grid table (B, dB, 1/dB, ...) as last uploaded into
// its scratch, and the device address it went to: a step re-uploads it (and
// waits for the copy) only when either changed.
std::vector<double> &vg_cache(grist_mesh_s *m);
const void *&vg_ptr(grist_mesh_s *m);

// Tracer-step context (tuning, device tables, graph cache) kept in the
// handle; defined in tracer.cu.
struct TracerCtx;
TracerCtx *&tracer_ctx(grist_mesh_s *m);
void tracer_ctx_free(TracerCtx *c);

// Per-kernel event timing (grist_profile_enable): when profiling is on, the
// scope records an event before and after the launch it encloses.
struct ProfScope {
    grist_mesh_s *h;
    int slot;
    cudaStream_t st;
    ProfScope(grist_mesh_s *h, const char *name, cudaStream_t st);
    ~ProfScope();
};
}  // namespace grist

#define GRIST_LAUNCH(h, name, st, ...)                     \
    do {                                                   \
        ::grist::ProfScope prof_scope_(h, name, st);       \
        __VA_ARGS__;                                       \
    } while (0)

#define GRIST_CUDA_TRY(x)                                  \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return GRIST_ECUDA;         \
    } while (0)
