// dycore.cu - GRIST dry dynamical core steps (Eqs. 3-9, Sec. 2.1):
// hydrostatic (RK3 + Mesinger forward-backward) and non-hydrostatic
// (horizontally explicit, vertically implicit) on the Voronoi C-grid, in
// FP64 or the paper's mixed precision (Sec. 2.3): advective terms in the
// policy's single-precision type, pressure gradient / gravity, vertical
// integrals, the equation of state, the column solve, surface pressure and
// layer mass in FP64.
//
// Layer fields [entity][ld], interface fields [cell][ld_int]; one thread per
// (entity, level) for the horizontal stencils, one warp per column for the
// vertical scans (continuity prefix, hydrostatic integral) and one thread
// per column for the tridiagonal solve.
//
// FP64 arithmetic is the scarce resource on this GPU (about 1/60 of the FP32
// rate), so divisions by layer masses are replaced by products with
// reciprocals formed once per column / edge / vertex (1/(ps - pi_top)) and
// once per level (1/dB), and the equation of state inside a stage is
// evaluated relative to the stage-input state (see pow1p_near0).
#include <cmath>
#include <vector>

#include "common.cuh"

#define PN(n) (P::DF ? n "/mixdf" : (sizeof(TA) == 4 ? (sizeof(TM) == 8 ? n "/mixdbl" : n "/mix") : n "/fp64"))

namespace grist {
namespace {

constexpr int kBlock = 256;
constexpr int kNHMax = 128;  // levels supported by the column solver

struct DyPar {
    int L, ld, ldi;
    double pi_top, p0, rd, cp, g, beta, kappa, gamma;
    const double *B;      // [L+1] interface coordinate
    const double *dB;     // [L]   layer thickness in B
    const double *rdB;    // [L]   1/dB
    const double *hrdBi;  // [L+1] 1/(dB[j-1] + dB[j]) at interior interfaces j (half the reciprocal mean)
    const double *dBi;    // [L+1] (dB[j-1] + dB[j])/2 at interior interfaces j
    const float *dBf;     // [L]   dB rounded to single precision
    const double *phis;   // [nC]  surface geopotential
    uint32_t emu;         // GRIST_ROW_* rows rounded to binary32 (precision search)
};

// Storage-rounding emulation of a single-precision row (precision search,
// Sec. 2.2 Eqs. 1-2): in the emulating FP64 policy (E) a double value of a
// row whose bit is set is rounded to binary32 where it is produced; the
// production policies compile to the plain value.
template <bool E> __device__ __forceinline__ double emu(double x, uint32_t mask, uint32_t bit) {
    if (E) return (mask & bit) ? (double)(float)x : x;
    return x;
}
template <bool E> __device__ __forceinline__ float emu(float x, uint32_t, uint32_t) { return x; }

// GRIST_MIX_DF: a double field that the momentum equation only differences
// (layer phi, K) is stored as its double-float split (h, l) in the same
// 8-byte slot, read back as a float2.
__device__ __forceinline__ double pack_split(double x) {
    float h, l;
    split_df(x, h, l);
    return __hiloint2double(__float_as_int(l), __float_as_int(h));
}

// Compensated single-precision accumulation (Knuth's TwoSum): a value is
// hi + lo with |lo| <= ulp(hi)/2, so a sum of FP32 terms carries about 48
// significant bits - as accurate as FP64 accumulation of the same FP32
// terms - while running on the FP32 pipe (FP64 instructions, conversions
// included, are the scarce resource on this GPU).
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = e + a.lo + b.lo;
    const float hi = s + lo;
    return F2{hi, lo - (hi - s)};
}
__device__ __forceinline__ F2 f2_shfl_xor(F2 v, int o) {
    return F2{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ F2 f2_shfl_up(F2 v, int o) {
    return F2{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}

// Column sum of a level-indexed value over the warp's lanes: FP64 terms
// are added in FP64; FP32 terms in compensated FP32, converted once.
__device__ __forceinline__ double col_reduce(double part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    return part;
}

// r^g for a ratio r close to 1 by the binomial series
// (1 + x)^g = sum_n C(g, n) x^n, Horner in FP64, with the binomial
// coefficients C(g, n) = C(g, n-1) (g - n + 1)/n formed on the host.  For
// |g| < 2 the coefficients stay below 4 in magnitude up to n = 16, so after N
// terms the omitted tail is below 4 |x|^N / (1 - |x|): the warp takes the
// shortest series with 4 |x|^N <= 2^-58 for the largest |x| among its lanes
// (N = 4, 5, 6, 8, 10 for |x| < 2^-15, 2^-12, 2^-10, 2^-8, 2^-6) - a
// warp-uniform branch, so no FP64 issue slot is spent on terms no lane
// needs.  A lane with |x| > 2^-6 uses the library pow().  mask: the lanes
// executing the call.
struct Binom {
    double c[10];
    float f[6];   // the same coefficients in binary32 (GRIST_MIX_DF increments)
};

template <int N> __device__ __forceinline__ double horner(double x, const Binom &B) {
    double s = B.c[N - 1];
#pragma unroll
    for (int n = N - 2; n >= 0; n--) s = fma(s, x, B.c[n]);
    return s;
}

// (1 + x)^g for a small x given directly.
__device__ __forceinline__ double pow1p_near0(double x, double g, const Binom &B, unsigned mask) {
    // high word of |x|: exponent and leading fraction bits, monotone in |x|
    const unsigned hx = (unsigned)__double2hiint(x) & 0x7fffffffu;
    const unsigned hm = __reduce_max_sync(mask, hx);
    if (hm < 0x3f000000u) return horner<4>(x, B);    // |x| < 2^-15
    if (hm < 0x3f300000u) return horner<5>(x, B);    // 2^-12
    if (hm < 0x3f500000u) return horner<6>(x, B);    // 2^-10
    if (hm < 0x3f700000u) return horner<8>(x, B);    // 2^-8
    if (hx > 0x3f900000u || (hx == 0x3f900000u && __double2loint(x) != 0)) return pow(1.0 + x, g);
    return horner<10>(x, B);
}

Binom binomial(double g) {
    Binom b;
    b.c[0] = 1.0;
    for (int n = 1; n < 10; n++) b.c[n] = b.c[n - 1] * (g - (n - 1)) / n;
    for (int n = 0; n < 6; n++) b.f[n] = (float)b.c[n];
    return b;
}

// GRIST_MIX_DF form of p (1 + x)^g for |x| <= 2^-6: the increment
// (1 + x)^g - 1 = x (C1 + x (C2 + ... + x C5)) in binary32 (the omitted
// terms are below 2^-30 of it), added to p in FP64 - the increment's
// binary32 rounding, about 2^-23 |g x|, is ~1e-10 of p for |x| ~ 1e-3.
// Larger |x| (none in a stable step) falls back to the FP64 pow.
__device__ __forceinline__ double scale_near1_df(double p, double x, double g, const Binom &B) {
    const unsigned hx = (unsigned)__double2hiint(x) & 0x7fffffffu;
    if (hx > 0x3f900000u) return p * pow(1.0 + x, g);
    const float xf = d2f(x);
    float s = B.f[5];
#pragma unroll
    for (int n = 4; n >= 1; n--) s = fmaf(s, xf, B.f[n]);
    return fma(p, f2d(s * xf), p);
}

// ---------------------------------------------------------------------------
// Eq. 3: mass flux at edges F = dpi_e u, dpi_e = mean of the two cells'
// layer mass = dB_k (ps1 + ps2 - 2 pi_top)/2.  One warp takes 32 edges: the
// per-edge FP64 work (column factor, the reciprocal 1/(ps1 + ps2 - 2 pi_top)
// for the momentum equation) runs one edge per lane - an FP64 instruction
// costs the FP64 pipe a full warp slot however few lanes are active - then
// the warp walks its edges with the lanes over levels, forming the product
// in the mass-flux type and the edge's column sum sum_k F_k by a fixed
// butterfly (both cells of the edge later use the same value, so the global
// mass change cancels to round-off).  In the final stage fscale times the
// flux is accumulated for the tracer solver (Sec. 2.3: single computed,
// saved double).
template <class P>
__global__ void k_mass_edge(DevMesh m, DyPar d, const double *__restrict__ ps_s,
                            const typename P::TU *__restrict__ u_s, typename P::TM *__restrict__ F,
                            double *__restrict__ Facc, double fscale, double *__restrict__ rsum_e,
                            double *__restrict__ Fcol) {
    const bool scaled = fscale != 1.0;
    using TM = typename P::TM;
    const int e0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    const int lane = threadIdx.x & 31;
    if (e0 >= m.nE) return;
    const int ne = min(32, m.nE - e0);
    TM hs_l = 0;
    if (lane < ne) {
        const int2 c = ldg(m.coe + e0 + lane);
        const double sum = (ldg(ps_s + c.x) - d.pi_top) + (ldg(ps_s + c.y) - d.pi_top);
        hs_l = cv<TM>(0.5 * sum);
        rsum_e[e0 + lane] = 0.5 * rcp(sum);   // 1 / (2 dpi_e / dB)
    }
    double col64 = 0.0;
    float col_hi = 0.f, col_lo = 0.f;
    for (int j = 0; j < ne; j++) {
        const int e = e0 + j;
        const TM hs = __shfl_sync(0xffffffffu, hs_l, j);
        if (sizeof(TM) == 8) {
            double col = 0.0;
            for (int k = lane; k < d.L; k += 32) {
                const size_t x = (size_t)e * d.ld + k;
                const TM f = emu<P::EMU>((TM)ldg(d.dB + k) * hs * cv<TM>(u_s[x]), d.emu, GRIST_ROW_MASS_FLUX);
                F[x] = f;
                col += (double)f;
                if (Facc) Facc[x] += scaled ? fscale * (double)f : (double)f;
            }
            col = col_reduce(col);
            if (lane == j) col64 = col;
        } else {
            F2 col{0.f, 0.f};
            for (int k = lane; k < d.L; k += 32) {
                const size_t x = (size_t)e * d.ld + k;
                const TM f = ldg(d.dBf + k) * hs * cv<TM>(u_s[x]);
                F[x] = f;
                col = f2_add(col, F2{cv<float>(f), 0.f});
                if (Facc) Facc[x] += scaled ? fscale * cv<double>(f) : cv<double>(f);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) col = f2_add(col, f2_shfl_xor(col, o));
            if (lane == j) {
                col_hi = col.hi;
                col_lo = col.lo;
            }
        }
    }
    if (lane < ne) Fcol[e0 + lane] = sizeof(TM) == 8 ? col64 : f2d(col_hi) + f2d(col_lo);
}

// Eq. 3 column part.  One warp takes 32 cells; the per-cell FP64 work (the
// surface pressure tendency -sum_j s dv/A (column sum of edge j), its stage
// update, 1/(ps - pi_top)) runs one cell per lane, then the warp walks its
// cells with the lanes over levels: layer divergence D_k (mass-flux type),
// vertical mass flux M_{k+1/2} = -B_{k+1/2} dps/dt - sum_{l<=k} D_l by a
// warp scan, theta = (dpi theta)/dpi of the stage input for Eq. 4.
template <class P>
__global__ void k_mass_col(DevMesh m, DyPar d, const typename P::TM *__restrict__ F,
                           const double *__restrict__ Fcol, const double *__restrict__ ps_s,
                           const double *__restrict__ ps_n, double *__restrict__ ps_out,
                           const double *__restrict__ th_s, typename P::TA *__restrict__ theta,
                           double *__restrict__ Mv, double dts, double *__restrict__ dpi_out,
                           double *__restrict__ rdps_out, double *__restrict__ rth_out,
                           double *__restrict__ Macc, double fscale) {
    using TM = typename P::TM;
    using TA = typename P::TA;
    const int i0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    const int lane = threadIdx.x & 31;
    if (i0 >= m.nC) return;
    const int nci = min(32, m.nC - i0);
    double pst_l = 0.0, dps_l = 0.0, rdps_l = 0.0;
    if (lane < nci) {
        const int i = i0 + lane;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) pst_l -= ldg(m.cdiv + i * 6 + j) * ldg(Fcol + ldg(m.eoc + i * 6 + j));
        dps_l = ldg(ps_s + i) - d.pi_top;
        rdps_l = rcp(dps_l);
        ps_out[i] = ps_n[i] + dts * pst_l;
        rdps_out[i] = rdps_l;
        Mv[(size_t)i * d.ldi] = 0.0;
        Mv[(size_t)i * d.ldi + d.L] = 0.0;
    }
    const int nch = (d.L + 31) >> 5;
    for (int c = 0; c < nci; c++) {
        const int i = i0 + c;
        const double pst = __shfl_sync(0xffffffffu, pst_l, c);
        const double dps = __shfl_sync(0xffffffffu, dps_l, c);
        const double rdps = __shfl_sync(0xffffffffu, rdps_l, c);
        int eidx[GRIST_MAXE];
        TM cw[GRIST_MAXE];
        load_row6(m.eoc8, i, eidx);
        load_row6(Coef<TM>::cdiv8(m), i, cw);
        double run = 0.0;
        F2 runf{0.f, 0.f};
        for (int ch = 0; ch < nch; ch++) {
            const int k = ch * 32 + lane;
            TM s = 0;
            if (k < d.L) {
#pragma unroll
                for (int j = 0; j < GRIST_MAXE; j++) s += cw[j] * ldg(F + (size_t)eidx[j] * d.ld + k);
                s = emu<P::EMU>(s, d.emu, GRIST_ROW_MASS_FLUX);
                const size_t x = (size_t)i * d.ld + k;
                theta[x] = emu<P::EMU>(cv<TA>(th_s[x] * ldg(d.rdB + k) * rdps), d.emu, GRIST_ROW_THETA);
                if (dpi_out) dpi_out[x] = ldg(d.dB + k) * dps;
                if (rth_out) rth_out[x] = rcp(th_s[x]);
            }
            // inclusive prefix of D over the chunk, carried across chunks:
            // FP64 terms in FP64, FP32 terms in compensated FP32
            if (sizeof(TM) == 8) {
                double v = (double)s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const double t = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += t;
                }
                if (k < d.L - 1) {
                    const double mk = -ldg(d.B + k + 1) * pst - (run + v);
                    Mv[(size_t)i * d.ldi + k + 1] = mk;
                    if (Macc) Macc[(size_t)i * d.ldi + k + 1] += fscale * mk;
                }
                run += __shfl_sync(0xffffffffu, v, 31);
            } else {
                // the earlier chunks' total is carried as a compensated pair
                // too, so the prefix reaches FP64 once, at M
                F2 v{cv<float>(s), 0.f};
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const F2 t = f2_shfl_up(v, o);
                    if (lane >= o) v = f2_add(v, t);
                }
                v = f2_add(v, runf);
                if (k < d.L - 1) {
                    const double mk = -ldg(d.B + k + 1) * pst - (f2d(v.hi) + f2d(v.lo));
                    Mv[(size_t)i * d.ldi + k + 1] = mk;
                    if (Macc) Macc[(size_t)i * d.ldi + k + 1] += fscale * mk;
                }
                runf = F2{__shfl_sync(0xffffffffu, v.hi, 31), __shfl_sync(0xffffffffu, v.lo, 31)};
            }
        }
    }
}

// Eq. 4 horizontal flux: third-order upwind (beta = 1) edge value of theta
// times the mass flux.  A thread takes levels kg and kg + Lh (Lh = ceil(L/2))
// of one edge, so the upwind stencil row (4 vector loads) serves both
// levels unless their fluxes run opposite ways.
template <class P>
__global__ void k_theta_flux(DevMesh m, DyPar d, LevelDiv Dh, const typename P::TM *__restrict__ F,
                             const typename P::TA *__restrict__ th, typename P::TA *__restrict__ Fth) {
    using TA = typename P::TA;
    const int Lh = (int)Dh.d;
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nE * (uint32_t)Lh) return;
    int e, kg;
    split_index(n, Dh, e, kg);
    int c[GRIST_D2P];
    TA w[GRIST_D2P];
    int loaded = -1;
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int k = kg + u * Lh;
        if (k >= d.L) break;
        const size_t x = (size_t)e * d.ld + k;
        const TA f = cv<TA>(F[x]);
        const int side = f >= (TA)0 ? 0 : 1;
        TA te;
        if (m.d2w_ok) {
            // one weighted sum over the upwind side's stencil (the mean of
            // the edge's two cells folded into the weights)
            if (side != loaded) {
                load_d2w(m, e, side, c, w);
                loaded = side;
            }
            te = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) te += w[j] * ldg(th + (size_t)c[j] * d.ld + k);
        } else {
            const int32_t *st = m.d2i + (size_t)e * 14 + side * GRIST_D2P;
            const int2 ce = ldg(m.coe + e);
            const TA *cf = Coef<TA>::d2c(m) + (size_t)e * 14 + side * GRIST_D2P;
            TA sm = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) sm += ldg(cf + j) * ldg(th + (size_t)ldg(st + j) * d.ld + k);
            te = (TA)0.5 * (ldg(th + (size_t)ce.x * d.ld + k) + ldg(th + (size_t)ce.y * d.ld + k)) -
                 (TA)2 * ldg(Coef<TA>::dc2(m) + e) * sm;
        }
        Fth[x] = emu<P::EMU>(f * te, d.emu, GRIST_ROW_THETA);
    }
}

// Eq. 4 update: dpi theta^(s) = dpi theta^n + dt_s (-div F_theta - delta(M theta)).
template <class P>
__global__ void k_theta_update(DevMesh m, DyPar d, LevelDiv Dh, const typename P::TA *__restrict__ Fth,
                               const typename P::TA *__restrict__ th, const double *__restrict__ Mv,
                               const double *__restrict__ th_n, double *__restrict__ th_out, double dts) {
    using TA = typename P::TA;
    const int Lh = (int)Dh.d;
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)Lh) return;
    int i, kg;
    split_index(n, Dh, i, kg);
    // the cell's row once for its two levels kg and kg + Lh
    int eidx[GRIST_MAXE];
    TA cw[GRIST_MAXE];
    load_row6(m.eoc8, i, eidx);
    load_row6(Coef<TA>::cdiv8(m), i, cw);
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int k = kg + u * Lh;
        if (k >= d.L) break;
        TA div = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) div += cw[j] * ldg(Fth + (size_t)eidx[j] * d.ld + k);
        const size_t x = (size_t)i * d.ld + k;
        const TA tk = th[x];
        TA top = 0, bot = 0;
        if (k > 0) top = cv<TA>(Mv[(size_t)i * d.ldi + k]) * ((TA)0.5 * (th[x - 1] + tk));
        if (k < d.L - 1) bot = cv<TA>(Mv[(size_t)i * d.ldi + k + 1]) * ((TA)0.5 * (tk + th[x + 1]));
        const TA tend = -div - (bot - top);
        th_out[x] = th_n[x] + dts * cv<double>(tend);
    }
}

// Eq. 8 (hydrostatic diagnostics), one warp per column: mid-layer pressure,
// alpha = Rd theta (p/p0)^kappa / p, geopotential integrated upward from
// phi_s by a suffix scan, layer geopotential = mean of its interfaces.
template <bool EMU, bool DF>
__global__ void k_hydro_diag(DevMesh m, DyPar d, const double *__restrict__ ps, const double *__restrict__ th,
                             double *__restrict__ p, double *__restrict__ al, double *__restrict__ phl) {
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= m.nC) return;
    const double dps = ps[i] - d.pi_top;
    const double rdps = rcp(dps);
    const int nch = (d.L + 31) >> 5;
    double carry = ldg(d.phis + i);
    for (int ch = nch - 1; ch >= 0; ch--) {
        const int k = ch * 32 + lane;
        double contrib = 0.0, a = 0.0, pk = 0.0;
        if (k < d.L) {
            const double pt = d.pi_top + ldg(d.B + k) * dps, pb = d.pi_top + ldg(d.B + k + 1) * dps;
            const double dp = pb - pt;
            pk = 0.5 * (pt + pb);
            a = d.rd * (th[(size_t)i * d.ld + k] * ldg(d.rdB + k) * rdps) * pow(pk / d.p0, d.kappa) / pk;
            contrib = a * dp;
        }
        // inclusive suffix sum within the chunk
        double v = contrib;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o < 32) v += t;
        }
        if (k < d.L) {
            const size_t x = (size_t)i * d.ld + k;
            p[x] = emu<EMU>(pk, d.emu, GRIST_ROW_EOS);
            al[x] = emu<EMU>(a, d.emu, GRIST_ROW_EOS);
            const double ph = carry + (v - contrib) + 0.5 * contrib;
            phl[x] = DF ? pack_split(ph) : emu<EMU>(ph, d.emu, GRIST_ROW_EOS);
        }
        carry += __shfl_sync(0xffffffffu, v, 0);
    }
}

// Column reciprocal of the kite-remapped vertex layer mass:
// 1 / sum_i kite(i,v)/A_v (ps_i - pi_top); the layer value is dB_k times it.
template <bool EMU>
__global__ void k_vertex_mass(DevMesh m, DyPar d, const double *__restrict__ ps_s, double *__restrict__ rdpv) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.nV) return;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++) s += ldg(m.ckite + v * 3 + j) * (ldg(ps_s + ldg(m.cov + v * 3 + j)) - d.pi_top);
    rdpv[v] = emu<EMU>(rcp(s), d.emu, GRIST_ROW_DPI_PV);
}

// Vertex PV, Sec. 2.3: zeta_p = (zeta + f) / dpi_v, the relative vorticity
// from the circulation of u (advective type), dpi_v the kite-weighted remap
// of the FP64 layer mass (dpi must be double for zeta_p).  In a binary32
// advective type the FP64 factor 1/dpi_v = (1/dB_k)(1/dpi_col) is formed
// first and rounded once, then the rest is binary32 arithmetic (Sec. 2.2
// (ii): no mixed-kind expression): one FP64 product per vertex-level.
template <class P>
__global__ void k_vort(DevMesh m, DyPar d, LevelDiv Dh, const typename P::TU *__restrict__ u,
                       const double *__restrict__ rdpv, typename P::TA *__restrict__ qv) {
    using TA = typename P::TA;
    const int Lh = (int)Dh.d;
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nV * (uint32_t)Lh) return;
    int v, kg;
    split_index(n, Dh, v, kg);
    // the vertex's edges and weights once for its two levels kg and kg + Lh
    int ev[3];
    TA cc[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        ev[j] = ldg(m.eov + v * 3 + j);
        cc[j] = ldg(Coef<TA>::ccurl(m) + v * 3 + j);
    }
    const double rv = ldg(rdpv + v);
#pragma unroll
    for (int w = 0; w < 2; w++) {
        const int k = kg + w * Lh;
        if (k >= d.L) break;
        TA z = 0;
#pragma unroll
        for (int j = 0; j < 3; j++) z += cc[j] * cv<TA>(ldg(u + (size_t)ev[j] * d.ld + k));
        if constexpr (sizeof(TA) == 4) {
            qv[(size_t)v * d.ld + k] = (z + ldg(m.fv_f + v)) * d2f(ldg(d.rdB + k) * rv);
        } else {
            qv[(size_t)v * d.ld + k] = emu<P::EMU>(cv<TA>((cv<double>(z) + ldg(m.fv + v)) * (ldg(d.rdB + k) * rv)),
                                                   d.emu, GRIST_ROW_PV_FLUX);
        }
    }
}

// Cell kinetic energy, stored doubled: 2K = sum (dc dv / 2A) u^2 (FP64:
// boxed term of Eq. 5).
template <class P>
__global__ void k_ke(DevMesh m, DyPar d, LevelDiv Dv, const typename P::TU *__restrict__ u, double *__restrict__ K) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)d.L) return;
    int i, k;
    split_index(n, Dv, i, k);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        const double ue = cv<double>(ldg(u + (size_t)ldg(m.eoc + i * 6 + j) * d.ld + k));
        s += ldg(m.kec2 + i * 6 + j) * ue * ue;
    }
    K[(size_t)i * d.ld + k] = P::DF ? pack_split(s) : emu<P::EMU>(s, d.emu, GRIST_ROW_KE_GRAD);
}

// PV at edge-level (e, k): the mean of the PV at the edge's two vertices.
template <class P>
__device__ __forceinline__ typename P::TA pv_at_edge(const DevMesh &m, const DyPar &d,
                                                     const typename P::TA *__restrict__ qv, int e, int k) {
    using TA = typename P::TA;
    const int2 v = ldg(m.voe + e);
    return emu<P::EMU>((TA)0.5 * (ldg(qv + (size_t)v.x * d.ld + k) + ldg(qv + (size_t)v.y * d.ld + k)), d.emu,
                       GRIST_ROW_PV_FLUX);
}

// Eq. 5 momentum tendency and stage update:
//   PV flux (1/dc) sum w dv' F' (q_e + q_e')/2          [advective type]
//   - dK/dn - eta-dot du/deta                              [FP64, boxed]
//   - alpha_e dp/dn - (dp/dpi)_e dphi/dn                   [FP64]
// with the tendency rounded to the wind's type (Sec. 2.3: boxed terms are
// computed in double, their tendency saved in single).  The edge layer mass
// in the vertical advection is dB_k (ps1 + ps2 - 2 pi_top)/2, entered as
// the product of the per-level and per-edge reciprocals.
template <class P, bool NH>
__global__ void k_momentum(DevMesh m, DyPar d, LevelDiv Dv, const typename P::TU *__restrict__ u_s,
                           const typename P::TU *u_n, typename P::TU *u_out, const typename P::TM *__restrict__ F,
                           const typename P::TA *__restrict__ qv, const double *__restrict__ K,
                           const double *__restrict__ Mv, const double *__restrict__ rsum_e,
                           const double *__restrict__ p, const double *__restrict__ al,
                           const double *__restrict__ phl, const double *__restrict__ dpp, double dts,
                           uint32_t *status) {
    using TA = typename P::TA;
    using TU = typename P::TU;
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nE * (uint32_t)d.L) return;
    int e, k;
    split_index(n, Dv, e, k);
    const size_t x = (size_t)e * d.ld + k;
    const int2 c = ldg(m.coe + e);
    // the edge PV values come from the vertex PV (the mean of the two
    // vertices, formed here: this kernel is bound by the FP64 pipe and has
    // load slots to spare, so no separate edge-PV pass is needed)
    const TA qee = pv_at_edge<P>(m, d, qv, e, k);
    TA pv = 0;
#pragma unroll
    for (int j = 0; j < GRIST_MAXEOE; j++) {
        const int e2 = ldg(m.eoe + e * 10 + j);
        const size_t y = (size_t)e2 * d.ld + k;
        pv += ldg(Coef<TA>::wpv(m) + e * 10 + j) * cv<TA>(ldg(F + y)) * ((TA)0.5 * (qee + pv_at_edge<P>(m, d, qv, e2, k)));
    }
    const size_t a1 = (size_t)c.x * d.ld + k, a2 = (size_t)c.y * d.ld + k;
    if (P::DF) {
        // GRIST_MIX_DF: the slow tendency in binary32; the differences of the
        // double fields p, layer phi and K from their double-float splits
        // (p split here, phi and K stored split), the factors that are only
        // multiplied truncated to binary32, every other operation in binary32
        // - no FP64 instruction
        const float uk = (float)ldg(u_s + x);
        float va32 = 0.f;
        if (k < d.L - 1)
            va32 = (d2f_trunc(ldg(Mv + (size_t)c.x * d.ldi + k + 1)) +
                    d2f_trunc(ldg(Mv + (size_t)c.y * d.ldi + k + 1))) *
                   ((float)ldg(u_s + x + 1) - uk);
        if (k > 0)
            va32 = fmaf(d2f_trunc(ldg(Mv + (size_t)c.x * d.ldi + k)) + d2f_trunc(ldg(Mv + (size_t)c.y * d.ldi + k)),
                        uk - (float)ldg(u_s + x - 1), va32);
        va32 *= d2f_trunc(ldg(d.rdB + k)) * d2f_trunc(ldg(rsum_e + e));
        float p1h, p1l, p2h, p2l;
        split_df(ldg(p + a1), p1h, p1l);
        split_df(ldg(p + a2), p2h, p2l);
        const float2 f1 = ldg(reinterpret_cast<const float2 *>(phl) + a1);
        const float2 f2 = ldg(reinterpret_cast<const float2 *>(phl) + a2);
        const float2 k1 = ldg(reinterpret_cast<const float2 *>(K) + a1);
        const float2 k2 = ldg(reinterpret_cast<const float2 *>(K) + a2);
        const float de = NH ? d2f_trunc(ldg(dpp + a1)) + d2f_trunc(ldg(dpp + a2)) : 2.f;
        const float grad = fmaf(d2f_trunc(ldg(al + a1)) + d2f_trunc(ldg(al + a2)), diff_df(p2h, p2l, p1h, p1l),
                                fmaf(de, diff_df(f2.x, f2.y, f1.x, f1.y), diff_df(k2.x, k2.y, k1.x, k1.y)));
        const float tend = (float)pv + fmaf(d2f_trunc(ldg(m.hrdc + e)), grad, -va32);
        const float v = (float)u_n[x] + d2f(dts) * tend;
        if (!isfinite(v)) atomicOr(status, GRIST_FLAG_NONFINITE);
        u_out[x] = (TU)v;
        return;
    }
    const double uk = cv<double>(ldg(u_s + x));
    double va = 0.0;
    if (k < d.L - 1)
        va = (ldg(Mv + (size_t)c.x * d.ldi + k + 1) + ldg(Mv + (size_t)c.y * d.ldi + k + 1)) *
             (cv<double>(ldg(u_s + x + 1)) - uk);
    if (k > 0)
        va = fma(ldg(Mv + (size_t)c.x * d.ldi + k) + ldg(Mv + (size_t)c.y * d.ldi + k),
                 uk - cv<double>(ldg(u_s + x - 1)), va);
    // [M sums](du) / (2 dpi_e) with dpi_e = dB (sum)/2, M_e = (M1 + M2)/2;
    // rsum_e holds 1/(2 sum)
    va *= ldg(d.rdB + k) * ldg(rsum_e + e);
    va = emu<P::EMU>(va, d.emu, GRIST_ROW_VADV_U);
    // dK/dn + alpha_e dp/dn + (dp/dpi)_e dphi/dn with the two means folded
    // into -1/(2 dc) (hrdc) and K stored doubled
    double grad;
    if (!P::EMU || !(d.emu & GRIST_ROW_PGF)) {
        const double de = NH ? ldg(dpp + a1) + ldg(dpp + a2) : 2.0;
        grad = fma(ldg(al + a1) + ldg(al + a2), ldg(p + a2) - ldg(p + a1),
                   fma(de, ldg(phl + a2) - ldg(phl + a1), ldg(K + a2) - ldg(K + a1)));
    } else {
        // pressure gradient and gravity from binary32 inputs, summed and
        // rounded to binary32 (precision search)
        const uint32_t r = GRIST_ROW_PGF;
        const double de = NH ? emu<P::EMU>(ldg(dpp + a1), d.emu, r) + emu<P::EMU>(ldg(dpp + a2), d.emu, r) : 2.0;
        const double pgf = emu<P::EMU>(fma(emu<P::EMU>(ldg(al + a1), d.emu, r) + emu<P::EMU>(ldg(al + a2), d.emu, r),
                                   emu<P::EMU>(ldg(p + a2), d.emu, r) - emu<P::EMU>(ldg(p + a1), d.emu, r),
                                   de * (emu<P::EMU>(ldg(phl + a2), d.emu, r) - emu<P::EMU>(ldg(phl + a1), d.emu, r))),
                               d.emu, r);
        grad = pgf + (ldg(K + a2) - ldg(K + a1));
    }
    const double slow = fma(ldg(m.hrdc + e), grad, -va);
    const TA tend = emu<P::EMU>(pv, d.emu, GRIST_ROW_PV_FLUX) + cv<TA>(slow);
    const TU v = emu<P::EMU>(cv<TU>(cv<TA>(u_n[x]) + cv<TA>(dts) * tend), d.emu, GRIST_ROW_WIND);
    if (!isfinite(v)) atomicOr(status, GRIST_FLAG_NONFINITE);
    u_out[x] = v;
}

// ---------------------------------------------------------------------------
// Non-hydrostatic pieces (Eqs. 6, 7, 9)

// Eq. 9 at time level n: p = p0 (Rd dpi_theta / (p0 dphi))^gamma, as
// p0 exp(gamma log(.)).
template <bool EMU>
__global__ void k_eos(DevMesh m, DyPar d, LevelDiv Dv, const double *__restrict__ th, const double *__restrict__ phi,
                      double *__restrict__ p) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)d.L) return;
    int i, k;
    split_index(n, Dv, i, k);
    const double dphi = phi[(size_t)i * d.ldi + k] - phi[(size_t)i * d.ldi + k + 1];
    p[(size_t)i * d.ld + k] =
        emu<EMU>(d.p0 * exp(d.gamma * log(d.rd * th[(size_t)i * d.ld + k] / (d.p0 * dphi))), d.emu, GRIST_ROW_EOS);
}

// A binary32 advective type takes the differences of the FP64 fields from
// their truncating double-float splits (split_trunc; accurate to about 2^-24
// of the difference before its binary32 rounding) instead of FP64
// subtractions, so the binary32 advection issues no FP64 instruction.
template <typename TA> struct AdvVal;
template <> struct AdvVal<double> {
    double v;
    __device__ __forceinline__ explicit AdvVal(double x) : v(x) {}
};
template <> struct AdvVal<float> {
    float h, l;
    __device__ __forceinline__ explicit AdvVal(double x) { split_trunc(x, h, l); }
};
__device__ __forceinline__ double adv_diff(const AdvVal<double> &a, const AdvVal<double> &b) { return a.v - b.v; }
__device__ __forceinline__ float adv_diff(const AdvVal<float> &a, const AdvVal<float> &b) {
    return diff_df(a.h, a.l, b.h, b.l);
}

// Explicit parts of Eqs. 6-7 at every interface: horizontal advection
// V.grad(x) = (1/A) sum s dv u^int (x_nb - x)/2 and vertical advection
// M (x_{j+1} - x_{j-1}) / (dpi_{j-1} + dpi_j) of w and phi from the stage
// input (advective type; the differences of the FP64 fields are formed to
// about 2^-24 of themselves before the rounding to that type), plus the (1 - beta) share of g (dp/dpi - 1) and g w at t^n.  The
// t^n forcing g (dp/dpi - 1) is formed in the first stage (FIRST) from the
// t^n pressure and kept for the later stages.
template <class P, bool FIRST>
__global__ void k_nh_explicit(DevMesh m, DyPar d, LevelDiv Dv, const typename P::TU *__restrict__ u_s,
                              const double *__restrict__ rdps_s, const double *__restrict__ Mv,
                              const double *__restrict__ w_s, const double *__restrict__ phi_s,
                              const double *__restrict__ w_n, const double *__restrict__ phi_n,
                              const double *__restrict__ p_n, double *__restrict__ fw_n, double *__restrict__ wst,
                              double *__restrict__ phst, double dts) {
    using TA = typename P::TA;
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    const int Li = d.L + 1;
    if (n >= (uint32_t)m.nC * (uint32_t)Li) return;
    int i, j;
    split_index(n, Dv, i, j);
    const size_t xi = (size_t)i * d.ldi + j;
    if (j == d.L) {
        wst[xi] = 0.0;
        phst[xi] = ldg(d.phis + i);
        return;
    }
    const AdvVal<TA> wi(w_s[xi]), pi(phi_s[xi]);
    TA hw = 0, hp = 0;
#pragma unroll
    for (int s = 0; s < GRIST_MAXE; s++) {
        const int e = ldg(m.eoc + i * 6 + s);
        const int nb = ldg(m.coc + i * 6 + s);
        TA ui;
        const size_t ue = (size_t)e * d.ld;
        if (j == 0) ui = cv<TA>(ldg(u_s + ue));
        else ui = (TA)0.5 * (cv<TA>(ldg(u_s + ue + j - 1)) + cv<TA>(ldg(u_s + ue + j)));
        const TA cu = ldg(Coef<TA>::cdiv(m) + i * 6 + s) * ui * (TA)0.5;
        const size_t y = (size_t)nb * d.ldi + j;
        hw += cu * adv_diff(AdvVal<TA>(ldg(w_s + y)), wi);
        hp += cu * adv_diff(AdvVal<TA>(ldg(phi_s + y)), pi);
    }
    TA vw = 0, vp = 0;
    double fw = 0.0;
    if (j > 0) {
        const double rd2 = ldg(d.hrdBi + j) * ldg(rdps_s + i);   // 1/(dpi_{j-1} + dpi_j)
        const TA r = cv<TA>(Mv[(size_t)i * d.ldi + j] * rd2);
        vw = r * adv_diff(AdvVal<TA>(w_s[xi + 1]), AdvVal<TA>(w_s[xi - 1]));
        vp = r * adv_diff(AdvVal<TA>(phi_s[xi + 1]), AdvVal<TA>(phi_s[xi - 1]));
        if (FIRST) {
            // first stage: the stage input is t^n, so rdps_s is 1/(ps^n - pi_top)
            fw = d.g * fma(p_n[(size_t)i * d.ld + j] - p_n[(size_t)i * d.ld + j - 1], 2.0 * rd2, -1.0);
            fw_n[xi] = fw;
        } else {
            fw = fw_n[xi];
        }
    }
    wst[xi] = w_n[xi] + dts * (cv<double>(emu<P::EMU>(-hw - vw, d.emu, GRIST_ROW_NH_ADV)) + (1.0 - d.beta) * fw);
    phst[xi] = phi_n[xi] + dts * (cv<double>(emu<P::EMU>(-hp - vp, d.emu, GRIST_ROW_NH_ADV)) + (1.0 - d.beta) * d.g * w_n[xi]);
}

// Staging of a [32 columns][kSolveKC levels] tile between global memory
// (rows of stride S, one row per column) and shared memory
// sm[level * 33 + column]: each step moves kSolveKC consecutive levels
// (32 bytes, one sector) of 32 / kSolveKC columns, so every global sector
// is used whole; the 33-wide rows keep the shared-memory side free of bank
// conflicts.  Four-level chunks keep a block's shared memory at 6.6 KB so
// that 24 one-warp blocks fit on an SM.
#ifndef GRIST_SOLVE_KC
#define GRIST_SOLVE_KC 4          // levels per staged chunk (1, 2, 4 or 8)
#endif
#ifndef GRIST_SOLVE_MIN_BLOCKS
#define GRIST_SOLVE_MIN_BLOCKS 24 // resident one-warp blocks per SM the registers must allow
#endif
constexpr int kSolveCols = 32;
constexpr int kSolveKC = GRIST_SOLVE_KC;
constexpr int kSolveColsPerStep = 32 / kSolveKC;
constexpr int kRow = 33;
constexpr int kStage = kSolveKC * kRow;
constexpr int kSolveMinBlocks = GRIST_SOLVE_MIN_BLOCKS;
static_assert(kSolveKC == 1 || kSolveKC == 2 || kSolveKC == 4 || kSolveKC == 8, "chunk of 1, 2, 4 or 8 levels");

__device__ __forceinline__ void stage_in(const double *X, size_t S, int col0, int ncol, int k0, int nk, double *sm) {
    const int lane = threadIdx.x & 31, kk = lane % kSolveKC;
#pragma unroll
    for (int it = 0; it < kSolveKC; it++) {
        const int col = it * kSolveColsPerStep + lane / kSolveKC;
        double v = 0.0;
        if (col < ncol && kk < nk) v = X[(size_t)(col0 + col) * S + k0 + kk];
        sm[kk * kRow + col] = v;
    }
}

__device__ __forceinline__ void stage_out(double *X, size_t S, int col0, int ncol, int k0, int nk, const double *sm) {
    const int lane = threadIdx.x & 31, kk = lane % kSolveKC;
#pragma unroll
    for (int it = 0; it < kSolveKC; it++) {
        const int col = it * kSolveColsPerStep + lane / kSolveKC;
        if (col < ncol && kk < nk) X[(size_t)(col0 + col) * S + k0 + kk] = sm[kk * kRow + col];
    }
}

// Implicit part of Eqs. 6-7 and Eq. 9, one thread per column (a block is
// one warp of 32 consecutive columns), FP64.  Column data moves through
// shared memory in kSolveKC-level chunks (whole-sector global access).
// Equation of state relative to the t^n state (1/th_r, phi_r, p_r):
//   p** = p_r ((th dphi_r) / (th_r dphi**))^gamma     (pow1p_near0)
// linearised about phi**: p_k = p**_k - C_k (w_k - w_{k+1}),
// C_k = gamma p**_k beta dt g / dphi**_k; tridiagonal rows for interior
// interfaces j = 1..L-1 (w = 0 at top and ground),
//   -a_j C_{j-1} w_{j-1} + (1 + a_j (C_{j-1} + C_j)) w_j - a_j C_j w_{j+1}
//       = w**_j + a_j (p**_j - p**_{j-1}) - beta dt g,
// a_j = beta dt g / dpi_j at the interface; each row is divided by a_j
// (off-diagonals -C, no product per row) and the system solved by the
// Thomas algorithm; phi = phi** + beta dt g w; the full EOS then gives
//   p = p** (dphi / dphi**)^(-gamma),  dphi = dphi** + beta dt g (w_k - w_{k+1});
// finally alpha = dphi/dpi, layer phi and dp/dpi averaged to layers
// (interface value 1 at top and bottom) for the momentum equation.  phi_out
// may be phi_r and p may be p_r (the last stage writes the state in place):
// each block reads all reference values of its columns before writing them.
template <bool EMU, bool DF>
__global__ void __launch_bounds__(32, kSolveMinBlocks) k_nh_solve(DevMesh m, DyPar d, const double *__restrict__ wst,
                                                 const double *__restrict__ phst, const double *__restrict__ th,
                                                 const double *__restrict__ rth_r, const double *phi_r,
                                                 const double *p_r, const double *__restrict__ ps, double dts,
                                                 double *w_out, double *phi_out, double *p, double *__restrict__ al,
                                                 double *__restrict__ phl, double *__restrict__ dpp, Binom bg_pos,
                                                 Binom bg_neg) {
    __shared__ double sA[6 * kStage + kRow];
    const int lane = threadIdx.x;
    const int col0 = blockIdx.x * kSolveCols;
    const int ncol = min(kSolveCols, m.nC - col0);
    const int i = col0 + lane;
    const bool act = lane < ncol;
    const int L = d.L;
    const double bg = d.beta * dts * d.g;
    const double gbg = d.gamma * bg;
    const double dps = act ? ps[i] - d.pi_top : 1.0;
    const double rdps = rcp(dps);
    const double psg = dps * rcp(bg);   // 1/a_j = dBi_j psg
    const unsigned amask = __ballot_sync(0xffffffffu, act);
    double cp[kNHMax], dd[kNHMax], pst[kNHMax], rdf[kNHMax];
    double ftop = act ? phst[(size_t)i * d.ldi] : 0.0, rtop = act ? phi_r[(size_t)i * d.ldi] : 0.0;
    const double phi_top0 = ftop;
    double pst_prev = 0.0, C_prev = 0.0;
    // forward sweep
    for (int k0 = 0; k0 < L; k0 += kSolveKC) {
        const int nk = min(kSolveKC, L - k0);
        __syncwarp();
        stage_in(phst, d.ldi, col0, ncol, k0 + 1, nk, sA + 0 * kStage);
        stage_in(phi_r, d.ldi, col0, ncol, k0 + 1, nk, sA + 1 * kStage);
        stage_in(th, d.ld, col0, ncol, k0, nk, sA + 2 * kStage);
        stage_in(rth_r, d.ld, col0, ncol, k0, nk, sA + 3 * kStage);
        stage_in(p_r, d.ld, col0, ncol, k0, nk, sA + 4 * kStage);
        stage_in(wst, d.ldi, col0, ncol, k0, nk, sA + 5 * kStage);
        __syncwarp();
        if (act) {
            for (int kk = 0; kk < nk; kk++) {
                const int j = k0 + kk;
                const int o = kk * kRow + lane;
                const double fbot = sA[0 * kStage + o], rbot = sA[1 * kStage + o];
                const double rdfj = rcp_nr(ftop - fbot);
                // x = th dphi_r / (th_r dphi**) - 1, the ratio's offset from 1
                const double x = fma(sA[2 * kStage + o] * sA[3 * kStage + o], (rtop - rbot) * rdfj, -1.0);
                const double pstj = DF ? scale_near1_df(sA[4 * kStage + o], x, d.gamma, bg_pos)
                                       : sA[4 * kStage + o] * pow1p_near0(x, d.gamma, bg_pos, amask);
                pst[j] = pstj;
                rdf[j] = rdfj;
                const double C = gbg * pstj * rdfj;
                if (j >= 1) {
                    // row j / a_j: -C_{j-1} w_{j-1} + (1/a_j + C_{j-1} + C_j) w_j - C_j w_{j+1}
                    //            = (w**_j - beta dt g)/a_j + p**_j - p**_{j-1}
                    // (no w_{j+1} term in the last row: w_L = 0)
                    const double sj = ldg(d.dBi + j) * psg;
                    const double b = sj + (C_prev + C);
                    const double rhs = fma(sA[5 * kStage + o] - bg, sj, pstj - pst_prev);
                    const double cq = (j == L - 1) ? 0.0 : C;
                    const int r = j - 1;
                    if (r == 0) {
                        const double rb = rcp_nr(b);
                        cp[0] = -cq * rb;
                        dd[0] = rhs * rb;
                    } else {
                        const double rden = rcp_nr(fma(C_prev, cp[r - 1], b));
                        cp[r] = -cq * rden;
                        dd[r] = fma(C_prev, dd[r - 1], rhs) * rden;
                    }
                }
                pst_prev = pstj;
                C_prev = C;
                ftop = fbot;
                rtop = rbot;
            }
        }
    }
    // back substitution, bottom to top, w written chunk by chunk
    // (interfaces 0..L; w = 0 at 0 and L)
    double wn = 0.0;
    for (int k0 = (L / kSolveKC) * kSolveKC; k0 >= 0; k0 -= kSolveKC) {
        const int nk = min(kSolveKC, L + 1 - k0);
        __syncwarp();
        for (int kk = nk - 1; kk >= 0; kk--) {
            const int jf = k0 + kk;
            double wv = 0.0;
            if (act && jf >= 1 && jf <= L - 1) {
                wn = fma(-cp[jf - 1], wn, dd[jf - 1]);
                wv = wn;
            }
            sA[kk * kRow + lane] = wv;
        }
        __syncwarp();
        stage_out(w_out, d.ldi, col0, ncol, k0, nk, sA);
    }
    // phi, EOS and momentum diagnostics, top to bottom
    if (act) phi_out[(size_t)i * d.ldi] = phi_top0;
    // halves of dp/dpi at the interfaces (1 at top and ground), so that the
    // layer mean is one addition
    double phi_top = phi_top0, htop = 0.5, pprev = 0.0;
    for (int k0 = 0; k0 < L; k0 += kSolveKC) {
        const int nk = min(kSolveKC, L - k0);
        __syncwarp();
        stage_in(phst, d.ldi, col0, ncol, k0 + 1, nk, sA + 0 * kStage);
        stage_in(w_out, d.ldi, col0, ncol, k0, nk, sA + 1 * kStage);   // w at interfaces k0..k0+nk-1
        if (lane < ncol) sA[6 * kStage + lane] = w_out[(size_t)i * d.ldi + k0 + nk];   // interface k0+nk
        __syncwarp();
        if (act) {
            for (int kk = 0; kk < nk; kk++) {
                const int k = k0 + kk;
                const int o = kk * kRow + lane;
                const double w_top = sA[1 * kStage + o];
                const double w_bot = (kk + 1 < nk) ? sA[1 * kStage + o + kRow] : sA[6 * kStage + lane];
                const double phi_bot = (k + 1 < L) ? fma(bg, w_bot, sA[o]) : ldg(d.phis + i);
                const double xk = bg * (w_top - w_bot) * rdf[k];
                const double pk = DF ? scale_near1_df(pst[k], xk, -d.gamma, bg_neg)
                                     : pst[k] * pow1p_near0(xk, -d.gamma, bg_neg, amask);
                double hcur = 0.5;
                if (k > 0) {
                    hcur = (pk - pprev) * (ldg(d.hrdBi + k) * rdps);
                    const double dv = htop + hcur;
                    if (kk > 0) sA[5 * kStage + o - kRow] = emu<EMU>(dv, d.emu, GRIST_ROW_EOS);   // layer k-1 of this chunk
                    else dpp[(size_t)i * d.ld + k - 1] = emu<EMU>(dv, d.emu, GRIST_ROW_EOS);        // of the previous chunk
                }
                sA[2 * kStage + o] = emu<EMU>(pk, d.emu, GRIST_ROW_EOS);
                const double dphi = phi_top - phi_bot;
                sA[3 * kStage + o] = emu<EMU>(dphi * (ldg(d.rdB + k) * rdps), d.emu, GRIST_ROW_EOS);
                const double phm = fma(0.5, dphi, phi_bot);   // layer mean (phi_top + phi_bot)/2
                sA[4 * kStage + o] = DF ? pack_split(phm) : emu<EMU>(phm, d.emu, GRIST_ROW_EOS);
                sA[1 * kStage + o] = phi_bot;   // w_top of this row is no longer needed
                htop = hcur;
                pprev = pk;
                phi_top = phi_bot;
            }
        }
        __syncwarp();
        stage_out(phi_out, d.ldi, col0, ncol, k0 + 1, nk, sA + 1 * kStage);
        stage_out(p, d.ld, col0, ncol, k0, nk, sA + 2 * kStage);
        stage_out(al, d.ld, col0, ncol, k0, nk, sA + 3 * kStage);
        stage_out(phl, d.ld, col0, ncol, k0, nk, sA + 4 * kStage);
        stage_out(dpp, d.ld, col0, ncol, k0, nk - 1, sA + 5 * kStage);
    }
    if (act) dpp[(size_t)i * d.ld + L - 1] = emu<EMU>(htop + 0.5, d.emu, GRIST_ROW_EOS);
}

// Relative vorticity at the vertices (diagnostic): zeta_v = sum_j ccurl u,
// ccurl = t(e,v) dc_e / A_v, in FP64.
template <typename TU>
__global__ void k_diag_vort(DevMesh m, int L, int ld, LevelDiv Dv, const TU *__restrict__ u, double *__restrict__ vor) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nV * (uint32_t)L) return;
    int v, k;
    split_index(n, Dv, v, k);
    double z = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++) z += ldg(m.ccurl + v * 3 + j) * (double)ldg(u + (size_t)ldg(m.eov + v * 3 + j) * ld + k);
    vor[(size_t)v * ld + k] = z;
}

__global__ void k_add_scalar(double *x, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *x += v;
}

template <class P, bool NH>
int dycore_step(grist_mesh_s *h, grist_dycore_state *S, const grist_dycore_params *prm, double dt, cudaStream_t st) {
    using TU = typename P::TU;
    using TA = typename P::TA;
    using TM = typename P::TM;
    const DevMesh &m = dev_mesh(h);
    const int L = prm->n_levels, ld = prm->ld, ldi = prm->ld_int;
    const size_t nCL = (size_t)m.nC * ld, nEL = (size_t)m.nE * ld, nVL = (size_t)m.nV * ld, nCI = (size_t)m.nC * ldi;

    // scratch layout
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += al(bytes); return o; };
    const size_t nvg = 5 * (size_t)L + 3 + ((size_t)L + 1) / 2;   // doubles, then L floats
    const size_t o_vg = take(sizeof(double) * nvg);
    const size_t o_uA = take(nEL * sizeof(TU)), o_uB = take(nEL * sizeof(TU));
    const size_t o_psA = take(m.nC * 8), o_psB = take(m.nC * 8), o_psN = take(m.nC * 8);
    const size_t o_rdps = take(m.nC * 8), o_rsum = take(m.nE * 8), o_rdpv = take(m.nV * 8),
                 o_fcol = take(m.nE * 8);
    const size_t o_thA = take(nCL * 8), o_thB = take(nCL * 8);
    const size_t o_F = take(nEL * sizeof(TM)), o_M = take(nCI * 8);
    const size_t o_theta = take(nCL * sizeof(TA)), o_Fth = take(nEL * sizeof(TA));
    const size_t o_p = take(nCL * 8), o_al = take(nCL * 8), o_phl = take(nCL * 8), o_dpp = take(nCL * 8);
    const size_t o_qv = take(nVL * sizeof(TA)), o_K = take(nCL * 8);
    size_t o_wA = 0, o_wB = 0, o_phA = 0, o_phB = 0, o_wst = 0, o_phst = 0, o_pn = 0, o_fw = 0, o_rth = 0;
    if (NH) {
        o_wA = take(nCI * 8); o_wB = take(nCI * 8); o_phA = take(nCI * 8); o_phB = take(nCI * 8);
        o_wst = take(nCI * 8); o_phst = take(nCI * 8); o_pn = take(nCL * 8); o_fw = take(nCI * 8);
        o_rth = take(nCL * 8);
    }
    char *s = (char *)scratch(h, 1, off);
    if (!s) return GRIST_ENOMEM;

    // vertical grid: B (L+1) | dB (L) | 1/dB (L) | 1/(dB[j-1]+dB[j]) (L+1) | (dB[j-1]+dB[j])/2 (L+1)
    std::vector<double> vg(nvg, 0.0);
    double *hB = vg.data(), *hdB = hB + L + 1, *hrdB = hdB + L, *hhrdBi = hrdB + L, *hdBi = hhrdBi + L + 1;
    for (int k = 0; k <= L; k++) hB[k] = prm->b_interface[k];
    for (int k = 0; k < L; k++) {
        hdB[k] = prm->b_interface[k + 1] - prm->b_interface[k];
        hrdB[k] = 1.0 / hdB[k];
    }
    for (int j = 1; j < L; j++) {
        hhrdBi[j] = 1.0 / (hdB[j - 1] + hdB[j]);
        hdBi[j] = 0.5 * (hdB[j - 1] + hdB[j]);
    }
    float *hdBf = reinterpret_cast<float *>(hdBi + L + 1);
    for (int k = 0; k < L; k++) hdBf[k] = (float)hdB[k];
    double *dvg = (double *)(s + o_vg);
    if (vg_ptr(h) != dvg || vg_cache(h) != vg) {
        // ordered after this stream's earlier steps, which read the old table
        GRIST_CUDA_TRY(cudaMemcpyAsync(dvg, vg.data(), vg.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        GRIST_CUDA_TRY(cudaStreamSynchronize(st));  // vg is a host temporary
        vg_cache(h) = vg;
        vg_ptr(h) = dvg;
    }

    DyPar d;
    d.L = L; d.ld = ld; d.ldi = ldi;
    d.pi_top = prm->pi_top; d.p0 = prm->p0; d.rd = prm->rd; d.cp = prm->cp; d.g = prm->g;
    d.beta = prm->offcentre_beta; d.kappa = prm->rd / prm->cp; d.gamma = prm->cp / (prm->cp - prm->rd);
    d.B = dvg; d.dB = dvg + L + 1; d.rdB = dvg + 2 * L + 1; d.hrdBi = dvg + 3 * L + 1; d.dBi = dvg + 4 * L + 2;
    d.phis = prm->phi_surface;
    d.dBf = reinterpret_cast<const float *>(dvg + 5 * L + 3);
    d.emu = prm->emulate_fp32_rows;

    TU *uA = (TU *)(s + o_uA), *uB = (TU *)(s + o_uB);
    double *psA = (double *)(s + o_psA), *psB = (double *)(s + o_psB), *psN = (double *)(s + o_psN);
    double *rdps = (double *)(s + o_rdps), *rsum = (double *)(s + o_rsum), *rdpv = (double *)(s + o_rdpv),
           *fcol = (double *)(s + o_fcol);
    double *thA = (double *)(s + o_thA), *thB = (double *)(s + o_thB);
    TM *F = (TM *)(s + o_F);
    double *Mv = (double *)(s + o_M);
    TA *theta = (TA *)(s + o_theta), *Fth = (TA *)(s + o_Fth);
    double *p = (double *)(s + o_p), *alp = (double *)(s + o_al), *phl = (double *)(s + o_phl),
           *dpp = (double *)(s + o_dpp);
    TA *qv = (TA *)(s + o_qv);
    double *K = (double *)(s + o_K);
    double *wA = (double *)(s + o_wA), *wB = (double *)(s + o_wB), *phA = (double *)(s + o_phA),
           *phB = (double *)(s + o_phB), *wst = (double *)(s + o_wst), *phst = (double *)(s + o_phst),
           *pn = (double *)(s + o_pn), *fwn = (double *)(s + o_fw), *rthn = (double *)(s + o_rth);

    TU *u = (TU *)S->u;
    uint32_t *status = status_word(h);
    const LevelDiv DL = make_div((uint32_t)L), DI = make_div((uint32_t)(L + 1)), DH = make_div((uint32_t)(L + 1) / 2);
    const unsigned gC = grid_for((long long)m.nC * L, kBlock), gE = grid_for((long long)m.nE * L, kBlock),
                   gV = grid_for((long long)m.nV * L, kBlock), gW = grid_for((long long)m.nC * 32, kBlock),
                   gI = grid_for((long long)m.nC * (L + 1), kBlock), gSolve = grid_for(m.nC, kSolveCols),
                   gVx = grid_for(m.nV, kBlock), gE32 = grid_for((long long)m.nE + 31, kBlock),
                   gC32 = grid_for((long long)m.nC + 31, kBlock), gEH = grid_for((long long)m.nE * DH.d, kBlock),
                   gCH = grid_for((long long)m.nC * DH.d, kBlock), gVH = grid_for((long long)m.nV * DH.d, kBlock);
    const double dts[3] = {dt / 3.0, dt / 2.0, dt};
    const double ascale = S->accum_scale != 0.0 ? S->accum_scale : 1.0;

    GRIST_CUDA_TRY(cudaMemcpyAsync(psN, S->ps, m.nC * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // t^n pressure: carried in the state when valid, else from the EOS
    const double *p_n = pn;
    if (NH) {
        if (S->p_nh && S->p_nh_valid) {
            p_n = S->p_nh;
        } else {
            double *dst = S->p_nh ? S->p_nh : pn;
            GRIST_LAUNCH(h, PN("k_eos"), st, k_eos<P::EMU><<<gC, kBlock, 0, st>>>(m, d, DL, S->dpi_theta, S->phi, dst));
            p_n = dst;
        }
    }
    const Binom bpos = binomial(d.gamma), bneg = binomial(-d.gamma);

    double *p_outs[3] = {p, p, (NH && S->p_nh) ? S->p_nh : p};

    const TU *u_in = u;
    const double *ps_in = psN, *th_in = S->dpi_theta, *w_in = S->w, *phi_in = S->phi;
    TU *u_outs[3] = {uA, uB, u};
    double *ps_outs[3] = {psA, psB, S->ps};
    double *th_outs[3] = {thA, thB, S->dpi_theta};
    double *w_outs[3] = {wA, wB, S->w};
    double *phi_outs[3] = {phA, phB, S->phi};
    for (int s3 = 0; s3 < 3; s3++) {
        const double h3 = dts[s3];
        GRIST_LAUNCH(h, PN("k_mass_edge"), st, k_mass_edge<P><<<gE32, kBlock, 0, st>>>(
            m, d, ps_in, u_in, F, s3 == 2 ? S->mass_flux_accum : nullptr, ascale, rsum, fcol));
        GRIST_LAUNCH(h, PN("k_mass_col"), st, k_mass_col<P><<<gC32, kBlock, 0, st>>>(
            m, d, F, fcol, ps_in, psN, ps_outs[s3], th_in, theta, Mv, h3, s3 == 0 ? S->dpi_start : nullptr, rdps,
            (NH && s3 == 0) ? rthn : nullptr, s3 == 2 ? S->vmass_flux_accum : nullptr, ascale));
        GRIST_LAUNCH(h, PN("k_theta_flux"), st, k_theta_flux<P><<<gEH, kBlock, 0, st>>>(m, d, DH, F, theta, Fth));
        GRIST_LAUNCH(h, PN("k_theta_update"), st, k_theta_update<P><<<gCH, kBlock, 0, st>>>(
            m, d, DH, Fth, theta, Mv, S->dpi_theta, th_outs[s3], h3));
        if (NH) {
            if (s3 == 0)
                GRIST_LAUNCH(h, PN("k_nh_explicit"), st, k_nh_explicit<P, true><<<gI, kBlock, 0, st>>>(
                    m, d, DI, u_in, rdps, Mv, w_in, phi_in, S->w, S->phi, p_n, fwn, wst, phst, h3));
            else
                GRIST_LAUNCH(h, PN("k_nh_explicit"), st, k_nh_explicit<P, false><<<gI, kBlock, 0, st>>>(
                    m, d, DI, u_in, rdps, Mv, w_in, phi_in, S->w, S->phi, p_n, fwn, wst, phst, h3));
            GRIST_LAUNCH(h, PN("k_nh_solve"), st, k_nh_solve<P::EMU, P::DF><<<gSolve, kSolveCols, 0, st>>>(
                m, d, wst, phst, th_outs[s3], rthn, S->phi, p_n, ps_outs[s3], h3, w_outs[s3],
                phi_outs[s3], p_outs[s3], alp, phl, dpp, bpos, bneg));
        } else {
            GRIST_LAUNCH(h, PN("k_hydro_diag"), st, k_hydro_diag<P::EMU, P::DF><<<gW, kBlock, 0, st>>>(
                m, d, ps_outs[s3], th_outs[s3], p, alp, phl));
        }
        GRIST_LAUNCH(h, PN("k_vertex_mass"), st, k_vertex_mass<P::EMU><<<gVx, kBlock, 0, st>>>(m, d, ps_in, rdpv));
        GRIST_LAUNCH(h, PN("k_vort"), st, k_vort<P><<<gVH, kBlock, 0, st>>>(m, d, DH, u_in, rdpv, qv));
        GRIST_LAUNCH(h, PN("k_ke"), st, k_ke<P><<<gC, kBlock, 0, st>>>(m, d, DL, u_in, K));
        GRIST_LAUNCH(h, PN("k_momentum"), st, k_momentum<P, NH><<<gE, kBlock, 0, st>>>(
            m, d, DL, u_in, u, u_outs[s3], F, qv, K, Mv, rsum, p_outs[s3], alp, phl, dpp, h3, status));
        u_in = u_outs[s3];
        ps_in = ps_outs[s3];
        th_in = th_outs[s3];
        w_in = w_outs[s3];
        phi_in = phi_outs[s3];
    }
    if (S->accum_weight) GRIST_LAUNCH(h, PN("k_add_scalar"), st, k_add_scalar<<<1, 32, 0, st>>>(S->accum_weight, ascale));
    if (cudaGetLastError() != cudaSuccess) return GRIST_ECUDA;
    if (NH && S->p_nh) S->p_nh_valid = 1;
    return GRIST_OK;
}

int check(grist_mesh h, grist_dycore_state *S, const grist_dycore_params *prm, grist_precision prec, double dt,
          bool nh) {
    if (!h || !S || !prm) return GRIST_EINVAL;
    if (!(dt > 0) || !std::isfinite(dt)) return GRIST_EINVAL;
    if (prec != GRIST_FP64 && prec != GRIST_MIX && prec != GRIST_MIX_DBL_MASS && prec != GRIST_MIX_DF)
        return GRIST_EINVAL;
    const int L = prm->n_levels;
    if (L < 2 || L > GRIST_MAXL || prm->ld < L || prm->ld_int < L + 1) return GRIST_EINVAL;
    if (nh && L > kNHMax) return GRIST_EUNSUPPORTED;
    if (!S->u || !S->ps || !S->dpi_theta || !prm->b_interface || !prm->phi_surface) return GRIST_EINVAL;
    if (nh && (!S->w || !S->phi)) return GRIST_EINVAL;
    if (prm->b_interface[0] != 0.0 || prm->b_interface[L] != 1.0) return GRIST_EINVAL;
    for (int k = 0; k < L; k++)
        if (!(prm->b_interface[k + 1] > prm->b_interface[k])) return GRIST_EINVAL;
    if (!(prm->pi_top >= 0) || !(prm->p0 > 0) || !(prm->rd > 0) || !(prm->cp > prm->rd) || !(prm->g > 0))
        return GRIST_EINVAL;
    if (nh && !(prm->offcentre_beta > 0 && prm->offcentre_beta <= 1)) return GRIST_EINVAL;
    if (!std::isfinite(S->accum_scale) || S->accum_scale < 0) return GRIST_EINVAL;
    if (prm->emulate_fp32_rows & ~GRIST_ROW_ALL) return GRIST_EINVAL;
    return GRIST_OK;
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_dycore_step_hydro(grist_mesh h, grist_dycore_state *S, const grist_dycore_params *prm,
                                       grist_precision prec, double dt, void *stream) {
    int rc = check(h, S, prm, prec, dt, false);
    if (rc != GRIST_OK) return rc;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (prm->emulate_fp32_rows) {
        if (prec != GRIST_FP64) return GRIST_EUNSUPPORTED;
        return dycore_step<PolFP64EMU, false>(h, S, prm, dt, st);
    }
    switch (prec) {
        case GRIST_FP64: return dycore_step<PolFP64, false>(h, S, prm, dt, st);
        case GRIST_MIX: return dycore_step<PolMIX, false>(h, S, prm, dt, st);
        case GRIST_MIX_DF: return dycore_step<PolMIXDF, false>(h, S, prm, dt, st);
        default: return dycore_step<PolMIXDBL, false>(h, S, prm, dt, st);
    }
}

extern "C" int grist_dycore_step_nh(grist_mesh h, grist_dycore_state *S, const grist_dycore_params *prm,
                                    grist_precision prec, double dt, void *stream) {
    int rc = check(h, S, prm, prec, dt, true);
    if (rc != GRIST_OK) return rc;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (prm->emulate_fp32_rows) {
        if (prec != GRIST_FP64) return GRIST_EUNSUPPORTED;
        return dycore_step<PolFP64EMU, true>(h, S, prm, dt, st);
    }
    switch (prec) {
        case GRIST_FP64: return dycore_step<PolFP64, true>(h, S, prm, dt, st);
        case GRIST_MIX: return dycore_step<PolMIX, true>(h, S, prm, dt, st);
        case GRIST_MIX_DF: return dycore_step<PolMIXDF, true>(h, S, prm, dt, st);
        default: return dycore_step<PolMIXDBL, true>(h, S, prm, dt, st);
    }
}

extern "C" int grist_diag_vorticity(grist_mesh h, const void *u, grist_precision prec, int32_t n_levels, int32_t ld,
                                    double *vor, void *stream) {
    if (!h || !u || !vor || n_levels < 1 || n_levels > GRIST_MAXL || ld < n_levels) return GRIST_EINVAL;
    if (prec != GRIST_FP64 && prec != GRIST_MIX && prec != GRIST_MIX_DBL_MASS && prec != GRIST_MIX_DF)
        return GRIST_EINVAL;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    const DevMesh &m = dev_mesh(h);
    cudaStream_t st = (cudaStream_t)stream;
    const LevelDiv Dv = make_div((uint32_t)n_levels);
    const unsigned grid = grid_for((long long)m.nV * n_levels, kBlock);
    if (prec == GRIST_FP64)
        k_diag_vort<double><<<grid, kBlock, 0, st>>>(m, n_levels, ld, Dv, (const double *)u, vor);
    else
        k_diag_vort<float><<<grid, kBlock, 0, st>>>(m, n_levels, ld, Dv, (const float *)u, vor);
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}
