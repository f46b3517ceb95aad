// tracer.cu - tracer transport, Eq. 10 (horizontal part), Sec. 2.1:
// third-order upwind edge flux, Wicker-Skamarock RK3, Zalesak FCT on the
// final stage; FP64 or single-precision tracers (Sec. 2.3) with an FP64
// mass flux and FP64 layer mass.
//
// Data layout: q [T][nC][ld], dpi [nC][ld], mass flux [nE][ld], edge
// fluxes [T][nE][ld]; one thread per (entity, level) with the level index
// innermost, so a warp reads consecutive levels of neighbouring entities
// (coalesced), and a thread loops over the member's tracers so the
// per-(entity, level) geometry and mass-flux loads are shared by all of
// them.
#include <cmath>

#include "common.cuh"

#define PN(n) (sizeof(TC) == 4 ? n "/mix" : n "/fp64")

namespace grist {
namespace {

constexpr int kBlock = 256;

// Cell divergence of the (time-mean) mass flux, FP64: the tracer solver's
// own continuity, dpi^(s) = dpi^n - dt_s divF.
__global__ void k_div_mass(DevMesh m, int L, int ld, LevelDiv D, const double *__restrict__ F,
                           double *__restrict__ divF) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)L) return;
    int i, k;
    split_index(n, D, i, k);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++)
        s += ldg(m.cdiv + i * 6 + j) * ldg(F + (size_t)ldg(m.eoc + i * 6 + j) * ld + k);
    divF[(size_t)i * ld + k] = s;
}

// Third-order upwind edge flux (Skamarock-Gassmann form):
//   q_e = (q1 + q2)/2 - (dc^2/12)(q''1 + q''2) + sgn(F) beta (dc^2/12)(q''2 - q''1)
//   F^H = F q_e
// With beta = 1 only the upwind side's second derivative survives:
//   q_e = (q1 + q2)/2 - 2 (dc^2/12) q''_upwind.
template <typename TQ, typename TC, bool BETA1>
__global__ void k_edge_flux(DevMesh m, int T, int L, int ld, LevelDiv D, const TQ *__restrict__ q, size_t qs,
                            const double *__restrict__ F, TC beta, TC *__restrict__ FH, size_t fs) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nE * (uint32_t)L) return;
    int e, k;
    split_index(n, D, e, k);
    const int2 c = ldg(m.coe + e);
    const TC f = (TC)ldg(F + (size_t)e * ld + k);
    const TC dc2 = ldg(Coef<TC>::dc2(m) + e);
    const int32_t *st = m.d2i + (size_t)e * 14;
    const TC *cf = Coef<TC>::d2c(m) + (size_t)e * 14;
    if (BETA1) {
        const int side = f >= (TC)0 ? 0 : 1;
        int idx[GRIST_D2P];
        TC w[GRIST_D2P];
#pragma unroll
        for (int j = 0; j < GRIST_D2P; j++) {
            idx[j] = ldg(st + side * GRIST_D2P + j);
            w[j] = ldg(cf + side * GRIST_D2P + j);
        }
        for (int t = 0; t < T; t++) {
            const TQ *qt = q + (size_t)t * qs;
            TC d = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) d += w[j] * (TC)ldg(qt + (size_t)idx[j] * ld + k);
            TC q1 = (TC)ldg(qt + (size_t)c.x * ld + k), q2 = (TC)ldg(qt + (size_t)c.y * ld + k);
            TC qe = (TC)0.5 * (q1 + q2) - (TC)2 * dc2 * d;
            FH[(size_t)t * fs + (size_t)e * ld + k] = f * qe;
        }
    } else {
        const TC sgn = f >= (TC)0 ? (TC)1 : (TC)-1;
        for (int t = 0; t < T; t++) {
            const TQ *qt = q + (size_t)t * qs;
            TC d1 = 0, d2 = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) {
                d1 += ldg(cf + j) * (TC)ldg(qt + (size_t)ldg(st + j) * ld + k);
                d2 += ldg(cf + GRIST_D2P + j) * (TC)ldg(qt + (size_t)ldg(st + GRIST_D2P + j) * ld + k);
            }
            TC q1 = (TC)ldg(qt + (size_t)c.x * ld + k), q2 = (TC)ldg(qt + (size_t)c.y * ld + k);
            TC qe = (TC)0.5 * (q1 + q2) - dc2 * (d1 + d2) + sgn * beta * dc2 * (d2 - d1);
            FH[(size_t)t * fs + (size_t)e * ld + k] = f * qe;
        }
    }
}

// RK stage update: q^(s) = (dpi^n q^n - dt_s div F^H) / dpi^(s),
// written as r1 q^n - r2 div with r1 = dpi^n/dpi^(s), r2 = dt_s/dpi^(s)
// taken once per (cell, level) in FP64 and rounded to the tracer type
// (Sec. 2.2 (ii): no mixed-kind products inside the tracer loop).
template <typename TQ, typename TC>
__global__ void k_stage_update(DevMesh m, int T, int L, int ld, LevelDiv D, const TQ *__restrict__ qn, TQ *qout,
                               size_t qs, const TC *__restrict__ FH, size_t fs, const double *__restrict__ dpi,
                               const double *__restrict__ divF, double dts, uint32_t *status) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)L) return;
    int i, k;
    split_index(n, D, i, k);
    const size_t x = (size_t)i * ld + k;
    const double dp = dpi[x];
    const double rinv = 1.0 / (dp - dts * divF[x]);
    const TC r1 = (TC)(dp * rinv), r2 = (TC)(dts * rinv);
    int eidx[GRIST_MAXE];
    TC cw[GRIST_MAXE];
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        eidx[j] = ldg(m.eoc + i * 6 + j);
        cw[j] = ldg(Coef<TC>::cdiv(m) + i * 6 + j);
    }
    bool bad = false;
    for (int t = 0; t < T; t++) {
        const TC *ft = FH + (size_t)t * fs;
        TC div = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) div += cw[j] * ldg(ft + (size_t)eidx[j] * ld + k);
        TC v = r1 * (TC)qn[(size_t)t * qs + x] - r2 * div;
        bad |= !isfinite(v);
        qout[(size_t)t * qs + x] = (TQ)v;
    }
    if (bad) atomicOr(status, GRIST_FLAG_NONFINITE);
}

// Low-order (first-order upwind) flux of edge j of cell i from q^n.
// The upwind cell of an edge is c1 when F >= 0, c2 otherwise; cell i is c1
// of its edge exactly when the divergence coefficient is positive.
template <typename TQ, typename TC>
__device__ __forceinline__ TC upwind_flux(TC f, TC cw, int i, int nb, const TQ *qt, int ld, int k) {
    const bool i_is_c1 = cw > (TC)0;
    const int up = ((f >= (TC)0) == i_is_c1) ? i : nb;
    return f * (TC)ldg(qt + (size_t)up * ld + k);
}

// FCT step 1: low-order solution q^td = (dpi^n q^n - dt div F^L) / dpi^(3).
template <typename TQ, typename TC>
__global__ void k_fct_lowres(DevMesh m, int T, int L, int ld, LevelDiv D, const TQ *__restrict__ qn, size_t qs,
                             const double *__restrict__ F, const double *__restrict__ dpi,
                             const double *__restrict__ divF, double dt, TQ *__restrict__ qtd) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)L) return;
    int i, k;
    split_index(n, D, i, k);
    const size_t x = (size_t)i * ld + k;
    const double dp = dpi[x];
    const double rinv = 1.0 / (dp - dt * divF[x]);
    const TC r1 = (TC)(dp * rinv), r2 = (TC)(dt * rinv);
    int nb[GRIST_MAXE];
    TC cw[GRIST_MAXE], fe[GRIST_MAXE];
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        int e = ldg(m.eoc + i * 6 + j);
        nb[j] = ldg(m.coc + i * 6 + j);
        cw[j] = ldg(Coef<TC>::cdiv(m) + i * 6 + j);
        fe[j] = (TC)ldg(F + (size_t)e * ld + k);
    }
    for (int t = 0; t < T; t++) {
        const TQ *qt = qn + (size_t)t * qs;
        TC div = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) div += cw[j] * upwind_flux<TQ, TC>(fe[j], cw[j], i, nb[j], qt, ld, k);
        qtd[(size_t)t * qs + x] = (TQ)(r1 * (TC)qt[x] - r2 * div);
    }
}

// FCT step 2: local bounds over the cell and its neighbours of {q^n, q^td};
// antidiffusive in/out sums P+-, allowed changes Q+-, ratios
// R+- = min(1, Q / (P + TINY)) (Sec. 2.2 (iii): TINY of the working type).
template <typename TQ, typename TC>
__global__ void k_fct_ratios(DevMesh m, int T, int L, int ld, LevelDiv D, const TQ *__restrict__ qn,
                             const TQ *__restrict__ qtd, size_t qs, const TC *__restrict__ FH, size_t fs,
                             const double *__restrict__ F, const double *__restrict__ dpi,
                             const double *__restrict__ divF, double dt, TC *__restrict__ Rp,
                             TC *__restrict__ Rm) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)L) return;
    int i, k;
    split_index(n, D, i, k);
    const size_t x = (size_t)i * ld + k;
    const TC dp3 = (TC)(dpi[x] - dt * divF[x]);
    const TC dtc = (TC)dt;
    int nb[GRIST_MAXE], eidx[GRIST_MAXE];
    TC cw[GRIST_MAXE], fe[GRIST_MAXE];
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        eidx[j] = ldg(m.eoc + i * 6 + j);
        nb[j] = ldg(m.coc + i * 6 + j);
        cw[j] = ldg(Coef<TC>::cdiv(m) + i * 6 + j);
        fe[j] = (TC)ldg(F + (size_t)eidx[j] * ld + k);
    }
    for (int t = 0; t < T; t++) {
        const TQ *qt = qn + (size_t)t * qs;
        const TQ *qd = qtd + (size_t)t * qs;
        const TC *ft = FH + (size_t)t * fs;
        TC qtd_i = (TC)qd[x];
        TC qmax = fmax_((TC)qt[x], qtd_i), qmin = fmin_((TC)qt[x], qtd_i);
        TC pp = 0, pm = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            size_t y = (size_t)nb[j] * ld + k;
            TC a = (TC)ldg(qt + y), b = (TC)ldg(qd + y);
            qmax = fmax_(qmax, fmax_(a, b));
            qmin = fmin_(qmin, fmin_(a, b));
            TC ae = ldg(ft + (size_t)eidx[j] * ld + k) - upwind_flux<TQ, TC>(fe[j], cw[j], i, nb[j], qt, ld, k);
            TC out = cw[j] * ae;  // outward antidiffusive flux / A_i (sign and dv folded in)
            pp += fmax_((TC)0, -out);
            pm += fmax_((TC)0, out);
        }
        pp *= dtc;
        pm *= dtc;
        TC Qp = (qmax - qtd_i) * dp3, Qm = (qtd_i - qmin) * dp3;
        Rp[(size_t)t * qs + x] = fmin_((TC)1, Qp / (pp + Coef<TC>::tiny()));
        Rm[(size_t)t * qs + x] = fmin_((TC)1, Qm / (pm + Coef<TC>::tiny()));
    }
}

// FCT step 3: limited flux F^L + C A with C = min(R-(c1), R+(c2)) when the
// antidiffusive flux A runs c1 -> c2 (A >= 0), min(R+(c1), R-(c2)) else;
// final update q^{n+1} = (dpi^n q^n - dt div(F^L + C A)) / dpi^(3).
template <typename TQ, typename TC>
__global__ void k_fct_final(DevMesh m, int T, int L, int ld, LevelDiv D, const TQ *__restrict__ qn,
                            TQ *__restrict__ qout, size_t qs, const TC *__restrict__ FH, size_t fs,
                            const double *__restrict__ F, const double *__restrict__ dpi,
                            const double *__restrict__ divF, double dt, const TC *__restrict__ Rp,
                            const TC *__restrict__ Rm, uint32_t *status) {
    uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (uint32_t)m.nC * (uint32_t)L) return;
    int i, k;
    split_index(n, D, i, k);
    const size_t x = (size_t)i * ld + k;
    const double dp = dpi[x];
    const double rinv = 1.0 / (dp - dt * divF[x]);
    const TC r1 = (TC)(dp * rinv), r2 = (TC)(dt * rinv);
    int nb[GRIST_MAXE], eidx[GRIST_MAXE];
    TC cw[GRIST_MAXE], fe[GRIST_MAXE];
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        eidx[j] = ldg(m.eoc + i * 6 + j);
        nb[j] = ldg(m.coc + i * 6 + j);
        cw[j] = ldg(Coef<TC>::cdiv(m) + i * 6 + j);
        fe[j] = (TC)ldg(F + (size_t)eidx[j] * ld + k);
    }
    bool bad = false;
    for (int t = 0; t < T; t++) {
        const TQ *qt = qn + (size_t)t * qs;
        const TC *ft = FH + (size_t)t * fs;
        const TC *rp = Rp + (size_t)t * qs, *rm = Rm + (size_t)t * qs;
        const TC rp_i = rp[x], rm_i = rm[x];
        TC div = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            size_t y = (size_t)nb[j] * ld + k;
            TC fl = upwind_flux<TQ, TC>(fe[j], cw[j], i, nb[j], qt, ld, k);
            TC ae = ldg(ft + (size_t)eidx[j] * ld + k) - fl;
            const bool i_is_c1 = cw[j] > (TC)0;
            TC rp1 = i_is_c1 ? rp_i : ldg(rp + y), rm1 = i_is_c1 ? rm_i : ldg(rm + y);
            TC rp2 = i_is_c1 ? ldg(rp + y) : rp_i, rm2 = i_is_c1 ? ldg(rm + y) : rm_i;
            TC c = ae >= (TC)0 ? fmin_(rm1, rp2) : fmin_(rp1, rm2);
            div += cw[j] * (fl + c * ae);
        }
        TC v = r1 * (TC)qt[x] - r2 * div;
        bad |= !isfinite(v);
        qout[(size_t)t * qs + x] = (TQ)v;
    }
    if (bad) atomicOr(status, GRIST_FLAG_NONFINITE);
}

template <typename T>
__global__ void k_copy(const T *__restrict__ src, T *__restrict__ dst, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = src[i];
}

template <typename TQ, typename TC>
int member_step(grist_mesh_s *h, const grist_tracer_member &mb, int limiter, double beta, double dt,
                cudaStream_t st) {
    const DevMesh &m = dev_mesh(h);
    const int L = mb.n_levels, T = mb.n_tracers, ld = mb.ld;
    if (T == 0 || L == 0) return GRIST_OK;
    const size_t qs = (size_t)m.nC * ld, fs = (size_t)m.nE * ld;
    // scratch: divF | qA | qB | FH | Rp | Rm
    size_t b_div = qs * sizeof(double), b_q = (size_t)T * qs * sizeof(TQ), b_fh = (size_t)T * fs * sizeof(TC),
           b_r = (size_t)T * qs * sizeof(TC);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t total = al(b_div) + 2 * al(b_q) + al(b_fh) + 2 * al(b_r);
    char *s = (char *)scratch(h, 0, total);
    if (!s) return GRIST_ENOMEM;
    double *divF = (double *)s;
    TQ *qA = (TQ *)(s + al(b_div));
    TQ *qB = (TQ *)((char *)qA + al(b_q));
    TC *FH = (TC *)((char *)qB + al(b_q));
    TC *Rp = (TC *)((char *)FH + al(b_fh));
    TC *Rm = (TC *)((char *)Rp + al(b_r));
    TQ *q = (TQ *)mb.q;
    uint32_t *status = status_word(h);

    const LevelDiv D = make_div((uint32_t)L);
    const unsigned gC = grid_for((long long)m.nC * L, kBlock), gE = grid_for((long long)m.nE * L, kBlock);
    const bool b1 = beta == 1.0;
    const double dts[3] = {dt / 3.0, dt / 2.0, dt};

    GRIST_LAUNCH(h, PN("k_div_mass"), st, k_div_mass<<<gC, kBlock, 0, st>>>(m, L, ld, D, mb.mass_flux, divF));
    const TQ *in = q;
    TQ *outs[2] = {qA, qB};
    for (int s3 = 0; s3 < 3; s3++) {
        if (b1)
            GRIST_LAUNCH(h, PN("k_edge_flux"), st, k_edge_flux<TQ, TC, true><<<gE, kBlock, 0, st>>>(m, T, L, ld, D, in, qs, mb.mass_flux, (TC)beta, FH, fs));
        else
            GRIST_LAUNCH(h, PN("k_edge_flux"), st, k_edge_flux<TQ, TC, false><<<gE, kBlock, 0, st>>>(m, T, L, ld, D, in, qs, mb.mass_flux, (TC)beta, FH, fs));
        if (s3 < 2) {
            GRIST_LAUNCH(h, PN("k_stage_update"), st, k_stage_update<TQ, TC><<<gC, kBlock, 0, st>>>(m, T, L, ld, D, q, outs[s3], qs, FH, fs, mb.dpi, divF,
                                                         dts[s3], status));
            in = outs[s3];
        } else if (!limiter) {
            // final stage without limiter: each thread reads only its own q^n
            GRIST_LAUNCH(h, PN("k_stage_update"), st, k_stage_update<TQ, TC><<<gC, kBlock, 0, st>>>(m, T, L, ld, D, q, q, qs, FH, fs, mb.dpi, divF, dt,
                                                         status));
        } else {
            GRIST_LAUNCH(h, PN("k_fct_lowres"), st, k_fct_lowres<TQ, TC><<<gC, kBlock, 0, st>>>(m, T, L, ld, D, q, qs, mb.mass_flux, mb.dpi, divF, dt, qA));
            GRIST_LAUNCH(h, PN("k_fct_ratios"), st, k_fct_ratios<TQ, TC><<<gC, kBlock, 0, st>>>(m, T, L, ld, D, q, qA, qs, FH, fs, mb.mass_flux, mb.dpi,
                                                       divF, dt, Rp, Rm));
            GRIST_LAUNCH(h, PN("k_fct_final"), st, k_fct_final<TQ, TC><<<gC, kBlock, 0, st>>>(m, T, L, ld, D, q, qB, qs, FH, fs, mb.mass_flux, mb.dpi,
                                                      divF, dt, Rp, Rm, status));
            GRIST_LAUNCH(h, PN("k_copy"), st, k_copy<TQ><<<1024, kBlock, 0, st>>>(qB, q, (size_t)T * qs));
        }
    }
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_tracer_step(grist_mesh h, const grist_tracer_batch *b, double dt, void *stream) {
    if (!h || !b || (b->n_members > 0 && !b->members) || b->n_members < 0) return GRIST_EINVAL;
    if (!(dt > 0) || !std::isfinite(dt)) return GRIST_EINVAL;
    if (b->prec != GRIST_FP64 && b->prec != GRIST_MIX && b->prec != GRIST_MIX_DBL_MASS) return GRIST_EINVAL;
    for (int i = 0; i < b->n_members; i++) {
        const grist_tracer_member &mb = b->members[i];
        if (mb.n_levels < 0 || mb.n_tracers < 0 || mb.n_levels > GRIST_MAXL || mb.ld < mb.n_levels) return GRIST_EINVAL;
        if (mb.n_levels > 0 && mb.n_tracers > 0 && (!mb.q || !mb.dpi || !mb.mass_flux)) return GRIST_EINVAL;
    }
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < b->n_members; i++) {
        int rc = b->prec == GRIST_FP64
                     ? member_step<double, double>(h, b->members[i], b->limiter, b->beta_upwind, dt, st)
                     : member_step<float, float>(h, b->members[i], b->limiter, b->beta_upwind, dt, st);
        if (rc != GRIST_OK) return rc;
    }
    return GRIST_OK;
}
