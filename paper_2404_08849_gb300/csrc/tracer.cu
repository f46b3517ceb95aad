// tracer.cu - tracer transport, Eq. 10 (horizontal part), Sec. 2.1:
// third-order upwind edge flux, Wicker-Skamarock RK3, Zalesak FCT on the
// final stage; FP64 or single-precision tracers (Sec. 2.3) with an FP64
// mass flux and FP64 layer mass.
//
// Batching (ensembles of uneven members, Sec. 4.3 ensemble runs): every
// phase of the step is one pass over a flat work list that concatenates,
// for each member m and tracer group g (tracers_per_thread tracers), the
// (entity, level) index space of that member; a segment table maps a flat
// index to (m, g) by binary search, cached per thread across grid-stride
// iterations.  The phases run either as one launch each or inside one
// persistent cooperative kernel separated by bounded grid barriers.
//
// These kernels are bound by instruction issue and latency, not by the FP64
// pipe, so they keep the hardware binary32/binary64 conversions (one issue
// slot each) rather than the integer ones the FP64-bound dycore kernels use.
//
// Data layout: q [T][nC][ld], dpi [nC][ld], mass flux [nE][ld], edge
// fluxes [T][nE][ld]; consecutive threads take consecutive levels of one
// entity (coalesced rows), neighbour rows are gathered through L1/L2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

#define PN(n) (sizeof(TC) == 4 ? n "/mix" : n "/fp64")

namespace grist {

struct MemberDev {
    void *q;                // [T][nC][ld] caller's tracers (q^n in, q^{n+1} out)
    const double *dpi;      // [nC][ld]
    const double *F;        // [nE][ld]
    void *qA, *qB;          // scratch stage tracers [T][nC][ld]
    void *FH;               // scratch edge fluxes [T][nE][ld]; A = F^H - F^L in a limited final stage
    void *R2;               // scratch FCT ratios {R+, R-} [T][nC][ld] pairs in the compute type
    void *X2;               // scratch FCT local bounds {max, min}(q^n, q^td) [T][nC][ld] pairs
    void *DFL;              // scratch FCT div F^L [T][nC][ld] in the compute type
    const void *Ff;         // mass flux in the compute type [nE][ld]: a binary32 copy (scratch) or F itself
    void *DV;               // scratch {dpi, div F} pairs in the compute type [nC][ld]
    int L, T, ld, pad;
    const double *Mv;       // time-mean vertical mass flux [nC][ldi] or null (no vertical step)
    int ldi;
    LevelDiv DL;            // division by Lg
    int Lg;                 // level groups: a thread takes levels g, g + Lg, ... (levels_per_thread of them)
    unsigned long long qs, fs;  // nC*ld, nE*ld
};

// A flat work space: segment s covers [start[s], start[s+1]) and belongs to
// member mg[s].x, tracer group mg[s].y; within a segment the local index r
// is entity * L + level.
struct Space {
    const unsigned long long *start;  // [nseg + 1]
    const int2 *mg;                   // [nseg]
    int nseg;
    unsigned long long total;
};

// Tiles of consecutive (space-filling-curve) cells for the fused stage
// kernel: per tile the halo cells its edge fluxes read (the tile, its
// neighbours and theirs), its edges, and for every tile edge the halo-local
// indices of c1, c2 and the two deriv-two stencils; per tile cell the
// tile-local index of each of its six edges.
constexpr int kTileCells = 32;

struct TileMesh {
    int ntiles, Hmax, Emax;
    const int *hoff;           // [ntiles + 1]
    const int *halo;           // global cell ids
    const int *eoff;           // [ntiles + 1]
    const int *tedge;          // global edge ids
    const uint16_t *eloc;      // [edges][16]: c1, c2, stencil side 0 (7), side 1 (7)
    const uint16_t *cle;       // [ntiles * kTileCells][6]
};

struct TracerCtx {
    grist_tracer_tuning tune{128, 4, 0, 0, 0, 2, 1};
    // tile tables (built on first use)
    char *dtile = nullptr;
    TileMesh tiles{};
    // work-list tables (member descriptors, segment tables), one device copy
    // per distinct batch, never rewritten: a step recorded in a graph keeps
    // reading the table it was recorded with, whatever other batches run
    // in between.  cur: the table of the last planned batch.
    struct Table {
        std::vector<char> host;
        char *dev = nullptr;
    };
    std::vector<Table> tabs;
    int cur = -1;
    unsigned *barrier = nullptr;  // [0] arrival count, [1] generation, [2] abort, [3] self-test word
    // graph cache: the last few captured steps, keyed by their signature
    // (buffers, sizes, dt, tuning, stream) - alternating buffer sets, as in
    // a pipelined caller, each keep their graph
    struct GraphEntry {
        std::vector<unsigned long long> sig;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<GraphEntry> graphs;
    bool graph_failed = false;
    std::vector<unsigned long long> failed_sig;

    void drop_graphs() {
        for (auto &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
        }
        graphs.clear();
    }
};

constexpr size_t kGraphCache = 4;
constexpr size_t kTableCache = 64;   // distinct batches whose tables a handle keeps

void tracer_ctx_free(TracerCtx *c) {
    if (!c) return;
    c->drop_graphs();
    for (auto &t : c->tabs)
        if (t.dev) cudaFree(t.dev);
    if (c->dtile) cudaFree(c->dtile);
    if (c->barrier) cudaFree(c->barrier);
    delete c;
}

namespace {

constexpr long long kBarrierSpinLimit = 20000000;  // x ~64 ns sleep: about a second
constexpr int kVertMaxL = 128;   // levels supported by the vertical transport
// Largest block of the work-list kernels (their register use, at most 128
// per thread, lets every block up to this size launch).
constexpr int kTracerMaxBlock = 512;

struct Batch {
    const MemberDev *mem;
    int nm;
    Space D, C, E;  // D: cell x level (no groups); C: cell x level x group; E: edge x level x group
    Space T;        // blocks of the fused stage kernel: segment start = first block of (member, group)
    int tpt;
    int lpt;        // levels per thread of the work-list phases (1 or 2; the persistent launch takes 1)
    double dt;
    double dt3;     // dt / 3, the first RK stage (formed on the host)
    int fct;
    int beta1;
    int ring;       // the edge phases run cell-centrically (item_edge_ring) over the space C
    double beta;
    double cmax;    // vertical transport: largest explicit Courant number
};

// Cached segment lookup: returns the segment of flat index n, reusing seg
// when n still lies inside it.
__device__ __forceinline__ int find_seg(const Space &S, unsigned long long n, int seg) {
    if (seg >= 0 && n >= S.start[seg] && n < S.start[seg + 1]) return seg;
    int lo = 0, hi = S.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.start[mid] <= n) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Loads of arrays that a phase writes and a later phase reads.  Inside the
// persistent kernel such data changes during the launch, so it is read
// coherently at L2 (ld.global.cg); across separate launches the read-only
// path is safe.
template <bool PERS, typename T> __device__ __forceinline__ T lds(const T *p) {
    return PERS ? __ldcg(p) : __ldg(p);
}

template <typename TC> __device__ __forceinline__ TC tiny_of();
template <> __device__ __forceinline__ double tiny_of<double>() { return 2.2250738585072014e-308; }
template <> __device__ __forceinline__ float tiny_of<float>() { return 1.17549435e-38f; }

// ---------------------------------------------------------------------------
// phase bodies (one work item each)

// {dpi, div F} pair in the compute type.
template <typename TC> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// Stage ratios r1 = dpi^n / dpi^(s) and r2 = dt_s / dpi^(s) of the update
// q^(s) = r1 q^n - r2 div F^H, with dpi^(s) = dpi^n - dt_s div F: FP64 in the
// FP64 policy (the oracle's arithmetic); in the binary32 policy in binary32
// from the rounded pair, so the binary32 phases issue no FP64 instruction
// (the ratios are rounded to binary32 either way).
__device__ __forceinline__ void stage_ratios(double2 dv, double dts, float, double &r1, double &r2) {
    const double rinv = rcp(dv.x - dts * dv.y);
    r1 = dv.x * rinv;
    r2 = dts * rinv;
}
__device__ __forceinline__ void stage_ratios(float2 dv, double, float dtsf, float &r1, float &r2) {
    const float rinv = __frcp_rn(fmaf(-dtsf, dv.y, dv.x));
    r1 = dv.x * rinv;
    r2 = dtsf * rinv;
}
// Layer mass at the end of the step, dpi^n - dt div F, in the compute type.
__device__ __forceinline__ double end_mass(double2 dv, double dt, float) { return dv.x - dt * dv.y; }
__device__ __forceinline__ float end_mass(float2 dv, double, float dtf) { return fmaf(-dtf, dv.y, dv.x); }

template <bool PERS, typename TC>
__device__ __forceinline__ typename Vec2<TC>::T dv_at(const MemberDev &mb, size_t x) {
    return lds<PERS>((const typename Vec2<TC>::T *)mb.DV + x);
}

// A cell's edges, neighbours and divergence weights, read once per work
// item (rows of 8, 16-byte vectors) and shared by its levels.
static_assert(GRIST_MAXE == 6, "cell rows hold 6 entries");
template <typename TW> struct CellRow {
    int e[GRIST_MAXE], nb[GRIST_MAXE];
    TW cw[GRIST_MAXE];
};
template <bool NB, typename TW>
__device__ __forceinline__ void load_cell_row(const DevMesh &m, int i, CellRow<TW> &r) {
    load_row6(m.eoc8, i, r.e);
    if (NB) load_row6(m.coc8, i, r.nb);
    load_row6(Coef<TW>::cdiv8(m), i, r.cw);
}

// Tracer continuity of the member: div F of the FP64 time-mean mass flux,
// summed in FP64, stored with dpi^n as the {dpi, div F} pair of the later
// phases (rounded to binary32 in the binary32 policy).  In that policy each
// edge's flux is also rounded once to binary32 for the later phases (by the
// cell it leaves: positive divergence coefficient), so they read 4 bytes
// per edge-level instead of 8.
template <typename TC>
__device__ __forceinline__ void item_div(const MemberDev &mb, const CellRow<double> &r, int i, int k) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) {
        const int e = r.e[j];
        const double cw = r.cw[j];
        const double f = ldg(mb.F + (size_t)e * mb.ld + k);
        s += cw * f;
        if (sizeof(TC) == 4 && cw > 0.0) ((float *)mb.Ff)[(size_t)e * mb.ld + k] = cv<float>(f);
    }
    const size_t x = (size_t)i * mb.ld + k;
    if (sizeof(TC) == 4) ((float2 *)mb.DV)[x] = make_float2(cv<float>(ldg(mb.dpi + x)), cv<float>(s));
    else ((double2 *)mb.DV)[x] = make_double2(ldg(mb.dpi + x), s);
}

// Mass flux of edge-level x in the compute type: the binary32 copy made by
// the continuity phase (read coherently inside the persistent launch, which
// wrote it), or the caller's FP64 array.
template <bool PERS, typename TC>
__device__ __forceinline__ TC flux_at(const MemberDev &mb, size_t x) {
    if (sizeof(TC) == 4) return (TC)lds<PERS>((const float *)mb.Ff + x);
    return (TC)ldg(mb.F + x);
}

// Products and sums of the limiter written with explicit rounding, so the
// edge-centric and cell-centric forms (different kernels) give the same
// bits: F^L = F q^n_upwind, A = F^H - F^L with F^H = F q_e, div F^L summed
// by fused multiply-adds in edge order, q^td = r1 q^n - r2 div F^L.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename TC> __device__ __forceinline__ TC antidiff(TC f, TC qe, TC qup) {
    return mul_rn(f, qe) - mul_rn(f, qup);
}
template <typename TC> __device__ __forceinline__ TC lowres_value(TC r1, TC r2, TC qn, TC divl) {
    return fma_rn(r1, qn, -mul_rn(r2, divl));
}

// Third-order upwind edge flux (Skamarock-Gassmann form):
//   q_e = (q1 + q2)/2 - (dc^2/12)(q''1 + q''2) + sgn(F) beta (dc^2/12)(q''2 - q''1)
// F^H = F q_e.  With beta = 1 only the upwind side's second derivative
// survives: q_e = (q1 + q2)/2 - 2 (dc^2/12) q''_upwind.
// In the final stage of a limited step (qn = q^n) the phase stores the
// antidiffusive flux A = F^H - F^L instead of F^H.
template <bool PERS, typename TQ, typename TC>
__device__ __forceinline__ void item_edge(const DevMesh &m, const MemberDev &mb, const TQ *q, const TQ *qn, int t0,
                                          int t1, int e, int k, bool beta1, TC beta) {
    const int ld = mb.ld;
    const int2 c = ldg(m.coe + e);
    const TC f = flux_at<PERS, TC>(mb, (size_t)e * ld + k);
    const TC dc2 = ldg(Coef<TC>::dc2(m) + e);
    const int32_t *st = m.d2i + (size_t)e * 14;
    const TC *cf = Coef<TC>::d2c(m) + (size_t)e * 14;
    TC *FH = (TC *)mb.FH;
    if (beta1 && m.d2w_ok) {
        // one weighted sum over the upwind side's stencil (the mean of c1 and
        // c2 folded into the weights)
        const int side = f >= (TC)0 ? 0 : 1;
        int idx[GRIST_D2P];
        TC w[GRIST_D2P];
        load_d2w(m, e, side, idx, w);
        for (int t = t0; t < t1; t++) {
            const TQ *qt = q + (size_t)t * mb.qs;
            TC v = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) v += w[j] * static_cast<TC>(lds<PERS>(qt + (size_t)idx[j] * ld + k));
            FH[(size_t)t * mb.fs + (size_t)e * ld + k] =
                qn ? antidiff(f, v, static_cast<TC>(qn[(size_t)t * mb.qs + (size_t)idx[0] * ld + k])) : f * v;
        }
    } else if (beta1) {
        const int side = f >= (TC)0 ? 0 : 1;
        int idx[GRIST_D2P];
        TC w[GRIST_D2P];
#pragma unroll
        for (int j = 0; j < GRIST_D2P; j++) {
            idx[j] = ldg(st + side * GRIST_D2P + j);
            w[j] = ldg(cf + side * GRIST_D2P + j);
        }
        for (int t = t0; t < t1; t++) {
            const TQ *qt = q + (size_t)t * mb.qs;
            TC d = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) d += w[j] * static_cast<TC>(lds<PERS>(qt + (size_t)idx[j] * ld + k));
            const TC q1 = static_cast<TC>(lds<PERS>(qt + (size_t)c.x * ld + k)), q2 = static_cast<TC>(lds<PERS>(qt + (size_t)c.y * ld + k));
            const TC qe = (TC)0.5 * (q1 + q2) - (TC)2 * dc2 * d;
            FH[(size_t)t * mb.fs + (size_t)e * ld + k] =
                qn ? antidiff(f, qe, static_cast<TC>(qn[(size_t)t * mb.qs + (size_t)(f >= (TC)0 ? c.x : c.y) * ld + k]))
                   : f * qe;
        }
    } else {
        const TC sgn = f >= (TC)0 ? (TC)1 : (TC)-1;
        for (int t = t0; t < t1; t++) {
            const TQ *qt = q + (size_t)t * mb.qs;
            TC d1 = 0, d2 = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) {
                d1 += ldg(cf + j) * static_cast<TC>(lds<PERS>(qt + (size_t)ldg(st + j) * ld + k));
                d2 += ldg(cf + GRIST_D2P + j) * static_cast<TC>(lds<PERS>(qt + (size_t)ldg(st + GRIST_D2P + j) * ld + k));
            }
            const TC q1 = static_cast<TC>(lds<PERS>(qt + (size_t)c.x * ld + k)), q2 = static_cast<TC>(lds<PERS>(qt + (size_t)c.y * ld + k));
            const TC qe = (TC)0.5 * (q1 + q2) - dc2 * (d1 + d2) + sgn * beta * dc2 * (d2 - d1);
            FH[(size_t)t * mb.fs + (size_t)e * ld + k] =
                qn ? antidiff(f, qe, static_cast<TC>(qn[(size_t)t * mb.qs + (size_t)(f >= (TC)0 ? c.x : c.y) * ld + k]))
                   : f * qe;
        }
    }
}

// The edge item over a thread's LPT levels kg, kg + Lg, ...  With the
// combined weights, the upwind side's stencil (4 vector loads) is read once
// and read again only for a level whose flux runs the other way.
template <bool PERS, typename TQ, typename TC, int LPT>
__device__ __forceinline__ void item_edge_levels(const DevMesh &m, const MemberDev &mb, const TQ *q, const TQ *qn,
                                                 int t0, int t1, int e, int kg, bool beta1, TC beta) {
    if (!(beta1 && m.d2w_ok)) {
#pragma unroll
        for (int u = 0; u < LPT; u++) {
            const int k = kg + u * mb.Lg;
            if (LPT > 1 && k >= mb.L) break;
            item_edge<PERS, TQ, TC>(m, mb, q, qn, t0, t1, e, k, beta1, beta);
        }
        return;
    }
    const int ld = mb.ld;
    TC *FH = (TC *)mb.FH;
    int idx[GRIST_D2P];
    TC w[GRIST_D2P];
    int loaded = -1;
#pragma unroll
    for (int u = 0; u < LPT; u++) {
        const int k = kg + u * mb.Lg;
        if (LPT > 1 && k >= mb.L) break;
        const TC f = flux_at<PERS, TC>(mb, (size_t)e * ld + k);
        const int side = f >= (TC)0 ? 0 : 1;
        if (side != loaded) {
            load_d2w(m, e, side, idx, w);
            loaded = side;
        }
        for (int t = t0; t < t1; t++) {
            const TQ *qt = q + (size_t)t * mb.qs;
            TC v = 0;
#pragma unroll
            for (int j = 0; j < GRIST_D2P; j++) v += w[j] * static_cast<TC>(lds<PERS>(qt + (size_t)idx[j] * ld + k));
            FH[(size_t)t * mb.fs + (size_t)e * ld + k] =
                qn ? antidiff(f, v, static_cast<TC>(qn[(size_t)t * mb.qs + (size_t)idx[0] * ld + k])) : f * v;
        }
    }
}

// Cell-centric form of the edge flux (beta = 1, combined weights, every
// stencil the upwind cell's ring {i, neighbours} in the order of the cell's
// neighbour list): the thread of cell i gathers q over its ring and forms
// the flux of each edge whose flux leaves the cell, so each edge-level is
// written once, by its upwind cell, with the weights and the summation
// order of the edge-centric form (bit-identical), from 7 gathers per
// cell-level instead of 7 per edge-level.  The ring values of up to
// kRingT tracers are gathered first, so each drained edge's weights are
// read once for them; the cell's divergence signs are kept as two masks
// (real edge; i is c1).  In the final stage of a limited step (qn = q^n)
// the phase stores A = F^H - F^L, F^L = F q^n_i.
#ifndef GRIST_TR_RING_T
#define GRIST_TR_RING_T 2
#endif
constexpr int kRingT = GRIST_TR_RING_T;
template <bool PERS, typename TQ, typename TC, int LPT>
__device__ __forceinline__ void item_edge_ring(const DevMesh &m, const MemberDev &mb, const int (&e)[GRIST_MAXE],
                                               const int (&nb)[GRIST_MAXE], unsigned real, unsigned c1,
                                               const TQ *q, const TQ *qn, int t0, int t1, int i, int kg) {
    const int ld = mb.ld;
    TC *FH = (TC *)mb.FH;
#pragma unroll
    for (int u = 0; u < LPT; u++) {
        const int k = kg + u * mb.Lg;
        if (LPT > 1 && k >= mb.L) break;
        TC f[GRIST_MAXE];
        unsigned out = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            f[j] = flux_at<PERS, TC>(mb, (size_t)e[j] * ld + k);
            if (((real >> j) & 1u) && ((f[j] >= (TC)0) == (((c1 >> j) & 1u) != 0))) out |= 1u << j;
        }
        for (int tb = t0; tb < t1; tb += kRingT) {
            const int nt = min(kRingT, t1 - tb);
            TC qr[kRingT][GRIST_D2P], qup[kRingT];
#pragma unroll
            for (int a = 0; a < kRingT; a++) {
                if (a >= nt) break;
                const TQ *qt = q + (size_t)(tb + a) * mb.qs;
                qr[a][0] = static_cast<TC>(lds<PERS>(qt + (size_t)i * ld + k));
#pragma unroll
                for (int j = 0; j < GRIST_MAXE; j++) qr[a][1 + j] = static_cast<TC>(lds<PERS>(qt + (size_t)nb[j] * ld + k));
                qup[a] = qn ? static_cast<TC>(qn[(size_t)(tb + a) * mb.qs + (size_t)i * ld + k]) : (TC)0;
            }
#pragma unroll
            for (int j = 0; j < GRIST_MAXE; j++) {
                if (!(out & (1u << j))) continue;
                TC w[GRIST_D2P];
                load_d2w_weights(m, e[j], ((c1 >> j) & 1u) ? 0 : 1, w);
#pragma unroll
                for (int a = 0; a < kRingT; a++) {
                    if (a >= nt) break;
                    TC v = 0;
#pragma unroll
                    for (int p = 0; p < GRIST_D2P; p++) v += w[p] * qr[a][p];
                    FH[(size_t)(tb + a) * mb.fs + (size_t)e[j] * ld + k] = qn ? antidiff(f[j], v, qup[a]) : f[j] * v;
                }
            }
        }
    }
}

// RK stage update: q^(s) = (dpi^n q^n - dt_s div F^H) / dpi^(s),
// written as r1 q^n - r2 div with r1 = dpi^n/dpi^(s), r2 = dt_s/dpi^(s)
// taken once per (cell, level) in FP64 and rounded to the tracer type
// (Sec. 2.2 (ii): no mixed-kind products inside the tracer loop).
template <bool PERS, typename TQ, typename TC>
__device__ __forceinline__ bool item_update(const CellRow<TC> &r, const MemberDev &mb, TQ *qout, int t0, int t1, int i,
                                            int k, double dts, float dtsf) {
    const int ld = mb.ld;
    const size_t x = (size_t)i * ld + k;
    TC r1, r2;
    stage_ratios(dv_at<PERS, TC>(mb, x), dts, dtsf, r1, r2);
    const int *eidx = r.e;
    const TC *cw = r.cw;
    const TQ *qn = (const TQ *)mb.q;
    const TC *FH = (const TC *)mb.FH;
    bool bad = false;
    for (int t = t0; t < t1; t++) {
        const TC *ft = FH + (size_t)t * mb.fs;
        TC div = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) div += cw[j] * lds<PERS>(ft + (size_t)eidx[j] * ld + k);
        const TC v = r1 * static_cast<TC>(qn[(size_t)t * mb.qs + x]) - r2 * div;
        bad |= !isfinite(v);
        qout[(size_t)t * mb.qs + x] = static_cast<TQ>(v);
    }
    return bad;
}

// FCT 1: low-order solution q^td = (dpi^n q^n - dt div F^L) / dpi^(3),
// with F^L the first-order upwind flux of q^n (the upwind cell is c1 when
// F >= 0, c2 otherwise; cell i is c1 of its edge exactly when its
// divergence coefficient is positive), stored as the cell's local bounds
// {max, min}(q^n, q^td) (X2: q^td is the member of the pair that is not
// q^n, or q^n itself), and div F^L (DFL) for the later phases.
template <bool PERS, typename TQ, typename TC>
__device__ __forceinline__ void item_lowres(const CellRow<TC> &r, const MemberDev &mb, int t0, int t1, int i, int k,
                                            double dt, float dtf) {
    using T2 = typename Vec2<TC>::T;
    const int ld = mb.ld;
    const size_t x = (size_t)i * ld + k;
    TC r1, r2;
    stage_ratios(dv_at<PERS, TC>(mb, x), dt, dtf, r1, r2);
    TC fe[GRIST_MAXE];
#pragma unroll
    for (int j = 0; j < GRIST_MAXE; j++) fe[j] = flux_at<PERS, TC>(mb, (size_t)r.e[j] * ld + k);
    const TQ *qn = (const TQ *)mb.q;
    T2 *X2 = (T2 *)mb.X2;
    TC *DFL = (TC *)mb.DFL;
    for (int t = t0; t < t1; t++) {
        const TQ *qt = qn + (size_t)t * mb.qs;
        TC divl = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            const int up = ((fe[j] >= (TC)0) == (r.cw[j] > (TC)0)) ? i : r.nb[j];
            divl = fma_rn(r.cw[j], mul_rn(fe[j], static_cast<TC>(lds<PERS>(qt + (size_t)up * ld + k))), divl);
        }
        const TC qi = static_cast<TC>(qt[x]);
        const TC qd = static_cast<TC>(static_cast<TQ>(lowres_value(r1, r2, qi, divl)));
        X2[(size_t)t * mb.qs + x] = T2{fmax_(qi, qd), fmin_(qi, qd)};
        DFL[(size_t)t * mb.qs + x] = divl;
    }
}

// FCT 2: bounds over the cell and its neighbours of {q^n, q^td} (from the
// cells' local bounds); antidiffusive in/out sums P+- of A = F^H - F^L (as
// the final edge phase stored it); allowed changes Q+-; ratios
// R+- = min(1, Q / (P + TINY)) (Sec. 2.2 (iii): TINY of the working type),
// stored as the pair {R+, R-}.
template <bool PERS, typename TQ, typename TC>
__device__ __forceinline__ void item_ratios(const CellRow<TC> &r, const MemberDev &mb, int t0, int t1, int i, int k,
                                            double dt, float dtf) {
    using T2 = typename Vec2<TC>::T;
    const int ld = mb.ld;
    const size_t x = (size_t)i * ld + k;
    const TC dp3 = static_cast<TC>(end_mass(dv_at<PERS, TC>(mb, x), dt, dtf));
    const TC dtc = sizeof(TC) == 4 ? (TC)dtf : (TC)dt;
    const T2 *X2 = (const T2 *)mb.X2;
    const TQ *qn = (const TQ *)mb.q;
    const TC *A = (const TC *)mb.FH;
    T2 *R2 = (T2 *)mb.R2;
    for (int t = t0; t < t1; t++) {
        const T2 *xt = X2 + (size_t)t * mb.qs;
        const TC *at = A + (size_t)t * mb.fs;
        const T2 bi = lds<PERS>(xt + x);
        TC qmax = bi.x, qmin = bi.y;
        TC pp = 0, pm = 0;
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            const T2 bn = lds<PERS>(xt + (size_t)r.nb[j] * ld + k);
            qmax = fmax_(qmax, bn.x);
            qmin = fmin_(qmin, bn.y);
            const TC out = r.cw[j] * lds<PERS>(at + (size_t)r.e[j] * ld + k);  // outward A / A_i
            pp += fmax_((TC)0, -out);
            pm += fmax_((TC)0, out);
        }
        pp *= dtc;
        pm *= dtc;
        const TC qn_i = static_cast<TC>(qn[(size_t)t * mb.qs + x]);
        const TC qtd_i = bi.x == qn_i ? bi.y : bi.x;
        const TC Qp = (qmax - qtd_i) * dp3, Qm = (qtd_i - qmin) * dp3;
        R2[(size_t)t * mb.qs + x] = T2{fmin_((TC)1, Qp / (pp + tiny_of<TC>())), fmin_((TC)1, Qm / (pm + tiny_of<TC>()))};
    }
}

// FCT 3: limited flux F^L + C A with C = min(R-(c1), R+(c2)) when A runs
// c1 -> c2 (A >= 0), min(R+(c1), R-(c2)) else; q^{n+1} = (dpi^n q^n - dt
// div(F^L + C A)) / dpi^(3), with div F^L from the low-order phase, written
// over q^n in place (each thread reads only its own cell's q^n).
template <bool PERS, typename TQ, typename TC>
__device__ __forceinline__ bool item_final(const CellRow<TC> &r, const MemberDev &mb, int t0, int t1, int i, int k,
                                           double dt, float dtf) {
    using T2 = typename Vec2<TC>::T;
    const int ld = mb.ld;
    const size_t x = (size_t)i * ld + k;
    TC r1, r2;
    stage_ratios(dv_at<PERS, TC>(mb, x), dt, dtf, r1, r2);
    TQ *q = (TQ *)mb.q;
    const TC *A = (const TC *)mb.FH, *DFL = (const TC *)mb.DFL;
    const T2 *R2 = (const T2 *)mb.R2;
    bool bad = false;
    for (int t = t0; t < t1; t++) {
        const TC *at = A + (size_t)t * mb.fs;
        const T2 *rt = R2 + (size_t)t * mb.qs;
        const T2 ri = lds<PERS>(rt + x);
        TC div = lds<PERS>(DFL + (size_t)t * mb.qs + x);
#pragma unroll
        for (int j = 0; j < GRIST_MAXE; j++) {
            const TC ae = lds<PERS>(at + (size_t)r.e[j] * ld + k);
            const T2 rn = lds<PERS>(rt + (size_t)r.nb[j] * ld + k);
            const bool i_is_c1 = r.cw[j] > (TC)0;
            const TC rp1 = i_is_c1 ? ri.x : rn.x, rm1 = i_is_c1 ? ri.y : rn.y;
            const TC rp2 = i_is_c1 ? rn.x : ri.x, rm2 = i_is_c1 ? rn.y : ri.y;
            const TC c = ae >= (TC)0 ? fmin_(rm1, rp2) : fmin_(rp1, rm2);
            div += r.cw[j] * (c * ae);
        }
        const size_t y = (size_t)t * mb.qs + x;
        const TC v = r1 * static_cast<TC>(q[y]) - r2 * div;
        bad |= !isfinite(v);
        q[y] = static_cast<TQ>(v);
    }
    return bad;
}

// ---------------------------------------------------------------------------
// phases: grid-stride loops over a work space

enum Phase { P_DIV = 0, P_EDGE0, P_UPD0, P_EDGE1, P_UPD1, P_EDGE2, P_UPD2, P_LOWRES, P_RATIOS, P_FINAL, P_NPHASE };

// One pass over a work space.  A work item is (entity, level group g) of a
// member and tracer group; the thread takes the LPT levels g, g + Lg, ...
// (Lg = ceil(L / LPT)), so consecutive threads still touch consecutive
// levels, and the entity's tables are read once for its LPT levels.
// RING: the form of an edge phase, -1 = as B.ring says (the persistent
// launch), 0 / 1 = compiled for one form (the per-phase kernels, so that a
// kernel's registers serve the form it runs).
template <bool PERS, typename TQ, typename TC, int PH, int LPT = 1, int RING = -1>
__device__ void run_phase(const DevMesh &m, const Batch &B, uint32_t *status) {
    const bool ring = RING < 0 ? (B.ring != 0) : (RING == 1);
    const Space &S = (PH == P_DIV) ? B.D : ((PH == P_EDGE0 || PH == P_EDGE1 || PH == P_EDGE2) && !ring) ? B.E : B.C;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    int seg = -1;
    bool bad = false;
    const double dts = PH <= P_UPD0 ? B.dt3 : (PH <= P_UPD1 ? 0.5 * B.dt : B.dt);
    const float dtsf = cv<float>(dts), dtf = cv<float>(B.dt);
    const TC beta = static_cast<TC>(B.beta);
    for (unsigned long long n = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; n < S.total; n += stride) {
        seg = find_seg(S, n, seg);
        const int2 mg = S.mg[seg];
        const MemberDev &mb = B.mem[mg.x];
        int ent, kg;
        split_index((uint32_t)(n - S.start[seg]), mb.DL, ent, kg);
        const int t0 = mg.y * B.tpt;
        const int t1 = min(mb.T, t0 + B.tpt);
        if constexpr (PH == P_EDGE0 || PH == P_EDGE1 || PH == P_EDGE2) {
            const TQ *qs = (const TQ *)(PH == P_EDGE0 ? mb.q : (PH == P_EDGE1 ? mb.qA : mb.qB));
            // the final stage of a limited step stores A = F^H - F^L
            const TQ *qn = (PH == P_EDGE2 && B.fct) ? (const TQ *)mb.q : nullptr;
            if (ring) {
                int e[GRIST_MAXE], nb[GRIST_MAXE];
                TC cw[GRIST_MAXE];
                load_row6(m.eoc8, ent, e);
                load_row6(m.coc8, ent, nb);
                load_row6(Coef<TC>::cdiv8(m), ent, cw);
                unsigned real = 0, c1 = 0;
#pragma unroll
                for (int j = 0; j < GRIST_MAXE; j++) {
                    if (cw[j] != (TC)0) real |= 1u << j;
                    if (cw[j] > (TC)0) c1 |= 1u << j;
                }
                item_edge_ring<PERS, TQ, TC, LPT>(m, mb, e, nb, real, c1, qs, qn, t0, t1, ent, kg);
            } else {
                item_edge_levels<PERS, TQ, TC, LPT>(m, mb, qs, qn, t0, t1, ent, kg, B.beta1, beta);
            }
            continue;
        }
        // the cell's row, once for its LPT levels (FP64 weights for the
        // continuity phase); the limited-flux phase, the one with the most
        // live values per level, reads it again for each level instead
        using TW = typename std::conditional<PH == P_DIV, double, TC>::type;
        constexpr bool kNb = PH == P_LOWRES || PH == P_RATIOS || PH == P_FINAL;
        constexpr bool kRowPerLevel = PH == P_FINAL;
        CellRow<TW> r;
        if (!kRowPerLevel) load_cell_row<kNb>(m, ent, r);
#pragma unroll
        for (int u = 0; u < LPT; u++) {
        const int k = kg + u * mb.Lg;
        if (LPT > 1 && k >= mb.L) break;
        if (kRowPerLevel) load_cell_row<kNb>(m, ent, r);
        if constexpr (PH == P_DIV) item_div<TC>(mb, r, ent, k);
        if constexpr (PH == P_UPD0) bad |= item_update<PERS, TQ, TC>(r, mb, (TQ *)mb.qA, t0, t1, ent, k, dts, dtsf);
        if constexpr (PH == P_UPD1) bad |= item_update<PERS, TQ, TC>(r, mb, (TQ *)mb.qB, t0, t1, ent, k, dts, dtsf);
        if constexpr (PH == P_UPD2) bad |= item_update<PERS, TQ, TC>(r, mb, (TQ *)mb.q, t0, t1, ent, k, dts, dtsf);
        if constexpr (PH == P_LOWRES) item_lowres<PERS, TQ, TC>(r, mb, t0, t1, ent, k, B.dt, dtf);
        if constexpr (PH == P_RATIOS) item_ratios<PERS, TQ, TC>(r, mb, t0, t1, ent, k, B.dt, dtf);
        if constexpr (PH == P_FINAL) bad |= item_final<PERS, TQ, TC>(r, mb, t0, t1, ent, k, B.dt, dtf);
        }
    }
    if (bad) atomicOr(status, GRIST_FLAG_NONFINITE);
}

// Register cap of a work-list phase kernel in the binary32 policy.  These
// kernels are bound by the latency of their neighbour gathers: a cap trades
// the loads each thread keeps in flight against resident warps, and the best
// point differs per phase (measured on the level-9 mesh, 60 levels, 4
// tracers).  Compile-time, per phase; 0 = only the limit that lets a block
// of kTracerMaxBlock threads launch (65536 registers per SM), which is also
// the FP64 policy's cap.
#ifndef GRIST_TR_REGS_EDGE   // edge fluxes, edge-centric form
#define GRIST_TR_REGS_EDGE 56
#endif
#ifndef GRIST_TR_REGS_RING   // edge fluxes, cell-centric form
#define GRIST_TR_REGS_RING 72
#endif
#ifndef GRIST_TR_REGS_UPD
#define GRIST_TR_REGS_UPD 64
#endif
#ifndef GRIST_TR_REGS_LOWRES
#define GRIST_TR_REGS_LOWRES 64
#endif
#ifndef GRIST_TR_REGS_RATIOS
#define GRIST_TR_REGS_RATIOS 72
#endif
#ifndef GRIST_TR_REGS_FINAL
#define GRIST_TR_REGS_FINAL 0
#endif
constexpr int kTracerRegLimit = 65536 / kTracerMaxBlock;
constexpr int cap_or_none(int r) { return r > 0 && r < kTracerRegLimit ? r : kTracerRegLimit; }
template <typename TC, int PH, int RING> constexpr int tracer_phase_regs() {
    return sizeof(TC) != 4                                      ? kTracerRegLimit
           : (PH == P_EDGE0 || PH == P_EDGE1 || PH == P_EDGE2)
               ? cap_or_none(RING == 1 ? GRIST_TR_REGS_RING : GRIST_TR_REGS_EDGE)
           : (PH == P_UPD0 || PH == P_UPD1 || PH == P_UPD2)    ? cap_or_none(GRIST_TR_REGS_UPD)
           : PH == P_LOWRES                                    ? cap_or_none(GRIST_TR_REGS_LOWRES)
           : PH == P_RATIOS                                    ? cap_or_none(GRIST_TR_REGS_RATIOS)
           : PH == P_FINAL                                     ? cap_or_none(GRIST_TR_REGS_FINAL)
                                                               : kTracerRegLimit;
}

template <typename TQ, typename TC, int PH, int LPT, int RING>
__global__ void __maxnreg__((tracer_phase_regs<TC, PH, RING>())) k_tracer_phase(DevMesh m, Batch B, uint32_t *status) {
    run_phase<false, TQ, TC, PH, LPT, RING>(m, B, status);
}

// Fused RK stage (no limiter) on one tile x 32 levels x the tracers of one
// group: the stage input on the tile's halo goes to shared memory, every
// tile edge's third-order flux is computed once into shared memory, and the
// cell update gathers from there (boundary edges of a tile are computed by
// both tiles that share them).  Same arithmetic as item_edge + item_update.
template <typename TQ, typename TC, bool BETA1>
__global__ void __launch_bounds__(256) k_tr_tile_stage(DevMesh m, TileMesh tm, Batch B, int stage,
                                                       uint32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TC *qs = (TC *)smem_raw;              // [Hmax][32]
    TC *fs = qs + (size_t)tm.Hmax * 32;   // [Emax][32]
    __shared__ int s_seg;
    if (threadIdx.x == 0) s_seg = find_seg(B.T, blockIdx.x, -1);
    __syncthreads();
    const int seg = s_seg;
    const int2 mg = B.T.mg[seg];
    const MemberDev &mb = B.mem[mg.x];
    const unsigned r = blockIdx.x - (unsigned)B.T.start[seg];
    const int nch = (mb.L + 31) >> 5;
    const int tile = (int)(r / nch), chunk = (int)(r % nch);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = chunk * 32 + lane;
    const bool kin = k < mb.L;
    const int ld = mb.ld;
    const int h0 = tm.hoff[tile], H = tm.hoff[tile + 1] - h0;
    const int e0 = tm.eoff[tile], E = tm.eoff[tile + 1] - e0;
    const int c0 = tile * kTileCells;
    const int nc = min(kTileCells, m.nC - c0);
    const TQ *qin = stage == 0 ? (const TQ *)mb.q : (stage == 1 ? (const TQ *)mb.qA : (const TQ *)mb.qB);
    TQ *qout = stage == 0 ? (TQ *)mb.qA : (stage == 1 ? (TQ *)mb.qB : (TQ *)mb.q);
    const TQ *qn = (const TQ *)mb.q;
    const double dts = stage == 0 ? B.dt3 : (stage == 1 ? 0.5 * B.dt : B.dt);
    const TC beta = static_cast<TC>(B.beta);
    // stage ratios of this warp's cells (same for every tracer)
    constexpr int kCpw = kTileCells / 4;   // cells per warp for blocks of >= 4 warps
    TC r1v[kCpw], r2v[kCpw];
#pragma unroll
    for (int idx = 0; idx < kCpw; idx++) {
        const int ci = warp + idx * nw;
        r1v[idx] = r2v[idx] = (TC)0;
        if (ci < nc && kin) {
            const size_t x = (size_t)(c0 + ci) * ld + k;
            stage_ratios(((const typename Vec2<TC>::T *)mb.DV)[x], dts, cv<float>(dts), r1v[idx], r2v[idx]);
        }
    }
    const int t0 = mg.y * B.tpt, t1 = min(mb.T, t0 + B.tpt);
    bool bad = false;
    for (int t = t0; t < t1; t++) {
        const TQ *qt = qin + (size_t)t * mb.qs;
        for (int hh = warp; hh < H; hh += nw)
            qs[hh * 32 + lane] = kin ? static_cast<TC>(ldg(qt + (size_t)ldg(tm.halo + h0 + hh) * ld + k)) : (TC)0;
        __syncthreads();
        for (int j = warp; j < E; j += nw) {
            if (kin) {
                const int e = ldg(tm.tedge + e0 + j);
                const uint16_t *loc = tm.eloc + (size_t)(e0 + j) * 16;
                const TC f = static_cast<TC>(ldg(mb.F + (size_t)e * ld + k));
                const TC dc2 = ldg(Coef<TC>::dc2(m) + e);
                const TC *cf = Coef<TC>::d2c(m) + (size_t)e * 14;
                const TC q1 = qs[loc[0] * 32 + lane], q2 = qs[loc[1] * 32 + lane];
                TC qe;
                if (BETA1) {
                    const int side = f >= (TC)0 ? 0 : 1;
                    TC d = 0;
#pragma unroll
                    for (int i = 0; i < GRIST_D2P; i++)
                        d += ldg(cf + side * GRIST_D2P + i) * qs[loc[2 + side * GRIST_D2P + i] * 32 + lane];
                    qe = (TC)0.5 * (q1 + q2) - (TC)2 * dc2 * d;
                } else {
                    const TC sgn = f >= (TC)0 ? (TC)1 : (TC)-1;
                    TC d1 = 0, d2 = 0;
#pragma unroll
                    for (int i = 0; i < GRIST_D2P; i++) {
                        d1 += ldg(cf + i) * qs[loc[2 + i] * 32 + lane];
                        d2 += ldg(cf + GRIST_D2P + i) * qs[loc[2 + GRIST_D2P + i] * 32 + lane];
                    }
                    qe = (TC)0.5 * (q1 + q2) - dc2 * (d1 + d2) + sgn * beta * dc2 * (d2 - d1);
                }
                fs[j * 32 + lane] = f * qe;
            }
        }
        __syncthreads();
#pragma unroll
        for (int idx = 0; idx < kCpw; idx++) {
            const int ci = warp + idx * nw;
            if (ci < nc && kin) {
                const int cell = c0 + ci;
                const uint16_t *le = tm.cle + (size_t)cell * 6;
                TC div = 0;
#pragma unroll
                for (int j = 0; j < GRIST_MAXE; j++) div += ldg(Coef<TC>::cdiv(m) + cell * 6 + j) * fs[le[j] * 32 + lane];
                const size_t x = (size_t)cell * ld + k;
                const TC v = r1v[idx] * static_cast<TC>(qn[(size_t)t * mb.qs + x]) - r2v[idx] * div;
                bad |= !isfinite(v);
                qout[(size_t)t * mb.qs + x] = static_cast<TQ>(v);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(status, GRIST_FLAG_NONFINITE);
}

// ---------------------------------------------------------------------------
// Vertical transport, the delta(M q) term of Eq. 10, by an adaptively
// implicit upwind scheme (Sec. 2.1; the reading): at interior interface j
// (between layers j-1 above and j below, M_j > 0 carrying mass downward)
// the donor layer is j-1 if M_j > 0, else j, with Courant number
// c_j = |M_j| dt / dpi*_donor; the share Me_j = min(1, cmax / c_j) M_j moves
// explicitly (first-order upwind from q at the start), the rest
// Mi_j = M_j - Me_j by backward-Euler upwind, so per column
//   dpi+_k q+_k + dt (Fi_{k+1} - Fi_k) = dpi*_k q_k - dt (Fe_{k+1} - Fe_k),
//   dpi*_k = dpi_k - dt div(F)_k (the horizontal step's end),
//   dpi+_k = dpi*_k - dt (M_{k+1} - M_k),
// a tridiagonal M-matrix system solved by the Thomas algorithm.  Arithmetic
// in the tracer compute type.
__device__ __forceinline__ double vinv(double x) { return rcp(x); }   // correctly rounded, as 1.0 / x
__device__ __forceinline__ float vinv(float x) { return 1.0f / x; }

// One warp per column, lanes over levels (level k = lane + 32 r, r < R;
// R = 2 up to 64 levels, else 4).  Each lane forms the flux split
// at the two interfaces of its layers (an interface shared by two layers is
// split by both from the same operands, so identically).  When no interface
// of the column has an implicit share (every Courant number <= cmax, the
// usual case) the tridiagonal system is diagonal: the Thomas sweep then
// reduces exactly to q+_k = rhs_k * (1 / b_k), which every lane evaluates for
// its own levels in parallel.  Otherwise the rows go through shared memory
// and one lane runs the Thomas sweep of the column; the diagonal case is
// exactly what that sweep computes when the off-diagonals vanish.
constexpr int kVertWarps = 8;

template <typename TQ, typename TC, int kVertR>
__global__ void __launch_bounds__(kVertWarps * 32) k_tr_vertical(DevMesh m, MemberDev mb, double dt, double cmax,
                                                                uint32_t *status) {
    __shared__ TC sA[kVertWarps][kVertMaxL], sB[kVertWarps][kVertMaxL], sC[kVertWarps][kVertMaxL],
        sD[kVertWarps][kVertMaxL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kVertWarps + warp;
    if (i >= m.nC) return;   // whole warps only: no block barrier below
    const int L = mb.L, ld = mb.ld, ldi = mb.ldi;
    const TC dtc = cv<TC>(dt), cm = cv<TC>(cmax);
    const size_t row = (size_t)i * ld, irow = (size_t)i * ldi;
    // start layer mass of the vertical step: the end of the horizontal one
    const typename Vec2<TC>::T *DV = (const typename Vec2<TC>::T *)mb.DV;
    const float dtf = cv<float>(dt);
    auto dstar = [&](int kk) -> TC { return (TC)end_mass(DV[row + kk], dt, dtf); };
    // interface j between layers j-1 (above) and j (below), with those
    // layers' start masses: explicit and implicit shares
    auto split = [&](int j, TC above, TC below, TC &me, TC &mi) {
        const TC Mj = (j > 0 && j < L) ? cv<TC>(mb.Mv[irow + j]) : (TC)0;
        me = mi = (TC)0;
        if (Mj != (TC)0) {
            const TC cour = fabs(Mj) * dtc / (Mj > (TC)0 ? above : below);
            const TC f = cour <= cm ? (TC)1 : cm / cour;
            me = f * Mj;
            mi = Mj - me;
        }
    };
    TC dps[kVertR], met[kVertR], mit[kVertR], meb[kVertR], mib[kVertR], a[kVertR], b[kVertR], c[kVertR];
    bool implicit = false;
#pragma unroll
    for (int r = 0; r < kVertR; r++) {
        const int k = lane + 32 * r;
        dps[r] = met[r] = mit[r] = meb[r] = mib[r] = a[r] = c[r] = (TC)0;
        b[r] = (TC)1;
        if (k < L) {
            const TC d0 = dstar(k);
            const TC dm = k > 0 ? dstar(k - 1) : (TC)0, dp = k + 1 < L ? dstar(k + 1) : (TC)0;
            dps[r] = d0;
            split(k, dm, d0, met[r], mit[r]);
            split(k + 1, d0, dp, meb[r], mib[r]);
            const TC Mt = met[r] + mit[r], Mb = meb[r] + mib[r];
            const TC dpn = d0 - dtc * (Mb - Mt);
            a[r] = -dtc * fmax_((TC)0, mit[r]);
            b[r] = dpn + dtc * (fmax_((TC)0, mib[r]) - fmin_((TC)0, mit[r]));
            c[r] = dtc * fmin_((TC)0, mib[r]);
            implicit |= (mit[r] != (TC)0) | (mib[r] != (TC)0);
        }
    }
    implicit = __any_sync(0xffffffffu, implicit);
    TC rb[kVertR];
#pragma unroll
    for (int r = 0; r < kVertR; r++) rb[r] = vinv(b[r]);
    bool bad = false;
    for (int t = 0; t < mb.T; t++) {
        TQ *qt = (TQ *)mb.q + (size_t)t * mb.qs + row;
        TC rhs[kVertR];
#pragma unroll
        for (int r = 0; r < kVertR; r++) {
            const int k = lane + 32 * r;
            rhs[r] = (TC)0;
            if (k < L) {
                const TC qk = (TC)qt[k];
                const TC qm = k > 0 ? (TC)qt[k - 1] : (TC)0, qp = k + 1 < L ? (TC)qt[k + 1] : (TC)0;
                const TC Mt = met[r] + mit[r], Mb = meb[r] + mib[r];
                const TC q_top = Mt > (TC)0 ? qm : qk;
                const TC q_bot = Mb > (TC)0 ? qk : qp;
                rhs[r] = dps[r] * qk - dtc * (meb[r] * q_bot - met[r] * q_top);
            }
        }
        __syncwarp();   // every lane has read the column before any lane writes it
        if (!implicit) {
#pragma unroll
            for (int r = 0; r < kVertR; r++) {
                const int k = lane + 32 * r;
                if (k < L) {
                    const TC x = rhs[r] * rb[r];
                    bad |= !isfinite(x);
                    qt[k] = (TQ)x;
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < kVertR; r++) {
                const int k = lane + 32 * r;
                if (k < L) {
                    sA[warp][k] = a[r];
                    sB[warp][k] = b[r];
                    sC[warp][k] = c[r];
                    sD[warp][k] = rhs[r];
                }
            }
            __syncwarp();
            if (lane == 0) {
                // Thomas sweep (forward elimination into sC / sD, back
                // substitution into sD), the arithmetic of k_tr_vertical
                for (int k = 0; k < L; k++) {
                    const TC rden = vinv(k == 0 ? sB[warp][k] : sB[warp][k] - sA[warp][k] * sC[warp][k - 1]);
                    const TC cpk = sC[warp][k] * rden;
                    sD[warp][k] = (k == 0 ? sD[warp][k] : sD[warp][k] - sA[warp][k] * sD[warp][k - 1]) * rden;
                    sC[warp][k] = cpk;
                }
                TC qb = (TC)0;
                for (int k = L - 1; k >= 0; k--) {
                    qb = (k == L - 1) ? sD[warp][k] : sD[warp][k] - sC[warp][k] * qb;
                    sD[warp][k] = qb;
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < kVertR; r++) {
                const int k = lane + 32 * r;
                if (k < L) {
                    const TC x = sD[warp][k];
                    bad |= !isfinite(x);
                    qt[k] = (TQ)x;
                }
            }
            __syncwarp();   // the next tracer reuses the rows
        }
    }
    if (bad) atomicOr(status, GRIST_FLAG_NONFINITE);
}

// Bounded wait until *gen differs from g: at most `limit` polls (~64 ns
// apart); on giving up (or when another block already gave up) raises
// GRIST_FLAG_TIMEOUT and returns false.
__device__ bool bounded_wait_change(volatile unsigned *gen, unsigned g, long long limit, unsigned *abort_word,
                                    uint32_t *status) {
    long long it = 0;
    while (*gen == g) {
        if (++it > limit || *(volatile unsigned *)abort_word) {
            atomicExch(abort_word, 1u);
            atomicOr(status, GRIST_FLAG_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Grid barrier for a cooperative launch (all blocks co-resident).  bar[0]
// counts arrivals, bar[1] is the generation, bar[2] the launch's abort word
// (both bar[0] and bar[2] are zeroed before every launch).  Thread 0 of each
// block arrives on the counter; the last arrival resets it and bumps the
// generation.  The wait is bounded (bounded_wait_change), so the kernel
// always ends; after a timeout every block returns false.
__device__ bool grid_sync(unsigned *bar, uint32_t *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else if (!bounded_wait_change(gen, g, kBarrierSpinLimit, bar + 2, status)) {
            ok = 0;
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Self-test of the bounded wait: one thread waits on a word nothing writes.
__global__ void k_wait_selftest(unsigned *word, unsigned *abort_word, long long limit, uint32_t *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        bounded_wait_change(word, *(volatile unsigned *)word, limit, abort_word, status);
}

// One cooperative launch for the whole step: the phases in order with a
// grid barrier between consecutive ones.
template <typename TQ, typename TC>
__global__ void k_tracer_persistent(DevMesh m, Batch B, unsigned *bar, uint32_t *status) {
    run_phase<true, TQ, TC, P_DIV>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_EDGE0>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_UPD0>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_EDGE1>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_UPD1>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_EDGE2>(m, B, status);
    if (!grid_sync(bar, status)) return;
    if (!B.fct) {
        run_phase<true, TQ, TC, P_UPD2>(m, B, status);
        return;
    }
    run_phase<true, TQ, TC, P_LOWRES>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_RATIOS>(m, B, status);
    if (!grid_sync(bar, status)) return;
    run_phase<true, TQ, TC, P_FINAL>(m, B, status);
}

// ---------------------------------------------------------------------------
// host side

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct HostPlan {
    std::vector<MemberDev> mem;
    std::vector<unsigned long long> sD, sC, sE, sT;
    std::vector<int2> mD, mC, mE, mT;
    size_t scratch_bytes = 0;
};

template <typename TQ, typename TC>
int plan_batch(const DevMesh &m, const grist_tracer_batch *b, int tpt, int lpt, HostPlan &P) {
    P = HostPlan();
    size_t off = 0;
    unsigned long long tD = 0, tC = 0, tE = 0, tT = 0;
    const unsigned long long ntiles = ((unsigned long long)m.nC + kTileCells - 1) / kTileCells;
    for (int i = 0; i < b->n_members; i++) {
        const grist_tracer_member &u = b->members[i];
        if (u.n_levels == 0 || u.n_tracers == 0) continue;
        MemberDev d{};
        d.q = u.q;
        d.dpi = u.dpi;
        d.F = u.mass_flux;
        d.L = u.n_levels;
        d.T = u.n_tracers;
        d.ld = u.ld;
        d.Mv = u.vmass_flux;
        d.ldi = u.ld_int;
        d.Lg = (u.n_levels + lpt - 1) / lpt;
        d.DL = make_div((uint32_t)d.Lg);
        d.qs = (unsigned long long)m.nC * u.ld;
        d.fs = (unsigned long long)m.nE * u.ld;
        // scratch offsets (relative, resolved after allocation)
        const size_t bq = (size_t)d.T * d.qs * sizeof(TQ), bf = (size_t)d.T * d.fs * sizeof(TC),
                     br = (size_t)d.T * d.qs * sizeof(TC);
        d.qA = (void *)(uintptr_t)off; off += al256(bq);
        d.qB = (void *)(uintptr_t)off; off += al256(bq);
        d.FH = (void *)(uintptr_t)off; off += al256(bf);
        d.R2 = (void *)(uintptr_t)off; off += al256(2 * br);
        d.X2 = (void *)(uintptr_t)off; off += al256(2 * br);
        d.DFL = (void *)(uintptr_t)off; off += al256(br);
        if (sizeof(TC) == 4) { d.Ff = (const void *)(uintptr_t)off; off += al256(d.fs * sizeof(float)); }
        d.DV = (void *)(uintptr_t)off; off += al256(d.qs * 2 * sizeof(TC));
        const int idx = (int)P.mem.size();
        const int G = (d.T + tpt - 1) / tpt;
        P.sD.push_back(tD); P.mD.push_back(make_int2(idx, 0));
        tD += (unsigned long long)m.nC * d.Lg;
        for (int g = 0; g < G; g++) {
            P.sC.push_back(tC); P.mC.push_back(make_int2(idx, g));
            tC += (unsigned long long)m.nC * d.Lg;
            P.sE.push_back(tE); P.mE.push_back(make_int2(idx, g));
            tE += (unsigned long long)m.nE * d.Lg;
            P.sT.push_back(tT); P.mT.push_back(make_int2(idx, g));
            tT += ntiles * (unsigned long long)((d.L + 31) / 32);
        }
        P.mem.push_back(d);
    }
    P.sD.push_back(tD);
    P.sC.push_back(tC);
    P.sE.push_back(tE);
    P.sT.push_back(tT);
    P.scratch_bytes = off;
    return GRIST_OK;
}

// Upload the plan's tables (member descriptors with resolved scratch
// pointers, segment tables) into the context's device table; returns the
// Batch with device pointers.  Synchronous when the tables change.
template <typename TQ, typename TC>
int upload_plan(grist_mesh_s *h, TracerCtx *c, HostPlan &P, const grist_tracer_batch *b, double dt, Batch &B,
                cudaStream_t st) {
    char *scr = (char *)scratch(h, 0, P.scratch_bytes + 256);
    if (!scr) return GRIST_ENOMEM;
    for (auto &d : P.mem) {
        d.qA = scr + (uintptr_t)d.qA;
        d.qB = scr + (uintptr_t)d.qB;
        d.FH = scr + (uintptr_t)d.FH;
        d.R2 = scr + (uintptr_t)d.R2;
        d.X2 = scr + (uintptr_t)d.X2;
        d.DFL = scr + (uintptr_t)d.DFL;
        d.Ff = sizeof(TC) == 4 ? (const void *)(scr + (uintptr_t)d.Ff) : (const void *)d.F;
        d.DV = scr + (uintptr_t)d.DV;
    }
    const size_t nm = P.mem.size();
    size_t o = 0;
    const size_t o_mem = o; o += al256(nm * sizeof(MemberDev));
    const size_t o_sD = o; o += al256(P.sD.size() * 8);
    const size_t o_sC = o; o += al256(P.sC.size() * 8);
    const size_t o_sE = o; o += al256(P.sE.size() * 8);
    const size_t o_mD = o; o += al256(P.mD.size() * sizeof(int2));
    const size_t o_mC = o; o += al256(P.mC.size() * sizeof(int2));
    const size_t o_mE = o; o += al256(P.mE.size() * sizeof(int2));
    const size_t o_sT = o; o += al256(P.sT.size() * 8);
    const size_t o_mT = o; o += al256(P.mT.size() * sizeof(int2));
    std::vector<char> ht(o, 0);
    std::memcpy(ht.data() + o_mem, P.mem.data(), nm * sizeof(MemberDev));
    std::memcpy(ht.data() + o_sD, P.sD.data(), P.sD.size() * 8);
    std::memcpy(ht.data() + o_sC, P.sC.data(), P.sC.size() * 8);
    std::memcpy(ht.data() + o_sE, P.sE.data(), P.sE.size() * 8);
    std::memcpy(ht.data() + o_mD, P.mD.data(), P.mD.size() * sizeof(int2));
    std::memcpy(ht.data() + o_mC, P.mC.data(), P.mC.size() * sizeof(int2));
    std::memcpy(ht.data() + o_mE, P.mE.data(), P.mE.size() * sizeof(int2));
    std::memcpy(ht.data() + o_sT, P.sT.data(), P.sT.size() * 8);
    std::memcpy(ht.data() + o_mT, P.mT.data(), P.mT.size() * sizeof(int2));
    int ti = -1;
    for (size_t x = 0; x < c->tabs.size() && ti < 0; x++)
        if (c->tabs[x].host.size() == o && std::memcmp(c->tabs[x].host.data(), ht.data(), o) == 0) ti = (int)x;
    if (ti < 0) {
        // a batch not seen before: its table is made outside any stream
        // capture (a recorded step must have run once without capture)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        GRIST_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone) return GRIST_EUNSUPPORTED;
        if (c->tabs.size() >= kTableCache) {
            // drop the oldest table (and the tracer graphs, which may read it)
            GRIST_CUDA_TRY(cudaDeviceSynchronize());
            c->drop_graphs();
            cudaFree(c->tabs.front().dev);
            c->tabs.erase(c->tabs.begin());
        }
        TracerCtx::Table t;
        if (cudaMalloc(&t.dev, o) != cudaSuccess) return GRIST_ENOMEM;
        if (cudaMemcpy(t.dev, ht.data(), o, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(t.dev);
            return GRIST_ECUDA;
        }
        t.host = ht;
        c->tabs.push_back(std::move(t));
        ti = (int)c->tabs.size() - 1;
    }
    c->cur = ti;
    char *dtab = c->tabs[ti].dev;
    if (!c->barrier) {
        if (cudaMalloc(&c->barrier, 4 * sizeof(unsigned)) != cudaSuccess) return GRIST_ENOMEM;
        GRIST_CUDA_TRY(cudaMemset(c->barrier, 0, 4 * sizeof(unsigned)));
    }
    B.mem = (const MemberDev *)(dtab + o_mem);
    B.nm = (int)nm;
    B.D = Space{(const unsigned long long *)(dtab + o_sD), (const int2 *)(dtab + o_mD), (int)P.mD.size(), P.sD.back()};
    B.C = Space{(const unsigned long long *)(dtab + o_sC), (const int2 *)(dtab + o_mC), (int)P.mC.size(), P.sC.back()};
    B.E = Space{(const unsigned long long *)(dtab + o_sE), (const int2 *)(dtab + o_mE), (int)P.mE.size(), P.sE.back()};
    B.T = Space{(const unsigned long long *)(dtab + o_sT), (const int2 *)(dtab + o_mT), (int)P.mT.size(), P.sT.back()};
    B.tpt = c->tune.tracers_per_thread;
    B.lpt = c->tune.persistent ? 1 : c->tune.levels_per_thread;
    B.dt = dt;
    B.dt3 = dt / 3.0;
    B.fct = b->limiter ? 1 : 0;
    B.beta1 = b->beta_upwind == 1.0 ? 1 : 0;
    B.ring = (c->tune.cell_edges && B.beta1 && dev_mesh(h).ring_ok) ? 1 : 0;
    B.beta = b->beta_upwind;
    B.cmax = b->vertical_courant_max;
    return GRIST_OK;
}

int sm_count(int dev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int build_tiles(grist_mesh_s *h, TracerCtx *c);

// Enqueue the horizontal phases (no host synchronisation: capturable).
template <typename TQ, typename TC>
int enqueue_horizontal(grist_mesh_s *h, TracerCtx *c, const Batch &B, cudaStream_t st) {
    const DevMesh &m = dev_mesh(h);
    uint32_t *status = status_word(h);
    const int block = c->tune.block;
    const int dev = mesh_device(h);
    if (B.nm == 0) return GRIST_OK;
    if (c->tune.persistent) {
        int per_sm = 0;
        GRIST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tracer_persistent<TQ, TC>, block, 0));
        if (per_sm < 1) return GRIST_EUNSUPPORTED;
        const int grid = per_sm * sm_count(dev);
        DevMesh mm = m;
        Batch bb = B;
        unsigned *bar = c->barrier;
        GRIST_CUDA_TRY(cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st));
        void *args[] = {&mm, &bb, &bar, &status};
        GRIST_LAUNCH(h, PN("k_tracer_persistent"), st,
                     GRIST_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_tracer_persistent<TQ, TC>, grid, block,
                                                                args, 0, st)));
        return GRIST_OK;
    }
    static const char *names_f[] = {"k_tr_div/mix", "k_tr_edge/mix", "k_tr_update/mix", "k_tr_edge/mix",
                                    "k_tr_update/mix", "k_tr_edge/mix", "k_tr_update/mix", "k_tr_lowres/mix",
                                    "k_tr_ratios/mix", "k_tr_final/mix"};
    static const char *names_d[] = {"k_tr_div/fp64", "k_tr_edge/fp64", "k_tr_update/fp64", "k_tr_edge/fp64",
                                    "k_tr_update/fp64", "k_tr_edge/fp64", "k_tr_update/fp64", "k_tr_lowres/fp64",
                                    "k_tr_ratios/fp64", "k_tr_final/fp64"};
    const int sms = sm_count(dev);
    const bool fused = c->tune.fused != 0;
    if (fused) {
        int rc = build_tiles(h, c);
        if (rc != GRIST_OK) return rc;
    }
    const size_t tile_smem = (size_t)(c->tiles.Hmax + c->tiles.Emax) * 32 * sizeof(TC);
    auto launch_tile = [&](int stage) -> int {
        if (B.T.total == 0) return GRIST_OK;
        const unsigned grid = (unsigned)B.T.total;
        if (B.beta1) {
            GRIST_CUDA_TRY(cudaFuncSetAttribute(k_tr_tile_stage<TQ, TC, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
            GRIST_LAUNCH(h, sizeof(TC) == 4 ? "k_tr_tile_stage/mix" : "k_tr_tile_stage/fp64", st,
                         k_tr_tile_stage<TQ, TC, true><<<grid, 256, tile_smem, st>>>(m, c->tiles, B, stage, status));
        } else {
            GRIST_CUDA_TRY(cudaFuncSetAttribute(k_tr_tile_stage<TQ, TC, false>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
            GRIST_LAUNCH(h, sizeof(TC) == 4 ? "k_tr_tile_stage/mix" : "k_tr_tile_stage/fp64", st,
                         k_tr_tile_stage<TQ, TC, false><<<grid, 256, tile_smem, st>>>(m, c->tiles, B, stage, status));
        }
        return GRIST_OK;
    };
    for (int ph = P_DIV; ph < P_NPHASE; ph++) {
        if (!B.fct && ph > P_UPD2) break;
        if (B.fct && ph == P_UPD2) continue;
        if (fused && (ph == P_EDGE0 || ph == P_EDGE1 || (!B.fct && ph == P_EDGE2))) continue;
        if (fused && (ph == P_UPD0 || ph == P_UPD1 || ph == P_UPD2)) {
            const int rc = launch_tile(ph == P_UPD0 ? 0 : (ph == P_UPD1 ? 1 : 2));
            if (rc != GRIST_OK) return rc;
            continue;
        }
        const Space &S = (ph == P_DIV) ? B.D : ((ph == P_EDGE0 || ph == P_EDGE1 || ph == P_EDGE2) && !B.ring) ? B.E : B.C;
        long long want = (long long)((S.total + block - 1) / block);
        const long long cap = (long long)sms * 2048 * 32 / block;  // enough blocks to fill every SM many times
        const unsigned grid = (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
        const char *nm = sizeof(TC) == 4 ? names_f[ph] : names_d[ph];
        switch (ph) {
#define GRIST_PHASE_LAUNCH(P_, R_) \
        if (B.lpt == 2) GRIST_LAUNCH(h, nm, st, (k_tracer_phase<TQ, TC, P_, 2, R_><<<grid, block, 0, st>>>(m, B, status))); \
        else GRIST_LAUNCH(h, nm, st, (k_tracer_phase<TQ, TC, P_, 1, R_><<<grid, block, 0, st>>>(m, B, status)));
#define GRIST_PHASE_CASE(P_) \
    case P_:                                                                                                   \
        if constexpr (P_ == P_EDGE0 || P_ == P_EDGE1 || P_ == P_EDGE2) {                                       \
            if (B.ring) {                                                                                      \
                GRIST_PHASE_LAUNCH(P_, 1)                                                                      \
            } else {                                                                                           \
                GRIST_PHASE_LAUNCH(P_, 0)                                                                      \
            }                                                                                                  \
        } else {                                                                                               \
            GRIST_PHASE_LAUNCH(P_, 0)                                                                          \
        }                                                                                                      \
        break;
            GRIST_PHASE_CASE(P_DIV)
            GRIST_PHASE_CASE(P_EDGE0)
            GRIST_PHASE_CASE(P_UPD0)
            GRIST_PHASE_CASE(P_EDGE1)
            GRIST_PHASE_CASE(P_UPD1)
            GRIST_PHASE_CASE(P_EDGE2)
            GRIST_PHASE_CASE(P_UPD2)
            GRIST_PHASE_CASE(P_LOWRES)
            GRIST_PHASE_CASE(P_RATIOS)
            GRIST_PHASE_CASE(P_FINAL)
#undef GRIST_PHASE_CASE
#undef GRIST_PHASE_LAUNCH
        }
    }
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

// The step: the horizontal phases, then the vertical transport of every
// member that has a vertical mass flux (one launch per such member; the
// members' resolved descriptors are the host mirror of the device table).
template <typename TQ, typename TC>
int enqueue_step(grist_mesh_s *h, TracerCtx *c, const Batch &B, cudaStream_t st) {
    int rc = enqueue_horizontal<TQ, TC>(h, c, B, st);
    if (rc != GRIST_OK) return rc;
    const DevMesh &m = dev_mesh(h);
    const MemberDev *hm = reinterpret_cast<const MemberDev *>(c->tabs[c->cur].host.data());
    for (int j = 0; j < B.nm; j++) {
        if (!hm[j].Mv) continue;
        const unsigned gv = grid_for(m.nC, kVertWarps);
        if (hm[j].L <= 64)
            GRIST_LAUNCH(h, sizeof(TC) == 4 ? "k_tr_vertical/mix" : "k_tr_vertical/fp64", st,
                         (k_tr_vertical<TQ, TC, 2><<<gv, kVertWarps * 32, 0, st>>>(m, hm[j], B.dt, B.cmax,
                                                                                   status_word(h))));
        else
            GRIST_LAUNCH(h, sizeof(TC) == 4 ? "k_tr_vertical/mix" : "k_tr_vertical/fp64", st,
                         (k_tr_vertical<TQ, TC, kVertMaxL / 32><<<gv, kVertWarps * 32, 0, st>>>(
                             m, hm[j], B.dt, B.cmax, status_word(h))));
    }
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

// Build the tile tables of the mesh (once per handle) and upload them.
int build_tiles(grist_mesh_s *h, TracerCtx *c) {
    if (c->dtile) return GRIST_OK;
    const HostTables &ht = host_tables(h);
    const int nC = ht.nC;
    const int nt = (nC + kTileCells - 1) / kTileCells;
    std::vector<int> hoff(nt + 1, 0), eoff(nt + 1, 0), halo, tedge;
    std::vector<uint16_t> eloc, cle((size_t)nt * kTileCells * 6, 0);
    int Hmax = 0, Emax = 0;
    std::vector<int> cells, edges;
    for (int t = 0; t < nt; t++) {
        const int c0 = t * kTileCells, c1 = std::min(nC, c0 + kTileCells);
        edges.clear();
        for (int i = c0; i < c1; i++)
            for (int j = 0; j < 6; j++) edges.push_back(ht.eoc[(size_t)i * 6 + j]);
        std::sort(edges.begin(), edges.end());
        edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
        cells.clear();
        for (int e : edges) {
            cells.push_back(ht.coe[e].x);
            cells.push_back(ht.coe[e].y);
            for (int q = 0; q < 14; q++) cells.push_back(ht.d2i[(size_t)e * 14 + q]);
        }
        std::sort(cells.begin(), cells.end());
        cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
        if (cells.size() > 65535 || edges.size() > 65535) return GRIST_EUNSUPPORTED;
        auto loc = [&](int cell) {
            return (uint16_t)(std::lower_bound(cells.begin(), cells.end(), cell) - cells.begin());
        };
        for (int e : edges) {
            eloc.push_back(loc(ht.coe[e].x));
            eloc.push_back(loc(ht.coe[e].y));
            for (int q = 0; q < 14; q++) eloc.push_back(loc(ht.d2i[(size_t)e * 14 + q]));
        }
        for (int i = c0; i < c1; i++)
            for (int j = 0; j < 6; j++)
                cle[(size_t)i * 6 + j] = (uint16_t)(std::lower_bound(edges.begin(), edges.end(),
                                                                     ht.eoc[(size_t)i * 6 + j]) - edges.begin());
        halo.insert(halo.end(), cells.begin(), cells.end());
        tedge.insert(tedge.end(), edges.begin(), edges.end());
        hoff[t + 1] = (int)halo.size();
        eoff[t + 1] = (int)tedge.size();
        Hmax = std::max(Hmax, (int)cells.size());
        Emax = std::max(Emax, (int)edges.size());
    }
    size_t o = 0;
    const size_t o_hoff = o; o += al256(hoff.size() * 4);
    const size_t o_halo = o; o += al256(halo.size() * 4);
    const size_t o_eoff = o; o += al256(eoff.size() * 4);
    const size_t o_tedge = o; o += al256(tedge.size() * 4);
    const size_t o_eloc = o; o += al256(eloc.size() * 2);
    const size_t o_cle = o; o += al256(cle.size() * 2);
    std::vector<char> hb(o, 0);
    std::memcpy(hb.data() + o_hoff, hoff.data(), hoff.size() * 4);
    std::memcpy(hb.data() + o_halo, halo.data(), halo.size() * 4);
    std::memcpy(hb.data() + o_eoff, eoff.data(), eoff.size() * 4);
    std::memcpy(hb.data() + o_tedge, tedge.data(), tedge.size() * 4);
    std::memcpy(hb.data() + o_eloc, eloc.data(), eloc.size() * 2);
    std::memcpy(hb.data() + o_cle, cle.data(), cle.size() * 2);
    char *d = nullptr;
    if (cudaMalloc(&d, o) != cudaSuccess) return GRIST_ENOMEM;
    if (cudaMemcpy(d, hb.data(), o, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return GRIST_ECUDA;
    }
    c->dtile = d;
    TileMesh &T = c->tiles;
    T.ntiles = nt;
    T.Hmax = Hmax;
    T.Emax = Emax;
    T.hoff = (const int *)(d + o_hoff);
    T.halo = (const int *)(d + o_halo);
    T.eoff = (const int *)(d + o_eoff);
    T.tedge = (const int *)(d + o_tedge);
    T.eloc = (const uint16_t *)(d + o_eloc);
    T.cle = (const uint16_t *)(d + o_cle);
    return GRIST_OK;
}

TracerCtx *ctx_of(grist_mesh_s *h) {
    TracerCtx *&c = tracer_ctx(h);
    if (!c) c = new TracerCtx();
    return c;
}

template <typename TQ, typename TC>
int tracer_step_t(grist_mesh_s *h, const grist_tracer_batch *b, double dt, cudaStream_t st) {
    TracerCtx *c = ctx_of(h);
    const DevMesh &m = dev_mesh(h);
    HostPlan P;
    int rc = plan_batch<TQ, TC>(m, b, c->tune.tracers_per_thread, c->tune.persistent ? 1 : c->tune.levels_per_thread, P);
    if (rc != GRIST_OK) return rc;
    Batch B;
    rc = upload_plan<TQ, TC>(h, c, P, b, dt, B, st);
    if (rc != GRIST_OK) return rc;
    if (!c->tune.use_graph || profiling(h)) return enqueue_step<TQ, TC>(h, c, B, st);
    // graph path: signature = batch contents + tuning + dt + stream
    std::vector<unsigned long long> sig;
    sig.push_back((unsigned long long)b->prec);
    sig.push_back((unsigned long long)b->limiter);
    unsigned long long u;
    std::memcpy(&u, &b->beta_upwind, 8); sig.push_back(u);
    std::memcpy(&u, &dt, 8); sig.push_back(u);
    std::memcpy(&u, &b->vertical_courant_max, 8); sig.push_back(u);
    sig.push_back((unsigned long long)(uintptr_t)st);
    sig.push_back(((unsigned long long)c->tune.block << 32) | (unsigned)c->tune.tracers_per_thread);
    sig.push_back((unsigned long long)c->tune.persistent | ((unsigned long long)c->tune.levels_per_thread << 8) |
                  ((unsigned long long)c->tune.fused << 16) | ((unsigned long long)c->tune.cell_edges << 24));
    for (int i = 0; i < b->n_members; i++) {
        const grist_tracer_member &mm = b->members[i];
        sig.push_back((unsigned long long)(uintptr_t)mm.q);
        sig.push_back((unsigned long long)(uintptr_t)mm.dpi);
        sig.push_back((unsigned long long)(uintptr_t)mm.mass_flux);
        sig.push_back(((unsigned long long)mm.n_levels << 40) | ((unsigned long long)mm.n_tracers << 20) |
                      (unsigned long long)mm.ld);
        sig.push_back((unsigned long long)(uintptr_t)mm.vmass_flux);
        sig.push_back((unsigned long long)mm.ld_int);
    }
    sig.push_back((unsigned long long)(uintptr_t)c->tabs[c->cur].dev);
    // inside a caller's capture (a whole-step graph) the kernels are
    // recorded directly into that graph
    cudaStreamCaptureStatus cs;
    GRIST_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone || st == nullptr) return enqueue_step<TQ, TC>(h, c, B, st);
    for (auto &ge : c->graphs)
        if (ge.sig == sig) {
            GRIST_CUDA_TRY(cudaGraphLaunch(ge.exec, st));
            return GRIST_OK;
        }
    if (c->graph_failed && sig == c->failed_sig) return enqueue_step<TQ, TC>(h, c, B, st);
    GRIST_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int erc = enqueue_step<TQ, TC>(h, c, B, st);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (erc != GRIST_OK || ce != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        // this batch cannot be captured (e.g. the cooperative launch): run
        // it directly and remember not to retry the capture
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->graph_failed = true;
        c->failed_sig = sig;
        return enqueue_step<TQ, TC>(h, c, B, st);
    }
    if (c->graphs.size() >= kGraphCache) {
        // evict the oldest; its last replay may still be queued on a stream
        GRIST_CUDA_TRY(cudaDeviceSynchronize());
        cudaGraphExecDestroy(c->graphs.front().exec);
        cudaGraphDestroy(c->graphs.front().graph);
        c->graphs.erase(c->graphs.begin());
    }
    TracerCtx::GraphEntry ge;
    ge.sig = sig;
    ge.graph = g;
    ge.exec = ex;
    c->graphs.push_back(ge);
    GRIST_CUDA_TRY(cudaGraphLaunch(ex, st));
    return GRIST_OK;
}

int validate(const grist_tracer_batch *b, double dt) {
    if (!b || (b->n_members > 0 && !b->members) || b->n_members < 0) return GRIST_EINVAL;
    if (b->n_members > GRIST_MAX_MEMBERS) return GRIST_EUNSUPPORTED;
    if (!(dt > 0) || !std::isfinite(dt)) return GRIST_EINVAL;
    if (b->prec != GRIST_FP64 && b->prec != GRIST_MIX && b->prec != GRIST_MIX_DBL_MASS && b->prec != GRIST_MIX_DF)
        return GRIST_EINVAL;
    if (!std::isfinite(b->beta_upwind)) return GRIST_EINVAL;
    for (int i = 0; i < b->n_members; i++) {
        const grist_tracer_member &mb = b->members[i];
        if (mb.n_levels < 0 || mb.n_tracers < 0 || mb.n_levels > GRIST_MAXL || mb.ld < mb.n_levels) return GRIST_EINVAL;
        if (mb.n_levels > 0 && mb.n_tracers > 0 && (!mb.q || !mb.dpi || !mb.mass_flux)) return GRIST_EINVAL;
        if (mb.vmass_flux && mb.ld_int < mb.n_levels + 1) return GRIST_EINVAL;
        if (mb.vmass_flux && mb.n_levels > kVertMaxL) return GRIST_EUNSUPPORTED;
    }
    if (!(b->vertical_courant_max >= 0.0)) return GRIST_EINVAL;   // NaN and negatives; +inf: explicit only
    return GRIST_OK;
}

int dispatch(grist_mesh_s *h, const grist_tracer_batch *b, double dt, cudaStream_t st) {
    return b->prec == GRIST_FP64 ? tracer_step_t<double, double>(h, b, dt, st) : tracer_step_t<float, float>(h, b, dt, st);
}

int check_tuning(const grist_tracer_tuning *t) {
    if (!t) return GRIST_EINVAL;
    if (t->block < 64 || t->block > kTracerMaxBlock || t->block % 32) return GRIST_EINVAL;
    if (t->tracers_per_thread < 1 || t->tracers_per_thread > 64) return GRIST_EINVAL;
    if (t->persistent != 0 && t->persistent != 1) return GRIST_EINVAL;
    if (t->use_graph != 0 && t->use_graph != 1) return GRIST_EINVAL;
    if (t->fused != 0 && t->fused != 1) return GRIST_EINVAL;
    if (t->levels_per_thread != 1 && t->levels_per_thread != 2) return GRIST_EINVAL;
    if (t->cell_edges != 0 && t->cell_edges != 1) return GRIST_EINVAL;
    return GRIST_OK;
}

}  // namespace
}  // namespace grist

using namespace grist;

extern "C" int grist_tracer_step(grist_mesh h, const grist_tracer_batch *b, double dt, void *stream) {
    if (!h) return GRIST_EINVAL;
    int rc = validate(b, dt);
    if (rc != GRIST_OK) return rc;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    return dispatch(h, b, dt, (cudaStream_t)stream);
}

extern "C" int grist_selftest_bounded_wait(grist_mesh h, int64_t spin_limit, void *stream) {
    if (!h || spin_limit < 1 || spin_limit > 100000000) return GRIST_EINVAL;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    TracerCtx *c = ctx_of(h);
    if (!c->barrier) {
        if (cudaMalloc(&c->barrier, 4 * sizeof(unsigned)) != cudaSuccess) return GRIST_ENOMEM;
        GRIST_CUDA_TRY(cudaMemset(c->barrier, 0, 4 * sizeof(unsigned)));
    }
    // word 3 is written by no kernel; word 2 is cleared first so the wait
    // runs to its own limit
    cudaStream_t st = (cudaStream_t)stream;
    GRIST_CUDA_TRY(cudaMemsetAsync(c->barrier + 2, 0, sizeof(unsigned), st));
    k_wait_selftest<<<1, 32, 0, st>>>(c->barrier + 3, c->barrier + 2, (long long)spin_limit, status_word(h));
    return cudaGetLastError() == cudaSuccess ? GRIST_OK : GRIST_ECUDA;
}

extern "C" int grist_tracer_set_tuning(grist_mesh h, const grist_tracer_tuning *t) {
    if (!h) return GRIST_EINVAL;
    int rc = check_tuning(t);
    if (rc != GRIST_OK) return rc;
    TracerCtx *c = ctx_of(h);
    c->tune = *t;
    return GRIST_OK;
}

extern "C" int grist_tracer_get_tuning(grist_mesh h, grist_tracer_tuning *t) {
    if (!h || !t) return GRIST_EINVAL;
    *t = ctx_of(h)->tune;
    return GRIST_OK;
}

extern "C" int grist_tracer_autotune(grist_mesh h, const grist_tracer_batch *b, double dt, int32_t steps,
                                     void *stream, grist_tracer_tuning *best, double *best_ms) {
    if (!h || !best || steps < 1) return GRIST_EINVAL;
    int rc = validate(b, dt);
    if (rc != GRIST_OK) return rc;
    if (cudaSetDevice(mesh_device(h)) != cudaSuccess) return GRIST_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    TracerCtx *c = ctx_of(h);
    const grist_tracer_tuning saved = c->tune;
    const DevMesh &m = dev_mesh(h);
    // private copies of the tracers
    std::vector<grist_tracer_member> mem(b->members, b->members + b->n_members);
    std::vector<void *> copies;
    const size_t es = b->prec == GRIST_FP64 ? 8 : 4;
    int maxT = 1;
    for (auto &mb : mem) {
        if (mb.n_levels == 0 || mb.n_tracers == 0) continue;
        maxT = mb.n_tracers > maxT ? mb.n_tracers : maxT;
        const size_t bytes = (size_t)mb.n_tracers * m.nC * mb.ld * es;
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            for (void *q : copies) cudaFree(q);
            return GRIST_ENOMEM;
        }
        cudaMemcpyAsync(p, mb.q, bytes, cudaMemcpyDeviceToDevice, st);
        copies.push_back(p);
        mb.q = p;
    }
    grist_tracer_batch bb = *b;
    bb.members = mem.data();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_cfg = [&](const grist_tracer_tuning &t, double *ms) -> int {
        c->tune = t;
        int r = dispatch(h, &bb, dt, st);  // warm-up (and graph capture)
        if (r != GRIST_OK) return r;
        cudaEventRecord(e0, st);
        for (int i = 0; i < steps; i++) {
            r = dispatch(h, &bb, dt, st);
            if (r != GRIST_OK) return r;
        }
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return GRIST_ECUDA;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f / steps;
        return GRIST_OK;
    };
    grist_tracer_tuning bestt = saved;
    double bestms = 1e300;
    const int blocks[] = {128, 256, 512};
    const int tpts[] = {1, 2, 4, 8};
    for (int fu = 0; fu <= 1; fu++) {
        for (int bl : blocks) {
            for (int tp : tpts) {
                if (tp > 1 && tp / 2 >= maxT) continue;
                grist_tracer_tuning t{bl, tp, 0, 0, fu, 1, 1};
                double ms = 0;
                if (time_cfg(t, &ms) == GRIST_OK && ms < bestms) { bestms = ms; bestt = t; }
            }
        }
    }
    // two levels per thread (work-list phases) at the best tracers per
    // thread, every block size
    {
        const int tp = bestt.tracers_per_thread, fu = bestt.fused;
        for (int bl : blocks) {
            grist_tracer_tuning t{bl, tp, 0, 0, fu, 2, 1};
            double ms = 0;
            if (time_cfg(t, &ms) == GRIST_OK && ms < bestms) { bestms = ms; bestt = t; }
        }
    }
    // the edge-centric form of the edge fluxes at the best so far
    {
        grist_tracer_tuning t = bestt;
        t.cell_edges = 0;
        double ms = 0;
        if (time_cfg(t, &ms) == GRIST_OK && ms < bestms) { bestms = ms; bestt = t; }
    }
    for (int pers = 0; pers <= 1; pers++) {
        for (int gr = 0; gr <= 1; gr++) {
            if (pers == 0 && gr == 0) continue;
            grist_tracer_tuning t = bestt;
            t.persistent = pers;
            t.use_graph = gr;
            if (pers) {
                t.fused = 0;
                t.levels_per_thread = 1;
            }
            double ms = 0;
            if (time_cfg(t, &ms) == GRIST_OK && ms < bestms) { bestms = ms; bestt = t; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    for (void *q : copies) cudaFree(q);
    // the cached graphs may refer to the freed copies: drop them
    c->drop_graphs();
    c->tune = bestt;
    *best = bestt;
    if (best_ms) *best_ms = bestms;
    uint32_t flags = 0;
    cudaMemcpy(&flags, status_word(h), sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (flags & GRIST_FLAG_TIMEOUT) return GRIST_ETIMEOUT;
    return GRIST_OK;
}
