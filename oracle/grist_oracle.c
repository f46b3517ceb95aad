/*
 * grist_oracle.c - plain, slow, FP64 CPU oracle of the GRIST hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code with the CUDA library.
 *
 * Written from the paper's statement of the method (arXiv 2404.08849):
 *   Sec. 2.1  : hexagonal Arakawa-C grid, RK + Mesinger forward-backward
 *               hydrostatic solver, HEVI non-hydrostatic solver, tracer
 *               transport split from the dycore with a third-order upwind
 *               flux and the Flux-Corrected-Transport limiter.
 *   Eqs. 3-10 : continuity (3), theta_m transport (4), momentum (5),
 *               w (6), phi (7), hydrostatic relation (8), equation of
 *               state (9), tracer transport (10).
 *   Sec. 2.3  : precision semantics (the oracle is all-FP64).
 * The paper defers every discrete operator to Zhang et al. (2019, 2020);
 * the discrete forms below are the readings listed in the design notes
 * (TRiSK-family C-grid operators, Skamarock-Gassmann third-order flux,
 * Zalesak FCT, Wicker-Skamarock RK3).
 *
 * Layout: every field is [entity][level] (level innermost, leading dimension
 * = number of levels); interface fields are [cell][L+1], interface 0 at the
 * model top.  Entities are in the mesh generator's original numbering.
 * Loops are scalar and ordered; OpenMP only splits independent entity loops
 * (each output element is written by exactly one iteration).
 *
 * Parity status: every function here is pinned by tests (invariants,
 * closed forms, library routines) - see the test suite.  The whole-dycore
 * solution against a true solution is not pinned (no analytic solution);
 * only its invariants are.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXE 6
#define MAXEOE 10
#define D2P 7

typedef struct {
    int32_t nC, nE, nV;
    double radius;
    const double *cell_area, *vertex_area, *dc, *dv, *f_vertex;
    const int32_t *cells_on_edge, *vertices_on_edge, *n_edges_on_cell, *edges_on_cell,
        *cells_on_cell, *edges_on_vertex, *cells_on_vertex;
    const double *edge_sign_on_cell, *edge_sign_on_vertex, *kite_area;
    const int32_t *n_edges_on_edge, *edges_on_edge;
    const double *trisk_weight;
    const int32_t *d2_stencil;
    const double *d2_coef;
} orc_mesh;

typedef struct {
    int32_t L;
    double pi_top, p0, rd, cp, g, beta; /* beta: off-centring weight of the implicit terms */
    const double *b_int;                /* [L+1], 0 at top, 1 at the surface */
    const double *phi_s;                /* [nC] surface geopotential */
} orc_params;

static void *xalloc(size_t n) {
    void *p = calloc(n ? n : 1, 1);
    return p;
}

/* ------------------------------------------------------------------------
 * Basic C-grid operators (Sec. 2.1: Arakawa-C staggering; TRiSK family)
 * ---------------------------------------------------------------------- */

/* Cell divergence of an edge flux: D_i = (1/A_i) sum_e s(e,i) dv_e F_e. */
void orc_divergence(const orc_mesh *m, int L, const double *F, double *out) {
#pragma omp parallel for
    for (int i = 0; i < m->nC; i++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->n_edges_on_cell[i]; j++) {
                int e = m->edges_on_cell[i * MAXE + j];
                s += m->edge_sign_on_cell[i * MAXE + j] * m->dv[e] * F[(size_t)e * L + k];
            }
            out[(size_t)i * L + k] = s / m->cell_area[i];
        }
    }
}

/* Edge gradient of a cell field: (h(c2) - h(c1)) / dc_e. */
void orc_gradient(const orc_mesh *m, int L, const double *h, double *out) {
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
        for (int k = 0; k < L; k++)
            out[(size_t)e * L + k] = (h[(size_t)c2 * L + k] - h[(size_t)c1 * L + k]) / m->dc[e];
    }
}

/* Vertex relative vorticity: zeta_v = (1/A_v) sum_e t(e,v) dc_e u_e. */
void orc_vorticity(const orc_mesh *m, int L, const double *u, double *out) {
#pragma omp parallel for
    for (int v = 0; v < m->nV; v++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < 3; j++) {
                int e = m->edges_on_vertex[3 * v + j];
                s += m->edge_sign_on_vertex[3 * v + j] * m->dc[e] * u[(size_t)e * L + k];
            }
            out[(size_t)v * L + k] = s / m->vertex_area[v];
        }
    }
}

/* Kite-weighted cell -> vertex remap: x_v = (1/A_v) sum_i kite(i,v) x_i. */
void orc_cell_to_vertex(const orc_mesh *m, int L, const double *x, double *out) {
#pragma omp parallel for
    for (int v = 0; v < m->nV; v++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < 3; j++)
                s += m->kite_area[3 * v + j] * x[(size_t)m->cells_on_vertex[3 * v + j] * L + k];
            out[(size_t)v * L + k] = s / m->vertex_area[v];
        }
    }
}

/* Cell kinetic energy: K_i = (1/A_i) sum_e (1/4) dc_e dv_e u_e^2. */
void orc_kinetic_energy(const orc_mesh *m, int L, const double *u, double *out) {
#pragma omp parallel for
    for (int i = 0; i < m->nC; i++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->n_edges_on_cell[i]; j++) {
                int e = m->edges_on_cell[i * MAXE + j];
                double ue = u[(size_t)e * L + k];
                s += 0.25 * m->dc[e] * m->dv[e] * ue * ue;
            }
            out[(size_t)i * L + k] = s / m->cell_area[i];
        }
    }
}

/* Tangential (perpendicular) mass flux at edges, TRiSK reconstruction:
 * Fperp_e = (1/dc_e) sum_e' w(e,e') dv_e' F_e'. */
void orc_perp_flux(const orc_mesh *m, int L, const double *F, double *out) {
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->n_edges_on_edge[e]; j++) {
                int e2 = m->edges_on_edge[e * MAXEOE + j];
                s += m->trisk_weight[e * MAXEOE + j] * m->dv[e2] * F[(size_t)e2 * L + k];
            }
            out[(size_t)e * L + k] = s / m->dc[e];
        }
    }
}

/* Potential-vorticity flux term of Eq. 5 (zeta_p dpi u_t), energy-neutral
 * form: (1/dc_e) sum_e' w(e,e') dv_e' F_e' (q_e + q_e')/2 with q_e the mean
 * of the PV at the edge's two vertices.  Returned as +tendency of u_n
 * (d u_n / dt = + zeta_a u_t with t = k x n). */
void orc_pv_flux(const orc_mesh *m, int L, const double *F, const double *qv, double *out) {
    double *qe = (double *)xalloc(sizeof(double) * (size_t)m->nE * L);
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        int v1 = m->vertices_on_edge[2 * e], v2 = m->vertices_on_edge[2 * e + 1];
        for (int k = 0; k < L; k++)
            qe[(size_t)e * L + k] = 0.5 * (qv[(size_t)v1 * L + k] + qv[(size_t)v2 * L + k]);
    }
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->n_edges_on_edge[e]; j++) {
                int e2 = m->edges_on_edge[e * MAXEOE + j];
                s += m->trisk_weight[e * MAXEOE + j] * m->dv[e2] * F[(size_t)e2 * L + k] * 0.5 *
                     (qe[(size_t)e * L + k] + qe[(size_t)e2 * L + k]);
            }
            out[(size_t)e * L + k] = s / m->dc[e];
        }
    }
    free(qe);
}

/* ------------------------------------------------------------------------
 * Third-order upwind edge flux (Sec. 2.1: "third-order upwind flux
 * operator").  Normal second derivative of q at each side of the edge from
 * the deriv-two stencil: q''_s = sum_j D(e,s,j) q(stencil_j).  Edge value
 *   q_e = (q1+q2)/2 - (dc^2/12)(q''_1 + q''_2)
 *         + sgn(F) beta (dc^2/12)(q''_2 - q''_1),
 * flux = F_e q_e.  beta = 1 gives the pure third-order scheme; beta = 0 the
 * fourth-order centred one.
 * ---------------------------------------------------------------------- */
void orc_edge_flux_3rd(const orc_mesh *m, int L, const double *q, const double *F, double beta,
                       double *out) {
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
        double dc2 = m->dc[e] * m->dc[e] / 12.0;
        for (int k = 0; k < L; k++) {
            double d[2];
            for (int s = 0; s < 2; s++) {
                double acc = 0.0;
                for (int j = 0; j < D2P; j++) {
                    int c = m->d2_stencil[(e * 2 + s) * D2P + j];
                    if (c < 0) continue;
                    acc += m->d2_coef[(e * 2 + s) * D2P + j] * q[(size_t)c * L + k];
                }
                d[s] = acc;
            }
            double f = F[(size_t)e * L + k];
            double sgn = f >= 0.0 ? 1.0 : -1.0;
            double qe = 0.5 * (q[(size_t)c1 * L + k] + q[(size_t)c2 * L + k]) - dc2 * (d[0] + d[1]) +
                        sgn * beta * dc2 * (d[1] - d[0]);
            out[(size_t)e * L + k] = f * qe;
        }
    }
}

/* ------------------------------------------------------------------------
 * Tracer transport, Eq. 10 (horizontal part), Sec. 2.1.
 * Wicker-Skamarock RK3 (dt/3, dt/2, dt).  Layer mass at stage s follows the
 * tracer solver's own continuity with the same (time-mean) mass flux:
 *   dpi^(s) = dpi^n - dt_s * div(F),
 * so a constant q stays constant.  Stage update:
 *   q^(s) = (dpi^n q^n - dt_s div(F q_e(q^(s-1)))) / dpi^(s).
 * FCT (Zalesak) on the final stage only when fct != 0:
 *   F^L = F * q^n(upwind); A = F^H - F^L; q^td from F^L;
 *   q^max/min over the cell and its neighbours of {q^n, q^td};
 *   P+ = dt/A_i sum l max(0, -s A), P- = dt/A_i sum l max(0, s A),
 *   Q+ = (q^max - q^td) dpi^(3), Q- = (q^td - q^min) dpi^(3),
 *   R+- = min(1, Q/(P + TINY));  C_e = min(R-(c1), R+(c2)) if A >= 0 else
 *   min(R+(c1), R-(c2));  final update with F^L + C A.
 * q: [T][nC][L] in/out; dpi: [nC][L]; F: [nE][L].
 * ---------------------------------------------------------------------- */
void orc_tracer_step(const orc_mesh *m, int L, int T, double *q, const double *dpi,
                     const double *F, double dt, double beta, int fct) {
    size_t nCL = (size_t)m->nC * L, nEL = (size_t)m->nE * L;
    double *divF = (double *)xalloc(sizeof(double) * nCL);
    double *dpis = (double *)xalloc(sizeof(double) * nCL * 3);
    double *qs = (double *)xalloc(sizeof(double) * nCL);
    double *qnew = (double *)xalloc(sizeof(double) * nCL);
    double *FH = (double *)xalloc(sizeof(double) * nEL);
    double *divH = (double *)xalloc(sizeof(double) * nCL);
    double *FL = (double *)xalloc(sizeof(double) * nEL);
    double *AE = (double *)xalloc(sizeof(double) * nEL);
    double *qtd = (double *)xalloc(sizeof(double) * nCL);
    double *divL = (double *)xalloc(sizeof(double) * nCL);
    double *Rp = (double *)xalloc(sizeof(double) * nCL);
    double *Rm = (double *)xalloc(sizeof(double) * nCL);
    double *FC = (double *)xalloc(sizeof(double) * nEL);
    const double dts[3] = {dt / 3.0, dt / 2.0, dt};

    orc_divergence(m, L, F, divF);
    for (int s = 0; s < 3; s++)
        for (size_t x = 0; x < nCL; x++) dpis[s * nCL + x] = dpi[x] - dts[s] * divF[x];

    for (int t = 0; t < T; t++) {
        double *qn = q + (size_t)t * nCL;
        memcpy(qs, qn, sizeof(double) * nCL);
        for (int s = 0; s < 3; s++) {
            orc_edge_flux_3rd(m, L, qs, F, beta, FH);
            const double *dpn = dpis + s * nCL;
            if (s < 2 || !fct) {
                orc_divergence(m, L, FH, divH);
                for (size_t x = 0; x < nCL; x++)
                    qnew[x] = (dpi[x] * qn[x] - dts[s] * divH[x]) / dpn[x];
                memcpy(qs, qnew, sizeof(double) * nCL);
                continue;
            }
            /* FCT, final stage */
#pragma omp parallel for
            for (int e = 0; e < m->nE; e++) {
                int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
                for (int k = 0; k < L; k++) {
                    double f = F[(size_t)e * L + k];
                    double qu = f >= 0.0 ? qn[(size_t)c1 * L + k] : qn[(size_t)c2 * L + k];
                    FL[(size_t)e * L + k] = f * qu;
                    AE[(size_t)e * L + k] = FH[(size_t)e * L + k] - FL[(size_t)e * L + k];
                }
            }
            orc_divergence(m, L, FL, divL);
            for (size_t x = 0; x < nCL; x++) qtd[x] = (dpi[x] * qn[x] - dt * divL[x]) / dpn[x];
#pragma omp parallel for
            for (int i = 0; i < m->nC; i++) {
                for (int k = 0; k < L; k++) {
                    size_t x = (size_t)i * L + k;
                    double qmax = fmax(qn[x], qtd[x]), qmin = fmin(qn[x], qtd[x]);
                    double pp = 0.0, pm = 0.0;
                    for (int j = 0; j < m->n_edges_on_cell[i]; j++) {
                        int nb = m->cells_on_cell[i * MAXE + j];
                        size_t y = (size_t)nb * L + k;
                        qmax = fmax(qmax, fmax(qn[y], qtd[y]));
                        qmin = fmin(qmin, fmin(qn[y], qtd[y]));
                        int e = m->edges_on_cell[i * MAXE + j];
                        double out = m->edge_sign_on_cell[i * MAXE + j] * AE[(size_t)e * L + k];
                        pp += m->dv[e] * fmax(0.0, -out);
                        pm += m->dv[e] * fmax(0.0, out);
                    }
                    pp *= dt / m->cell_area[i];
                    pm *= dt / m->cell_area[i];
                    double Qp = (qmax - qtd[x]) * dpn[x];
                    double Qm = (qtd[x] - qmin) * dpn[x];
                    Rp[x] = fmin(1.0, Qp / (pp + DBL_MIN));
                    Rm[x] = fmin(1.0, Qm / (pm + DBL_MIN));
                }
            }
#pragma omp parallel for
            for (int e = 0; e < m->nE; e++) {
                int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
                for (int k = 0; k < L; k++) {
                    size_t x = (size_t)e * L + k;
                    double a = AE[x];
                    double c = a >= 0.0 ? fmin(Rm[(size_t)c1 * L + k], Rp[(size_t)c2 * L + k])
                                        : fmin(Rp[(size_t)c1 * L + k], Rm[(size_t)c2 * L + k]);
                    FC[x] = FL[x] + c * a;
                }
            }
            orc_divergence(m, L, FC, divH);
            for (size_t x = 0; x < nCL; x++) qnew[x] = (dpi[x] * qn[x] - dt * divH[x]) / dpn[x];
            memcpy(qs, qnew, sizeof(double) * nCL);
        }
        memcpy(qn, qs, sizeof(double) * nCL);
    }
    free(divF); free(dpis); free(qs); free(qnew); free(FH); free(divH); free(FL); free(AE);
    free(qtd); free(divL); free(Rp); free(Rm); free(FC);
}

/* ------------------------------------------------------------------------
 * Dycore pieces
 * ---------------------------------------------------------------------- */

/* Layer mass thickness from the sigma-mass coordinate (Sec. 2.1 hybrid
 * sigma-mass; pure-sigma reading): pi_{k+1/2} = pi_t + B_{k+1/2}(ps - pi_t),
 * dpi_k = pi_{k+1/2} - pi_{k-1/2}. */
static void layer_mass(const orc_params *P, int nC, const double *ps, double *dpi) {
    int L = P->L;
    for (int i = 0; i < nC; i++)
        for (int k = 0; k < L; k++)
            dpi[(size_t)i * L + k] = (P->pi_top + P->b_int[k + 1] * (ps[i] - P->pi_top)) -
                                     (P->pi_top + P->b_int[k] * (ps[i] - P->pi_top));
}

/* Continuity, Eq. 3 (flux form): F_e = dpi_e u_e with dpi_e the mean of the
 * two cells; D_i,k = div(F); ps tendency = -(1/A_i) sum_e s dv (sum_k F_e,k);
 * vertical mass flux at interfaces from the layer continuity equation
 *   M_{k+1/2} = -B_{k+1/2} dps/dt - sum_{l<=k} D_l,  M_top = M_surf = 0
 * (positive downward, towards larger pi). */
void orc_mass(const orc_mesh *m, const orc_params *P, const double *ps, const double *u,
              double *dpi, double *F, double *D, double *ps_tend, double *M) {
    int L = P->L;
    layer_mass(P, m->nC, ps, dpi);
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
        for (int k = 0; k < L; k++)
            F[(size_t)e * L + k] =
                0.5 * (dpi[(size_t)c1 * L + k] + dpi[(size_t)c2 * L + k]) * u[(size_t)e * L + k];
    }
    orc_divergence(m, L, F, D);
#pragma omp parallel for
    for (int i = 0; i < m->nC; i++) {
        double s = 0.0;
        for (int j = 0; j < m->n_edges_on_cell[i]; j++) {
            int e = m->edges_on_cell[i * MAXE + j];
            double col = 0.0;
            for (int k = 0; k < L; k++) col += F[(size_t)e * L + k];
            s += m->edge_sign_on_cell[i * MAXE + j] * m->dv[e] * col;
        }
        ps_tend[i] = -s / m->cell_area[i];
        double acc = 0.0;
        M[(size_t)i * (L + 1)] = 0.0;
        for (int k = 0; k < L; k++) {
            acc += D[(size_t)i * L + k];
            M[(size_t)i * (L + 1) + k + 1] = -P->b_int[k + 1] * ps_tend[i] - acc;
        }
        M[(size_t)i * (L + 1) + L] = 0.0;
    }
}

/* theta_m tendency, Eq. 4: horizontal third-order upwind flux of theta =
 * (dpi theta)/dpi with the mass flux F, vertical flux M_{k+1/2} times the
 * mean of the two adjacent layers' theta. */
void orc_theta_tend(const orc_mesh *m, int L, const double *dpi_theta, const double *dpi,
                    const double *F, const double *M, double beta, double *tend) {
    size_t nCL = (size_t)m->nC * L;
    double *th = (double *)xalloc(sizeof(double) * nCL);
    double *FT = (double *)xalloc(sizeof(double) * (size_t)m->nE * L);
    double *dv = (double *)xalloc(sizeof(double) * nCL);
    for (size_t x = 0; x < nCL; x++) th[x] = dpi_theta[x] / dpi[x];
    orc_edge_flux_3rd(m, L, th, F, beta, FT);
    orc_divergence(m, L, FT, dv);
#pragma omp parallel for
    for (int i = 0; i < m->nC; i++) {
        for (int k = 0; k < L; k++) {
            double top = 0.0, bot = 0.0;
            if (k > 0)
                top = M[(size_t)i * (L + 1) + k] * 0.5 * (th[(size_t)i * L + k - 1] + th[(size_t)i * L + k]);
            if (k < L - 1)
                bot = M[(size_t)i * (L + 1) + k + 1] * 0.5 *
                      (th[(size_t)i * L + k] + th[(size_t)i * L + k + 1]);
            tend[(size_t)i * L + k] = -dv[(size_t)i * L + k] - (bot - top);
        }
    }
    free(th); free(FT); free(dv);
}

/* Hydrostatic diagnostics (Eq. 8 with p = pi): mid-layer pressure
 * p_k = (pi_{k-1/2} + pi_{k+1/2})/2, Exner (p/p0)^kappa, specific volume
 * alpha_k = Rd theta_k (p_k/p0)^kappa / p_k, geopotential integrated upward
 * from phi_s: phi_{k-1/2} = phi_{k+1/2} + alpha_k dpi_k; layer phi = mean of
 * its interfaces.  Outputs p, alpha, phi_layer [nC][L]; phi_int [nC][L+1]. */
void orc_hydro_diag(const orc_params *P, int nC, const double *ps, const double *dpi_theta,
                    double *p, double *alpha, double *phi_layer, double *phi_int) {
    int L = P->L;
    double kappa = P->rd / P->cp;
#pragma omp parallel for
    for (int i = 0; i < nC; i++) {
        phi_int[(size_t)i * (L + 1) + L] = P->phi_s[i];
        for (int k = L - 1; k >= 0; k--) {
            double pt = P->pi_top + P->b_int[k] * (ps[i] - P->pi_top);
            double pb = P->pi_top + P->b_int[k + 1] * (ps[i] - P->pi_top);
            double dp = pb - pt;
            double pk = 0.5 * (pt + pb);
            double th = dpi_theta[(size_t)i * L + k] / dp;
            double a = P->rd * th * pow(pk / P->p0, kappa) / pk;
            p[(size_t)i * L + k] = pk;
            alpha[(size_t)i * L + k] = a;
            phi_int[(size_t)i * (L + 1) + k] = phi_int[(size_t)i * (L + 1) + k + 1] + a * dp;
            phi_layer[(size_t)i * L + k] =
                0.5 * (phi_int[(size_t)i * (L + 1) + k] + phi_int[(size_t)i * (L + 1) + k + 1]);
        }
    }
}

/* Equation of state, Eq. 9, with dphi_k = phi_{k-1/2} - phi_{k+1/2} > 0
 * (the paper's dphi runs along increasing pi, hence its minus sign):
 * p_k = p0 (Rd dpi_theta_k / (p0 dphi_k))^gamma, gamma = cp/(cp - Rd). */
void orc_eos(const orc_params *P, int nC, const double *dpi_theta, const double *phi, double *p) {
    int L = P->L;
    double gam = P->cp / (P->cp - P->rd);
#pragma omp parallel for
    for (int i = 0; i < nC; i++)
        for (int k = 0; k < L; k++) {
            double dphi = phi[(size_t)i * (L + 1) + k] - phi[(size_t)i * (L + 1) + k + 1];
            p[(size_t)i * L + k] = P->p0 * pow(P->rd * dpi_theta[(size_t)i * L + k] / (P->p0 * dphi), gam);
        }
}

/* Momentum tendency, Eq. 5.
 *   du/dt = PV flux (zeta_p dpi u_t term)
 *           - (K(c2) - K(c1))/dc                                 (dKE/dn)
 *           - [M_{k+1/2}(u_{k+1}-u_k) + M_{k-1/2}(u_k-u_{k-1})]/(2 dpi_e,k)
 *                                                    (eta-dot du/deta)
 *           - alpha_e (p(c2) - p(c1))/dc - dpdpi_e (phi(c2) - phi(c1))/dc
 *                                        (pressure gradient and gravity)
 * with M, dpi at edges the mean of the two cells and alpha_e, dpdpi_e the
 * mean of the two cells' layer values (dpdpi = 1 in the hydrostatic case).
 * zeta_p = (zeta + f)/dpi_v with the kite-remapped vertex mass (Sec. 2.3:
 * zeta_p is highly sensitive to the precision of dpi). */
void orc_momentum_tend(const orc_mesh *m, int L, const double *u, const double *dpi,
                       const double *F, const double *M, const double *p, const double *alpha,
                       const double *phi_layer, const double *dpdpi, double *tend) {
    size_t nVL = (size_t)m->nV * L, nCL = (size_t)m->nC * L, nEL = (size_t)m->nE * L;
    double *zeta = (double *)xalloc(sizeof(double) * nVL);
    double *dpv = (double *)xalloc(sizeof(double) * nVL);
    double *K = (double *)xalloc(sizeof(double) * nCL);
    double *pv = (double *)xalloc(sizeof(double) * nEL);
    orc_vorticity(m, L, u, zeta);
    orc_cell_to_vertex(m, L, dpi, dpv);
    for (int v = 0; v < m->nV; v++)
        for (int k = 0; k < L; k++) {
            size_t x = (size_t)v * L + k;
            zeta[x] = (zeta[x] + m->f_vertex[v]) / dpv[x];
        }
    orc_kinetic_energy(m, L, u, K);
    orc_pv_flux(m, L, F, zeta, pv);
#pragma omp parallel for
    for (int e = 0; e < m->nE; e++) {
        int c1 = m->cells_on_edge[2 * e], c2 = m->cells_on_edge[2 * e + 1];
        double rdc = 1.0 / m->dc[e];
        for (int k = 0; k < L; k++) {
            size_t x = (size_t)e * L + k;
            size_t a1 = (size_t)c1 * L + k, a2 = (size_t)c2 * L + k;
            double ke = (K[a2] - K[a1]) * rdc;
            double dpe = 0.5 * (dpi[a1] + dpi[a2]);
            double va = 0.0;
            if (k < L - 1) {
                double Mb = 0.5 * (M[(size_t)c1 * (L + 1) + k + 1] + M[(size_t)c2 * (L + 1) + k + 1]);
                va += Mb * (u[x + 1] - u[x]);
            }
            if (k > 0) {
                double Mt = 0.5 * (M[(size_t)c1 * (L + 1) + k] + M[(size_t)c2 * (L + 1) + k]);
                va += Mt * (u[x] - u[x - 1]);
            }
            va /= 2.0 * dpe;
            double ae = 0.5 * (alpha[a1] + alpha[a2]);
            double de = dpdpi ? 0.5 * (dpdpi[a1] + dpdpi[a2]) : 1.0;
            double pgf = -ae * (p[a2] - p[a1]) * rdc - de * (phi_layer[a2] - phi_layer[a1]) * rdc;
            tend[x] = pv[x] - ke - va + pgf;
        }
    }
    free(zeta); free(dpv); free(K); free(pv);
}

/* ------------------------------------------------------------------------
 * Hydrostatic dycore step (Sec. 2.1: Runge-Kutta + Mesinger forward-
 * backward, fully explicit).  Wicker-Skamarock RK3; inside each stage the
 * mass (Eq. 3) and theta (Eq. 4) are advanced first, the diagnostics
 * (Eq. 8) are taken from the new-stage mass and theta, then the momentum
 * (Eq. 5) uses the stage-input wind for its advective terms and the new
 * pressure / geopotential for the pressure-gradient and gravity terms.
 * The final stage's mass flux is added to flux_accum (time-mean flux for
 * the tracer solver), its vertical mass flux M [nC][L+1] (the delta(M q)
 * flux of Eq. 10) to vflux_accum when given, and *accum_weight is
 * incremented.
 * ps [nC], u [nE][L], dpi_theta [nC][L]: in/out.
 * ---------------------------------------------------------------------- */
void orc_dycore_step_hydro(const orc_mesh *m, const orc_params *P, double *ps, double *u,
                           double *dpi_theta, double *flux_accum, double *vflux_accum,
                           double *accum_weight, double dt) {
    int L = P->L;
    size_t nC = m->nC, nCL = nC * L, nEL = (size_t)m->nE * L;
    double *ps_n = (double *)xalloc(sizeof(double) * nC), *u_n = (double *)xalloc(sizeof(double) * nEL),
           *th_n = (double *)xalloc(sizeof(double) * nCL);
    double *dpi = (double *)xalloc(sizeof(double) * nCL), *dpi_new = (double *)xalloc(sizeof(double) * nCL);
    double *F = (double *)xalloc(sizeof(double) * nEL), *D = (double *)xalloc(sizeof(double) * nCL);
    double *pst = (double *)xalloc(sizeof(double) * nC), *M = (double *)xalloc(sizeof(double) * nC * (L + 1));
    double *tht = (double *)xalloc(sizeof(double) * nCL);
    double *p = (double *)xalloc(sizeof(double) * nCL), *al = (double *)xalloc(sizeof(double) * nCL),
           *phl = (double *)xalloc(sizeof(double) * nCL), *phi = (double *)xalloc(sizeof(double) * nC * (L + 1));
    double *ut = (double *)xalloc(sizeof(double) * nEL);
    double *ps_s = (double *)xalloc(sizeof(double) * nC), *u_s = (double *)xalloc(sizeof(double) * nEL),
           *th_s = (double *)xalloc(sizeof(double) * nCL);
    const double dts[3] = {dt / 3.0, dt / 2.0, dt};
    memcpy(ps_n, ps, sizeof(double) * nC);
    memcpy(u_n, u, sizeof(double) * nEL);
    memcpy(th_n, dpi_theta, sizeof(double) * nCL);
    memcpy(ps_s, ps, sizeof(double) * nC);
    memcpy(u_s, u, sizeof(double) * nEL);
    memcpy(th_s, dpi_theta, sizeof(double) * nCL);
    for (int s = 0; s < 3; s++) {
        orc_mass(m, P, ps_s, u_s, dpi, F, D, pst, M);
        orc_theta_tend(m, L, th_s, dpi, F, M, 1.0, tht);
        for (size_t i = 0; i < nC; i++) ps[i] = ps_n[i] + dts[s] * pst[i];
        for (size_t x = 0; x < nCL; x++) dpi_theta[x] = th_n[x] + dts[s] * tht[x];
        orc_hydro_diag(P, m->nC, ps, dpi_theta, p, al, phl, phi);
        orc_momentum_tend(m, L, u_s, dpi, F, M, p, al, phl, NULL, ut);
        for (size_t x = 0; x < nEL; x++) u[x] = u_n[x] + dts[s] * ut[x];
        if (s == 2 && flux_accum) {
            for (size_t x = 0; x < nEL; x++) flux_accum[x] += F[x];
            if (accum_weight) *accum_weight += 1.0;
        }
        if (s == 2 && vflux_accum)
            for (size_t x = 0; x < nC * (L + 1); x++) vflux_accum[x] += M[x];
        memcpy(ps_s, ps, sizeof(double) * nC);
        memcpy(u_s, u, sizeof(double) * nEL);
        memcpy(th_s, dpi_theta, sizeof(double) * nCL);
    }
    (void)dpi_new;
    free(ps_n); free(u_n); free(th_n); free(dpi); free(dpi_new); free(F); free(D); free(pst); free(M);
    free(tht); free(p); free(al); free(phl); free(phi); free(ut); free(ps_s); free(u_s); free(th_s);
}

/* ------------------------------------------------------------------------
 * Non-hydrostatic pieces (Eqs. 6, 7, 9; Sec. 2.1 HEVI)
 * ---------------------------------------------------------------------- */

/* Horizontal advection V.grad(x) of an interface field x [nC][L+1]
 * (advective form): (1/A_i) sum_e s(e,i) dv_e u_e^int (x(nbr) - x(i))/2,
 * with u at interfaces the mean of the two adjacent layers (top and bottom
 * interfaces take the nearest layer). */
void orc_interface_hadv(const orc_mesh *m, int L, const double *u, const double *x, double *out) {
    int Li = L + 1;
#pragma omp parallel for
    for (int i = 0; i < m->nC; i++) {
        for (int k = 0; k < Li; k++) {
            double s = 0.0;
            for (int j = 0; j < m->n_edges_on_cell[i]; j++) {
                int e = m->edges_on_cell[i * MAXE + j];
                int nb = m->cells_on_cell[i * MAXE + j];
                double ui;
                if (k == 0) ui = u[(size_t)e * L];
                else if (k == L) ui = u[(size_t)e * L + L - 1];
                else ui = 0.5 * (u[(size_t)e * L + k - 1] + u[(size_t)e * L + k]);
                s += m->edge_sign_on_cell[i * MAXE + j] * m->dv[e] * ui * 0.5 *
                     (x[(size_t)nb * Li + k] - x[(size_t)i * Li + k]);
            }
            out[(size_t)i * Li + k] = s / m->cell_area[i];
        }
    }
}

/* Vertical advection eta-dot dx/deta = M dx/dpi at interior interfaces
 * (centred): M_{k} (x_{k+1} - x_{k-1}) / (dpi_{k-1} + dpi_k); zero at the
 * top and bottom interfaces where M = 0. */
void orc_interface_vadv(int nC, int L, const double *M, const double *dpi, const double *x,
                        double *out) {
    int Li = L + 1;
#pragma omp parallel for
    for (int i = 0; i < nC; i++) {
        out[(size_t)i * Li] = 0.0;
        out[(size_t)i * Li + L] = 0.0;
        for (int k = 1; k < L; k++)
            out[(size_t)i * Li + k] = M[(size_t)i * Li + k] *
                                      (x[(size_t)i * Li + k + 1] - x[(size_t)i * Li + k - 1]) /
                                      (dpi[(size_t)i * L + k - 1] + dpi[(size_t)i * L + k]);
    }
}

/* Thomas algorithm for a tridiagonal system (no pivoting; the HEVI system
 * is diagonally dominant): a = sub-, b = main, c = super-diagonal, d = rhs;
 * x = solution.  n >= 1. */
void orc_thomas(int n, const double *a, const double *b, const double *c, const double *d, double *x) {
    double *cp = (double *)xalloc(sizeof(double) * n), *dp = (double *)xalloc(sizeof(double) * n);
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int i = 1; i < n; i++) {
        double den = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / den;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp); free(dp);
}

/* Vertical implicit solve of one HEVI stage for every column (Eqs. 6, 7, 9).
 * Inputs: w_star, phi_star = explicit parts (w**, phi**) [nC][L+1];
 * dpi_theta, dpi of the new stage [nC][L]; dts = stage step; beta =
 * implicit weight.  Linearising the EOS about phi**:
 *   p_k = p**_k - C_k (w_k - w_{k+1}),  C_k = gamma p**_k beta dts g / dphi**_k,
 * the w equation at interior interface j (between layers j-1 and j),
 * a_j = beta dts g / dpi_j^int, dpi_j^int = (dpi_{j-1} + dpi_j)/2:
 *   -a_j C_{j-1} w_{j-1} + (1 + a_j C_{j-1} + a_j C_j) w_j - a_j C_j w_{j+1}
 *     = w**_j + a_j (p**_j - p**_{j-1}) - beta dts g,
 * w = 0 at the rigid lid (j = 0) and the flat ground (j = L).  Then
 * phi_j = phi**_j + beta dts g w_j (phi_L = phi_s kept) and the final
 * pressure from the full EOS.  Outputs w, phi [nC][L+1], p [nC][L]. */
void orc_vertical_solve(const orc_params *P, int nC, const double *w_star, const double *phi_star,
                        const double *dpi_theta, const double *dpi, double dts, double *w,
                        double *phi, double *p) {
    int L = P->L, Li = L + 1;
    double gam = P->cp / (P->cp - P->rd), bg = P->beta * dts * P->g;
#pragma omp parallel for
    for (int i = 0; i < nC; i++) {
        double *pst = (double *)xalloc(sizeof(double) * L), *C = (double *)xalloc(sizeof(double) * L);
        int n = L - 1;
        double *a = (double *)xalloc(sizeof(double) * (n + 1)), *b = (double *)xalloc(sizeof(double) * (n + 1)),
               *c = (double *)xalloc(sizeof(double) * (n + 1)), *d = (double *)xalloc(sizeof(double) * (n + 1)),
               *x = (double *)xalloc(sizeof(double) * (n + 1));
        for (int k = 0; k < L; k++) {
            double dphi = phi_star[(size_t)i * Li + k] - phi_star[(size_t)i * Li + k + 1];
            pst[k] = P->p0 * pow(P->rd * dpi_theta[(size_t)i * L + k] / (P->p0 * dphi), gam);
            C[k] = gam * pst[k] * bg / dphi;
        }
        for (int j = 1; j < L; j++) {
            double dpint = 0.5 * (dpi[(size_t)i * L + j - 1] + dpi[(size_t)i * L + j]);
            double aj = bg / dpint;
            a[j - 1] = -aj * C[j - 1];
            c[j - 1] = -aj * C[j];
            b[j - 1] = 1.0 + aj * C[j - 1] + aj * C[j];
            d[j - 1] = w_star[(size_t)i * Li + j] + aj * (pst[j] - pst[j - 1]) - bg;
        }
        if (n > 0) {
            a[0] = 0.0;
            c[n - 1] = 0.0;
            orc_thomas(n, a, b, c, d, x);
        }
        w[(size_t)i * Li] = 0.0;
        w[(size_t)i * Li + L] = 0.0;
        for (int j = 1; j < L; j++) w[(size_t)i * Li + j] = x[j - 1];
        for (int j = 0; j < L; j++) phi[(size_t)i * Li + j] = phi_star[(size_t)i * Li + j] + bg * w[(size_t)i * Li + j];
        phi[(size_t)i * Li + L] = P->phi_s[i];
        free(pst); free(C); free(a); free(b); free(c); free(d); free(x);
    }
    orc_eos(P, nC, dpi_theta, phi, p);
}

/* d p / d pi averaged to layers (the paper's L operator in Eq. 5, reading:
 * mean of the two interface values, interface value (p_j - p_{j-1}) /
 * dpi_j^int in the interior and 1 at the top and bottom). */
void orc_dpdpi_layer(int nC, int L, const double *p, const double *dpi, double *out) {
    for (int i = 0; i < nC; i++)
        for (int k = 0; k < L; k++) {
            double top = 1.0, bot = 1.0;
            if (k > 0)
                top = (p[(size_t)i * L + k] - p[(size_t)i * L + k - 1]) /
                      (0.5 * (dpi[(size_t)i * L + k - 1] + dpi[(size_t)i * L + k]));
            if (k < L - 1)
                bot = (p[(size_t)i * L + k + 1] - p[(size_t)i * L + k]) /
                      (0.5 * (dpi[(size_t)i * L + k] + dpi[(size_t)i * L + k + 1]));
            out[(size_t)i * L + k] = 0.5 * (top + bot);
        }
}

/* ------------------------------------------------------------------------
 * Non-hydrostatic dycore step (Sec. 2.1: horizontally explicit, vertically
 * implicit).  WS-RK3; in each stage:
 *   1. mass (Eq. 3) and theta (Eq. 4) from the stage input -> new stage;
 *   2. w, phi explicit parts (Eqs. 6, 7): advection (horizontal + vertical)
 *      from the stage input and the (1 - beta) share of the vertical
 *      pressure-gradient / gravity and w g terms at time level n;
 *   3. the implicit beta share by one tridiagonal solve per column, then the
 *      full EOS (Eq. 9) for p;
 *   4. momentum (Eq. 5) with the stage-input wind for the advective terms
 *      and the new p, phi, alpha = dphi/dpi, dp/dpi for the pressure-
 *      gradient and gravity terms.
 * ps [nC], u [nE][L], dpi_theta [nC][L], w, phi [nC][L+1]: in/out.
 * ---------------------------------------------------------------------- */
void orc_dycore_step_nh(const orc_mesh *m, const orc_params *P, double *ps, double *u,
                        double *dpi_theta, double *w, double *phi, double *flux_accum,
                        double *vflux_accum, double *accum_weight, double dt) {
    int L = P->L, Li = L + 1;
    size_t nC = m->nC, nCL = nC * L, nEL = (size_t)m->nE * L, nCI = nC * Li;
    double *ps_n = (double *)xalloc(sizeof(double) * nC), *u_n = (double *)xalloc(sizeof(double) * nEL),
           *th_n = (double *)xalloc(sizeof(double) * nCL), *w_n = (double *)xalloc(sizeof(double) * nCI),
           *phi_n = (double *)xalloc(sizeof(double) * nCI);
    double *ps_s = (double *)xalloc(sizeof(double) * nC), *u_s = (double *)xalloc(sizeof(double) * nEL),
           *th_s = (double *)xalloc(sizeof(double) * nCL), *w_s = (double *)xalloc(sizeof(double) * nCI),
           *phi_s = (double *)xalloc(sizeof(double) * nCI);
    double *dpi = (double *)xalloc(sizeof(double) * nCL), *dpi_new = (double *)xalloc(sizeof(double) * nCL),
           *dpi_n = (double *)xalloc(sizeof(double) * nCL);
    double *F = (double *)xalloc(sizeof(double) * nEL), *D = (double *)xalloc(sizeof(double) * nCL);
    double *pst = (double *)xalloc(sizeof(double) * nC), *M = (double *)xalloc(sizeof(double) * nCI);
    double *tht = (double *)xalloc(sizeof(double) * nCL);
    double *p_n = (double *)xalloc(sizeof(double) * nCL), *p = (double *)xalloc(sizeof(double) * nCL);
    double *hw = (double *)xalloc(sizeof(double) * nCI), *vw = (double *)xalloc(sizeof(double) * nCI),
           *hp = (double *)xalloc(sizeof(double) * nCI), *vp = (double *)xalloc(sizeof(double) * nCI);
    double *wst = (double *)xalloc(sizeof(double) * nCI), *pstar = (double *)xalloc(sizeof(double) * nCI);
    double *al = (double *)xalloc(sizeof(double) * nCL), *phl = (double *)xalloc(sizeof(double) * nCL),
           *dpp = (double *)xalloc(sizeof(double) * nCL);
    double *ut = (double *)xalloc(sizeof(double) * nEL);
    const double dts[3] = {dt / 3.0, dt / 2.0, dt};
    double g = P->g, beta = P->beta;

    memcpy(ps_n, ps, sizeof(double) * nC); memcpy(u_n, u, sizeof(double) * nEL);
    memcpy(th_n, dpi_theta, sizeof(double) * nCL); memcpy(w_n, w, sizeof(double) * nCI);
    memcpy(phi_n, phi, sizeof(double) * nCI);
    memcpy(ps_s, ps, sizeof(double) * nC); memcpy(u_s, u, sizeof(double) * nEL);
    memcpy(th_s, dpi_theta, sizeof(double) * nCL); memcpy(w_s, w, sizeof(double) * nCI);
    memcpy(phi_s, phi, sizeof(double) * nCI);
    /* time-level-n pressure and layer mass for the explicit (1 - beta) share */
    layer_mass(P, m->nC, ps_n, dpi_n);
    orc_eos(P, m->nC, th_n, phi_n, p_n);

    for (int s = 0; s < 3; s++) {
        double h = dts[s];
        orc_mass(m, P, ps_s, u_s, dpi, F, D, pst, M);
        orc_theta_tend(m, L, th_s, dpi, F, M, 1.0, tht);
        for (size_t i = 0; i < nC; i++) ps[i] = ps_n[i] + h * pst[i];
        for (size_t x = 0; x < nCL; x++) dpi_theta[x] = th_n[x] + h * tht[x];
        layer_mass(P, m->nC, ps, dpi_new);
        /* explicit parts of w and phi */
        orc_interface_hadv(m, L, u_s, w_s, hw);
        orc_interface_vadv(m->nC, L, M, dpi, w_s, vw);
        orc_interface_hadv(m, L, u_s, phi_s, hp);
        orc_interface_vadv(m->nC, L, M, dpi, phi_s, vp);
        for (size_t i = 0; i < nC; i++) {
            for (int j = 0; j < Li; j++) {
                size_t x = i * Li + j;
                double fw = 0.0;
                if (j > 0 && j < L) {
                    double dpint = 0.5 * (dpi_n[i * L + j - 1] + dpi_n[i * L + j]);
                    fw = g * ((p_n[i * L + j] - p_n[i * L + j - 1]) / dpint - 1.0);
                }
                wst[x] = w_n[x] + h * (-hw[x] - vw[x] + (1.0 - beta) * fw);
                pstar[x] = phi_n[x] + h * (-hp[x] - vp[x] + (1.0 - beta) * g * w_n[x]);
            }
            pstar[i * Li + L] = P->phi_s[i];
        }
        orc_vertical_solve(P, m->nC, wst, pstar, dpi_theta, dpi_new, h, w, phi, p);
        /* momentum with the new pressure and geopotential */
        for (size_t i = 0; i < nC; i++)
            for (int k = 0; k < L; k++) {
                double dphi = phi[i * Li + k] - phi[i * Li + k + 1];
                al[i * L + k] = dphi / dpi_new[i * L + k];
                phl[i * L + k] = 0.5 * (phi[i * Li + k] + phi[i * Li + k + 1]);
            }
        orc_dpdpi_layer(m->nC, L, p, dpi_new, dpp);
        orc_momentum_tend(m, L, u_s, dpi, F, M, p, al, phl, dpp, ut);
        for (size_t x = 0; x < nEL; x++) u[x] = u_n[x] + h * ut[x];
        if (s == 2 && flux_accum) {
            for (size_t x = 0; x < nEL; x++) flux_accum[x] += F[x];
            if (accum_weight) *accum_weight += 1.0;
        }
        if (s == 2 && vflux_accum)
            for (size_t x = 0; x < nCI; x++) vflux_accum[x] += M[x];
        memcpy(ps_s, ps, sizeof(double) * nC); memcpy(u_s, u, sizeof(double) * nEL);
        memcpy(th_s, dpi_theta, sizeof(double) * nCL); memcpy(w_s, w, sizeof(double) * nCI);
        memcpy(phi_s, phi, sizeof(double) * nCI);
    }
    free(ps_n); free(u_n); free(th_n); free(w_n); free(phi_n); free(ps_s); free(u_s); free(th_s);
    free(w_s); free(phi_s); free(dpi); free(dpi_new); free(dpi_n); free(F); free(D); free(pst); free(M);
    free(tht); free(p_n); free(p); free(hw); free(vw); free(hp); free(vp); free(wst); free(pstar);
    free(al); free(phl); free(dpp); free(ut);
}

/* ------------------------------------------------------------------------
 * Vertical tracer transport: the delta(M q) term of Eq. 10.  Sec. 2.1 names
 * "an adaptively implicit method" for the vertical (after Li and Zhang
 * 2022, not available here); the reading is a Courant-number-dependent
 * split of the vertical mass flux:
 *   at interior interface j (between layers j-1 above and j below; M_j > 0
 *   carries mass from j-1 into j) the donor layer is j-1 if M_j > 0, else j;
 *   its Courant number c_j = |M_j| dt / dpi_donor; the explicit share is
 *   Me_j = f_j M_j with f_j = min(1, cmax / c_j), the implicit share
 *   Mi_j = M_j - Me_j (zero wherever c_j <= cmax).
 *   Both shares are first-order upwind: the explicit one from q at the start
 *   of the step, the implicit one from q at the end (backward Euler), so for
 *   each layer k (M_0 = M_L = 0)
 *     dpi+_k q+_k + dt (Fi_{k+1} - Fi_k) = dpi_k q_k - dt (Fe_{k+1} - Fe_k),
 *     dpi+_k = dpi_k - dt (M_{k+1} - M_k),
 *   F_j = M_j q(donor of j): a tridiagonal M-matrix system per column,
 *   solved by the Thomas algorithm.  Constants stay constant, column mass
 *   sum_k dpi+ q+ = sum_k dpi q is conserved, and no new extrema appear.
 * q [T][nC][L] in/out; dpi [nC][L] the layer mass at the start of the
 * step; Mv [nC][L+1] the (time-mean) vertical mass flux.
 * ---------------------------------------------------------------------- */
void orc_tracer_vertical(int nC, int L, int T, double *q, const double *dpi, const double *Mv, double dt,
                         double cmax) {
    const int Li = L + 1;
#pragma omp parallel for
    for (int i = 0; i < nC; i++) {
        double *me = (double *)xalloc(sizeof(double) * Li), *mi = (double *)xalloc(sizeof(double) * Li);
        double *dpn = (double *)xalloc(sizeof(double) * L);
        double *a = (double *)xalloc(sizeof(double) * L), *b = (double *)xalloc(sizeof(double) * L),
               *c = (double *)xalloc(sizeof(double) * L), *d = (double *)xalloc(sizeof(double) * L),
               *x = (double *)xalloc(sizeof(double) * L);
        const double *Mi = Mv + (size_t)i * Li, *dp = dpi + (size_t)i * L;
        for (int j = 0; j < Li; j++) {
            me[j] = 0.0;
            mi[j] = 0.0;
            if (j == 0 || j == L || Mi[j] == 0.0) continue;
            const int donor = Mi[j] > 0.0 ? j - 1 : j;
            const double cour = fabs(Mi[j]) * dt / dp[donor];
            const double f = cour <= cmax ? 1.0 : cmax / cour;
            me[j] = f * Mi[j];
            mi[j] = Mi[j] - me[j];
        }
        for (int k = 0; k < L; k++) dpn[k] = dp[k] - dt * (Mi[k + 1] - Mi[k]);
        for (int t = 0; t < T; t++) {
            double *qt = q + ((size_t)t * nC + i) * L;
            for (int k = 0; k < L; k++) {
                const double qtop = (k > 0) ? (Mi[k] > 0.0 ? qt[k - 1] : qt[k]) : 0.0;
                const double qbot = (k < L - 1) ? (Mi[k + 1] > 0.0 ? qt[k] : qt[k + 1]) : 0.0;
                d[k] = dp[k] * qt[k] - dt * (me[k + 1] * qbot - me[k] * qtop);
                a[k] = -dt * fmax(mi[k], 0.0);
                b[k] = dpn[k] + dt * (fmax(mi[k + 1], 0.0) - fmin(mi[k], 0.0));
                c[k] = dt * fmin(mi[k + 1], 0.0);
            }
            orc_thomas(L, a, b, c, d, x);
            memcpy(qt, x, sizeof(double) * L);
        }
        free(me); free(mi); free(dpn); free(a); free(b); free(c); free(d); free(x);
    }
}

/* ------------------------------------------------------------------------
 * Global sums (Sec. 2.3: mass conserved to double-precision round-off).
 * Neumaier compensated summation in index order of w_i * x_i; returns the
 * sum and the accumulated compensation term in out[0], out[1].
 * ---------------------------------------------------------------------- */
void orc_compensated_sum(int64_t n, const double *x, const double *w, double *out) {
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double v = w ? w[i] * x[i] : x[i];
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    out[0] = s + c;
    out[1] = c;
}

/* Dry mass sum_i A_i (ps_i - pi_top) and tracer mass
 * sum_{i,k} A_i dpi_{i,k} q_{i,k}, both compensated in index order. */
void orc_dry_mass(const orc_mesh *m, const double *ps, double pi_top, double *out) {
    double *x = (double *)xalloc(sizeof(double) * m->nC);
    for (int i = 0; i < m->nC; i++) x[i] = ps[i] - pi_top;
    orc_compensated_sum(m->nC, x, m->cell_area, out);
    free(x);
}

void orc_tracer_mass(const orc_mesh *m, int L, const double *q, const double *dpi, double *out) {
    size_t n = (size_t)m->nC * L;
    double *x = (double *)xalloc(sizeof(double) * n), *w = (double *)xalloc(sizeof(double) * n);
    for (int i = 0; i < m->nC; i++)
        for (int k = 0; k < L; k++) {
            x[(size_t)i * L + k] = q[(size_t)i * L + k];
            w[(size_t)i * L + k] = m->cell_area[i] * dpi[(size_t)i * L + k];
        }
    orc_compensated_sum((int64_t)n, x, w, out);
    free(x); free(w);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
