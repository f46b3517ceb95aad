/*
 * grist.h - C ABI of the GB300 (sm_103a) GRIST hot-path library.
 *
 * The library advances the explicit horizontal operators of the GRIST
 * dynamical core (arXiv 2404.08849) on the icosahedral Voronoi C-grid over
 * every vertical level:
 *   - tracer transport, Eq. 10 (third-order upwind edge flux, FCT limiter,
 *     cell-divergence gather; Sec. 2.1),
 *   - the hydrostatic dycore (Eqs. 3-5, 8; RK + Mesinger forward-backward,
 *     Sec. 2.1) and the non-hydrostatic dycore (Eqs. 3-7, 9; horizontally
 *     explicit, vertically implicit, Sec. 2.1),
 *   - compensated global mass sums (Sec. 2.3: mass conserved to FP64
 *     round-off),
 * in FP64 or in the paper's mixed precision (Sec. 2.2-2.3).
 *
 * General conventions
 *   - Every function returns a grist_status (0 = success, < 0 = error).
 *     Nothing aborts, exits or throws across the ABI.
 *   - "device" pointers are CUDA global-memory pointers on the mesh's
 *     device, owned by the caller (e.g. PyTorch tensors), and must stay
 *     valid until the enqueued work has finished.  "host" pointers are
 *     ordinary CPU memory, read during the call only.
 *   - Field layout is structure-of-arrays with the level index innermost:
 *     a layer field is [entity][ld] (ld >= n_levels, entries k >= n_levels
 *     are never read or written); an interface field is [cell][ld_int]
 *     (ld_int >= n_levels + 1, interface 0 = model top).
 *   - Fields are in the library's internal numbering (cells renumbered along
 *     a space-filling curve, see grist_mesh_permutation).
 *   - Step calls are asynchronous on the given CUDA stream (NULL = legacy
 *     default stream); the return code covers argument validation and launch
 *     errors.  Numerical faults are reported by grist_last_step_status
 *     after the stream has been synchronised.
 *   - Calls on one mesh handle must not overlap from several host threads.
 *     The dycore steps and the tracer steps keep separate device scratch in
 *     the handle, so a tracer step may run on one stream while a dycore step
 *     runs on another (e.g. the tracers of step n beside the dycore of step
 *     n + 1, with their fluxes in separate buffers); two dycore steps, or
 *     two tracer steps, of one handle must not overlap.
 */
#ifndef GRIST_H
#define GRIST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRIST_OK = 0,
    GRIST_EINVAL = -1,       /* bad argument or inconsistent mesh tables */
    GRIST_ECUDA = -2,        /* a CUDA runtime call failed */
    GRIST_ENOMEM = -3,       /* device or host allocation failed */
    GRIST_ENUMERIC = -4,     /* non-finite values produced */
    GRIST_ETIMEOUT = -5,     /* a bounded device-side wait gave up */
    GRIST_EUNSUPPORTED = -6  /* valid but not supported request */
} grist_status;

/* Precision policy (Sec. 2.2: the KIND parameter "ns"; Sec. 2.3: the
 * compile switch for the mass-flux divergence).
 *   GRIST_FP64          every array and operation in double precision.
 *   GRIST_MIX           advective terms, winds u_n and tracers stored and
 *                       computed in single precision; pressure gradient,
 *                       gravity, vertical integrals, the equation of state,
 *                       the implicit column solve, surface pressure, layer
 *                       mass and all global sums in double (Sec. 2.3).
 *   GRIST_MIX_DBL_MASS  as GRIST_MIX but the mass flux dpi*V and its
 *                       divergence in double (Sec. 2.3, Sec. 4.4).
 *   GRIST_MIX_DF        as GRIST_MIX but the pressure-gradient, gravity
 *                       and kinetic-energy-gradient terms of Eq. 5, which
 *                       GRIST_MIX computes in double, in single-precision
 *                       arithmetic whose differences of nearly equal double
 *                       fields (p, layer phi, K) come from double-float
 *                       splits (about 48 bits), and the non-hydrostatic
 *                       equation of state (Eq. 9) as a double base value
 *                       plus a single-precision increment; no counterpart
 *                       in the paper (an FP32-dominant variant of its
 *                       double rows).  Tracers: as GRIST_MIX. */
typedef enum { GRIST_FP64 = 0, GRIST_MIX = 1, GRIST_MIX_DBL_MASS = 2, GRIST_MIX_DF = 3 } grist_precision;

/* ---------------------------------------------------------------------- */
/* Mesh (Sec. 2.1: hexagonal Arakawa-C grid; Table 1 grid sizes)           */
/* ---------------------------------------------------------------------- */

typedef struct grist_mesh_s *grist_mesh; /* opaque, library-owned */

/* Host tables of one icosahedral Voronoi mesh, 0-based, original numbering.
 * Orientation: cells_on_edge[e] = (c1, c2), the normal points c1 -> c2;
 * t = k x n and vertices_on_edge[e] = (v1, v2) with v2 - v1 along t.
 * Per-cell lists are counter-clockwise seen from outside; slot 5 of a
 * pentagon is -1.  edge_sign_on_cell = +1 where the normal leaves the cell;
 * edge_sign_on_vertex = +1 where the normal turns counter-clockwise about
 * the vertex.  The TRiSK weights w(e,e') give the tangential mass flux
 * (1/dc_e) sum_e' w(e,e') dv_e' F_e'; the deriv-two stencil gives the
 * normal second derivative at side s of edge e as sum_j coef q(stencil_j).
 * All arrays are copied by grist_mesh_create; the caller keeps ownership. */
typedef struct {
    int32_t n_cells, n_edges, n_vertices, max_edges; /* max_edges must be 6 */
    double radius;                                    /* sphere radius [m] */
    const double *cell_xyz;                           /* [nC][3] unit vectors */
    const double *cell_area;                          /* [nC] m^2 */
    const double *vertex_xyz;                         /* [nV][3] */
    const double *vertex_area;                        /* [nV] m^2 (dual triangle) */
    const double *edge_dc;                            /* [nE] cell-centre distance */
    const double *edge_dv;                            /* [nE] Voronoi edge length */
    const double *f_vertex;                           /* [nV] Coriolis parameter */
    const int32_t *cells_on_edge;                     /* [nE][2] */
    const int32_t *vertices_on_edge;                  /* [nE][2] */
    const int32_t *n_edges_on_cell;                   /* [nC] 5 or 6 */
    const int32_t *edges_on_cell;                     /* [nC][6] */
    const int32_t *cells_on_cell;                     /* [nC][6] */
    const int32_t *edges_on_vertex;                   /* [nV][3] */
    const int32_t *cells_on_vertex;                   /* [nV][3] */
    const double *edge_sign_on_cell;                  /* [nC][6] +-1, 0 padding */
    const double *edge_sign_on_vertex;                /* [nV][3] +-1 */
    const double *kite_area;                          /* [nV][3] aligned with cells_on_vertex */
    const int32_t *n_edges_on_edge;                   /* [nE] <= 10 */
    const int32_t *edges_on_edge;                     /* [nE][10] */
    const double *trisk_weight;                       /* [nE][10] */
    const int32_t *d2_stencil;                        /* [nE][2][7], -1 padding */
    const double *d2_coef;                            /* [nE][2][7] */
    int32_t sfc_reorder;                              /* 1 = renumber along a Hilbert curve */
} grist_mesh_desc;

/* Validate and copy the tables (counts, index ranges, Euler characteristic,
 * pentagon count, area sums), renumber them (sfc_reorder), pack them
 * structure-of-arrays and upload them to `device`.  On success *out holds a
 * handle owning all device tables and the step scratch; GRIST_EINVAL for
 * inconsistent tables, GRIST_ECUDA / GRIST_ENOMEM on device failures.
 * Allocates device memory; not stream-ordered (synchronous). */
int grist_mesh_create(const grist_mesh_desc *desc, int device, grist_mesh *out);

/* Free every device and host resource of the handle (synchronises the
 * device first).  NULL is accepted. */
int grist_mesh_destroy(grist_mesh mesh);

/* Host copies of the renumbering: new index of every original cell, edge
 * and vertex (arrays of n_cells / n_edges / n_vertices; any may be NULL). */
int grist_mesh_permutation(grist_mesh mesh, int32_t *cell_new_of_old, int32_t *edge_new_of_old,
                           int32_t *vertex_new_of_old);

/* Entity counts of the handle (any pointer may be NULL). */
int grist_mesh_counts(grist_mesh mesh, int32_t *n_cells, int32_t *n_edges, int32_t *n_vertices);

/* Properties of the mesh's stencils found at creation, as bits of *flags:
 *   GRIST_MESH_COMBINED_STENCIL  every edge side's stencil contains c1 and
 *                                c2, so with beta_upwind = 1 the edge value
 *                                is one weighted sum (Sec. 2.1's third-order
 *                                flux, the cell mean folded into the weights)
 *   GRIST_MESH_RING_STENCIL      in addition every edge side's stencil is its
 *                                cell's neighbour ring in the cell's order,
 *                                and the cell is c1 exactly when its
 *                                divergence sign is positive (the condition
 *                                of grist_tracer_tuning.cell_edges)
 * GRIST_EINVAL for a NULL argument.  Host only. */
#define GRIST_MESH_COMBINED_STENCIL 1u
#define GRIST_MESH_RING_STENCIL 2u
int grist_mesh_features(grist_mesh mesh, uint32_t *flags);

/* ---------------------------------------------------------------------- */
/* Tracer transport (Eq. 10, horizontal; Sec. 2.1, Sec. 2.3)               */
/* ---------------------------------------------------------------------- */

/* One ensemble member: a set of n_tracers tracers on n_levels levels.
 *   q          device, in/out, [n_tracers][n_cells][ld]; double for
 *              GRIST_FP64, float for the mixed policies (Sec. 2.3: tracer
 *              transport mostly in single precision).
 *   dpi        device, in, [n_cells][ld] double: layer mass at t^n.
 *   mass_flux  device, in, [n_edges][ld] double: time-mean mass flux
 *              dpi*V_n at edges (Sec. 2.3: accumulated from the continuity
 *              equation, used in double).
 *   vmass_flux device, in, [n_cells][ld_int] double, or NULL: time-mean
 *              vertical mass flux M at the interfaces (M > 0 downward, 0 at
 *              the top and the surface; e.g. the dycore's
 *              vmass_flux_accum).  When given, the horizontal step is
 *              followed by the vertical transport delta(M q) of Eq. 10 over
 *              the same dt (see grist_tracer_batch.vertical_courant_max).
 *   ld_int     leading dimension of vmass_flux (>= n_levels + 1).
 * The layer mass at each RK stage follows the tracer solver's continuity
 * with the same flux, dpi^(s) = dpi - dt_s div(mass_flux); the vertical
 * step starts from dpi - dt div(mass_flux) and ends at that minus
 * dt (M_{k+1} - M_k), the dycore's layer mass when the fluxes are its
 * accumulated ones. */
typedef struct {
    int32_t n_levels, n_tracers, ld;
    void *q;
    const double *dpi;
    const double *mass_flux;
    const double *vmass_flux;
    int32_t ld_int;
} grist_tracer_member;

/* A batch of members (uneven tracer and level counts allowed) advanced in
 * one call.  limiter: 1 = FCT on the final RK stage, 0 = none.
 * beta_upwind: upwind weight of the third-order flux (1 = third order,
 * 0 = fourth-order centred).  prec: GRIST_FP64 or a mixed policy.
 * vertical_courant_max: the vertical transport (Sec. 2.1 "adaptively
 * implicit") moves the share of M up to this Courant number |M| dt / dpi
 * of the donor layer explicitly (first-order upwind) and the rest by
 * backward-Euler upwind (one tridiagonal system per column): constants stay
 * constant, column mass is conserved, no new extrema for values <= 1.
 * 0 = fully implicit; negative or NaN: GRIST_EINVAL (only read when a
 * member has a vertical mass flux; the Python binding's default is 1). */
typedef struct {
    int32_t n_members;
    const grist_tracer_member *members; /* host array of n_members */
    grist_precision prec;
    int32_t limiter;
    double beta_upwind;
    double vertical_courant_max;        /* >= 0 (see below) */
} grist_tracer_batch;

/* Advance every member by dt with Wicker-Skamarock RK3 (dt/3, dt/2, dt),
 * the third-order upwind flux each stage and, if limiter, the Zalesak FCT
 * on the final stage.  All members advance together: each phase of the
 * step is one pass over a work list of (member, tracer group, entity,
 * level), either as one kernel launch per phase or as one persistent
 * cooperative launch per step (see grist_tracer_tuning).  At most
 * GRIST_MAX_MEMBERS members.  Asynchronous on `stream`.  GRIST_EINVAL on
 * bad sizes or NULL pointers; a persistent launch whose bounded grid
 * barrier gave up raises GRIST_FLAG_TIMEOUT (grist_last_step_status). */
#define GRIST_MAX_MEMBERS 64
int grist_tracer_step(grist_mesh mesh, const grist_tracer_batch *batch, double dt, void *stream);

/* Launch configuration of the tracer step (the batching design of this
 * library; no counterpart in the paper).
 *   block               threads per block (64..512, multiple of 32)
 *   tracers_per_thread  tracers one thread carries through a phase (>= 1)
 *   persistent          0 = one launch per phase; 1 = one cooperative
 *                       persistent launch per step with grid barriers
 *   use_graph           1 = capture the step's launches in a CUDA graph on
 *                       the first call with a given batch (same buffers,
 *                       sizes, dt, precision, limiter, beta) and replay it
 *                       afterwards; the first call must not itself be
 *                       inside a stream capture.
 *   fused               1 = RK stages without the limiter run as one tiled
 *                       kernel each (edge fluxes of a tile of cells kept in
 *                       shared memory, never written to global memory);
 *                       ignored when persistent = 1.
 *   levels_per_thread   1 or 2: levels one thread of a per-phase launch
 *                       carries (levels g and g + ceil(L/2) for 2; the
 *                       entity's stencil tables are read once for both);
 *                       the persistent launch uses 1.
 *   cell_edges          1 = with beta_upwind = 1 the edge fluxes are formed
 *                       cell-centrically: the thread of a cell gathers q over
 *                       the cell and its neighbours once and writes the flux
 *                       of every edge whose flux leaves the cell (same
 *                       weights, same summation order: bit-identical to 0,
 *                       the edge-centric form, which is also used whenever
 *                       beta_upwind != 1 or the mesh's stencils are not the
 *                       upwind cell's neighbour ring). */
typedef struct {
    int32_t block, tracers_per_thread, persistent, use_graph, fused, levels_per_thread, cell_edges;
} grist_tracer_tuning;

/* Set / get the tuning used by later grist_tracer_step calls on the mesh
 * (default: block 128, tracers_per_thread 4, persistent 0, use_graph 0,
 * fused 0, levels_per_thread 2, cell_edges 1 - the autotuner's choice on
 * the level-9 mesh with 60 levels and 4 tracers).
 * GRIST_EINVAL for out-of-range values. */
int grist_tracer_set_tuning(grist_mesh mesh, const grist_tracer_tuning *tuning);
int grist_tracer_get_tuning(grist_mesh mesh, grist_tracer_tuning *tuning);

/* Autotuner: time candidate tunings (block sizes - hence cells per block -
 * tracers per thread, fused tiles on/off, then levels per thread at the
 * best of those, the edge-flux form, then per-phase vs persistent launch
 * and graph on/off) on
 * `steps` tracer steps of
 * the given batch, keep the fastest as the mesh's tuning and return it in
 * *best (and its mean step time in milliseconds in *best_ms, may be NULL).
 * Works on private copies of the tracer arrays (allocates them), so the
 * caller's q is unchanged; synchronises `stream`. */
int grist_tracer_autotune(grist_mesh mesh, const grist_tracer_batch *batch, double dt, int32_t steps, void *stream,
                          grist_tracer_tuning *best, double *best_ms);

/* ---------------------------------------------------------------------- */
/* Dycore (Eqs. 3-9; Sec. 2.1, Sec. 2.3)                                   */
/* ---------------------------------------------------------------------- */

/* Constants and vertical grid.  Pure sigma-mass coordinate:
 * pi_{k+1/2} = pi_top + b_interface[k] (ps - pi_top), b = 0 at the top,
 * 1 at the surface. */
typedef struct {
    int32_t n_levels, ld, ld_int;  /* ld >= L, ld_int >= L + 1 */
    double pi_top;                 /* [Pa] constant model-top pressure */
    double p0, rd, cp, g;          /* reference pressure, gas constant, heat capacity, gravity */
    double offcentre_beta;         /* implicit weight of the NH vertical terms (0.5..1) */
    const double *b_interface;     /* host, [L+1] */
    const double *phi_surface;     /* device, [nC] surface geopotential */
    uint32_t emulate_fp32_rows;    /* GRIST_ROW_* bits; 0 = none (see below) */
} grist_dycore_params;

/* Rows of the precision map (Sec. 2.3) for the iterative precision search
 * of Sec. 2.2 (Eqs. 1-2).  With a bit set, every FP64 value of that row is
 * rounded to binary32 where it is produced (storage-rounding emulation:
 * the arithmetic between roundings stays in the policy's type), so the
 * accuracy cost of a single-precision row can be measured on the FP64
 * path without a kernel per combination.  A nonzero mask needs GRIST_FP64
 * (else GRIST_EUNSUPPORTED) and runs a separately compiled emulating
 * variant of the FP64 kernels; 0 runs the production kernels unchanged. */
#define GRIST_ROW_MASS_FLUX 0x001u  /* dpi V at edges and its layer divergence (Eq. 3) */
#define GRIST_ROW_WIND 0x002u       /* u_n after each stage update (Eq. 5) */
#define GRIST_ROW_PV_FLUX 0x004u    /* vertex and edge PV, tangential PV flux (Eq. 5) */
#define GRIST_ROW_KE_GRAD 0x008u    /* cell kinetic energy (Eq. 5) */
#define GRIST_ROW_VADV_U 0x010u     /* vertical advection of momentum (Eq. 5) */
#define GRIST_ROW_PGF 0x020u        /* pressure gradient and gravity terms, inputs and sum (Eq. 5) */
#define GRIST_ROW_THETA 0x040u      /* theta and its edge flux (Eq. 4) */
#define GRIST_ROW_DPI_PV 0x080u     /* vertex layer mass dividing the PV (Sec. 2.3 "green") */
#define GRIST_ROW_EOS 0x100u        /* p, alpha, layer phi, dp/dpi (Eqs. 8-9) */
#define GRIST_ROW_NH_ADV 0x200u     /* advection of w and phi (Eqs. 6-7) */
#define GRIST_ROW_ALL 0x3ffu

/* Prognostic state (device, in/out, caller-owned).
 *   u           [nE][ld] edge-normal wind: double (FP64) or float (mixed)
 *   ps          [nC] double, dry surface pressure
 *   dpi_theta   [nC][ld] double, mass-weighted potential temperature
 *   w, phi      [nC][ld_int] double, NH vertical velocity and geopotential
 *               at interfaces (ignored by the hydrostatic step)
 *   mass_flux_accum [nE][ld] double or NULL: accum_scale times the
 *               final-stage mass flux of the step is added to it (time-mean
 *               flux for the tracer, Sec. 2.1 / Sec. 2.3 "accumulated and
 *               averaged"): n steps with accum_scale = 1/n leave the mean
 *               flux over the n steps, the flux that carries the tracers
 *               over one tracer step of n dycore time steps.
 *   accum_weight device double or NULL: accum_scale is added per step.
 *   dpi_start   [nC][ld] double or NULL: receives the layer mass dpi at
 *               the start of the step (the tracer solver's dpi^n).
 *   p_nh        [nC][ld] double or NULL (NH only): the non-hydrostatic
 *               pressure of the state, Eq. 9.  If p_nh_valid is nonzero
 *               on entry the step uses it as the t^n pressure instead of
 *               evaluating the equation of state; on return it holds the
 *               pressure of the new state and p_nh_valid is set to 1.  Set
 *               p_nh_valid to 0 whenever dpi_theta or phi change outside
 *               the step.
 *   accum_scale weight of this step's flux in mass_flux_accum and
 *               accum_weight; 0 is read as 1.
 *   vmass_flux_accum [nC][ld_int] double or NULL: accum_scale times the
 *               final stage's vertical mass flux M at the interfaces (the
 *               delta(M q) flux of Eq. 10; M > 0 carries mass downward, 0 at
 *               the top and the surface) is added to it - the flux of the
 *               tracers' vertical transport. */
typedef struct {
    void *u;
    double *ps;
    double *dpi_theta;
    double *w;
    double *phi;
    double *mass_flux_accum;
    double *accum_weight;
    double *dpi_start;
    double *p_nh;
    int32_t p_nh_valid;
    double accum_scale;
    double *vmass_flux_accum;
} grist_dycore_state;

/* Hydrostatic step: WS-RK3, Mesinger forward-backward inside each stage
 * (mass and theta first, then the hydrostatic diagnostics Eq. 8 from the
 * new mass, then momentum Eq. 5).  Asynchronous on `stream`. */
int grist_dycore_step_hydro(grist_mesh mesh, grist_dycore_state *state, const grist_dycore_params *params,
                            grist_precision prec, double dt, void *stream);

/* Non-hydrostatic step: WS-RK3 with, per stage, mass and theta, the
 * explicit parts of w and phi (Eqs. 6-7), one FP64 tridiagonal solve per
 * column for the implicit part (off-centred by offcentre_beta), the
 * equation of state Eq. 9, then momentum Eq. 5 with the new pressure and
 * geopotential.  Asynchronous on `stream`. */
int grist_dycore_step_nh(grist_mesh mesh, grist_dycore_state *state, const grist_dycore_params *params,
                         grist_precision prec, double dt, void *stream);

/* Diagnostic: relative vorticity at the vertices, zeta_v = (1/A_v) sum over
 * the vertex's edges of t(e,v) dc_e u_e, on every level (the velocity
 * diagnostic of Eq. 1).
 *   u       device, in, [nE][ld] double (u_prec GRIST_FP64) or float
 *           (GRIST_MIX / GRIST_MIX_DBL_MASS).
 *   vor     device, out, [nV][ld] double.
 * Asynchronous on `stream`. */
int grist_diag_vorticity(grist_mesh mesh, const void *u, grist_precision u_prec, int32_t n_levels, int32_t ld,
                         double *vor, void *stream);

/* ---------------------------------------------------------------------- */
/* Whole-step CUDA graphs (no counterpart in the paper)                    */
/* ---------------------------------------------------------------------- */

/* Record everything enqueued on `stream` between grist_capture_begin and
 * grist_capture_end - e.g. one coupled model step: a dycore step and the
 * tracer step that uses its fluxes - as one CUDA graph, and replay it with
 * grist_graph_launch: one launch per step on the host instead of one per
 * kernel.  Rules:
 *   - `stream` must be a created stream (not the legacy default stream);
 *     capture runs in thread-local mode.
 *   - Make every recorded call once before capturing it: first calls size
 *     the handle's scratch and upload tables (allocations and copies that a
 *     capture cannot hold).
 *   - A replay repeats the recorded calls with the recorded arguments
 *     (buffers, sizes, dt, precision, tuning, and host-side choices such as
 *     a carried NH pressure being valid); capture again when one changes.
 *     The handle's scratch must not grow after the capture (make the
 *     largest call first), the dycore's vertical grid (b_interface) must be
 *     the one recorded, and a handle keeps the work-list tables of its last
 *     64 distinct tracer batches: a graph that recorded a tracer step of a
 *     batch dropped since then must be recorded again.  A tracer step of a
 *     batch the handle has not run outside a capture returns
 *     GRIST_EUNSUPPORTED inside the capture.  Keep per-kernel profiling
 *     (grist_profile_enable) off while capturing.
 *   - The steps enqueued while capturing do not run; the graph runs them.
 * grist_capture_end returns GRIST_ECUDA when the capture failed (e.g. a
 * recorded call needed an allocation); the stream is then no longer
 * capturing. */
typedef struct grist_graph_s *grist_graph;
int grist_capture_begin(void *stream);
int grist_capture_end(void *stream, grist_graph *out);
/* Enqueue one replay of the graph on `stream` (asynchronous). */
int grist_graph_launch(grist_graph graph, void *stream);
/* Free the graph (NULL accepted); replays already enqueued are not waited
 * for by this call - synchronise first. */
int grist_graph_destroy(grist_graph graph);

/* ---------------------------------------------------------------------- */
/* Global sums (Sec. 2.3: global mass conserved to round-off)              */
/* ---------------------------------------------------------------------- */

typedef enum {
    GRIST_SUM_DRY_MASS = 0,      /* sum_i A_i (field_i - offset), field [nC] double */
    GRIST_SUM_TRACER_MASS = 1,   /* sum_{i,k} A_i dpi_{i,k} field_{i,k}, field [nC][ld] */
    GRIST_SUM_AREA_WEIGHTED = 2  /* sum_{i,k} A_i field_{i,k}, field [nC][ld] (n_levels >= 1) */
} grist_sum_kind;

/* Deterministic compensated (Neumaier / double-double) global sum over all
 * cells (and levels) in a fixed order.  field: device, double (field_prec
 * GRIST_FP64) or float (mixed); dpi: device [nC][ld] double, only for the
 * tracer mass.  out_sum_and_err: host double[2] = {sum, compensation term}.
 * Enqueued on `stream`, then waits for the stream (the result is on the
 * host when the call returns). */
int grist_global_sums(grist_mesh mesh, grist_sum_kind kind, const void *field, const double *dpi,
                      int32_t n_levels, int32_t ld, grist_precision field_prec, double offset,
                      double *out_sum_and_err, void *stream);

/* ---------------------------------------------------------------------- */
/* Measurement aid (no counterpart in the paper)                           */
/* ---------------------------------------------------------------------- */

/* Enable (1) or disable (0) per-kernel timing on this handle.  While
 * enabled, every kernel launch of the step calls is bracketed by a pair of
 * CUDA events on the launching stream; enabling clears earlier totals.
 * Costs about one event record per launch; leave it off for production. */
int grist_profile_enable(grist_mesh mesh, int enable);

/* Synchronise the device and report the per-kernel totals gathered since
 * the last grist_profile_enable(mesh, 1): for entry j < *n_entries,
 * names + 64*j is a NUL-terminated kernel name, launches[j] the launch
 * count and total_ms[j] the summed event time in milliseconds.  At most
 * max_entries entries are written (host arrays, caller-owned). */
int grist_profile_read(grist_mesh mesh, int32_t max_entries, char *names, int32_t *launches, double *total_ms,
                       int32_t *n_entries);

/* FP64 throughput probe: launch `blocks` x `threads` threads (threads a
 * multiple of 32, at most 1024), each running GRIST_BENCH_FP64_CHAINS
 * independent chains of `iters` fused multiply-adds in double precision,
 * and write one double per thread to out (device, [blocks * threads], the
 * chains' sums, so the work cannot be optimised away).  FP64 flop per
 * launch = 2 * GRIST_BENCH_FP64_CHAINS * iters * blocks * threads; timing
 * the launch with events on `stream` gives the GPU's FP64 FMA rate, the
 * measured peak of the FP64-pipe roofline.  Asynchronous; GRIST_EINVAL for
 * sizes out of range (iters in 1..2^40, blocks in 1..2^20). */
#define GRIST_BENCH_FP64_CHAINS 8
int grist_bench_fp64_fma(int64_t iters, int32_t blocks, int32_t threads, double *out, void *stream);

/* ---------------------------------------------------------------------- */
/* Allocation-free weighted sum (no counterpart in the paper)              */
/* ---------------------------------------------------------------------- */

/* Upper bound on n for grist_weighted_sum_noalloc, and the number of terms
 * one block of its kernel sums. */
#define GRIST_NOALLOC_CHUNK 65536
#define GRIST_NOALLOC_MAX_TERMS (4096 * 65536)

/* sum_i w[i] * x[i] (w NULL: sum_i x[i]) over n device doubles, with the
 * compensated method of grist_global_sums (Neumaier accumulation plus a
 * TwoSum tree) in a fixed order of its own - bitwise reproducible run to
 * run, but not bitwise equal to grist_global_sums - without allocating any
 * memory.  For callers that cannot allocate device memory:
 * programs whose device memory is owned by another allocator that reserves
 * it up front, and code that must not pay the device-wide synchronisation a
 * cudaMalloc / cudaFree can imply.  No mesh handle is needed.
 *   x, w             device, in, n doubles (w may be NULL).
 *   n                0 <= n <= GRIST_NOALLOC_MAX_TERMS, else GRIST_EINVAL
 *                    (checked before anything is launched).
 *   out_sum_and_err  device, out, 2 doubles = {sum, compensation term},
 *                    written on `stream`; the call does not wait.
 * Partial sums live in one fixed device array per device (about 64 KB,
 * kept until the process exits) that every call shares: calls whose GPU
 * work overlaps race on it, so serialise them.  Each call writes every
 * partial it reads, so nothing needs clearing between calls.  The first
 * call on a device looks up the array's address with that device current
 * and keeps it for the life of the process (a cudaDeviceReset in between
 * would invalidate it); make that first call before any stream capture.
 * Uses the current device (cudaSetDevice). */
int grist_weighted_sum_noalloc(const double *x, const double *w, int64_t n, double *out_sum_and_err, void *stream);

/* ---------------------------------------------------------------------- */
/* Status                                                                  */
/* ---------------------------------------------------------------------- */

#define GRIST_FLAG_NONFINITE 0x1u  /* a step wrote NaN or Inf */
#define GRIST_FLAG_TIMEOUT 0x2u    /* a bounded device wait gave up */

/* Diagnostic: launch one thread that waits, with at most spin_limit polls
 * (about 64 ns apart; 1 <= spin_limit <= 1e8), for a device word that
 * nothing writes - the same bounded wait the persistent tracer launch uses
 * at its grid barriers.  The kernel always ends; afterwards
 * grist_last_step_status reports GRIST_FLAG_TIMEOUT and the context stays
 * usable.  Asynchronous on `stream`.  No counterpart in the paper. */
int grist_selftest_bounded_wait(grist_mesh mesh, int64_t spin_limit, void *stream);

/* Diagnostic: check the library's integer-arithmetic conversions between
 * binary32 and binary64 (the mixed-precision kernels use them in place of
 * the hardware conversion instructions, which issue on the FP64 pipe)
 * against the hardware conversions, on the current device:
 *   binary32 -> binary64 over all 2^32 bit patterns;
 *   binary64 -> binary32 over, for every binary32 pattern f, the value f,
 *   the midpoint between f and the next binary32 away from zero and the
 *   two binary64 neighbours of that midpoint (every rounding boundary,
 *   ties included), plus n_random pseudo-random binary64 patterns
 *   (splitmix64 of seed + i; half of them with exponents inside and around
 *   the binary32 range).
 * Bit-exact agreement is required, except that any NaN matches any NaN.
 *   out_checked[2], out_mismatch[2]  host, out: conversions checked and
 *                    mismatches for {binary32->binary64, binary64->binary32}.
 * Synchronous (uses and synchronises the default stream); allocates and
 * frees 32 bytes of device memory.  No counterpart in the paper. */
int grist_selftest_conversions(uint64_t n_random, uint64_t seed, uint64_t *out_checked, uint64_t *out_mismatch);

/* Diagnostic: check the library's FMA-refined approximate reciprocal (used
 * in the FP64 column solve in place of the correctly rounded one) against
 * the IEEE quotient 1.0 / x on n pseudo-random binary64 values (splitmix64
 * of seed + i; any sign and fraction, |x| in [2^-1020, 2^1021)), on the
 * current device.
 *   out_checked     host, out: values checked.
 *   out_over_1ulp   host, out: results more than one ulp from 1.0 / x.
 *   out_max_ulp     host, out: largest distance seen, in ulps.
 * Synchronous (default stream); allocates and frees 24 bytes of device
 * memory.  No counterpart in the paper. */
int grist_selftest_reciprocal(uint64_t n, uint64_t seed, uint64_t *out_checked, uint64_t *out_over_1ulp,
                              uint64_t *out_max_ulp);

/* Diagnostic: check the double-float splits x ~ h + l on n pseudo-random
 * binary64 values (splitmix64 of seed + i; |x| in [2^-74, 2^127), any sign
 * and fraction): the rounding split used by GRIST_MIX_DF (h = x rounded to
 * binary32, l = the residual rounded to binary32) and the truncating split
 * of the binary32 advection of w and phi (h = x truncated toward zero).
 * Counts values where either h differs from the hardware conversion (to
 * nearest, toward zero) or either |x - (h + l)| exceeds 2^-47 |x|.
 * Synchronous (default stream); allocates and frees 16 bytes of device
 * memory.  No counterpart in the paper. */
int grist_selftest_split(uint64_t n, uint64_t seed, uint64_t *out_checked, uint64_t *out_bad);

/* Flags raised by the steps since the previous call (read after the stream
 * has been synchronised; synchronises the device and clears the flags). */
int grist_last_step_status(grist_mesh mesh, uint32_t *flags);

/* Static description of a status code. */
const char *grist_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* GRIST_H */
