// mesh.cu - mesh handle: validation, space-filling-curve renumbering,
// structure-of-arrays packing and upload of the icosahedral Voronoi C-grid
// tables (Sec. 2.1 hexagonal Arakawa-C grid), device scratch, status word.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

using namespace grist;

struct grist_mesh_s {
    int device = 0;
    int nC = 0, nE = 0, nV = 0;
    std::vector<int32_t> cell_new, edge_new, vertex_new;  // new index of each original entity
    DevMesh d{};
    void *arena = nullptr;
    void *scr[8] = {nullptr};
    size_t scr_bytes[8] = {0};
    uint32_t *status = nullptr;
    TracerCtx *tctx = nullptr;
    HostTables ht;
    // the dycore's vertical-grid table as last uploaded, and where
    std::vector<double> vg_cache;
    const void *vg_ptr = nullptr;
    // profiling
    bool prof_on = false;
    std::vector<cudaEvent_t> ev;            // pool, pairs (2j, 2j+1)
    std::vector<int> pend_name;             // name id of each pending pair
    std::vector<std::string> prof_names;
    std::vector<double> prof_ms;
    std::vector<int> prof_count;
};

namespace grist {
const DevMesh &dev_mesh(grist_mesh_s *m) { return m->d; }
int mesh_device(grist_mesh_s *m) { return m->device; }
uint32_t *status_word(grist_mesh_s *m) { return m->status; }
bool profiling(grist_mesh_s *m) { return m->prof_on; }
TracerCtx *&tracer_ctx(grist_mesh_s *m) { return m->tctx; }
const HostTables &host_tables(grist_mesh_s *m) { return m->ht; }
std::vector<double> &vg_cache(grist_mesh_s *m) { return m->vg_cache; }
const void *&vg_ptr(grist_mesh_s *m) { return m->vg_ptr; }

static const int kEventPairs = 4096;

static void prof_drain(grist_mesh_s *m) {
    if (m->pend_name.empty()) return;
    cudaDeviceSynchronize();
    for (size_t j = 0; j < m->pend_name.size(); j++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m->ev[2 * j], m->ev[2 * j + 1]) == cudaSuccess) {
            m->prof_ms[m->pend_name[j]] += ms;
            m->prof_count[m->pend_name[j]] += 1;
        }
    }
    m->pend_name.clear();
}

ProfScope::ProfScope(grist_mesh_s *h_, const char *name, cudaStream_t st_) : h(h_), slot(-1), st(st_) {
    if (!h || !h->prof_on) return;
    if ((int)h->pend_name.size() >= kEventPairs) prof_drain(h);
    int id = -1;
    for (size_t j = 0; j < h->prof_names.size(); j++)
        if (h->prof_names[j] == name) { id = (int)j; break; }
    if (id < 0) {
        h->prof_names.push_back(name);
        h->prof_ms.push_back(0.0);
        h->prof_count.push_back(0);
        id = (int)h->prof_names.size() - 1;
    }
    slot = (int)h->pend_name.size();
    h->pend_name.push_back(id);
    cudaEventRecord(h->ev[2 * slot], st);
}

ProfScope::~ProfScope() {
    if (slot >= 0) cudaEventRecord(h->ev[2 * slot + 1], st);
}

void *scratch(grist_mesh_s *m, int slot, size_t bytes) {
    if (slot < 0 || slot >= 8) return nullptr;
    if (bytes == 0) bytes = 256;
    if (m->scr_bytes[slot] >= bytes) return m->scr[slot];
    if (m->scr[slot]) {
        cudaDeviceSynchronize();
        cudaFree(m->scr[slot]);
        m->scr[slot] = nullptr;
        m->scr_bytes[slot] = 0;
    }
    // a fresh allocation may reuse the freed address: whatever was uploaded
    // into scratch (the dycore's vertical-grid table) is gone
    m->vg_cache.clear();
    m->vg_ptr = nullptr;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    m->scr[slot] = p;
    m->scr_bytes[slot] = bytes;
    return p;
}
}  // namespace grist

namespace {

// 3-D Hilbert index of a point with 21-bit integer coordinates, after
// J. Skilling, "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004):
// convert the coordinates to the "transposed" Hilbert form (undo the
// excess work of each bit level, then Gray-encode) and interleave the bits.
uint64_t hilbert3(uint32_t x[3], int bits) {
    const int n = 3;
    uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < n; i++) {
            if (x[i] & Q) {
                x[0] ^= P;
            } else {
                uint32_t t = (x[0] ^ x[i]) & P;
                x[0] ^= t;
                x[i] ^= t;
            }
        }
    }
    for (int i = 1; i < n; i++) x[i] ^= x[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (x[n - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < n; i++) x[i] ^= t;
    uint64_t h = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int i = 0; i < n; i++) h = (h << 1) | ((x[i] >> b) & 1u);
    return h;
}

struct Arena {
    std::vector<std::pair<size_t, size_t>> parts;  // offset, bytes
    size_t total = 0;
    size_t add(size_t bytes) {
        size_t off = (total + 255) & ~size_t(255);
        total = off + bytes;
        return off;
    }
};

int validate(const grist_mesh_desc *d) {
    if (!d) return GRIST_EINVAL;
    if (d->max_edges != GRIST_MAXE) return GRIST_EUNSUPPORTED;
    const int nC = d->n_cells, nE = d->n_edges, nV = d->n_vertices;
    if (nC < 4 || nE < 6 || nV < 4) return GRIST_EINVAL;
    if ((long long)nE * GRIST_MAXL >= (1ll << 31)) return GRIST_EUNSUPPORTED;
    if (nV - nE + nC != 2) return GRIST_EINVAL;  // Euler characteristic of the sphere
    const void *ptrs[] = {d->cell_xyz, d->cell_area, d->vertex_area, d->edge_dc, d->edge_dv, d->f_vertex,
                          d->cells_on_edge, d->vertices_on_edge, d->n_edges_on_cell, d->edges_on_cell,
                          d->cells_on_cell, d->edges_on_vertex, d->cells_on_vertex, d->edge_sign_on_cell,
                          d->edge_sign_on_vertex, d->kite_area, d->n_edges_on_edge, d->edges_on_edge,
                          d->trisk_weight, d->d2_stencil, d->d2_coef};
    for (const void *p : ptrs)
        if (!p) return GRIST_EINVAL;
    long long sum_eoc = 0;
    for (int i = 0; i < nC; i++) {
        int n = d->n_edges_on_cell[i];
        if (n < 3 || n > GRIST_MAXE) return GRIST_EINVAL;
        sum_eoc += n;
        for (int j = 0; j < n; j++) {
            int e = d->edges_on_cell[i * 6 + j], c = d->cells_on_cell[i * 6 + j];
            if (e < 0 || e >= nE || c < 0 || c >= nC) return GRIST_EINVAL;
            int a = d->cells_on_edge[2 * e], b = d->cells_on_edge[2 * e + 1];
            if (!((a == i && b == c) || (b == i && a == c))) return GRIST_EINVAL;
            double s = d->edge_sign_on_cell[i * 6 + j];
            if (s != (a == i ? 1.0 : -1.0)) return GRIST_EINVAL;
        }
        if (!(d->cell_area[i] > 0)) return GRIST_EINVAL;
    }
    if (sum_eoc != 2ll * nE) return GRIST_EINVAL;
    for (int e = 0; e < nE; e++) {
        for (int s = 0; s < 2; s++) {
            int c = d->cells_on_edge[2 * e + s], v = d->vertices_on_edge[2 * e + s];
            if (c < 0 || c >= nC || v < 0 || v >= nV) return GRIST_EINVAL;
            for (int j = 0; j < GRIST_D2P; j++) {
                int q = d->d2_stencil[(2 * e + s) * GRIST_D2P + j];
                if (q < -1 || q >= nC) return GRIST_EINVAL;
            }
        }
        int n = d->n_edges_on_edge[e];
        if (n < 0 || n > GRIST_MAXEOE) return GRIST_EINVAL;
        for (int j = 0; j < n; j++) {
            int q = d->edges_on_edge[e * GRIST_MAXEOE + j];
            if (q < 0 || q >= nE) return GRIST_EINVAL;
        }
        if (!(d->edge_dc[e] > 0) || !(d->edge_dv[e] > 0)) return GRIST_EINVAL;
    }
    double asum = 0, vsum = 0;
    for (int v = 0; v < nV; v++) {
        for (int j = 0; j < 3; j++) {
            int e = d->edges_on_vertex[3 * v + j], c = d->cells_on_vertex[3 * v + j];
            if (e < 0 || e >= nE || c < 0 || c >= nC) return GRIST_EINVAL;
        }
        if (!(d->vertex_area[v] > 0)) return GRIST_EINVAL;
        vsum += d->vertex_area[v];
    }
    for (int i = 0; i < nC; i++) asum += d->cell_area[i];
    double sphere = 4.0 * M_PI * d->radius * d->radius;
    if (std::fabs(asum / sphere - 1.0) > 1e-9 || std::fabs(vsum / sphere - 1.0) > 1e-9) return GRIST_EINVAL;
    return GRIST_OK;
}

template <typename T> T *place(char *base, size_t off) { return reinterpret_cast<T *>(base + off); }

}  // namespace

extern "C" int grist_mesh_create(const grist_mesh_desc *desc, int device, grist_mesh *out) {
    if (!out) return GRIST_EINVAL;
    *out = nullptr;
    int rc = validate(desc);
    if (rc != GRIST_OK) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GRIST_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return GRIST_ECUDA;

    const int nC = desc->n_cells, nE = desc->n_edges, nV = desc->n_vertices;
    grist_mesh_s *m = new (std::nothrow) grist_mesh_s();
    if (!m) return GRIST_ENOMEM;
    m->device = device;
    m->nC = nC; m->nE = nE; m->nV = nV;

    // ---- renumbering ---------------------------------------------------
    std::vector<int32_t> cold(nC);  // original index of each new cell
    std::iota(cold.begin(), cold.end(), 0);
    if (desc->sfc_reorder) {
        std::vector<uint64_t> key(nC);
        for (int i = 0; i < nC; i++) {
            uint32_t x[3];
            for (int a = 0; a < 3; a++) {
                double c = 0.5 * (desc->cell_xyz[3 * i + a] + 1.0);
                c = std::min(std::max(c, 0.0), 1.0);
                x[a] = (uint32_t)std::min(c * 2097152.0, 2097151.0);
            }
            key[i] = hilbert3(x, 21);
        }
        std::stable_sort(cold.begin(), cold.end(), [&](int a, int b) { return key[a] < key[b]; });
    }
    m->cell_new.assign(nC, 0);
    for (int i = 0; i < nC; i++) m->cell_new[cold[i]] = i;
    const std::vector<int32_t> &cn = m->cell_new;

    std::vector<int32_t> eold(nE), vold(nV);
    std::iota(eold.begin(), eold.end(), 0);
    std::iota(vold.begin(), vold.end(), 0);
    if (desc->sfc_reorder) {
        std::vector<uint64_t> ek(nE), vk(nV);
        for (int e = 0; e < nE; e++) {
            uint64_t a = cn[desc->cells_on_edge[2 * e]], b = cn[desc->cells_on_edge[2 * e + 1]];
            ek[e] = (std::min(a, b) << 32) | std::max(a, b);
        }
        for (int v = 0; v < nV; v++) {
            uint64_t c[3];
            for (int j = 0; j < 3; j++) c[j] = cn[desc->cells_on_vertex[3 * v + j]];
            std::sort(c, c + 3);
            vk[v] = (c[0] << 42) | (c[1] << 21) | c[2];
        }
        std::stable_sort(eold.begin(), eold.end(), [&](int a, int b) { return ek[a] < ek[b]; });
        std::stable_sort(vold.begin(), vold.end(), [&](int a, int b) { return vk[a] < vk[b]; });
    }
    m->edge_new.assign(nE, 0);
    m->vertex_new.assign(nV, 0);
    for (int e = 0; e < nE; e++) m->edge_new[eold[e]] = e;
    for (int v = 0; v < nV; v++) m->vertex_new[vold[v]] = v;
    const std::vector<int32_t> &en = m->edge_new, &vn = m->vertex_new;

    // ---- host packing (new numbering) ---------------------------------
    std::vector<int32_t> eoc(6 * (size_t)nC), coc(6 * (size_t)nC);
    std::vector<double> cdiv(6 * (size_t)nC), kec(6 * (size_t)nC), area(nC);
    std::vector<float> cdiv_f(6 * (size_t)nC);
    for (int i = 0; i < nC; i++) {
        int o = cold[i];
        int n = desc->n_edges_on_cell[o];
        double A = desc->cell_area[o];
        area[i] = A;
        for (int j = 0; j < 6; j++) {
            size_t x = (size_t)i * 6 + j;
            if (j < n) {
                int e = desc->edges_on_cell[o * 6 + j];
                eoc[x] = en[e];
                coc[x] = cn[desc->cells_on_cell[o * 6 + j]];
                cdiv[x] = desc->edge_sign_on_cell[o * 6 + j] * desc->edge_dv[e] / A;
                kec[x] = 0.5 * desc->edge_dc[e] * desc->edge_dv[e] / A;
            } else {
                eoc[x] = en[desc->edges_on_cell[o * 6]];
                coc[x] = i;
                cdiv[x] = 0.0;
                kec[x] = 0.0;
            }
            cdiv_f[x] = (float)cdiv[x];
        }
    }
    // padded rows of 8 of the per-cell lists (entries 6 and 7: eoc[i][0],
    // the cell itself, weight 0) for 16-byte vector reads
    std::vector<int32_t> eoc8(8 * (size_t)nC), coc8(8 * (size_t)nC);
    std::vector<double> cdiv8(8 * (size_t)nC);
    std::vector<float> cdiv8_f(8 * (size_t)nC);
    for (int i = 0; i < nC; i++) {
        for (int j = 0; j < 8; j++) {
            const size_t x = (size_t)i * 8 + j, y = (size_t)i * 6 + j;
            eoc8[x] = j < 6 ? eoc[y] : eoc[(size_t)i * 6];
            coc8[x] = j < 6 ? coc[y] : i;
            cdiv8[x] = j < 6 ? cdiv[y] : 0.0;
            cdiv8_f[x] = (float)cdiv8[x];
        }
    }
    std::vector<int2> coe(nE), voe(nE);
    std::vector<double> rdc(nE), hrdc(nE), dc2(nE), d2c(14 * (size_t)nE), wpv(10 * (size_t)nE);
    std::vector<float> dc2_f(nE), d2c_f(14 * (size_t)nE), wpv_f(10 * (size_t)nE);
    std::vector<int32_t> d2i(14 * (size_t)nE), eoe(10 * (size_t)nE);
    std::vector<int32_t> d2wi(16 * (size_t)nE);
    std::vector<double> d2w(16 * (size_t)nE);
    std::vector<float> d2w_f(16 * (size_t)nE);
    int d2w_ok = 1;
    for (int e = 0; e < nE; e++) {
        int o = eold[e];
        coe[e] = make_int2(cn[desc->cells_on_edge[2 * o]], cn[desc->cells_on_edge[2 * o + 1]]);
        voe[e] = make_int2(vn[desc->vertices_on_edge[2 * o]], vn[desc->vertices_on_edge[2 * o + 1]]);
        double dc = desc->edge_dc[o];
        rdc[e] = 1.0 / dc;
        hrdc[e] = -0.5 / dc;
        dc2[e] = dc * dc / 12.0;
        dc2_f[e] = (float)dc2[e];
        for (int s = 0; s < 2; s++) {
            int centre = desc->cells_on_edge[2 * o + s];
            for (int j = 0; j < GRIST_D2P; j++) {
                size_t x = ((size_t)e * 2 + s) * GRIST_D2P + j;
                int c = desc->d2_stencil[(2 * o + s) * GRIST_D2P + j];
                d2i[x] = cn[c >= 0 ? c : centre];
                d2c[x] = c >= 0 ? desc->d2_coef[(2 * o + s) * GRIST_D2P + j] : 0.0;
                d2c_f[x] = (float)d2c[x];
            }
            // combined weights: the mean of the edge's two cells folded into
            // the upwind side's stencil (first entry of each cell)
            // (rows of 8: the eighth entry is padding, the side's centre cell
            // with weight 0, so that a row is two 16-byte index vectors)
            const size_t b0 = ((size_t)e * 2 + s) * GRIST_D2P, w0 = ((size_t)e * 2 + s) * 8;
            for (int j = 0; j < GRIST_D2P; j++) {
                d2wi[w0 + j] = d2i[b0 + j];
                d2w[w0 + j] = -2.0 * dc2[e] * d2c[b0 + j];
            }
            d2wi[w0 + 7] = cn[centre];
            d2w[w0 + 7] = 0.0;
            const int ends[2] = {coe[e].x, coe[e].y};
            for (int q = 0; q < 2; q++) {
                int at = -1;
                for (int j = 0; j < GRIST_D2P && at < 0; j++)
                    if (d2i[b0 + j] == ends[q]) at = j;
                if (at < 0) d2w_ok = 0;
                else d2w[w0 + at] += 0.5;
            }
            for (int j = 0; j < 8; j++) d2w_f[w0 + j] = (float)d2w[w0 + j];
        }
        int n = desc->n_edges_on_edge[o];
        for (int j = 0; j < GRIST_MAXEOE; j++) {
            size_t x = (size_t)e * 10 + j;
            if (j < n) {
                int e2 = desc->edges_on_edge[o * 10 + j];
                eoe[x] = en[e2];
                wpv[x] = desc->trisk_weight[o * 10 + j] * desc->edge_dv[e2] / dc;
            } else {
                eoe[x] = e;
                wpv[x] = 0.0;
            }
            wpv_f[x] = (float)wpv[x];
        }
    }
    std::vector<int32_t> eov(3 * (size_t)nV), cov(3 * (size_t)nV);
    std::vector<double> ccurl(3 * (size_t)nV), ckite(3 * (size_t)nV), fv(nV);
    std::vector<float> fv_f(nV);
    std::vector<float> ccurl_f(3 * (size_t)nV);
    for (int v = 0; v < nV; v++) {
        int o = vold[v];
        double Av = desc->vertex_area[o];
        fv[v] = desc->f_vertex[o];
        fv_f[v] = (float)fv[v];
        for (int j = 0; j < 3; j++) {
            size_t x = (size_t)v * 3 + j;
            int e = desc->edges_on_vertex[3 * o + j];
            eov[x] = en[e];
            cov[x] = cn[desc->cells_on_vertex[3 * o + j]];
            ccurl[x] = desc->edge_sign_on_vertex[3 * o + j] * desc->edge_dc[e] / Av;
            ccurl_f[x] = (float)ccurl[x];
            ckite[x] = desc->kite_area[3 * o + j] / Av;
        }
    }

    // Every edge side's stencil is its cell's ring {cell, neighbours in the
    // order of the cell's neighbour list}, and the cell is c1 of its edge
    // exactly when its divergence coefficient is positive: then the edge
    // flux can be formed cell-centrically by the upwind cell.
    int ring_ok = d2w_ok;
    for (int i = 0; i < nC && ring_ok; i++) {
        for (int j = 0; j < 6 && ring_ok; j++) {
            const size_t x = (size_t)i * 6 + j;
            if (cdiv[x] == 0.0) continue;   // padding of a pentagon
            const int e = eoc[x];
            const int s = coe[e].x == i ? 0 : (coe[e].y == i ? 1 : -1);
            if (s < 0 || (cdiv[x] > 0.0) != (s == 0)) { ring_ok = 0; break; }
            const int32_t *row = d2wi.data() + ((size_t)e * 2 + s) * 8;
            if (row[0] != i) ring_ok = 0;
            for (int q = 0; q < 6; q++)
                if (row[1 + q] != coc[(size_t)i * 6 + q]) ring_ok = 0;
        }
    }

    // ---- upload into one arena -------------------------------------------
    Arena ar;
    size_t o_eoc = ar.add(eoc.size() * 4), o_coc = ar.add(coc.size() * 4), o_cdiv = ar.add(cdiv.size() * 8),
           o_cdivf = ar.add(cdiv_f.size() * 4), o_kec = ar.add(kec.size() * 8), o_area = ar.add(area.size() * 8),
           o_coe = ar.add(coe.size() * 8), o_voe = ar.add(voe.size() * 8), o_rdc = ar.add(rdc.size() * 8),
           o_hrdc = ar.add(hrdc.size() * 8),
           o_dc2 = ar.add(dc2.size() * 8), o_dc2f = ar.add(dc2_f.size() * 4), o_d2i = ar.add(d2i.size() * 4),
           o_d2c = ar.add(d2c.size() * 8), o_d2cf = ar.add(d2c_f.size() * 4), o_eoe = ar.add(eoe.size() * 4),
           o_d2w = ar.add(d2w.size() * 8), o_d2wf = ar.add(d2w_f.size() * 4), o_d2wi = ar.add(d2wi.size() * 4),
           o_wpv = ar.add(wpv.size() * 8), o_wpvf = ar.add(wpv_f.size() * 4), o_eov = ar.add(eov.size() * 4),
           o_cov = ar.add(cov.size() * 4), o_ccurl = ar.add(ccurl.size() * 8), o_ccurlf = ar.add(ccurl_f.size() * 4),
           o_ckite = ar.add(ckite.size() * 8), o_fv = ar.add(fv.size() * 8), o_fvf = ar.add(fv_f.size() * 4), o_eoc8 = ar.add(eoc8.size() * 4),
           o_coc8 = ar.add(coc8.size() * 4), o_cdiv8 = ar.add(cdiv8.size() * 8), o_cdiv8f = ar.add(cdiv8_f.size() * 4);
    std::vector<char> host(ar.total);
    auto put = [&](size_t off, const void *src, size_t bytes) { std::memcpy(host.data() + off, src, bytes); };
    put(o_eoc, eoc.data(), eoc.size() * 4); put(o_coc, coc.data(), coc.size() * 4);
    put(o_cdiv, cdiv.data(), cdiv.size() * 8); put(o_cdivf, cdiv_f.data(), cdiv_f.size() * 4);
    put(o_kec, kec.data(), kec.size() * 8); put(o_area, area.data(), area.size() * 8);
    put(o_coe, coe.data(), coe.size() * 8); put(o_voe, voe.data(), voe.size() * 8);
    put(o_rdc, rdc.data(), rdc.size() * 8); put(o_dc2, dc2.data(), dc2.size() * 8);
    put(o_hrdc, hrdc.data(), hrdc.size() * 8);
    put(o_dc2f, dc2_f.data(), dc2_f.size() * 4); put(o_d2i, d2i.data(), d2i.size() * 4);
    put(o_d2c, d2c.data(), d2c.size() * 8); put(o_d2cf, d2c_f.data(), d2c_f.size() * 4);
    put(o_d2w, d2w.data(), d2w.size() * 8); put(o_d2wf, d2w_f.data(), d2w_f.size() * 4);
    put(o_d2wi, d2wi.data(), d2wi.size() * 4);
    put(o_eoe, eoe.data(), eoe.size() * 4); put(o_wpv, wpv.data(), wpv.size() * 8);
    put(o_wpvf, wpv_f.data(), wpv_f.size() * 4); put(o_eov, eov.data(), eov.size() * 4);
    put(o_cov, cov.data(), cov.size() * 4); put(o_ccurl, ccurl.data(), ccurl.size() * 8);
    put(o_ccurlf, ccurl_f.data(), ccurl_f.size() * 4); put(o_ckite, ckite.data(), ckite.size() * 8);
    put(o_fv, fv.data(), fv.size() * 8); put(o_fvf, fv_f.data(), fv_f.size() * 4);
    put(o_eoc8, eoc8.data(), eoc8.size() * 4); put(o_coc8, coc8.data(), coc8.size() * 4);
    put(o_cdiv8, cdiv8.data(), cdiv8.size() * 8); put(o_cdiv8f, cdiv8_f.data(), cdiv8_f.size() * 4);

    char *dev = nullptr;
    if (cudaMalloc(&dev, ar.total) != cudaSuccess) { delete m; return GRIST_ENOMEM; }
    if (cudaMemcpy(dev, host.data(), ar.total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dev); delete m; return GRIST_ECUDA;
    }
    if (cudaMalloc(&m->status, 256) != cudaSuccess || cudaMemset(m->status, 0, 256) != cudaSuccess) {
        cudaFree(dev); delete m; return GRIST_ENOMEM;
    }
    m->arena = dev;
    m->ht.nC = nC; m->ht.nE = nE; m->ht.nV = nV;
    m->ht.eoc = eoc;
    m->ht.coe = coe;
    m->ht.d2i = d2i;
    DevMesh &D = m->d;
    D.nC = nC; D.nE = nE; D.nV = nV;
    D.eoc = place<int32_t>(dev, o_eoc); D.coc = place<int32_t>(dev, o_coc);
    D.cdiv = place<double>(dev, o_cdiv); D.cdiv_f = place<float>(dev, o_cdivf);
    D.eoc8 = place<int32_t>(dev, o_eoc8); D.coc8 = place<int32_t>(dev, o_coc8);
    D.cdiv8 = place<double>(dev, o_cdiv8); D.cdiv8_f = place<float>(dev, o_cdiv8f);
    D.kec2 = place<double>(dev, o_kec); D.area = place<double>(dev, o_area);
    D.coe = place<int2>(dev, o_coe); D.voe = place<int2>(dev, o_voe);
    D.rdc = place<double>(dev, o_rdc); D.hrdc = place<double>(dev, o_hrdc);
    D.dc2 = place<double>(dev, o_dc2); D.dc2_f = place<float>(dev, o_dc2f);
    D.d2i = place<int32_t>(dev, o_d2i); D.d2c = place<double>(dev, o_d2c); D.d2c_f = place<float>(dev, o_d2cf);
    D.d2w = place<double>(dev, o_d2w); D.d2w_f = place<float>(dev, o_d2wf); D.d2wi = place<int32_t>(dev, o_d2wi);
    D.d2w_ok = d2w_ok;
    D.ring_ok = ring_ok;
    D.eoe = place<int32_t>(dev, o_eoe); D.wpv = place<double>(dev, o_wpv); D.wpv_f = place<float>(dev, o_wpvf);
    D.eov = place<int32_t>(dev, o_eov); D.cov = place<int32_t>(dev, o_cov);
    D.ccurl = place<double>(dev, o_ccurl); D.ccurl_f = place<float>(dev, o_ccurlf);
    D.ckite = place<double>(dev, o_ckite); D.fv = place<double>(dev, o_fv); D.fv_f = place<float>(dev, o_fvf);
    *out = m;
    return GRIST_OK;
}

extern "C" int grist_profile_enable(grist_mesh m, int enable) {
    if (!m) return GRIST_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return GRIST_ECUDA;
    if (enable && m->ev.empty()) {
        m->ev.resize(2 * kEventPairs);
        for (auto &e : m->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return GRIST_ECUDA;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return GRIST_ECUDA;
    m->pend_name.clear();
    m->prof_names.clear();
    m->prof_ms.clear();
    m->prof_count.clear();
    m->prof_on = enable != 0;
    return GRIST_OK;
}

extern "C" int grist_profile_read(grist_mesh m, int32_t max_entries, char *names, int32_t *launches,
                                  double *total_ms, int32_t *n_entries) {
    if (!m || !n_entries || max_entries < 0) return GRIST_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return GRIST_ECUDA;
    prof_drain(m);
    int n = (int)std::min<size_t>(m->prof_names.size(), (size_t)max_entries);
    for (int j = 0; j < n; j++) {
        if (names) {
            std::strncpy(names + 64 * j, m->prof_names[j].c_str(), 63);
            names[64 * j + 63] = 0;
        }
        if (launches) launches[j] = m->prof_count[j];
        if (total_ms) total_ms[j] = m->prof_ms[j];
    }
    *n_entries = n;
    return GRIST_OK;
}

extern "C" int grist_mesh_destroy(grist_mesh m) {
    if (!m) return GRIST_OK;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (auto &e : m->ev) cudaEventDestroy(e);
    tracer_ctx_free(m->tctx);
    for (int s = 0; s < 8; s++)
        if (m->scr[s]) cudaFree(m->scr[s]);
    if (m->arena) cudaFree(m->arena);
    if (m->status) cudaFree(m->status);
    delete m;
    return GRIST_OK;
}

extern "C" int grist_mesh_permutation(grist_mesh m, int32_t *cell_new_of_old, int32_t *edge_new_of_old,
                                      int32_t *vertex_new_of_old) {
    if (!m) return GRIST_EINVAL;
    if (cell_new_of_old) std::memcpy(cell_new_of_old, m->cell_new.data(), sizeof(int32_t) * m->nC);
    if (edge_new_of_old) std::memcpy(edge_new_of_old, m->edge_new.data(), sizeof(int32_t) * m->nE);
    if (vertex_new_of_old) std::memcpy(vertex_new_of_old, m->vertex_new.data(), sizeof(int32_t) * m->nV);
    return GRIST_OK;
}

extern "C" int grist_mesh_counts(grist_mesh m, int32_t *nC, int32_t *nE, int32_t *nV) {
    if (!m) return GRIST_EINVAL;
    if (nC) *nC = m->nC;
    if (nE) *nE = m->nE;
    if (nV) *nV = m->nV;
    return GRIST_OK;
}

extern "C" int grist_mesh_features(grist_mesh m, uint32_t *flags) {
    if (!m || !flags) return GRIST_EINVAL;
    *flags = (m->d.d2w_ok ? GRIST_MESH_COMBINED_STENCIL : 0u) | (m->d.ring_ok ? GRIST_MESH_RING_STENCIL : 0u);
    return GRIST_OK;
}

extern "C" int grist_last_step_status(grist_mesh m, uint32_t *flags) {
    if (!m || !flags) return GRIST_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return GRIST_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GRIST_ECUDA;
    if (cudaMemcpy(flags, m->status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return GRIST_ECUDA;
    if (cudaMemset(m->status, 0, sizeof(uint32_t)) != cudaSuccess) return GRIST_ECUDA;
    return GRIST_OK;
}

extern "C" const char *grist_status_string(int s) {
    switch (s) {
        case GRIST_OK: return "ok";
        case GRIST_EINVAL: return "invalid argument or mesh tables";
        case GRIST_ECUDA: return "CUDA runtime error";
        case GRIST_ENOMEM: return "out of memory";
        case GRIST_ENUMERIC: return "non-finite values produced";
        case GRIST_ETIMEOUT: return "bounded device wait gave up";
        case GRIST_EUNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}
