"""Pins of the grid tables and the oracle's C-grid operators (CPU only).

I1  counts, Euler characteristic, 12 pentagons, areas (Table 1 counts)
I2  div(curl psi) = 0 for any vertex stream function
I3  curl(grad h) = 0 on vertices
I4  TRiSK tangential reconstruction: antisymmetry / energy neutrality and
    the dual-divergence identity (perp flux out of each dual triangle equals
    the kite-weighted share of the primal divergence)
I8  deriv-two stencils are exact for tangent-plane quadratics
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from grist_inputs import mesh as gm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cells.txt")


def _table1():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, lev, split, ncell, res = line.split()
        rows.append((name, int(lev), int(split), int(ncell), float(res)))
    return rows


def test_table1_cell_counts():
    """Cells = 10 * (split^2) * 4^n + 2 reproduces every count of Table 1."""
    for name, lev, split, ncell, res in _table1():
        assert 10 * split * split * 4 ** lev + 2 == ncell, name
        if split == 1:
            assert gm.n_cells(lev) == ncell
        # resolution ~ sqrt(cell area): within 10% of the printed spacing
        spacing = math.sqrt(4 * math.pi * gm.EARTH_RADIUS ** 2 / ncell) / 1e3
        assert abs(spacing / res - 1.0) < 0.12, (name, spacing)


@pytest.mark.parametrize("level", [0, 1, 3, 5])
def test_counts_euler_pentagons(mesh_cache, level):
    m = mesh_cache(level)
    nC, nE, nV = m["n_cells"], m["n_edges"], m["n_vertices"]
    assert (nC, nE, nV) == (gm.n_cells(level), gm.n_edges(level), gm.n_vertices(level))
    assert nV - nE + nC == 2
    assert np.sum(m["n_edges_on_cell"] == 5) == 12
    assert np.sum(m["n_edges_on_cell"] == 6) == nC - 12
    # every edge appears in exactly two cells' edge lists and 2 triangles
    eoc = m["edges_on_cell"][m["edges_on_cell"] >= 0]
    assert np.all(np.bincount(eoc, minlength=nE) == 2)
    assert np.all(np.bincount(m["edges_on_vertex"].ravel(), minlength=nE) == 2)


@pytest.mark.parametrize("level", [2, 5])
def test_areas(mesh_cache, level):
    m = mesh_cache(level)
    R = m["radius"]
    sphere = 4 * math.pi * R * R
    assert abs(m["cell_area"].sum() / sphere - 1) < 1e-12
    assert abs(m["vertex_area"].sum() / sphere - 1) < 1e-12
    # cell area from kites == polygon area by fan triangulation (independent)
    xc, xv = m["cell_xyz"], m["vertex_xyz"]
    voc = m["vertices_on_cell"]
    poly = np.zeros(m["n_cells"])
    for k in range(6):
        a = voc[:, k]
        b = np.where(k + 1 < m["n_edges_on_cell"], voc[:, (k + 1) % 6], voc[:, 0])
        ok = a >= 0
        pa, pb = xv[np.where(ok, a, 0)], xv[np.where(ok, b, 0)]
        num = np.abs(np.sum(xc * np.cross(pa, pb), 1))
        den = 1 + np.sum(xc * pa, 1) + np.sum(pa * pb, 1) + np.sum(pb * xc, 1)
        poly += np.where(ok, 2 * np.arctan2(num, den), 0.0)
    assert np.max(np.abs(poly * R * R / m["cell_area"] - 1)) < 1e-10
    # dual triangle area == spherical triangle of the three generators
    cv = m["cells_on_vertex"]
    a, b, c = xc[cv[:, 0]], xc[cv[:, 1]], xc[cv[:, 2]]
    tri = 2 * np.arctan2(np.abs(np.sum(a * np.cross(b, c), 1)),
                         1 + np.sum(a * b, 1) + np.sum(b * c, 1) + np.sum(c * a, 1))
    assert np.max(np.abs(tri * R * R / m["vertex_area"] - 1)) < 1e-10
    # Voronoi property: each circumcentre is equidistant from its 3 generators
    d = [np.arccos(np.clip(np.sum(xv * p, 1), -1, 1)) for p in (a, b, c)]
    assert np.max(np.abs(d[0] - d[1])) < 1e-12 and np.max(np.abs(d[0] - d[2])) < 1e-12


def test_orientation_conventions(mesh_cache):
    m = mesh_cache(3)
    xc, xv, xe, ne = m["cell_xyz"], m["vertex_xyz"], m["edge_xyz"], m["edge_normal_xyz"]
    c1, c2 = m["cells_on_edge"].T
    v1, v2 = m["vertices_on_edge"].T
    assert np.all(np.sum((xc[c2] - xc[c1]) * ne, 1) > 0)          # n: c1 -> c2
    t = np.cross(xe, ne)
    assert np.all(np.sum((xv[v2] - xv[v1]) * t, 1) > 0)          # t = k x n: v1 -> v2
    # dc, dv are great-circle lengths
    R = m["radius"]
    assert np.allclose(m["edge_dc"], R * np.arccos(np.clip(np.sum(xc[c1] * xc[c2], 1), -1, 1)), rtol=1e-10)


@pytest.mark.parametrize("level", [2, 4])
def test_div_curl_zero(mesh_cache, level):
    """I2: u from any vertex stream function has zero discrete divergence."""
    m = mesh_cache(level)
    M = O.Mesh(m)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((m["n_vertices"], 3)) * 1e7
    v1, v2 = m["vertices_on_edge"].T
    u = -(psi[v2] - psi[v1]) / m["edge_dv"][:, None]
    div = O.divergence(M, u * 1000.0)
    scale = np.max(np.abs(u * 1000.0)) * np.max(m["edge_dv"]) / np.min(m["cell_area"])
    assert np.max(np.abs(div)) / scale < 1e-14


@pytest.mark.parametrize("level", [2, 4])
def test_curl_grad_zero(mesh_cache, level):
    """I3: the circulation of a discrete gradient vanishes at every vertex."""
    m = mesh_cache(level)
    M = O.Mesh(m)
    h = np.random.default_rng(2).standard_normal((m["n_cells"], 2)) * 1e4
    g = O.gradient(M, h)
    z = O.vorticity(M, g)
    scale = np.max(np.abs(g)) * np.max(m["edge_dc"]) / np.min(m["vertex_area"])
    assert np.max(np.abs(z)) / scale < 1e-14


def test_trisk_antisymmetric_energy_neutral(mesh_cache):
    """I4: w(e,e') = -w(e',e) and the PV flux does no work:
    sum_e dc dv F_e (PV flux)_e = 0 for any F and vertex PV."""
    m = mesh_cache(3)
    M = O.Mesh(m)
    W = {}
    eoe, w = m["edges_on_edge"], m["trisk_weight"]
    for e in range(m["n_edges"]):
        for j in range(m["n_edges_on_edge"][e]):
            W[(e, eoe[e, j])] = w[e, j]
    assert max(abs(W[(a, b)] + W[(b, a)]) for (a, b) in W) < 1e-14
    rng = np.random.default_rng(3)
    F = rng.standard_normal((m["n_edges"], 2)) * 1e4
    qv = rng.standard_normal((m["n_vertices"], 2)) * 1e-7
    pv = O.pv_flux(M, F, qv)
    work = np.sum(m["edge_dc"][:, None] * m["edge_dv"][:, None] * F * pv, 0)
    scale = np.sum(np.abs(m["edge_dc"][:, None] * m["edge_dv"][:, None] * F * pv), 0)
    assert np.all(np.abs(work) / scale < 1e-13)


@pytest.mark.parametrize("level", [1, 3])
def test_trisk_dual_divergence(mesh_cache, level):
    """I4: the tangential flux leaving each dual triangle equals the
    kite-weighted remap of the primal divergence (the defining property of
    the TRiSK weights), for an arbitrary edge flux."""
    m = mesh_cache(level)
    M = O.Mesh(m)
    F = np.random.default_rng(4).standard_normal((m["n_edges"], 1))
    fp = O.perp_flux(M, F)[:, 0] * m["edge_dc"]          # flux through the full dual edge, +t
    v1, v2 = m["vertices_on_edge"].T
    dual_out = np.zeros(m["n_vertices"])
    np.add.at(dual_out, v1, fp)       # triangle of v1 lies on the -t side: outward = +t
    np.add.at(dual_out, v2, -fp)
    div = O.divergence(M, F)
    remap = O.cell_to_vertex(M, div)[:, 0] * m["vertex_area"]
    assert np.max(np.abs(dual_out - remap)) < 1e-12 * np.max(np.abs(remap))


@pytest.mark.parametrize("level", [3, 5])
def test_deriv_two_quadratic_exact(mesh_cache, level):
    """I8: the deriv-two coefficients return the exact second derivative along
    the edge direction for any quadratic in the cell's gnomonic plane."""
    m = mesh_cache(level)
    R = m["radius"]
    xc = m["cell_xyz"]
    rng = np.random.default_rng(5)
    for side in (0, 1):
        es = rng.choice(m["n_edges"], 300, replace=False)
        for e in es:
            c = m["cells_on_edge"][e, side]
            o = m["cells_on_edge"][e, 1 - side]
            p = xc[c]
            ax = np.zeros(3); ax[np.argmin(np.abs(p))] = 1.0
            e1 = np.cross(ax, p); e1 /= np.linalg.norm(e1); e2 = np.cross(p, e1)
            st = m["d2_stencil"][e, side]
            cf = m["d2_coef"][e, side]
            pts = xc[st[st >= 0]]
            x = R * (pts @ e1) / (pts @ p); y = R * (pts @ e2) / (pts @ p)
            A, B, C, D, E, Fq = rng.standard_normal(6) * np.array([1, 1e-5, 1e-5, 1e-10, 1e-10, 1e-10])
            q = A + B * x + C * y + D * x * x + E * x * y + Fq * y * y
            ox = R * (xc[o] @ e1) / (xc[o] @ p); oy = R * (xc[o] @ e2) / (xc[o] @ p)
            nx, ny = ox / math.hypot(ox, oy), oy / math.hypot(ox, oy)
            exact = 2 * (D * nx * nx + E * nx * ny + Fq * ny * ny)
            got = np.dot(cf[st >= 0], q)
            assert abs(got - exact) < 1e-8 * (abs(D) + abs(E) + abs(Fq)), (e, side)
            assert abs(np.sum(cf)) < 1e-9 * np.max(np.abs(cf))        # constants -> 0


@pytest.mark.parametrize("level", [3, 5])
def test_stencils_are_upwind_cell_rings(mesh_cache, level):
    """The property the cell-centric edge fluxes rely on: the deriv-two
    stencil of side s of every edge is the ring of its cell c_s - the cell
    itself, then its neighbours in the order of cells_on_cell - and the cell
    is c1 of an edge exactly when its edge sign is +1 (so the upwind cell of
    an edge, F >= 0 -> c1, is known from the sign alone)."""
    m = mesh_cache(level)
    c12 = m["cells_on_edge"]
    st = m["d2_stencil"]
    ring = np.concatenate([np.arange(m["n_cells"])[:, None], m["cells_on_cell"]], 1)
    for s in range(2):
        assert np.array_equal(st[:, s, :], ring[c12[:, s]])
    eoc, sgn = m["edges_on_cell"], m["edge_sign_on_cell"]
    valid = eoc >= 0
    cells = np.broadcast_to(np.arange(m["n_cells"])[:, None], eoc.shape)
    is_c1 = c12[np.where(valid, eoc, 0), 0] == cells
    assert np.array_equal((sgn > 0)[valid], is_c1[valid])
    assert np.all(sgn[valid] != 0) and np.all(sgn[~valid] == 0)
