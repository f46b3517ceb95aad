"""Icosahedral spherical Voronoi C-grid generator (input data, FP64, host).

The paper runs GRIST on the hexagonal Arakawa-C grid of a recursively bisected
icosahedron (Sec. 2.1; Table 1 lists G6 = 40,962, G7 = 163,842, G8 = 655,362
cells, i.e. 10*4^n + 2 cells at bisection level n).  This module builds that
grid and every static table the operators read:

* the triangular (Delaunay) mesh of generators by n bisections of the
  icosahedron, every new point the normalised midpoint of its parent edge;
* its Voronoi dual: one cell per generator, one Voronoi vertex per triangle at
  the spherical circumcentre, one edge per triangle side;
* lengths, kite / cell / vertex areas, orientation signs;
* the tangential-reconstruction (TRiSK-family) weights of each edge and the
  deriv-two stencils (normal second derivative at each side of an edge from a
  least-squares quadratic fit in the cell's gnomonic tangent plane).

Conventions (shared by every consumer of the tables):

* ``cells_on_edge[e] = (c1, c2)``; the edge normal ``n_e`` points c1 -> c2 and
  a positive normal velocity blows from c1 to c2.
* ``t_e = k x n_e`` (k the outward radial unit vector);
  ``vertices_on_edge[e] = (v1, v2)`` with ``v2 - v1`` along ``t_e``.
* ``edges_on_cell`` / ``cells_on_cell`` / ``vertices_on_cell`` are in
  counter-clockwise order seen from outside; vertex k lies between edge k and
  edge k+1.  Pentagons pad slot 5 with -1 (sign 0, weights 0).
* ``edge_sign_on_cell[i][k] = +1`` when ``n_e`` points out of cell i.
* ``edge_sign_on_vertex[v][j] = +1`` when ``n_e`` points counter-clockwise
  around v (positive circulation).
* Arrays are returned in the generator's own numbering; a consumer that wants
  a different order permutes them itself.

Everything is vectorised NumPy in float64 / int32.  Nothing here is part of
the time step: these are the grid description handed to ``grist_mesh_create``.
"""
from __future__ import annotations

import math

import numpy as np

EARTH_RADIUS = 6.371e6
OMEGA = 7.292e-5

MAX_EDGES = 6      # hexagon; pentagons pad one slot
MAX_EOE = 10       # edges_on_edge: (n1 - 1) + (n2 - 1)
D2_PTS = 7         # cell + up to 6 neighbours


def n_cells(level: int) -> int:
    return 10 * 4 ** level + 2


def n_edges(level: int) -> int:
    return 30 * 4 ** level


def n_vertices(level: int) -> int:
    return 20 * 4 ** level


# ----------------------------------------------------------------------------
# triangular mesh
# ----------------------------------------------------------------------------

def _icosahedron():
    """12 vertices on the unit sphere and the 20 faces, each ordered
    counter-clockwise seen from outside.  Faces are found as the triples of
    mutually nearest vertices rather than typed in."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            pts += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    xyz = np.array(pts, dtype=np.float64)
    xyz /= np.linalg.norm(xyz, axis=1, keepdims=True)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    edge_len = np.min(d[d > 1e-9])
    adj = np.abs(d - edge_len) < 1e-9
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    a, b, c = xyz[i], xyz[j], xyz[k]
                    if np.dot(np.cross(b - a, c - a), a + b + c) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    faces = np.array(faces, dtype=np.int64)
    assert faces.shape == (20, 3)
    return xyz, faces


def _bisect(xyz, faces):
    """One bisection: every triangle splits into four; new points are the
    normalised midpoints of the parent edges (shared edges dedup'd)."""
    nv = xyz.shape[0]
    a, b, c = faces[:, 0], faces[:, 1], faces[:, 2]
    ends = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 0)
    lo = np.minimum(ends[..., 0], ends[..., 1])
    hi = np.maximum(ends[..., 0], ends[..., 1])
    key = lo * nv + hi
    uniq, inv = np.unique(key.ravel(), return_inverse=True)
    ulo, uhi = uniq // nv, uniq % nv
    mid = xyz[ulo] + xyz[uhi]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    new_xyz = np.concatenate([xyz, mid], 0)
    m = inv.reshape(3, -1) + nv
    mab, mbc, mca = m[0], m[1], m[2]
    f = np.concatenate([
        np.stack([a, mab, mca], 1),
        np.stack([b, mbc, mab], 1),
        np.stack([c, mca, mbc], 1),
        np.stack([mab, mbc, mca], 1),
    ], 0)
    return new_xyz, f


def triangular_mesh(level: int):
    xyz, faces = _icosahedron()
    for _ in range(level):
        xyz, faces = _bisect(xyz, faces)
    return xyz, faces


# ----------------------------------------------------------------------------
# spherical geometry helpers (unit vectors)
# ----------------------------------------------------------------------------

def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _arc(a, b):
    """Great-circle angle between unit vectors (robust atan2 form)."""
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def _tri_area(a, b, c):
    """Spherical excess of the triangle (a, b, c) on the unit sphere
    (Van Oosterom & Strackee)."""
    num = np.abs(np.sum(a * np.cross(b, c), axis=-1))
    den = 1.0 + np.sum(a * b, -1) + np.sum(b * c, -1) + np.sum(c * a, -1)
    return 2.0 * np.arctan2(num, den)


def _tangent_basis(p):
    """Orthonormal (e1, e2) tangent to the unit sphere at p with (e1, e2, p)
    right-handed, so increasing atan2(y, x) is counter-clockwise from outside."""
    ax = np.zeros_like(p)
    small = np.argmin(np.abs(p), axis=1)
    ax[np.arange(p.shape[0]), small] = 1.0
    e1 = _unit(np.cross(ax, p))
    e2 = np.cross(p, e1)
    return e1, e2


# ----------------------------------------------------------------------------
# Voronoi C-grid
# ----------------------------------------------------------------------------

def build_mesh(level: int, radius: float = EARTH_RADIUS, omega: float = OMEGA):
    """Return a dict with every grid table (original numbering)."""
    xc, faces = triangular_mesh(level)
    nC = xc.shape[0]
    nV = faces.shape[0]
    R = float(radius)

    # Voronoi vertices: spherical circumcentres of the (ccw) triangles
    fa, fb, fc = xc[faces[:, 0]], xc[faces[:, 1]], xc[faces[:, 2]]
    xv = _unit(np.cross(fb - fa, fc - fa))

    # directed half-edges a->b of every face, face id and slot
    src = faces.ravel()
    dst = faces[:, [1, 2, 0]].ravel()
    hface = np.repeat(np.arange(nV, dtype=np.int64), 3)
    dkey = src * nC + dst
    order = np.argsort(dkey, kind="stable")
    dkey_sorted = dkey[order]
    face_of_sorted = hface[order]

    def face_of(a, b):
        k = a.astype(np.int64) * nC + b.astype(np.int64)
        pos = np.searchsorted(dkey_sorted, k)
        assert np.all(dkey_sorted[pos] == k)
        return face_of_sorted[pos]

    # undirected edges: c1 = smaller generator id, c2 = larger
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    ukey = np.unique(lo * nC + hi)
    c1 = ukey // nC
    c2 = ukey % nC
    nE = c1.shape[0]
    # face on the left of c1->c2 (the +t side) is v2, the other is v1
    v2 = face_of(c1, c2)
    v1 = face_of(c2, c1)

    cells_on_edge = np.stack([c1, c2], 1)
    vertices_on_edge = np.stack([v1, v2], 1)

    x1, x2 = xc[c1], xc[c2]
    xe = _unit(x1 + x2)                       # edge point: midpoint of the c1-c2 arc
    dc = R * _arc(x1, x2)
    dv = R * _arc(xv[v1], xv[v2])
    ne = _unit((x2 - x1) - np.sum((x2 - x1) * xe, -1, keepdims=True) * xe)

    def edge_id(a, b):
        k = np.minimum(a, b).astype(np.int64) * nC + np.maximum(a, b)
        pos = np.searchsorted(ukey, k)
        assert np.all(ukey[pos] == k)
        return pos

    # --- cells: edges in counter-clockwise order --------------------------
    inc_cell = np.concatenate([c1, c2])
    inc_nbr = np.concatenate([c2, c1])
    inc_edge = np.concatenate([np.arange(nE), np.arange(nE)])
    e1b, e2b = _tangent_basis(xc)
    dvec = xc[inc_nbr] - xc[inc_cell]
    ang = np.arctan2(np.sum(dvec * e2b[inc_cell], -1), np.sum(dvec * e1b[inc_cell], -1))
    srt = np.lexsort((ang, inc_cell))
    inc_cell, inc_nbr, inc_edge = inc_cell[srt], inc_nbr[srt], inc_edge[srt]
    n_eoc = np.bincount(inc_cell, minlength=nC).astype(np.int32)
    start = np.concatenate([[0], np.cumsum(n_eoc)[:-1]])
    slot = np.arange(inc_cell.shape[0]) - start[inc_cell]
    edges_on_cell = -np.ones((nC, MAX_EDGES), np.int64)
    cells_on_cell = -np.ones((nC, MAX_EDGES), np.int64)
    edges_on_cell[inc_cell, slot] = inc_edge
    cells_on_cell[inc_cell, slot] = inc_nbr
    # vertex between edge k and k+1 = face holding the half-edge cell->nbr_k
    vertices_on_cell = -np.ones((nC, MAX_EDGES), np.int64)
    vertices_on_cell[inc_cell, slot] = face_of(inc_cell, inc_nbr)
    edge_sign_on_cell = np.zeros((nC, MAX_EDGES), np.float64)
    valid = edges_on_cell >= 0
    ee = np.where(valid, edges_on_cell, 0)
    edge_sign_on_cell[valid] = np.where(c1[ee[valid]] == np.nonzero(valid)[0], 1.0, -1.0)

    # --- vertices: the triangle corners / sides in ccw order ----------------
    cells_on_vertex = faces.copy()
    edges_on_vertex = np.stack([edge_id(faces[:, 0], faces[:, 1]),
                                edge_id(faces[:, 1], faces[:, 2]),
                                edge_id(faces[:, 2], faces[:, 0])], 1)
    trav_from = faces
    trav_to = faces[:, [1, 2, 0]]
    edge_sign_on_vertex = np.where(c1[edges_on_vertex] == trav_from, 1.0, -1.0)
    assert np.all((c1[edges_on_vertex] == trav_from) | (c1[edges_on_vertex] == trav_to))

    # kite of corner j of triangle v: bounded by the sides (j-1 -> j) and (j -> j+1)
    kite = np.zeros((nV, 3), np.float64)
    for j in range(3):
        ca = xc[faces[:, j]]
        e_out = edges_on_vertex[:, j]            # side j -> j+1
        e_in = edges_on_vertex[:, (j + 2) % 3]   # side j-1 -> j
        kite[:, j] = (_tri_area(ca, xe[e_out], xv) + _tri_area(ca, xv, xe[e_in])) * R * R
    vertex_area = kite.sum(1)
    cell_area = np.zeros(nC, np.float64)
    np.add.at(cell_area, faces.ravel(), kite.ravel())

    # kite of cell i at vertices_on_cell[i][k]
    kite_on_cell = np.zeros((nC, MAX_EDGES), np.float64)
    vv = np.where(valid, vertices_on_cell, 0)
    corner = np.argmax(cells_on_vertex[vv] == np.arange(nC)[:, None, None], axis=2)
    kite_on_cell = np.where(valid, kite[vv, corner], 0.0)

    # --- TRiSK tangential-reconstruction weights ----------------------------
    # For cell i with edges e_1..e_m (ccw) and vertex v_k between e_k, e_{k+1},
    # R_k = kite(i, v_k) / A_i.  For edge e = e_p of i and another edge
    # e' = e_{p+j}, S = R_p + ... + R_{p+j-1} (vertices passed going ccw from
    # e to e') and w(e, e') = n(e,i) n(e',i) (1/2 - S).  The tangential mass
    # flux at e is (1/dc_e) sum_e' w(e,e') dv_e' F_e' summed over both cells.
    eoe = -np.ones((nE, MAX_EOE), np.int64)
    weo = np.zeros((nE, MAX_EOE), np.float64)
    n_eoe = np.zeros(nE, np.int32)
    rk = kite_on_cell / cell_area[:, None]
    pos_in_cell = np.full((nE, 2), -1, np.int64)
    for side, cc in enumerate((c1, c2)):
        hit = edges_on_cell[cc] == np.arange(nE)[:, None]
        pos_in_cell[:, side] = np.argmax(hit, 1)
        assert np.all(hit.any(1))
    fill = np.zeros(nE, np.int64)
    for side, cc in enumerate((c1, c2)):
        m = n_eoc[cc].astype(np.int64)
        p = pos_in_cell[:, side]
        s_e = edge_sign_on_cell[cc, p]
        S = np.zeros(nE)
        for j in range(1, MAX_EDGES):
            ok = j < m
            prev = (p + j - 1) % np.maximum(m, 1)
            S = S + np.where(ok, rk[cc, prev], 0.0)
            q = (p + j) % np.maximum(m, 1)
            e2 = edges_on_cell[cc, q]
            s_e2 = edge_sign_on_cell[cc, q]
            w = s_e * s_e2 * (0.5 - S)
            rows = np.nonzero(ok)[0]
            eoe[rows, fill[rows]] = e2[rows]
            weo[rows, fill[rows]] = w[rows]
            fill[rows] += 1
    n_eoe[:] = fill

    # --- deriv-two stencils --------------------------------------------------
    # Per cell: least-squares fit of a + bx + cy + dx^2 + exy + fy^2 over the
    # cell and its neighbours in gnomonic coordinates of the cell's tangent
    # plane.  q'' along direction (nx, ny) = 2 (d nx^2 + e nx ny + f ny^2).
    stencil = np.concatenate([np.arange(nC)[:, None], cells_on_cell], 1)   # [nC, 7]
    sval = stencil >= 0
    pts = xc[np.where(sval, stencil, 0)]                                   # [nC, 7, 3]
    dotc = np.sum(pts * xc[:, None, :], -1)
    gx = R * np.sum(pts * e1b[:, None, :], -1) / dotc
    gy = R * np.sum(pts * e2b[:, None, :], -1) / dotc
    h = R * np.sqrt(cell_area / R ** 2)                                     # ~ cell size
    sx, sy = gx / h[:, None], gy / h[:, None]
    V = np.stack([np.ones_like(sx), sx, sy, sx * sx, sx * sy, sy * sy], -1)
    V = V * sval[..., None]
    VtV = np.einsum("nki,nkj->nij", V, V)
    P = np.linalg.solve(VtV, np.transpose(V, (0, 2, 1)))                   # [nC, 6, 7]
    P2 = P[:, 3:6, :] / (h * h)[:, None, None]                               # d, e, f rows, physical

    d2_stencil = -np.ones((nE, 2, D2_PTS), np.int64)
    d2_coef = np.zeros((nE, 2, D2_PTS), np.float64)
    for side, (cc, other) in enumerate(((c1, c2), (c2, c1))):
        ox = R * np.sum(xc[other] * e1b[cc], -1) / np.sum(xc[other] * xc[cc], -1)
        oy = R * np.sum(xc[other] * e2b[cc], -1) / np.sum(xc[other] * xc[cc], -1)
        nrm = np.sqrt(ox * ox + oy * oy)
        nx, ny = ox / nrm, oy / nrm
        coef = 2.0 * (nx[:, None] * nx[:, None] * P2[cc, 0, :]
                      + nx[:, None] * ny[:, None] * P2[cc, 1, :]
                      + ny[:, None] * ny[:, None] * P2[cc, 2, :])
        d2_stencil[:, side, :] = stencil[cc]
        d2_coef[:, side, :] = np.where(sval[cc], coef, 0.0)

    lat_v = np.arcsin(np.clip(xv[:, 2], -1.0, 1.0))
    f_vertex = 2.0 * omega * np.sin(lat_v)

    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    return {
        "level": level,
        "n_cells": nC, "n_edges": nE, "n_vertices": nV, "max_edges": MAX_EDGES,
        "radius": R, "omega": float(omega),
        "cell_xyz": f64(xc), "vertex_xyz": f64(xv), "edge_xyz": f64(xe),
        "edge_normal_xyz": f64(ne),
        "cell_area": f64(cell_area), "vertex_area": f64(vertex_area),
        "edge_dc": f64(dc), "edge_dv": f64(dv), "f_vertex": f64(f_vertex),
        "cells_on_edge": i32(cells_on_edge), "vertices_on_edge": i32(vertices_on_edge),
        "n_edges_on_cell": i32(n_eoc), "edges_on_cell": i32(edges_on_cell),
        "cells_on_cell": i32(cells_on_cell), "vertices_on_cell": i32(vertices_on_cell),
        "edge_sign_on_cell": f64(edge_sign_on_cell),
        "edges_on_vertex": i32(edges_on_vertex), "cells_on_vertex": i32(cells_on_vertex),
        "edge_sign_on_vertex": f64(edge_sign_on_vertex), "kite_area": f64(kite),
        "n_edges_on_edge": i32(n_eoe), "edges_on_edge": i32(eoe), "trisk_weight": f64(weo),
        "d2_stencil": i32(d2_stencil), "d2_coef": f64(d2_coef),
    }


def lonlat(xyz):
    lon = np.arctan2(xyz[:, 1], xyz[:, 0])
    lat = np.arcsin(np.clip(xyz[:, 2], -1.0, 1.0))
    return lon, lat


_CACHE: dict = {}


def get_mesh(level: int, cache_dir: str | None = None):
    """Memoised ``build_mesh(level)`` for the default Earth radius; with
    ``cache_dir`` (or the GRIST_MESH_CACHE environment variable) the tables
    are also kept on disk as one uncompressed .npz per level."""
    import os
    if level in _CACHE:
        return _CACHE[level]
    cache_dir = cache_dir or os.environ.get("GRIST_MESH_CACHE")
    path = os.path.join(cache_dir, "grist_mesh_L%d.npz" % level) if cache_dir else None
    if path and os.path.exists(path):
        with np.load(path) as z:
            m = {k: (z[k] if z[k].ndim else z[k].item()) for k in z.files}
        for k in ("level", "n_cells", "n_edges", "n_vertices", "max_edges"):
            m[k] = int(m[k])
        for k in ("radius", "omega"):
            m[k] = float(m[k])
    else:
        m = build_mesh(level)
        if path:
            os.makedirs(cache_dir, exist_ok=True)
            tmp = path + ".%d.tmp.npz" % os.getpid()
            np.savez(tmp, **m)
            os.replace(tmp, path)
    _CACHE[level] = m
    return m
