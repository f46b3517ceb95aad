"""Pins of the oracle's tracer transport (Eq. 10, Sec. 2.1) - CPU only.

I5  free-stream preservation (constant q stays constant, FCT on/off, even
    for a divergent mass flux)
I6  global tracer-mass conservation to round-off
I7  FCT: no new extrema (slotted cylinder); without FCT overshoots appear
I8  third-order flux reduces to (-q[i-1] + 5 q[i] + 2 q[i+1])/6 on a uniform
    1-D stencil (and the fourth-order centred form at beta = 0)
I9  solid-body rotation: the bell's centre moves to lon 300 after one day
I10 convergence order of a smooth hill under rotation across mesh levels
I11 the RK3 step is the polynomial 1 + z + z^2/2 + z^3/6 of the spatial
    operator (Wicker-Skamarock stage weights dt/3, dt/2, dt)
I15 compensated sums agree with math.fsum
"""
import math

import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S
from grist_inputs.mesh import lonlat


def _ring_mesh(n, dx):
    """Periodic 1-D ring of n cells written as a mesh table set: edge e joins
    cell e (c1) and cell e+1 (c2); deriv-two stencil = (q[c-1] - 2 q[c] +
    q[c+1]) / dx^2 on both sides."""
    nC = nE = n
    cells_on_edge = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    st = -np.ones((nE, 2, 7), np.int32)
    cf = np.zeros((nE, 2, 7))
    for s in range(2):
        c = cells_on_edge[:, s]
        st[:, s, 0], st[:, s, 1], st[:, s, 2] = c, (c - 1) % n, (c + 1) % n
        cf[:, s, 0], cf[:, s, 1], cf[:, s, 2] = -2 / dx ** 2, 1 / dx ** 2, 1 / dx ** 2
    eoc = -np.ones((nC, 6), np.int32)
    eoc[:, 0] = np.arange(n); eoc[:, 1] = (np.arange(n) - 1) % n
    coc = -np.ones((nC, 6), np.int32)
    coc[:, 0] = (np.arange(n) + 1) % n; coc[:, 1] = (np.arange(n) - 1) % n
    sgn = np.zeros((nC, 6)); sgn[:, 0] = 1.0; sgn[:, 1] = -1.0
    z1 = np.zeros((1, 3), np.int32)
    return {
        "n_cells": nC, "n_edges": nE, "n_vertices": 1, "radius": 1.0,
        "cell_area": np.full(nC, dx), "vertex_area": np.ones(1), "edge_dc": np.full(nE, dx),
        "edge_dv": np.ones(nE), "f_vertex": np.zeros(1), "cells_on_edge": cells_on_edge,
        "vertices_on_edge": np.zeros((nE, 2), np.int32), "n_edges_on_cell": np.full(nC, 2, np.int32),
        "edges_on_cell": eoc, "cells_on_cell": coc, "edge_sign_on_cell": sgn,
        "edges_on_vertex": z1, "cells_on_vertex": z1, "edge_sign_on_vertex": np.zeros((1, 3)),
        "kite_area": np.zeros((1, 3)), "n_edges_on_edge": np.zeros(nE, np.int32),
        "edges_on_edge": -np.ones((nE, 10), np.int32), "trisk_weight": np.zeros((nE, 10)),
        "d2_stencil": st, "d2_coef": cf,
    }


def test_third_order_flux_1d_reduction():
    n, dx = 16, 3.0
    M = O.Mesh(_ring_mesh(n, dx))
    q = np.random.default_rng(7).standard_normal((n, 1))
    i = np.arange(n)
    qm, q0, qp, qpp = q[(i - 1) % n, 0], q[i, 0], q[(i + 1) % n, 0], q[(i + 2) % n, 0]
    pos = O.edge_flux_3rd(M, q, np.ones((n, 1)), beta=1.0)[:, 0]
    assert np.allclose(pos, (-qm + 5 * q0 + 2 * qp) / 6, rtol=0, atol=1e-14)
    neg = O.edge_flux_3rd(M, q, -np.ones((n, 1)), beta=1.0)[:, 0]
    assert np.allclose(-neg, (2 * q0 + 5 * qp - qpp) / 6, rtol=0, atol=1e-14)
    cen = O.edge_flux_3rd(M, q, np.ones((n, 1)), beta=0.0)[:, 0]
    assert np.allclose(cen, (-qm + 7 * q0 + 7 * qp - qpp) / 12, rtol=0, atol=1e-14)


@pytest.mark.parametrize("fct", [False, True])
def test_free_stream_divergent_flux(mesh_cache, fct):
    m = mesh_cache(3)
    M = O.Mesh(m)
    L = 4
    rng = np.random.default_rng(8)
    F = rng.standard_normal((m["n_edges"], L)) * 3e4       # divergent, ~10 m/s x 3000 Pa
    dpi = np.full((m["n_cells"], L), 3000.0)
    q = np.full((2, m["n_cells"], L), 1.234)
    out = O.tracer_step(M, q, dpi, F, 600.0, fct=fct)
    assert np.max(np.abs(out - 1.234)) < 1e-13


@pytest.mark.parametrize("fct", [False, True])
def test_tracer_mass_conservation(mesh_cache, fct):
    m = mesh_cache(4)
    M = O.Mesh(m)
    L = 3
    rng = np.random.default_rng(9)
    F = rng.standard_normal((m["n_edges"], L)) * 1e4
    dpi = 3000.0 + rng.uniform(0, 100, (m["n_cells"], L))
    q = S.tracer_mixture(m, 2, L, rng)
    dt = 300.0
    out = O.tracer_step(M, q, dpi, F, dt, fct=fct)
    dpi_new = dpi - dt * O.divergence(M, F)
    for t in range(2):
        before = O.tracer_mass(M, q[t], dpi)[0]
        after = O.tracer_mass(M, out[t], dpi_new)[0]
        assert abs(after - before) / abs(before) < 1e-13


def test_fct_no_new_extrema(mesh_cache):
    m = mesh_cache(4)
    M = O.Mesh(m)
    R = m["radius"]
    c = S.tracer_rotation_case(m, n_levels=1)
    cyl = S.slotted_cylinder(m, math.radians(270), 0.0, R / 2, 1.0, 0.15, 0.4)
    q0 = np.stack([cyl[:, None], (0.5 + 0.5 * (S.cosine_bell(m, math.radians(200), 0.3, R / 3, 1.0)))[:, None]])
    lo, hi = q0.min(axis=(1, 2)), q0.max(axis=(1, 2))
    q = q0.copy()
    for _ in range(24):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], c["dt"], fct=True)
    for t in range(2):
        assert q[t].min() >= lo[t] - 1e-12 * (hi[t] - lo[t])
        assert q[t].max() <= hi[t] + 1e-12 * (hi[t] - lo[t])
    # without the limiter the third-order scheme over/undershoots
    q = q0.copy()
    for _ in range(24):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], c["dt"], fct=False)
    assert q[0].min() < -1e-3 or q[0].max() > 1 + 1e-3


def test_rk3_polynomial(mesh_cache):
    m = mesh_cache(2)
    M = O.Mesh(m)
    nC = m["n_cells"]
    c = S.tracer_rotation_case(m, n_levels=1)
    F, dpi, dt = c["mass_flux"], c["dpi"], 4 * 3600.0
    A = np.zeros((nC, nC))
    S1 = np.zeros((nC, nC))
    for j in range(nC):
        e = np.zeros((nC, 1)); e[j] = 1.0
        A[:, j] = -O.divergence(M, O.edge_flux_3rd(M, e, F))[:, 0] / dpi[:, 0]
        S1[:, j] = O.tracer_step(M, e[None], dpi, F, dt, fct=False)[0, :, 0]
    hA = dt * A
    P = np.eye(nC) + hA + hA @ hA / 2 + hA @ hA @ hA / 6
    assert np.max(np.abs(S1 - P)) < 1e-12
    assert np.max(np.abs(hA)) > 0.1            # the test is not trivially small


def test_rotation_one_day_and_revolution(mesh_cache):
    m = mesh_cache(4)
    M = O.Mesh(m)
    c = S.tracer_rotation_case(m, n_levels=1)
    q = c["q"].copy()
    for _ in range(48):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], c["dt"])
    lon, lat = lonlat(m["cell_xyz"])
    w = q[0, :, 0] / q[0, :, 0].sum()
    # mass-weighted centre of the bell (on the equator)
    x = np.sum(w * np.cos(lon) * np.cos(lat)); y = np.sum(w * np.sin(lon) * np.cos(lat))
    assert abs(math.degrees(math.atan2(y, x)) % 360 - 300.0) < 1.0
    ex = S.bell_exact(m, 48 * c["dt"], c["u0"])
    assert O.error_norms(q[0, :, 0], ex, m["cell_area"])[1] < 0.12
    for _ in range(576 - 48):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], c["dt"])
    l1, l2, linf = O.error_norms(q[0, :, 0], c["q"][0, :, 0], m["cell_area"])
    assert l2 < 0.5 and q.min() > -1e-10 and q.max() <= 1000.0


def _hill_rotation_error(m, steps_per_day):
    M = O.Mesh(m)
    R = m["radius"]
    c = S.tracer_rotation_case(m, n_levels=1)
    lon0, lat0, width = math.radians(270.0), 0.0, R / 6
    q = S.gaussian_hill(m, lon0, lat0, width, 1.0)[None, :, None]
    dt = 86400.0 / steps_per_day
    for _ in range(steps_per_day):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], dt, fct=False)
    ex = S.gaussian_hill(m, lon0 + c["u0"] * 86400.0 / R, lat0, width, 1.0)
    return O.error_norms(q[0, :, 0], ex, m["cell_area"])


def test_convergence_order(mesh_cache):
    errs = [_hill_rotation_error(mesh_cache(lev), 12 * 2 ** (lev - 3)) for lev in (3, 4, 5, 6)]
    l2 = np.array([e[1] for e in errs])
    order = np.log2(l2[:-1] / l2[1:])
    assert order[-1] >= 1.8, (l2, order)
    assert np.all(order > 1.5), (l2, order)


def test_compensated_sum_vs_fsum():
    rng = np.random.default_rng(11)
    for trial in range(20):
        n = 10000
        big = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 12, n)
        x = np.concatenate([big, -big[: n // 2] * (1 + 1e-9), rng.standard_normal(100)])
        rng.shuffle(x)
        got = O.compensated_sum(x)[0]
        exact = math.fsum(x)
        assert abs(got - exact) <= 2 * np.spacing(abs(exact)), (got, exact)
    w = rng.uniform(1, 2, 5000)
    x = rng.standard_normal(5000)
    assert abs(O.compensated_sum(x, w)[0] - math.fsum(w * x)) <= 2 * np.spacing(abs(math.fsum(w * x))) + \
        4 * np.finfo(float).eps * np.sum(np.abs(w * x)) * 1e-3
