"""Pins of the oracle's vertical tracer transport (the delta(M q) term of
Eq. 10, adaptively implicit upwind; orc_tracer_vertical) and of the
vertical mass flux the dycore accumulates for it:

* fully implicit limit (cmax = 0) with uniform downward flow: the textbook
  backward-Euler upwind recursion q_k = (q*_k + c q_{k-1}) / (1 + c);
* explicit limit (Courant numbers below cmax) with uniform flow: forward-
  time backward-space upwind q_k = q*_k - c (q*_k - q*_{k-1});
* flipping a column and the sign of its flux flips the result (catches a
  wrong donor or sign in the upward branch);
* any flux and any cmax: constants stay constant, column mass is conserved,
  no new extrema;
* the dycore's accumulated horizontal and vertical final-stage fluxes close
  the layer continuity: dpi^{n+1} = dpi^n - dt (div F + M_{k+1} - M_k).
"""
import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S


def _uniform_column(L, m, delta):
    Mv = np.zeros((1, L + 1))
    Mv[0, 1:L] = m
    return Mv, np.full((1, L), delta)


def test_fully_implicit_uniform_downward_flow_is_backward_euler_upwind():
    L, delta, m, dt = 12, 800.0, 3.0, 600.0        # c = m dt / delta = 2.25
    Mv, dpi = _uniform_column(L, m, delta)
    q0 = np.random.default_rng(1).uniform(0.0, 1.0, (1, 1, L))
    got = O.tracer_vertical_step(q0, dpi, Mv, dt, cmax=0.0)[0, 0]
    c = m * dt / delta
    ref = np.empty(L)
    ref[0] = q0[0, 0, 0]                              # no inflow through the lid
    for k in range(1, L):
        ref[k] = (q0[0, 0, k] + c * ref[k - 1]) / (1.0 + c)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


def test_explicit_limit_uniform_flow_is_upwind():
    L, delta, m, dt = 10, 1000.0, 2.0, 200.0       # c = 0.4 < cmax
    Mv, dpi = _uniform_column(L, m, delta)
    q0 = np.random.default_rng(2).uniform(0.0, 1.0, (1, 1, L))
    got = O.tracer_vertical_step(q0, dpi, Mv, dt, cmax=1.0)[0, 0]
    c = m * dt / delta
    q = q0[0, 0]
    # interior layers: mass unchanged, FTBS; top layer loses mass, keeps q;
    # bottom layer gains mass through its top
    ref = q.copy()
    ref[1:L - 1] = q[1:L - 1] - c * (q[1:L - 1] - q[0:L - 2])
    ref[L - 1] = (delta * q[L - 1] + dt * m * q[L - 2]) / (delta + dt * m)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("cmax", [0.0, 0.7, 1e9])
def test_flip_symmetry(cmax):
    rng = np.random.default_rng(3)
    L, dt = 15, 300.0
    Mv = np.zeros((4, L + 1))
    Mv[:, 1:L] = rng.uniform(-5, 5, (4, L - 1))
    dpi = rng.uniform(500, 1500, (4, L))
    q0 = rng.uniform(0, 1, (2, 4, L))
    a = O.tracer_vertical_step(q0, dpi, Mv, dt, cmax)
    b = O.tracer_vertical_step(q0[:, :, ::-1], dpi[:, ::-1], -Mv[:, ::-1], dt, cmax)
    np.testing.assert_allclose(a, b[:, :, ::-1], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("cmax", [0.0, 0.5, 1.0, 1e9])
def test_invariants_random_columns(cmax):
    rng = np.random.default_rng(4)
    nC, L, dt = 50, 40, 400.0
    # a large column-wide flux of either sign, tapered to zero at the lid and
    # the ground (Courant numbers up to ~6), plus a small convergent /
    # divergent part, so no layer empties
    prof = np.sin(np.pi * np.arange(L + 1) / L)
    Mv = rng.uniform(-10, 10, (nC, 1)) * prof[None, :]
    Mv[:, 1:L] += rng.uniform(-0.2, 0.2, (nC, L - 1))
    Mv[:, 0] = Mv[:, L] = 0.0
    dpi = rng.uniform(600, 1200, (nC, L))
    dpn = dpi - dt * np.diff(Mv, axis=1)
    assert dpn.min() > 0
    # free stream
    const = O.tracer_vertical_step(np.full((1, nC, L), 2.5), dpi, Mv, dt, cmax)
    assert np.max(np.abs(const - 2.5)) <= 1e-13
    # column mass and bounds
    q0 = rng.uniform(0.1, 1.0, (3, nC, L))
    q1 = O.tracer_vertical_step(q0, dpi, Mv, dt, cmax)
    m0 = np.sum(dpi[None] * q0, axis=2)
    m1 = np.sum(dpn[None] * q1, axis=2)
    assert np.max(np.abs(m1 - m0) / m0) <= 1e-13
    lo, hi = q0.min(axis=2, keepdims=True), q0.max(axis=2, keepdims=True)
    if cmax <= 1.0:                                      # explicit share within its CFL limit
        assert np.all(q1 >= lo - 1e-13) and np.all(q1 <= hi + 1e-13)


def test_dycore_vertical_flux_closes_layer_continuity(mesh_cache):
    m = mesh_cache(3)
    M = O.Mesh(m)
    L = 15
    for nh in (False, True):
        st = S.dycore_jet_case(m, L, nonhydrostatic=nh, bubble=nh)
        P = O.Params(L, st["b_int"], st["pi_top"], st["phi_s"])
        fa = np.zeros((m["n_edges"], L))
        va = np.zeros((m["n_cells"], L + 1))
        dt = 60.0 if nh else 300.0
        r = (O.dycore_step_nh if nh else O.dycore_step_hydro)(M, P, st, dt, flux_accum=fa, vflux_accum=va)
        def dpi_of(ps):
            return np.diff(st["pi_top"] + st["b_int"][None, :] * (ps[:, None] - st["pi_top"]), axis=1)
        lhs = dpi_of(r["ps"])
        rhs = dpi_of(st["ps"]) - dt * (O.divergence(M, fa) + np.diff(va, axis=1))
        assert np.max(np.abs(lhs - rhs)) / np.max(lhs) <= 1e-13, nh
        assert np.all(va[:, 0] == 0) and np.all(va[:, L] == 0)
