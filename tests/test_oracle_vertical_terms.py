"""Closed-form pins of the oracle's vertical and interface terms - CPU only.

Each term below reaches an exact value on a field whose continuous answer
is known, so a dropped factor, a flipped sign or a shifted interface index
in the oracle fails here (nothing else in the CPU suite reaches these terms
with a non-trivial input):

- eta-dot du/deta in the momentum tendency (Eq. 5): for u linear in the
  layer's mid-level pressure and M linear in pressure on uniform layers the
  M-dependent part of the tendency is -M(pi_k) du/dpi at interior layers;
  at the top and bottom layers only the inner interface carries mass, so
  the term is half of it there (the closed ends of the column).
- the centred vertical advection of interface fields (explicit parts of
  Eqs. 6-7): for x linear in the interface pressure it is M_j dx/dpi at
  every interior interface, for any layer thicknesses, and 0 at the ends.
- the horizontal advection of interface fields (Eqs. 6-7): the Cartesian
  coordinate X of the cell centre under eastward solid-body rotation
  u0 cos(lat) has V.grad X = -(u0/R) Y; the discrete operator converges to
  it under refinement: area-weighted l1 at about order 1.7 and l2 at first
  order over levels 3 -> 6.  The maximum error stays near 6 % on the cells
  along the icosahedron's edges, where the plain bisection mesh is not
  smooth (a property of the mesh, not of the operator; the tracer
  convergence pins see the same).
- the L operator (dp/dpi averaged to layers, Eq. 5): for p equal to c times
  the mid-layer pressure of a hydrostatic column it is c in the interior
  and (1 + c)/2 in the top and bottom layers (interface value 1 at the
  column's ends); c = 1 (the hydrostatic case) gives 1 everywhere.
"""
import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S
from grist_inputs.mesh import build_mesh


def _layer_column(nC, L, ps, pi_top=225.0, b_int=None):
    b = S.sigma_uniform(L) if b_int is None else b_int
    pint = pi_top + b[None, :] * (ps[:, None] - pi_top)
    return pint, np.diff(pint, axis=1), 0.5 * (pint[:, 1:] + pint[:, :-1])


def _vadv_part(m, L, u, dpi, Mv):
    """The M-dependent part of the momentum tendency: the tendency with the
    vertical mass flux Mv minus the tendency with Mv = 0, every other input
    equal (no mass flux, uniform pressure and geopotential)."""
    M = O.Mesh(m)
    nC, nE = m["n_cells"], m["n_edges"]
    F = np.zeros((nE, L))
    p = np.full((nC, L), 5.0e4)
    alpha = np.full((nC, L), 0.8)
    phl = np.full((nC, L), 1.0e4)
    with_m = O.momentum_tend(M, L, u, dpi, F, Mv, p, alpha, phl, dpdpi=None)
    without = O.momentum_tend(M, L, u, dpi, F, np.zeros_like(Mv), p, alpha, phl, dpdpi=None)
    return with_m - without


@pytest.mark.parametrize("m_slope", [0.0, 3.0e-6])
def test_momentum_vertical_advection_closed_form(mesh_cache, m_slope):
    m = mesh_cache(2)
    nC, nE = m["n_cells"], m["n_edges"]
    L = 12
    ps = np.full(nC, 1.0e5)                       # flat: every layer has the same mass at every cell
    pint, dpi, pmid = _layer_column(nC, L, ps)
    b = 1.0e-3                                    # du/dpi [m s^-1 Pa^-1]
    u = np.repeat((b * (pmid[0] - 5.0e4))[None, :], nE, axis=0)
    # M linear in the interface pressure (uniform when m_slope = 0); the
    # top and bottom values are never read (closed column ends)
    M0 = 0.5
    Mv = np.repeat((M0 + m_slope * (pint[0] - 5.0e4))[None, :], nC, axis=0)
    Mv[:, 0] = 123.0
    Mv[:, L] = -321.0
    got = _vadv_part(m, L, u, dpi, Mv)
    m_mid = M0 + m_slope * (pmid[0] - 5.0e4)       # M at the layer centre (linear M)
    m_top_face = Mv[0, 1]                          # interior interface below the top layer
    m_bot_face = Mv[0, L - 1]                      # interior interface above the bottom layer
    expect = -b * m_mid.copy()
    expect[0] = -b * m_top_face / 2
    expect[L - 1] = -b * m_bot_face / 2
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(got - expect[None, :])) <= 1e-13 * scale, np.max(np.abs(got - expect[None, :])) / scale


def test_interface_vertical_advection_closed_form():
    rng = np.random.default_rng(21)
    nC, L = 7, 15
    # uneven layers: thicknesses drawn at random, so a wrong pair of layers
    # in the denominator cannot pass
    dpi = rng.uniform(200.0, 3000.0, (nC, L))
    pint = np.concatenate([np.full((nC, 1), 300.0), 300.0 + np.cumsum(dpi, axis=1)], axis=1)
    slope = -2.5                                   # dx/dpi
    x = 1.0e4 + slope * pint
    Mv = rng.uniform(-1.0, 1.0, (nC, L + 1))
    got = O.interface_vadv(L, Mv, dpi, x)
    expect = Mv * slope
    expect[:, 0] = 0.0
    expect[:, L] = 0.0
    assert np.max(np.abs(got - expect)) <= 1e-13 * np.max(np.abs(expect))


def _hadv_errors(level, L=3):
    m = build_mesh(level)
    u0 = 40.0
    ue = S.normal_wind_from_psi(m, S.solid_body_psi(m, u0))
    a = np.array([1.0, -0.5, 2.0])[:L]                       # layer wind factors
    u = ue[:, None] * a[None, :]
    c = np.array([1.0, 3.0, -2.0, 0.5])[:L + 1]              # interface field factors
    X, Y = m["cell_xyz"][:, 0], m["cell_xyz"][:, 1]
    x = X[:, None] * c[None, :]
    got = O.interface_hadv(O.Mesh(m), L, u, x)
    # interface wind: the mean of the two adjacent layers, the nearest layer
    # at the top and the bottom
    ui = np.concatenate([[a[0]], 0.5 * (a[:-1] + a[1:]), [a[-1]]])
    expect = (-(u0 / m["radius"]) * Y)[:, None] * (ui * c)[None, :]
    return O.error_norms(got, expect, m["cell_area"])


def test_interface_horizontal_advection_converges():
    errs = np.array([_hadv_errors(lev) for lev in (3, 4, 5, 6)])   # rows: l1, l2, linf
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order[:, 0] >= 1.5), (errs, order)
    assert np.all(order[:, 1] >= 0.95), (errs, order)
    assert errs[-1, 0] < 1e-3 and np.all(errs[:, 2] < 0.1), errs


@pytest.mark.parametrize("c", [1.0, 0.7])
def test_dpdpi_layer_closed_form(c):
    rng = np.random.default_rng(22)
    nC, L = 5, 20
    ps = rng.uniform(8.0e4, 1.03e5, nC)
    b = np.concatenate([[0.0], np.sort(rng.uniform(0.0, 1.0, L - 1)), [1.0]])   # uneven sigma levels
    pint, dpi, pmid = _layer_column(nC, L, ps, b_int=b)
    got = O.dpdpi_layer(c * pmid, dpi)
    expect = np.full((nC, L), c)
    expect[:, 0] = expect[:, L - 1] = 0.5 * (1.0 + c)
    assert np.max(np.abs(got - expect)) <= 1e-12, np.max(np.abs(got - expect))
