"""Pins of the oracle's theta-transport tendency (Eq. 4) and cell kinetic
energy (Eq. 5) - CPU only.

theta tendency, d(dpi theta)/dt = -div(F theta_e) - delta(M theta):
- a constant theta is carried with the mass: the tendency equals theta0
  times the layer-mass tendency -div F - (M_{k+1/2} - M_{k-1/2}) of the
  continuity equation (Eq. 3), so theta = (dpi theta)/dpi stays theta0 (the
  third-order edge value of a constant is the constant); a dropped theta
  factor or a flipped sign of either part fails;
- with no horizontal flux the vertical fluxes telescope: every column's
  sum of the tendency is 0 (a shifted interface index fails);
- with no vertical flux the horizontal fluxes cancel pairwise: the
  area-weighted global sum is 0 on every level.

cell kinetic energy K_i = (1/A_i) sum_e (dc dv / 4) u_e^2: for the normal
components of solid-body rotation V = k x r on the unit sphere it converges
to |V|^2 / 2 = (1 - z^2)/2 at the cell centres - area-weighted l1 at about
order 1.7 and l2 at first order over levels 3 -> 6; the maximum error stays
near 6 % along the icosahedron's edges, where the bisection mesh is not
smooth (the interface-advection pin sees the same).  A wrong weight
(dc dv / 2, dc^2, a missing area) is off by O(1).
"""
import numpy as np
import pytest

import oracle as O


def _random_fields(m, L, rng):
    nC, nE = m["n_cells"], m["n_edges"]
    dpi = 1000.0 + rng.uniform(0.0, 200.0, (nC, L))
    F = rng.standard_normal((nE, L)) * 1.0e3
    Mv = rng.standard_normal((nC, L + 1)) * 10.0
    Mv[:, 0] = 0.0
    Mv[:, L] = 0.0
    return dpi, F, Mv


@pytest.mark.parametrize("theta0", [300.0, -2.5])
def test_theta_tendency_of_a_constant_is_theta0_times_the_mass_tendency(mesh_cache, theta0):
    m = mesh_cache(3)
    L = 7
    dpi, F, Mv = _random_fields(m, L, np.random.default_rng(11))
    M = O.Mesh(m)
    got = O.theta_tend(M, L, theta0 * dpi, dpi, F, Mv)
    mass_tend = -O.divergence(M, F) - (Mv[:, 1:] - Mv[:, :-1])
    scale = np.max(np.abs(theta0 * mass_tend))
    assert np.max(np.abs(got - theta0 * mass_tend)) <= 1e-13 * scale


def test_theta_vertical_fluxes_telescope_in_each_column(mesh_cache):
    m = mesh_cache(3)
    L = 9
    rng = np.random.default_rng(12)
    dpi, _, Mv = _random_fields(m, L, rng)
    theta = 250.0 + rng.uniform(0.0, 100.0, (m["n_cells"], L))
    got = O.theta_tend(O.Mesh(m), L, theta * dpi, dpi, np.zeros((m["n_edges"], L)), Mv)
    assert np.max(np.abs(got)) > 1.0                       # the fluxes are not trivial
    col = got.sum(axis=1)
    assert np.max(np.abs(col)) <= 1e-12 * np.max(np.abs(got))


def test_theta_horizontal_fluxes_cancel_globally(mesh_cache):
    m = mesh_cache(3)
    L = 4
    rng = np.random.default_rng(13)
    dpi, F, _ = _random_fields(m, L, rng)
    theta = 250.0 + rng.uniform(0.0, 100.0, (m["n_cells"], L))
    got = O.theta_tend(O.Mesh(m), L, theta * dpi, dpi, F, np.zeros((m["n_cells"], L + 1)))
    a = m["cell_area"][:, None]
    tot = (a * got).sum(axis=0)
    assert np.max(np.abs(got)) > 1.0
    assert np.max(np.abs(tot)) <= 1e-12 * np.sum(a * np.abs(got), axis=0).max()


def _ke_errors(level):
    from grist_inputs.mesh import build_mesh
    m = build_mesh(level)
    xe = m["edge_xyz"] / np.linalg.norm(m["edge_xyz"], axis=1, keepdims=True)
    V = np.stack([-xe[:, 1], xe[:, 0], np.zeros(len(xe))], 1)
    u = np.sum(V * m["edge_normal_xyz"], axis=1)[:, None]
    K = O.kinetic_energy(O.Mesh(m), u)[:, 0]
    xc = m["cell_xyz"] / np.linalg.norm(m["cell_xyz"], axis=1, keepdims=True)
    ex = 0.5 * (1.0 - xc[:, 2] ** 2)
    a = m["cell_area"]
    err = K - ex
    return (np.sum(a * np.abs(err)) / np.sum(a * np.abs(ex)), np.sqrt(np.sum(a * err ** 2) / np.sum(a * ex ** 2)),
            np.max(np.abs(err)) / np.max(np.abs(ex)))


def test_kinetic_energy_converges_to_half_speed_squared():
    errs = np.array([_ke_errors(lev) for lev in (3, 4, 5, 6)])   # rows: levels; cols: l1, l2, linf
    l1_order = np.log2(errs[:-1, 0] / errs[1:, 0])
    l2_order = np.log2(errs[:-1, 1] / errs[1:, 1])
    assert np.all(l1_order >= 1.4), l1_order
    assert np.all(l2_order >= 0.9), l2_order
    assert errs[-1, 0] < 3e-4 and errs[-1, 1] < 2e-3
    assert np.all(errs[:, 2] < 0.1), errs[:, 2]
