"""Pins of the oracle's dycore (Eqs. 3-9, Sec. 2.1) - CPU only.

I6   dry-mass conservation (sum A (ps - pi_t)) to FP64 round-off, HDC and NDC
I12  resting, horizontally uniform, discretely hydrostatic atmosphere stays
     at rest (HDC and NDC)
I13  isothermal column: the hydrostatic geopotential integral converges at
     second order to phi_s + Rd T ln(ps / pi)
I14  Thomas solver vs numpy.linalg.solve; the HEVI column solve satisfies
     the w equation with the full equation of state to linearisation error
     Equation of state (Eq. 9) inverts the hydrostatic thickness exactly
     Theta transport is consistent with continuity (uniform theta stays
     uniform)
     Balanced solid-body flow: the net momentum tendency is a small residual
     of its pressure-gradient part and shrinks with resolution (pins the
     signs of the PV, kinetic-energy and pressure-gradient terms)
I17  hydrostatic limit: one NDC step stays close to the HDC step
"""
import math

import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S
from grist_inputs.mesh import lonlat


def _params(st, L, beta=0.55):
    return O.Params(L, st["b_int"], st["pi_top"], st["phi_s"], beta=beta)


def _solid_body_state(m, L=20, u0=20.0, T0=300.0):
    """Isothermal zonal solid-body flow in gradient-wind balance on a flat
    surface: ps = p0 exp(-(a Omega u0 + u0^2/2) sin^2(lat) / (Rd T0))."""
    R, Om = m["radius"], m["omega"]
    B, pit = S.sigma_uniform(L), 225.0
    _, latc = lonlat(m["cell_xyz"])
    ps = S.P0 * np.exp(-(R * Om * u0 + u0 * u0 / 2) * np.sin(latc) ** 2 / (S.RD * T0))
    pint = pit + B[None, :] * (ps[:, None] - pit)
    dpi = np.diff(pint, axis=1)
    pm = 0.5 * (pint[:, 1:] + pint[:, :-1])
    th = T0 * (S.P0 / pm) ** S.KAPPA
    u = S.normal_wind_from_psi(m, S.solid_body_psi(m, u0))
    return {"ps": ps, "u": np.repeat(u[:, None], L, 1), "dpi_theta": dpi * th, "b_int": B,
            "pi_top": pit, "phi_s": np.zeros(m["n_cells"])}


def test_dry_mass_conservation_hydro(mesh_cache):
    m = mesh_cache(4)
    M = O.Mesh(m)
    st = S.dycore_jet_case(m, 30)
    P = _params(st, 30)
    m0 = O.dry_mass(M, st["ps"], st["pi_top"])[0]
    s = st
    for _ in range(5):
        s = O.dycore_step_hydro(M, P, s, 300.0)
    m1 = O.dry_mass(M, s["ps"], st["pi_top"])[0]
    assert abs(m1 - m0) / m0 < 1e-13
    assert np.max(np.abs(s["ps"] - st["ps"])) > 1e-3          # mass did move


def test_dry_mass_conservation_nh(mesh_cache):
    m = mesh_cache(3)
    M = O.Mesh(m)
    st = S.dycore_jet_case(m, 20, nonhydrostatic=True, bubble=True)
    P = _params(st, 20)
    m0 = O.dry_mass(M, st["ps"], st["pi_top"])[0]
    s = st
    for _ in range(4):
        s = O.dycore_step_nh(M, P, s, 300.0)
    assert abs(O.dry_mass(M, s["ps"], st["pi_top"])[0] - m0) / m0 < 1e-13


@pytest.mark.parametrize("nh", [False, True])
def test_resting_atmosphere(mesh_cache, nh):
    m = mesh_cache(3)
    M = O.Mesh(m)
    L = 30
    st = S.resting_case(m, L, nonhydrostatic=nh)
    P = _params(st, L)
    s = st
    for _ in range(3):
        s = O.dycore_step_nh(M, P, s, 120.0) if nh else O.dycore_step_hydro(M, P, s, 300.0)
    assert np.max(np.abs(s["u"])) < 1e-12
    assert np.max(np.abs(s["ps"] - st["ps"])) < 1e-9
    assert np.max(np.abs(s["dpi_theta"] - st["dpi_theta"])) < 1e-9 * np.max(st["dpi_theta"])
    if nh:
        assert np.max(np.abs(s["w"])) < 1e-10
        assert np.max(np.abs(s["phi"] - st["phi"])) < 1e-9 * np.max(st["phi"])


def test_isothermal_geopotential_second_order():
    errs = []
    T0 = 250.0
    for L in (15, 30, 60):
        B = S.sigma_uniform(L)
        ps = np.array([1.0e5, 0.9e5])
        pit = 2.0e4          # keeps dp / p small in every layer (asymptotic regime)
        P = O.Params(L, B, pit, np.zeros(2))
        pint = pit + B[None, :] * (ps[:, None] - pit)
        dpi = np.diff(pint, axis=1)
        pm = 0.5 * (pint[:, 1:] + pint[:, :-1])
        th = T0 * (1.0e5 / pm) ** (287.04 / 1004.64)
        d = O.hydro_diag(P, ps, dpi * th)
        exact = 287.04 * T0 * np.log(ps[:, None] / pint)
        errs.append(np.max(np.abs(d["phi_int"] - exact)) / np.max(exact))
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert np.all(order > 1.8), (errs, order)


def test_eos_inverts_hydrostatic_thickness(mesh_cache):
    """Eq. 9 with the phi of a discretely hydrostatic column returns the
    mid-layer pressure (ideal gas + Poisson relation, gamma = cp/cv)."""
    m = mesh_cache(2)
    st = S.dycore_jet_case(m, 40, nonhydrostatic=True, bubble=True)
    P = _params(st, 40)
    p = O.eos(P, st["dpi_theta"], st["phi"])
    assert np.max(np.abs(p / st["pmid"] - 1)) < 1e-12
    d = O.hydro_diag(P, st["ps"], st["dpi_theta"])
    assert np.max(np.abs(d["phi_int"] - st["phi"])) < 1e-9 * np.max(st["phi"])


def test_thomas_vs_dense_solve():
    rng = np.random.default_rng(12)
    for n in (1, 2, 5, 59, 200):
        a = rng.uniform(-1, 1, n); c = rng.uniform(-1, 1, n)
        b = np.abs(a) + np.abs(c) + rng.uniform(0.5, 2, n)
        a[0] = 0.0; c[-1] = 0.0
        d = rng.standard_normal(n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        ref = np.linalg.solve(A, d)
        assert np.max(np.abs(O.thomas(a, b, c, d) - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_vertical_solve_satisfies_w_equation(mesh_cache):
    """After the HEVI column solve, the residual of the w equation
    w - w** - beta dt g ((p_j - p_{j-1}) / dpi_j - 1) with p from the FULL
    equation of state is the EOS linearisation error alone: it is second
    order in the departure from balance (halving the departure divides it
    by ~4) while the implicit increment itself is first order."""
    m = mesh_cache(2)
    L = 30
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    P = _params(st, L, beta=0.55)
    rng = np.random.default_rng(13)
    nC = m["n_cells"]
    dw = np.zeros((nC, L + 1)); dw[:, 1:L] = rng.standard_normal((nC, L - 1)) * 0.5
    dphi = np.concatenate([rng.standard_normal((nC, L)) * 2.0, np.zeros((nC, 1))], 1)
    dts = 60.0
    bg = 0.55 * dts * 9.80616
    dpint = 0.5 * (st["dpi"][:, :-1] + st["dpi"][:, 1:])
    res, inc = [], []
    for amp in (1.0, 0.5):
        w_star, phi_star = amp * dw, st["phi"] + amp * dphi
        w, phi, p = O.vertical_solve(P, w_star, phi_star, st["dpi_theta"], st["dpi"], dts)
        r = w[:, 1:L] - w_star[:, 1:L] - bg * ((p[:, 1:] - p[:, :-1]) / dpint - 1.0)
        res.append(np.max(np.abs(r)))
        inc.append(np.max(np.abs(w[:, 1:L] - w_star[:, 1:L])))
        assert np.all(w[:, 0] == 0) and np.all(w[:, L] == 0)
        assert np.allclose(phi[:, :L], phi_star[:, :L] + bg * w[:, :L], rtol=0, atol=1e-9)
        assert np.all(phi[:, L] == st["phi_s"])
        assert np.allclose(p, O.eos(P, st["dpi_theta"], phi), rtol=1e-14, atol=0)
    assert res[0] / res[1] > 3.5, res
    assert 1.8 < inc[0] / inc[1] < 2.2, inc
    assert res[0] < 0.05 * inc[0]


@pytest.mark.parametrize("nh", [False, True])
def test_uniform_theta_stays_uniform(mesh_cache, nh):
    m = mesh_cache(3)
    M = O.Mesh(m)
    L = 12
    st = S.dycore_jet_case(m, L, nonhydrostatic=nh)
    th0 = 300.0
    st = dict(st)
    st["dpi_theta"] = st["dpi"] * th0
    if nh:
        P = _params(st, L)
        alpha = 287.04 * th0 * (st["pmid"] / 1e5) ** (287.04 / 1004.64) / st["pmid"]
        phi = np.zeros((m["n_cells"], L + 1))
        for k in range(L - 1, -1, -1):
            phi[:, k] = phi[:, k + 1] + alpha[:, k] * st["dpi"][:, k]
        st["phi"] = phi
        s = O.dycore_step_nh(M, P, st, 200.0)
    else:
        P = _params(st, L)
        s = O.dycore_step_hydro(M, P, st, 300.0)
    pint = st["pi_top"] + st["b_int"][None, :] * (s["ps"][:, None] - st["pi_top"])
    th = s["dpi_theta"] / np.diff(pint, axis=1)
    assert np.max(np.abs(th - th0)) < 1e-10 * th0


def _explicit_u_tend(m, st, L):
    M = O.Mesh(m)
    P = _params(st, L)
    ms = O.mass(M, P, st["ps"], st["u"])
    d = O.hydro_diag(P, st["ps"], st["dpi_theta"])
    full = O.momentum_tend(M, L, st["u"], ms["dpi"], ms["F"], ms["M"], d["p"], d["alpha"], d["phi_layer"])
    pgf = O.momentum_tend(M, L, 0 * st["u"], ms["dpi"], 0 * ms["F"], ms["M"], d["p"], d["alpha"], d["phi_layer"])
    return full, pgf


def test_balanced_solid_body_residual(mesh_cache):
    ratios = []
    for lev in (3, 4, 5):
        m = mesh_cache(lev)
        full, pgf = _explicit_u_tend(m, _solid_body_state(m), 20)
        ratios.append(np.sqrt(np.mean(full ** 2)) / np.sqrt(np.mean(pgf ** 2)))
    assert ratios[0] < 0.1 and ratios[1] < ratios[0] and ratios[2] < ratios[1], ratios


def test_hydrostatic_limit(mesh_cache):
    m = mesh_cache(4)
    M = O.Mesh(m)
    st = S.dycore_jet_case(m, 40, nonhydrostatic=True)
    P = _params(st, 40)
    a = O.dycore_step_hydro(M, P, st, 60.0)
    b = O.dycore_step_nh(M, P, st, 60.0)
    du = np.max(np.abs(a["u"] - st["u"]))
    assert np.max(np.abs(a["u"] - b["u"])) < 0.01 * du
    assert np.max(np.abs(a["ps"] - b["ps"])) < 0.01 * np.max(np.abs(a["ps"] - st["ps"]))
    assert np.max(np.abs(b["w"])) < 0.05
