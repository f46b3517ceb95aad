"""GPU: vertical tracer transport (the delta(M q) term of Eq. 10,
adaptively implicit upwind; Sec. 2.1) against the oracle, alone and after
the horizontal step, in FP64 (1e-12) and the mixed policy (2e-5); and
coupled to the dycore's accumulated horizontal and vertical fluxes: a
constant tracer stays constant and the global tracer mass is conserved with
the dycore's own final layer mass (the tracer continuity, horizontal then
vertical, lands on it)."""
import math

import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    return G


def _column_flux(rng, nC, L, dt, dpi_min, courant):
    """Tapered vertical mass flux of either sign with Courant numbers up to
    `courant` (capped so that no layer loses more than ~half its mass:
    dt |M_{k+1} - M_k| <= dt amp pi / L <= 0.4 dpi_min), and a small
    convergent/divergent part."""
    prof = np.sin(np.pi * np.arange(L + 1) / L)
    amp = min(courant * dpi_min / dt, 0.4 * dpi_min * L / (np.pi * dt))
    Mv = rng.uniform(-amp, amp, (nC, 1)) * prof[None, :]
    Mv[:, 1:L] += rng.uniform(-0.02 * amp, 0.02 * amp, (nC, L - 1))
    Mv[:, 0] = Mv[:, L] = 0.0
    return Mv


def _member(mesh, q, dpi, F, Mv, prec, ld, ldi):
    import torch
    from gpu_cases import to_dev
    dq = torch.float64 if prec == "fp64" else torch.float32
    return {"q": to_dev(mesh, q, "cell", 1, dq, ld), "dpi": to_dev(mesh, dpi, "cell", 0, torch.float64, ld),
            "mass_flux": to_dev(mesh, F, "edge", 0, torch.float64, ld),
            "vmass_flux": to_dev(mesh, Mv, "cell", 0, torch.float64, ldi), "n_levels": q.shape[2]}


@pytest.mark.parametrize("prec", ["fp64", "mix"])
@pytest.mark.parametrize("cmax,courant", [(0.0, 6.0), (0.5, 6.0), (1.0, 6.0), (1e9, 0.9)])
def test_vertical_step_against_oracle(G, mesh_cache, prec, cmax, courant):
    """cmax 0: fully implicit; 0.5, 1: split; 1e9 (explicit only) with
    Courant numbers below 1, its stability limit."""
    import torch
    from gpu_cases import from_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(11)
    dt = 400.0
    cases = [(3, 30, 32, 33), (2, 17, 17, 20)]          # (T, L, ld, ld_int): ragged chunks, padding
    members, refs = [], []
    for T, L, ld, ldi in cases:
        dpi = rng.uniform(600, 1200, (m["n_cells"], L))
        Mv = _column_flux(rng, m["n_cells"], L, dt, 600.0, courant)
        q = rng.uniform(0.1, 1.0, (T, m["n_cells"], L))
        F = np.zeros((m["n_edges"], L))                  # horizontal no-op
        members.append(_member(mesh, q, dpi, F, Mv, prec, ld, ldi))
        refs.append(O.tracer_vertical_step(q, dpi, Mv, dt, cmax))
    mesh.tracer_step(members, dt, prec=prec, vertical_courant_max=cmax)
    torch.cuda.synchronize()
    assert mesh.last_status() == 0
    tol = 1e-12 if prec == "fp64" else 2e-5
    for mb, ref in zip(members, refs):
        got = from_dev(mesh, mb["q"], "cell", 1, n=mb["n_levels"])
        assert O.max_rel_diff(got, ref) <= tol
    mesh.close()


@pytest.mark.parametrize("prec", ["fp64", "mix"])
def test_horizontal_then_vertical_against_oracle(G, mesh_cache, prec):
    import torch
    from gpu_cases import from_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(12)
    L, dt = 24, 300.0
    c = S.tracer_rotation_case(m, n_levels=L)
    dpi = c["dpi"]
    F = c["mass_flux"]
    Mv = _column_flux(rng, m["n_cells"], L, dt, float(dpi.min()), 3.0)
    q = S.tracer_mixture(m, 3, L, rng)
    mb = _member(mesh, q, dpi, F, Mv, prec, L, L + 1)
    mesh.tracer_step([mb], dt, prec=prec, vertical_courant_max=0.8)
    torch.cuda.synchronize()
    M = O.Mesh(m)
    qh = O.tracer_step(M, q, dpi, F, dt)
    ref = O.tracer_vertical_step(qh, dpi - dt * O.divergence(M, F), Mv, dt, 0.8)
    got = from_dev(mesh, mb["q"], "cell", 1)
    assert O.max_rel_diff(got, ref) <= (1e-12 if prec == "fp64" else 2e-5)
    mesh.close()


def test_coupled_with_dycore_fluxes(G, mesh_cache):
    """Three NH dycore steps accumulate the mean horizontal and vertical
    mass fluxes; one tracer step of 3 dt (horizontal + vertical) keeps a
    constant tracer constant and conserves tracer mass with the dycore's
    final layer mass."""
    import torch
    from gpu_cases import dycore_params, from_dev, to_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    L, dt, n = 30, 60.0, 3
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    s = {"u": to_dev(mesh, st["u"], "edge", 0, torch.float64), "ps": to_dev(mesh, st["ps"]),
         "dpi_theta": to_dev(mesh, st["dpi_theta"]), "w": to_dev(mesh, st["w"]), "phi": to_dev(mesh, st["phi"]),
         "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
         "vmass_flux_accum": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
         "accum_scale": 1.0 / n}
    dpi0 = torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda")
    P = dycore_params(mesh, st, L)
    for i in range(n):
        s["dpi_start"] = dpi0 if i == 0 else None
        mesh.dycore_step_nh(s, P, dt)
    q0 = S.tracer_mixture(m, 2, L, np.random.default_rng(9))
    q0 = np.concatenate([q0, np.full((1, m["n_cells"], L), 1.7)])
    q = to_dev(mesh, q0, "cell", 1, torch.float64)
    mesh.tracer_step([{"q": q, "dpi": dpi0, "mass_flux": s["mass_flux_accum"], "vmass_flux": s["vmass_flux_accum"],
                       "n_levels": L}], n * dt, prec="fp64")
    torch.cuda.synchronize()
    assert mesh.last_status() == 0
    got = from_dev(mesh, q, "cell", 1)
    assert np.max(np.abs(got[2] - 1.7)) <= 1e-12
    ps = from_dev(mesh, s["ps"])
    dpi_end = np.diff(st["pi_top"] + st["b_int"][None, :] * (ps[:, None] - st["pi_top"]), axis=1)
    dpi_start = from_dev(mesh, dpi0)
    A = m["cell_area"][:, None]
    for t in range(2):
        before = math.fsum((A * dpi_start * q0[t]).ravel())
        after = math.fsum((A * dpi_end * got[t]).ravel())
        assert abs(after - before) / abs(before) <= 1e-12
    mesh.close()


def test_vertical_validation(G, mesh_cache):
    import torch
    from gpu_cases import to_dev
    m = mesh_cache(3)
    mesh = G.Mesh(m)
    L = 10
    q = to_dev(mesh, np.ones((1, m["n_cells"], L)), "cell", 1, torch.float64)
    dpi = to_dev(mesh, np.full((m["n_cells"], L), 1000.0))
    F = torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda")
    short = torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda")    # needs L + 1 interfaces
    with pytest.raises(G.GristError):
        mesh.tracer_step([{"q": q, "dpi": dpi, "mass_flux": F, "vmass_flux": short, "n_levels": L}], 60.0)
    with pytest.raises(G.GristError):
        mesh.tracer_step([{"q": q, "dpi": dpi, "mass_flux": F,
                           "vmass_flux": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
                           "n_levels": L}], 60.0, vertical_courant_max=float("nan"))
    with pytest.raises(G.GristError):
        mesh.tracer_step([{"q": q, "dpi": dpi, "mass_flux": F,
                           "vmass_flux": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
                           "n_levels": L}], 60.0, vertical_courant_max=-1.0)
    mesh.close()
