"""GPU: checkpoint / resume and fault flags of the coupled step.

* The prognostic state is caller-owned and the library keeps no hidden state
  between steps: 4 coupled NH steps (dycore accumulating the horizontal and
  vertical mass fluxes, then the tracers' horizontal and vertical transport)
  in one run equal, bit for bit, 2 steps + a copy of the whole state to host
  memory + a new mesh handle (fresh scratch) + the copy back + 2 more steps,
  in FP64 and in the mixed policy.  The carried NH pressure is part of the
  saved state.
* A non-finite wind raises GRIST_FLAG_NONFINITE in the dycore step (the
  failure is made on the host: no GPU fault is involved).
"""
import numpy as np
import pytest

from grist_inputs import states as S

pytestmark = pytest.mark.gpu

L, DT = 20, 60.0
KEYS = ("u", "ps", "dpi_theta", "w", "phi", "q", "p_nh")


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    return G


def _state(mesh, st, q0, prec):
    import torch
    from gpu_cases import to_dev
    fdt = torch.float64 if prec == "fp64" else torch.float32
    return {"u": to_dev(mesh, st["u"], "edge", 0, fdt), "ps": to_dev(mesh, st["ps"]),
            "dpi_theta": to_dev(mesh, st["dpi_theta"]), "w": to_dev(mesh, st["w"]), "phi": to_dev(mesh, st["phi"]),
            "q": to_dev(mesh, q0, "cell", 1, fdt),
            "p_nh": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"), "p_nh_valid": False,
            "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
            "vmass_flux_accum": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
            "dpi_start": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda")}


def _steps(mesh, s, P, prec, n):
    for _ in range(n):
        s["mass_flux_accum"].zero_()
        s["vmass_flux_accum"].zero_()
        mesh.dycore_step_nh(s, P, DT, prec=prec)
        mesh.tracer_step([{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                           "vmass_flux": s["vmass_flux_accum"], "n_levels": L}], DT, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mix"])
def test_resume_is_bit_exact(G, mesh_cache, prec):
    import torch
    from gpu_cases import dycore_params
    m = mesh_cache(4)
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    q0 = S.tracer_mixture(m, 3, L, np.random.default_rng(21))
    # straight run
    mesh = G.Mesh(m)
    P = dycore_params(mesh, st, L)
    s = _state(mesh, st, q0, prec)
    _steps(mesh, s, P, prec, 4)
    torch.cuda.synchronize()
    straight = {k: s[k].cpu().numpy() for k in KEYS}
    assert mesh.last_status() == 0
    mesh.close()
    # 2 steps, checkpoint to the host, new handle, restore, 2 steps
    mesh = G.Mesh(m)
    P = dycore_params(mesh, st, L)
    s = _state(mesh, st, q0, prec)
    _steps(mesh, s, P, prec, 2)
    torch.cuda.synchronize()
    ckpt = {k: s[k].cpu().numpy().copy() for k in KEYS}
    ckpt_valid = s["p_nh_valid"]
    mesh.close()
    del s
    mesh = G.Mesh(m)
    P = dycore_params(mesh, st, L)
    s = _state(mesh, st, q0, prec)
    for k in KEYS:
        s[k].copy_(torch.from_numpy(ckpt[k]))
    s["p_nh_valid"] = ckpt_valid
    _steps(mesh, s, P, prec, 2)
    torch.cuda.synchronize()
    for k in KEYS:
        assert np.array_equal(s[k].cpu().numpy(), straight[k]), k
    assert mesh.last_status() == 0
    mesh.close()


def test_nonfinite_wind_is_flagged(G, mesh_cache):
    import torch
    from gpu_cases import dycore_params
    m = mesh_cache(3)
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    mesh = G.Mesh(m)
    P = dycore_params(mesh, st, L)
    s = _state(mesh, st, np.zeros((1, m["n_cells"], L)), "fp64")
    mesh.last_status()
    s["u"][7, 3] = float("nan")
    mesh.dycore_step_nh(s, P, DT)
    torch.cuda.synchronize()
    assert mesh.last_status() & G.GRIST_FLAG_NONFINITE
    # the handle stays usable: a clean state steps without flags
    s = _state(mesh, st, np.zeros((1, m["n_cells"], L)), "fp64")
    mesh.dycore_step_nh(s, P, DT)
    torch.cuda.synchronize()
    assert mesh.last_status() == 0
    mesh.close()
