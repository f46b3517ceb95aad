"""GPU: dycore / tracer time splitting (Sec. 2.1: the tracers advance with
the mass flux accumulated and averaged over the dycore steps of one tracer
step; Sec. 2.3: that flux is computed in the dycore's precision and saved in
double).  n non-hydrostatic dycore steps add accum_scale = 1/n of their
final-stage flux to mass_flux_accum, the first of them also writes the layer
mass dpi^n; one tracer step of n dycore time steps then carries the tracers
with the mean flux.

Checked against the oracle (n oracle dycore steps summing the final-stage
flux, the mean taken here, one oracle tracer step of n dt) element by
element, and by properties of the hand-off: the tracer solver's own
continuity, summed over a column, lands on the dycore's column mass after
the n steps (ps - pi_top), and the global tracer mass is conserved.
Tolerances as in test_gpu_parity.py."""
import math

import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    return G


def _split_window(mesh, st, q0, L, dt, n, prec):
    """n NH dycore steps accumulating the mean flux, then one tracer step of
    n dt; returns host arrays in generator numbering."""
    import torch
    from gpu_cases import dycore_params, from_dev, to_dev
    fdt = torch.float64 if prec == "fp64" else torch.float32
    s = {"u": to_dev(mesh, st["u"], "edge", 0, fdt), "ps": to_dev(mesh, st["ps"]),
         "dpi_theta": to_dev(mesh, st["dpi_theta"]), "w": to_dev(mesh, st["w"]), "phi": to_dev(mesh, st["phi"]),
         "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
         "accum_weight": torch.zeros(1, dtype=torch.float64, device="cuda"),
         "p_nh": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"), "p_nh_valid": False,
         "accum_scale": 1.0 / n}
    dpi0 = torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda")
    P = dycore_params(mesh, st, L)
    for i in range(n):
        s["dpi_start"] = dpi0 if i == 0 else None
        mesh.dycore_step_nh(s, P, dt, prec=prec)
    q = to_dev(mesh, q0, "cell", 1, fdt)
    mesh.tracer_step([{"q": q, "dpi": dpi0, "mass_flux": s["mass_flux_accum"], "n_levels": L}], n * dt, prec=prec)
    torch.cuda.synchronize()
    out = {k: from_dev(mesh, s[k], kind) for k, kind in
           (("u", "edge"), ("ps", "cell"), ("dpi_theta", "cell"), ("w", "cell"), ("phi", "cell"),
            ("mass_flux_accum", "edge"))}
    out["dpi_start"] = from_dev(mesh, dpi0)
    out["q"] = from_dev(mesh, q, "cell", 1)
    out["weight"] = float(s["accum_weight"].item())
    out["status"] = mesh.last_status()
    return out


def _oracle_window(m, st, q0, L, dt, n):
    from gpu_cases import oracle_params
    M = O.Mesh(m)
    P = oracle_params(st, L)
    fa = np.zeros((m["n_edges"], L))
    ref = dict(st)
    for _ in range(n):
        r = O.dycore_step_nh(M, P, ref, dt, flux_accum=fa)
        ref.update({k: r[k] for k in ("ps", "u", "dpi_theta", "w", "phi")})
    pint = st["pi_top"] + st["b_int"][None, :] * (st["ps"][:, None] - st["pi_top"])
    dpi0 = np.diff(pint, axis=1)
    ref["mass_flux_mean"] = fa / n
    ref["dpi0"] = dpi0
    ref["q"] = O.tracer_step(M, q0, dpi0, fa / n, n * dt)
    return ref


@pytest.mark.parametrize("prec", ["fp64", "mix"])
def test_split_three_dycore_steps_per_tracer_step(G, mesh_cache, prec):
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    L, dt, n = 30, 60.0, 3
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    q0 = S.tracer_mixture(m, 3, L, np.random.default_rng(5))
    got = _split_window(mesh, st, q0, L, dt, n, prec)
    ref = _oracle_window(m, st, q0, L, dt, n)
    assert got["status"] == 0
    assert abs(got["weight"] - 1.0) <= 1e-15
    assert O.max_rel_diff(got["dpi_start"], ref["dpi0"]) <= 1e-13
    if prec == "fp64":
        for k in ("u", "ps", "dpi_theta", "phi", "mass_flux_accum", "q"):
            r = ref["mass_flux_mean"] if k == "mass_flux_accum" else ref[k]
            assert O.max_rel_diff(got[k], r) <= FP64_TOL, k
        assert O.max_rel_diff(got["w"], ref["w"]) <= 1e-9
    else:
        assert O.max_rel_diff(got["u"], ref["u"]) <= 2e-5
        assert O.max_rel_diff(got["ps"], ref["ps"]) <= 1e-7
        assert O.max_rel_diff(got["mass_flux_accum"], ref["mass_flux_mean"]) <= 2e-5
        assert O.max_rel_diff(got["q"], ref["q"]) <= 2e-5
        for k in ("dpi_theta", "phi"):
            assert O.max_rel_diff(got[k], ref[k]) <= 5e-7, k
    # the tracer solver's continuity over the window, summed over each
    # column, equals the dycore's column mass after the n steps
    M = O.Mesh(m)
    dpi_tr = got["dpi_start"] - n * dt * O.divergence(M, got["mass_flux_accum"])
    col_tr = dpi_tr.sum(axis=1)
    col_dy = got["ps"] - st["pi_top"]
    assert np.max(np.abs(col_tr - col_dy) / col_dy) <= (1e-12 if prec == "fp64" else 1e-9)
    # global tracer mass over the tracer step (FP64 storage only)
    if prec == "fp64":
        A = m["cell_area"][:, None]
        for t in range(q0.shape[0]):
            before = math.fsum((A * got["dpi_start"] * q0[t]).ravel())
            after = math.fsum((A * dpi_tr * got["q"][t]).ravel())
            assert abs(after - before) / abs(before) <= 1e-13
    mesh.close()


def test_accum_scale_default_and_validation(G, mesh_cache):
    """accum_scale 0 (a zero-initialised C struct) accumulates with weight
    1; a negative or non-finite scale is refused before any launch."""
    import torch
    from gpu_cases import dycore_params, to_dev
    m = mesh_cache(3)
    mesh = G.Mesh(m)
    L = 10
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)

    def state(scale):
        return {"u": to_dev(mesh, st["u"], "edge", 0, torch.float64), "ps": to_dev(mesh, st["ps"]),
                "dpi_theta": to_dev(mesh, st["dpi_theta"]), "w": to_dev(mesh, st["w"]),
                "phi": to_dev(mesh, st["phi"]),
                "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
                "accum_weight": torch.zeros(1, dtype=torch.float64, device="cuda"), "accum_scale": scale}
    P = dycore_params(mesh, st, L)
    a, b = state(0.0), state(1.0)
    mesh.dycore_step_nh(a, P, 60.0)
    mesh.dycore_step_nh(b, P, 60.0)
    torch.cuda.synchronize()
    assert float(a["accum_weight"].item()) == 1.0
    assert torch.equal(a["mass_flux_accum"], b["mass_flux_accum"])
    for bad in (-0.5, float("nan"), float("inf")):
        with pytest.raises(G.GristError):
            mesh.dycore_step_nh(state(bad), P, 60.0)
    mesh.close()
