"""GPU checks at the full sizes of the benchmark configurations.

* C2 hydrostatic jet, level-6 mesh (40,962 cells), 30 levels, dt 300 s and
  C3 non-hydrostatic jet + bubble, level-8 mesh (655,362 cells), 60 levels,
  dt 60 s: one step element-wise against a full oracle step.
* C4 uneven 16-member tracer ensemble on the level-7 mesh in one call (the
  benchmark's launch path, autotuned): sampled members element-wise against
  the oracle.
* C5 non-hydrostatic dycore + 4 tracers on the level-9 mesh (2,621,442
  cells), 60 levels, dt 30 s, in the benchmark's coupled step (horizontal
  and vertical tracer transport with the dycore's fluxes): properties
  that hold at any size (dry- and tracer-mass conservation, free stream of
  a constant tracer, mixed vs FP64 agreement), the oracle being too slow for
  an element-wise comparison there.
Tolerances as in test_gpu_parity.py.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S
from grist_inputs.mesh import get_mesh

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


def _rel(a, b):
    return O.max_rel_diff(a, b)


def test_c2_hydrostatic_full_size(G):
    from gpu_cases import oracle_params, run_dycore
    m = get_mesh(6)
    mesh = G.Mesh(m)
    L = 30
    st = S.dycore_jet_case(m, L)
    ref = O.dycore_step_hydro(O.Mesh(m), oracle_params(st, L), st, 300.0)
    got = run_dycore(mesh, st, L, 300.0, nh=False)
    for k in ("u", "ps", "dpi_theta"):
        assert _rel(got[k], ref[k]) <= FP64_TOL, k
    mix = run_dycore(mesh, st, L, 300.0, nh=False, prec="mix")
    assert _rel(mix["u"], ref["u"]) <= 2e-5
    assert _rel(mix["ps"], ref["ps"]) <= 1e-7
    mesh.close()


def test_c3_nonhydrostatic_full_size(G):
    from gpu_cases import oracle_params, run_dycore
    m = get_mesh(8)
    mesh = G.Mesh(m)
    L = 60
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    ref = O.dycore_step_nh(O.Mesh(m), oracle_params(st, L), st, 60.0)
    got = run_dycore(mesh, st, L, 60.0, nh=True)
    for k in ("u", "ps", "dpi_theta", "phi"):
        assert _rel(got[k], ref[k]) <= FP64_TOL, k
    from test_gpu_parity import check_w_fp64
    check_w_fp64(got["w"], ref["w"], 60.0)
    mix = run_dycore(mesh, st, L, 60.0, nh=True, prec="mix")
    assert _rel(mix["u"], ref["u"]) <= 2e-5
    assert _rel(mix["ps"], ref["ps"]) <= 1e-7
    for k in ("dpi_theta", "phi"):
        assert _rel(mix[k], ref[k]) <= 5e-7, k
    from test_gpu_parity import check_w_mixed
    check_w_mixed(mix["w"], ref["w"], 60.0)
    mesh.close()


def test_nh_carried_pressure_two_steps(G, mesh_cache):
    """Two NH steps carrying the pressure in the state (the second step skips
    the equation-of-state pass) match two oracle steps."""
    import torch
    from gpu_cases import dycore_params, from_dev, oracle_params, to_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    L = 40
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    M = O.Mesh(m)
    P = oracle_params(st, L)
    ref = dict(st)
    for _ in range(2):
        r = O.dycore_step_nh(M, P, ref, 90.0)
        ref.update({k: r[k] for k in ("ps", "u", "dpi_theta", "w", "phi")})
    s = {"u": to_dev(mesh, st["u"], "edge", 0, torch.float64), "ps": to_dev(mesh, st["ps"]),
         "dpi_theta": to_dev(mesh, st["dpi_theta"]), "w": to_dev(mesh, st["w"]), "phi": to_dev(mesh, st["phi"]),
         "p_nh": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"), "p_nh_valid": False}
    Pd = dycore_params(mesh, st, L)
    for _ in range(2):
        mesh.dycore_step_nh(s, Pd, 90.0)
        assert s["p_nh_valid"]
    for k, kind in (("u", "edge"), ("ps", "cell"), ("dpi_theta", "cell"), ("phi", "cell")):
        assert _rel(from_dev(mesh, s[k], kind), ref[k]) <= FP64_TOL, k
    p_ref = O.eos(P, ref["dpi_theta"], ref["phi"])
    assert _rel(from_dev(mesh, s["p_nh"]), p_ref) <= FP64_TOL
    mesh.close()


def test_c4_batched_ensemble_full_size(G):
    import torch
    from gpu_cases import from_dev
    m = get_mesh(7)
    mesh = G.Mesh(m)
    members, dt = S.ensemble_members(m, n_members=16)
    dev = [{"q": torch.from_numpy(mesh.to_internal(mb["q"], "cell", 1)).to("cuda", torch.float32),
            "dpi": torch.from_numpy(mesh.to_internal(mb["dpi"])).cuda(),
            "mass_flux": torch.from_numpy(mesh.to_internal(mb["mass_flux"], "edge")).cuda(),
            "n_levels": mb["n_levels"]} for mb in members]
    mesh.autotune_tracer(dev, dt, prec="mix", steps=2)
    mesh.tracer_step(dev, dt, prec="mix")
    torch.cuda.synchronize()
    assert mesh.last_status() == 0
    M = O.Mesh(m)
    # sampled members: the two smallest and the first 25-tracer member
    order = sorted(range(16), key=lambda i: members[i]["n_tracers"] * members[i]["n_levels"])
    sample = order[:2] + [next(i for i in range(16) if members[i]["n_tracers"] == 25)]
    for i in sample:
        mb = members[i]
        ref = O.tracer_step(M, mb["q"], mb["dpi"], mb["mass_flux"], dt)
        got = from_dev(mesh, dev[i]["q"], "cell", 1)
        assert _rel(got, ref) <= 2e-5, i
    mesh.close()


def _coupled_step(mesh, s, P, prec):
    s["mass_flux_accum"].zero_()
    s["vmass_flux_accum"].zero_()
    mesh.dycore_step_nh(s, P, 30.0, prec=prec)
    mesh.tracer_step([{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                       "vmass_flux": s["vmass_flux_accum"], "n_levels": 60}], 30.0, prec=prec)


def test_c5_level9_coupled_properties(G):
    import torch
    from gpu_cases import dycore_params
    m = get_mesh(9)
    mesh = G.Mesh(m)
    L = 60
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    q = S.tracer_mixture(m, 3, L, np.random.default_rng(7))
    q = np.concatenate([q, np.full((1, m["n_cells"], L), 1.5)])     # 4th tracer: constant
    P = dycore_params(mesh, st, L)
    out = {}
    for prec in ("fp64", "mix"):
        fdt = torch.float64 if prec == "fp64" else torch.float32
        s = {"u": torch.from_numpy(mesh.to_internal(st["u"], "edge")).to("cuda", fdt),
             "ps": torch.from_numpy(mesh.to_internal(st["ps"])).cuda(),
             "dpi_theta": torch.from_numpy(mesh.to_internal(st["dpi_theta"])).cuda(),
             "w": torch.from_numpy(mesh.to_internal(st["w"])).cuda(),
             "phi": torch.from_numpy(mesh.to_internal(st["phi"])).cuda(),
             "q": torch.from_numpy(mesh.to_internal(q, "cell", 1)).to("cuda", fdt),
             "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
             "vmass_flux_accum": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
             "dpi_start": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"),
             "p_nh": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"), "p_nh_valid": False}
        dry0 = mesh.global_sum(G.GRIST_SUM_DRY_MASS, s["ps"], offset=st["pi_top"])[0]
        q0 = s["q"][0].clone()
        _coupled_step(mesh, s, P, prec)
        torch.cuda.synchronize()
        assert mesh.last_status() == 0
        dry1 = mesh.global_sum(G.GRIST_SUM_DRY_MASS, s["ps"], offset=st["pi_top"])[0]
        assert abs(dry1 - dry0) / dry0 <= 1e-13, prec
        # free stream of the constant tracer (the tracer step's own continuity)
        dev = float((s["q"][3].double() - 1.5).abs().max())
        assert dev <= (1e-12 if prec == "fp64" else 2e-6), (prec, dev)
        if prec == "fp64":
            # tracer mass over the horizontal and vertical transport: the
            # tracer continuity ends on the dycore's new layer mass,
            # sum A dpi^n q^n == sum A dpi^{n+1} q^{n+1}
            dpi_n = mesh.from_internal(s["dpi_start"].cpu().numpy())
            ps1 = mesh.from_internal(s["ps"].cpu().numpy())
            dpi1 = np.diff(st["pi_top"] + st["b_int"][None, :] * (ps1[:, None] - st["pi_top"]), axis=1)
            # the tracer solver's own end layer mass: dpi^n - dt div(F) -
            # dt (M_{k+1} - M_k) from the fluxes it was given
            Fh = mesh.from_internal(s["mass_flux_accum"].cpu().numpy(), "edge")
            Mv = mesh.from_internal(s["vmass_flux_accum"].cpu().numpy())
            dpi_tr = dpi_n - 30.0 * O.divergence(O.Mesh(m), Fh) - 30.0 * (Mv[:, 1:] - Mv[:, :-1])
            q1 = mesh.from_internal(s["q"][0].cpu().numpy())
            A = m["cell_area"][:, None]
            before = math.fsum((A * dpi_n * mesh.from_internal(q0.cpu().numpy())).ravel())
            after_own = math.fsum((A * dpi_tr * q1).ravel())
            after_dy = math.fsum((A * dpi1 * q1).ravel())
            print("C5 tracer mass: own continuity %.3e, dycore layer mass %.3e, max|dpi_tr/dpi1 - 1| %.3e" % (
                (after_own - before) / before, (after_dy - before) / before, np.max(np.abs(dpi_tr / dpi1 - 1))))
            assert abs(after_own - before) / abs(before) <= 1e-13
            assert abs(after_dy - before) / abs(before) <= 1e-13
        out[prec] = {k: s[k].double().cpu().numpy() for k in ("u", "ps", "dpi_theta", "w", "phi", "q")}
        del s
        torch.cuda.empty_cache()
    a, b = out["mix"], out["fp64"]
    assert _rel(a["u"], b["u"]) <= 2e-5
    assert _rel(a["q"], b["q"]) <= 2e-5
    assert _rel(a["ps"], b["ps"]) <= 1e-7
    for k in ("dpi_theta", "phi"):
        assert _rel(a[k], b[k]) <= 5e-7, k
    mesh.close()
