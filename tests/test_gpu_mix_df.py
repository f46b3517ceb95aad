"""GPU: the FP32-dominant policy GRIST_MIX_DF (the pressure-gradient,
gravity and kinetic-energy-gradient terms in binary32 arithmetic with their
differences of double fields taken from double-float splits; the NH
equation of state as a double base plus a binary32 increment).  One step of
the hydrostatic and the non-hydrostatic core against the FP64 oracle within
the mixed-policy tolerances, and against the GRIST_MIX step (which computes
those terms in FP64): the two agree to single-precision rounding of the
tendencies."""
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


@pytest.mark.parametrize("nh", [False, True])
def test_mix_df_step_against_oracle_and_mix(G, mesh_cache, nh):
    from gpu_cases import oracle_params, run_dycore
    m = mesh_cache(5)
    mesh = G.Mesh(m)
    L = 30
    dt = 60.0 if nh else 300.0
    st = S.dycore_jet_case(m, L, nonhydrostatic=nh, bubble=nh)
    M = O.Mesh(m)
    P = oracle_params(st, L)
    ref = O.dycore_step_nh(M, P, st, dt) if nh else O.dycore_step_hydro(M, P, st, dt)
    df = run_dycore(mesh, st, L, dt, nh=nh, prec="mix_df")
    mix = run_dycore(mesh, st, L, dt, nh=nh, prec="mix")
    assert O.max_rel_diff(df["u"], ref["u"]) <= 2e-5
    assert O.max_rel_diff(df["ps"], ref["ps"]) <= 1e-7
    assert O.max_rel_diff(df["dpi_theta"], ref["dpi_theta"]) <= 5e-7
    if nh:
        assert O.max_rel_diff(df["phi"], ref["phi"]) <= 5e-7
    # against GRIST_MIX: the same except for the binary32 rounding inside
    # the slow tendency (~2^-24 of it), far below the policy's own error
    assert O.max_rel_diff(df["u"], mix["u"]) <= 2e-6
    # the surface pressure sees the wind difference only through the column
    # mass flux: |d ps / dt| changes by at most max_i sum_j (dv_j / A_i) *
    # (ps - pi_top) * max|du| per unit time, so over the step
    # |dps| / ps <= dt * max_i sum_j dv_j / A_i * max|du|
    import numpy as np
    dv = m["edge_dv"][np.maximum(m["edges_on_cell"], 0)] * (m["edges_on_cell"] >= 0)
    perim = np.max(dv.sum(axis=1) / m["cell_area"])
    du = float(np.max(np.abs(df["u"] - mix["u"])))
    assert O.max_rel_diff(df["ps"], mix["ps"]) <= dt * perim * du, (O.max_rel_diff(df["ps"], mix["ps"]),
                                                                     dt * perim * du)
    mesh.close()
