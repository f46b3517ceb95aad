"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances
* FP64 path: max|x_gpu - x_oracle| / max|x_oracle| <= 1e-12 per field after
  one step (the stated per-step bound; differences come only from the order
  of FP64 operations and the libm pow).
* Mixed path: single-precision storage of u and q and FP32 advective
  arithmetic give ~1e-7 relative rounding per operation; after one step the
  normalised l-infinity error against the FP64 oracle is bounded by 2e-5
  (tracers, winds).  The FP64-kept fields (ps, dpi_theta) see the FP32
  rounding only through their tendency: a mass flux dpi*u ~ 1e5 Pa m/s per
  level rounded at 6e-8, summed over ~30 levels and 6 edges with
  dv/A ~ 1e-5 1/m, gives ~1e-6 Pa/s, i.e. ~6e-9 of ps after a 300 s step;
  bound 1e-7 (measured 2.6e-9).  dpi_theta and phi take FP32 theta (rounded
  at eps32 ~ 6e-8) through ~8 flux terms per cell-level (6 horizontal, 2
  vertical), each up to the layer content times a Courant number ~0.5:
  bound 5e-7 (measured up to 1.5e-7 on the level-9 mesh).
Sizes span several CTAs and a ragged level count with padding (ld > L).
"""
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


@pytest.fixture(scope="module")
def dev_meshes(G, mesh_cache):
    cache = {}

    def get(level):
        if level not in cache:
            cache[level] = (G.Mesh(mesh_cache(level)), mesh_cache(level))
        return cache[level]
    return get


def _rel(a, b):
    return O.max_rel_diff(a, b)


# ---------------------------------------------------------------------------
# tracer

@pytest.mark.parametrize("fct", [True, False])
def test_tracer_fp64_rotation_case(dev_meshes, fct):
    from gpu_cases import run_tracer
    mesh, m = dev_meshes(4)
    c = S.tracer_rotation_case(m, n_levels=30)
    ref = O.tracer_step(O.Mesh(m), c["q"], c["dpi"], c["mass_flux"], c["dt"], fct=fct)
    got = run_tracer(mesh, m, c["q"], c["dpi"], c["mass_flux"], c["dt"], fct=fct)
    assert _rel(got, ref) <= FP64_TOL


@pytest.mark.parametrize("beta", [1.0, 0.25])
def test_tracer_fp64_ragged_divergent(dev_meshes, beta):
    """Several tracers, 37 levels padded to ld = 40, divergent mass flux,
    varying layer mass, level 5 mesh (many CTAs)."""
    from gpu_cases import run_tracer
    mesh, m = dev_meshes(5)
    rng = np.random.default_rng(21)
    L = 37
    F = rng.standard_normal((m["n_edges"], L)) * 2e4
    dpi = 3000.0 + rng.uniform(0, 200, (m["n_cells"], L))
    q = S.tracer_mixture(m, 3, L, rng)
    ref = O.tracer_step(O.Mesh(m), q, dpi, F, 400.0, beta=beta, fct=True)
    got = run_tracer(mesh, m, q, dpi, F, 400.0, beta=beta, fct=True, ld=40)
    assert _rel(got, ref) <= FP64_TOL


def test_tracer_mix_accuracy(dev_meshes):
    from gpu_cases import run_tracer
    mesh, m = dev_meshes(5)
    rng = np.random.default_rng(22)
    L = 30
    members, dt = S.ensemble_members(m, n_members=1, seed=S.SEED + 5)
    mb = members[0]
    ref = O.tracer_step(O.Mesh(m), mb["q"], mb["dpi"], mb["mass_flux"], dt)
    got = run_tracer(mesh, m, mb["q"], mb["dpi"], mb["mass_flux"], dt, prec="mix")
    assert _rel(got, ref) <= 2e-5


def test_tracer_mix_below_discretisation_error(dev_meshes):
    """One day of solid-body rotation: the mixed-precision solution's
    distance from the FP64 oracle is far below the FP64 solution's own
    error against the analytic bell (the paper's acceptance idea, Sec. 2.2,
    with the discretisation error as the yardstick)."""
    from gpu_cases import run_tracer
    mesh, m = dev_meshes(4)
    c = S.tracer_rotation_case(m, n_levels=4)
    M = O.Mesh(m)
    q = c["q"]
    for _ in range(48):
        q = O.tracer_step(M, q, c["dpi"], c["mass_flux"], c["dt"])
    got = run_tracer(mesh, m, c["q"], c["dpi"], c["mass_flux"], c["dt"], prec="mix", steps=48)
    exact = S.bell_exact(m, 48 * c["dt"], c["u0"])
    disc = max(O.error_norms(q[0, :, 0], exact, m["cell_area"]))
    mix = max(O.error_norms(got[0, :, 0], q[0, :, 0], m["cell_area"]))
    assert mix < 1e-3 * disc, (mix, disc)


def test_tracer_mass_and_free_stream_gpu(G, dev_meshes):
    import torch
    from gpu_cases import to_dev
    mesh, m = dev_meshes(5)
    rng = np.random.default_rng(23)
    L = 8
    F = rng.standard_normal((m["n_edges"], L)) * 1e4
    dpi = 3000.0 + rng.uniform(0, 100, (m["n_cells"], L))
    q = np.concatenate([S.tracer_mixture(m, 1, L, rng), np.full((1, m["n_cells"], L), 2.5)])
    qd = to_dev(mesh, q, "cell", 1, torch.float64)
    dpid = to_dev(mesh, dpi, "cell", 0, torch.float64)
    Fd = to_dev(mesh, F, "edge", 0, torch.float64)
    m0 = mesh.global_sum(G.GRIST_SUM_TRACER_MASS, qd[0], dpid, n_levels=L)[0]
    dt = 300.0
    mesh.tracer_step([{"q": qd, "dpi": dpid, "mass_flux": Fd, "n_levels": L}], dt)
    dpi_new = dpi - dt * O.divergence(O.Mesh(m), F)
    m1 = mesh.global_sum(G.GRIST_SUM_TRACER_MASS, qd[0], to_dev(mesh, dpi_new, "cell", 0, torch.float64),
                         n_levels=L)[0]
    assert abs(m1 - m0) / abs(m0) < 1e-13
    assert float((qd[1] - 2.5).abs().max()) < 1e-13


# ---------------------------------------------------------------------------
# dycore

@pytest.mark.parametrize("ld", [None, 33])
def test_hydro_fp64_parity(dev_meshes, ld):
    from gpu_cases import oracle_params, run_dycore
    mesh, m = dev_meshes(4)
    L = 30
    st = S.dycore_jet_case(m, L)
    fa = np.zeros((m["n_edges"], L))
    ref = O.dycore_step_hydro(O.Mesh(m), oracle_params(st, L), st, 300.0, flux_accum=fa)
    got = run_dycore(mesh, st, L, 300.0, nh=False, ld=ld, accum=True)
    for k in ("u", "ps", "dpi_theta"):
        assert _rel(got[k], ref[k]) <= FP64_TOL, k
    assert _rel(got["mass_flux_accum"], fa) <= FP64_TOL
    assert got["accum_weight"] == 1.0


@pytest.mark.parametrize("prec", ["mix", "mix_dbl_mass"])
def test_hydro_mix_accuracy(dev_meshes, prec):
    from gpu_cases import oracle_params, run_dycore
    mesh, m = dev_meshes(5)
    L = 30
    st = S.dycore_jet_case(m, L)
    ref = O.dycore_step_hydro(O.Mesh(m), oracle_params(st, L), st, 300.0)
    got = run_dycore(mesh, st, L, 300.0, nh=False, prec=prec)
    assert _rel(got["u"], ref["u"]) <= 2e-5
    assert _rel(got["ps"], ref["ps"]) <= 1e-7
    assert _rel(got["dpi_theta"], ref["dpi_theta"]) <= 5e-7


def test_nh_fp64_parity(dev_meshes):
    from gpu_cases import oracle_params, run_dycore, spun_up_nh
    mesh, m = dev_meshes(4)
    L = 60
    st = spun_up_nh(m, L)
    ref = O.dycore_step_nh(O.Mesh(m), oracle_params(st, L), st, 120.0)
    got = run_dycore(mesh, st, L, 120.0, nh=True)
    for k in ("u", "ps", "dpi_theta", "phi"):
        assert _rel(got[k], ref[k]) <= FP64_TOL, k
    check_w_fp64(got["w"], ref["w"], 120.0)


def check_w_fp64(w, w_ref, dt, beta=0.55):
    """w leaves the column solve as w** + beta dt g ((p_j - p_{j-1})/dpi_j - 1):
    the difference of two terms of size beta dt g each (dp/dpi ~ 1 in a
    near-hydrostatic column), so its rounding error scales with beta dt g,
    not with the small |w|.  The per-step bound of the FP64 path is held on
    that scale; the ratio beta dt g / max|w| is the cancellation factor."""
    scale = beta * dt * S.GRAVITY
    dw = float(np.max(np.abs(w - w_ref)))
    print("w: max|dw| %.3e m/s = %.2e of beta dt g (%.1f m/s); max|w| %.3e; cancellation factor %.3g"
          % (dw, dw / scale, scale, np.max(np.abs(w_ref)), scale / np.max(np.abs(w_ref))))
    assert dw <= FP64_TOL * scale


@pytest.mark.parametrize("prec", ["mix", "mix_dbl_mass"])
def test_nh_mix_accuracy(dev_meshes, prec):
    from gpu_cases import oracle_params, run_dycore, spun_up_nh
    mesh, m = dev_meshes(4)
    L = 60
    st = spun_up_nh(m, L)
    ref = O.dycore_step_nh(O.Mesh(m), oracle_params(st, L), st, 120.0)
    got = run_dycore(mesh, st, L, 120.0, nh=True, prec=prec)
    assert _rel(got["u"], ref["u"]) <= 2e-5
    assert _rel(got["ps"], ref["ps"]) <= 1e-7
    assert _rel(got["dpi_theta"], ref["dpi_theta"]) <= 5e-7
    assert _rel(got["phi"], ref["phi"]) <= 1e-9
    check_w_mixed(got["w"], ref["w"], 120.0)


def check_w_mixed(w, w_ref, dt, beta=0.55):
    """Mixed path: the advective increments of w and phi are formed in
    binary32, so each carries one binary32 rounding (2^-24 of itself) into
    the column solve, whose terms are of size beta dt g; w can therefore be
    off by up to 2^-24 beta dt g, but not more."""
    scale = beta * dt * S.GRAVITY
    dw = float(np.max(np.abs(w - w_ref)))
    print("mixed w: max|dw| %.3e m/s, %.2e of max|w|, %.2e of beta dt g" % (
        dw, dw / np.max(np.abs(w_ref)), dw / scale))
    assert dw <= 2.0 ** -24 * scale


@pytest.mark.parametrize("nh,prec", [(False, "fp64"), (False, "mix"), (True, "fp64"), (True, "mix")])
def test_dry_mass_conservation_gpu(G, dev_meshes, nh, prec):
    import torch
    from gpu_cases import dycore_params, to_dev
    mesh, m = dev_meshes(5)
    L = 30
    st = S.dycore_jet_case(m, L, nonhydrostatic=nh, bubble=nh)
    dt_u = torch.float64 if prec == "fp64" else torch.float32
    s = {"u": to_dev(mesh, st["u"], "edge", 0, dt_u), "ps": to_dev(mesh, st["ps"], "cell", 0, torch.float64),
         "dpi_theta": to_dev(mesh, st["dpi_theta"], "cell", 0, torch.float64)}
    if nh:
        s["w"] = to_dev(mesh, st["w"], "cell", 0, torch.float64)
        s["phi"] = to_dev(mesh, st["phi"], "cell", 0, torch.float64)
    P = dycore_params(mesh, st, L)
    m0 = mesh.global_sum(G.GRIST_SUM_DRY_MASS, s["ps"], offset=st["pi_top"])[0]
    for _ in range(5):
        (mesh.dycore_step_nh if nh else mesh.dycore_step_hydro)(s, P, 120.0 if nh else 300.0, prec=prec)
    m1 = mesh.global_sum(G.GRIST_SUM_DRY_MASS, s["ps"], offset=st["pi_top"])[0]
    assert abs(m1 - m0) / m0 <= 1e-13
    assert mesh.last_status() == 0


# ---------------------------------------------------------------------------
# sums, status, validation

def test_global_sums_vs_fsum(G, dev_meshes):
    import torch
    from gpu_cases import to_dev
    mesh, m = dev_meshes(5)
    rng = np.random.default_rng(24)
    ps = 1e5 + rng.standard_normal(m["n_cells"]) * 1e3
    got = mesh.global_sum(G.GRIST_SUM_DRY_MASS, to_dev(mesh, ps, "cell", 0, torch.float64), offset=225.0)[0]
    exact = math.fsum(m["cell_area"] * (ps - 225.0))
    assert abs(got - exact) <= 4 * np.spacing(abs(exact))
    L = 7
    q = rng.standard_normal((m["n_cells"], L))
    dpi = rng.uniform(100, 5000, (m["n_cells"], L))
    got = mesh.global_sum(G.GRIST_SUM_TRACER_MASS, to_dev(mesh, q, "cell", 0, torch.float64),
                          to_dev(mesh, dpi, "cell", 0, torch.float64), n_levels=L)[0]
    exact = math.fsum((m["cell_area"][:, None] * dpi * q).ravel())
    assert abs(got - exact) <= 4 * np.spacing(abs(exact)) + 1e-15 * np.sum(np.abs(m["cell_area"][:, None] * dpi * q))
    # determinism
    again = mesh.global_sum(G.GRIST_SUM_TRACER_MASS, to_dev(mesh, q, "cell", 0, torch.float64),
                            to_dev(mesh, dpi, "cell", 0, torch.float64), n_levels=L)[0]
    assert again == got


def test_nonfinite_flag(G, dev_meshes):
    import torch
    from gpu_cases import to_dev
    mesh, m = dev_meshes(3)
    L = 4
    q = np.ones((1, m["n_cells"], L))
    q[0, 5, 2] = np.nan
    qd = to_dev(mesh, q, "cell", 1, torch.float64)
    F = np.zeros((m["n_edges"], L))
    dpi = np.full((m["n_cells"], L), 1000.0)
    mesh.last_status()
    mesh.tracer_step([{"q": qd, "dpi": to_dev(mesh, dpi), "mass_flux": to_dev(mesh, F, "edge"), "n_levels": L}],
                     10.0, limiter=False)
    assert mesh.last_status() & G.GRIST_FLAG_NONFINITE
    assert mesh.last_status() == 0


def test_invalid_arguments(G, dev_meshes):
    import torch
    mesh, m = dev_meshes(3)
    q = torch.zeros((1, mesh.nC, 4), dtype=torch.float64, device="cuda")
    dpi = torch.ones((mesh.nC, 4), dtype=torch.float64, device="cuda")
    F = torch.zeros((mesh.nE, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GristError) as e:
        mesh.tracer_step([{"q": q, "dpi": dpi, "mass_flux": F, "n_levels": 4}], -1.0)
    assert e.value.code == -1
    with pytest.raises(G.GristError):
        mesh.tracer_step([{"q": q, "dpi": dpi, "mass_flux": F, "n_levels": 5}], 1.0)   # ld < L
