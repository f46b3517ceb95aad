"""GPU: batched uneven tracer ensembles in one call (work list over members
and tracer groups), in every launch mode (per-phase launches, persistent
cooperative launch, CUDA-graph replay), against the FP64 oracle member by
member; the autotuner; the bounded device wait."""
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


def _members(m, rng, shapes):
    """Uneven members: (T, L, ld) each, divergent fluxes, varying dpi."""
    out = []
    for T, L, ld in shapes:
        F = rng.standard_normal((m["n_edges"], L)) * 2e4
        dpi = 3000.0 + rng.uniform(0, 200, (m["n_cells"], L))
        q = S.tracer_mixture(m, T, L, rng)
        out.append({"q": q, "dpi": dpi, "F": F, "L": L, "ld": ld})
    return out


def _run(G, mesh, members, dt, prec, steps=1, tuning=None, limiter=True):
    import torch
    from gpu_cases import from_dev, to_dev
    if tuning:
        mesh.set_tracer_tuning(**tuning)
    dq = torch.float64 if prec == "fp64" else torch.float32
    dev = []
    for mb in members:
        dev.append({"q": to_dev(mesh, mb["q"], "cell", 1, dq, mb["ld"]),
                    "dpi": to_dev(mesh, mb["dpi"], "cell", 0, torch.float64, mb["ld"]),
                    "mass_flux": to_dev(mesh, mb["F"], "edge", 0, torch.float64, mb["ld"]),
                    "n_levels": mb["L"]})
    for _ in range(steps):
        mesh.tracer_step(dev, dt, prec=prec, limiter=limiter)
    torch.cuda.synchronize()
    return [from_dev(mesh, d["q"], "cell", 1, n=mb["L"]) for d, mb in zip(dev, members)]


SHAPES = [(1, 30, 30), (4, 60, 60), (10, 37, 40), (3, 8, 8), (25, 12, 16)]
TUNINGS = [None,
           {"block": 128, "tracers_per_thread": 1, "fused": False},
           {"block": 512, "tracers_per_thread": 8, "fused": False},
           {"block": 256, "tracers_per_thread": 3, "fused": True},
           {"block": 256, "tracers_per_thread": 4, "persistent": True},
           {"block": 256, "tracers_per_thread": 2, "use_graph": True},
           {"block": 256, "tracers_per_thread": 4, "persistent": True, "use_graph": True},
           {"block": 256, "tracers_per_thread": 4, "levels_per_thread": 2},
           {"block": 512, "tracers_per_thread": 1, "levels_per_thread": 2, "use_graph": True},
           {"block": 128, "tracers_per_thread": 4, "levels_per_thread": 2, "cell_edges": False},
           {"block": 256, "tracers_per_thread": 2, "persistent": True, "cell_edges": False}]


@pytest.mark.parametrize("tuning", TUNINGS)
def test_uneven_batch_fp64_parity(G, mesh_cache, tuning):
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(41)
    members = _members(m, rng, SHAPES)
    M = O.Mesh(m)
    steps = 2
    refs = []
    for mb in members:
        q = mb["q"]
        for _ in range(steps):
            q = O.tracer_step(M, q, mb["dpi"], mb["F"], 300.0)
        refs.append(q)
    got = _run(G, mesh, members, 300.0, "fp64", steps=steps, tuning=tuning)
    for g, r in zip(got, refs):
        assert O.max_rel_diff(g, r) <= FP64_TOL
    assert mesh.last_status() == 0
    mesh.close()


@pytest.mark.parametrize("fused", [True, False])
def test_uneven_batch_no_limiter_fp64(G, mesh_cache, fused):
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(43)
    members = _members(m, rng, [(2, 30, 32), (5, 45, 45)])
    M = O.Mesh(m)
    got = _run(G, mesh, members, 300.0, "fp64", steps=2, limiter=False,
               tuning={"block": 256, "tracers_per_thread": 2, "fused": fused})
    for g, mb in zip(got, members):
        q = mb["q"]
        for _ in range(2):
            q = O.tracer_step(M, q, mb["dpi"], mb["F"], 300.0, fct=False)
        assert O.max_rel_diff(g, q) <= FP64_TOL
    mesh.close()


def test_uneven_batch_mix(G, mesh_cache):
    m = mesh_cache(5)
    mesh = G.Mesh(m)
    members, dt = S.ensemble_members(m, n_members=6, seed=S.SEED + 100)
    M = O.Mesh(m)
    batch = [{"q": mb["q"], "dpi": mb["dpi"], "F": mb["mass_flux"], "L": mb["n_levels"], "ld": mb["n_levels"]}
             for mb in members]
    got = _run(G, mesh, batch, dt, "mix", tuning={"block": 256, "tracers_per_thread": 4, "persistent": True})
    for g, mb in zip(got, members):
        ref = O.tracer_step(M, mb["q"], mb["dpi"], mb["mass_flux"], dt)
        assert O.max_rel_diff(g, ref) <= 2e-5
    mesh.close()


def test_autotune_keeps_caller_data_and_picks_valid_tuning(G, mesh_cache, tmp_path):
    import torch
    from gpu_cases import to_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(42)
    members = _members(m, rng, [(4, 30, 30), (10, 60, 60)])
    dev = [{"q": to_dev(mesh, mb["q"], "cell", 1, torch.float32),
            "dpi": to_dev(mesh, mb["dpi"], "cell", 0, torch.float64),
            "mass_flux": to_dev(mesh, mb["F"], "edge", 0, torch.float64), "n_levels": mb["L"]} for mb in members]
    before = [d["q"].clone() for d in dev]
    cache = str(tmp_path / "tune.json")
    t, ms = mesh.autotune_tracer(dev, 300.0, prec="mix", steps=2, cache_path=cache, cache_key="L4-test")
    assert t["block"] in (128, 256, 512) and t["tracers_per_thread"] in (1, 2, 4, 8)
    assert t["levels_per_thread"] in (1, 2)
    assert ms is not None and ms > 0
    for d, b in zip(dev, before):
        assert torch.equal(d["q"], b)
    # cached choice is reused without re-timing
    t2, ms2 = mesh.autotune_tracer(dev, 300.0, prec="mix", cache_path=cache, cache_key="L4-test")
    assert t2 == t and ms2 == ms
    # a step with the tuned configuration still matches the default one
    from gpu_cases import from_dev
    mesh.tracer_step(dev, 300.0, prec="mix")
    tuned = [from_dev(mesh, d["q"], "cell", 1) for d in dev]
    mesh.set_tracer_tuning()
    for d, b in zip(dev, before):
        d["q"].copy_(b)
    mesh.tracer_step(dev, 300.0, prec="mix")
    plain = [from_dev(mesh, d["q"], "cell", 1) for d in dev]
    for a, b in zip(tuned, plain):
        assert O.max_rel_diff(a, b) <= 2e-6
    assert mesh.last_status() == 0
    mesh.close()


def test_bounded_wait_times_out_and_context_survives(G, mesh_cache):
    import torch
    m = mesh_cache(3)
    mesh = G.Mesh(m)
    mesh.last_status()
    mesh.selftest_bounded_wait(spin_limit=20000)
    assert mesh.last_status() & G.GRIST_FLAG_TIMEOUT
    # the context is still usable: a normal step runs and reports no flags
    from gpu_cases import run_tracer
    c = S.tracer_rotation_case(m, n_levels=4)
    ref = O.tracer_step(O.Mesh(m), c["q"], c["dpi"], c["mass_flux"], c["dt"])
    got = run_tracer(mesh, m, c["q"], c["dpi"], c["mass_flux"], c["dt"])
    assert O.max_rel_diff(got, ref) <= FP64_TOL
    assert mesh.last_status() == 0
    mesh.close()


def test_tuning_rejects_unlaunchable_block(G, mesh_cache):
    """Blocks above 512 threads are refused when set, not at launch."""
    m = mesh_cache(3)
    mesh = G.Mesh(m)
    for bad in (1024, 544, 48, 100):
        with pytest.raises(G.GristError):
            mesh.set_tracer_tuning(block=bad, tracers_per_thread=4)
    mesh.set_tracer_tuning(block=512, tracers_per_thread=8)
    assert mesh.tracer_tuning()["block"] == 512
    mesh.close()
