"""GPU: the two forms of the tracer edge fluxes (Sec. 2.1 third-order upwind
flux with beta = 1).  Edge-centric: one thread per edge-level gathers the
upwind cell's stencil.  Cell-centric (grist_tracer_tuning.cell_edges): the
upwind cell's thread gathers its neighbour ring once and writes the flux of
every edge whose flux leaves it.  Both use the same weights in the same
order, so a tracer step gives the same bits either way, in every launch
mode and precision; and the edge-centric form alone also matches the FP64
oracle (the default, cell-centric form is checked against it by the other
tracer tests)."""
import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S

pytestmark = pytest.mark.gpu

SHAPES = [(4, 60, 60), (3, 37, 40), (2, 8, 8)]   # (T, L, ld): ragged level groups, padded rows


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    return G


def _members(m, rng):
    out = []
    for T, L, ld in SHAPES:
        out.append({"q": S.tracer_mixture(m, T, L, rng), "dpi": 3000.0 + rng.uniform(0, 200, (m["n_cells"], L)),
                    "F": rng.standard_normal((m["n_edges"], L)) * 2e4, "L": L, "ld": ld})
    return out


def _run(mesh, members, prec, limiter, steps=2):
    import torch
    from gpu_cases import from_dev, to_dev
    dq = torch.float64 if prec == "fp64" else torch.float32
    dev = [{"q": to_dev(mesh, mb["q"], "cell", 1, dq, mb["ld"]),
            "dpi": to_dev(mesh, mb["dpi"], "cell", 0, torch.float64, mb["ld"]),
            "mass_flux": to_dev(mesh, mb["F"], "edge", 0, torch.float64, mb["ld"]), "n_levels": mb["L"]}
           for mb in members]
    for _ in range(steps):
        mesh.tracer_step(dev, 300.0, prec=prec, limiter=limiter)
    torch.cuda.synchronize()
    return [from_dev(mesh, d["q"], "cell", 1, n=mb["L"]) for d, mb in zip(dev, members)]


@pytest.mark.parametrize("level", [3, 4])
def test_meshes_have_ring_stencils(G, mesh_cache, level):
    mesh = G.Mesh(mesh_cache(level))
    assert mesh.features() == {"combined_stencil": True, "ring_stencil": True}
    mesh.close()


@pytest.mark.parametrize("prec", ["fp64", "mix"])
@pytest.mark.parametrize("limiter", [True, False])
@pytest.mark.parametrize("mode", [{"levels_per_thread": 2}, {"levels_per_thread": 1, "tracers_per_thread": 1},
                                  {"persistent": True}])
def test_cell_and_edge_forms_give_the_same_bits(G, mesh_cache, prec, limiter, mode):
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    members = _members(m, np.random.default_rng(71))
    tune = {"block": 128, "tracers_per_thread": 2}
    tune.update(mode)
    mesh.set_tracer_tuning(cell_edges=True, **tune)
    a = _run(mesh, members, prec, limiter)
    mesh.set_tracer_tuning(cell_edges=False, **tune)
    b = _run(mesh, members, prec, limiter)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    mesh.close()


def test_edge_form_fp64_parity(G, mesh_cache):
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    members = _members(m, np.random.default_rng(72))
    mesh.set_tracer_tuning(block=128, tracers_per_thread=2, levels_per_thread=2, cell_edges=False)
    got = _run(mesh, members, "fp64", True)
    M = O.Mesh(m)
    for g, mb in zip(got, members):
        q = mb["q"]
        for _ in range(2):
            q = O.tracer_step(M, q, mb["dpi"], mb["F"], 300.0)
        assert O.max_rel_diff(g, q) <= 1e-12
    mesh.close()
