"""GPU: a whole coupled step (dycore step, zeroed flux accumulators, tracer
step with the dycore's horizontal and vertical fluxes) recorded once as a
CUDA graph and replayed must give the same state, bit for bit, as the same
steps launched call by call; so must the tracer work list with two levels
per thread (against the oracle)."""
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


def _state(torch, mesh, st, q, L, prec):
    fdt = torch.float64 if prec == "fp64" else torch.float32
    to = mesh.to_internal
    return {"u": torch.from_numpy(to(st["u"], "edge")).to("cuda", fdt),
            "ps": torch.from_numpy(to(st["ps"])).cuda(),
            "dpi_theta": torch.from_numpy(to(st["dpi_theta"])).cuda(),
            "w": torch.from_numpy(to(st["w"])).cuda(), "phi": torch.from_numpy(to(st["phi"])).cuda(),
            "q": torch.from_numpy(to(q, "cell", 1)).to("cuda", fdt),
            "mass_flux_accum": torch.zeros((mesh.nE, L), dtype=torch.float64, device="cuda"),
            "vmass_flux_accum": torch.zeros((mesh.nC, L + 1), dtype=torch.float64, device="cuda"),
            "dpi_start": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"),
            "p_nh": torch.zeros((mesh.nC, L), dtype=torch.float64, device="cuda"), "p_nh_valid": False}


@pytest.mark.parametrize("prec", ["fp64", "mix"])
def test_captured_coupled_step_replays_bit_for_bit(G, mesh_cache, prec):
    import torch
    from gpu_cases import dycore_params
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    L, dt = 30, 120.0
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    q = S.tracer_mixture(m, 3, L, np.random.default_rng(3))
    P = dycore_params(mesh, st, L)
    stream = torch.cuda.Stream()
    # the tracer's own graph cache on: inside the whole-step capture its
    # kernels must be recorded, not a cached graph launched
    mesh.set_tracer_tuning(block=128, tracers_per_thread=4, use_graph=True, levels_per_thread=2)

    def step(s):
        s["mass_flux_accum"].zero_()
        s["vmass_flux_accum"].zero_()
        mesh.dycore_step_nh(s, P, dt, prec=prec)
        mesh.tracer_step([{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                           "vmass_flux": s["vmass_flux_accum"], "n_levels": L}], dt, prec=prec)

    keys = ("u", "ps", "dpi_theta", "w", "phi", "q", "p_nh")
    with torch.cuda.stream(stream):
        a = _state(torch, mesh, st, q, L, prec)
        b = _state(torch, mesh, st, q, L, prec)
        step(a)            # each buffer set's first call: scratch, tables, carried pressure
        step(b)
        for _ in range(3):
            step(a)
    graph = G.capture(lambda: step(b), stream)
    for _ in range(3):
        graph.launch()
    torch.cuda.synchronize()
    for k in keys:
        assert torch.equal(a[k], b[k]), k
    assert mesh.last_status() == 0
    # a buffer set that never ran outside a capture cannot be recorded: the
    # call reports it, the capture ends, and the stream stays usable
    with torch.cuda.stream(stream):
        c = _state(torch, mesh, st, q, L, prec)
        c["p_nh_valid"] = True
    with pytest.raises(G.GristError):
        G.capture(lambda: step(c), stream)
    with torch.cuda.stream(stream):
        step(a)
        graph.launch()                            # the recorded graph still replays b's step
    torch.cuda.synchronize()
    for k in keys:
        assert torch.equal(a[k], b[k]), k
    graph.close()
    mesh.close()


@pytest.mark.parametrize("limiter", [True, False])
def test_two_levels_per_thread_fp64_parity(G, mesh_cache, limiter):
    import torch
    from gpu_cases import run_tracer
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    rng = np.random.default_rng(44)
    L = 37                                        # odd: the last level group holds one level
    F = rng.standard_normal((m["n_edges"], L)) * 2e4
    dpi = 3000.0 + rng.uniform(0, 200, (m["n_cells"], L))
    q = S.tracer_mixture(m, 3, L, rng)
    mesh.set_tracer_tuning(block=128, tracers_per_thread=2, levels_per_thread=2)
    ref = O.tracer_step(O.Mesh(m), q, dpi, F, 300.0, fct=limiter)
    got = run_tracer(mesh, m, q, dpi, F, 300.0, fct=limiter, ld=40)
    assert O.max_rel_diff(got, ref) <= 1e-12
    mesh.close()
