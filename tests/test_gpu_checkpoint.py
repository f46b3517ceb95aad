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


class _Pipeline:
    """The coupled steps with the tracers of step n on a second stream beside
    the dycore of step n + 1.  The passive tracers never feed back into the
    dycore; the dycore of step n + 1 writes the other of two flux buffers
    (horizontal and vertical mass-flux accumulators, dpi^n), and waits for
    the tracer step that last read it.  Results are those of the sequential
    schedule (same kernels, same inputs)."""

    def __init__(self, torch, mesh, s, P, wl, prec):
        # torch, mesh handle, state dict, dycore params, workload dict, policy
        self.torch, self.mesh, self.s, self.P, self.wl, self.prec = torch, mesh, s, P, wl, prec
        self.side = torch.cuda.Stream(device=s["ps"].device)
        self.bufs = [{k: s[k].clone() for k in ("mass_flux_accum", "vmass_flux_accum", "dpi_start")}
                     for _ in range(2)]
        self.dyc_done = [torch.cuda.Event(), torch.cuda.Event()]
        self.trc_done = [None, None]
        self.n = 0

    def step(self):
        torch, s, wl = self.torch, self.s, self.wl
        main = torch.cuda.current_stream()
        i = self.n % 2
        b = self.bufs[i]
        if self.trc_done[i] is not None:
            main.wait_event(self.trc_done[i])            # the tracer step that read this buffer
        b["mass_flux_accum"].zero_()
        b["vmass_flux_accum"].zero_()
        st = dict(s, **b)
        if wl["nh"]:
            self.mesh.dycore_step_nh(st, self.P, wl["dt"], prec=self.prec)
            s["p_nh_valid"] = st["p_nh_valid"]
        else:
            self.mesh.dycore_step_hydro(st, self.P, wl["dt"], prec=self.prec)
        self.dyc_done[i].record(main)
        self.side.wait_event(self.dyc_done[i])
        self.mesh.tracer_step([{"q": s["q"], "dpi": b["dpi_start"], "mass_flux": b["mass_flux_accum"],
                                "vmass_flux": b["vmass_flux_accum"], "n_levels": wl["L"]}], wl["dt"],
                              prec=self.prec, limiter=True, stream=self.side)
        ev = torch.cuda.Event()
        ev.record(self.side)
        self.trc_done[i] = ev
        self.n += 1

    def join(self):
        """Make the caller's stream wait for the last tracer step."""
        for ev in self.trc_done:
            if ev is not None:
                self.torch.cuda.current_stream().wait_event(ev)


@pytest.mark.parametrize("use_graph", [False, True])
def test_two_stream_pipeline_equals_sequential(G, mesh_cache, use_graph):
    """A caller may run the tracers of step n on a second stream beside the
    dycore of step n + 1 (separate scratch; fluxes double-buffered): the
    state equals the sequential schedule's bit for bit, with and without the
    tracer step's graph replay (its cache then holds one graph per buffer)."""
    import os
    import sys
    import torch
    from gpu_cases import dycore_params
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    m = mesh_cache(4)
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    q0 = S.tracer_mixture(m, 3, L, np.random.default_rng(22))
    wl = {"nh": True, "T": 3, "L": L, "dt": DT}
    out = []
    for pipelined in (False, True):
        mesh = G.Mesh(m)
        mesh.set_tracer_tuning(block=256, tracers_per_thread=4, use_graph=use_graph)
        P = dycore_params(mesh, st, L)
        s = _state(mesh, st, q0, "mix")
        if pipelined:
            pipe = _Pipeline(torch, mesh, s, P, wl, "mix")
            for _ in range(5):
                pipe.step()
            pipe.join()
        else:
            for _ in range(5):
                bench.step(mesh, s, P, wl, "mix")
        torch.cuda.synchronize()
        assert mesh.last_status() == 0
        out.append({k: s[k].cpu().numpy() for k in KEYS})
        mesh.close()
    for k in KEYS:
        assert np.array_equal(out[0][k], out[1][k]), k
