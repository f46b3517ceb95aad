"""Shared set-up for the GPU parity tests: builds the same seeded inputs for
the oracle (original numbering, NumPy) and the CUDA library (internal
numbering, torch CUDA tensors), runs both, maps results back."""
import numpy as np

import oracle as O
from grist_inputs import states as S


def torch_mod():
    import torch
    return torch


def to_dev(mesh, a, kind="cell", axis=0, dtype=None, ld=None):
    """NumPy array in generator numbering -> CUDA tensor in internal
    numbering (optionally padded along the last axis to ld)."""
    torch = torch_mod()
    b = mesh.to_internal(a, kind, axis)
    if ld is not None and b.shape[-1] < ld:
        pad = np.full(b.shape[:-1] + (ld - b.shape[-1],), np.nan)
        b = np.concatenate([b, pad], axis=-1)
    t = torch.from_numpy(np.ascontiguousarray(b))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def from_dev(mesh, t, kind="cell", axis=0, n=None):
    a = t.detach().cpu().numpy().astype(np.float64)
    if n is not None:
        a = a[..., :n]
    return mesh.from_internal(a, kind, axis)


def run_tracer(mesh, m, q, dpi, F, dt, prec="fp64", fct=True, beta=1.0, ld=None, steps=1):
    torch = torch_mod()
    T, nC, L = q.shape
    ld = ld or L
    dt_q = torch.float64 if prec == "fp64" else torch.float32
    qd = to_dev(mesh, q, "cell", 1, dt_q, ld)
    mb = {"q": qd, "dpi": to_dev(mesh, dpi, "cell", 0, torch.float64, ld),
          "mass_flux": to_dev(mesh, F, "edge", 0, torch.float64, ld), "n_levels": L}
    for _ in range(steps):
        mesh.tracer_step([mb], dt, prec=prec, limiter=fct, beta=beta)
    torch.cuda.synchronize()
    return from_dev(mesh, qd, "cell", 1, n=L)


def dycore_params(mesh, st, L, beta=0.55, ld=None, ld_int=None):
    import paper_2404_08849_gb300 as G
    torch = torch_mod()
    phis = to_dev(mesh, st["phi_s"], "cell", 0, torch.float64)
    return G.DycoreParams(L, st["b_int"], st["pi_top"], phis, ld=ld, ld_int=ld_int, beta=beta)


def run_dycore(mesh, st, L, dt, nh, prec="fp64", steps=1, ld=None, ld_int=None, accum=False):
    torch = torch_mod()
    ld = ld or L
    ld_int = ld_int or (L + 1)
    dt_u = torch.float64 if prec == "fp64" else torch.float32
    s = {"u": to_dev(mesh, st["u"], "edge", 0, dt_u, ld),
         "ps": to_dev(mesh, st["ps"], "cell", 0, torch.float64),
         "dpi_theta": to_dev(mesh, st["dpi_theta"], "cell", 0, torch.float64, ld)}
    if nh:
        s["w"] = to_dev(mesh, st["w"], "cell", 0, torch.float64, ld_int)
        s["phi"] = to_dev(mesh, st["phi"], "cell", 0, torch.float64, ld_int)
    if accum:
        s["mass_flux_accum"] = torch.zeros((mesh.nE, ld), dtype=torch.float64, device="cuda")
        s["accum_weight"] = torch.zeros(1, dtype=torch.float64, device="cuda")
    P = dycore_params(mesh, st, L, ld=ld, ld_int=ld_int)
    for _ in range(steps):
        if nh:
            mesh.dycore_step_nh(s, P, dt, prec=prec)
        else:
            mesh.dycore_step_hydro(s, P, dt, prec=prec)
    torch.cuda.synchronize()
    out = {"u": from_dev(mesh, s["u"], "edge", 0, n=L), "ps": from_dev(mesh, s["ps"], "cell", 0),
           "dpi_theta": from_dev(mesh, s["dpi_theta"], "cell", 0, n=L)}
    if nh:
        out["w"] = from_dev(mesh, s["w"], "cell", 0, n=L + 1)
        out["phi"] = from_dev(mesh, s["phi"], "cell", 0, n=L + 1)
    if accum:
        out["mass_flux_accum"] = from_dev(mesh, s["mass_flux_accum"], "edge", 0, n=L)
        out["accum_weight"] = float(s["accum_weight"].item())
    return out


def oracle_params(st, L, beta=0.55):
    return O.Params(L, st["b_int"], st["pi_top"], st["phi_s"], beta=beta)


def spun_up_nh(m, L, steps=3, dt=120.0):
    """NH jet + bubble advanced a few oracle steps so that w and the
    non-hydrostatic pressure are non-trivial."""
    st = S.dycore_jet_case(m, L, nonhydrostatic=True, bubble=True)
    M = O.Mesh(m)
    P = oracle_params(st, L)
    s = dict(st)
    for _ in range(steps):
        s2 = O.dycore_step_nh(M, P, s, dt)
        s.update({k: s2[k] for k in ("ps", "u", "dpi_theta", "w", "phi")})
    return s
