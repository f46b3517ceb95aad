"""Iterative precision search (Sec. 2.2, Eqs. 1-2) on the library's dycore.

The FP64 run is the truth.  Candidate precision reductions - rows of the
precision map, each emulated by rounding that row's FP64 results to binary32
where they are produced (``grist_dycore_params.emulate_fp32_rows``) - are
tried one at a time on top of the configuration accepted so far; a run of
the same case gives the overall error

    E = max(L(ps), L(vor)),   L(x) = max(l1, l2, linf)          (Eqs. 1-2)

against the FP64 run (normalised norms, area-weighted: cells for the
surface pressure, vertices for the relative vorticity on every level).  A
candidate with E <= alpha (0.05 in the paper) is kept and the next reduction
builds on it; otherwise it is abandoned.

Usage (GPU):  python -m paper_2404_08849_gb300.precision --level 5 --steps 288
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import GRIST_ROWS, DycoreParams, Mesh

# candidate order: advective rows first, then the "boxed" tendencies, the
# vertex layer mass under the PV, and the pressure-gradient / EOS rows
DEFAULT_ORDER = ("theta", "pv_flux", "nh_adv", "mass_flux", "wind", "ke_grad", "vadv_u", "dpi_pv", "pgf", "eos")


def error_norms(x, ref, weight):
    """Normalised (l1, l2, linf) of x against ref: l1 = I|x - r| / I|r|,
    l2 = sqrt(I(x - r)^2 / I r^2), linf = max|x - r| / max|r|, with I the
    weighted sum (weight broadcast over trailing axes)."""
    x = np.asarray(x, np.float64)
    r = np.asarray(ref, np.float64)
    w = np.asarray(weight, np.float64)
    w = w.reshape(w.shape + (1,) * (x.ndim - w.ndim))
    d = x - r
    l1 = float(np.sum(w * np.abs(d)) / np.sum(w * np.abs(r)))
    l2 = float(math.sqrt(np.sum(w * d * d) / np.sum(w * r * r)))
    linf = float(np.max(np.abs(d)) / np.max(np.abs(r)))
    return l1, l2, linf


def error_level(x, ref, weight):
    """L(x) of Eq. 2; a non-finite norm (a run that blew up) counts as
    infinitely wrong (Python's max would silently skip a NaN)."""
    n = error_norms(x, ref, weight)
    return max(n) if all(math.isfinite(v) for v in n) else math.inf


def overall_error(ps, ps_ref, vor, vor_ref, cell_area, vertex_area):
    """E of Eq. 1."""
    return max(error_level(ps, ps_ref, cell_area), error_level(vor, vor_ref, vertex_area))


class Experiment:
    """One dycore case run from the same initial state for every candidate.
    m: mesh tables (generator numbering); state: the initial state in the
    generator's numbering (u, ps, dpi_theta, and w, phi for the NH core,
    b_int, pi_top, phi_s)."""

    def __init__(self, m, state, n_levels, dt, steps, nonhydrostatic, device=0):
        import torch
        self.torch = torch
        self.mesh = Mesh(m, device=device)
        self.m, self.st, self.L, self.dt, self.steps, self.nh = m, state, n_levels, dt, steps, nonhydrostatic
        self.device = device
        to = self.mesh.to_internal
        self.host = {"u": to(state["u"], "edge"), "ps": to(state["ps"]), "dpi_theta": to(state["dpi_theta"])}
        if nonhydrostatic:
            self.host["w"] = to(state["w"])
            self.host["phi"] = to(state["phi"])
        self.phis = torch.from_numpy(to(state["phi_s"])).to(device)
        self.cell_area = to(m["cell_area"])
        self.vertex_area = to(m["vertex_area"], "vertex")

    def run(self, mask=0, prec="fp64"):
        """Advance `steps` steps with the emulated rows `mask`; returns the
        final (ps [nC], vor [nV][L]) on the host, internal numbering."""
        torch = self.torch
        fdt = torch.float64 if prec == "fp64" else torch.float32
        s = {k: torch.from_numpy(v).to(self.device) for k, v in self.host.items()}
        s["u"] = s["u"].to(fdt)
        if self.nh:
            s["p_nh"] = torch.zeros((self.mesh.nC, self.L), dtype=torch.float64, device=self.device)
            s["p_nh_valid"] = False
        P = DycoreParams(self.L, self.st["b_int"], self.st["pi_top"], self.phis, emulate_fp32_rows=mask)
        step = self.mesh.dycore_step_nh if self.nh else self.mesh.dycore_step_hydro
        for _ in range(self.steps):
            step(s, P, self.dt, prec=prec)
        vor = self.mesh.vorticity(s["u"], self.L)
        torch.cuda.synchronize()
        return s["ps"].cpu().numpy(), vor.cpu().numpy()

    def error(self, result, truth):
        return overall_error(result[0], truth[0], result[1], truth[1], self.cell_area, self.vertex_area)

    def close(self):
        self.mesh.close()


def iterative_search(exp, rows=DEFAULT_ORDER, alpha=0.05, truth=None):
    """The procedure of Sec. 2.2: returns (accepted mask, accepted row names,
    table of {row, mask, E, accepted} in trial order)."""
    truth = truth if truth is not None else exp.run(0)
    config, kept, table = 0, [], []
    for name in rows:
        cand = config | GRIST_ROWS[name]
        e = exp.error(exp.run(cand), truth)
        ok = e <= alpha
        if ok:
            config, kept = cand, kept + [name]
        table.append({"row": name, "mask": cand, "E": e, "accepted": ok})
    return config, kept, table


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--level", type=int, default=5)
    ap.add_argument("--levels", type=int, default=30)
    ap.add_argument("--nh", action="store_true", help="non-hydrostatic core (default hydrostatic)")
    ap.add_argument("--dt", type=float, default=None)
    ap.add_argument("--steps", type=int, default=288)
    ap.add_argument("--alpha", type=float, default=0.05)
    args = ap.parse_args()
    from grist_inputs import states as S
    from grist_inputs.mesh import get_mesh
    m = get_mesh(args.level)
    dt = args.dt or (60.0 if args.nh else 300.0)
    st = S.dycore_jet_case(m, args.levels, nonhydrostatic=args.nh, bubble=args.nh)
    exp = Experiment(m, st, args.levels, dt, args.steps, args.nh)
    truth = exp.run(0)
    config, kept, table = iterative_search(exp, alpha=args.alpha, truth=truth)
    single = {name: exp.error(exp.run(GRIST_ROWS[name]), truth) for name in DEFAULT_ORDER}
    policies = {p: exp.error(exp.run(0, prec=p), truth) for p in ("mix", "mix_dbl_mass", "mix_df")}
    print(json.dumps({"case": {"mesh_level": args.level, "n_levels": args.levels, "nonhydrostatic": args.nh,
                               "dt_s": dt, "steps": args.steps, "alpha": args.alpha},
                      "trials": table, "accepted_rows": kept, "accepted_mask": config,
                      "E_single_row": single, "E_policies": policies}))
    exp.close()


if __name__ == "__main__":
    main()
