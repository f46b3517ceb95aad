#!/usr/bin/env python
"""Throughput of the GRIST hot path on one GB300 (and N independent replicas).

Workload (default ``g9nh``): the mixed-precision non-hydrostatic dycore plus
four tracers on the level-9 icosahedral mesh (2,621,442 cells, 7,864,320
edges, 5,242,880 vertices), 60 levels on a stretched 30 km-top grid, dt =
30 s, seeded jet + perturbation + warm bubble, tracers = bell / slotted
cylinder / 2 Gaussians.  One step = one NH dycore step (which accumulates the
horizontal and vertical mass fluxes and hands dpi to the tracer solver) + one
tracer step of the 4 tracers with those fluxes (horizontal RK3 + FCT, then
the vertical transport).  The FP64 GPU path runs the same step on the
same inputs side by side.

Metric: cell-level-steps/s = n_cells * n_levels * steps / time.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the reference arm), on host cores, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-level-steps/s mixed vs FP64 on 1 GB300 at stated error; HBM GB/s vs peak"
UNIT = "cell-level-steps/s"

WORKLOADS = {
    # name: mesh level, levels, non-hydrostatic, tracers, dt
    "g9nh": dict(level=9, L=60, nh=True, T=4, dt=30.0,
                 phys="NH dycore + 4 tracers (3rd-order + FCT horizontal, adaptively implicit vertical), dt 30 s",
                 desc="NH dycore + 4 tracers (3rd-order + FCT horizontal, adaptively implicit vertical), "
                      "L9 mesh 2621442 cells, 60 levels, dt 30 s"),
    "g8nh": dict(level=8, L=60, nh=True, T=0, dt=60.0, phys="NH dycore, dt 60 s",
                 desc="NH dycore, L8 mesh 655362 cells, 60 levels, dt 60 s"),
    "g6hdc": dict(level=6, L=30, nh=False, T=0, dt=300.0, phys="hydrostatic dycore, dt 300 s",
                  desc="hydrostatic dycore, L6 mesh 40962 cells, 30 levels, dt 300 s"),
}


def algorithmic_bytes(name, nC, nE, nV, L, T, prec):
    """Compulsory bytes of one launch: every array the kernel declares read
    or written once (stencil re-reads, padding and index tables excluded)."""
    base = name.split("/")[0]
    sU = sA = sM = 8
    if prec in ("mix", "mix_dbl_mass", "mix_df"):
        sU = sA = 4
        sM = 8 if prec == "mix_dbl_mass" else 4
    sQ = sC = 8 if prec == "fp64" else 4
    CL, EL, VL, CI = nC * L, nE * L, nV * L, nC * (L + 1)
    table = {
        "k_mass_edge": 2 * nC * 8 + EL * (sU + sM),                       # + accumulation counted below
        "k_mass_col": EL * sM + CL * 8 + 2 * nC * 8 + nC * 8 + CL * sA + CI * 8,
        "k_theta_flux": EL * sM + CL * sA + EL * sA,
        "k_theta_update": EL * sA + CL * sA + CI * 8 + 2 * CL * 8,
        "k_hydro_diag": nC * 8 + CL * 8 + 3 * CL * 8,
        "k_vort": EL * sU + nC * 8 + VL * sA,
        "k_ke": EL * sU + CL * 8,
        # u_s, u_n, F, vertex PV (edge PV formed in the kernel), K, M, 1/sum,
        # p, alpha, layer phi, dp/dpi, u_out
        "k_momentum": 2 * EL * sU + EL * sM + VL * sA + CL * 8 + CI * 8 + nC * 8 + 4 * CL * 8 + EL * sU,
        "k_eos": CL * 8 + CI * 8 + CL * 8,
        "k_nh_explicit": EL * sU + 2 * nC * 8 + CI * 8 + 4 * CI * 8 + CL * 8 + 2 * CI * 8,
        "k_nh_solve": 2 * CI * 8 + CL * 8 + nC * 8 + 2 * CI * 8 + 4 * CL * 8,
        "k_add_scalar": 16,
        "k_vertex_mass": nC * 8 + nV * 8,
        # F, dpi^n -> the {dpi^n, div F} pair (+ the binary32 flux copy)
        "k_tr_div": EL * 8 + CL * 8 + 2 * CL * sC + (EL * 4 if sC == 4 else 0),
        "k_tr_edge": T * CL * sQ + EL * sC + T * EL * sC,
        "k_tr_update": T * EL * sC + T * CL * sQ + 2 * CL * sC + T * CL * sQ,
        # limiter: q^n, F, {dpi, div F} -> local bounds {max, min}(q^n, q^td), div F^L
        "k_tr_lowres": T * CL * sQ + EL * sC + 2 * CL * sC + 2 * T * CL * sC + T * CL * sC,
        # q^n, bounds, A, {dpi, div F} -> {R+, R-}
        "k_tr_ratios": T * CL * sQ + 2 * T * CL * sC + T * EL * sC + 2 * CL * sC + 2 * T * CL * sC,
        # q^n, div F^L, A, {R+, R-}, {dpi, div F} -> q^{n+1} in place
        "k_tr_final": T * CL * sQ + T * CL * sC + T * EL * sC + 2 * T * CL * sC + 2 * CL * sC + T * CL * sQ,
        "k_tr_vertical": 2 * CL * sC + CI * 8 + 2 * T * CL * sQ,
    }
    return table.get(base)


# FP64 work of the kernels of the mixed step that are bound by the FP64 pipe
# (ncu: sm__pipe_fp64_cycles_active 64-92 % of peak, DRAM well below its
# peak): FP64 flops = 2 DFMA + DADD + DMUL executed thread instructions, and
# DRAM bytes (read + write), per unit of work, both counted by ncu on the
# level-7 mesh (163,842 cells, 60 levels) of the same workload and step.
# Units: cell-levels "c", edge-levels "e", vertex-levels "v", cell-interfaces
# (L + 1 per column) "i".  Per-launch figures scale with the units processed.
# Only kernels whose arithmetic is unchanged since their capture are listed
# (the vertex PV, the mass-column prefix and the tracer stage ratios have
# since lost FP64 work; the tracer limiter passes now issue none).
FP64_WORK_MIX = {
    # kernel: (unit, FP64 flop per unit, DRAM bytes per unit)
    "k_nh_solve": ("c", 63.70, 280.8),
    "k_momentum": ("e", 19.88, 36.9),      # DRAM: the capture with the edge PV formed in the kernel
    "k_nh_explicit": ("i", 13.38, 73.4),
    "k_ke": ("c", 18.00, 18.3),
    "k_eos": ("c", 93.0, 21.1),
    "k_tr_div": ("c", 12.00, 31.5),
}

SM_COUNT = 152
DFMA_PER_SM_CLK = 2     # ncu: smsp__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained = 304 / GPU


def fp64_peak_tflops(sm_mhz):
    """FP64 peak from the unit counts and clock: 152 SMs x 2 DFMA per clock
    x 2 flop at the given SM clock."""
    return SM_COUNT * DFMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


# Algorithmic FP64 work of the double-precision terms of the mixed step, per
# unit, counted from the discrete formulas as written (every +, -, *, / one
# flop, a pow one flop; the factoring, reciprocal tables and series the
# kernels use instead are not counted):
#   k_momentum (Eq. 5, FP64 terms of the mixed policy): -(K2 - K1)/dc (2);
#     eta-dot du/deta = [Mb(u+ - u) + Mt(u - u-)]/(2 dpi_e) with the cell
#     means Mb, Mt (2 x (1 add + 1 mul)), two differences, two products, a
#     sum, 2 dpi_e (1 add) and the division (11); -alpha_e (p2 - p1)/dc with
#     alpha_e a cell mean (5); -(dp/dpi)_e (phi2 - phi1)/dc (5 NH; 2 in the
#     hydrostatic core, dp/dpi = 1); the four terms summed (3): 26 NH / 23 HDC
#     per edge-level.
#   k_nh_solve (Eqs. 6, 7, 9 implicit part): dphi** (1), the EOS p** (5),
#     C = gamma p** beta dt g / dphi** (3), a = beta dt g / dpi at the
#     interface with the interface mass a mean (3), the row's diagonal and
#     right-hand side (8), Thomas forward (6) and back (2) sweeps,
#     phi = phi** + beta dt g w (2), the final EOS (6), alpha = dphi/dpi
#     (1), the layer phi (2), dp/dpi at the interface and its layer mean (4):
#     43 per cell-level.
#   k_ke (Eq. 5 KE): sum over 6 edges of (dc dv / 4A) u^2 (3 each): 18 per
#     cell-level.
#   k_nh_explicit (Eqs. 6-7 explicit part, FP64 share): the t^n forcing
#     g ((p_j - p_{j-1}) / dpi_j - 1) (4 + 2 for the interface mass), w** and
#     phi** updates (4 + 3): 13 per interface.
#   k_eos (Eq. 9): dphi, Rd dpi_theta / (p0 dphi) (3), the pow, p0 x: 6 per
#     cell-level.
#   k_mass_col (Eq. 3 column part, FP64 share): the vertical mass flux
#     M = -B dps/dt - sum D (3) and theta = dpi_theta / dpi (1): 4 per
#     cell-level.
#   k_tr_div (tracer continuity, Eq. 10 with the FP64 flux): 6 products and
#     5 sums: 11 per cell-level.
FP64_ALG = {
    "k_momentum": ("e", 26.0, 23.0),
    "k_nh_solve": ("c", 43.0, 43.0),
    "k_ke": ("c", 18.0, 18.0),
    "k_nh_explicit": ("i", 13.0, 13.0),
    "k_eos": ("c", 6.0, 6.0),
    "k_mass_col": ("c", 4.0, 4.0),
    "k_tr_div": ("c", 11.0, 11.0),
}


def measure_fp64_peak(G, torch, device, seconds=0.25):
    """FP64 FMA rate of this GPU from grist_bench_fp64_fma: 16 warps' worth
    of independent FMA chains per SM scheduler slot, timed with CUDA events
    on the launching stream (best of 5 after 3 warm-up launches), with the
    SM clock sampled during the timed launches."""
    blocks, threads = SM_COUNT * 8, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device=device)
    iters = 4096
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # size the launch to about `seconds`
    e0.record(st)
    fl = G.bench_fp64_fma(out, iters, blocks, threads)
    e1.record(st)
    torch.cuda.synchronize()
    iters = max(4096, int(iters * seconds / max(e0.elapsed_time(e1) * 1e-3, 1e-6)))
    for _ in range(3):
        G.bench_fp64_fma(out, iters, blocks, threads)
    cs = ClockSampler(device)
    cs.start()
    best = None
    for _ in range(5):
        e0.record(st)
        fl = G.bench_fp64_fma(out, iters, blocks, threads)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    clocks = cs.stop()
    assert bool(torch.isfinite(out).all())
    tf = fl / best / 1e12
    sm = clocks.get("sm_mhz")
    return {"tflops": round(tf, 4), "launch_ms": round(best * 1e3, 3), "flop_per_launch": fl,
            "sm_mhz": sm, "tflops_per_ghz": round(tf / (sm / 1e3), 4) if sm else None,
            "derived_tflops_at_max_clock": round(fp64_peak_tflops(2070.0), 4),
            "how": "grist_bench_fp64_fma: %d blocks x %d threads x 8 independent FMA chains x %d rounds, "
                   "CUDA events, best of 5" % (blocks, threads, iters)}


def units_of(kind, nC, nE, nV, L):
    return {"c": nC * L, "e": nE * L, "v": nV * L, "i": nC * (L + 1)}[kind]


# ---------------------------------------------------------------------------
# multi-rank aggregation (one process per GPU; each rank times its own K steps)

def reduce_max(x, dist, device):
    """The largest x over all ranks (every rank passes its own; None and a
    single-process run pass through).  device: where the collective's
    tensor lives (the rank's GPU for NCCL, "cpu" for gloo)."""
    if dist is None or x is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, secs_max):
    """Whole-job throughput: the units every rank processed, over the
    slowest rank's time (weak scaling: each rank has the same work)."""
    return world * units_per_rank / secs_max


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "grist_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm

def setup_case(G, torch, wl, seed, device):
    from grist_inputs import states as S
    from grist_inputs.mesh import get_mesh
    m = get_mesh(wl["level"])
    mesh = G.Mesh(m, device=device)
    L, T = wl["L"], wl["T"]
    st = S.dycore_jet_case(m, L, nonhydrostatic=wl["nh"], bubble=wl["nh"], seed=seed)
    q = S.tracer_mixture(m, T, L, np.random.default_rng(seed + 7)) if T else None
    host = {"u": mesh.to_internal(st["u"], "edge"), "ps": mesh.to_internal(st["ps"]),
            "dpi_theta": mesh.to_internal(st["dpi_theta"])}
    if wl["nh"]:
        host["w"] = mesh.to_internal(st["w"])
        host["phi"] = mesh.to_internal(st["phi"])
    if T:
        host["q"] = mesh.to_internal(q, "cell", 1)
    phis = torch.from_numpy(mesh.to_internal(st["phi_s"])).to(device)
    P = G.DycoreParams(L, st["b_int"], st["pi_top"], phis)
    return m, mesh, host, P


def make_state(torch, host, prec, device, nE, nC, L, T, nh):
    fdt = torch.float64 if prec == "fp64" else torch.float32
    s = {"u": torch.from_numpy(host["u"]).to(device=device, dtype=fdt),
         "ps": torch.from_numpy(host["ps"]).to(device),
         "dpi_theta": torch.from_numpy(host["dpi_theta"]).to(device)}
    if nh:
        s["w"] = torch.from_numpy(host["w"]).to(device)
        s["phi"] = torch.from_numpy(host["phi"]).to(device)
        s["p_nh"] = torch.zeros((nC, L), dtype=torch.float64, device=device)   # pressure carried by the state
        s["p_nh_valid"] = False
    if T:
        s["q"] = torch.from_numpy(host["q"]).to(device=device, dtype=fdt)
        s["mass_flux_accum"] = torch.zeros((nE, L), dtype=torch.float64, device=device)
        s["vmass_flux_accum"] = torch.zeros((nC, L + 1), dtype=torch.float64, device=device)
        s["dpi_start"] = torch.zeros((nC, L), dtype=torch.float64, device=device)
    return s


def step(mesh, s, P, wl, prec):
    """One step of the workload: dycore (accumulating the mass flux and
    handing dpi^n to the tracer solver) then the tracers."""
    if "mass_flux_accum" in s:
        s["mass_flux_accum"].zero_()
        s["vmass_flux_accum"].zero_()
    if wl["nh"]:
        mesh.dycore_step_nh(s, P, wl["dt"], prec=prec)
    else:
        mesh.dycore_step_hydro(s, P, wl["dt"], prec=prec)
    if wl["T"]:
        mesh.tracer_step([{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                           "vmass_flux": s["vmass_flux_accum"], "n_levels": wl["L"]}], wl["dt"], prec=prec,
                         limiter=True)


def timed(torch, fn, K, dist=None):
    st = torch.cuda.current_stream()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(K):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3


def gpu_arm(args, wl):
    import torch
    import paper_2404_08849_gb300 as G
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    device = local
    torch.cuda.set_device(device)
    G.load()
    from grist_inputs import states as S
    seed = S.SEED + rank      # each rank: an independent ensemble member
    m, mesh, host, P = setup_case(G, torch, wl, seed, device)
    nC, nE, nV, L, T = mesh.nC, mesh.nE, mesh.nV, wl["L"], wl["T"]
    K, W = args.steps, args.warmup

    tunings = {}
    fp64_peak = None if args.no_fp64_peak else measure_fp64_peak(G, torch, device)
    finals = {}

    side = torch.cuda.Stream(device)   # a created stream: the step graph is captured on it
    launch_mode = {}

    def run_prec(prec, sample_clocks=False):
      with torch.cuda.stream(side):
        s = make_state(torch, host, prec, device, nE, nC, L, T, wl["nh"])
        if args.tracer_tuning:
            mesh.set_tracer_tuning(**json.loads(args.tracer_tuning))
            tunings[prec] = mesh.tracer_tuning()
        for w in range(W):
            step(mesh, s, P, wl, prec)
            if w == 0 and T and not args.no_autotune and not args.tracer_tuning:
                # the tracer launch configuration from the library's autotuner,
                # on this step's own tracer inputs (restored after timing)
                tunings[prec] = mesh.autotune_tracer(
                    [{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                      "vmass_flux": s["vmass_flux_accum"], "n_levels": L}], wl["dt"], prec=prec, steps=2)[0]
        torch.cuda.synchronize()
        # the timed steps: replays of one captured coupled step (the
        # library's whole-step graph), else the calls one by one
        graph = None
        if not args.eager:
            try:
                graph = G.capture(lambda: step(mesh, s, P, wl, prec), side)
            except G.GristError:
                graph = None
        launch_mode[prec] = "CUDA graph of one coupled step, replayed" if graph else "library calls per step"
        cs = ClockSampler(device) if sample_clocks else None
        if cs:
            cs.start()
        secs = timed(torch, (graph.launch if graph else (lambda: step(mesh, s, P, wl, prec))), K, dist)
        clocks = cs.stop() if cs else None
        if graph:
            graph.close()
        status = mesh.last_status()
        # per-kernel event timing over a second pass of K steps
        mesh.profile(True)
        for _ in range(K):
            step(mesh, s, P, wl, prec)
        prof = mesh.profile_read()
        mesh.profile(False)
        # conservation and the end state, for the mixed-vs-FP64 error norms
        dry = mesh.global_sum(G.GRIST_SUM_DRY_MASS, s["ps"], offset=float(P.c.pi_top))[0]
        fin = {"ps": s["ps"].clone(), "dpi_theta": s["dpi_theta"].clone(),
               "vor": mesh.vorticity(s["u"], L), "steps": W + 2 * K}
        if wl["nh"]:
            fin["w"] = s["w"].clone()
        finals[prec] = fin
        del s
        torch.cuda.empty_cache()
        return secs, clocks, prof, status, dry

    dry_start = mesh.global_sum(G.GRIST_SUM_DRY_MASS, torch.from_numpy(host["ps"]).to(device),
                                offset=float(P.c.pi_top))[0]
    secs_mix, clocks, prof_mix, st_mix, dry_mix = run_prec(args.prec, sample_clocks=True)
    secs_64, _, prof_64, st_64, dry_64 = (run_prec("fp64") if not args.no_fp64 else (None, None, {}, 0, None))
    accuracy = None
    if "fp64" in finals and args.prec in finals and args.prec != "fp64":
        accuracy = mixed_vs_fp64(torch, mesh, m, finals[args.prec], finals["fp64"], P, wl, device)
        accuracy["dry_mass_drift"] = {args.prec: (dry_mix - dry_start) / dry_start,
                                      "fp64": (dry_64 - dry_start) / dry_start}
    finals.clear()
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers: every step, the
    # whole model state (u, ps, dpi theta, and for the NH core w, phi and the
    # carried pressure; the tracers) comes in from pinned host memory and
    # goes back.  The tracers' copy in runs on a copy stream while the dycore
    # step runs, the dycore fields' copy out while the tracer step runs; the
    # step ends when all of its outputs are on the host.
    e2e = None
    if not args.no_e2e:
        s = make_state(torch, host, args.prec, device, nE, nC, L, T, wl["nh"])
        dy_keys = ["u", "ps", "dpi_theta"] + (["w", "phi", "p_nh"] if wl["nh"] else [])
        tr_keys = ["q"] if T else []
        pinned = {k: torch.empty(s[k].shape, dtype=s[k].dtype, pin_memory=True).copy_(s[k])
                  for k in dy_keys + tr_keys}
        h2d = sum(v.numel() * v.element_size() for v in pinned.values())
        cstream = torch.cuda.Stream(device)
        carried = {"p": False}   # the host copy of the pressure is valid after the first step

        def e2e_step():
            main = torch.cuda.current_stream()
            cstream.wait_stream(main)
            q_in = None
            if tr_keys:
                with torch.cuda.stream(cstream):
                    s["q"].copy_(pinned["q"], non_blocking=True)
                    q_in = cstream.record_event()
            for k in dy_keys:
                s[k].copy_(pinned[k], non_blocking=True)
            s["p_nh_valid"] = carried["p"]
            if "mass_flux_accum" in s:
                s["mass_flux_accum"].zero_()
                s["vmass_flux_accum"].zero_()
            if wl["nh"]:
                mesh.dycore_step_nh(s, P, wl["dt"], prec=args.prec)
            else:
                mesh.dycore_step_hydro(s, P, wl["dt"], prec=args.prec)
            dy_done = main.record_event()
            with torch.cuda.stream(cstream):
                cstream.wait_event(dy_done)
                for k in dy_keys:
                    pinned[k].copy_(s[k], non_blocking=True)
            if tr_keys:
                main.wait_event(q_in)
                mesh.tracer_step([{"q": s["q"], "dpi": s["dpi_start"], "mass_flux": s["mass_flux_accum"],
                                   "vmass_flux": s["vmass_flux_accum"], "n_levels": L}], wl["dt"],
                                 prec=args.prec, limiter=True)
                pinned["q"].copy_(s["q"], non_blocking=True)
            main.wait_stream(cstream)
            carried["p"] = bool(wl["nh"])
        for _ in range(W):
            e2e_step()
        secs_e2e = reduce_max(timed(torch, e2e_step, K, dist), dist, device)
        e2e = {"value": whole_job_rate(nC * L * K, world, secs_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d),
               "copies": "state in from pinned host memory and out every step; tracers in during the "
                         "dycore step and dycore fields out during the tracer step (copy stream)"}
        del s, pinned

    # max over ranks
    secs_mix = reduce_max(secs_mix, dist, device)
    secs_64 = reduce_max(secs_64, dist, device)

    total_units = world * nC * L * K
    value = whole_job_rate(nC * L * K, world, secs_mix)

    # roofline of the dominant kernel of the mixed step
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    f64_peak = fp64_peak["tflops"] if fp64_peak else fp64_peak_tflops(sm_max)
    f64_src = ("measured: " + fp64_peak["how"]) if fp64_peak else (
        "derived: %d SMs x %d DFMA/clk x 2 flop x %.0f MHz" % (SM_COUNT, DFMA_PER_SM_CLK, sm_max))
    fp64_table = FP64_WORK_MIX if args.prec != "fp64" else {}
    kernels = []
    for name, (launches, ms) in sorted(prof_mix.items(), key=lambda kv: -kv[1][1]):
        b = algorithmic_bytes(name, nC, nE, nV, L, T, args.prec)
        avg = ms / max(launches, 1)
        row = {"kernel": name, "launches": launches, "total_ms": round(ms, 3),
               "avg_ms": round(avg, 4), "share": None,
               "gbs": round(b / (avg * 1e-3) / 1e9, 1) if b else None}
        # FP64 work: algorithmic (formulas) and executed (ncu count of the
        # GRIST_MIX kernels)
        base = name.split("/")[0]
        a = FP64_ALG.get(base)
        if a and args.prec != "fp64":
            fl = (a[1] if wl["nh"] else a[2]) * units_of(a[0], nC, nE, nV, L)
            row["fp64_alg_tflops"] = round(fl / (avg * 1e-3) / 1e12, 4)
        w = fp64_table.get(base) if name.endswith("/mix") else None
        if w:
            row["fp64_exec_tflops"] = round(w[1] * units_of(w[0], nC, nE, nV, L) / (avg * 1e-3) / 1e12, 4)
        kernels.append(row)
    tot = sum(k["total_ms"] for k in kernels) or 1.0
    for k in kernels:
        k["share"] = round(k["total_ms"] / tot, 4)
    dom = kernels[0] if kernels else None
    roofline = None
    if dom:
        hbm_ctx = ({"achieved": dom["gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(dom["gbs"] / hbm_peak, 4), "peak_source": peak_src}
                   if dom["gbs"] is not None else None)
        w = fp64_table.get(dom["kernel"].split("/")[0]) if dom["kernel"].endswith("/mix") else None
        a = FP64_ALG.get(dom["kernel"].split("/")[0]) if args.prec != "fp64" else None
        if a and "fp64_alg_tflops" in dom:
            units = units_of(a[0], nC, nE, nV, L)
            per_unit = a[1] if wl["nh"] else a[2]
            roofline = {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["fp64_alg_tflops"],
                        "peak": round(f64_peak, 4), "unit": "TFLOP/s",
                        "frac": round(dom["fp64_alg_tflops"] / f64_peak, 4),
                        "traffic": (int(w[2] * units) if w and w[2] is not None else None),
                        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per unit on the "
                                          "level-7 case, times this launch's units",
                        "algorithmic_bytes": algorithmic_bytes(dom["kernel"], nC, nE, nV, L, T, args.prec),
                        "work": "algorithmic FP64 flop per launch %.4g (%.1f per unit, from the formulas)%s" % (
                            per_unit * units, per_unit,
                            ("; executed %.1f per unit (ncu), %.4g TFLOP/s executed" % (w[1], dom["fp64_exec_tflops"]))
                            if w else ""),
                        "peak_source": f64_src, "hbm": hbm_ctx}
        elif hbm_ctx:
            roofline = dict({"bound": "hbm", "kernel": dom["kernel"], "traffic": None}, **hbm_ctx)
    launches_per_step = sum(k["launches"] for k in kernels) / max(K, 1)

    # time splitting: n dycore steps accumulate the mean mass flux
    # (accum_scale = 1/n), then one tracer step of n dycore time steps
    split = None
    if T and args.split > 1:
        n = args.split
        s = make_state(torch, host, args.prec, device, nE, nC, L, T, wl["nh"])
        s["accum_scale"] = 1.0 / n
        dpi0 = s.pop("dpi_start")

        def window():
            s["mass_flux_accum"].zero_()
            s["vmass_flux_accum"].zero_()
            for i in range(n):
                s["dpi_start"] = dpi0 if i == 0 else None
                if wl["nh"]:
                    mesh.dycore_step_nh(s, P, wl["dt"], prec=args.prec)
                else:
                    mesh.dycore_step_hydro(s, P, wl["dt"], prec=args.prec)
            mesh.tracer_step([{"q": s["q"], "dpi": dpi0, "mass_flux": s["mass_flux_accum"],
                               "vmass_flux": s["vmass_flux_accum"], "n_levels": L}], n * wl["dt"], prec=args.prec,
                             limiter=True)
        for _ in range(max(1, W // n)):
            window()
        secs_w = reduce_max(timed(torch, window, K, dist), dist, device)
        split = {"dycore_steps_per_tracer_step": n, "tracer_dt_s": n * wl["dt"],
                 "value": whole_job_rate(nC * L * n * K, world, secs_w), "unit": UNIT + " (dycore steps)",
                 "ms_per_window": secs_w / K * 1e3, "status_flags": mesh.last_status()}
        del s, dpi0
        torch.cuda.empty_cache()

    mesh.close()
    del mesh
    torch.cuda.empty_cache()
    batched = None if args.no_batched else batched_ensemble(G, torch, device, args, dist)
    secondary = None
    if not args.no_secondary and args.workload == "g9nh" and args.mesh_level is None:
        secondary = [secondary_line(G, torch, name, args, device, dist) for name in ("g6hdc", "g8nh")]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, level=args.cpu_level, steps=args.cpu_steps)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
               "ms_per_step": secs_mix / K * 1e3, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "mixed f32/f64" if args.prec != "fp64" else "f64",
               "data": "synthetic (seeded jet + perturbation + warm bubble, tracer mixture)",
               "config": {"workload": wl["desc"], "precision": args.prec, "n_cells": nC, "n_edges": nE,
                          "launch": launch_mode,
                          "n_levels": L, "n_tracers": T, "dt_s": wl["dt"],
                          "l2_policy": "inputs larger than L2 (state >> 129 MB), no flush",
                          "tracer_tuning": tunings or "library default",
                          "parallelism": "independent ensemble member per GPU" if world > 1 else "single GPU"},
               "fp64": ({"value": total_units / secs_64, "ms_per_step": secs_64 / K * 1e3,
                         "speedup_mix_over_fp64": secs_64 / secs_mix} if secs_64 else None),
               "roofline": roofline, "kernels": kernels, "gpu_launches": int(round(launches_per_step * K)),
               "batched_ensemble": batched, "split_coupling": split,
               "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "fp64_peak": fp64_peak,
               "accuracy_vs_fp64": accuracy, "secondary": secondary,
               "status_flags": {"mix": st_mix, "fp64": st_64},
               "dry_mass_end": {"mix": dry_mix, "fp64": dry_64}}
        print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def norms_dev(torch, x, ref, w):
    """Normalised (l1, l2, linf) of x against ref on the device in float64
    (Eq. 2 read as the Williamson norms: I|x - r| / I|r|,
    sqrt(I(x - r)^2 / I r^2), max|x - r| / max|r|; I the weighted sum)."""
    d = x - ref
    l1 = (w * d.abs()).sum() / (w * ref.abs()).sum()
    l2 = torch.sqrt((w * d * d).sum() / (w * ref * ref).sum())
    linf = d.abs().max() / ref.abs().max()
    return [float(l1), float(l2), float(linf)]


def mixed_vs_fp64(torch, mesh, m, mix, ref, P, wl, device):
    """Error of the mixed run's end state against the FP64 GPU run's (same
    inputs, same number of steps; the FP64 path matches the oracle to 1e-12
    per step): normalised l1/l2/linf of the surface pressure, the relative
    vorticity, theta and w, and the paper's E = max(L(ps), L(vor)) (Eqs. 1-2)
    against its acceptance threshold 0.05."""
    ca = torch.from_numpy(mesh.to_internal(m["cell_area"])).to(device)
    va = torch.from_numpy(mesh.to_internal(m["vertex_area"], "vertex")).to(device)
    b = torch.from_numpy(np.asarray(P.b, np.float64)).to(device)
    db = b[1:] - b[:-1]
    pit = float(P.c.pi_top)

    def theta(f):
        dpi = (f["ps"] - pit)[:, None] * db[None, :]
        return f["dpi_theta"] / dpi, dpi
    th_m, _ = theta(mix)
    th_r, dpi_r = theta(ref)
    out = {"steps": mix["steps"], "simulated_s": mix["steps"] * wl["dt"],
           "ps": norms_dev(torch, mix["ps"], ref["ps"], ca),
           "vorticity": norms_dev(torch, mix["vor"], ref["vor"], va[:, None]),
           "theta": norms_dev(torch, th_m, th_r, ca[:, None] * dpi_r)}
    if "w" in mix:
        out["w"] = norms_dev(torch, mix["w"], ref["w"], ca[:, None])
    E = max(max(out["ps"]), max(out["vorticity"]))
    out["E"] = E
    out["E_le_alpha_0.05"] = bool(E <= 0.05)
    return out


def secondary_line(G, torch, name, args, device, dist):
    """A further benchmark configuration (hydrostatic L6 or non-hydrostatic
    L8 dycore): the mixed and the FP64 step side by side, W untimed and K
    timed steps each, inputs resident on the device."""
    wl = WORKLOADS[name]
    from grist_inputs import states as S
    m, mesh, host, P = setup_case(G, torch, wl, S.SEED, device)
    nC, nE, L = mesh.nC, mesh.nE, wl["L"]
    res = {"workload": wl["desc"], "unit": UNIT}
    side = torch.cuda.Stream(device)
    for prec in (args.prec, "fp64"):
      with torch.cuda.stream(side):
        s = make_state(torch, host, prec, device, nE, nC, L, 0, wl["nh"])
        for _ in range(args.warmup):
            step(mesh, s, P, wl, prec)
        secs_e = reduce_max(timed(torch, lambda: step(mesh, s, P, wl, prec), args.steps, dist), dist, device)
        graph = None if args.eager else G.capture(lambda: step(mesh, s, P, wl, prec), side)
        secs = (reduce_max(timed(torch, graph.launch, args.steps, dist), dist, device) if graph else secs_e)
        if graph:
            graph.close()
        res[prec] = {"ms_per_step": secs / args.steps * 1e3, "value": nC * L * args.steps / secs,
                     "eager_ms_per_step": secs_e / args.steps * 1e3,
                     "launch": "CUDA graph of one step" if graph else "library calls per step",
                     "status_flags": mesh.last_status()}
        del s
        torch.cuda.empty_cache()
    res["speedup_mix_over_fp64"] = res["fp64"]["ms_per_step"] / res[args.prec]["ms_per_step"]
    mesh.close()
    return res


def batched_ensemble(G, torch, device, args, dist):
    """Uneven ensemble of tracer sets on the level-7 mesh (163,842 cells):
    16 members with tracer counts from {1, 4, 10, 25} and level counts from
    {30, 60}, seeded deformational non-divergent winds (amplitude +-20%),
    FP32 tracers with FCT, all members advanced by one call per step; the
    launch configuration comes from the library's autotuner.  Unit:
    tracer-cell-level-steps/s summed over members."""
    from grist_inputs import states as S
    from grist_inputs.mesh import get_mesh
    rank = int(os.environ.get("RANK", "0"))
    m = get_mesh(7)
    mesh = G.Mesh(m, device=device)
    members, dt = S.ensemble_members(m, n_members=16, seed=S.SEED + 1000 * rank)
    dev = []
    units = 0
    for mb in members:
        dev.append({"q": torch.from_numpy(mesh.to_internal(mb["q"], "cell", 1)).to(device=device,
                                                                                 dtype=torch.float32),
                    "dpi": torch.from_numpy(mesh.to_internal(mb["dpi"])).to(device),
                    "mass_flux": torch.from_numpy(mesh.to_internal(mb["mass_flux"], "edge")).to(device),
                    "n_levels": mb["n_levels"]})
        units += mb["n_tracers"] * mb["n_levels"] * mesh.nC
    tuning, tune_ms = mesh.autotune_tracer(dev, dt, prec="mix", steps=3)
    for _ in range(args.warmup):
        mesh.tracer_step(dev, dt, prec="mix")
    secs = timed(torch, lambda: mesh.tracer_step(dev, dt, prec="mix"), args.steps, dist)
    mass = [mesh.global_sum(G.GRIST_SUM_TRACER_MASS, d["q"][0], d["dpi"], n_levels=d["n_levels"])[0]
            for d in dev[:2]]
    status = mesh.last_status()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    secs = reduce_max(secs, dist, device)
    out = {"workload": "16-member uneven tracer ensemble, L7 mesh 163842 cells, T in {1,4,10,25}, "
                       "L in {30,60}, FP32 tracers + FCT, dt %.1f s" % dt,
           "value": whole_job_rate(units * args.steps, world, secs), "unit": "tracer-cell-level-steps/s",
           "ms_per_step": secs / args.steps * 1e3, "tuning": tuning, "autotune_ms_per_step": tune_ms,
           "members": [[mb["n_tracers"], mb["n_levels"]] for mb in members], "status_flags": status}
    mesh.close()
    del dev
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)

class OracleCase:
    """The workload's physics on a given mesh level for the FP64 CPU oracle:
    mesh, state and parameters built once; step() advances one coupled step
    (dycore accumulating the horizontal and vertical mass fluxes, then the
    tracers' horizontal and vertical transport) and times only that."""

    def __init__(self, wl, level):
        import oracle as O
        from grist_inputs import states as S
        from grist_inputs.mesh import get_mesh
        self.O, self.wl = O, wl
        self.m = m = get_mesh(level)
        self.M = O.Mesh(m)
        self.L, self.T = wl["L"], wl["T"]
        self.st = S.dycore_jet_case(m, self.L, nonhydrostatic=wl["nh"], bubble=wl["nh"])
        self.P = O.Params(self.L, self.st["b_int"], self.st["pi_top"], self.st["phi_s"])
        self.q = S.tracer_mixture(m, self.T, self.L, np.random.default_rng(S.SEED + 7)) if self.T else None
        self.s = dict(self.st)
        self.level = level
        self.units = m["n_cells"] * self.L

    def step(self):
        """One oracle step; returns its wall time in seconds."""
        O, wl, m, L, st = self.O, self.wl, self.m, self.L, self.st
        s = self.s
        t0 = time.perf_counter()
        fa = np.zeros((m["n_edges"], L))
        va = np.zeros((m["n_cells"], L + 1))
        if wl["nh"]:
            s2 = O.dycore_step_nh(self.M, self.P, s, wl["dt"], flux_accum=fa, vflux_accum=va)
        else:
            s2 = O.dycore_step_hydro(self.M, self.P, s, wl["dt"], flux_accum=fa, vflux_accum=va)
        if self.T:
            pint = st["pi_top"] + st["b_int"][None, :] * (s["ps"][:, None] - st["pi_top"])
            dpi = np.diff(pint, axis=1)
            q = O.tracer_step(self.M, self.q, dpi, fa, wl["dt"])
            self.q = O.tracer_vertical_step(q, dpi - wl["dt"] * O.divergence(self.M, fa), va, wl["dt"], 1.0)
        self.s = dict(s, **{k: s2[k] for k in s2 if k != "accum_weight"})
        return time.perf_counter() - t0

    def sample(self, steps):
        return "%d step(s) of the same %s physics on the level-%d mesh (%d cells x %d levels), timed per step " \
               "(mesh and state built once, outside the timing)" % (
                   steps, "NH dycore + %d tracers" % self.T if self.wl["nh"] else "HDC", self.level,
                   self.m["n_cells"], self.L)


def cpu_baseline(wl, level, steps=1):
    c = OracleCase(wl, level)
    secs = sum(c.step() for _ in range(steps))
    return {"value": c.units * steps / secs, "unit": UNIT, "cores": c.O.num_threads(), "kind": "oracle",
            "sample": c.sample(steps), "ms_per_step": secs / steps * 1e3}


def reference_arm(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = OracleCase(wl, args.ref_level)
    for _ in range(args.warmup):
        c.step()
    secs = sum(c.step() for _ in range(args.steps))
    value = c.units * args.steps / secs
    sample = c.sample(args.steps)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "%s; timed on a bounded sample: the level-%d mesh (%d cells), %d levels" % (
                       wl["phys"], c.level, c.m["n_cells"], c.L),
                   "full_workload": wl["desc"], "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": c.O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="g9nh", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mix", choices=["mix", "mix_dbl_mass", "mix_df", "fp64"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default tracer launch configuration")
    ap.add_argument("--tracer-tuning", default=None,
                    help="tracer launch configuration as JSON (keys of Mesh.set_tracer_tuning), no autotuning")
    ap.add_argument("--no-fp64-peak", action="store_true", help="skip the FP64 FMA-rate measurement")
    ap.add_argument("--no-secondary", action="store_true", help="skip the L6 hydrostatic and L8 NH lines")
    ap.add_argument("--eager", action="store_true",
                    help="time the library calls step by step instead of a captured step graph")
    ap.add_argument("--split", type=int, default=3,
                    help="dycore steps per tracer step of the time-splitting measurement (1 = skip it)")
    ap.add_argument("--mesh-level", type=int, default=None,
                    help="override the workload's mesh level (small cases for profiling)")
    ap.add_argument("--cpu-level", type=int, default=8)
    ap.add_argument("--cpu-steps", type=int, default=1,
                    help="oracle steps of the cpu_baseline sample (4 at --cpu-level 9 is the level-9 subset)")
    ap.add_argument("--ref-level", type=int, default=7)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    os.environ.setdefault("GRIST_MESH_CACHE", "/tmp/grist_mesh_cache")
    wl = dict(WORKLOADS[args.workload])
    if args.mesh_level is not None:
        wl["level"] = args.mesh_level
        wl["desc"] = wl["phys"] + ", level-%d mesh (profiling case)" % args.mesh_level
    if args.impl == "reference":
        reference_arm(args, wl)
    else:
        gpu_arm(args, wl)


if __name__ == "__main__":
    main()
