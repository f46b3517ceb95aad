"""FP64 CPU oracle of the GRIST hot path - TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  The CUDA library
never calls it and shares no code with it; the two meet only on the mesh
tables and seeded inputs produced by ``grist_inputs``.

The arithmetic lives in ``grist_oracle.c`` (plain scalar C, FP64,
``-O2 -ffp-contract=off``, OpenMP only over independent entity loops).  This
module compiles it with gcc on first use, loads it with ctypes and wraps
each entry point for NumPy arrays in the generator's original numbering.

Also here, in NumPy: the paper's error metric (Eqs. 1-2; Sec. 2.2),
normalised l1 / l2 / linf norms against an FP64 reference.

Parity: every oracle function is pinned by tests against closed forms,
invariants or library routines; the whole-dycore trajectory has no true
solution to compare with and is pinned only through its invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grist_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


_P = ctypes.POINTER
_D = ctypes.c_double
_I = ctypes.c_int32


class OrcMesh(ctypes.Structure):
    _fields_ = [("nC", _I), ("nE", _I), ("nV", _I), ("radius", _D),
                ("cell_area", _P(_D)), ("vertex_area", _P(_D)), ("dc", _P(_D)), ("dv", _P(_D)),
                ("f_vertex", _P(_D)),
                ("cells_on_edge", _P(_I)), ("vertices_on_edge", _P(_I)), ("n_edges_on_cell", _P(_I)),
                ("edges_on_cell", _P(_I)), ("cells_on_cell", _P(_I)), ("edges_on_vertex", _P(_I)),
                ("cells_on_vertex", _P(_I)),
                ("edge_sign_on_cell", _P(_D)), ("edge_sign_on_vertex", _P(_D)), ("kite_area", _P(_D)),
                ("n_edges_on_edge", _P(_I)), ("edges_on_edge", _P(_I)), ("trisk_weight", _P(_D)),
                ("d2_stencil", _P(_I)), ("d2_coef", _P(_D))]


class OrcParams(ctypes.Structure):
    _fields_ = [("L", _I), ("pi_top", _D), ("p0", _D), ("rd", _D), ("cp", _D), ("g", _D),
                ("beta", _D), ("b_int", _P(_D)), ("phi_s", _P(_D))]


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(_D))


def _ip(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(_I))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Mesh:
    """ctypes view of a mesh dict from ``grist_inputs.mesh.build_mesh``."""

    def __init__(self, m):
        self.m = m
        self.nC, self.nE, self.nV = m["n_cells"], m["n_edges"], m["n_vertices"]
        self._keep = {k: m[k] for k in m if isinstance(m[k], np.ndarray)}
        s = OrcMesh()
        s.nC, s.nE, s.nV, s.radius = self.nC, self.nE, self.nV, m["radius"]
        for name, key in [("cell_area", "cell_area"), ("vertex_area", "vertex_area"), ("dc", "edge_dc"),
                          ("dv", "edge_dv"), ("f_vertex", "f_vertex"), ("edge_sign_on_cell", "edge_sign_on_cell"),
                          ("edge_sign_on_vertex", "edge_sign_on_vertex"), ("kite_area", "kite_area"),
                          ("trisk_weight", "trisk_weight"), ("d2_coef", "d2_coef")]:
            setattr(s, name, _dp(m[key]))
        for name in ["cells_on_edge", "vertices_on_edge", "n_edges_on_cell", "edges_on_cell", "cells_on_cell",
                     "edges_on_vertex", "cells_on_vertex", "n_edges_on_edge", "edges_on_edge", "d2_stencil"]:
            setattr(s, name, _ip(m[name]))
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


class Params:
    """Dycore constants (one struct; the same values cross the CUDA ABI)."""

    def __init__(self, n_levels, b_int, pi_top, phi_s, p0=1.0e5, rd=287.04, cp=1004.64, g=9.80616,
                 beta=0.55):
        self.b_int = _f64(b_int)
        self.phi_s = _f64(phi_s)
        s = OrcParams()
        s.L, s.pi_top, s.p0, s.rd, s.cp, s.g, s.beta = n_levels, pi_top, p0, rd, cp, g, beta
        s.b_int, s.phi_s = _dp(self.b_int), _dp(self.phi_s)
        self.s = s
        self.L = n_levels

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _setup():
    L = lib()
    M = _P(OrcMesh)
    Pp = _P(OrcParams)
    pd = _P(_D)
    sig = {
        "orc_divergence": [M, _I, pd, pd],
        "orc_gradient": [M, _I, pd, pd],
        "orc_vorticity": [M, _I, pd, pd],
        "orc_cell_to_vertex": [M, _I, pd, pd],
        "orc_kinetic_energy": [M, _I, pd, pd],
        "orc_perp_flux": [M, _I, pd, pd],
        "orc_pv_flux": [M, _I, pd, pd, pd],
        "orc_edge_flux_3rd": [M, _I, pd, pd, _D, pd],
        "orc_tracer_step": [M, _I, _I, pd, pd, pd, _D, _D, _I],
        "orc_mass": [M, Pp, pd, pd, pd, pd, pd, pd, pd],
        "orc_theta_tend": [M, _I, pd, pd, pd, pd, _D, pd],
        "orc_hydro_diag": [Pp, _I, pd, pd, pd, pd, pd, pd],
        "orc_eos": [Pp, _I, pd, pd, pd],
        "orc_momentum_tend": [M, _I, pd, pd, pd, pd, pd, pd, pd, pd, pd],
        "orc_dycore_step_hydro": [M, Pp, pd, pd, pd, pd, pd, pd, _D],
        "orc_tracer_vertical": [_I, _I, _I, pd, pd, pd, _D, _D],
        "orc_interface_hadv": [M, _I, pd, pd, pd],
        "orc_interface_vadv": [_I, _I, pd, pd, pd, pd],
        "orc_thomas": [_I, pd, pd, pd, pd, pd],
        "orc_dpdpi_layer": [_I, _I, pd, pd, pd],
        "orc_vertical_solve": [Pp, _I, pd, pd, pd, pd, _D, pd, pd, pd],
        "orc_dycore_step_nh": [M, Pp, pd, pd, pd, pd, pd, pd, pd, pd, _D],
        "orc_compensated_sum": [ctypes.c_int64, pd, pd, pd],
        "orc_dry_mass": [M, pd, _D, pd],
        "orc_tracer_mass": [M, _I, pd, pd, pd],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = None
    L.orc_num_threads.restype = ctypes.c_int
    return L


_fns = None


def _f():
    global _fns
    if _fns is None:
        _fns = _setup()
    return _fns


def num_threads() -> int:
    return int(_f().orc_num_threads())


# ---------------------------------------------------------------------------
# operator wrappers (shape [entity][L])
# ---------------------------------------------------------------------------

def _lev(a):
    return a.shape[1] if a.ndim == 2 else 1


def divergence(M: Mesh, F):
    F = _f64(F); L = _lev(F)
    out = np.empty((M.nC, L))
    _f().orc_divergence(M.ref, L, _dp(F), _dp(out))
    return out


def gradient(M: Mesh, h):
    h = _f64(h); L = _lev(h)
    out = np.empty((M.nE, L))
    _f().orc_gradient(M.ref, L, _dp(h), _dp(out))
    return out


def vorticity(M: Mesh, u):
    u = _f64(u); L = _lev(u)
    out = np.empty((M.nV, L))
    _f().orc_vorticity(M.ref, L, _dp(u), _dp(out))
    return out


def cell_to_vertex(M: Mesh, x):
    x = _f64(x); L = _lev(x)
    out = np.empty((M.nV, L))
    _f().orc_cell_to_vertex(M.ref, L, _dp(x), _dp(out))
    return out


def kinetic_energy(M: Mesh, u):
    u = _f64(u); L = _lev(u)
    out = np.empty((M.nC, L))
    _f().orc_kinetic_energy(M.ref, L, _dp(u), _dp(out))
    return out


def perp_flux(M: Mesh, F):
    F = _f64(F); L = _lev(F)
    out = np.empty((M.nE, L))
    _f().orc_perp_flux(M.ref, L, _dp(F), _dp(out))
    return out


def pv_flux(M: Mesh, F, qv):
    F = _f64(F); qv = _f64(qv); L = _lev(F)
    out = np.empty((M.nE, L))
    _f().orc_pv_flux(M.ref, L, _dp(F), _dp(qv), _dp(out))
    return out


def edge_flux_3rd(M: Mesh, q, F, beta=1.0):
    q = _f64(q); F = _f64(F); L = _lev(q)
    out = np.empty((M.nE, L))
    _f().orc_edge_flux_3rd(M.ref, L, _dp(q), _dp(F), beta, _dp(out))
    return out


def tracer_step(M: Mesh, q, dpi, F, dt, beta=1.0, fct=True):
    """One RK3 (+FCT) tracer step; q [T][nC][L] is copied, returned new."""
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    T, nC, L = q.shape
    _f().orc_tracer_step(M.ref, L, T, _dp(q), _dp(_f64(dpi)), _dp(_f64(F)), dt, beta, 1 if fct else 0)
    return q


def tracer_vertical_step(q, dpi, Mv, dt, cmax=1.0):
    """Vertical transport delta(M q) of Eq. 10 (adaptively implicit upwind,
    see orc_tracer_vertical); q [T][nC][L] copied and returned, dpi [nC][L]
    the layer mass at the start, Mv [nC][L+1] the vertical mass flux."""
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    T, nC, L = q.shape
    _f().orc_tracer_vertical(nC, L, T, _dp(q), _dp(_f64(dpi)), _dp(_f64(Mv)), dt, cmax)
    return q


def mass(M: Mesh, P: Params, ps, u):
    L = P.L
    dpi = np.empty((M.nC, L)); F = np.empty((M.nE, L)); D = np.empty((M.nC, L))
    pst = np.empty(M.nC); Mv = np.empty((M.nC, L + 1))
    _f().orc_mass(M.ref, P.ref, _dp(_f64(ps)), _dp(_f64(u)), _dp(dpi), _dp(F), _dp(D), _dp(pst), _dp(Mv))
    return {"dpi": dpi, "F": F, "D": D, "ps_tend": pst, "M": Mv}


def theta_tend(M: Mesh, L, dpi_theta, dpi, F, Mv, beta=1.0):
    out = np.empty((M.nC, L))
    _f().orc_theta_tend(M.ref, L, _dp(_f64(dpi_theta)), _dp(_f64(dpi)), _dp(_f64(F)), _dp(_f64(Mv)), beta,
                        _dp(out))
    return out


def hydro_diag(P: Params, ps, dpi_theta):
    nC = ps.shape[0]; L = P.L
    p = np.empty((nC, L)); al = np.empty((nC, L)); phl = np.empty((nC, L)); phi = np.empty((nC, L + 1))
    _f().orc_hydro_diag(P.ref, nC, _dp(_f64(ps)), _dp(_f64(dpi_theta)), _dp(p), _dp(al), _dp(phl), _dp(phi))
    return {"p": p, "alpha": al, "phi_layer": phl, "phi_int": phi}


def eos(P: Params, dpi_theta, phi):
    nC = dpi_theta.shape[0]
    p = np.empty((nC, P.L))
    _f().orc_eos(P.ref, nC, _dp(_f64(dpi_theta)), _dp(_f64(phi)), _dp(p))
    return p


def momentum_tend(M: Mesh, L, u, dpi, F, Mv, p, alpha, phi_layer, dpdpi=None):
    out = np.empty((M.nE, L))
    dpp = _dp(_f64(dpdpi)) if dpdpi is not None else None
    _f().orc_momentum_tend(M.ref, L, _dp(_f64(u)), _dp(_f64(dpi)), _dp(_f64(F)), _dp(_f64(Mv)), _dp(_f64(p)),
                           _dp(_f64(alpha)), _dp(_f64(phi_layer)), dpp, _dp(out))
    return out


def dycore_step_hydro(M: Mesh, P: Params, state, dt, flux_accum=None, vflux_accum=None):
    """One HDC step; state dict with ps, u, dpi_theta (copied, returned).
    flux_accum [nE][L] / vflux_accum [nC][L+1]: the final stage's horizontal
    / vertical mass flux is added in place."""
    ps = np.array(state["ps"], np.float64, copy=True)
    u = np.array(state["u"], np.float64, copy=True)
    th = np.array(state["dpi_theta"], np.float64, copy=True)
    wgt = np.zeros(1)
    fa = flux_accum if flux_accum is not None else None
    va = vflux_accum if vflux_accum is not None else None
    _f().orc_dycore_step_hydro(M.ref, P.ref, _dp(ps), _dp(u), _dp(th), _dp(fa) if fa is not None else None,
                               _dp(va) if va is not None else None, _dp(wgt), dt)
    return {"ps": ps, "u": u, "dpi_theta": th, "accum_weight": float(wgt[0])}


def interface_hadv(M: Mesh, L, u, x):
    out = np.empty((M.nC, L + 1))
    _f().orc_interface_hadv(M.ref, L, _dp(_f64(u)), _dp(_f64(x)), _dp(out))
    return out


def interface_vadv(L, Mv, dpi, x):
    nC = x.shape[0]
    out = np.empty((nC, L + 1))
    _f().orc_interface_vadv(nC, L, _dp(_f64(Mv)), _dp(_f64(dpi)), _dp(_f64(x)), _dp(out))
    return out


def thomas(a, b, c, d):
    n = len(b)
    x = np.empty(n)
    _f().orc_thomas(n, _dp(_f64(a)), _dp(_f64(b)), _dp(_f64(c)), _dp(_f64(d)), _dp(x))
    return x


def vertical_solve(P: Params, w_star, phi_star, dpi_theta, dpi, dts):
    nC = w_star.shape[0]; L = P.L
    w = np.empty((nC, L + 1)); phi = np.empty((nC, L + 1)); p = np.empty((nC, L))
    _f().orc_vertical_solve(P.ref, nC, _dp(_f64(w_star)), _dp(_f64(phi_star)), _dp(_f64(dpi_theta)),
                            _dp(_f64(dpi)), dts, _dp(w), _dp(phi), _dp(p))
    return w, phi, p


def dpdpi_layer(p, dpi):
    """dp/dpi averaged to layers (the L operator of Eq. 5): p, dpi [nC][L]."""
    p = _f64(p); nC, L = p.shape
    out = np.empty((nC, L))
    _f().orc_dpdpi_layer(nC, L, _dp(p), _dp(_f64(dpi)), _dp(out))
    return out


def dycore_step_nh(M: Mesh, P: Params, state, dt, flux_accum=None, vflux_accum=None):
    """One NDC step; state dict with ps, u, dpi_theta, w, phi (copied)."""
    ps = np.array(state["ps"], np.float64, copy=True)
    u = np.array(state["u"], np.float64, copy=True)
    th = np.array(state["dpi_theta"], np.float64, copy=True)
    w = np.array(state["w"], np.float64, copy=True)
    phi = np.array(state["phi"], np.float64, copy=True)
    wgt = np.zeros(1)
    fa = flux_accum if flux_accum is not None else None
    va = vflux_accum if vflux_accum is not None else None
    _f().orc_dycore_step_nh(M.ref, P.ref, _dp(ps), _dp(u), _dp(th), _dp(w), _dp(phi),
                            _dp(fa) if fa is not None else None, _dp(va) if va is not None else None, _dp(wgt), dt)
    return {"ps": ps, "u": u, "dpi_theta": th, "w": w, "phi": phi, "accum_weight": float(wgt[0])}


def compensated_sum(x, w=None):
    x = _f64(np.ravel(x))
    out = np.empty(2)
    _f().orc_compensated_sum(x.size, _dp(x), _dp(_f64(np.ravel(w))) if w is not None else None, _dp(out))
    return out


def dry_mass(M: Mesh, ps, pi_top):
    out = np.empty(2)
    _f().orc_dry_mass(M.ref, _dp(_f64(ps)), pi_top, _dp(out))
    return out


def tracer_mass(M: Mesh, q, dpi):
    q = _f64(q); L = q.shape[1]
    out = np.empty(2)
    _f().orc_tracer_mass(M.ref, L, _dp(q), _dp(_f64(dpi)), _dp(out))
    return out


# ---------------------------------------------------------------------------
# error metric (Eqs. 1-2, Sec. 2.2)
# ---------------------------------------------------------------------------

def error_norms(x, ref, weight):
    """Normalised l1, l2, linf of x against ref with area (x mass) weights:
    l1 = I|x - r| / I|r|,  l2 = sqrt(I (x - r)^2 / I r^2),
    linf = max|x - r| / max|r|; I = weighted global sum."""
    x = np.asarray(x, np.float64); ref = np.asarray(ref, np.float64)
    wgt = np.broadcast_to(np.asarray(weight, np.float64).reshape(
        weight.shape + (1,) * (x.ndim - np.ndim(weight))), x.shape)
    d = x - ref
    l1 = np.sum(wgt * np.abs(d)) / np.sum(wgt * np.abs(ref))
    l2 = np.sqrt(np.sum(wgt * d * d) / np.sum(wgt * ref * ref))
    linf = np.max(np.abs(d)) / np.max(np.abs(ref))
    return float(l1), float(l2), float(linf)


def error_level(x, ref, weight):
    """L(x) = max(l1, l2, linf) of Eq. 2."""
    return max(error_norms(x, ref, weight))


def max_rel_diff(x, ref):
    """max|x - ref| / max|ref| (per-field parity measure)."""
    x = np.asarray(x, np.float64); ref = np.asarray(ref, np.float64)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))
