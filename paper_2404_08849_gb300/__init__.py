"""GB300 (sm_103a) GRIST hot-path library - Python binding.

Thin wrapper over the C ABI of ``libgrist_gb300.so`` (``include/grist.h``):
it marshals NumPy mesh tables and PyTorch device tensors (pointers, sizes,
the current CUDA stream) into the C structs and raises on a non-zero status.
All computation runs in the library's CUDA kernels; there is no CPU path.

Numbering: the library renumbers cells / edges / vertices along a
space-filling curve.  ``Mesh.to_internal`` / ``Mesh.from_internal`` permute
host arrays between the generator's numbering and the internal one.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (GRIST_FLAG_NONFINITE, GRIST_FLAG_TIMEOUT, GRIST_FP64, GRIST_MIX, GRIST_MIX_DBL_MASS, GRIST_MIX_DF,
                   GRIST_ROW_ALL,
                   GRIST_ROWS, GRIST_SUM_AREA_WEIGHTED, GRIST_SUM_DRY_MASS, GRIST_SUM_TRACER_MASS, GristError)

__all__ = ["Mesh", "DycoreParams", "GRIST_FP64", "GRIST_MIX", "GRIST_MIX_DBL_MASS", "GRIST_MIX_DF", "GristError",
           "GRIST_SUM_DRY_MASS", "GRIST_SUM_TRACER_MASS", "GRIST_SUM_AREA_WEIGHTED", "load",
           "GRIST_FLAG_NONFINITE", "GRIST_FLAG_TIMEOUT", "GRIST_ROWS", "GRIST_ROW_ALL"]

PREC = {"fp64": GRIST_FP64, "mix": GRIST_MIX, "mix_dbl_mass": GRIST_MIX_DBL_MASS, "mix_df": GRIST_MIX_DF}


def load():
    return _lib.load()


def _ptr(t):
    return ctypes.c_void_p(int(t.data_ptr())) if t is not None else None


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def selftest_conversions(n_random=1 << 28, seed=2404_08849):
    """grist_selftest_conversions: the library's integer binary32 <->
    binary64 conversions against the hardware ones on the current device.
    Returns {"f2d": (checked, mismatches), "d2f": (checked, mismatches)}."""
    lib = _lib.load()
    checked = (ctypes.c_uint64 * 2)()
    bad = (ctypes.c_uint64 * 2)()
    _lib.check("grist_selftest_conversions", lib.grist_selftest_conversions(int(n_random), int(seed), checked, bad))
    return {"f2d": (int(checked[0]), int(bad[0])), "d2f": (int(checked[1]), int(bad[1]))}


def selftest_split(n=1 << 28, seed=2404_08849):
    """grist_selftest_split: the rounding and truncating double-float splits
    against RN32 / RZ32 and their 2^-47 error bound.  Returns (checked,
    failures)."""
    lib = _lib.load()
    c, b = ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check("grist_selftest_split", lib.grist_selftest_split(int(n), int(seed), ctypes.byref(c), ctypes.byref(b)))
    return int(c.value), int(b.value)


def selftest_reciprocal(n=1 << 28, seed=2404_08849):
    """grist_selftest_reciprocal: the FMA-refined reciprocal against 1.0 / x.
    Returns (checked, results more than one ulp off, largest ulp distance)."""
    lib = _lib.load()
    c, b, w = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _lib.check("grist_selftest_reciprocal", lib.grist_selftest_reciprocal(int(n), int(seed), ctypes.byref(c),
                                                                          ctypes.byref(b), ctypes.byref(w)))
    return int(c.value), int(b.value), int(w.value)


class StepGraph:
    """A recorded sequence of library calls (grist_capture_begin/end),
    replayed with launch(); see capture()."""

    def __init__(self, handle, stream):
        self.handle = handle
        self.stream = stream

    def launch(self):
        _lib.check("grist_graph_launch", _lib.load().grist_graph_launch(self.handle, _stream_handle(self.stream)))

    def close(self):
        if self.handle:
            _lib.load().grist_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def capture(fn, stream):
    """Record the library calls fn() enqueues on `stream` (a created torch
    CUDA stream, made current for the recording) into one CUDA graph and
    return it as a StepGraph; fn's calls do not run now - the graph runs
    them at each launch().  Make the same calls once before capturing them
    (first calls allocate scratch and upload tables)."""
    import torch
    lib = _lib.load()
    h = _stream_handle(stream)
    with torch.cuda.stream(stream):
        _lib.check("grist_capture_begin", lib.grist_capture_begin(h))
        g = ctypes.c_void_p()
        try:
            fn()
        except BaseException:
            # end the capture and drop what was recorded
            if lib.grist_capture_end(h, ctypes.byref(g)) == 0:
                lib.grist_graph_destroy(g)
            raise
        rc = lib.grist_capture_end(h, ctypes.byref(g))
    _lib.check("grist_capture_end", rc)
    return StepGraph(g, stream)


FP64_FMA_CHAINS = 8   # GRIST_BENCH_FP64_CHAINS


def bench_fp64_fma(out, iters, blocks, threads=256, stream=None):
    """grist_bench_fp64_fma: enqueue the FP64 FMA throughput kernel on
    `stream` (default: the current stream).  out: CUDA float64 tensor of at
    least blocks * threads elements.  Returns the FP64 flop of the launch."""
    lib = _lib.load()
    assert out.dtype.itemsize == 8 and out.numel() >= blocks * threads and out.is_cuda
    _lib.check("grist_bench_fp64_fma", lib.grist_bench_fp64_fma(int(iters), int(blocks), int(threads), _ptr(out),
                                                                _stream_handle(stream)))
    return 2 * FP64_FMA_CHAINS * int(iters) * int(blocks) * int(threads)


class Mesh:
    """Device copy of one icosahedral Voronoi mesh (``grist_mesh_create``)."""

    def __init__(self, m: dict, device: int = 0, sfc_reorder: bool = True):
        lib = _lib.load()
        self.m = m
        self.nC, self.nE, self.nV = int(m["n_cells"]), int(m["n_edges"]), int(m["n_vertices"])
        d = _lib.MeshDesc()
        self._keep = []

        def dp(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

        def ip(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

        d.n_cells, d.n_edges, d.n_vertices, d.max_edges = self.nC, self.nE, self.nV, int(m["max_edges"])
        d.radius = float(m["radius"])
        for f in ("cell_xyz", "cell_area", "vertex_xyz", "vertex_area", "edge_dc", "edge_dv", "f_vertex",
                  "edge_sign_on_cell", "edge_sign_on_vertex", "kite_area", "trisk_weight", "d2_coef"):
            setattr(d, f, dp(m[f]))
        for f in ("cells_on_edge", "vertices_on_edge", "n_edges_on_cell", "edges_on_cell", "cells_on_cell",
                  "edges_on_vertex", "cells_on_vertex", "n_edges_on_edge", "edges_on_edge", "d2_stencil"):
            setattr(d, f, ip(m[f]))
        d.sfc_reorder = 1 if sfc_reorder else 0
        h = ctypes.c_void_p()
        _lib.check("grist_mesh_create", lib.grist_mesh_create(ctypes.byref(d), int(device), ctypes.byref(h)))
        self._keep = []
        self.handle = h
        self.device = device
        self.cell_new = np.empty(self.nC, np.int32)
        self.edge_new = np.empty(self.nE, np.int32)
        self.vertex_new = np.empty(self.nV, np.int32)
        P = ctypes.POINTER(ctypes.c_int32)
        _lib.check("grist_mesh_permutation", lib.grist_mesh_permutation(
            h, self.cell_new.ctypes.data_as(P), self.edge_new.ctypes.data_as(P), self.vertex_new.ctypes.data_as(P)))
        self.cell_old = np.argsort(self.cell_new).astype(np.int64)
        self.edge_old = np.argsort(self.edge_new).astype(np.int64)
        self.vertex_old = np.argsort(self.vertex_new).astype(np.int64)

    def features(self):
        """Stencil properties found at creation (grist_mesh_features):
        {"combined_stencil": bool, "ring_stencil": bool}."""
        f = ctypes.c_uint32()
        _lib.check("grist_mesh_features", _lib.load().grist_mesh_features(self.handle, ctypes.byref(f)))
        return {"combined_stencil": bool(f.value & 1), "ring_stencil": bool(f.value & 2)}

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().grist_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- numbering ---------------------------------------------------------
    def _old(self, kind):
        return {"cell": self.cell_old, "edge": self.edge_old, "vertex": self.vertex_old}[kind]

    def _new(self, kind):
        return {"cell": self.cell_new, "edge": self.edge_new, "vertex": self.vertex_new}[kind]

    def to_internal(self, a, kind="cell", axis=0):
        """Array in the generator's numbering -> internal numbering."""
        return np.ascontiguousarray(np.take(np.asarray(a), self._old(kind), axis=axis))

    def from_internal(self, a, kind="cell", axis=0):
        return np.ascontiguousarray(np.take(np.asarray(a), self._new(kind), axis=axis))

    # ---- steps ---------------------------------------------------------------
    @staticmethod
    def _batch(members, prec, limiter, beta, cmax=1.0):
        arr = (_lib.TracerMember * max(1, len(members)))()
        for i, mb in enumerate(members):
            q = mb["q"]
            arr[i].n_levels = int(mb["n_levels"])
            arr[i].n_tracers = int(q.shape[0])
            arr[i].ld = int(q.shape[2])
            arr[i].q = _ptr(q)
            arr[i].dpi = _ptr(mb["dpi"])
            arr[i].mass_flux = _ptr(mb["mass_flux"])
            vm = mb.get("vmass_flux")
            arr[i].vmass_flux = _ptr(vm)
            arr[i].ld_int = int(vm.shape[-1]) if vm is not None else 0
        b = _lib.TracerBatch()
        b.n_members = len(members)
        b.members = arr
        b.prec = _prec(prec)
        b.limiter = 1 if limiter else 0
        b.beta_upwind = float(beta)
        b.vertical_courant_max = float(cmax)
        return b, arr

    def tracer_step(self, members, dt, prec="fp64", limiter=True, beta=1.0, vertical_courant_max=1.0,
                    stream=None):
        """members: list of dicts with torch CUDA tensors q [T][nC][ld]
        (float64 for fp64, float32 for the mixed policies), dpi [nC][ld]
        and mass_flux [nE][ld] (float64), int n_levels, and optionally
        vmass_flux [nC][ld_int] (float64) for the vertical transport."""
        lib = _lib.load()
        b, keep = self._batch(members, prec, limiter, beta, vertical_courant_max)
        _lib.check("grist_tracer_step", lib.grist_tracer_step(self.handle, ctypes.byref(b), float(dt),
                                                              _stream_handle(stream)))

    def set_tracer_tuning(self, block=128, tracers_per_thread=4, persistent=False, use_graph=False, fused=False,
                          levels_per_thread=2, cell_edges=True):
        t = _lib.TracerTuning(int(block), int(tracers_per_thread), int(bool(persistent)), int(bool(use_graph)),
                              int(bool(fused)), int(levels_per_thread), int(bool(cell_edges)))
        _lib.check("grist_tracer_set_tuning", _lib.load().grist_tracer_set_tuning(self.handle, ctypes.byref(t)))

    def tracer_tuning(self):
        t = _lib.TracerTuning()
        _lib.check("grist_tracer_get_tuning", _lib.load().grist_tracer_get_tuning(self.handle, ctypes.byref(t)))
        return {"block": t.block, "tracers_per_thread": t.tracers_per_thread, "persistent": bool(t.persistent),
                "use_graph": bool(t.use_graph), "fused": bool(t.fused), "levels_per_thread": t.levels_per_thread,
                "cell_edges": bool(t.cell_edges)}

    def autotune_tracer(self, members, dt, prec="mix", limiter=True, beta=1.0, steps=3, stream=None,
                        cache_path=None, cache_key=None):
        """Run the library's autotuner on this batch (or reuse the choice
        stored in the JSON file cache_path under cache_key) and make it the
        mesh's tracer tuning.  Returns (tuning dict, ms per step or None)."""
        import json
        import os
        if cache_path and cache_key and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if cache_key in cache:
                t = cache[cache_key]["tuning"]
                self.set_tracer_tuning(**t)
                return t, cache[cache_key].get("ms")
        lib = _lib.load()
        b, keep = self._batch(members, prec, limiter, beta)
        best = _lib.TracerTuning()
        ms = ctypes.c_double()
        _lib.check("grist_tracer_autotune", lib.grist_tracer_autotune(
            self.handle, ctypes.byref(b), float(dt), int(steps), _stream_handle(stream), ctypes.byref(best),
            ctypes.byref(ms)))
        t = self.tracer_tuning()
        if cache_path and cache_key:
            cache = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    cache = json.load(f)
            cache[cache_key] = {"tuning": t, "ms": ms.value}
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        return t, ms.value

    def selftest_bounded_wait(self, spin_limit=100000, stream=None):
        _lib.check("grist_selftest_bounded_wait", _lib.load().grist_selftest_bounded_wait(
            self.handle, int(spin_limit), _stream_handle(stream)))

    def _dycore(self, fn, state, params, prec, dt, stream):
        lib = _lib.load()
        s = _lib.DycoreState()
        s.u, s.ps, s.dpi_theta = _ptr(state["u"]), _ptr(state["ps"]), _ptr(state["dpi_theta"])
        s.w, s.phi = _ptr(state.get("w")), _ptr(state.get("phi"))
        s.mass_flux_accum = _ptr(state.get("mass_flux_accum"))
        s.accum_weight = _ptr(state.get("accum_weight"))
        s.dpi_start = _ptr(state.get("dpi_start"))
        s.p_nh = _ptr(state.get("p_nh"))
        s.p_nh_valid = 1 if state.get("p_nh_valid") else 0
        s.accum_scale = float(state.get("accum_scale", 1.0))
        s.vmass_flux_accum = _ptr(state.get("vmass_flux_accum"))
        _lib.check(fn, getattr(lib, fn)(self.handle, ctypes.byref(s), ctypes.byref(params.c), _prec(prec),
                                        float(dt), _stream_handle(stream)))
        if state.get("p_nh") is not None:
            state["p_nh_valid"] = bool(s.p_nh_valid)

    def dycore_step_hydro(self, state, params, dt, prec="fp64", stream=None):
        self._dycore("grist_dycore_step_hydro", state, params, prec, dt, stream)

    def dycore_step_nh(self, state, params, dt, prec="fp64", stream=None):
        self._dycore("grist_dycore_step_nh", state, params, prec, dt, stream)

    def vorticity(self, u, n_levels, out=None, stream=None):
        """Relative vorticity at the vertices, [nV][ld] float64 on the device
        (grist_diag_vorticity); u is [nE][ld] float64 or float32."""
        import torch
        ld = int(u.shape[-1])
        if out is None:
            out = torch.empty((self.nV, ld), dtype=torch.float64, device=u.device)
        prec = GRIST_FP64 if u.dtype == torch.float64 else GRIST_MIX
        _lib.check("grist_diag_vorticity", _lib.load().grist_diag_vorticity(
            self.handle, _ptr(u), prec, int(n_levels), ld, _ptr(out), _stream_handle(stream)))
        return out

    def global_sum(self, kind, field, dpi=None, n_levels=1, offset=0.0, stream=None):
        """Compensated deterministic sum; returns (sum, compensation)."""
        import torch
        lib = _lib.load()
        out = (ctypes.c_double * 2)()
        prec = GRIST_FP64 if field.dtype == torch.float64 else GRIST_MIX
        ld = int(field.shape[-1]) if field.dim() > 1 else 1
        _lib.check("grist_global_sums", lib.grist_global_sums(
            self.handle, int(kind), _ptr(field), _ptr(dpi), int(n_levels), ld, prec, float(offset), out,
            _stream_handle(stream)))
        return float(out[0]), float(out[1])

    def profile(self, enable: bool):
        """Turn per-kernel CUDA-event timing on (clears totals) or off."""
        _lib.check("grist_profile_enable", _lib.load().grist_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self, max_entries: int = 128):
        """{kernel name: (launches, total_ms)} since profiling was enabled."""
        lib = _lib.load()
        names = ctypes.create_string_buffer(64 * max_entries)
        launches = (ctypes.c_int32 * max_entries)()
        ms = (ctypes.c_double * max_entries)()
        n = ctypes.c_int32()
        _lib.check("grist_profile_read", lib.grist_profile_read(self.handle, max_entries, names, launches, ms,
                                                                ctypes.byref(n)))
        out = {}
        for j in range(n.value):
            nm = names.raw[64 * j:64 * (j + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(launches[j]), float(ms[j]))
        return out

    def last_status(self):
        lib = _lib.load()
        f = ctypes.c_uint32()
        _lib.check("grist_last_step_status", lib.grist_last_step_status(self.handle, ctypes.byref(f)))
        return int(f.value)


class DycoreParams:
    """grist_dycore_params; b_interface kept on the host, phi_surface a
    device tensor [nC] (internal numbering)."""

    def __init__(self, n_levels, b_interface, pi_top, phi_surface, ld=None, ld_int=None, p0=1.0e5, rd=287.04,
                 cp=1004.64, g=9.80616, beta=0.55, emulate_fp32_rows=0):
        self.b = np.ascontiguousarray(b_interface, dtype=np.float64)
        self.phi_surface = phi_surface
        c = _lib.DycoreParams()
        c.n_levels = int(n_levels)
        c.ld = int(ld if ld is not None else n_levels)
        c.ld_int = int(ld_int if ld_int is not None else n_levels + 1)
        c.pi_top, c.p0, c.rd, c.cp, c.g, c.offcentre_beta = pi_top, p0, rd, cp, g, beta
        c.b_interface = self.b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.phi_surface = _ptr(phi_surface)
        c.emulate_fp32_rows = int(emulate_fp32_rows)
        self.c = c
