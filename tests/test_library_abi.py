"""CPU-side checks of the C-ABI boundary: the library builds for sm_103a,
loads, and exports every entry point declared in include/grist.h (no
compute calls: there is no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^(?:int|const char \*)\s*(grist_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("grist_mesh_create", "grist_tracer_step", "grist_dycore_step_hydro", "grist_dycore_step_nh",
              "grist_global_sums"):
        assert n in names


def test_library_builds_loads_and_exports():
    from paper_2404_08849_gb300 import build, _lib
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) == set(_declared())


def test_status_strings_without_gpu():
    from paper_2404_08849_gb300 import _lib
    lib = _lib.load()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.grist_status_string(code)
    assert lib.grist_mesh_destroy(None) == 0
    assert lib.grist_mesh_create(None, 0, ctypes.byref(ctypes.c_void_p())) == -1


def test_mesh_create_rejects_bad_tables_before_touching_a_gpu(mesh_cache):
    """Validation runs on the host before any CUDA call: corrupt tables are
    refused with GRIST_EINVAL even on a machine without a GPU."""
    import numpy as np
    import paper_2404_08849_gb300 as G
    m = dict(mesh_cache(2))
    bad = m["cells_on_edge"].copy()
    bad[3, 0] = m["n_cells"] + 7
    m["cells_on_edge"] = bad
    try:
        G.Mesh(m)
    except G.GristError as e:
        assert e.code == -1
    else:
        raise AssertionError("corrupt mesh accepted")
    m = dict(mesh_cache(2))
    area = m["cell_area"].copy()
    area[0] *= 1.5
    m["cell_area"] = area
    try:
        G.Mesh(m)
    except G.GristError as e:
        assert e.code == -1
    else:
        raise AssertionError("area sum mismatch accepted")
