"""The mixed-precision dycore against the FP64 discretisation error.

The paper accepts a reduced-precision configuration when its error against
the double-precision run stays small (Sec. 2.2, Eqs. 1-2).  The yardstick
used here is the FP64 discretisation error at the same mesh level: the FP64
solution on level L against the FP64 solution on level L + 1 injected onto
level L (bisection keeps every generator, so the level-L cell centres are
the first cells of level L + 1, and injection needs no interpolation).  For
the surface pressure, the relative vorticity (kite-averaged to cells, whose
positions nest across levels), theta and w, every normalised norm (l1, l2,
linf) of mixed - FP64 on level L must lie below the same norm of
FP64_L - inject(FP64_{L+1}).

Cases: the hydrostatic jet on levels 5 -> 6 (30 levels, dt 300 s, one day)
and the non-hydrostatic jet + bubble on levels 4 -> 5 (60 levels, dt 120 s,
six hours), both seeded synthetic states evaluated at the cells' positions,
so the two levels start from the same continuous fields.
"""
import numpy as np
import pytest

import oracle as O
from grist_inputs import states as S
from grist_inputs.mesh import get_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    G.load()
    return G


def _cell_vorticity(m, vor_v):
    """Kite-weighted average of the vertex vorticity over each cell."""
    acc = np.zeros((m["n_cells"],) + vor_v.shape[1:])
    for j in range(3):
        np.add.at(acc, m["cells_on_vertex"][:, j], m["kite_area"][:, j, None] * vor_v)
    return acc / m["cell_area"][:, None]


def _run(G, m, L, nh, prec, dt, steps):
    import torch
    from gpu_cases import run_dycore
    mesh = G.Mesh(m)
    st = S.dycore_jet_case(m, L, nonhydrostatic=nh, bubble=nh)
    out = run_dycore(mesh, st, L, dt, nh=nh, prec=prec, steps=steps)
    u = torch.from_numpy(mesh.to_internal(out["u"], "edge")).cuda()
    vor = mesh.vorticity(u, L)
    torch.cuda.synchronize()
    vor_v = mesh.from_internal(vor.cpu().numpy(), "vertex")
    mesh.close()
    pint = st["pi_top"] + st["b_int"][None, :] * (out["ps"][:, None] - st["pi_top"])
    dpi = np.diff(pint, axis=1)
    res = {"ps": out["ps"], "vor": _cell_vorticity(m, vor_v), "theta": out["dpi_theta"] / dpi, "dpi": dpi}
    if nh:
        res["w"] = out["w"]
    return res


@pytest.mark.parametrize("nh,level,L,dt,steps", [(False, 5, 30, 300.0, 288), (True, 4, 60, 120.0, 180)])
def test_mixed_error_below_discretisation_error(G, nh, level, L, dt, steps):
    coarse, fine = get_mesh(level), get_mesh(level + 1)
    nC = coarse["n_cells"]
    ref = _run(G, coarse, L, nh, "fp64", dt, steps)
    mix = _run(G, coarse, L, nh, "mix", dt, steps)
    hi = _run(G, fine, L, nh, "fp64", dt, steps)
    area = coarse["cell_area"]
    fields = ["ps", "vor", "theta"] + (["w"] if nh else [])
    report = {}
    for f in fields:
        inj = hi[f][:nC]
        wgt = area if f in ("ps", "vor", "w") else area[:, None] * ref["dpi"]
        disc = O.error_norms(ref[f], inj, wgt)
        err = O.error_norms(mix[f], ref[f], wgt)
        report[f] = (err, disc)
        for e, d, name in zip(err, disc, ("l1", "l2", "linf")):
            assert e < d, (f, name, e, d)
    print("mixed vs FP64 (l1, l2, linf) | FP64 L vs L+1:",
          {k: (["%.2e" % x for x in v[0]], ["%.2e" % x for x in v[1]]) for k, v in report.items()})
