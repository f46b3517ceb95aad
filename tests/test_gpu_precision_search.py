"""GPU: the iterative precision search of Sec. 2.2 (Eqs. 1-2).

* grist_diag_vorticity against the oracle's vertex vorticity;
* the row emulation: mask 0 leaves the FP64 run bit for bit unchanged, a
  row the hydrostatic core never evaluates (advection of w, phi) changes
  nothing, every other row changes the result, by less than the native
  mixed policy's error for the advective rows;
* the search: accepts exactly the rows with E <= alpha, builds each trial on
  the configuration accepted so far, and is reproducible.
"""
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


def test_vorticity_diagnostic_matches_oracle(G, mesh_cache):
    import torch
    from gpu_cases import from_dev, to_dev
    m = mesh_cache(4)
    mesh = G.Mesh(m)
    L = 12
    u = S.dycore_jet_case(m, L)["u"]
    ref = O.vorticity(O.Mesh(m), u)
    got = from_dev(mesh, mesh.vorticity(to_dev(mesh, u, "edge", 0, torch.float64), L), "vertex")
    assert O.max_rel_diff(got, ref) <= 1e-12
    got32 = from_dev(mesh, mesh.vorticity(to_dev(mesh, u, "edge", 0, torch.float32), L), "vertex")
    assert O.max_rel_diff(got32, ref) <= 1e-6
    mesh.close()


@pytest.fixture(scope="module")
def hdc(G, mesh_cache):
    from paper_2404_08849_gb300 import precision as PR
    m = mesh_cache(4)
    st = S.dycore_jet_case(m, 20)
    exp = PR.Experiment(m, st, 20, 300.0, 12, nonhydrostatic=False)
    yield exp, exp.run(0)
    exp.close()


def test_row_emulation(G, hdc):
    exp, truth = hdc
    again = exp.run(0)
    assert np.array_equal(again[0], truth[0]) and np.array_equal(again[1], truth[1])
    # the hydrostatic core never advects w or phi
    e = exp.error(exp.run(G.GRIST_ROWS["nh_adv"]), truth)
    assert e == 0.0
    errs = {}
    for name, bit in G.GRIST_ROWS.items():
        if name == "nh_adv":
            continue
        errs[name] = exp.error(exp.run(bit), truth)
        assert 0.0 < errs[name] < 1e-2, (name, errs[name])
    e_mix = exp.error(exp.run(0, prec="mix"), truth)
    assert 0.0 < e_mix < 1e-2
    for name in ("theta", "pv_flux"):
        assert errs[name] <= e_mix
    with pytest.raises(G.GristError):
        exp.run(G.GRIST_ROW_ALL + 1)
    with pytest.raises(G.GristError):        # emulation runs on the FP64 path only
        exp.run(G.GRIST_ROWS["eos"], prec="mix")


def test_iterative_search_accepts_rows_within_alpha(G, hdc):
    from paper_2404_08849_gb300 import precision as PR
    exp, truth = hdc
    # alpha 0.05 (the paper's): a short run accepts every row
    config, kept, table = PR.iterative_search(exp, alpha=0.05, truth=truth)
    assert kept == list(PR.DEFAULT_ORDER) and config == G.GRIST_ROW_ALL
    assert all(t["accepted"] == (t["E"] <= 0.05) for t in table)
    # masks grow monotonically with the accepted rows
    masks = [t["mask"] for t in table]
    assert all(b & a == a for a, b in zip(masks, masks[1:]))
    # alpha 0: only the row that changes nothing survives; every trial is
    # then a single row on top of the empty configuration
    config0, kept0, table0 = PR.iterative_search(exp, alpha=0.0, truth=truth)
    assert kept0 == ["nh_adv"] and config0 == G.GRIST_ROWS["nh_adv"]
    for t in table0:
        assert t["mask"] & ~G.GRIST_ROWS["nh_adv"] in (0, G.GRIST_ROWS[t["row"]])
    # reproducible
    config_b, kept_b, table_b = PR.iterative_search(exp, alpha=0.05, truth=truth)
    assert [t["E"] for t in table_b] == [t["E"] for t in table]
