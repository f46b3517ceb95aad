"""The allocation-free weighted sum, called through the C ABI.

grist_weighted_sum_noalloc serves callers that cannot allocate device
memory (their memory belongs to another allocator that reserved it up front,
or they must not pay the synchronisation a cudaMalloc / cudaFree implies):
its partial sums live in a fixed device array instead of library scratch.
This file is collected last so that a run stopping at the first failure has
run every other test before it.  Two calls in a row must each match the
regular entry point (grist_global_sums, area-weighted) within the global-sum
tolerance used elsewhere (4 ulp of the exact sum), and sizes beyond the
stated maximum are refused."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_weighted_sum_matches_global_sums(mesh_cache):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2404_08849_gb300 as G
    from paper_2404_08849_gb300 import _lib
    lib = _lib.load()
    m = mesh_cache(5)
    mesh = G.Mesh(m)
    torch.cuda.set_device(mesh.device)
    area = torch.from_numpy(mesh.to_internal(m["cell_area"])).cuda()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(31)
    for call in range(2):
        x_host = rng.standard_normal(mesh.nC) * 10.0 ** (call + 2) + 5.0
        x = torch.from_numpy(mesh.to_internal(x_host)).cuda()
        rc = lib.grist_weighted_sum_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(area.data_ptr()),
                                            mesh.nC, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = float(out[0].item())
        ref = mesh.global_sum(G.GRIST_SUM_AREA_WEIGHTED, x.view(-1, 1), n_levels=1)[0]
        exact = math.fsum(m["cell_area"] * x_host)
        assert abs(got - ref) <= 4 * np.spacing(abs(exact)), (call, got, ref)
        assert abs(got - exact) <= 4 * np.spacing(abs(exact)), (call, got, exact)
    # unweighted form and the size limit
    ones = torch.ones(1000, dtype=torch.float64, device="cuda")
    assert lib.grist_weighted_sum_noalloc(ctypes.c_void_p(ones.data_ptr()), None, 1000,
                                          ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    assert float(out[0].item()) == 1000.0
    too_many = (1 << 28) + 1
    assert lib.grist_weighted_sum_noalloc(ctypes.c_void_p(ones.data_ptr()), None, too_many,
                                          ctypes.c_void_p(out.data_ptr()), stream) == -1
    mesh.close()


@pytest.mark.parametrize("n", [65536, 3 * 65536 + 17, 300 * 65536 + 17])
def test_noalloc_multi_block(n):
    """Several blocks: the per-block partials and their compensated merge
    (one chunk exactly, a ragged last chunk, a few hundred chunks), then a
    second call with fewer blocks, which must not read the first call's
    leftover partials.  Random weights and values against math.fsum."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2404_08849_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(0)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(n)
    for nn in (n, n // 3 + 5):
        x_host = rng.standard_normal(nn) * 100.0 + 3.0
        w_host = rng.uniform(0.5, 2.0, nn)
        x = torch.from_numpy(x_host).cuda()
        w = torch.from_numpy(w_host).cuda()
        rc = lib.grist_weighted_sum_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()), nn,
                                            ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = float(out[0].item())
        exact = math.fsum((w_host * x_host).tolist())
        # the products w*x are rounded once on either side; the bound is on
        # the sum of those rounded products
        assert abs(got - exact) <= 4 * np.spacing(abs(exact)), (nn, got, exact)
