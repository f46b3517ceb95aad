"""The benchmark's per-kernel accounting covers every kernel the library's
step paths launch: each name passed to the library's launch macro (the
profiling names) has its compulsory bytes in bench.algorithmic_bytes, so a
renamed, added or removed kernel cannot silently drop out of the GB/s and
share columns.  The two whole-stage / whole-step launches of the optional
modes (fused tiles, persistent kernel) have no per-phase byte count."""
import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

WHOLE_STEP = {"k_tr_tile_stage", "k_tracer_persistent"}


def _launched_names():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "paper_2404_08849_gb300", "csrc", "*.cu")):
        src = open(path).read()
        names |= set(re.findall(r'PN\("(k_[a-z0-9_]+)"\)', src))
        names |= set(re.findall(r'"(k_[a-z0-9_]+)/(?:mix|fp64)"', src))
    return names


def test_every_launched_kernel_has_algorithmic_bytes():
    import bench
    names = _launched_names()
    assert {"k_momentum", "k_nh_solve", "k_tr_edge", "k_tr_final"} <= names
    missing = []
    for n in sorted(names - WHOLE_STEP):
        for prec in ("mix", "fp64"):
            b = bench.algorithmic_bytes(n + "/" + prec, 40962, 122880, 81920, 30, 4, prec)
            if not b or b <= 0:
                missing.append((n, prec))
    assert not missing, missing


def test_executed_fp64_table_names_launched_kernels():
    import bench
    names = _launched_names()
    assert set(bench.FP64_WORK_MIX) <= names
    assert set(bench.FP64_ALG) <= names
