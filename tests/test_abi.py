"""The C-ABI library builds, loads and exports every entry point that
include/fastpc.h declares; host-only logic is checked without a GPU."""
import math
import os
import re
import statistics

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastpc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_04626_gb300 import build as b
    from paper_2109_04626_gb300 import fastpc
    b.build()
    return fastpc.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pc_create", "pc_corr", "pc_skeleton", "pc_ci_batch", "pc_destroy",
                     "pc_set_opt", "pc_set_stream", "pc_sepsets_get", "pc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_threshold_matches_two_independent_routes(lib):
    from paper_2109_04626_gb300 import fastpc
    nd = statistics.NormalDist()
    for a in (0.5, 0.2, 0.05, 0.01, 1e-3, 1e-4, 1e-6, 1e-10):
        q = fastpc.pc_fisher_threshold(a)
        assert q == pytest.approx(-nd.inv_cdf(a / 2), rel=1e-13)
        assert q == pytest.approx(oracle.threshold(a), rel=1e-13)
    assert math.isnan(fastpc.pc_fisher_threshold(0.0))
    assert math.isnan(fastpc.pc_fisher_threshold(1.0))


def test_status_strings(lib):
    from paper_2109_04626_gb300 import fastpc
    for i, name in enumerate(fastpc.STATUS):
        assert lib.pc_status_string(i).decode() == name


def test_launch_counter_starts_without_gpu_work(lib):
    from paper_2109_04626_gb300 import fastpc
    assert fastpc.pc_kernel_launches() >= 0
