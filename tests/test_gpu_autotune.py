"""Launch-shape autotuner (pc_autotune): the chosen shape comes from the candidate
sets, and the skeleton and sepsets are the same under every shape."""
import numpy as np
import pytest
import torch

from paper_2109_04626_gb300 import sem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    from paper_2109_04626_gb300 import fastpc
    fastpc.load()
    return fastpc


@pytest.mark.parametrize("cfg,order", [(2, 1), (3, 0)])
def test_autotune_keeps_result(fp, cfg, order):
    w = sem.WORKLOADS[cfg]
    X = sem.make(cfg).X
    n, p = X.shape
    with fp.PC(n, p, w["alpha"], w["max_level"], order=order) as pc:
        pc.corr(torch.from_numpy(np.ascontiguousarray(X)).cuda())
        adj0, st0 = pc.skeleton()
        sep0 = pc.sepsets()
        r = fp.pc_autotune(pc.h, 1)
        assert r["lane_chunk"] in (4, 8, 16, 32)
        assert r["lane_rounds"] in (4, 16, 32, 64, 256)
        assert r["lane_blocks"] in (4, 8, 16)
        assert r["direct_warps"] in (2, 4, 8)
        assert r["ms_best"] <= r["ms_default"] and r["runs"] >= 2
        for k in ("lane_chunk", "lane_rounds", "lane_blocks", "direct_warps"):
            assert fp.pc_get_opt(pc.h, k) == r[k]
        adj1, st1 = pc.skeleton()
        assert np.array_equal(adj0, adj1)
        assert pc.sepsets() == sep0
        assert st1["tests_canonical"] == st0["tests_canonical"]
        # an extreme shape still gives the same skeleton
        for k, v in (("lane_chunk", 1), ("lane_rounds", 0), ("lane_blocks", 1), ("direct_warps", 1)):
            fp.pc_set_opt(pc.h, k, v)
        adj2, _ = pc.skeleton()
        assert np.array_equal(adj0, adj2)
        assert pc.sepsets() == sep0


def test_autotune_bad_args(fp):
    X = sem.make(1).X
    n, p = X.shape
    with fp.PC(n, p, 0.01, -1) as pc:
        with pytest.raises(fp.PCError):
            fp.pc_autotune(pc.h, 1)                          # before pc_corr
        pc.corr(torch.from_numpy(np.ascontiguousarray(X)).cuda())
        with pytest.raises(fp.PCError):
            fp.pc_autotune(pc.h, 0)
        for k, v in (("lane_chunk", 0), ("lane_rounds", -1), ("lane_blocks", 33), ("direct_warps", 3)):
            with pytest.raises(fp.PCError):
                fp.pc_set_opt(pc.h, k, v)


@pytest.mark.parametrize("cfg,order", [(2, 1), (4, 0)])
def test_warp_kernel_only_same_result(fp, cfg, order):
    """Every stage on the one-warp-per-test kernel (the plain form's kernel) gives
    the same skeleton, sepsets and canonical count as the small-stage kernel."""
    w = sem.WORKLOADS[cfg]
    X = sem.make(cfg).X
    n, p = X.shape
    out = []
    for lane in (1, 0):
        with fp.PC(n, p, w["alpha"], w["max_level"], order=order, small_stage_kernel=lane) as pc:
            pc.corr(torch.from_numpy(np.ascontiguousarray(X)).cuda())
            adj, st = pc.skeleton()
            out.append((adj, pc.sepsets(), st["tests_canonical"]))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert out[0][2] == out[1][2]
