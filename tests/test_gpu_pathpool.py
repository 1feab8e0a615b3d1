"""The path-restricted candidate pools adj(G,i,j) n path(G,i,j) of Algorithms 1
and 2 (Sec. 2.1 notation) on the GPU (option "path_pool"), element by element
against the oracle's PATHPOOL search: skeleton, separating sets (level, side,
rank in the pool's lexicographic order, members), test counts per run and the
stages visited, in both schedules."""
import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04626_gb300 import build
    from paper_2109_04626_gb300 import fastpc
    build.build()
    fastpc.load()
    return fastpc


def _case(seed, p, n, prob):
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    return np.ascontiguousarray(sem.sample(W, order, n, rng))


def _check(fp, X, order, alpha=0.01, max_level=-1):
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, alpha, max_level, reversed_order=bool(order), flags=oracle.PATHPOOL)
    with fp.PC(n, p, alpha, max_level, order=order, path_pool=1) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        adj, st = pc.skeleton()
        seps = pc.sepsets()
    np.testing.assert_array_equal(adj, R["adj"])
    assert seps == R["sepsets"]
    assert st["tests_canonical"] == R["tests_total"]
    assert st["levels_run"] == len(R["levels"])
    return R


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_pathpool_small_sems_equal_oracle(fp, seed, order):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(6, 14))
    X = _case(70 + seed, p, int(rng.integers(200, 3000)), float(rng.uniform(0.15, 0.4)))
    _check(fp, X, order)


def test_pathpool_conventional_larger(fp):
    # p = 60, sparse: pools of several components, many pairs, stages up to a few
    X = _case(91, 60, 4000, 0.06)
    R = _check(fp, X, 0)
    assert len(R["levels"]) >= 3 and len(R["sepsets"]) > 100


def test_pathpool_max_level_and_fp32_data(fp):
    X = _case(93, 30, 1500, 0.15).astype(np.float32)
    for order in (0, 1):
        for ml in (0, 1, 2):
            _check(fp, X, order, max_level=ml)


def test_pathpool_option_checks(fp):
    X = _case(95, 8, 500, 0.3)
    n, p = X.shape
    with fp.PC(n, p, 0.01, -1, order=0, path_pool=1) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        fp.pc_mlp_set_params(pc.h, np.zeros(fp.pc_mlp_nparam(), dtype=np.float32))
        pc.set(learned=1)
        with pytest.raises(fp.PCError):               # the proposal order has no pair pools
            pc.skeleton()
    with fp.PCBatch([500, 400], [8, 6], 0.01, -1) as pb:
        with pytest.raises(fp.PCError):
            fp.pc_set_opt(pb.h, "path_pool", 1)
