"""The paper's own workloads through the C-ABI, element by element against the
FP64 oracle: the simulation of Sec. 6.1-6.3 (graphs of mean degree 5 with two
hubs of 10 neighbours, weights +-U[0.2,0.8], alpha = 1e-3, both orders) and the
power experiment of Sec. 6.4 (the substitute 10-node graph, N = 100000,
alpha = 1e-3): skeleton, separating sets, canonical test counts, the partial
correlations of the four tests the text discusses, and Phase II."""
import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ALPHA = 1e-3


@pytest.fixture(scope="module")
def fp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04626_gb300 import build
    from paper_2109_04626_gb300 import fastpc
    build.build()
    fastpc.load()
    return fastpc


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("p", [15, 40, 95, 100])
def test_sweep_graphs_equal_oracle(fp, p, order):
    for m in range(3):
        s = sem.make_sweep(p, m)
        X = s.X
        n = X.shape[0]
        C = oracle.pearson(X)
        R = oracle.skeleton(C, n, ALPHA, -1, reversed_order=bool(order))
        with fp.PC(n, p, ALPHA, -1, order=order) as pc:
            pc.corr(torch.from_numpy(X).cuda())
            adj, st = pc.skeleton()
            seps = pc.sepsets()
            codes, _ = pc.orient()
        np.testing.assert_array_equal(adj, R["adj"])
        assert seps == R["sepsets"]
        assert st["tests_canonical"] == R["tests_total"]
        assert st["levels_run"] == len(R["levels"])
        np.testing.assert_array_equal(codes, oracle.orient(R["adj"], R["sepsets"])[0])


POWER_TESTS = [(5, 6, [0]), (5, 6, [0, 1, 2, 3, 4, 7, 8]), (8, 9, [0]), (8, 9, list(range(8)))]


@pytest.mark.parametrize("precision", [0, 2])
def test_power_datasets_equal_oracle(fp, precision):
    for m in range(4):
        s = sem.make_power(m)
        X = s.X
        n = X.shape[0]
        C = oracle.pearson(X)
        for order in (0, 1):
            R = oracle.skeleton(C, n, ALPHA, -1, reversed_order=bool(order))
            with fp.PC(n, 10, ALPHA, -1, order=order, precision=precision) as pc:
                pc.corr(torch.from_numpy(X).cuda())
                if order == 0:
                    for a, b, S in POWER_TESTS:
                        ij = torch.tensor([[a, b]], dtype=torch.int32, device="cuda")
                        Sd = torch.tensor([S], dtype=torch.int32, device="cuda")
                        r, ind, z = pc.ci_batch(ij, Sd, len(S))
                        ok, r64, z64, _ = oracle.ci_test(C, n, ALPHA, a, b, S)
                        assert abs(float(r.item()) - r64) <= 1e-5
                        assert bool(ind.item()) == ok
                adj, st = pc.skeleton()
                seps = pc.sepsets()
            np.testing.assert_array_equal(adj, R["adj"])
            assert seps == R["sepsets"]
            assert st["tests_canonical"] == R["tests_total"]
