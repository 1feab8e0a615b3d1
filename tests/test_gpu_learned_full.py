"""The learned proposal order at the full sizes of the benchmark workloads: the
p=1000 ER SEM (n=20000) with a network trained as that workload prescribes (on
200 seeded p=200 SEMs of the same expected degree), and the 64 independent
SEMs (p in [50,400]) with the proposal on in every handle and in the batched
handle.  The skeleton must equal the FP64 oracle's (Eq. 1 decides removal,
Sec. 2.2.2, whatever the order in which the sets are tried), every recorded
separating set must be independent by the oracle's own test, and each pair must
be removed at the oracle's stage (PC-stable: the order within a stage cannot
change which stage removes a pair)."""
import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import proposal, sem

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


def _check_learned(C, n, alpha, adj, seps, R):
    np.testing.assert_array_equal(adj, R["adj"])
    assert set(seps) == set(R["sepsets"])
    by_l = {}
    for (a, b), (lv, side, rank, nodes) in seps.items():
        assert lv == R["sepsets"][(a, b)][0], (a, b)
        if lv > 0:
            by_l.setdefault(lv, []).append((a, b, nodes))
    for lv, rows in by_l.items():
        ij = np.array([(a, b) for a, b, _ in rows], dtype=np.int32)
        S = np.array([nodes for _, _, nodes in rows], dtype=np.int32)
        r, z, indep, degen = oracle.ci_batch(C, n, alpha, ij, S)
        assert np.all(indep), lv


def _c4_training_X(sd):
    # the p=1000 workload's training recipe: p=200 ER SEMs of expected degree 10
    rng = np.random.Generator(np.random.PCG64(4100 + sd))
    dag, W, order = sem.er_dag(200, 10.0 / 199, rng)
    return sem.sample(W, order, 5000, rng).astype(np.float32)


def test_p1000_learned_order_equals_oracle(fp):
    feats, labels = proposal.collect(_c4_training_X, range(200), 0.01, order=0, max_rows_per_seed=100_000)
    s = sem.make(4)
    X = s.X
    n, p = X.shape
    with fp.PC(n, p, 0.01, -1, order=0, precision=2) as pc:
        loss = proposal.train(pc.h, feats, labels, epochs=6, batch=8192, lr=2e-3, seed=1)
        assert loss < 0.2
        pc.corr(torch.from_numpy(X).cuda())
        adj_p, st_p = pc.skeleton()
        fp.pc_set_opt(pc.h, "learned", 1)
        adj, st = pc.skeleton()
        seps = pc.sepsets()
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=False)
    np.testing.assert_array_equal(adj_p, R["adj"])
    assert st_p["tests_canonical"] == R["tests_total"]
    _check_learned(C, n, 0.01, adj, seps, R)
    # the proposal order reaches the separating sets with fewer tests
    assert st["tests_canonical"] < st_p["tests_canonical"]


def test_many64_learned_order_equals_oracle(fp):
    # network trained on other seeds of the 64-instance recipe
    train = sem.make_many(24, base_seed=9000)
    feats, labels = proposal.collect(lambda i: train[i].X, range(len(train)), 0.01, order=0,
                                     max_rows_per_seed=50_000)
    inst = sem.make_many(64)
    ns = [x.X.shape[0] for x in inst]
    ps = [x.X.shape[1] for x in inst]
    with fp.PC(ns[0], ps[0], 0.01, -1, order=0) as pc0:
        proposal.train(pc0.h, feats, labels, epochs=4, batch=8192, lr=2e-3, seed=2)
        theta = fp.pc_mlp_get_params(pc0.h)
    opts = {"learned": 1, "learned_min_tests": 0, "learned_min_ratio": 0}   # score every stage
    pcs, streams = [], [torch.cuda.Stream() for _ in range(8)]
    for i, x in enumerate(inst):
        pc = fp.PC(ns[i], ps[i], 0.01, -1, order=0, precision=2)
        fp.pc_mlp_set_params(pc.h, theta)
        pc.set(**opts)
        fp.pc_set_stream(pc.h, streams[i % len(streams)])
        pc.corr(torch.from_numpy(x.X).cuda())
        pcs.append(pc)
    torch.cuda.synchronize()
    adjs, stats, status = fp.pc_skeleton_many([pc.h for pc in pcs], ps)
    assert all(x == 0 for x in status)
    seps_many = [pc.sepsets() for pc in pcs]
    for pc in pcs:
        pc.close()
    with fp.PCBatch(ns, ps, 0.01, -1, precision=2) as pb:
        fp.pc_mlp_set_params(pb.h, theta)
        pb.set(**opts)
        for i, x in enumerate(inst):
            pb.corr_block(i, torch.from_numpy(x.X).cuda())
        adj_b, _ = pb.skeleton()
        blocks, seps_b = pb.split(adj_b, pb.sepsets())
    for i, x in enumerate(inst):
        C = oracle.pearson(x.X)
        R = oracle.skeleton(C, ns[i], 0.01, -1, reversed_order=False)
        _check_learned(C, ns[i], 0.01, adjs[i], seps_many[i], R)
        _check_learned(C, ns[i], 0.01, blocks[i], seps_b[i], R)
