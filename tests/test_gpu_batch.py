"""Batched problems (pc_create_batch / pc_corr_block): one handle over
independent instances laid out block-diagonally.  The skeleton, sepsets and
canonical test count of every instance must equal the FP64 oracle run on that
instance alone (conventional order, Algorithm 1)."""
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
    from paper_2109_04626_gb300 import fastpc
    fastpc.load()
    return fastpc


def _instances(k, seed, p_range=(20, 60), prob_range=(0.05, 0.3), n_range=(300, 4000)):
    return sem.make_many(k, base_seed=seed, p_range=p_range, prob_range=prob_range, n_range=n_range)


def _oracle(X, alpha, max_level):
    n, p = X.shape
    return oracle.skeleton(oracle.pearson(X), n, alpha, max_level, reversed_order=False)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batch_equals_oracle_per_instance(fp, precision):
    inst = _instances(7, 900 + precision)
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    with fp.PCBatch(ns, ps, 0.01, -1, precision=precision) as pb:
        assert pb.offsets == list(np.concatenate([[0], np.cumsum(ps)]))
        for i, s in enumerate(inst):
            pb.corr_block(i, torch.from_numpy(s.X).cuda() if i % 2 else s.X)   # device and host input
        adj, st = pb.skeleton()
        adjs, seps = pb.split(adj, pb.sepsets())
    P = sum(ps)
    o = pb.offsets
    # nothing outside the diagonal blocks
    mask = np.zeros((P, P), dtype=bool)
    for i in range(len(ps)):
        mask[o[i]:o[i + 1], o[i]:o[i + 1]] = True
    assert not adj[~mask].any()
    canon = 0
    for i, s in enumerate(inst):
        R = _oracle(s.X, 0.01, -1)
        np.testing.assert_array_equal(adjs[i], R["adj"])
        assert seps[i] == R["sepsets"], i
        canon += R["tests_total"]
    assert st["tests_canonical"] == canon


def test_batch_corr_blocks_and_max_level(fp):
    inst = _instances(5, 950, p_range=(10, 40), n_range=(200, 2000))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    with fp.PCBatch(ns, ps, 0.05, 2) as pb:
        for i, s in enumerate(inst):
            pb.corr_block(i, s.X)
        C32, C64 = pb.corr_get()
        adj, _ = pb.skeleton()
        adjs, seps = pb.split(adj, pb.sepsets())
    o = pb.offsets
    for i, s in enumerate(inst):
        Co = oracle.pearson(s.X)
        blk = C64[o[i]:o[i + 1], o[i]:o[i + 1]]
        assert np.abs(blk - Co).max() <= 1e-12
        assert np.abs(C32[o[i]:o[i + 1], o[i]:o[i + 1]] - Co).max() <= 2e-6
        R = _oracle(s.X, 0.05, 2)
        np.testing.assert_array_equal(adjs[i], R["adj"])
        assert seps[i] == R["sepsets"]


def test_batch_learned_order_keeps_skeleton(fp):
    from paper_2109_04626_gb300 import proposal
    inst = _instances(4, 970, p_range=(40, 80), prob_range=(0.15, 0.3), n_range=(2000, 6000))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    with fp.PCBatch(ns, ps, 0.01, -1) as pb:
        for i, s in enumerate(inst):
            pb.corr_block(i, s.X)
        adj0, st0 = pb.skeleton()
        fp.pc_mlp_set_params(pb.h, proposal.initial_params(3))
        fp.pc_set_opt(pb.h, "learned", 1)
        fp.pc_set_opt(pb.h, "learned_min_tests", 0)
        fp.pc_set_opt(pb.h, "learned_min_ratio", 0)
        adj1, st1 = pb.skeleton()
    np.testing.assert_array_equal(adj0, adj1)


def test_batch_ci_batch_and_errors(fp):
    inst = _instances(3, 990, p_range=(12, 20), n_range=(500, 800))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    pb = fp.PCBatch(ns, ps, 0.01, -1)
    with pytest.raises(fp.PCError):
        pb.skeleton()                                   # no data yet
    with pytest.raises(fp.PCError):
        fp.pc_corr(pb.h, inst[0].X)                     # per-instance data only
    with pytest.raises(fp.PCError):
        pb.corr_block(3, inst[0].X)                     # no such instance
    with pytest.raises(fp.PCError):
        fp.pc_set_opt(pb.h, "order", 1)                 # conventional order only
    for i, s in enumerate(inst):
        pb.corr_block(i, s.X)
    o = pb.offsets
    # raw tests inside instance 1 against the oracle on that instance alone
    rng = np.random.Generator(np.random.PCG64(4))
    p1 = ps[1]
    ij = np.array([rng.choice(p1, 2, replace=False) for _ in range(50)], dtype=np.int32)
    S = np.array([[k for k in rng.permutation(p1) if k not in t][:2] for t in ij], dtype=np.int32)
    r, ind, z = pb.ci_batch(torch.from_numpy(ij + o[1]).cuda(), torch.from_numpy(S + o[1]).cuda(), 2)
    ro, zo, io, do = oracle.ci_batch(oracle.pearson(inst[1].X), ns[1], 0.01, ij, S)
    assert np.abs(r.cpu().numpy() - ro).max() <= 1e-5
    np.testing.assert_array_equal(ind.cpu().numpy().astype(bool), np.asarray(io, dtype=bool))
    # a test across instances is rejected
    with pytest.raises(fp.PCError):
        pb.ci_batch(torch.tensor([[o[0], o[1]]], dtype=torch.int32).cuda(), None, 0)
    pb.close()


def test_many64_full_size_equals_oracle(fp):
    """The 64-instance workload at its full sizes: every instance's skeleton and
    sepsets from the batched handle and from 64 concurrent handles equal the
    FP64 oracle's (conventional order)."""
    inst = sem.make_many(64)
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    pcs = []
    streams = [torch.cuda.Stream() for _ in range(8)]
    for i, s in enumerate(inst):
        pc = fp.PC(ns[i], ps[i], 0.01, -1, order=0)
        fp.pc_set_stream(pc.h, streams[i % len(streams)])
        pc.corr(torch.from_numpy(s.X).cuda())
        pcs.append(pc)
    torch.cuda.synchronize()
    adjs, stats, status = fp.pc_skeleton_many([pc.h for pc in pcs], ps)
    assert all(x == 0 for x in status)
    seps_many = [pc.sepsets() for pc in pcs]
    for pc in pcs:
        pc.close()
    with fp.PCBatch(ns, ps, 0.01, -1) as pb:
        for i, s in enumerate(inst):
            pb.corr_block(i, torch.from_numpy(s.X).cuda())
        adj_b, _ = pb.skeleton()
        blocks, seps_b = pb.split(adj_b, pb.sepsets())
    for i, s in enumerate(inst):
        R = _oracle(s.X, 0.01, -1)
        np.testing.assert_array_equal(adjs[i], R["adj"])
        np.testing.assert_array_equal(blocks[i], R["adj"])
        assert seps_many[i] == R["sepsets"], i
        assert seps_b[i] == R["sepsets"], i
        assert stats[i]["tests_canonical"] == R["tests_total"], i


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_corr_blocks_equals_per_instance_calls(fp, precision):
    """pc_corr_blocks (the instances' correlation steps on the handle's side
    streams) gives bit for bit the correlations of one pc_corr_block per
    instance, and the skeleton of every instance equals the oracle's.  Twelve
    instances of mixed sizes: more than the side streams, so a stream's
    workspaces serve several instances and grow between them."""
    inst = _instances(12, 1010 + precision, p_range=(8, 70), n_range=(150, 5000))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    Xs = [torch.from_numpy(s.X).cuda() if i % 3 else s.X for i, s in enumerate(inst)]   # host and device
    with fp.PCBatch(ns, ps, 0.01, -1, precision=precision) as pa:
        for i, X in enumerate(Xs):
            pa.corr_block(i, X)
        C32a, C64a = pa.corr_get()
        adj_a, st_a = pa.skeleton()
    with fp.PCBatch(ns, ps, 0.01, -1, precision=precision) as pb:
        pb.corr_blocks(Xs)
        C32b, C64b = pb.corr_get()
        adj_b, st_b = pb.skeleton()
        adjs, seps = pb.split(adj_b, pb.sepsets())
        pb.corr_blocks(Xs)                               # again, on the same side streams
        C32c, _ = pb.corr_get()
    np.testing.assert_array_equal(C32a, C32b)
    np.testing.assert_array_equal(C64a, C64b)
    np.testing.assert_array_equal(C32b, C32c)
    np.testing.assert_array_equal(adj_a, adj_b)
    assert st_a["tests_canonical"] == st_b["tests_canonical"]
    for i, s in enumerate(inst):
        R = _oracle(s.X, 0.01, -1)
        np.testing.assert_array_equal(adjs[i], R["adj"])
        assert seps[i] == R["sepsets"], i


def test_corr_blocks_errors(fp):
    inst = _instances(3, 1030, p_range=(10, 16), n_range=(300, 600))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    with fp.PCBatch(ns, ps, 0.01, -1) as pb:
        with pytest.raises(ValueError):
            pb.corr_blocks([s.X for s in inst[:2]])                 # one array per instance
        with pytest.raises(fp.PCError):
            fp.pc_corr_blocks(pb.h, [s.X for s in inst[:2]] + [inst[2].X[:, :5]])  # ld < p_2
        with pytest.raises(fp.PCError):
            pb.skeleton()                                           # nothing was issued
        pb.corr_blocks([s.X for s in inst])
        adj, _ = pb.skeleton()
    with fp.PC(ns[0], ps[0], 0.01, -1) as pc:
        with pytest.raises(fp.PCError):
            fp.pc_corr_blocks(pc.h, [inst[0].X])                    # not a batched handle
