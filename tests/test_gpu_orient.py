"""GPU parity of Phase II (Algorithm 1, Phase II; pc_orient) against the oracle's
Phase II: the orientation codes are compared entry by entry (bit-exact), on the
GPU's own skeleton and separation sets (any stage order, precision or proposal
order) and, where the sets are the canonical ones, end to end against the
oracle's skeleton as well."""
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


def _case(seed, p, n, prob, dtype=np.float32):
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    return np.ascontiguousarray(sem.sample(W, order, n, rng).astype(dtype))


def _run(fp, X, order, precision=2, alpha=0.01, learned_theta=None):
    n, p = X.shape
    with fp.PC(n, p, alpha, -1, order=order, precision=precision) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        if learned_theta is not None:
            fp.pc_mlp_set_params(pc.h, learned_theta)
            fp.pc_set_opt(pc.h, "learned", 1)
            fp.pc_set_opt(pc.h, "learned_min_tests", 0)
            fp.pc_set_opt(pc.h, "learned_min_ratio", 0)
        adj, _ = pc.skeleton()
        seps = pc.sepsets()
        codes, rounds = pc.orient()
        codes_d = torch.empty((p, p), dtype=torch.int8, device="cuda")
        pc.orient(codes_d)
    np.testing.assert_array_equal(codes_d.cpu().numpy(), codes)
    return adj, seps, codes, rounds


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("shape", [(1000, 20, 0.2, np.float64), (5000, 95, 0.3, np.float32),
                                   (3001, 70, 0.08, np.float32), (2000, 133, 0.04, np.float32),
                                   (600, 40, 0.35, np.float32)])
def test_orient_equals_oracle(fp, order, shape):
    n, p, prob, dt = shape
    X = _case(31 + p, p, n, prob, dt)
    adj, seps, codes, rounds = _run(fp, X, order)
    ref, ref_rounds = oracle.orient(adj, seps)
    np.testing.assert_array_equal(codes, ref)
    assert rounds == ref_rounds
    # the canonical sets: the oracle's own Phase I gives the same graph
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=bool(order))
    np.testing.assert_array_equal(codes, oracle.orient(R["adj"], R["sepsets"])[0])
    assert np.count_nonzero(codes == 2) > 0 or p <= 20


@pytest.mark.parametrize("precision", [0, 1])
def test_orient_other_precisions(fp, precision):
    X = _case(77, 60, 2500, 0.15)
    adj, seps, codes, rounds = _run(fp, X, 1, precision=precision)
    np.testing.assert_array_equal(codes, oracle.orient(adj, seps)[0])


def test_orient_proposal_order_sets(fp):
    # a proposal order (random network parameters) finds other separating sets than the
    # lexicographic one; Phase II on them matches the oracle's Phase II on the same sets
    X = _case(91, 150, 4000, 0.07)
    theta = np.random.default_rng(4).standard_normal(fp.pc_mlp_nparam()).astype(np.float32) * 0.2
    adj, seps, codes, rounds = _run(fp, X, 0, learned_theta=theta)
    ref, ref_rounds = oracle.orient(adj, seps)
    np.testing.assert_array_equal(codes, ref)
    assert rounds == ref_rounds


def test_orient_empty_and_dense_graphs(fp):
    # independent columns: no edge survives; codes all zero
    X = np.random.default_rng(2).standard_normal((3000, 30)).astype(np.float32)
    adj, seps, codes, rounds = _run(fp, X, 0, alpha=1e-6)
    np.testing.assert_array_equal(codes, oracle.orient(adj, seps)[0])
    # few samples of a dense graph: many edges kept, colliders and rules on dense rows
    X = _case(5, 48, 120, 0.6)
    adj, seps, codes, rounds = _run(fp, X, 1, alpha=0.2)
    np.testing.assert_array_equal(codes, oracle.orient(adj, seps)[0])


def test_orient_batched_instances(fp):
    inst = sem.make_many(5, base_seed=414, p_range=(20, 90), n_range=(800, 4000))
    ns = [s.X.shape[0] for s in inst]
    ps = [s.X.shape[1] for s in inst]
    with fp.PCBatch(ns, ps, 0.01, -1) as pb:
        for i, s in enumerate(inst):
            pb.corr_block(i, s.X)
        adj, _ = pb.skeleton()
        codes, _ = pb.orient()
        blocks = pb.split(codes)
        adjs = pb.split(adj)
    off = np.cumsum([0] + ps)
    # no code outside the diagonal blocks
    mask = np.zeros_like(codes, dtype=bool)
    for i in range(len(ps)):
        mask[off[i]:off[i + 1], off[i]:off[i + 1]] = True
    assert not codes[~mask].any()
    for i, s in enumerate(inst):
        C = oracle.pearson(s.X)
        R = oracle.skeleton(C, s.X.shape[0], 0.01, -1, reversed_order=False)
        np.testing.assert_array_equal(adjs[i], R["adj"])
        np.testing.assert_array_equal(blocks[i], oracle.orient(R["adj"], R["sepsets"])[0])


def test_orient_errors(fp):
    X = _case(3, 12, 500, 0.3)
    with fp.PC(500, 12, 0.01, -1) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        with pytest.raises(fp.PCError):
            pc.orient()                                  # before pc_skeleton
        pc.skeleton()
        assert fp.load().pc_orient(pc.h, None, None) != 0    # no output buffer


def test_orient_full_size_p1000(fp):
    # the p = 1000, n = 20000 workload (expected degree 10), conventional order
    s = sem.make(4)
    adj, seps, codes, rounds = _run(fp, np.ascontiguousarray(s.X), 0)
    ref, ref_rounds = oracle.orient(adj, seps)
    np.testing.assert_array_equal(codes, ref)
    assert rounds == ref_rounds
    assert np.count_nonzero(codes == 2) > 100
