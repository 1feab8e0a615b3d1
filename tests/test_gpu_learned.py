"""GPU tests of the conditioning-set proposal network: forward on the tensor
cores against the FP64 reference (with the same BF16 roundings), gradients
against the reference backward pass, training, and the learned skeleton
search (identical skeleton, re-verified sepsets, fewer tests)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
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


def bf16(x):
    x = np.asarray(x, np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def ref_forward_bf16(theta, X):
    """FP64 forward with the roundings the tensor-core path applies: BF16 inputs,
    W1, W2 and h1."""
    P = mlp.unpack(theta.astype(np.float64))
    a1 = bf16(X) @ bf16(P["W1"]).T + P["b1"]
    h1 = bf16(np.maximum(a1, 0))
    h2 = np.maximum(h1 @ bf16(P["W2"]).T + P["b2"], 0)
    return h2 @ P["w3"] + P["b3"][0]


def _handle(fp, p=8):
    X = np.random.default_rng(0).standard_normal((50, p)).astype(np.float32)
    pc = fp.PC(50, p, 0.01)
    pc.corr(torch.from_numpy(X).cuda())
    return pc


@pytest.mark.parametrize("R", [1, 127, 128, 1000, 4099])
def test_forward_matches_reference(fp, R):
    pc = _handle(fp)
    theta = (mlp.init(11) * 0.5).astype(np.float32)
    theta[mlp.NPARAM - 1] = 0.3
    fp.pc_mlp_set_params(pc.h, theta)
    X = np.random.default_rng(R).uniform(-1, 2, (R, 16)).astype(np.float32)
    s = fp.pc_mlp_forward(pc.h, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = ref_forward_bf16(theta, X)
    assert np.abs(s - ref).max() <= 2e-3 * max(1.0, np.abs(ref).max())
    pc.close()


@pytest.mark.parametrize("backward", [0, 1], ids=["fp32_cuda_cores", "bf16_tensor_cores"])
@pytest.mark.parametrize("R", [1, 300, 3001, 20000])
def test_gradient_matches_reference_elementwise(fp, R, backward):
    pc = _handle(fp)
    fp.pc_set_opt(pc.h, "mlp_backward", backward)
    theta = (mlp.init(12) * 0.5).astype(np.float32)
    fp.pc_mlp_set_params(pc.h, theta)
    rng = np.random.default_rng(4 + R)
    X = rng.uniform(-1, 2, (R, 16)).astype(np.float32)
    y = (rng.random(R) < 0.3).astype(np.float32)
    g, loss = fp.pc_mlp_grad(pc.h, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    # FP64 reference at the parameters and roundings the GPU uses: BF16 inputs,
    # BF16 W1 and W2, h1 stored in BF16 (the second layer's operand) and, on the
    # tensor-core backward, the back-propagated signals stored in BF16 (the
    # operands of its products, formed in FP32 first)
    P = mlp.unpack(theta.astype(np.float64))
    P["W1"], P["W2"] = bf16(P["W1"]), bf16(P["W2"])
    dh_store = (lambda a: bf16(np.asarray(a, np.float32))) if backward else None
    gr = mlp.grad(mlp.pack(P), bf16(X), y, h1_store=bf16, dh_store=dh_store)
    lr = mlp.loss(mlp.pack(P), bf16(X), y, h1_store=bf16)
    assert abs(loss - lr) <= 1e-5 * abs(lr) + 1e-7
    # element by element, per parameter block: the GPU accumulates in FP32 (in
    # another order) where the reference accumulates in FP64; with BF16 signals an
    # element whose FP32 and FP64 values round to neighbouring BF16 numbers moves
    # its products by one BF16 step (2^-8), hence the wider band there
    rtol, atol = (1e-3, 1e-4) if backward == 0 else (4e-3, 4e-4)
    o = 0
    for name, shape in mlp.SIZES:
        k = int(np.prod(shape))
        gb, rb = g[o:o + k].astype(np.float64), gr[o:o + k]
        scale = float(np.abs(rb).max())
        np.testing.assert_allclose(gb, rb, rtol=rtol, atol=atol * scale + 1e-9, err_msg=name)
        o += k
    pc.close()


def test_tensor_core_and_fp32_backward_train_alike(fp):
    # the two backward paths give the same training curve to BF16 accuracy
    rng = np.random.default_rng(21)
    X = rng.uniform(0, 1, (30000, 16)).astype(np.float32)
    y = ((X[:, 2] - 0.5 * X[:, 5] + 0.3 * X[:, 9]) > 0.3).astype(np.float32)
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    losses = []
    for backward in (0, 1):
        pc = _handle(fp)
        fp.pc_set_opt(pc.h, "mlp_backward", backward)
        fp.pc_mlp_set_params(pc.h, proposal.initial_params(2))
        fp.pc_mlp_train(pc.h, Xt, yt, 4, 2048, 3e-3)
        losses.append(fp.pc_mlp_grad(pc.h, Xt, yt)[1])
        pc.close()
    assert losses[1] < 0.3 and abs(losses[1] - losses[0]) <= 0.1 * losses[0], losses


def test_training_reduces_loss(fp):
    pc = _handle(fp)
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 1, (20000, 16)).astype(np.float32)
    y = ((X[:, 4] - 0.6 * X[:, 0] + 0.2 * X[:, 7]) > 0.2).astype(np.float32)
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    fp.pc_mlp_set_params(pc.h, proposal.initial_params(1))
    _, l0 = fp.pc_mlp_grad(pc.h, Xt, yt)
    l1 = fp.pc_mlp_train(pc.h, Xt, yt, 6, 2048, 3e-3)
    _, l2 = fp.pc_mlp_grad(pc.h, Xt, yt)
    assert l2 < 0.5 * l0 and l2 < 0.3, (l0, l1, l2)
    pc.close()


def _er_X(seed, p=120, n=4000):
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, 10.0 / (p - 1), rng)
    return sem.sample(W, order, n, rng).astype(np.float32)


@pytest.fixture(scope="module")
def trained(fp):
    feats, labels = proposal.collect(_er_X, range(600, 624), 0.01, order=0)
    X = _er_X(600)
    pc = fp.PC(X.shape[0], X.shape[1], 0.01, -1, order=0)
    loss = proposal.train(pc.h, feats, labels, epochs=6, batch=8192, lr=2e-3, seed=3)
    theta = fp.pc_mlp_get_params(pc.h)
    pc.close()
    return theta, loss, int(labels.shape[0])


def test_learned_skeleton_identical_and_fewer_tests(fp, trained):
    theta, loss, rows = trained
    assert rows > 1000 and loss < 0.5
    plain_tot = learned_tot = 0
    for seed in (700, 701, 702):
        X = _er_X(seed)
        n, p = X.shape
        C = oracle.pearson(X)
        R = oracle.skeleton(C, n, 0.01, -1, reversed_order=False)
        with fp.PC(n, p, 0.01, -1, order=0) as pc:
            pc.corr(torch.from_numpy(X).cuda())
            adj_p, st_p = pc.skeleton()
            fp.pc_mlp_set_params(pc.h, theta)
            fp.pc_set_opt(pc.h, "learned", 1)
            fp.pc_set_opt(pc.h, "learned_min_tests", 0)   # score every stage
            fp.pc_set_opt(pc.h, "learned_min_ratio", 0)
            adj_l, st_l = pc.skeleton()               # sepsets re-verified in FP64 inside
            seps = pc.sepsets()
        np.testing.assert_array_equal(adj_p, R["adj"])
        np.testing.assert_array_equal(adj_l, R["adj"])
        assert set(seps) == set(R["sepsets"])
        for (a, b), (lv, side, rank, nodes) in seps.items():
            assert lv == R["sepsets"][(a, b)][0]        # removed at the same stage
            assert oracle.ci_test(C, n, 0.01, a, b, list(nodes))[0]
        plain_tot += st_p["tests_canonical"]
        learned_tot += st_l["tests_canonical"]
    assert learned_tot < plain_tot, (learned_tot, plain_tot)


def test_learned_reversed_order_identical(fp, trained):
    theta, _, _ = trained
    X = sem.make(2).X
    n, p = X.shape
    C = oracle.pearson(X)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=True)
    with fp.PC(n, p, 0.01, -1, order=1) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        fp.pc_mlp_set_params(pc.h, theta)
        fp.pc_set_opt(pc.h, "learned", 1)
        fp.pc_set_opt(pc.h, "learned_min_tests", 0)
        fp.pc_set_opt(pc.h, "learned_min_ratio", 0)
        adj, st = pc.skeleton()
        seps = pc.sepsets()
    np.testing.assert_array_equal(adj, R["adj"])
    assert set(seps) == set(R["sepsets"])
    for (a, b), (lv, side, rank, nodes) in seps.items():
        assert oracle.ci_test(C, n, 0.01, a, b, list(nodes))[0]
