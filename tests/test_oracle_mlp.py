"""Pins for the FP64 reference of the proposal network: the hand-written
backward pass agrees with central finite differences of the loss."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    theta = mlp.init(3) * 0.5
    X = rng.standard_normal((40, mlp.NF))
    y = (rng.random(40) < 0.3).astype(float)
    g = mlp.grad(theta, X, y)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 2048]])       # b3, a W1 entry, b1[0]
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y) - mlp.loss(tm, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_is_bce_of_sigmoid():
    theta = mlp.init(1)
    X = np.random.default_rng(2).standard_normal((7, mlp.NF))
    y = np.array([0, 1, 1, 0, 1, 0, 0], dtype=float)
    s, _ = mlp.forward(theta, X)
    sig = 1 / (1 + np.exp(-s))
    ref = -np.mean(y * np.log(sig) + (1 - y) * np.log(1 - sig))
    assert abs(mlp.loss(theta, X, y) - ref) < 1e-12


def test_pack_unpack_roundtrip():
    theta = mlp.init(9)
    assert theta.size == mlp.NPARAM == 18817
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(theta)), theta)


def test_stored_h1_gradient_matches_finite_differences():
    # with a storage map of derivative one (here a fixed offset added to h1), the
    # chain rule through the stored h1 is the exact gradient of the loss
    rng = np.random.default_rng(6)
    theta = mlp.init(4) * 0.5
    X = rng.standard_normal((30, mlp.NF))
    y = (rng.random(30) < 0.4).astype(float)
    off = 1e-3 * rng.standard_normal((30, mlp.NH))
    store = lambda h: h + off                                     # noqa: E731
    g = mlp.grad(theta, X, y, h1_store=store)
    assert np.abs(g - mlp.grad(theta, X, y)).max() > 0            # the map is applied
    h = 1e-6
    for i in np.concatenate([rng.choice(mlp.NPARAM, size=40, replace=False), [0, 2048, mlp.NPARAM - 1]]):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, X, y, h1_store=store) - mlp.loss(tm, X, y, h1_store=store)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_stored_signals_identity_map_is_the_gradient():
    # the backward-signal storage map at the identity gives the exact gradient
    # (pinned above by finite differences); any other map is applied as stated
    rng = np.random.default_rng(7)
    theta = mlp.init(5) * 0.5
    X = rng.standard_normal((25, mlp.NF))
    y = (rng.random(25) < 0.5).astype(float)
    np.testing.assert_array_equal(mlp.grad(theta, X, y, dh_store=lambda a: a), mlp.grad(theta, X, y))
    g0 = mlp.grad(theta, X, y, dh_store=lambda a: np.zeros_like(a))
    P = mlp.unpack(g0)
    assert not P["W2"].any() and not P["W1"].any() and not P["b1"].any()   # nothing flows past a2
    assert P["w3"].any()                                                     # the last layer does not read them


def test_bf16_rounding_of_the_tests_equals_torch():
    # the BF16 rounding the GPU tests apply to their references (nearest, ties to
    # even) is torch's own conversion
    torch = pytest.importorskip("torch")
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_gpu_learned import bf16
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(bf16(x), ref)
