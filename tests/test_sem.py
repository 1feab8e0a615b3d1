"""The seeded input generators (no method arithmetic): the recipe of the paper's
simulation (Sec. 6.1) as stated there."""
import numpy as np

from paper_2109_04626_gb300 import sem


def test_sweep_graphs_follow_the_recipe():
    for p in (15, 50, 95):
        degs, hub_ok, mags = [], 0, []
        for m in range(20):
            s = sem.make_sweep(p, m, n=50)
            assert np.all(np.tril(s.dag) == 0)                 # the fixed order X_1..X_p
            d = (s.dag + s.dag.T).sum(1)
            degs.append(d.mean())
            hub_ok += int(np.sort(d)[-2] >= 10)                # two hubs of (at least) 10 neighbours
            mags.append(np.abs(s.weights[s.dag == 1]))
            assert s.X.shape == (50, p) and s.X.dtype == np.float32
        mags = np.concatenate(mags)
        assert mags.min() >= 0.2 and mags.max() <= 0.8
        assert abs(np.mean(degs) - 5.0) < 1.6                  # mean degree 5 (plus the hubs' excess)
        assert hub_ok == 20
    a = sem.make_sweep(40, 3)
    b = sem.make_sweep(40, 3)
    assert np.array_equal(a.X, b.X) and a.seed == b.seed       # seeded


def test_power_graph_has_the_stated_relations():
    # Sec. 6.4: X5 _|_ X6 | {X0} and | {X0,X1,X2,X3,X4,X7,X8}; X8, X9 dependent given
    # {X0} and given {X0..X7} -- checked by d-separation on the substitute DAG
    from tests.dsep import d_separated
    dag, W, order = sem.power_dag()
    assert d_separated(dag, 5, 6, [0])
    assert d_separated(dag, 5, 6, [0, 1, 2, 3, 4, 7, 8])
    assert not d_separated(dag, 5, 6, [])
    assert not d_separated(dag, 8, 9, [0])
    assert not d_separated(dag, 8, 9, list(range(8)))
    assert np.all((np.abs(W[dag == 1]) >= 0.2) & (np.abs(W[dag == 1]) <= 0.8))
    s = sem.make_power(0, n=1000)
    assert s.X.shape == (1000, 10)
