"""Pins for the oracle's Phase II (Algorithm 1, Phase II; shared by Algorithm 2,
Sec. 3.3): each check ties the orientation to something other than itself --
the essential graph of a DAG found by brute force over every orientation of its
skeleton, the paper's Proposition 2 (both stage orders give one CPDAG), hand-made
partially directed graphs for each rule, the 4-node example of Sec. 3.1, and
label-permutation invariance of the order-free reading (no GPU needed)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem

NONE, UND, FWD, BWD, BI = 0, 1, 2, 3, 4


def _acyclic(dirs, p):
    indeg = [0] * p
    out = [[] for _ in range(p)]
    for a, b in dirs:
        out[a].append(b)
        indeg[b] += 1
    stack = [v for v in range(p) if indeg[v] == 0]
    seen = 0
    while stack:
        v = stack.pop()
        seen += 1
        for w in out[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                stack.append(w)
    return seen == p


def _colliders(dirs, adj):
    par = {}
    for a, b in dirs:
        par.setdefault(b, set()).add(a)
    out = set()
    for c, ps in par.items():
        for a, b in itertools.combinations(sorted(ps), 2):
            if not adj[a, b]:
                out.add((a, c, b))
    return out


def essential_graph(dag):
    """The CPDAG of a DAG by definition: every DAG on its skeleton with its unshielded
    colliders is in the Markov class (Sec. 2.3, Markov equivalence); an edge is directed
    iff all of them orient it alike.  Brute force over the 2^|E| orientations."""
    p = dag.shape[0]
    adj = ((dag + dag.T) > 0).astype(np.uint8)
    edges = [(a, b) for a in range(p) for b in range(a + 1, p) if adj[a, b]]
    true_dirs = [(a, b) for a in range(p) for b in range(p) if dag[a, b]]
    target = _colliders(true_dirs, adj)
    members = []
    for bits in range(1 << len(edges)):
        dirs = [(a, b) if (bits >> t) & 1 else (b, a) for t, (a, b) in enumerate(edges)]
        if _acyclic(dirs, p) and _colliders(dirs, adj) == target:
            members.append(set(dirs))
    assert set(true_dirs) in members
    codes = np.zeros((p, p), dtype=np.int8)
    for a, b in edges:
        fwd = all((a, b) in m for m in members)
        bwd = all((b, a) in m for m in members)
        codes[a, b], codes[b, a] = (FWD, BWD) if fwd else (BWD, FWD) if bwd else (UND, UND)
    return codes


def _tiny_dags(count, seed0, pmin=4, pmax=7, max_edges=12):
    out = []
    s = 0
    while len(out) < count:
        rng = np.random.Generator(np.random.PCG64(seed0 + s))
        s += 1
        p = int(rng.integers(pmin, pmax + 1))
        dag, W, _ = sem.er_dag(p, float(rng.uniform(0.3, 0.7)), rng)
        if dag.sum() <= max_edges:
            out.append((dag, W))
    return out


@pytest.mark.parametrize("rev", [False, True])
def test_population_orientation_is_the_essential_graph(rev):
    # faithful population correlations: the skeleton and every separating set are exact
    # (pinned in test_oracle.py), so Phase II must return the DAG's CPDAG (Sec. 5.2)
    n_dir = 0
    for dag, W in _tiny_dags(40, 7100):
        C = sem.population_corr(W)
        R = oracle.skeleton(C, 10 ** 9, 0.01, -1, reversed_order=rev, tol=1e-10)
        codes, _ = oracle.orient(R["adj"], R["sepsets"])
        np.testing.assert_array_equal(codes, essential_graph(dag))
        n_dir += int((codes == FWD).sum())
    assert n_dir > 20                      # the cases do orient edges


def test_proposition_2_same_cpdag_both_orders():
    # Prop. 2: the reversed order's larger separating sets give the conventional order's
    # CPDAG (population version), although the sets themselves differ
    differ = 0
    for dag, W in _tiny_dags(30, 7300, pmin=5, pmax=8, max_edges=14):
        C = sem.population_corr(W)
        Rc = oracle.skeleton(C, 10 ** 9, 0.01, -1, reversed_order=False, tol=1e-10)
        Rr = oracle.skeleton(C, 10 ** 9, 0.01, -1, reversed_order=True, tol=1e-10)
        np.testing.assert_array_equal(Rc["adj"], Rr["adj"])
        differ += sum(Rc["sepsets"][k][3] != Rr["sepsets"][k][3] for k in Rc["sepsets"])
        np.testing.assert_array_equal(oracle.orient(Rc["adj"], Rc["sepsets"])[0],
                                      oracle.orient(Rr["adj"], Rr["sepsets"])[0])
    assert differ > 0


def test_four_node_example_has_no_collider():
    # Sec. 3.1: X1 _|_ X3 | X2 and X3 _|_ X4 | X2 on the skeleton 1-2, 2-3, 2-4, 1-4:
    # node 2 is in both separating sets, so no edge is oriented
    adj = np.zeros((4, 4), dtype=np.uint8)
    for a, b in [(0, 1), (1, 2), (1, 3), (0, 3)]:
        adj[a, b] = adj[b, a] = 1
    codes, rounds = oracle.orient(adj, {(0, 2): (1,), (2, 3): (1,)})
    assert rounds == 0
    assert np.all(codes[adj == 1] == UND) and np.all(codes[adj == 0] == NONE)


def _pdag(p, und=(), dirs=()):
    adj = np.zeros((p, p), dtype=np.uint8)
    mk = np.zeros((p, p), dtype=np.uint8)
    for a, b in und:
        adj[a, b] = adj[b, a] = 1
    for a, b in dirs:
        adj[a, b] = adj[b, a] = 1
        mk[a, b] = 1
    return adj, mk


def test_rule_1():
    # X_i -> X_j - X_k, X_i and X_k non-adjacent: X_j -> X_k
    adj, mk = _pdag(3, und=[(1, 2)], dirs=[(0, 1)])
    codes, rounds = oracle.meek(adj, mk)
    assert codes[1, 2] == FWD and codes[0, 1] == FWD and rounds == 1
    # X_i adjacent to X_k: R1 does not apply
    adj, mk = _pdag(3, und=[(1, 2), (0, 2)], dirs=[(0, 1)])
    codes, _ = oracle.meek(adj, mk)
    assert codes[1, 2] == UND and codes[0, 2] == UND


def test_rule_2():
    # X_i -> X_k -> X_j and X_i - X_j: X_i -> X_j
    adj, mk = _pdag(3, und=[(0, 1)], dirs=[(0, 2), (2, 1)])
    codes, _ = oracle.meek(adj, mk)
    assert codes[0, 1] == FWD


def test_rule_3():
    # X_i - X_k -> X_j, X_i - X_l -> X_j, X_k and X_l non-adjacent, X_i - X_j: X_i -> X_j
    i, j, k, l = 0, 1, 2, 3
    adj, mk = _pdag(4, und=[(i, k), (i, l), (i, j)], dirs=[(k, j), (l, j)])
    codes, _ = oracle.meek(adj, mk)
    assert codes[i, j] == FWD and codes[i, k] == UND and codes[i, l] == UND
    # X_k adjacent to X_l: R3 does not apply
    adj[k, l] = adj[l, k] = 1
    codes, _ = oracle.meek(adj, mk)
    assert codes[i, j] == UND


def test_rule_4():
    # X_i - X_k -> X_l -> X_j, X_k and X_j non-adjacent, X_i - X_j: X_i -> X_j
    i, j, k, l = 0, 1, 2, 3
    adj, mk = _pdag(4, und=[(i, k), (i, j), (i, l)], dirs=[(k, l), (l, j)])
    codes, _ = oracle.meek(adj, mk)
    assert codes[i, j] == FWD
    # X_k adjacent to X_j: R4 does not apply, and neither does any other rule to X_i - X_j
    adj[k, j] = adj[j, k] = 1
    mk[k, j] = 1
    codes, _ = oracle.meek(adj, mk)
    assert codes[i, j] == UND


def test_rules_repeat_until_nothing_changes():
    # a chain behind a collider: 0 -> 2 <- 1, then 2 - 3 - 4 - 5 oriented one R1 step per round
    adj = np.zeros((6, 6), dtype=np.uint8)
    for a, b in [(0, 2), (1, 2), (2, 3), (3, 4), (4, 5)]:
        adj[a, b] = adj[b, a] = 1
    seps = {(0, 1): (), (0, 3): (2,), (1, 3): (2,), (2, 4): (3,), (3, 5): (4,), (0, 4): (2,),
            (1, 4): (2,), (0, 5): (2,), (1, 5): (2,), (2, 5): (3,)}
    codes, rounds = oracle.orient(adj, seps)
    assert [codes[a, b] for a, b in [(0, 2), (1, 2), (2, 3), (3, 4), (4, 5)]] == [FWD] * 5
    assert rounds == 3


def test_conflicting_colliders_give_a_bidirected_edge():
    # d - a - c - b: S(a,b) empty orients a -> c <- b; S(d,c) empty orients d -> a <- c
    d, a, c, b = 0, 1, 2, 3
    adj = np.zeros((4, 4), dtype=np.uint8)
    for x, y in [(d, a), (a, c), (c, b)]:
        adj[x, y] = adj[y, x] = 1
    codes, _ = oracle.orient(adj, {(a, b): (), (d, c): (), (d, b): (a, c)})
    assert codes[a, c] == BI and codes[c, a] == BI
    assert codes[d, a] == FWD and codes[b, c] == FWD


def test_codes_are_antisymmetric_and_label_free():
    # sample-mode skeletons (errors and conflicts possible): the order-free reading gives
    # the same graph for the same skeleton and separating sets under any relabelling
    swap = np.array([0, 1, 3, 2, 4], dtype=np.int8)
    for seed in range(4):
        s = sem.make(1, instance=seed, n=400, p=18)
        C = oracle.pearson(s.X)
        R = oracle.skeleton(C, 400, 0.05, -1, reversed_order=bool(seed & 1))
        codes, _ = oracle.orient(R["adj"], R["sepsets"])
        np.testing.assert_array_equal(codes.T, swap[codes])
        p = R["adj"].shape[0]
        perm = np.random.default_rng(seed).permutation(p)        # new label i = old node perm[i]
        inv = np.argsort(perm)
        adj_p = R["adj"][np.ix_(perm, perm)]
        seps_p = {(min(inv[a], inv[b]), max(inv[a], inv[b])): tuple(int(inv[x]) for x in v[3])
                  for (a, b), v in R["sepsets"].items()}
        codes_p, _ = oracle.orient(adj_p, seps_p)
        np.testing.assert_array_equal(codes_p, codes[np.ix_(perm, perm)])
