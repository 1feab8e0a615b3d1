"""Pins for the oracle's path-restricted candidate pool (the paper's
adj(G,a,b) intersected with path(G,a,b), Sec. 2.1 notation, Algorithms 1 and 2;
flag PATHPOOL): one pool per pair -- the nodes adjacent to a or b that lie on
some simple a-b path of the frozen graph -- searched once per stage, PC-stable.

* Brute force: a plain enumeration written here finds every node on a simple
  a-b path by walking all simple paths, takes each decision from numpy's
  inverse of the correlation block, and runs both schedules; the skeleton, the
  separating sets, the visited stages and the test counts must equal the
  oracle's.
* Population: on faithful population correlations of small DAGs the restricted
  pool still recovers the true skeleton (every separating set the restriction
  drops lies off all a-b paths, so no needed set is lost).
(no GPU needed)"""
import itertools
import statistics

import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem
from tests.test_oracle_bruteforce import _indep
from tests.test_oracle_orient import _tiny_dags


def _path_nodes(adj, a, b):
    """Nodes (other than a, b) on some simple a-b path, by walking all of them."""
    p = adj.shape[0]
    on = set()
    stack = [(a, (a,))]
    while stack:
        x, path = stack.pop()
        for y in range(p):
            if not adj[x, y] or y in path:
                continue
            if y == b:
                on.update(path[1:])
            else:
                stack.append((y, path + (y,)))
    return on


def _pool(adj, a, b):
    p = adj.shape[0]
    near = {k for k in range(p) if k not in (a, b) and (adj[a, k] or adj[b, k])}
    return sorted(near & _path_nodes(adj, a, b))


def _stage(C, n, q, adj, l, seps):
    p = adj.shape[0]
    frozen = adj.copy()
    count, removed = 0, []
    for a in range(p):
        for b in range(a + 1, p):
            if not frozen[a, b]:
                continue
            for rank, S in enumerate(itertools.combinations(_pool(frozen, a, b), l)):
                count += 1
                if _indep(C, n, a, b, S, q)[0]:
                    seps[(a, b)] = (l, 0, rank, tuple(int(x) for x in S))
                    removed.append((a, b))
                    break
    for a, b in removed:
        adj[a, b] = adj[b, a] = False
    return count


def _largest(adj):
    p = adj.shape[0]
    return max((len(_pool(adj, a, b)) for a in range(p) for b in range(a + 1, p) if adj[a, b]), default=-1)


def brute_pathpool(C, n, alpha, reversed_order):
    p = C.shape[0]
    q = -statistics.NormalDist().inv_cdf(alpha / 2)
    adj = np.ones((p, p), dtype=bool)
    np.fill_diagonal(adj, False)
    seps, tests, levels = {}, {}, []
    if reversed_order:
        # closed-form stage: on the complete graph every other node is on an a-b path
        removed = []
        for a in range(p):
            for b in range(a + 1, p):
                rest = [w for w in range(p) if w not in (a, b)]
                if _indep(C, n, a, b, rest, q)[0]:
                    seps[(a, b)] = (p - 2, 0, 0, tuple(rest))
                    removed.append((a, b))
        for a, b in removed:
            adj[a, b] = adj[b, a] = False
        tests[p - 2] = p * (p - 1) // 2
        levels.append(p - 2)
        l = min(p - 3, _largest(adj))
        while l >= 0:
            levels.append(l)
            tests[l] = _stage(C, n, q, adj, l, seps)
            l = min(l - 1, _largest(adj))
    else:
        l = 0
        while _largest(adj) >= l:
            levels.append(l)
            tests[l] = _stage(C, n, q, adj, l, seps)
            l += 1
    return adj.astype(np.uint8), seps, tests, levels


@pytest.mark.parametrize("rev", [False, True])
@pytest.mark.parametrize("case", [(6101, 7, 400, 0.45), (6102, 8, 1500, 0.35), (6103, 9, 3000, 0.3)])
def test_pathpool_equals_brute_force(case, rev):
    seed, p, n, prob = case
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    C = oracle.pearson(sem.sample(W, order, n, rng))
    adj, seps, tests, levels = brute_pathpool(C, n, 0.01, rev)
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=rev, flags=oracle.PATHPOOL)
    np.testing.assert_array_equal(R["adj"], adj)
    assert R["sepsets"] == seps
    assert R["levels"] == levels
    assert {l: int(R["tests_level"][l]) for l in levels} == tests


def test_pathpool_restriction_is_active_somewhere():
    # the restriction does drop candidates on these graphs: the pools of some pair
    # differ from adj(a) u adj(b) minus {a, b} at some stage, so the counts differ
    differ = 0
    for seed in range(6200, 6212):
        rng = np.random.Generator(np.random.PCG64(seed))
        dag, W, order = sem.er_dag(9, 0.3, rng)
        n = 800
        C = oracle.pearson(sem.sample(W, order, n, rng))
        Rp = oracle.skeleton(C, n, 0.01, -1, reversed_order=False, flags=oracle.PATHPOOL)
        # the unrestricted union pool, by brute force, for comparison of the counts
        adj = np.ones((9, 9), dtype=bool)
        np.fill_diagonal(adj, False)
        q = -statistics.NormalDist().inv_cdf(0.005)
        seps, total, l = {}, 0, 0
        while True:
            frozen = adj.copy()
            pools = {(a, b): sorted(k for k in range(9) if k not in (a, b) and (frozen[a, k] or frozen[b, k]))
                     for a in range(9) for b in range(a + 1, 9) if frozen[a, b]}
            if not pools or max(len(v) for v in pools.values()) < l:
                break
            for (a, b), pool in pools.items():
                for S in itertools.combinations(pool, l):
                    total += 1
                    if _indep(C, n, a, b, S, q)[0]:
                        adj[a, b] = adj[b, a] = False
                        break
            l += 1
        differ += int(total != Rp["tests_total"])
    assert differ > 0


@pytest.mark.parametrize("rev", [False, True])
def test_pathpool_population_recovers_the_skeleton(rev):
    for dag, W in _tiny_dags(30, 7500, pmin=5, pmax=8, max_edges=12):
        C = sem.population_corr(W)
        R = oracle.skeleton(C, 10 ** 9, 0.01, -1, reversed_order=rev, tol=1e-10, flags=oracle.PATHPOOL)
        np.testing.assert_array_equal(R["adj"], ((dag + dag.T) > 0).astype(np.uint8))


def test_four_node_example_conventional_count_with_the_papers_pool():
    # Sec. 3.1: with the paper's own pool adj(G,i,j) on i-j paths, Algorithm 1 runs the
    # printed 17 tests (PC-stable and non-stable alike on this example); the reversed
    # order runs 13 against the printed 14 (Reading R12)
    from tests.test_oracle import _four_node
    spec, indeps, dag, W = _four_node()
    C = sem.population_corr(W)
    for flags in (oracle.PATHPOOL, oracle.PATHPOOL | oracle.NONSTABLE):
        R = oracle.skeleton(C, 10 ** 9, 0.01, -1, False, flags=flags, tol=1e-10)
        assert R["tests_total"] == int(spec["count_pc"][0]) == 17
    R = oracle.skeleton(C, 10 ** 9, 0.01, -1, True, flags=oracle.PATHPOOL | oracle.STAGEA_GENERIC, tol=1e-10)
    assert R["tests_total"] == 13 and int(spec["count_pc_reverse"][0]) == 14
