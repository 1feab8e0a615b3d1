"""Brute-force pin of the oracle's skeleton search in both schedules (Algorithm 1
and the reversed Algorithm 2, PC-stable, Sec. 2.2 and 3): a plain enumeration
written here -- every stage l freezes the adjacency, every adjacent pair tries
the l-subsets of adj(a)\\{b} and then of adj(b)\\{a} in lexicographic order, the
first independent set separates, all deletions of the stage happen at its end --
with each partial correlation taken from numpy's inverse of the (l+2)x(l+2)
correlation block instead of the oracle's elimination.  The removed pairs,
every separating set (stage, side, rank, members), the pairs that no set
separates and the sequential test counts per stage must agree (no GPU needed)."""
import itertools
import math
import statistics

import numpy as np
import pytest

import oracle
from paper_2109_04626_gb300 import sem


def _indep(C, n, u, v, S, q):
    """Fisher-z decision of X_u _|_ X_v | X_S from the inverse of the block (Sec. 2.2.2)."""
    idx = [u, v] + list(S)
    P = np.linalg.inv(C[np.ix_(idx, idx)])
    r = -P[0, 1] / math.sqrt(P[0, 0] * P[1, 1])
    z = math.sqrt(n - len(S) - 3) * abs(math.atanh(r))
    return z <= q, abs(z - q)


def _stable_stage(C, n, q, adj, l, seps):
    """One PC-stable stage l: every adjacent pair a < b tries the l-subsets of the
    frozen adj(a)\\{b}, then of adj(b)\\{a}, lexicographically; the first independent set
    separates; deletions happen after the whole stage.  Returns (tests, margin)."""
    p = C.shape[0]
    frozen = adj.copy()
    count, removed, margin = 0, [], math.inf
    for a in range(p):
        for b in range(a + 1, p):
            if not frozen[a, b]:
                continue
            found = None
            for side, (u, v) in enumerate(((a, b), (b, a))):
                cand = [w for w in range(p) if frozen[u, w] and w != v]
                for rank, S in enumerate(itertools.combinations(cand, l)):
                    count += 1
                    ind, m = _indep(C, n, u, v, S, q)
                    margin = min(margin, m)
                    if ind:
                        found = (l, side, rank, tuple(int(x) for x in S))
                        break
                if found:
                    break
            if found:
                seps[(a, b)] = found
                removed.append((a, b))
    for a, b in removed:
        adj[a, b] = adj[b, a] = False
    return count, margin


def _largest_candidate_set(adj):
    p = adj.shape[0]
    return max((int(adj[u].sum()) - 1 for u in range(p) for v in range(p) if adj[u, v]), default=-1)


def brute_pc_stable(C, n, alpha):
    """Algorithm 1: l = 0, 1, ... while some adjacent pair has |adj(u)\\{v}| >= l."""
    p = C.shape[0]
    q = -statistics.NormalDist().inv_cdf(alpha / 2)
    adj = np.ones((p, p), dtype=bool)
    np.fill_diagonal(adj, False)
    seps, tests_level, margin = {}, [], math.inf
    l = 0
    while _largest_candidate_set(adj) >= l:
        count, m = _stable_stage(C, n, q, adj, l, seps)
        tests_level.append(count)
        margin = min(margin, m)
        l += 1
    return adj.astype(np.uint8), seps, tests_level, margin


def brute_pc_reversed(C, n, alpha):
    """Algorithm 2 (reading R4): stage l = p-2 first, one test per pair with S every
    other node; then l = min(p-3, L*) and l <- min(l-1, L*) down to 0, L* the
    largest candidate set of the current graph.  Returns the visited levels too."""
    p = C.shape[0]
    q = -statistics.NormalDist().inv_cdf(alpha / 2)
    adj = np.ones((p, p), dtype=bool)
    np.fill_diagonal(adj, False)
    seps, tests = {}, {}
    margin = math.inf
    removed = []
    for a in range(p):
        for b in range(a + 1, p):
            rest = [w for w in range(p) if w != a and w != b]
            ind, m = _indep(C, n, a, b, rest, q)
            margin = min(margin, m)
            if ind:
                seps[(a, b)] = (p - 2, 0, 0, tuple(rest))
                removed.append((a, b))
    tests[p - 2] = p * (p - 1) // 2
    for a, b in removed:
        adj[a, b] = adj[b, a] = False
    levels = [p - 2]
    l = min(p - 3, _largest_candidate_set(adj))
    while l >= 0:
        levels.append(l)
        tests[l], m = _stable_stage(C, n, q, adj, l, seps)
        margin = min(margin, m)
        l = min(l - 1, _largest_candidate_set(adj))
    return adj.astype(np.uint8), seps, tests, levels, margin


@pytest.mark.parametrize("case", [(5101, 6, 300, 0.5), (5102, 8, 500, 0.45), (5103, 9, 2000, 0.4),
                                  (5104, 10, 800, 0.35), (5105, 7, 150, 0.6), (5106, 11, 5000, 0.3)])
def test_conventional_skeleton_equals_brute_force(case):
    seed, p, n, prob = case
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    X = sem.sample(W, order, n, rng)
    C = oracle.pearson(X)
    alpha = 0.01
    adj, seps, tests_level, margin = brute_pc_stable(C, n, alpha)
    # the two CI routes may round differently only for a statistic at the threshold itself
    assert margin > 1e-9
    R = oracle.skeleton(C, n, alpha, -1, reversed_order=False)
    np.testing.assert_array_equal(R["adj"], adj)
    assert R["sepsets"] == seps
    assert [int(t) for t in R["tests_level"][:len(tests_level)]] == tests_level
    assert R["tests_total"] == sum(tests_level)
    assert R["levels"] == list(range(len(tests_level)))


def test_brute_force_cases_reach_several_stages():
    # the cases above are not trivial: some remove pairs beyond stage 1
    deep = 0
    for seed, p, n, prob in [(5102, 8, 500, 0.45), (5104, 10, 800, 0.35), (5106, 11, 5000, 0.3)]:
        rng = np.random.Generator(np.random.PCG64(seed))
        dag, W, order = sem.er_dag(p, prob, rng)
        X = sem.sample(W, order, n, rng)
        _, seps, tests_level, _ = brute_pc_stable(oracle.pearson(X), n, 0.01)
        deep += sum(1 for v in seps.values() if v[0] >= 2)
        assert len(tests_level) >= 3
    assert deep > 0


@pytest.mark.parametrize("case", [(5201, 7, 400, 0.5), (5202, 9, 1500, 0.4), (5203, 10, 3000, 0.35),
                                  (5204, 8, 200, 0.6)])
def test_reversed_skeleton_equals_brute_force(case):
    seed, p, n, prob = case
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = sem.er_dag(p, prob, rng)
    X = sem.sample(W, order, n, rng)
    C = oracle.pearson(X)
    adj, seps, tests, levels, margin = brute_pc_reversed(C, n, 0.01)
    assert margin > 1e-9
    R = oracle.skeleton(C, n, 0.01, -1, reversed_order=True)
    assert R["stageA_ran"]
    np.testing.assert_array_equal(R["adj"], adj)
    assert R["sepsets"] == seps
    assert R["levels"] == levels
    assert {l: int(R["tests_level"][l]) for l in levels} == tests
    assert R["tests_total"] == sum(tests.values())
    # the reversed order really visits intermediate stages and removes pairs in them
    assert len(levels) >= 3 and any(0 < v[0] < p - 2 for v in seps.values())
