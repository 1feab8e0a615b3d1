"""Brute-force pin of the oracle's conventional skeleton search (Algorithm 1,
PC-stable, Sec. 2.2): a plain enumeration written here -- every stage l freezes
the adjacency, every adjacent pair tries the l-subsets of adj(a)\\{b} and then of
adj(b)\\{a} in lexicographic order, the first independent set separates, all
deletions of the stage happen at its end -- with each partial correlation taken
from numpy's inverse of the (l+2)x(l+2) correlation block instead of the
oracle's elimination.  The removed pairs, every separating set (stage, side,
rank, members), the pairs that no set separates and the sequential test counts
per stage must agree (no GPU needed)."""
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


def brute_pc_stable(C, n, alpha):
    p = C.shape[0]
    q = -statistics.NormalDist().inv_cdf(alpha / 2)
    adj = np.ones((p, p), dtype=bool)
    np.fill_diagonal(adj, False)
    seps, tests_level, margin = {}, [], math.inf
    l = 0
    while any(adj[u, v] and adj[u].sum() - 1 >= l for u in range(p) for v in range(p)):
        frozen = adj.copy()
        count, removed = 0, []
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
        tests_level.append(count)
        l += 1
    return adj.astype(np.uint8), seps, tests_level, margin


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
