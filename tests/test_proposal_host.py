"""Host logic of the proposal training data (no GPU): rows come from the pairs a
plain run removed, on the frozen graph of their stage."""
import numpy as np

import oracle
from paper_2109_04626_gb300 import proposal, sem


def test_training_rows_rebuild_the_frozen_candidate_sets():
    rng = np.random.Generator(np.random.PCG64(77))
    dag, W, order = sem.er_dag(14, 0.35, rng)
    X = sem.sample(W, order, 700, rng)
    C = oracle.pearson(X)
    for rev in (False, True):
        R = oracle.skeleton(C, 700, 0.01, -1, reversed_order=rev)
        q, y = proposal.training_rows(R["adj"], R["sepsets"], rev)
        # every positive row is a member of the recorded sepset of its pair
        for (u, v, k, ld), lab in zip(q, y):
            l, d = ld & 0xffff, ld >> 16
            a, b = min(u, v), max(u, v)
            lv, side, rank, nodes = R["sepsets"][(a, b)]
            assert lv == l and ((u == a) == (side == 0))
            assert (k in nodes) == bool(lab)
        # per (pair, side) the rows list exactly d candidates, l of them positive
        groups = {}
        for (u, v, k, ld), lab in zip(q, y):
            groups.setdefault((u, v, ld), []).append(lab)
        for (u, v, ld), labs in groups.items():
            assert len(labs) == ld >> 16 and sum(labs) == (ld & 0xffff)


def test_training_rows_reproduce_recorded_ranks():
    # the rebuilt candidate list of each pair, enumerated lexicographically, has the
    # recorded sepset at the recorded rank -- so it is the oracle's frozen list
    import itertools
    rng = np.random.Generator(np.random.PCG64(78))
    dag, W, order = sem.er_dag(13, 0.4, rng)
    X = sem.sample(W, order, 600, rng)
    C = oracle.pearson(X)
    for rev in (False, True):
        R = oracle.skeleton(C, 600, 0.01, -1, reversed_order=rev)
        q, y = proposal.training_rows(R["adj"], R["sepsets"], rev)
        groups = {}
        for (u, v, k, ld), lab in zip(q, y):
            groups.setdefault((int(u), int(v), int(ld) & 0xffff), []).append(int(k))
        assert groups
        for (u, v, l), cand in groups.items():
            a, b = min(u, v), max(u, v)
            lv, side, rank, nodes = R["sepsets"][(a, b)]
            assert tuple(sorted(nodes)) == list(itertools.combinations(sorted(cand), l))[rank]
