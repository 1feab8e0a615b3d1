"""bench.py's accuracy scores of an oriented graph against the true DAG (Sec. 6.3)."""
import numpy as np

import bench


def test_dag_scores_hand_case():
    dag = np.zeros((4, 4), np.uint8)
    dag[0, 1] = dag[1, 2] = dag[3, 2] = 1                      # 0 -> 1 -> 2 <- 3
    codes = np.zeros((4, 4), np.int8)
    codes[0, 1], codes[1, 0] = 2, 3                            # right direction
    codes[1, 2] = codes[2, 1] = 1                              # undirected: a difference
    codes[3, 2], codes[2, 3] = 2, 3                            # right direction
    codes[0, 3] = codes[3, 0] = 1                              # extra edge
    tpr, fpr, shd = bench.dag_scores(codes, dag)
    assert tpr == 1.0 and abs(fpr - 1 / 3) < 1e-12 and shd == 2
    rev = codes.copy()
    rev[0, 1], rev[1, 0] = 3, 2                                # reversed edge: a difference
    assert bench.dag_scores(rev, dag)[2] == 3
    assert bench.dag_scores(np.zeros((4, 4), np.int8), dag) == (0.0, 0.0, 3)
