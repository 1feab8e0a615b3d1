"""Training data and training loop for the conditioning-set proposal network.

The network (see include/fastpc.h, pc_mlp_*) scores every candidate k of an
ordered pair (u, v); the skeleton search then enumerates the sets of that pair
in the order the scores propose.  It learns from the outcomes of the plain
(lexicographic) search: for every pair a plain run removed at a stage l >= 1,
each candidate of the side that found the separating set S is one row, labelled
1 if it belongs to S.  The frozen graph of stage l is rebuilt from the final
skeleton and the removal stages (Algorithm 1: pairs removed at stages >= l were
still adjacent at stage l; Algorithm 2: those removed at stages <= l).

All arithmetic of features, forward, backward and Adam runs in libfastpc; this
module only assembles index rows and drives the calls.
"""
from __future__ import annotations

import numpy as np

from . import fastpc as fp


def training_rows(adj_final: np.ndarray, sepsets: dict, reversed_order: bool):
    """(quads int32 (R, 4), labels float32 (R,)) for the removed pairs of one run."""
    p = adj_final.shape[0]
    by_level: dict[int, list] = {}
    for (a, b), (lv, side, rank, nodes) in sepsets.items():
        by_level.setdefault(lv, []).append((a, b, side, nodes))
    quads, labels = [], []
    for l, items in by_level.items():
        if l < 1 or l >= p - 2:
            continue
        frozen = adj_final.astype(bool).copy()
        for lv2, items2 in by_level.items():
            if (lv2 <= l) if reversed_order else (lv2 >= l):
                for a, b, _, _ in items2:
                    frozen[a, b] = frozen[b, a] = True
        for a, b, side, nodes in items:
            u, v = (a, b) if side == 0 else (b, a)
            cand = [int(k) for k in np.nonzero(frozen[u])[0] if k != v]
            d = len(cand)
            S = set(nodes)
            for k in cand:
                quads.append((u, v, k, l | (d << 16)))
                labels.append(1.0 if k in S else 0.0)
    if not quads:
        return np.zeros((0, 4), np.int32), np.zeros(0, np.float32)
    return np.asarray(quads, dtype=np.int32), np.asarray(labels, dtype=np.float32)


def collect(make_X, seeds, alpha: float, order: int, max_level: int = -1, precision: int = 2):
    """Runs the plain search on each seeded input and returns the feature rows
    (torch CUDA tensors, concatenated) and labels.  make_X(seed) -> X (n x p)."""
    import torch
    feats, labs = [], []
    for sd in seeds:
        X = make_X(sd)
        n, p = X.shape
        with fp.PC(n, p, alpha, max_level, order=order, precision=precision) as pc:
            pc.corr(torch.from_numpy(np.ascontiguousarray(X)).cuda())
            adj, _ = pc.skeleton()
            q, y = training_rows(adj, pc.sepsets(), bool(order))
            if len(y) == 0:
                continue
            feats.append(fp.pc_mlp_features(pc.h, torch.from_numpy(q).cuda()))
            labs.append(torch.from_numpy(y).cuda())
    return torch.cat(feats), torch.cat(labs)


def initial_params(seed: int) -> np.ndarray:
    """He-uniform initial parameters from a seeded generator (an input, not arithmetic
    of the method)."""
    nh, nf = 128, 16
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.uniform(-1, 1, nh * nf) * np.sqrt(6.0 / nf), np.zeros(nh),
             rng.uniform(-1, 1, nh * nh) * np.sqrt(6.0 / nh), np.zeros(nh),
             rng.uniform(-1, 1, nh) * np.sqrt(6.0 / nh), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(handle, feats, labels, epochs: int = 8, batch: int = 16384, lr: float = 2e-3, seed: int = 0):
    """Shuffles the rows (seeded) and trains the handle's network with Adam; returns
    the mean loss of the last epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(feats.shape[0], generator=g).to(feats.device)
    f = feats[perm].contiguous()
    y = labels[perm].contiguous()
    fp.pc_mlp_set_params(handle, initial_params(seed))
    return fp.pc_mlp_train(handle, f, y, epochs, batch, lr)
