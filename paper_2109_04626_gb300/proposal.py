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
    """(quads int32 (R, 4), labels float32 (R,)) for the removed pairs of one run.
    Rows are grouped by stage (ascending), then by pair in the order of
    ``sepsets``, each pair's candidates ascending."""
    p = adj_final.shape[0]
    by_level: dict[int, list] = {}
    for (a, b), (lv, side, rank, nodes) in sepsets.items():
        by_level.setdefault(lv, []).append((a, b, side, nodes))
    base = adj_final.astype(bool)
    quads, labels = [], []
    for l in sorted(by_level):
        if l < 1 or l >= p - 2:
            continue
        items = by_level[l]
        # the frozen graph of stage l: pairs removed at this stage or later
        # (Algorithm 1), at this stage or earlier (Algorithm 2), were adjacent
        frozen = base.copy()
        for lv2, items2 in by_level.items():
            if (lv2 <= l) if reversed_order else (lv2 >= l):
                ab = np.array([(a, b) for a, b, _, _ in items2], dtype=np.int64)
                frozen[ab[:, 0], ab[:, 1]] = True
                frozen[ab[:, 1], ab[:, 0]] = True
        k = len(items)
        u = np.array([a if side == 0 else b for a, b, side, _ in items], dtype=np.int64)
        v = np.array([b if side == 0 else a for a, b, side, _ in items], dtype=np.int64)
        cand = frozen[u].copy()                  # (k, p): adj(u)
        cand[np.arange(k), v] = False            # \ {v}
        member = np.zeros((k, p), dtype=bool)
        for i, (_, _, _, nodes) in enumerate(items):
            member[i, list(nodes)] = True
        d = cand.sum(axis=1)
        pi, kk = np.nonzero(cand)
        q = np.empty((pi.size, 4), dtype=np.int32)
        q[:, 0] = u[pi]
        q[:, 1] = v[pi]
        q[:, 2] = kk
        q[:, 3] = l | (d[pi] << 16)
        quads.append(q)
        labels.append(member[pi, kk].astype(np.float32))
    if not quads:
        return np.zeros((0, 4), np.int32), np.zeros(0, np.float32)
    return np.concatenate(quads), np.concatenate(labels)


def collect(make_X, seeds, alpha: float, order: int, max_level: int = -1, precision: int = 2,
            max_rows_per_seed: int | None = None):
    """Runs the plain search on each seeded input and returns the feature rows
    (torch CUDA tensors, concatenated) and labels.  make_X(seed) -> X (n x p).
    max_rows_per_seed: keep at most this many rows of each run, drawn without
    replacement by a generator seeded with the run's seed (None: all rows)."""
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
            if max_rows_per_seed is not None and len(y) > max_rows_per_seed:
                keep = np.sort(np.random.Generator(np.random.PCG64(sd)).choice(len(y), max_rows_per_seed,
                                                                               replace=False))
                q, y = q[keep], y[keep]
            feats.append(fp.pc_mlp_features(pc.h, torch.from_numpy(np.ascontiguousarray(q)).cuda()))
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
