"""Seeded synthetic linear-Gaussian SEM inputs (the paper's Sec. 6.1 recipe family).

This module draws inputs only -- it holds none of the skeleton search's
arithmetic -- and is the one module both the CUDA path's callers and the
oracle's tests use.  Every draw comes from ``numpy.random.Generator(PCG64(seed))``.

Recipe (Sec. 6.1, with the sizes of the benchmark workloads):
  * a DAG over a random topological order (a random permutation of 0..p-1);
  * each edge i -> j with i earlier than j present with probability ``prob``
    (Erdos-Renyi on the order), or, for the power-law workload, an in-degree
    drawn from pmf ~ (k+1)^-gamma on 0..max_in truncated at the number of
    earlier nodes, with parents uniform among the earlier nodes;
  * weights a_ij uniform on [-hi,-lo] U [lo,hi];
  * X_j = sum_i a_ij X_i + eps_j, eps_j ~ N(0,1), drawn in FP64 and cast to
    the workload's storage type (FP64 or FP32) afterwards.

Workloads (seed of instance s of workload c is 1000*c + s):
  1 ``p20_fp64``      p=20,  n=1000,  ER prob 0.2,  FP64
  2 ``p95_dense``     p=95,  n=5000,  ER prob 0.3,  FP32
  3 ``p500_powerlaw`` p=500, n=10000, power law mean degree 6, max in 40, FP32
  4 ``p1000_er``      p=1000,n=20000, ER prob 10/999, FP32
  5 ``many64``        64 instances, p~U[50,400], prob~U[0.05,0.3], n~U[2000,20000]

The paper's own simulation (Sec. 6.1, ``make_sweep``): a fixed order X_1..X_p,
edges i -> j (i < j) Bernoulli(5/(p-1)) so that a node has 5 neighbours on
average, then two hub nodes drawn uniformly whose neighbour sets are replaced by
10 uniformly drawn other nodes (directions by the order), weights uniform on
[-0.8,-0.2] U [0.2,0.8], eps ~ N(0,1).  The sample size is not stated there;
n = 5000 (the p = 95 workload's) is used.  Instance m of size p has seed
100000 + 100 p + m.

The power experiment (Sec. 6.4) uses a 10-node graph shown only in a figure that
the text does not carry; ``power_dag`` is a substitute with the relations the text
states: X5 and X6 separated by {X0} and by {X0,X1,X2,X3,X4,X7,X8}, X8 and X9
adjacent (dependent given {X0} and given {X0,...,X7}).  Dataset m has seed
200000 + m.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SEM:
    X: np.ndarray          # n x p samples, row-major, float64 or float32
    dag: np.ndarray        # p x p uint8, dag[i, j] = 1 iff i -> j
    weights: np.ndarray    # p x p float64, weights[i, j] = a_ij
    order: np.ndarray      # topological order (node ids)
    seed: int

    @property
    def skeleton(self) -> np.ndarray:
        return ((self.dag + self.dag.T) > 0).astype(np.uint8)


def _weights(rng, k, lo=0.1, hi=1.0):
    mag = rng.uniform(lo, hi, size=k)
    sign = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    return mag * sign


def er_dag(p: int, prob: float, rng, lo=0.1, hi=1.0):
    order = rng.permutation(p)
    dag = np.zeros((p, p), dtype=np.uint8)
    W = np.zeros((p, p), dtype=np.float64)
    for t in range(1, p):
        j = order[t]
        mask = rng.random(t) < prob
        pars = order[:t][mask]
        dag[pars, j] = 1
        W[pars, j] = _weights(rng, pars.size, lo, hi)
    return dag, W, order


def _powerlaw_mean(gamma: float, p: int, max_in: int) -> float:
    k = np.arange(max_in + 1, dtype=np.float64)
    w = (k + 1.0) ** (-gamma)
    tot = 0.0
    for t in range(p):
        m = min(max_in, t)
        ww = w[: m + 1]
        tot += float((k[: m + 1] * ww).sum() / ww.sum())
    return tot / p


def powerlaw_gamma(p: int, mean_total_degree: float = 6.0, max_in: int = 40) -> float:
    """gamma such that the expected in-degree, after truncation at the number of
    earlier nodes, is mean_total_degree / 2 (bisection, deterministic)."""
    target = mean_total_degree / 2.0
    lo, hi = 0.01, 6.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if _powerlaw_mean(mid, p, max_in) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw_dag(p: int, rng, mean_total_degree=6.0, max_in=40, lo=0.1, hi=1.0):
    gamma = powerlaw_gamma(p, mean_total_degree, max_in)
    k = np.arange(max_in + 1, dtype=np.float64)
    w = (k + 1.0) ** (-gamma)
    order = rng.permutation(p)
    dag = np.zeros((p, p), dtype=np.uint8)
    W = np.zeros((p, p), dtype=np.float64)
    for t in range(1, p):
        m = min(max_in, t)
        pm = w[: m + 1] / w[: m + 1].sum()
        kin = int(rng.choice(m + 1, p=pm))
        if kin == 0:
            continue
        pars = order[:t][rng.choice(t, size=kin, replace=False)]
        j = order[t]
        dag[pars, j] = 1
        W[pars, j] = _weights(rng, kin, lo, hi)
    return dag, W, order


def sample(W: np.ndarray, order: np.ndarray, n: int, rng) -> np.ndarray:
    """X (n x p, FP64) from X_j = sum_i W[i,j] X_i + eps_j in topological order."""
    p = W.shape[0]
    X = np.empty((n, p), dtype=np.float64)
    eps = rng.standard_normal((n, p))
    for j in order:
        pars = np.nonzero(W[:, j])[0]
        if pars.size:
            X[:, j] = X[:, pars] @ W[pars, j] + eps[:, j]
        else:
            X[:, j] = eps[:, j]
    return X


WORKLOADS = {
    1: dict(name="p20_fp64", p=20, n=1000, prob=0.2, dtype="float64", alpha=0.01, max_level=-1),
    2: dict(name="p95_dense", p=95, n=5000, prob=0.3, dtype="float32", alpha=0.01, max_level=-1),
    3: dict(name="p500_powerlaw", p=500, n=10000, prob=None, dtype="float32", alpha=0.01,
            max_level=8),
    4: dict(name="p1000_er", p=1000, n=20000, prob=10.0 / 999.0, dtype="float32", alpha=0.01,
            max_level=-1),
}


def make(cfg: int, instance: int = 0, n: int | None = None, p: int | None = None) -> SEM:
    """Instance ``instance`` of workload ``cfg`` (1..4); n/p override the size
    (same recipe, used for small parity cases)."""
    w = WORKLOADS[cfg]
    seed = 1000 * cfg + instance
    rng = np.random.Generator(np.random.PCG64(seed))
    pp = p if p is not None else w["p"]
    nn = n if n is not None else w["n"]
    if w["prob"] is None:
        dag, W, order = powerlaw_dag(pp, rng)
    else:
        prob = w["prob"] if p is None or cfg != 4 else 10.0 / (pp - 1)
        dag, W, order = er_dag(pp, prob, rng)
    X = sample(W, order, nn, rng)
    X = X.astype(np.float32) if w["dtype"] == "float32" else X
    return SEM(X=np.ascontiguousarray(X), dag=dag, weights=W, order=order, seed=seed)


def make_many(count: int = 64, base_seed: int = 5000, p_range=(50, 400),
              prob_range=(0.05, 0.3), n_range=(2000, 20000)) -> list[SEM]:
    """Workload 5: ``count`` independent FP32 instances with p, prob, n drawn
    uniformly (instance s uses seed base_seed + s)."""
    out = []
    for s in range(count):
        seed = base_seed + s
        rng = np.random.Generator(np.random.PCG64(seed))
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        prob = float(rng.uniform(*prob_range))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        dag, W, order = er_dag(p, prob, rng)
        X = sample(W, order, n, rng).astype(np.float32)
        out.append(SEM(X=np.ascontiguousarray(X), dag=dag, weights=W, order=order, seed=seed))
    return out


def hub_dag(p: int, rng, mean_degree: float = 5.0, hubs: int = 2, hub_degree: int = 10,
            lo: float = 0.2, hi: float = 0.8):
    """The Sec. 6.1 graph: Bernoulli(mean_degree/(p-1)) edges along the order 0..p-1,
    then ``hubs`` nodes whose neighbours are replaced by ``hub_degree`` random others."""
    A = np.triu(rng.random((p, p)) < mean_degree / (p - 1), 1)
    H = rng.choice(p, size=hubs, replace=False)
    A[H, :] = False
    A[:, H] = False
    for h in H:
        others = np.array([x for x in range(p) if x != h])
        for x in rng.choice(others, size=min(hub_degree, p - 1), replace=False):
            A[min(h, x), max(h, x)] = True
    dag = A.astype(np.uint8)
    W = np.zeros((p, p), dtype=np.float64)
    ii, jj = np.nonzero(A)
    W[ii, jj] = _weights(rng, ii.size, lo, hi)
    return dag, W, np.arange(p)


def make_sweep(p: int, instance: int, n: int = 5000, dtype=np.float32) -> SEM:
    """Instance ``instance`` of size p of the paper's simulation (Sec. 6.1)."""
    seed = 100000 + 100 * p + instance
    rng = np.random.Generator(np.random.PCG64(seed))
    dag, W, order = hub_dag(p, rng)
    X = sample(W, order, n, rng).astype(dtype)
    return SEM(np.ascontiguousarray(X), dag, W, order, seed)


POWER_EDGES = [(0, 5), (0, 6), (0, 1), (1, 2), (2, 3), (3, 4), (4, 7), (7, 8), (8, 9), (0, 8)]


def power_dag(seed: int = 199999):
    """The substitute 10-node DAG of the power experiment: X0 a common cause of the
    leaves X5 and X6, a chain X0 -> X1 -> ... -> X4 -> X7 -> X8 -> X9, and X0 -> X8;
    weights uniform on [-0.8,-0.2] U [0.2,0.8] (Sec. 6.1) drawn once."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dag = np.zeros((10, 10), dtype=np.uint8)
    W = np.zeros((10, 10), dtype=np.float64)
    for a, b in POWER_EDGES:
        dag[a, b] = 1
    ii, jj = np.nonzero(dag)
    W[ii, jj] = _weights(rng, ii.size, 0.2, 0.8)
    return dag, W, np.arange(10)


def make_power(m: int, n: int = 100000, dtype=np.float32) -> SEM:
    """Dataset m of the power experiment (Sec. 6.4): n samples of the substitute graph."""
    dag, W, order = power_dag()
    seed = 200000 + m
    X = sample(W, order, n, np.random.Generator(np.random.PCG64(seed))).astype(dtype)
    return SEM(np.ascontiguousarray(X), dag, W, order, seed)


def population_corr(W: np.ndarray) -> np.ndarray:
    """Population correlation of the SEM: Sigma = (I - B)^-T (I - B)^-1 with
    B = W (X = B^T X + eps), normalised to unit diagonal.  Used by tests that
    pin the oracle against d-separation."""
    p = W.shape[0]
    A = np.linalg.inv(np.eye(p) - W)          # X^T = eps^T (I - W)^-1
    S = A.T @ A
    d = np.sqrt(np.diag(S))
    return S / np.outer(d, d)
