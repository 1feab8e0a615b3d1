"""Brute-force d-separation (Definition of d-separation, Sec. 2.1) used to pin the
oracle's population-mode decisions.  Independent of any correlation arithmetic:
X _||_ Y | Z  iff X and Y are disconnected in the moral graph of the ancestral
set of X u Y u Z after deleting Z (Lauritzen's criterion, equivalent to the
path-blocking definition)."""
import numpy as np


def ancestors(dag: np.ndarray, nodes) -> set:
    out = set(nodes)
    stack = list(nodes)
    while stack:
        v = stack.pop()
        for u in np.nonzero(dag[:, v])[0]:
            u = int(u)
            if u not in out:
                out.add(u)
                stack.append(u)
    return out


def d_separated(dag: np.ndarray, x: int, y: int, Z) -> bool:
    Z = set(int(z) for z in Z)
    an = ancestors(dag, {x, y} | Z)
    idx = sorted(an)
    # moral graph on the ancestral set
    nbr = {v: set() for v in idx}
    for v in idx:
        pars = [int(u) for u in np.nonzero(dag[:, v])[0] if int(u) in an]
        for u in pars:
            nbr[u].add(v)
            nbr[v].add(u)
        for i in range(len(pars)):
            for j in range(i + 1, len(pars)):
                nbr[pars[i]].add(pars[j])
                nbr[pars[j]].add(pars[i])
    seen = {x}
    stack = [x]
    while stack:
        v = stack.pop()
        if v == y:
            return False
        for w in nbr[v]:
            if w in Z or w in seen:
                continue
            seen.add(w)
            stack.append(w)
    return True
