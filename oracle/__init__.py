"""FP64 CPU oracle for the PC-stable skeleton search of arXiv 2109.04626.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference leg may import this package.  The
product path (``paper_2109_04626_gb300``) never imports, links or calls it, and
the two share no code.

The arithmetic lives in ``pc_oracle.c`` (plain C, FP64, optional OpenMP over
the edges of one PC-stable stage); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Paper passages followed (see the C file for each routine):
  * Pearson corr: Sec. 4 (definition of ``corr``).
  * Partial correlation: Sec. 4, H = H0 - H1 H2^-1 H1^T, rho = h12/sqrt(h11 h22).
  * Fisher-z test: Sec. 2.2.2, Eq. 1 and the rule that replaces Alg. 1's independence query.
  * Skeleton: Algorithm 1 (conventional) and Algorithm 2 (reversed order),
    PC-stable deletion at the end of each stage; the path-restricted pool
    adj(G,i,j) on i-j paths (Sec. 2.1 notation, switch PATHPOOL); Algorithm 3,
    the batched form of Algorithm 2 (Sec. 4, ``skeleton_batched``).
  * Orientation: Algorithm 1, Phase II (unshielded colliders, rules R1-R4),
    which Algorithm 2 shares (Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pc_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

REVERSED = 1
NONSTABLE = 2
ONESIDED_I = 4
ONESIDED_J = 8
STAGEA_GENERIC = 16
NO_STAGEA = 32
POPULATION = 64
PATHPOOL = 128     # one candidate pool per pair: adj(G,a,b) on a-b paths (PC-stable search)


def build(force: bool = False) -> str:
    """Compile pc_oracle.c into _liboracle.so with gcc (-O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_norm_ppf.restype = ctypes.c_double
        lib.oracle_norm_ppf.argtypes = [ctypes.c_double]
        lib.oracle_pearson.restype = None
        lib.oracle_pearson.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, dp]
        lib.oracle_partial_corr.restype = ctypes.c_int
        lib.oracle_partial_corr.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ip, ctypes.c_int32, dp, dp, dp]
        lib.oracle_ci_test.restype = ctypes.c_int
        lib.oracle_ci_test.argtypes = [dp, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ip,
                                       ctypes.c_int32, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_precision.restype = ctypes.c_int
        lib.oracle_precision.argtypes = [dp, ctypes.c_int32, dp]
        lib.oracle_skeleton.restype = ctypes.c_void_p
        lib.oracle_skeleton.argtypes = [dp, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int32, ctypes.c_int]
        lib.oracle_skeleton_batched.restype = ctypes.c_void_p
        lib.oracle_skeleton_batched.argtypes = [dp, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int32, ctypes.c_int64]
        lib.oracle_result_free.restype = None
        lib.oracle_result_free.argtypes = [ctypes.c_void_p]
        lib.oracle_result_copy.restype = None
        lib.oracle_result_copy.argtypes = [ctypes.c_void_p, u8p, ip, ip, lp, lp, lp, lp, ip]
        lib.oracle_result_pool_len.restype = ctypes.c_int64
        lib.oracle_result_pool_len.argtypes = [ctypes.c_void_p]
        lib.oracle_result_pool.restype = None
        lib.oracle_result_pool.argtypes = [ctypes.c_void_p, ip]
        lib.oracle_result_scalars.restype = None
        lib.oracle_result_scalars.argtypes = [ctypes.c_void_p, lp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        u8 = ctypes.POINTER(ctypes.c_uint8)
        i64 = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_meek.restype = ctypes.c_int32
        lib.oracle_meek.argtypes = [u8, u8, ctypes.c_int32]
        lib.oracle_codes.restype = None
        lib.oracle_codes.argtypes = [u8, u8, ctypes.c_int32, ctypes.POINTER(ctypes.c_int8)]
        lib.oracle_orient.restype = ctypes.c_int32
        lib.oracle_orient.argtypes = [u8, ctypes.c_int32, i64, ip, ip, ctypes.POINTER(ctypes.c_int8)]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def norm_ppf(p: float) -> float:
    """Phi^{-1}(p) by Wichura's AS241 (PPND16)."""
    return float(_load().oracle_norm_ppf(float(p)))


def threshold(alpha: float) -> float:
    """q = Phi^{-1}(1 - alpha/2), the two-sided Fisher-z threshold (Sec. 2.2.2).

    Evaluated as -Phi^{-1}(alpha/2) (symmetry of the normal law): the lower-tail
    argument alpha/2 is exact in floating point, whereas 1 - alpha/2 rounds."""
    return -norm_ppf(alpha / 2.0)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def pearson(X) -> np.ndarray:
    """Pearson correlation of the columns of X (n x p), FP64, diag = 1."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, p = X.shape
    C = np.empty((p, p), dtype=np.float64)
    _load().oracle_pearson(_dp(X), n, p, _dp(C))
    return C


def partial_corr(C, u: int, v: int, S):
    """(r, h11, h22, degenerate) for r_{uv.S} via the Schur complement of Sec. 4."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    S = np.ascontiguousarray(np.asarray(S, dtype=np.int32).reshape(-1))
    r = ctypes.c_double()
    h11 = ctypes.c_double()
    h22 = ctypes.c_double()
    dg = _load().oracle_partial_corr(_dp(C), C.shape[1], int(u), int(v), _ip(S), S.size,
                                     ctypes.byref(r), ctypes.byref(h11), ctypes.byref(h22))
    return r.value, h11.value, h22.value, bool(dg)


def ci_test(C, n: int, alpha: float, u: int, v: int, S, tol: float = -1.0):
    """(independent, r, z, degenerate) of one Gaussian CI test."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    S = np.ascontiguousarray(np.asarray(S, dtype=np.int32).reshape(-1))
    r = ctypes.c_double()
    z = ctypes.c_double()
    dg = ctypes.c_int()
    ind = _load().oracle_ci_test(_dp(C), C.shape[1], int(n), threshold(alpha), float(tol),
                                 int(u), int(v), _ip(S), S.size, ctypes.byref(r),
                                 ctypes.byref(z), ctypes.byref(dg))
    return bool(ind), r.value, z.value, bool(dg.value)


def ci_batch(C, n: int, alpha: float, ij, S):
    """Vectorised convenience over rows of (ij[b,2], S[b,l]): returns r, z, indep, degen."""
    ij = np.asarray(ij, dtype=np.int32)
    S = np.asarray(S, dtype=np.int32).reshape(ij.shape[0], -1)
    b = ij.shape[0]
    r = np.empty(b)
    z = np.empty(b)
    ind = np.empty(b, dtype=bool)
    dg = np.empty(b, dtype=bool)
    for k in range(b):
        ind[k], r[k], z[k], dg[k] = ci_test(C, n, alpha, ij[k, 0], ij[k, 1], S[k])
    return r, z, ind, dg


def precision(C):
    """(P, singular): P = C^{-1} by Gauss-Jordan elimination (FP64)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    p = C.shape[0]
    P = np.empty_like(C)
    sing = _load().oracle_precision(_dp(C), p, _dp(P))
    return P, bool(sing)


def skeleton(C, n: int, alpha: float, max_level: int = -1, reversed_order: bool = True,
             flags: int = 0, tol: float = -1.0) -> dict:
    """Run Phase I (Algorithm 1 or 2, PC-stable unless NONSTABLE is in flags).

    Returns a dict with ``adj`` (p x p uint8), ``sepsets`` {(a,b): (level, side,
    rank, nodes tuple)} for a<b, ``tests_level`` (int64 per level),
    ``removed_level``, ``tests_total``, ``degenerate``, ``stageA_ran`` and
    ``levels`` (the visited levels in order).  ``tol >= 0`` selects population
    mode (independent iff |r| <= tol).
    """
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    p = C.shape[0]
    f = int(flags) | (REVERSED if reversed_order else 0)
    if tol >= 0.0:
        f |= POPULATION
    q = threshold(alpha)
    R = lib.oracle_skeleton(_dp(C), p, int(n), q, float(tol), int(max_level), f)
    return _unpack(lib, R, p)


def skeleton_batched(C, n: int, alpha: float, batch: int, max_level: int = -1, tol: float = -1.0) -> dict:
    """Algorithm 3 (the batched form of Algorithm 2, Sec. 4): the tests of a stage
    are queued pair by pair over the path-restricted pools (Reading R19) and
    decided ``batch`` at a time, each batch's deletions applied before the next
    is formed (Reading R20 for the partial batches).  Same result dict as
    ``skeleton``; every separating set is recorded on side 0."""
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    p = C.shape[0]
    R = lib.oracle_skeleton_batched(_dp(C), p, int(n), threshold(alpha), float(tol), int(max_level), int(batch))
    return _unpack(lib, R, p)


def _unpack(lib, R, p: int) -> dict:
    try:
        pp = p * p
        adj = np.empty(pp, dtype=np.uint8)
        sl = np.empty(pp, dtype=np.int32)
        ss = np.empty(pp, dtype=np.int32)
        sr = np.empty(pp, dtype=np.int64)
        so = np.empty(pp, dtype=np.int64)
        tl = np.empty(p + 1, dtype=np.int64)
        rl = np.empty(p + 1, dtype=np.int64)
        ls = np.empty(p + 1, dtype=np.int32)
        lib.oracle_result_copy(R, adj.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _ip(sl),
                               _ip(ss), sr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               so.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               tl.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               rl.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ip(ls))
        plen = lib.oracle_result_pool_len(R)
        pool = np.empty(max(plen, 1), dtype=np.int32)
        lib.oracle_result_pool(R, _ip(pool))
        sc = np.empty(4, dtype=np.int64)
        lib.oracle_result_scalars(R, sc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    finally:
        lib.oracle_result_free(R)
    adj = adj.reshape(p, p)
    sl = sl.reshape(p, p)
    sepsets = {}
    for a in range(p):
        for b in range(a + 1, p):
            lv = int(sl[a, b])
            if lv < 0:
                continue
            off = int(so[a * p + b])
            if off < 0:
                nodes = tuple(w for w in range(p) if w != a and w != b)
            else:
                nodes = tuple(int(x) for x in pool[off:off + lv])
            sepsets[(a, b)] = (lv, int(ss[a * p + b]), int(sr[a * p + b]), nodes)
    return {
        "adj": adj,
        "sepsets": sepsets,
        "tests_level": tl,
        "removed_level": rl,
        "tests_total": int(sc[0]),
        "degenerate": int(sc[1]),
        "stageA_ran": bool(sc[2]),
        "levels": [int(x) for x in ls[: int(sc[3])]],
    }


# --------------------------------------------------------------------------- Phase II
# Codes of an oriented graph, per ordered pair (a, b): 0 no edge, 1 a - b,
# 2 a -> b, 3 a <- b, 4 a <-> b (two colliders or rules disagree).
NONE, UNDIRECTED, FORWARD, BACKWARD, BIDIRECTED = 0, 1, 2, 3, 4


def _u8p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def orient(adj, sepsets) -> tuple:
    """Phase II of Algorithm 1 on a skeleton and its separation sets.

    ``sepsets`` maps (a, b) to the separating set's nodes, or to a skeleton()
    record (level, side, rank, nodes); a pair missing from it decides no
    collider.  Returns (codes p x p int8, rule rounds)."""
    lib = _load()
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    p = adj.shape[0]
    off = np.full(p * p, -2, dtype=np.int64)
    ln = np.zeros(p * p, dtype=np.int32)
    pool = []
    for (a, b), v in sepsets.items():
        nodes = v[3] if isinstance(v, tuple) and len(v) == 4 and isinstance(v[3], tuple) else v
        e = min(a, b) * p + max(a, b)
        if nodes is None:
            off[e] = -1
            continue
        off[e] = len(pool)
        ln[e] = len(nodes)
        pool.extend(int(x) for x in nodes)
    pool_a = np.ascontiguousarray(pool if pool else [0], dtype=np.int32)
    out = np.empty(p * p, dtype=np.int8)
    rounds = lib.oracle_orient(_u8p(adj), p, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ip(ln),
                               _ip(pool_a), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return out.reshape(p, p), int(rounds)


def meek(adj, marks) -> tuple:
    """Rules R1-R4 (Algorithm 1, Phase II) on a partially directed graph given by
    its skeleton and arrowhead marks (marks[a, b] = 1: arrowhead at b on {a,b}).
    Returns (codes, rule rounds)."""
    lib = _load()
    adj = np.ascontiguousarray(adj, dtype=np.uint8)
    mk = np.ascontiguousarray(marks, dtype=np.uint8).copy()
    p = adj.shape[0]
    rounds = lib.oracle_meek(_u8p(adj), _u8p(mk), p)
    out = np.empty(p * p, dtype=np.int8)
    lib.oracle_codes(_u8p(adj), _u8p(mk), p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return out.reshape(p, p), int(rounds)
