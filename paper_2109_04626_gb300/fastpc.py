"""Thin ctypes binding of include/fastpc.h (argument marshalling only).

Every computation runs inside libfastpc.so (CUDA, sm_103a).  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is
missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfastpc.so")

PC_F32, PC_F64 = 0, 1
STATUS = ["PC_OK", "PC_ERR_ARG", "PC_ERR_CUDA", "PC_ERR_OOM", "PC_ERR_STATE", "PC_ERR_DOF",
          "PC_ERR_BUDGET", "PC_ERR_TIMEOUT", "PC_ERR_INTERNAL"]


class PCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")


class pc_stats(ctypes.Structure):
    _fields_ = [
        ("tests_executed", ctypes.c_uint64),
        ("tests_canonical", ctypes.c_uint64),
        ("tests_redecided", ctypes.c_uint64),
        ("band_hits", ctypes.c_uint64),
        ("guard_hits", ctypes.c_uint64),
        ("degenerate", ctypes.c_uint64),
        ("complement_tests", ctypes.c_uint64),
        ("edges_removed", ctypes.c_uint64),
        ("edges_kept", ctypes.c_uint64),
        ("max_abs_dz", ctypes.c_double),
        ("t_skeleton_ms", ctypes.c_double),
        ("flops", ctypes.c_double),
        ("flops_class", ctypes.c_double * 6),
        ("levels_run", ctypes.c_int32),
        ("stage_a_ran", ctypes.c_int32),
        ("first_level", ctypes.c_int32),
        ("queue_overflows", ctypes.c_int32),
        ("prec_builds", ctypes.c_uint64),
        ("prec_downdates", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["flops_class"] = list(self.flops_class)
        return d


_lib = None


def load():
    """Load libfastpc.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_2109_04626_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    cs = ctypes.c_char_p
    sig = {
        "pc_create": (i32, [i64, i32, dbl, i32, ctypes.POINTER(vp)]),
        "pc_destroy": (None, [vp]),
        "pc_set_opt": (i32, [vp, cs, dbl]),
        "pc_get_opt": (i32, [vp, cs, ctypes.POINTER(dbl)]),
        "pc_set_stream": (i32, [vp, vp]),
        "pc_corr": (i32, [vp, vp, i32, i64]),
        "pc_corr_get": (i32, [vp, vp, vp]),
        "pc_skeleton": (i32, [vp, vp, ctypes.POINTER(pc_stats)]),
        "pc_sepsets_count": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "pc_sepsets_get": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "pc_orient": (i32, [vp, vp, ctypes.POINTER(i32)]),
        "pc_ci_batch": (i32, [vp, vp, vp, i32, i64, vp, vp, vp]),
        "pc_last_stats": (i32, [vp, ctypes.POINTER(pc_stats)]),
        "pc_threshold": (dbl, [vp]),
        "pc_fisher_threshold": (dbl, [dbl]),
        "pc_kernel_launches": (i64, []),
        "pc_timing": (i32, [vp, vp, vp, i32]),
        "pc_corr_noalloc": (i32, [vp, i32, i64, i32, i64, vp, i64, vp]),
        "pc_skeleton_many": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(pc_stats),
                                   ctypes.POINTER(i32)]),
        "pc_autotune": (i32, [vp, i32, ctypes.POINTER(pc_tune_result)]),
        "pc_create_batch": (i32, [i32, vp, vp, dbl, i32, ctypes.POINTER(vp)]),
        "pc_corr_block": (i32, [vp, i32, vp, i32, i64]),
        "pc_corr_blocks": (i32, [vp, ctypes.POINTER(vp), vp, vp]),
        "pc_batch_layout": (i32, [vp, ctypes.POINTER(i32), vp]),
        "pc_mlp_nparam": (i32, []),
        "pc_mlp_set_params": (i32, [vp, vp, i64]),
        "pc_mlp_get_params": (i32, [vp, vp, i64]),
        "pc_mlp_features": (i32, [vp, vp, i64, vp]),
        "pc_mlp_forward": (i32, [vp, vp, i64, vp]),
        "pc_mlp_grad": (i32, [vp, vp, vp, i64, vp, ctypes.POINTER(dbl)]),
        "pc_mlp_train": (i32, [vp, vp, vp, i64, i32, i64, dbl, ctypes.POINTER(dbl)]),
        "pc_last_error": (cs, [vp]),
        "pc_status_string": (cs, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(h, st):
    if st != 0:
        msg = load().pc_last_error(h)
        raise PCError(st, msg.decode() if msg else "")


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()


def pc_create(n: int, p: int, alpha: float, max_level: int = -1):
    h = ctypes.c_void_p()
    st = load().pc_create(int(n), int(p), float(alpha), int(max_level), ctypes.byref(h))
    if st != 0:
        raise PCError(st, "pc_create")
    return h


def pc_destroy(h):
    load().pc_destroy(h)


def pc_set_opt(h, key: str, val: float):
    _check(h, load().pc_set_opt(h, key.encode(), float(val)))


def pc_get_opt(h, key: str) -> float:
    v = ctypes.c_double()
    _check(h, load().pc_get_opt(h, key.encode(), ctypes.byref(v)))
    return v.value


def pc_set_stream(h, stream):
    """stream: torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default)."""
    raw = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(h, load().pc_set_stream(h, ctypes.c_void_p(raw)))


def _x_args(X):
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X)
        assert X.dtype in (np.float32, np.float64)
        return X, (PC_F64 if X.dtype == np.float64 else PC_F32), X.shape[1]
    import torch
    assert X.dtype in (torch.float32, torch.float64) and X.stride(1) == 1
    return X, (PC_F64 if X.dtype == torch.float64 else PC_F32), X.stride(0)


def pc_create_batch(ns, ps, alpha: float, max_level: int = -1):
    """Batched handle over len(ns) independent problems (instance i: ns[i] x ps[i])."""
    k = len(ns)
    n_arr = np.ascontiguousarray(ns, dtype=np.int64)
    p_arr = np.ascontiguousarray(ps, dtype=np.int32)
    h = ctypes.c_void_p()
    st = load().pc_create_batch(k, n_arr.ctypes.data, p_arr.ctypes.data, float(alpha), int(max_level),
                                ctypes.byref(h))
    if st != 0:
        raise PCError(st, "pc_create_batch failed")
    return h


def pc_corr_block(h, i: int, X):
    """Instance i's data (n_i x p_i row-major, numpy host or torch CUDA tensor)."""
    X, dt, ld = _x_args(X)
    _check(h, load().pc_corr_block(h, int(i), ctypes.c_void_p(_ptr(X)), dt, int(ld)))


def pc_corr_blocks(h, Xs):
    """Every instance's data in one call (Xs[i] as pc_corr_block's X for instance i);
    the instances' correlation steps run concurrently on the handle's side streams."""
    args = [_x_args(X) for X in Xs]
    ptrs = (ctypes.c_void_p * len(args))(*[_ptr(a[0]) for a in args])
    dts = np.ascontiguousarray([a[1] for a in args], dtype=np.int32)
    lds = np.ascontiguousarray([a[2] for a in args], dtype=np.int64)
    _check(h, load().pc_corr_blocks(h, ptrs, dts.ctypes.data, lds.ctypes.data))


def pc_batch_layout(h):
    """First global node id of every instance plus the total (list of k + 1 ints)."""
    k = ctypes.c_int32()
    _check(h, load().pc_batch_layout(h, ctypes.byref(k), None))
    off = np.empty(k.value + 1, dtype=np.int32)
    _check(h, load().pc_batch_layout(h, ctypes.byref(k), off.ctypes.data))
    return [int(x) for x in off]


def pc_corr(h, X):
    """X: n x p row-major (torch CUDA tensor or numpy host array), float32 or float64."""
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X)
        dt = PC_F64 if X.dtype == np.float64 else PC_F32
        assert X.dtype in (np.float32, np.float64)
        ld = X.shape[1]
    else:
        import torch
        assert X.dtype in (torch.float32, torch.float64) and X.stride(1) == 1
        dt = PC_F64 if X.dtype == torch.float64 else PC_F32
        ld = X.stride(0)
    _check(h, load().pc_corr(h, ctypes.c_void_p(_ptr(X)), dt, int(ld)))


def pc_corr_get(h, p: int):
    C32 = np.empty((p, p), dtype=np.float32)
    C64 = np.empty((p, p), dtype=np.float64)
    _check(h, load().pc_corr_get(h, ctypes.c_void_p(_ptr(C32)), ctypes.c_void_p(_ptr(C64))))
    return C32, C64


def pc_skeleton(h, p: int, adj_out=None):
    """Returns (adjacency p x p uint8, stats dict).  adj_out may be a device tensor."""
    st = pc_stats()
    adj = adj_out if adj_out is not None else np.empty((p, p), dtype=np.uint8)
    _check(h, load().pc_skeleton(h, ctypes.c_void_p(_ptr(adj)), ctypes.byref(st)))
    return adj, st.as_dict()


def pc_skeleton_many(handles, ps, adj_out=True):
    """Concurrent searches of independent problems: handles (list of c_void_p, each
    after pc_corr, ideally each on its own stream), ps their p.  Returns
    (list of adjacency arrays or None, list of stats dicts, list of status codes);
    adj_out=False leaves the skeletons on the device (no copies)."""
    k = len(handles)
    H = (ctypes.c_void_p * k)(*[h.value for h in handles])
    S = (pc_stats * k)()
    st = (ctypes.c_int32 * k)()
    if adj_out:
        adjs = [np.empty((p, p), dtype=np.uint8) for p in ps]
        A = (ctypes.c_void_p * k)(*[a.ctypes.data for a in adjs])
        load().pc_skeleton_many(H, k, A, S, st)
    else:
        adjs = [None] * k
        load().pc_skeleton_many(H, k, None, S, st)
    status = [int(x) for x in st]
    return [a if s_ == 0 else None for a, s_ in zip(adjs, status)], [x.as_dict() for x in S], status


class pc_tune_result(ctypes.Structure):
    _fields_ = [("lane_chunk", ctypes.c_int32), ("lane_rounds", ctypes.c_int32),
                ("lane_blocks", ctypes.c_int32), ("direct_warps", ctypes.c_int32),
                ("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double), ("runs", ctypes.c_int32),
                ("learned_max_level", ctypes.c_int32)]


def pc_autotune(h, reps: int = 3) -> dict:
    """Launch-shape search of the test kernels (pc_autotune); returns the chosen
    shape and the mean skeleton times before and after."""
    r = pc_tune_result()
    _check(h, load().pc_autotune(h, int(reps), ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in pc_tune_result._fields_}


def pc_last_stats(h) -> dict:
    st = pc_stats()
    _check(h, load().pc_last_stats(h, ctypes.byref(st)))
    return st.as_dict()


def pc_sepsets(h, p: int) -> dict:
    """{(a, b): (level, side, rank, nodes tuple)} for every removed pair a < b."""
    lib = load()
    nr, pl = ctypes.c_int64(), ctypes.c_int64()
    _check(h, lib.pc_sepsets_count(h, ctypes.byref(nr), ctypes.byref(pl)))
    k = nr.value
    pairs = np.empty((max(k, 1), 2), dtype=np.int32)
    level = np.empty(max(k, 1), dtype=np.int32)
    side = np.empty(max(k, 1), dtype=np.int32)
    rank = np.empty(max(k, 1), dtype=np.int64)
    off = np.empty(max(k, 1), dtype=np.int64)
    pool = np.empty(max(pl.value, 1), dtype=np.int32)
    _check(h, lib.pc_sepsets_get(h, *(ctypes.c_void_p(_ptr(a)) for a in (pairs, level, side, rank, off, pool))))
    out = {}
    for i in range(k):
        a, b = int(pairs[i, 0]), int(pairs[i, 1])
        lv, o = int(level[i]), int(off[i])
        if o < 0:
            nodes = tuple(w for w in range(p) if w != a and w != b)
        else:
            nodes = tuple(int(x) for x in pool[o:o + lv])
        out[(a, b)] = (lv, int(side[i]), int(rank[i]), nodes)
    return out


# codes of pc_orient per ordered pair (a, b)
NO_EDGE, UNDIRECTED, FORWARD, BACKWARD, BIDIRECTED = 0, 1, 2, 3, 4


def pc_orient(h, p: int, out=None):
    """Phase II (Algorithm 1) on the last skeleton: (codes, rule rounds).  codes is a
    p x p int8 numpy array (or ``out``, a host array or CUDA tensor of that shape):
    0 no edge, 1 a - b, 2 a -> b, 3 a <- b, 4 a <-> b."""
    codes = out if out is not None else np.empty((p, p), dtype=np.int8)
    rounds = ctypes.c_int32()
    _check(h, load().pc_orient(h, ctypes.c_void_p(_ptr(codes)), ctypes.byref(rounds)))
    return codes, int(rounds.value)


def pc_ci_batch(h, ij, S, l: int, r_out=None, indep_out=None, z_out=None):
    """ij: (b,2) int32 CUDA tensor, S: (b,l) int32 CUDA tensor.  Returns (r, indep, z) tensors."""
    import torch
    b = ij.shape[0]
    dev = ij.device
    r = r_out if r_out is not None else torch.empty(b, dtype=torch.float64, device=dev)
    ind = indep_out if indep_out is not None else torch.empty(b, dtype=torch.uint8, device=dev)
    z = z_out if z_out is not None else torch.empty(b, dtype=torch.float32, device=dev)
    Sp = _ptr(S) if (S is not None and l > 0) else None
    _check(h, load().pc_ci_batch(h, ctypes.c_void_p(_ptr(ij)), ctypes.c_void_p(Sp), int(l), int(b),
                                 ctypes.c_void_p(_ptr(r)), ctypes.c_void_p(_ptr(ind)),
                                 ctypes.c_void_p(_ptr(z))))
    return r, ind, z


def pc_threshold(h) -> float:
    return float(load().pc_threshold(h))


def pc_fisher_threshold(alpha: float) -> float:
    """Phi^{-1}(1 - alpha/2) computed by the library's host code (no GPU needed)."""
    return float(load().pc_fisher_threshold(float(alpha)))


def pc_kernel_launches() -> int:
    return int(load().pc_kernel_launches())


# class "corr_gemm" (the correlation GEMM kernels alone) is a part of class "corr"
TIMING_CLASSES = ["corr", "stage_a", "prec", "ci_direct", "ci_complement", "bookkeeping", "scoring", "corr_gemm",
                  "stage_loop"]


def pc_timing(h, reset: bool = False) -> dict:
    """Per-kernel-class device ms and launch-group counts (option "timing" = 1)."""
    ms = np.zeros(len(TIMING_CLASSES), dtype=np.float64)
    cnt = np.zeros(len(TIMING_CLASSES), dtype=np.int64)
    _check(h, load().pc_timing(h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(cnt.ctypes.data),
                               1 if reset else 0))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(TIMING_CLASSES)}


def pc_corr_noalloc(X, C_out, stream=None):
    """FP64 correlation of X (n x p CUDA tensor, float32/float64, row-major)
    into C_out (p x p float64 CUDA tensor) with no device allocation; see
    include/fastpc.h.  Issued on ``stream`` (torch stream, raw handle or None)."""
    import torch
    if X.device.type != "cuda" or C_out.device != X.device:
        raise ValueError(f"pc_corr_noalloc: X and C_out must be CUDA tensors on one device "
                         f"(X on {X.device}, C_out on {C_out.device})")
    assert X.dtype in (torch.float32, torch.float64) and X.stride(1) == 1
    assert C_out.dtype == torch.float64 and C_out.stride(1) == 1
    n, p = X.shape
    dt = PC_F64 if X.dtype == torch.float64 else PC_F32
    raw = 0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    lib = load()
    with torch.cuda.device(X.device):          # the library checks both buffers against the current device
        st = lib.pc_corr_noalloc(ctypes.c_void_p(X.data_ptr()), dt, int(n), int(p), int(X.stride(0)),
                                 ctypes.c_void_p(C_out.data_ptr()), int(C_out.stride(0)),
                                 ctypes.c_void_p(raw))
    if st != 0:
        raise PCError(st, "pc_corr_noalloc: p must be <= 4096, n >= 2, device pointers of the current "
                          "device, valid dtype/strides")


def pc_mlp_nparam() -> int:
    return int(load().pc_mlp_nparam())


def pc_mlp_set_params(h, theta):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    _check(h, load().pc_mlp_set_params(h, ctypes.c_void_p(theta.ctypes.data), theta.size))


def pc_mlp_get_params(h) -> np.ndarray:
    out = np.empty(pc_mlp_nparam(), dtype=np.float32)
    _check(h, load().pc_mlp_get_params(h, ctypes.c_void_p(out.ctypes.data), out.size))
    return out


def pc_mlp_features(h, quads):
    """quads: (R, 4) int32 CUDA tensor (u, v, k, l | d << 16) -> (R, 16) float32 CUDA tensor."""
    import torch
    R = quads.shape[0]
    feats = torch.empty((R, 16), dtype=torch.float32, device=quads.device)
    _check(h, load().pc_mlp_features(h, ctypes.c_void_p(_ptr(quads)), R, ctypes.c_void_p(_ptr(feats))))
    return feats


def pc_mlp_forward(h, feats):
    import torch
    R = feats.shape[0]
    scores = torch.empty(R, dtype=torch.float32, device=feats.device)
    _check(h, load().pc_mlp_forward(h, ctypes.c_void_p(_ptr(feats)), R, ctypes.c_void_p(_ptr(scores))))
    return scores


def pc_mlp_grad(h, feats, labels):
    """(gradient as a numpy float32 vector, mean loss)."""
    g = np.empty(pc_mlp_nparam(), dtype=np.float32)
    loss = ctypes.c_double()
    _check(h, load().pc_mlp_grad(h, ctypes.c_void_p(_ptr(feats)), ctypes.c_void_p(_ptr(labels)),
                                 feats.shape[0], ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)))
    return g, loss.value


def pc_mlp_train(h, feats, labels, epochs: int, batch: int, lr: float) -> float:
    loss = ctypes.c_double()
    _check(h, load().pc_mlp_train(h, ctypes.c_void_p(_ptr(feats)), ctypes.c_void_p(_ptr(labels)),
                                  feats.shape[0], int(epochs), int(batch), float(lr), ctypes.byref(loss)))
    return loss.value


class PC:
    """Owning wrapper: ``with PC(n, p, alpha, max_level, order=1) as pc: ...``"""

    def __init__(self, n, p, alpha, max_level=-1, **opts):
        self.n, self.p = int(n), int(p)
        self.h = pc_create(n, p, alpha, max_level)
        for k, v in opts.items():
            pc_set_opt(self.h, k, v)

    def set(self, **opts):
        for k, v in opts.items():
            pc_set_opt(self.h, k, v)
        return self

    def corr(self, X):
        pc_corr(self.h, X)
        return self

    def skeleton(self, adj_out=None):
        return pc_skeleton(self.h, self.p, adj_out)

    def sepsets(self):
        return pc_sepsets(self.h, self.p)

    def orient(self, out=None):
        return pc_orient(self.h, self.p, out)

    def ci_batch(self, ij, S, l):
        return pc_ci_batch(self.h, ij, S, l)

    def corr_get(self):
        return pc_corr_get(self.h, self.p)

    @property
    def threshold(self):
        return pc_threshold(self.h)

    def close(self):
        if self.h is not None:
            pc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PCBatch(PC):
    """Batched handle over independent problems (pc_create_batch): instance i has
    ns[i] samples of ps[i] variables; give its data with corr_block(i, X)."""

    def __init__(self, ns, ps, alpha: float, max_level: int = -1, **opts):
        self.h = pc_create_batch(ns, ps, alpha, max_level)
        self.ns, self.ps = list(ns), list(ps)
        self.n, self.p = max(ns), int(sum(ps))
        self.offsets = pc_batch_layout(self.h)
        for k, v in opts.items():
            pc_set_opt(self.h, k, v)

    def corr(self, X):
        raise PCError(4, "a batched handle takes its data per instance: corr_block(i, X)")

    def corr_block(self, i, X):
        pc_corr_block(self.h, i, X)
        return self

    def corr_blocks(self, Xs):
        if len(Xs) != len(self.ps):
            raise ValueError("corr_blocks: one array per instance")
        pc_corr_blocks(self.h, Xs)
        return self

    def split(self, adj, sepsets=None):
        """Per-instance adjacency blocks and sepsets (local node ids)."""
        o = self.offsets
        adjs = [adj[o[i]:o[i + 1], o[i]:o[i + 1]] for i in range(len(self.ps))]
        if sepsets is None:
            return adjs
        seps = [dict() for _ in self.ps]
        import bisect
        for (a, b), (lv, side, rank, nodes) in sepsets.items():
            i = bisect.bisect_right(o, a) - 1
            seps[i][(a - o[i], b - o[i])] = (lv, side, rank, tuple(x - o[i] for x in nodes))
        return adjs, seps
