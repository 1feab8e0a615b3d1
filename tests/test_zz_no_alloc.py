"""pc_corr_noalloc: the correlation step for callers that cannot call
cudaMalloc (applications whose device memory is reserved by their own pool or
budget, loops where an allocation would synchronise the device).  It must give
what the allocating entry point pc_corr gives, call after call, although every
call shares one file-scope device array for its column statistics.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_2109_04626_gb300 import sem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12          # the FP64 correlation tolerance the other GPU tests use


@pytest.fixture(scope="module")
def fp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_04626_gb300 import build
    from paper_2109_04626_gb300 import fastpc
    build.build()
    fastpc.load()
    return fastpc


def _reference_c64(fp, X):
    n, p = X.shape
    with fp.PC(n, p, 0.01, -1, precision=0) as pc:
        pc.corr(torch.from_numpy(X).cuda())
        _, C64 = pc.corr_get()
    return C64


def test_noalloc_matches_pc_corr_on_two_calls_in_a_row(fp):
    # two different inputs back to back: the second call must not see the first
    # call's statistics left in the shared array
    X1 = sem.make(2).X                                    # p=95, n=5000, FP32
    X2 = np.ascontiguousarray(sem.make(1).X)              # p=20, n=1000, FP64
    out = []
    for X in (X1, X2):
        n, p = X.shape
        C = torch.full((p, p), float("nan"), dtype=torch.float64, device="cuda")
        fp.pc_corr_noalloc(torch.from_numpy(X).cuda(), C)
        torch.cuda.synchronize()
        out.append(C.cpu().numpy())
    for X, C in zip((X1, X2), out):
        ref = _reference_c64(fp, X)
        assert np.isfinite(C).all()
        assert np.abs(C - ref).max() <= TOL
        assert np.all(np.diag(C) == 1.0)


def test_noalloc_small_then_large_with_shifted_means(fp):
    # a small problem, then a larger one whose columns have different, large means:
    # the second call must use its own statistics for every column, including the
    # columns beyond the first call's p (a wrong offset into the shared array shows)
    rng = np.random.default_rng(5)
    Xs = rng.standard_normal((300, 12)) + np.arange(12) * 3.0
    Xl = rng.standard_normal((700, 150)) @ (np.eye(150) + 0.1 * rng.standard_normal((150, 150)))
    Xl = Xl + 1000.0 * (1 + np.arange(150))[None, :] - 40.0
    for X in (Xs, Xl):
        n, p = X.shape
        C = torch.full((p, p), float("nan"), dtype=torch.float64, device="cuda")
        fp.pc_corr_noalloc(torch.from_numpy(X).cuda(), C)
        torch.cuda.synchronize()
        assert np.abs(C.cpu().numpy() - _reference_c64(fp, X)).max() <= 1e-10


def test_noalloc_strided_rows_leave_padding_untouched(fp):
    # X and C_out with row strides above p (ld > p, ldc > p): the padding columns
    # of C_out keep their sentinel and the p x p part equals pc_corr's
    X = sem.make(2).X                                     # p=95, n=5000, FP32
    n, p = X.shape
    Xpad = torch.full((n, p + 13), 7.0, dtype=torch.float32, device="cuda")
    Xpad[:, :p] = torch.from_numpy(X).cuda()
    Cpad = torch.full((p, p + 5), -3.25, dtype=torch.float64, device="cuda")
    fp.pc_corr_noalloc(Xpad[:, :p], Cpad[:, :p])
    torch.cuda.synchronize()
    out = Cpad.cpu().numpy()
    assert np.all(out[:, p:] == -3.25)
    assert np.abs(out[:, :p] - _reference_c64(fp, X)).max() <= TOL


def test_noalloc_at_its_maximum_p(fp):
    # p = 4096, the size the fixed array is sized for (few samples keep it quick)
    rng = np.random.default_rng(9)
    X = rng.standard_normal((64, 4096)) * (1 + np.arange(4096) % 7) + np.arange(4096) % 11
    C = torch.empty((4096, 4096), dtype=torch.float64, device="cuda")
    fp.pc_corr_noalloc(torch.from_numpy(X).cuda(), C)
    torch.cuda.synchronize()
    assert np.abs(C.cpu().numpy() - _reference_c64(fp, X)).max() <= 1e-10


def test_noalloc_repeat_same_input_is_stable(fp):
    X = sem.make(1).X
    n, p = X.shape
    Xd = torch.from_numpy(X).cuda()
    A = torch.empty((p, p), dtype=torch.float64, device="cuda")
    B = torch.empty((p, p), dtype=torch.float64, device="cuda")
    fp.pc_corr_noalloc(Xd, A)
    fp.pc_corr_noalloc(Xd, B)
    torch.cuda.synchronize()
    assert torch.equal(A, B)


def test_noalloc_rejects_sizes_beyond_its_maximum(fp):
    X = torch.zeros((8, 4097), dtype=torch.float32, device="cuda")
    C = torch.zeros((1, 1), dtype=torch.float64, device="cuda")    # never written
    with pytest.raises(fp.PCError) as e:
        fp.pc_corr_noalloc(X, C)
    assert e.value.status == 1
    with pytest.raises(fp.PCError):                                 # host buffers
        lib = fp.load()
        import ctypes
        Xh = np.zeros((8, 4), dtype=np.float32)
        Ch = np.zeros((4, 4), dtype=np.float64)
        st = lib.pc_corr_noalloc(ctypes.c_void_p(Xh.ctypes.data), 0, 8, 4, 4,
                                 ctypes.c_void_p(Ch.ctypes.data), 4, None)
        if st != 0:
            raise fp.PCError(st, "host pointers rejected")
