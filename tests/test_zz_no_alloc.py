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
