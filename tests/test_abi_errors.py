"""Error behaviour of the C-ABI without a GPU: every entry point that takes a
handle returns PC_ERR_ARG for a NULL handle (null or zero arguments everywhere
else) instead of faulting; pc_destroy(NULL) is a no-op; invalid sizes are
rejected before any CUDA call; and valid arguments on a machine without a CUDA
device fail with PC_ERR_CUDA -- the library has no CPU fallback.  The calls run
in a child process, so a crash fails the test instead of ending the session."""
import json
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastpc.h")

CHILD = r"""
import ctypes, json, math, sys
sys.path.insert(0, ROOT)
from paper_2109_04626_gb300 import fastpc
lib = fastpc.load()
res = {}
def zero(t):
    if t is None:
        return 0
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and not isinstance(t._type_, str):
        return None
    return 0
for name in NAMES:
    f = getattr(lib, name)
    res[name] = int(f(*[zero(t) for t in f.argtypes]))
lib.pc_destroy(None)
res["pc_threshold"] = math.isnan(lib.pc_threshold(None))
lib.pc_last_error(None)                               # must not fault
h = ctypes.c_void_p()
res["create_bad_n"] = int(lib.pc_create(3, 10, 0.01, -1, ctypes.byref(h)))
res["create_bad_p"] = int(lib.pc_create(1000, 1, 0.01, -1, ctypes.byref(h)))
res["create_bad_alpha"] = int(lib.pc_create(1000, 10, 0.0, -1, ctypes.byref(h)))
res["create_null_out"] = int(lib.pc_create(1000, 10, 0.01, -1, None))
n = (ctypes.c_int64 * 2)(1000, 1000)
p = (ctypes.c_int32 * 2)(10, 1)
res["batch_bad_p"] = int(lib.pc_create_batch(2, ctypes.cast(n, ctypes.c_void_p), ctypes.cast(p, ctypes.c_void_p),
                                             0.01, -1, ctypes.byref(h)))
res["noalloc_bad"] = int(lib.pc_corr_noalloc(None, 0, 0, 0, 0, None, 0, None))
# valid sizes but buffers that are not device memory of the current device (host
# arrays here): rejected by the pointer check before any launch
Xh = (ctypes.c_float * 32)()
Ch = (ctypes.c_double * 16)()
res["noalloc_not_device"] = int(lib.pc_corr_noalloc(ctypes.cast(Xh, ctypes.c_void_p), 0, 8, 4, 4,
                                                    ctypes.cast(Ch, ctypes.c_void_p), 4, None))
if WITH_CREATE:
    st = int(lib.pc_create(1000, 10, 0.01, -1, ctypes.byref(h)))
    res["create_valid"] = st
    res["create_handle_null"] = h.value is None
print(json.dumps(res))
"""


def handle_functions():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = set(re.findall(r"\b(pc_[a-z_0-9]+)\s*\(\s*(?:const\s+)?pc_handle\s*\*\s*\*?\s*\w+", src))
    return sorted(names - {"pc_destroy", "pc_threshold", "pc_last_error"})


def test_entry_points_reject_null_handles_and_fail_without_a_device():
    torch = pytest.importorskip("torch")
    no_gpu = not torch.cuda.is_available()
    from paper_2109_04626_gb300 import build as b
    b.build()
    names = handle_functions()
    assert len(names) >= 20 and "pc_skeleton" in names and "pc_skeleton_many" in names
    code = CHILD.replace("ROOT", repr(ROOT)).replace("NAMES", repr(names)).replace("WITH_CREATE", repr(no_gpu))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    arg = 1                                            # PC_ERR_ARG
    bad = {k: v for k, v in res.items() if k in names and v != arg}
    assert not bad, bad
    assert res["pc_threshold"] is True
    for k in ("create_bad_n", "create_bad_p", "create_bad_alpha", "create_null_out", "batch_bad_p",
              "noalloc_bad", "noalloc_not_device"):
        assert res[k] == arg, (k, res[k])
    if no_gpu:
        assert res["create_valid"] == 2 and res["create_handle_null"]   # PC_ERR_CUDA, no handle


def test_noalloc_binding_rejects_buffers_off_one_cuda_device():
    # the binding issues the call with X's device current and refuses buffers that
    # are not both CUDA tensors of that device, before the library is called
    torch = pytest.importorskip("torch")
    from paper_2109_04626_gb300 import fastpc
    X = torch.zeros((8, 4), dtype=torch.float32)
    C = torch.zeros((4, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        fastpc.pc_corr_noalloc(X, C)
    with pytest.raises(ValueError):
        fastpc.pc_corr_noalloc(X.to("meta"), C.to("meta"))
