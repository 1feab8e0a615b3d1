"""The N>1 path of bench.py on CPU: two gloo ranks (one process each, rendezvous
on 127.0.0.1) run its barrier and its max / sum over ranks, and the reference
arm runs on rank 0 only."""
import contextlib
import io
import json
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(None)
    bench.barrier(w)
    mx = bench.max_over_ranks(1.5 + r, w)
    sm = bench.sum_over_ranks(10.0 * (r + 1), w)
    bench.barrier(w)
    dist.destroy_process_group()
    # reference arm: rank 0 prints one line, the other ranks exit without work
    out = io.StringIO()
    ns = bench.argparse.Namespace(workload="p20_fp64", steps=1, warmup=0, gpus=world, impl="reference")
    with contextlib.redirect_stdout(out):
        rc = bench.run_reference(ns)
    q.put((r, w, mx, sm, rc, out.getvalue()))


def test_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p_ in ps:
        p_.start()
    res = sorted(q.get(timeout=300) for _ in ps)
    for p_ in ps:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    (r0, w0, mx0, sm0, rc0, out0), (r1, w1, mx1, sm1, rc1, out1) = res
    assert (w0, w1) == (2, 2)
    assert mx0 == mx1 == 2.5
    assert sm0 == sm1 == 30.0
    assert rc0 == 0 and rc1 == 0
    assert out1 == ""                                   # rank 1: no reference work
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
