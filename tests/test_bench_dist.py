"""The benchmark's multi-process plumbing on the host: two ranks over gloo
(world size 2), as torchrun would start them, exercise the rendezvous, the
timing barrier, the max-over-ranks reduction and the whole-job rate, and
check that the reference arm runs on rank 0 only (the other ranks return 0
without work or output).  No GPU and no collective on the data path: the
benchmark runs independent replicas."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                           "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
        sys.path.insert(0, ROOT)
        import torch.distributed as dist

        import bench
        r, w, local = bench.dist_setup(world)
        bench.barrier(w)
        # ranks report different elapsed times; every rank must see the slowest
        t = bench.max_over_ranks(0.5 * (rank + 1), w)
        rate = bench.job_rate(3, w, t)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            ref = bench.reference_arm(types.SimpleNamespace(n=64, m=1, steps=1, warmup=0, gpus=w,
                                                            kappas="1e2")) if rank != 0 else None
        bench.barrier(w)
        dist.destroy_process_group()
        q.put((rank, r, w, local, dist.is_available(), t, rate, ref, out.getvalue()))
    except Exception as e:  # noqa: BLE001 -- reported to the parent
        q.put((rank, "error", repr(e)))


def test_two_ranks_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = {}
    try:
        for _ in range(world):
            item = q.get(timeout=180)
            res[item[0]] = item
    finally:
        for p in ps:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for rank in range(world):
        item = res[rank]
        assert item[1] != "error", item
        _, r, w, local, _, t, rate, ref, printed = item
        assert (r, w, local) == (rank, world, rank)
        assert t == pytest.approx(1.0)          # the slower rank's time, on both ranks
        assert rate == pytest.approx(6.0)       # 3 units per rank x 2 ranks / 1.0 s
        if rank != 0:
            assert ref == 0 and printed == ""   # the reference arm: rank 0 alone works and prints


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.get(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        for k in env:
            os.environ.pop(k, None)
        r, w, local = bench.dist_setup(1)
        assert (r, w, local) == (0, 1, 0)
        bench.barrier(w)
        assert bench.max_over_ranks(2.5, w) == 2.5
        assert bench.job_rate(3, 1, 0.1) == pytest.approx(30.0)
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v
