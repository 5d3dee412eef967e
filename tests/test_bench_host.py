"""Host-side logic of the benchmark's N-replica mode (one process per GPU):
the whole-job time is the slowest rank's and the work is summed.  Runs as
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, cells = bench.reduce_max_sum(dist, torch, 10.0 + rank, 1000.0 * (rank + 1), device="cpu")
    q.put((rank, t, cells))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, cells in out:
        assert t == 11.0 and cells == 3000.0


def test_single_process_passthrough():
    import torch
    import bench
    assert bench.reduce_max_sum(None, torch, 3.0, 7.0) == (3.0, 7.0)


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=5, warmup=3)
    assert bench.reference_arm(args) == 0
    assert capsys.readouterr().out == ""


def test_kernel_code_hash_follows_code_not_comments():
    """The roofline traffic is kept only while the kernel code is the one the
    ncu capture measured; comments and blank lines do not count."""
    import bench
    src = "int a = 1;  // one\n\n// note\nint b = a + 2;\n"
    same = "int a = 1;\n// another note\nint b = a + 2;   \n"
    changed = "int a = 1;\nint b = a + 3;\n"
    assert bench.kernel_code_hash(src) == bench.kernel_code_hash(same)
    assert bench.kernel_code_hash(src) != bench.kernel_code_hash(changed)
