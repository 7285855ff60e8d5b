"""The benchmark's multi-process path on CPU: two gloo ranks aggregate their
per-rank time (max) and work (sum) the way bench.py does for --gpus N."""

import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      ODP_BENCH_BACKEND="gloo")
    import bench

    r, w, local, dist = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist is not None
    bench.barrier(dist)
    t_max = bench.max_over_ranks(dist, 10.0 + rank)
    work = bench.sum_over_ranks(dist, 100.0 * (rank + 1))
    q.put((rank, t_max, work))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_reference_arm_runs_only_on_rank0(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")

    class A:
        steps = 1
        warmup = 1

    bench.run_reference(A())
    assert capsys.readouterr().out == ""
