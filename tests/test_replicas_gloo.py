"""Replicas-only multi-GPU plumbing of bench.py on CPU ranks (gloo,
world size 2): the process group, the timing barrier, the max over ranks
that the whole-job value divides by, and the reference arm's rank rule."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init(world, backend="gloo")
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    ms = bench.max_over_ranks(1.5 + rank, w)           # rank 1 is the slow one
    out[rank] = (ms, bench.whole_job_value(1000, 10, ms, w))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 2.5e-3)


def test_whole_job_value_single_rank():
    import bench
    assert bench.whole_job_value(846369, 320, 2.0, 1) == pytest.approx(846369 * 320 / 2e-3)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup, config = 2, 1, 0, "tiny"
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_bench_parses_and_clock_sampler_degrades_without_gpu():
    import bench
    c = bench.Clocks(0)
    c.start()
    res = c.stop()
    assert "reasons" in res and "sm_mhz" in res

