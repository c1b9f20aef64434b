"""The N > 1 path of the benchmark on CPU: two gloo ranks on 127.0.0.1 take the max of their
timings, compute the weak-scaling whole-job value the same way, and only rank 0 runs the
reference arm.  No GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    my_ms = 100.0 + 25.0 * rank                       # rank 1 is the slower one
    job_ms = bench.max_over_ranks(my_ms, ws, device="cpu")
    value = bench.weak_scaling_value(64_000_000, 10, ws, job_ms)
    assert bench.dist_info() == (ws, rank, rank)
    tdist.barrier()
    tdist.destroy_process_group()
    out.put((rank, job_ms, value))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [125.0, 125.0]
    # 2 ranks x 10 steps x 64 M rays in 125 ms
    assert res[0][2] == pytest.approx(2 * 10 * 64e6 / 0.125 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        views, steps, warmup, cpu_seconds, gpus = 1, 1, 0, 0.1, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
