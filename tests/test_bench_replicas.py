"""The N > 1 path of bench.py without a GPU: the benchmark path does not
shard (one replica of the workload per rank, no data-path collective), so
what multi-rank runs add is host logic.  Each rank's time is reduced to the
maximum over ranks, the throughput counts the units of all ranks over that
time, and the reference arm runs on rank 0 only.  Tested with world size 2
over gloo on the CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.replica_time_max(times[rank], world)
        q.put((rank, t, bench.replica_throughput(1000.0, world, t)))
    finally:
        dist.destroy_process_group()


def test_replica_time_is_the_max_over_ranks_and_throughput_sums_ranks():
    world, times = 2, [0.75, 1.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, t, v in out:
        assert t == max(times)
        assert abs(v - world * 1000.0 / max(times)) < 1e-9


def test_single_rank_is_unchanged():
    assert bench.replica_time_max(0.5, 1) == 0.5
    assert bench.replica_throughput(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    class Args:
        steps, warmup, gpus = 2, 1, 2
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda *a, **k: (_ for _ in ()).throw(AssertionError("ran")))
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
