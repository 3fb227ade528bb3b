"""The N > 1 path of bench.py on CPU: two gloo ranks run independent replicas
and the run is timed by the slowest rank while the work adds up (no
data-path collective; the update is one simulation per GPU)."""
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    bench.barrier()
    # rank r "processed" (r + 1) * 1e9 updates in (r + 1) * 0.5 s
    t, u = bench.aggregate(0.5 * (rank + 1), 1e9 * (rank + 1))
    q.put((rank, ws, r, local, t, u))
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, t, u in res:
        assert ws == 2 and r == rank and local == rank
        assert t == pytest.approx(1.0)      # the slowest rank's time
        assert u == pytest.approx(3e9)      # all ranks' work
    # whole-job throughput = 3e9 updates / 1.0 s
    assert res[0][5] / res[0][4] == pytest.approx(3e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm prints from rank 0; other ranks exit 0."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus, nr, ntheta = 1, 0, 2, 64, 64
    assert bench.run_reference(A) == 0
    assert capsys.readouterr().out == ""
