"""Host logic of the multi-GPU benchmark path on CPU: the path does not shard
into a collective (replicas only), so N > 1 runs N independent replicas and
reports the whole-job throughput over the slowest rank.  Two gloo ranks check
the MAX reduction and value = ranks / per-step seconds."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        # rank r took (r + 1) * 3 seconds for 3 steps: the job's per-step time is the slowest rank's
        value, per_step = bench.replica_throughput((rank + 1) * 3.0, 3, device="cpu")
        out.put((rank, value, per_step))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, per_step in res:
        assert per_step == pytest.approx(2.0)          # max over ranks: 6 s / 3 steps
        assert value == pytest.approx(ws / 2.0)        # two replicas' steps per 2 s


def test_single_process_is_its_own_job():
    import bench
    assert not dist.is_initialized()
    value, per_step = bench.replica_throughput(4.0, 2, device="cpu")
    assert per_step == 2.0 and value == 0.5
