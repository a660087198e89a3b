"""Host logic of the multi-GPU path, run as two gloo ranks on CPU: ranks take
disjoint shot ranges whose union is contiguous, and the reported time is the
maximum over ranks (no data-path collective is involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, steps, shots, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ranges = [(bench.shard_offset(rank, world, i, shots), shots) for i in range(steps)]
    t = torch.tensor([10.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, ranges, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shot_ranges_and_max_time():
    world, steps, shots = 2, 5, 16384
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, shots, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    starts = sorted(s for _, rr, _ in out for s, _ in rr)
    assert starts == [k * shots for k in range(world * steps)]
    assert all(offset % 64 == 0 for _, rr, _ in out for offset, _ in rr)
    assert all(tmax == 10.0 + world - 1 for _, _, tmax in out)
