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


def _oracle_worker(rank, world, port, steps, shots, text, q):
    import numpy as np

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = oracle.Circuit(text)
    out = []
    for i in range(steps):
        off = bench.shard_offset(rank, world, i, shots)
        meas, dets = c.sample(np.arange(shots), 99, shot_offset=off)
        out.append((off, meas, dets))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sample_the_same_shots_as_one():
    """Sharding by shot ranges needs no collective: two gloo ranks sampling
    their ranges (the oracle's keyed per-shot sampler) together produce
    exactly the bits one rank produces for all the shots."""
    import numpy as np

    import oracle
    from paper_2103_02202_gb300 import workloads as W
    text = W.surface_code_memory(3, 3, 0.02)
    world, steps, shots = 2, 3, 128
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_worker, args=(r, world, port, steps, shots, text, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pieces = sorted((off, m, d) for _, out in got for off, m, d in out)
    meas = np.concatenate([m for _, m, _ in pieces])
    dets = np.concatenate([d for _, _, d in pieces])
    om, od = oracle.Circuit(text).sample(np.arange(world * steps * shots), 99)
    np.testing.assert_array_equal(meas, om)
    np.testing.assert_array_equal(dets, od)
