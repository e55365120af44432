"""The multi-GPU path runs independent replicas: the job split and the
max-over-ranks timing, checked with two gloo ranks on CPU."""
import os

import pytest

torch = pytest.importorskip("torch")


def _worker(rank, world, port, njobs, q):
    import torch.distributed as dist
    from paper_1308_2864_gb300.replicas import max_over_ranks, shard, sum_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(njobs, rank, world)
    t = max_over_ranks(1.5 + rank)
    total = sum_over_ranks(len(mine))
    out = [None] * world
    dist.all_gather_object(out, mine)
    dist.destroy_process_group()
    q.put((rank, mine, t, total, out))


def test_two_gloo_ranks_split_jobs_and_take_the_max_time():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, njobs = 2, 7
    procs = [ctx.Process(target=_worker, args=(r, world, port, njobs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, t, total, gathered in res:
        assert t == 2.5
        assert total == njobs
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(njobs))
        assert set(gathered[0]).isdisjoint(gathered[1])


def test_shard_rejects_bad_rank():
    from paper_1308_2864_gb300.replicas import shard
    with pytest.raises(ValueError):
        shard(3, 2, 2)


def _leaving_worker(rank, world, port, q):
    # rank 1 leaves between steps (no collective in flight); rank 0's next
    # collective must end in an error within the process-group timeout
    import datetime
    import time
    import torch.distributed as dist
    from paper_1308_2864_gb300.replicas import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    max_over_ranks(1.0)                      # one step together
    if rank == 1:
        q.put((rank, "left", 0.0))
        q.close()
        q.join_thread()                      # flush before the hard exit
        os._exit(0)
    time.sleep(1.0)
    t0 = time.monotonic()
    try:
        max_over_ranks(2.0)
        q.put((rank, "no error", time.monotonic() - t0))
    except Exception as e:                   # gloo reports the lost peer
        q.put((rank, type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_ends_the_next_collective_with_an_error():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (what, sec)) for r, what, sec in (q.get(timeout=120) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
    assert res[1][0] == "left"
    what, sec = res[0]
    assert what != "no error", "the survivor's collective completed without its peer"
    assert sec < 30.0
