"""Host logic of the multi-GPU bench path, on CPU with gloo and two ranks: each rank gets
disjoint instances, and the reported time is the MAX and the work the SUM over ranks."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_2507_14051_b300.dist import instance_seeds


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2507_14051_b300.dist import env_rank_world, instance_seeds, reduce_elapsed_and_work
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, local, w = env_rank_world()
    seeds = instance_seeds(r, w, per_rank=3)
    elapsed, work = reduce_elapsed_and_work(1.5 + r, 100.0 * (r + 1))
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, local, w, seeds, elapsed, work))


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[2] == 2 for o in out)
    assert set(out[0][3]).isdisjoint(out[1][3])
    for o in out:
        assert o[4] == 2.5          # max over ranks of 1.5 + rank
        assert o[5] == 300.0        # sum of 100 * (rank + 1)


def test_single_process_defaults():
    assert instance_seeds(0, 1) == [0]
    with pytest.raises(ValueError):
        instance_seeds(2, 2)
