"""The multi-GPU bench path (replicas: one process per GPU, independent instances): the host
logic on CPU with gloo and two ranks (each rank gets disjoint instances; the reported time is
the MAX and the work the SUM over ranks), and two ranks solving their own LPs, with the oracle on
CPU and with the GPU solver (both ranks on the one GPU of a test box)."""
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


def _solve_worker(rank, world, port, q, use_gpu):
    """One rank of the replicas-only multi-GPU path: solves its own instances (disjoint seeds)
    and joins the host-side MAX / SUM reduction."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time
    import torch.distributed as dist
    from paper_2507_14051_b300 import gen
    from paper_2507_14051_b300.dist import env_rank_world, instance_seeds, reduce_elapsed_and_work
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, _, w = env_rank_world()
    seeds = instance_seeds(r, w, per_rank=2, base=10)
    got = []
    t0 = time.perf_counter()
    for sd in seeds:
        lp = gen.small_lp(sd)
        if use_gpu:
            import torch
            import paper_2507_14051_b300 as lpx
            torch.cuda.set_device(0)  # every rank on the one GPU: independent solves, nothing shared
            with lpx.Solver(lp) as s:
                s.solve(1e-8, 100000)
                res = s.result()
        else:
            import oracle
            res = oracle.solve(lp, tol=1e-8, max_iter=100000)
        got.append((sd, int(res["status"]), int(res["iters"]), res["x"].tobytes(), res["y"].tobytes()))
    elapsed, work = reduce_elapsed_and_work(time.perf_counter() - t0, float(sum(g[2] for g in got)))
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, got, elapsed, work))


def _run_ranks(use_gpu, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, world, port, q, use_gpu)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=600) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def _check_ranks(out, single):
    seeds = [g[0] for o in out for g in o[1]]
    assert len(seeds) == len(set(seeds)) == 4             # disjoint instances
    total = sum(g[2] for o in out for g in o[1])
    for o in out:
        assert o[3] == float(total)                        # SUM of the work over ranks
        assert o[2] == max(p[2] for p in out)              # the same MAX elapsed on every rank
        for sd, st, it, xb, yb in o[1]:
            ref = single(sd)
            assert st == ref[0] == 1 and it == ref[1]      # OPTIMAL, same iteration count
            assert xb == ref[2] and yb == ref[3]           # bit for bit: a rank solves like one process


def test_two_ranks_solve_their_own_instances_oracle():
    """Two gloo ranks on CPU, each solving its own small LPs (the oracle as the solver): disjoint
    instances, the host reduction of time and work, and per-rank results equal to one process's."""
    import oracle
    from paper_2507_14051_b300 import gen

    def single(sd):
        r = oracle.solve(gen.small_lp(sd), tol=1e-8, max_iter=100000)
        return int(r["status"]), int(r["iters"]), r["x"].tobytes(), r["y"].tobytes()

    _check_ranks(_run_ranks(False), single)


@pytest.mark.gpu
def test_two_ranks_solve_their_own_instances_gpu(cuda_device):
    """The same with the GPU solver: two processes (gloo for the host reduction) on the one GPU,
    each solving its own LPs through lp_create / lp_solve / lp_get; the ranks' kernels never wait
    on each other.  Each result equals the single-process solve of the same instance bit for bit."""
    import paper_2507_14051_b300 as lpx
    from paper_2507_14051_b300 import gen

    def single(sd):
        with lpx.Solver(gen.small_lp(sd)) as s:
            s.solve(1e-8, 100000)
            r = s.result()
        return int(r["status"]), int(r["iters"]), r["x"].tobytes(), r["y"].tobytes()

    _check_ranks(_run_ranks(True), single)
