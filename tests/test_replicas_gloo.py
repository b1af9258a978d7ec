"""The multi-GPU path of bench.py is N independent replicas; its only
collectives are the host-side timing barrier and the max over ranks of the
measured time (gloo). Two CPU ranks exercise them here."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    env = bench.dist_env()
    dist.init_process_group("gloo")
    t = bench.max_over_ranks(1.5 + rank, True)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, env, t))


def test_two_rank_barrier_and_max():
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
    assert [o[1] for o in out] == [(2, 0, 0), (2, 1, 1)]
    assert all(o[2] == 2.5 for o in out)                 # the slowest rank's time on every rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, False) == 3.25
