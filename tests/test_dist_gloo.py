"""Multi-rank host logic of bench.py as two gloo ranks on CPU: rank and
world from the launcher's environment, one event per rank, the job time as
the slowest rank's, and whole-job weak-scaling throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    # ranks time different amounts; the job's time is the slowest rank's
    t = bench.max_over_ranks(0.5 + r, dist, torch.device("cpu"))
    v = bench.weak_value(1000, w, 4, t)
    seeds = [None] * w
    dist.all_gather_object(seeds, bench.rank_seed_offset(r))
    dist.barrier()
    q.put((r, w, local, t, v, seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    for r, (rank, world, local, t, v, seeds) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert t == 1.5
        assert v == pytest.approx(1000 * 2 * 4 / 1.5)
        assert len(set(seeds)) == 2          # every rank tracks its own event


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25, None, None) == 0.25
    assert bench.weak_value(10, 1, 3, 2.0) == 15.0
