"""The N>1 path on CPU: two gloo ranks, frame sharding and max-over-ranks reporting."""
import os
import socket

import pytest

from paper_2602_17938_gb300 import dist as pdist


def test_frames_for_rank_disjoint_and_covering():
    for n in (1, 5, 64, 256):
        for world in (1, 2, 3, 8):
            parts = [pdist.frames_for_rank(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, rk, _ = pdist.env()
    t_local = 1.0 + rk  # rank 1 is the slowest
    t_max = pdist.max_over_ranks(t_local)
    seed = pdist.frame_seed(1, rk)
    out.put((rk, ws, t_max, seed, pdist.job_throughput(1_000_000, 4, ws, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == 2.0 for r in res)
    assert res[0][3] != res[1][3]  # each rank cleans its own frame
    assert res[0][4] == pytest.approx(2 * 1_000_000 * 4 / 1e6 / 2.0)
