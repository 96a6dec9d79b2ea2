"""bench.py's multi-process logic on the CPU: two gloo ranks (world size 2) reduce their
timings with a max over ranks and account the whole-job work (weak scaling: every rank
tracks its own bunch, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    t_local = 1.0 + rank          # rank 1 is the slower one
    t_max = bench.max_over_ranks(t_local, dist, device="cpu")
    units = 1000 * 10 * 3 * 2 * ws          # n x turns x schemes x steps x ranks
    out[rank] = (t_max, units / t_max)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(1000 * 10 * 3 * 2 * 2 / 2.0)


def test_max_over_ranks_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5
