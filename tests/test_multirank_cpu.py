"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas
only -- each rank solves its own request, the job time is the slowest
rank's and the value counts every rank's work."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [1.5, 2.5][rank]
    m = bench.max_over_ranks(elapsed, dist, "cpu")
    out.put((rank, m, bench.job_value(1e9, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 2e9 / 2.5) < 1e-3 for r in res)


def test_footprint_estimate_grows_with_the_problem():
    import paper_2606_31380_b300 as q
    import scenes
    sc = scenes.config(1)
    f1 = q.footprint(sc.bodies, 1)
    f4 = q.footprint(sc.bodies, 4)
    f_half = q.footprint(sc.bodies[:8], 1)
    blocks = sum(b.n_nodes ** 2 for b in sc.bodies) * 48  # self blocks + preconditioner, both precisions
    assert f4 > f1 > f_half
    assert blocks < f1 < 3 * blocks
