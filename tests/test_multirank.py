"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own seeded
Gauss points (no data-path collective), job time = max over ranks, units =
sum over ranks; the reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    import rve_inputs as ri
    w, r, l = bench.dist_setup()
    assert (w, r, l) == (world, rank, rank)
    T, c, t, size, p = ri.gauss_point_states(64, bench.SEED + r)
    t_local = 1.0 + r            # rank 1 is the slow one
    job = bench.max_over_ranks(t_local, w)
    units = bench.sum_over_ranks(64.0, w)
    bench.barrier(w)
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), w, r)
    out.put((r, float(T[0]), job, units, ref is None))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, T0, job0, u0, none0), (r1, T1, job1, u1, none1) = res
    assert job0 == job1 == 2.0          # max over ranks
    assert u0 == u1 == 128.0            # whole-job units
    assert T0 != T1                     # each rank draws its own points
    assert not none0 and none1          # the reference arm prints on rank 0 only
