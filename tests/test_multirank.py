"""The N > 1 path on CPU with two gloo ranks: job time = max over ranks, units =
sum over ranks, the reference arm on rank 0 only; and the sharding of one
batch of Gauss points into cost-balanced contiguous blocks whose results are
gathered back (the only data-path collective)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, l = bench.dist_setup()
    assert (w, r, l) == (world, rank, rank)
    t_local = 1.0 + r            # rank 1 is the slow one
    job = bench.max_over_ranks(t_local, w)
    units = bench.sum_over_ranks(64.0, w)
    bench.barrier(w)
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), w, r)
    out.put((r, job, units, ref is None))
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
    (r0, job0, u0, none0), (r1, job1, u1, none1) = res
    assert job0 == job1 == 2.0          # max over ranks
    assert u0 == u1 == 128.0            # whole-job units
    assert not none0 and none1          # the reference arm prints on rank 0 only


# ----------------------------------------------- sharding of one batch (N > 1)
def _point_results(T, c, t):
    """A deterministic stand-in for a cell solve (the GPU is not used on CPU):
    SPD tensors that depend on the point's state."""
    n = len(T)
    A = np.stack([np.stack([np.cos(T[i] * (a + 1) + c[i] * (b + 1)) + t[i] * 1e-4 * (a == b) for b in range(6)])
                  for i in range(n) for a in range(6)]).reshape(n, 6, 6)
    C = A @ np.swapaxes(A, 1, 2) + 6 * np.eye(6)
    K = C[:, :3, :3] + np.eye(3)
    D = C[:, 3:, 3:] * 1e-12
    return C, K, D, np.zeros(n, np.int32)


def _shard_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    import rve_inputs as ri
    from paper_1610_03484_gb300 import sharding
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    w, r, _ = bench.dist_setup()
    G = 300
    T, c, t, size, p = ri.gauss_point_states(G, bench.SEED)
    mid = size * 2 + (p - 1)
    grids = [g for g in ri.SIZE_CLASSES for _ in ri.P_CLASSES]
    ps = [q for _ in ri.SIZE_CLASSES for q in ri.P_CLASSES]
    dofs = [ri.mesh_counts(*g)[0] * 3 * q ** 3 for g, q in zip(grids, ps)]   # any positive per-mesh size
    cost = sharding.point_costs(dofs, grids, ps, mid)
    off, imb = rve.partition_blocks(cost, w)
    lo, hi = int(off[r]), int(off[r + 1])
    local = sharding.pack(*_point_results(T[lo:hi], c[lo:hi], t[lo:hi]))
    full = sharding.gather_blocks(local, off)
    out.put((r, full, off, imb, cost))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_sharded_batch_gathers_the_single_rank_result_bit_for_bit():
    torch = pytest.importorskip("torch")
    import rve_inputs as ri
    import bench
    from paper_1610_03484_gb300 import sharding
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (_, full0, off, imb, cost), (_, full1, off1, _, _) = res
    T, c, t, _, _ = ri.gauss_point_states(300, bench.SEED)
    single = sharding.pack(*_point_results(T, c, t))
    assert np.array_equal(full0, single) and np.array_equal(full1, single)
    assert np.array_equal(off, off1) and off[0] == 0 and off[-1] == 300
    # balanced: the larger block costs at most the mean plus one point's cost
    blocks = [cost[off[r]:off[r + 1]].sum() for r in range(2)]
    assert max(blocks) <= cost.sum() / 2 + cost.max() + 1e-9
    assert abs(imb - max(blocks) / (cost.sum() / 2)) < 1e-12
    C, K, D, st = sharding.unpack(full0)
    Cs, Ks, Ds, _ = _point_results(T, c, t)
    assert np.array_equal(C, Cs) and np.array_equal(K, Ks) and np.array_equal(D, Ds)


def test_partition_is_the_linear_partition_optimum():
    """Against brute force on small inputs: no contiguous split has a smaller
    largest block."""
    import itertools
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    rng = np.random.default_rng(4)
    for G, n in ((7, 2), (9, 3), (10, 4), (3, 5)):
        cost = rng.uniform(0.1, 5.0, G)
        off, imb = rve.partition_blocks(cost, n)
        got = max(cost[off[r]:off[r + 1]].sum() for r in range(n))
        best = np.inf
        for cuts in itertools.combinations_with_replacement(range(G + 1), n - 1):
            b = (0,) + cuts + (G,)
            best = min(best, max(cost[b[r]:b[r + 1]].sum() for r in range(n)))
        assert got <= best * (1 + 1e-9)
        assert list(off) == sorted(off) and off[0] == 0 and off[-1] == G
