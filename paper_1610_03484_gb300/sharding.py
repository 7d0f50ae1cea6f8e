"""Multi-process sharding of one batch of macro Gauss points (one GPU per
process): the batch is split into contiguous blocks balanced by estimated solve
cost (rve_partition_blocks), every rank homogenises its block, and the 33
independent FP64 values per point (upper triangles of C 6x6, K and D 3x3) plus
the status are gathered back to every rank over torch.distributed.  The gather
is the only collective on the data path; packing and unpacking are plain
marshalling."""
from __future__ import annotations

import numpy as np

_IU6 = np.triu_indices(6)
_IU3 = np.triu_indices(3)
WIDTH = 21 + 6 + 6 + 1          # the 33 tensor values and the status


def point_costs(n_dofs_per_mesh, grid_per_mesh, p_per_mesh, mesh_id):
    """Cost estimate per point: its RVE's mechanical DOFs times the expected PCG
    iteration count, taken proportional to the grid's largest dimension times p
    (the Jacobi-PCG count grows like 1/h)."""
    per_mesh = np.array([float(n) * max(g) * p for n, g, p in zip(n_dofs_per_mesh, grid_per_mesh, p_per_mesh)])
    return per_mesh[np.asarray(mesh_id)]


def pack(C, K, D, status):
    C = np.asarray(C).reshape(-1, 6, 6)
    K = np.asarray(K).reshape(-1, 3, 3)
    D = np.asarray(D).reshape(-1, 3, 3)
    out = np.empty((len(C), WIDTH))
    out[:, :21] = C[:, _IU6[0], _IU6[1]]
    out[:, 21:27] = K[:, _IU3[0], _IU3[1]]
    out[:, 27:33] = D[:, _IU3[0], _IU3[1]]
    out[:, 33] = np.asarray(status).reshape(-1)
    return out


def unpack(a):
    n = len(a)
    C = np.zeros((n, 6, 6))
    K = np.zeros((n, 3, 3))
    D = np.zeros((n, 3, 3))
    C[:, _IU6[0], _IU6[1]] = a[:, :21]
    C[:, _IU6[1], _IU6[0]] = a[:, :21]
    K[:, _IU3[0], _IU3[1]] = a[:, 21:27]
    K[:, _IU3[1], _IU3[0]] = a[:, 21:27]
    D[:, _IU3[0], _IU3[1]] = a[:, 27:33]
    D[:, _IU3[1], _IU3[0]] = a[:, 27:33]
    return C, K, D, a[:, 33].astype(np.int32)


def gather_blocks(local, offsets, group=None):
    """All-gather of each rank's block [offsets[r+1] - offsets[r], WIDTH] into
    the whole batch [offsets[-1], WIDTH] on every rank (blocks padded to the
    largest, FP64 on the host: a few hundred bytes per point)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = np.diff(np.asarray(offsets))
    mx = int(sizes.max()) if len(sizes) else 0
    buf = torch.zeros((mx, WIDTH), dtype=torch.float64)
    loc = torch.from_numpy(np.ascontiguousarray(local, np.float64))
    if len(loc):
        buf[:len(loc)] = loc
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([parts[r][:sizes[r]].numpy() for r in range(world)], axis=0)
