"""Batched homogenisation of a single RVE class, for profiling.

    python -m paper_1610_03484_gb300.profile_batch 32,32,10 2 8 [n_points] [rtol] [calls] [profile] [kernel]

loads the plain-weave RVE on the given grid at order p, periodic BC, nominal
constituents, and runs macro_update_gauss_points `calls` times (default 1) on the
same n_points seeded Gauss points (default: one batch) in batches of B, mixed
precision; prints the wall time and the solver statistics of each call.  With
more than one batch the later batches are warm-started, as in the batched
workload; the first call also forms the per-mesh caches.  With profile = 1 the
PCG iterations are launched one by one from the host (the context's profile
mode) instead of as the device-side graph loop, so that a profiler that does not
follow kernels inside conditional graph nodes sees every launch.  kernel selects
the operator of the FP32 inner solve: 0 automatic (the matrix-free CUDA-core
kernel unless a schedule was tuned), 1 the matrix-free CUDA-core kernel, 2 the
tensor-core kernel (p = 2, 3).
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

import rve_inputs as ri  # noqa: E402
import paper_1610_03484_gb300 as rve  # noqa: E402


def main(argv):
    grid = tuple(int(x) for x in (argv[1] if len(argv) > 1 else "32,32,10").split(","))
    p = int(argv[2]) if len(argv) > 2 else 2
    B = int(argv[3]) if len(argv) > 3 else 16
    n = int(argv[4]) if len(argv) > 4 else B
    rtol = float(argv[5]) if len(argv) > 5 else 1e-8
    calls = int(argv[6]) if len(argv) > 6 else 1
    profile = bool(int(argv[7])) if len(argv) > 7 else False
    kernel = int(argv[8]) if len(argv) > 8 else rve.KERNEL_AUTO
    ctx = rve.Context(precision=rve.PREC_MIXED, rtol=rtol, inner_rtol=min(1e-5, rtol), batch=B,
                      profile=profile, operator_kernel=kernel)
    xyz, tets, ph, tg = ri.weave_rve(*grid)
    m = ctx.mesh_load(xyz, tets, p, ph, tg)
    m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    m.set_bc(rve.BC_PERIODIC)
    T, c, t, _, _ = ri.gauss_point_states(n, 5)
    for call in range(calls):
        t0 = time.time()
        Cc, Kk, Dd, st, stats, rc = ctx.macro_update([m], T, c, t, np.zeros(n, np.int32))
        keep = ("iterations_mech", "iterations_scalar", "refine_sweeps", "converged", "rel_residual_mech",
                "kernel_launches", "graph_host_ms", "graphs")
        print(grid, p, B, n, "call", call, "time %.4f s" % (time.time() - t0),
              {k: stats[k] for k in keep})


if __name__ == "__main__":
    main(sys.argv)
