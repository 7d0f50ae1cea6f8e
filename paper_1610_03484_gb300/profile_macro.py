"""The macro elastic solve of the nested FE^2 step on the composite plate, for
profiling.

    python -m paper_1610_03484_gb300.profile_macro [nx,ny,nz] [max_iter] [solves]

builds the Kuhn-split plate of nx x ny x nz hexes (default 200,40,10: 480k
tetrahedra, 1.92M Gauss points), takes C_bar of the 16x16x6, p = 1 plain-weave
RVE at nominal constituents, scaled at every Gauss point by a seeded factor in
[0.3, 1] (a degraded plate), holds symmetry rollers on x = 0, y = 0, z = 0 and
pulls the end x = L with 100 MPa; then runs `solves` solves from rest of at
most max_iter PCG iterations (default 200, 2) and prints their times.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

import rve_inputs as ri  # noqa: E402
import paper_1610_03484_gb300 as rve  # noqa: E402


def main(argv):
    grid = tuple(int(x) for x in (argv[1] if len(argv) > 1 else "200,40,10").split(","))
    max_iter = int(argv[2]) if len(argv) > 2 else 200
    solves = int(argv[3]) if len(argv) > 3 else 2
    with rve.Context(precision=rve.PREC_FP64) as ctx:
        rx, rt, ph, tg = ri.weave_rve(16, 16, 6)
        mesh = ctx.mesh_load(rx, rt, 1, ph, tg)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
        mesh.set_bc(rve.BC_PERIODIC)
        C0 = mesh.homogenise().C
        mesh.free()
        xyz, tets, _ = ri.plate(*grid)
        w = np.random.default_rng(1).uniform(0.3, 1.0, len(tets) * 4)
        C = np.ascontiguousarray(w[:, None, None] * C0[None])
        m = ctx.macro_load(xyz, tets)
        m.mech_set_bc(np.stack([xyz[:, i] <= 1e-12 for i in range(3)], axis=1))
        m.mech_set_traction(xyz[:, 0] >= xyz[:, 0].max() * (1 - 1e-12), [1.0e8, 0.0, 0.0])
        for k in range(solves):
            m.mech_set_u(None)
            t0 = time.time()
            try:
                st = m.mech_solve(C, rtol=1e-10, max_iter=max_iter)
            except rve.RveError as e:
                if e.code != -4:
                    raise
                st = {"converged": 0}
            print(grid, "solve", k, "time %.4f s" % (time.time() - t0), st)
        m.free()


if __name__ == "__main__":
    main(sys.argv)
