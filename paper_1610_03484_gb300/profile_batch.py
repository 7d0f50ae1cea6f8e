"""One batched homogenisation of a single RVE class, for profiling.

    python -m paper_1610_03484_gb300.profile_batch 32,32,10 2 8

loads the plain-weave RVE on the given grid at order p, periodic BC, nominal
constituents, and runs macro_update_gauss_points on B seeded Gauss points
(mixed precision, rtol 1e-8); prints the wall time and the solver statistics.
"""
import sys, os, time
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np
import rve_inputs as ri
import paper_1610_03484_gb300 as rve
grid = tuple(int(x) for x in (sys.argv[1] if len(sys.argv) > 1 else "32,32,10").split(","))
p = int(sys.argv[2]) if len(sys.argv) > 2 else 2
B = int(sys.argv[3]) if len(sys.argv) > 3 else 16
ctx = rve.Context(precision=rve.PREC_MIXED, rtol=1e-8, inner_rtol=1e-5, batch=B)
xyz, tets, ph, tg = ri.weave_rve(*grid)
m = ctx.mesh_load(xyz, tets, p, ph, tg)
m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
m.set_bc(rve.BC_PERIODIC)
T, c, t, _, _ = ri.gauss_point_states(B, 5)
t0 = time.time()
Cc, Kk, Dd, st, stats, rc = ctx.macro_update([m], T, c, t, np.zeros(B, np.int32))
print(grid, p, B, "time %.3f s" % (time.time() - t0), stats)
