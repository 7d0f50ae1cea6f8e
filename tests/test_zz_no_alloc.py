"""The allocation-free operator entry point against the allocating one.

rve_operator_energy_noalloc serves callers that cannot allocate device memory
while they run (an application that owns all GPU memory through its own
pre-sized pool, or a loop that must not allocate): it uses only a static
device scratch array.  It must give the same y = K x as rve_apply_operator, and
energies x . K x, on two calls in a row (the scratch keeps the previous call's
contents, so the second call checks that nothing stale leaks through).
This file is collected last on purpose.
"""
import numpy as np
import pytest

import rve_inputs as ri

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("field", [0, 1])
def test_noalloc_matches_apply_operator(field):
    import torch
    import paper_1610_03484_gb300 as rve
    from paper_1610_03484_gb300 import _build
    _build.build()
    rve.load_library()
    grid, p = (6, 5, 4), 2
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    torch.cuda.init()
    stream = torch.cuda.current_stream()
    with rve.Context(precision=rve.PREC_FP64, stream=stream.cuda_stream) as ctx:
        mesh = ctx.mesh_load(xyz, tets, p, phase, tangent)
        mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN, T_C=45.0, c_wt=0.8, t_h=500.0)
        mesh.set_bc(rve.BC_PERIODIC)
        N = mesh.info()["n_scalar_dofs"]
        nc = 3 if field == 0 else 1
        rng = np.random.default_rng(10 + field)
        for call in range(2):
            ncols = 12 if call == 0 else 6
            x = rng.normal(size=(N * nc, ncols))
            if field == 0:
                want = mesh.apply_operator(0, x)
            else:
                want = np.zeros_like(x)
                th = [c for c in range(ncols) if c % 6 < 3]
                mo = [c for c in range(ncols) if c % 6 >= 3]
                want[:, th] = mesh.apply_operator(1, x[:, th])
                want[:, mo] = mesh.apply_operator(2, x[:, mo])
            xd = torch.tensor(x, dtype=torch.float64, device="cuda")
            yd = torch.full((N * nc, ncols), 7.0, dtype=torch.float64, device="cuda")   # stale values
            ed = torch.zeros(ncols, dtype=torch.float64, device="cuda")
            mesh.operator_energy_noalloc(field, ncols, xd.data_ptr(), yd.data_ptr(), ed.data_ptr())
            torch.cuda.synchronize()
            got = yd.cpu().numpy()
            scale = np.abs(want).max()
            assert np.abs(got - want).max() <= 1e-12 * scale
            energy = np.einsum("rc,rc->c", x, want)
            np.testing.assert_allclose(ed.cpu().numpy(), energy, rtol=1e-10)
        # sizes beyond the static scratch are rejected, not truncated
        big = torch.zeros((N * nc, 102), dtype=torch.float64, device="cuda")
        with pytest.raises(rve.RveError) as e:
            mesh.operator_energy_noalloc(field, 102, big.data_ptr(), big.data_ptr(), big.data_ptr())
        assert e.value.code == -1
        mesh.free()
