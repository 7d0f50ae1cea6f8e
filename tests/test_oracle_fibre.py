"""Pins of the potential-flow yarn-direction oracle (Sec. 6): cases whose
potential and direction are known exactly, and symmetries of the weave."""
import numpy as np

import rve_inputs as ri
from oracle import fibre as fo


def test_straight_prism_has_linear_potential_and_axis_direction():
    # a straight yarn with a constant (staircase) section: phi is exactly linear
    # along the axis, so every direction is the axis itself
    xyz, tets = ri.kuhn_grid(10, 6, 4, lengths=(2.0, 1.0, 1.0))
    c = ri.centroids(xyz, tets)
    yid = np.where((np.abs(c[:, 1] - 0.5) < 0.3) & (np.abs(c[:, 2] - 0.5) < 0.3), 0, -1).astype(np.int32)
    sel = np.nonzero(yid == 0)[0]
    nodes, loc = np.unique(tets[sel], return_inverse=True)
    phi, grad = fo.yarn_potential(xyz[nodes], loc.reshape(-1, 4), 0)
    assert np.abs(phi - xyz[nodes, 0] / 2.0).max() < 1e-12
    d = fo.yarn_directions(xyz, tets, yid, [0], np.zeros((len(tets), 3)))
    assert np.abs(d[sel] - [1.0, 0.0, 0.0]).max() < 1e-12
    assert (d[yid < 0] == 0).all()                   # matrix keeps its input


def test_weave_directions_are_unit_and_follow_the_yarns():
    xyz, tets = ri.kuhn_grid(16, 16, 6)
    yid, axes = ri.plain_weave_yarns(xyz, tets)
    phase, tangent = ri.plain_weave(xyz, tets)
    assert np.array_equal(yid >= 0, phase == 1)
    d = fo.yarn_directions(xyz, tets, yid, axes, tangent)
    y = yid >= 0
    assert np.allclose(np.linalg.norm(d[y], axis=1), 1.0)
    for k, ax in enumerate(axes):
        s = yid == k
        # the flow runs along the yarn's axis from its lower to its upper end
        assert (d[s, ax] > 0).mean() > 0.9
        assert d[s, ax].mean() > 0.8
        # and, like the centreline, up and down about equally over one period (the
        # Kuhn split's fixed diagonal breaks the symmetry a little)
        assert abs(d[s, 2].mean()) < 0.1
        # close to the analytic centreline tangent on average (cos > 0.95)
        assert np.einsum("ij,ij->i", d[s], tangent[s]).mean() > 0.95
