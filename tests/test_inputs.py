"""Seeded input generators and the stored surrogate weights (host only)."""
import json
import os

import numpy as np

import rve_inputs as ri

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_state_generators_ranges_and_seeding():
    T, c, t, size, p = ri.gauss_point_states(5000, 2)
    assert (T >= 20).all() and (T <= 60).all()
    assert (c >= 0).all() and (c <= 1.5).all()
    assert (t >= 1).all() and (t <= 1e4).all()
    assert set(np.unique(p)) <= set(ri.P_CLASSES)
    assert (size >= 0).all() and (size < len(ri.SIZE_CLASSES)).all()
    Ta, ca, ta = ri.aged_states(5000, 13)
    assert (Ta >= 40).all() and (Ta <= 60).all()
    assert (ca >= 0).all() and (ca <= 1.5).all()
    assert (ta >= 1e2).all() and (ta <= 1e4).all()
    Tb, cb, tb = ri.aged_states(5000, 13)
    assert (Ta == Tb).all() and (ca == cb).all() and (ta == tb).all()
    assert not (ri.aged_states(10, 14)[0] == Ta[:10]).all()


def test_stored_surrogate_report():
    """The committed weights carry their training report: held-out error of the
    gated points within the 1e-2 bound, for both held-out sets."""
    z = np.load(os.path.join(ROOT, "paper_1610_03484_gb300", "surrogate_24x24x8_p2.npz"))
    rep = json.loads(str(z["report"]))
    assert int(z["members"]) == rep["members"]
    assert rep["n_train"] + rep.get("n_aged", 0) >= 20000
    assert max(rep["gated_rel_err_max"]) <= 1e-2
    assert rep["gated_frac"] >= 0.95
    aged = rep["aged_heldout"]
    assert max(aged["gated_rel_err_max"]) <= 1e-2 and aged["gated_frac"] >= 0.95
    assert z["params"].dtype == np.float32 or z["params"].dtype == np.float64
