"""Plain, slow, FP64 CPU oracle for the RVE cell problems of Ullah et al.,
"Multi-scale computational homogenisation to predict the long-term durability
of composite structures" (arXiv 1610.03484).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (different basis, different integration route, assembled sparse
matrices instead of a matrix-free operator, elimination and bordered systems
instead of projections); the only common module is the seeded input generator
``rve_inputs``.

Contents
* ``materials``   -- isotropic and transversely isotropic stiffness, rotation to
                     the fibre frame, transport tensors, the degradation law
                     (Sec. 4, Eqs. Model_final1 / Model_RateForm) and the
                     least-squares fit of beta (Eq. alphaT_LSF).
* ``lagrange``    -- textbook Lagrange P_p basis on a tetrahedron in barycentric
                     coordinates with exact monomial integration.  It spans the
                     same space as the paper's hierarchic basis (Sec. 1, Sec. 7),
                     so homogenised tensors must agree.
* ``macro``       -- the coupled macro time step: linear-tetrahedron heat and
                     moisture transport (Eqs. Eq_field, Eq_field_disc) with one
                     backward-Euler step, and the degradation field 1 - omega at
                     the macro Gauss points by backward Euler of the rate form
                     (Eq. Eq_Model_RateForm), plus the equivalent exposure time
                     that hands a Gauss point to the RVE path.
* ``fibre``       -- yarn directions from the potential flow along each yarn
                     (Sec. 6): Laplace problem per yarn, unit gradient per tet.
* ``fem``         -- assembly, the three RVE boundary conditions of Sec. 2 in
                     fluctuation form (Eq. micro_disp), sparse direct / CG solves,
                     energy-form tensors (Eqs. Hill_prin, Eq_C_stress,
                     eq_homo_flux), volume-averaged stress (Eq. macro_stress) and
                     the paper's own bordered route [[K, C^T],[C, 0]] with
                     sigma = D^T lambda / V (Eqs. eq_RVE_disc_Eqs, eq_mat_C_and_D,
                     eq_homo_stress) for brute-force checks on tiny meshes.

Parity pins live in ``tests/test_oracle_*.py`` (closed forms, bounds, brute
force, printed constants).  Unpinned parts are listed in each module header.
"""
