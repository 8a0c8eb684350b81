"""Oracle for the compact finite-difference (CFD) hot path of arXiv 2302.14858.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method (FP64 numpy for the block operators, exact
rationals / mpmath for scheme design).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import, call or execute anything in it.  The CUDA
product path (``paper_2302_14858_gb300``) shares no code with it and never
routes through it.

Modules
-------
schemes   Taylor constraints (Sec. "Method", Eq. mdAnsatz / Eq. Tcons), the
          modified wavenumber (Eq. fdpwerrdef) and its relative error
          (Eq. relmodnormwavnum), spectral tuning as an equality-constrained
          quadratic programme (Eqs. sp_error, optfunc, gammacut) and the
          C_0-matched explicit closures (Eqs. errrelmodwavcent,
          errelmodwavecentmatch).
cfd       The block operator: ghost fill (matrix G, Eq. example_G), closed
          banded solve (Eq. sch_cent_om), hybrid iteration (Eq. iter_center_P),
          the embedded dense operators (Eqs. diff_mat_subL/R/MR,
          iter_scheme), 3D application with symmetrised mixed derivatives
          (Sec. "Z4c: system description"), and classical RK4 for the linear
          wave system.
timestep  Kreiss-Oliger dissipation (Eq. dissdef) and the two-register (2S)
          low-storage Runge-Kutta recurrence with its 4-stage 4th-order
          coefficients.
biased    Biased first-degree schemes: UCD slow/fast U_M, V_M (Eq.
          defChenSchemes), their xi closures (Eqs. ucd_slow_closure_chi,
          ucd_fast_closure_chi), CCU X_M (Eq. LCslowfast), the mirror rule, the
          bidiagonal block systems (Eq. closure_left_X and its right-biased
          counterpart), their iteration (Eq. iter_left_X) and the upwinded
          shift-advection term (Eq. biasderapproxadv).

Parity status: every function is pinned by ``tests/test_oracle_*.py``.  The 3D
path (``apply_uniform``, mixed ops and hybrid iteration included) is pinned on
separable and on general random data against the decomposed 1D operator applied
to global lines, which is itself pinned against the dense embedded operator
[i]D of Eq. iter_scheme.
"""
