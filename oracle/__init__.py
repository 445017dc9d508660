"""CPU oracle of the plane-wave multiple-scattering transport path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg, never by the product package.  It shares
no code with the CUDA path.

Modules:
* ``pw_oracle``: the path itself (Eqs. loc, transfer, scatter, recurrence;
  App. C), the dense matching solve, the adjoint, and the layer doubling of
  Eq. recurrence2;
* ``brute``: an independent 40-digit matrix-exponential solve of the slice
  model;
* ``continuum``: an independent finite-difference solve of the
  continuous-z problem (a convergence pin of the slice model);
* ``complex_bands``: periodic electrodes (App. B complex bands by Eq. cmp,
  tilted cells, band folding; App. C transmission between them);
* ``separable``: nonlocal separable projector terms (Eqs. nloc, gsol_p0,
  calm_0) in one matching system.

Parity status: every function is pinned (tests/test_oracle_*).
"""
