"""CPU oracle of the plane-wave multiple-scattering transport path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg, never by the product package.  It shares
no code with the CUDA path; see ``pw_oracle`` for what it computes and
``brute`` for the independent high-precision solve that pins it.

Parity status: every function in ``pw_oracle`` is pinned (tests/test_oracle_*).
"""
