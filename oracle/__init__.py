"""CPU fp64 oracle of the finite-volume compressible Navier-Stokes right-hand side and TVD-RK3 step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may use it.  It shares no code with the CUDA path.

Modules
-------
ns_fv          the discretisation (Section 2.1, Eq. NSE and Eq. ODE) written out plainly in numpy,
               generic over the scalar type (float64, or complex128 for complex-step derivatives)
exact_riemann  the exact solution of the Euler Riemann problem (used to pin the Sod case)

Every function is vectorised over whole arrays with plain slicing; there is no blocking, fusion or
reordering beyond what the definitions state, so each step can be checked against the paper by eye.
"""
from . import ns_fv, exact_riemann  # noqa: F401
