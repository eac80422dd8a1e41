"""Oracle for the particle-filter likelihood path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1606_08281_gb300``.

* ``oracle.pf_oracle``: ctypes front end of ``pf_oracle.c``, the plain
  single-threaded FP64 filter (Supp. I, algorithm "Likelihood Approximation
  using particle filter", with Gillespie's direct method for the simulation
  step).
* ``oracle.exact_bd``: exact likelihood of the birth-death network by the
  forward algorithm on a truncated state space (the verification route the
  paper names, FSP, Supp. "posterior verification").
* ``oracle.fsp``: the same forward algorithm for any network on a box of
  counts (finite state projection of the chemical master equation), with
  scipy's sparse matrix-exponential action as the propagation step; the
  reference for the CUDA FSP kernel.
* ``oracle.ode``: the deterministic likelihood of the Egf-Ras-Raf-Mek-Erk
  model (its reaction equations and FRET noise model) with scipy's
  Dormand-Prince integrator; the reference for the CUDA ODE kernel.
"""
