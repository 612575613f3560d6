"""Plain float64 CPU oracle of the four-way coupled LBM-DEM time step.

THIS PACKAGE IS TEST INFRASTRUCTURE. It restates the method of Rettinger &
Ruede (arXiv 2003.01490) equation by equation in slow, readable numpy so
that the CUDA path can be checked against it. Only the test suite, the
``smoke()`` check of ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it. The library in ``paper_2003_01490_gb300`` never
imports, calls or falls back to it, and the two share no code.

Modules:
  d3q19     lattice, moment matrix M, equilibrium moments, rate matrices
  lbm       equilibrium PDFs, moments, moment-space collision with forcing
  particles mapping, link fractions, lubrication and contact laws
  coupling  boundary conditions, momentum exchange, missing links, refill
  sim       Algorithm 1: the complete coupled time step

Every function is pinned by the ``-m "not gpu"`` tests in ``tests/`` against
closed forms, invariants, brute force or the paper's printed values. The
complete coupled step is pinned as a whole by exact solutions it must keep
(a sphere carried by a uniform flow, prescribed or free, stays in it with
zero force) and by the Stokes drag of a periodic sphere array. A general
trajectory of interacting particles is pinned only by its parts and by its
invariance under a rotation of the lattice that permutes the axes, a mirror
of one axis and a whole-cell translation along periodic axes, not by values (parity unpinned for the complete step
at the large configurations).
"""
from .d3q19 import C, W, OPP, M, M_INV, Q, CS2, RHO0  # noqa: F401
from .sim import Domain, Params, Simulation  # noqa: F401
