"""CPU FP64 oracle for the eeFU / CTMRG hot path (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain, obviously-correct statement of what the GPU
library computes.  It exists so that tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` can check and time
the CUDA path against it.  No product code imports it, and it imports nothing
from the product package: the two share no kernels, helpers, tables or
constants.  Only the seeded input generators in ``kh_inputs`` serve both.

Everything is numpy / scipy in float64.  Library primitives used as single
steps: ``numpy.einsum`` / ``tensordot`` (contractions), ``numpy.linalg.svd``
(LAPACK gesdd), ``numpy.linalg.qr``, ``scipy.linalg.expm`` and ``eigh``.

Module map (paper: Czarnik, Francuz, Dziarmaga, "Tensor network simulation of
the Kitaev-Heisenberg model at finite temperature", arXiv:1906.02220):

* ``model``        -- Eqs. (1)-(3), (5): bond Hamiltonians, bias, duality
                      Eq. (4); Sec. III Eq. (6): gates and the Trotter layers.
* ``peps``         -- Fig. 3: site tensors, the beta=0 purification; Fig. 4(b)
                      and Sec. III: the gamma-composite on the rhombic lattice.
* ``ctmrg``        -- Fig. 4(c) and Sec. III: square-lattice CTMRG on the
                      quadruple (double-layer) tensor; the environment metric;
                      the correlation length of Sec. IV from the channel
                      transfer matrix; the 2 x 2 cluster in its environment.
* ``bond``         -- Fig. 3(b) and Sec. III: the environment-weighted bond
                      update A'-B' -> A''-B''.
* ``observables``  -- energy per site, <S^a> per sublattice, the printed
                      order parameters, the specific heat along a
                      trajectory, products of operators on a 2 x 2
                      plaquette and the plaquette flux W (Sec. V).
* ``eefu``         -- the imaginary-time driver of Sec. III.
* ``exact``        -- independent pins: exact diagonalisation of honeycomb
                      clusters, Onsager's free energy, Yang's magnetisation,
                      closed forms for decoupled dimers and a pure field.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (see tests/test_oracle_*.py), except the
finite-chi / finite-D physics at the paper's own parameters, for which the
paper prints no observable values ("parity unpinned" for that use only).
"""
