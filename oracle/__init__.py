"""CPU oracle for the two-step Brillouin-zone TDKS propagation.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128
numpy/scipy restatement of what the GPU library computes; it exists so that
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
can check and time the GPU path against it.  Nothing in the product library
imports, links or runs it, and it imports nothing from the product library.
It shares only the seeded input generators in ``workloads``.

Modules (each function cites the paper passage it follows):
  fd        -- finite-difference weights (Fornberg) and their plane-wave symbols
  kpoints   -- Monkhorst-Pack and shifted grids (Eqs. 8, 10), Halton sequence
  cell      -- grid, local potential, Kleinman-Bylander projectors (Eq. 2)
  hxc       -- Hartree (FFT Poisson) and LDA (Perdew-Zunger 1981) potentials
  hamiltonian -- application of h_k(t) (Eq. 2) and its dense matrix
  scf       -- ground state (fixed occupations, Pulay mixing)
  dynamics  -- fields (Eqs. 11, 15), Taylor-4 and ETRS steps, density (Eq. 3),
               current (Eqs. 5-6), two-step driver (Eq. 9, Sec. II.B steps 1-4)
               and the standard error of the two-step mean (Sec. III.B)
  analysis  -- windowed Fourier transforms, eps(omega) (Eqs. 12-14),
               HHG spectrum (Eqs. 16-17), error metrics, free-electron closed form

Parity pinning status of every function is listed in the test modules
``tests/test_oracle_*.py``; the v_loc/projector tables are pinned by
symmetry, normalisation, Fourier-coefficient and isolated-atom checks, and
the SCF ground state by the free-electron closed form and a brute-force
dense-matrix SCF on a tiny cell (no paper values exist for it).
"""
from . import fd, kpoints, cell, hxc, hamiltonian, scf, dynamics, analysis  # noqa: F401
