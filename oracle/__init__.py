"""CPU oracle for the DDA hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct FP64 statement of what the GPU path
computes, written from the DDSCAT 7.2 user guide (Draine & Flatau 2012) and
the published DDA formulae it cites.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import, call or link anything in
this package; the product path never does, and this package imports nothing
from the product package.

Contents
  dda       -- sites, LDR polarizability, interaction tensor, dense matrix,
               pairwise O(N^2) matvec, incident field, BiCGstab over the
               pairwise matvec, cross sections, pair-sum and quadrature C_sca,
               adjoint dQ_abs/d(eps).
  mie       -- Mie-series efficiencies for a homogeneous sphere.
  lattice   -- Ewald evaluation of the dipole lattice sum that defines the
               LATTDR polarizability (pins its constants and the form of S).
  pairwise  -- the same pairwise matvec in plain C with OpenMP (for sizes where
               numpy is too slow: row samples of large targets, timed baseline).

Parity status per function is stated in each docstring ("pinned by ...").
"""
from . import dda, lattice, mie  # noqa: F401
