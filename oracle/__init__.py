"""CPU FP64 oracle for the preconditioned discrete dipole approximation.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, numpy/scipy
restatement of Groth, Polimeridis & White, "Preconditioning the discrete
dipole approximation" (arXiv 1903.09802).  It exists to check the CUDA path;
only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: the
only common module is ``dda_inputs`` (geometry and seeded random numbers).

Modules
-------
physics      Clausius-Mossotti / LDR polarizability, dyadic Green function
operator     Algorithm 1 tensor, dense DDA matrix, FFT (circulant-embedded)
             matvec of the BTTB operator
circulant    T. Chan optimal circulant (eq. 13), its multilevel extension
             (Chan-Olkin, Section 3), the 3-level and 2-level preconditioners
krylov       restarted GMRES with Givens rotations (modified Gram-Schmidt)
observables  incident plane wave, cross sections (standard DDA theory; the
             paper gives none) and a far-field quadrature for C_sca

Parity status
-------------
Every function is pinned by a test in ``tests/test_oracle_*.py`` against a
closed form, a brute-force definition, an invariant or a textbook result
(Mie series).  The 2-level preconditioner's iteration counts against the
paper's Tables 3/4 are a soft comparison only (the voxel-count rounding of
the tables is unstated).
"""
