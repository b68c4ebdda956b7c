"""Plain FP64 CPU oracle for the Chebyshev-filtered subspace iteration of the spherical
spectral Kohn-Sham method (Banerjee, Elliott, James, "A spectral scheme for Kohn-Sham
density functional theory of clusters").

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
baseline leg may import this package. The CUDA product never calls it, and it shares
no code, tables or constants with the CUDA product.

Every step is written from the paper's formulation in the paper's order, in float64,
with numpy matmul/einsum and numpy.linalg (eigh, cholesky) as the only library
primitives:
  special.py      - spherical Bessel functions, their zeros, Gauss rules, normalised
                    associated Legendre functions (Sec. 2.2.1, 2.2.2, 3.4.2)
  basis.py        - basis F_lmn = R_ln(r) Y_lm, the tensor-product grid, the inverse and
                    forward basis transforms (Sec. 2.2.1, 2.2.2, eqs. G_lmr, Ar_lm,
                    Arlm_to_coeff)
  hamiltonian.py  - the matrix-free product H.X (Sec. 2.2.4, eq. matvec_final) with the
                    Kleinman-Bylander projector pair (Sec. 2.3.2), and the explicit dense
                    H for tiny bases (eq. Hij_def)
  eigen.py        - scaled Chebyshev filter, Cholesky-QR with column scaling, Rayleigh-
                    Ritz, Lanczos bound and the ChFSI loop (Sec. 3.1.1, 3.2, 3.2.1)
  lobpcg.py       - LOBPCG with the Teter-Payne-Allan preconditioner (Sec. 3.1)
  learned_density.py - per-atom radial descriptors, fitted atom-centred density
                    corrections, a small MLP with Adam, and the predicted starting density
  scf.py          - electron density, Hartree potential (eqs. hartree_calc1,
                    zeta_definition), LDA exchange-correlation, Fermi-Dirac occupations,
                    Anderson mixing and the SCF loop (Sec. 2.1, 2.2.5, 2.3.1, 3.4.1)
  ozaki.py        - FP64 products A^T B of the dense steps (Sec. 3.2) from exact products of
                    small-integer slices (Ozaki, Ogita, Oishi, Rump 2012), with the FP32
                    accumulation bound a tensor-core kernel relies on

Parity status: every function is pinned by the -m "not gpu" tests in tests/ against
closed forms, an independent library (scipy.special), brute force, or invariants.
"""
