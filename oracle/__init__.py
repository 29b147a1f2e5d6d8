"""Plain FP64 CPU oracle for the optimal-dimensionality SHT (Khalid, Kennedy, McEwen).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import anything here.  The CUDA
library never calls into this package and this package never calls into the CUDA library; the two
share no code.  Every function is written from the paper's definitions and procedures, in the
paper's order, in float64, with numpy / scipy used only as library primitives (matmul, LU solve,
SVD / symmetric eigendecomposition, and - for brute force only - scipy's spherical harmonics).

Modules
  legendre  scaled associated Legendre functions P~_l^m(theta) = Y_l^m(theta, 0)   (Sec. III-G)
  sampling  ring layout, equiangular set, simple and greedy ring orderings        (Sec. III-A, III-E)
  sht       forward SHT (Procedure 1), inverse SHT (Procedure 2), dense system, adjoints
  ring      ring DFTs and their inverses by direct sums                      (Eqs. (11), (18))
  spin      spin-s transforms from the Wigner-d recursion                    (Sec. III-H, App. A)

Parity status: every function here is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, scipy's Y_l^m, mpmath, orthonormality by Gauss-Legendre quadrature,
dense brute force, exact-SVD greedy); none is "parity unpinned".
"""
