"""FP64 CPU oracle for the randomized ("augmented") block-CG method.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package. The CUDA
library never calls it and shares no code with it.

Everything here is plain NumPy/SciPy in float64 and follows the paper
("Preconditioning without a preconditioner using randomized block Krylov subspace
methods", Chen, Huber, Lin, Zaid). Citations name the paper's sections (1
Introduction ... 7 Numerical experiments, appendices A-C) and its equations and
definitions by their labels.

  operators   block products with A_mu = A + mu I (Eq. regularized_ls, Sec. 1.2)
  direct      O0: the result definitions (Cholesky solve of A_mu, eigendecomposition
              for the ridge path and for A^{1/2} B)
  bcg         O1: block-CG by the Hestenes-Stiefel/O'Leary recurrence on the
              augmented start block [b Omega] (Def. BCG, Thm. main, Sec. 3)
  lanczos     O2: block-Lanczos with full reorthogonalisation and the projected
              shifted solves of Eq. bcg_alg (Sec. 3.2, Thm. cost)
  galerkin    brute force: explicit block Krylov basis and Galerkin projection
              (Def. BCG as written)
  nystrom     O3: Nystrom approximation (Eq. nystromBKI_def), deflation
              preconditioner (Eq. precond_def), PCG (Def. PCG), CG (Def. CG)

Every function is pinned by tests marked ``not gpu`` (closed forms, special
cases, brute force, the paper's theorems); none is "parity unpinned".
"""
