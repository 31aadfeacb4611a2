"""Randomized ("augmented") block-CG for GB300 (sm_103a).

Solves (A + mu I) x = b by block-CG on the start block [b Omega] with a Gaussian
sketch Omega (Chen, Huber, Lin, Zaid, "Preconditioning without a preconditioner
using randomized block Krylov subspace methods", Sec. 3). The solver is the C-ABI
library libbk.so (include/bk.h); ``paper_2501_18717_gb300.bk`` is its Python
binding and ``paper_2501_18717_gb300.workloads`` draws the seeded synthetic inputs.
Submodules are imported on demand so the input generators work without the
compiled library.
"""
__all__ = ["bk", "workloads", "build"]
