"""Oracle for SOR-SVD: a plain, slow binary64 CPU implementation written from
the paper (Kaloorazi & de Lamare, "Subspace-Orbit Randomized Decomposition for
Low-rank Matrix Approximation").

TEST INFRASTRUCTURE, not part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path and
imports nothing from the package.

Modules: ``philox`` (Omega), ``linalg`` (Householder QR, Jacobi SVD),
``sor_svd`` (Algorithm 3; R-SVD and TSR-SVD, Algorithms 1 and 2), ``bounds`` (Theorems 4-7), ``rpca`` (Table 3).
Every function here is pinned by a ``-m "not gpu"`` test against something
other than itself (library routines, closed forms, invariants, the values the
paper prints).
"""
from .philox import gaussian_matrix, gaussian_elements, philox4x64_10, round_to  # noqa: F401
from .linalg import householder_qr, jacobi_svd  # noqa: F401
from .sor_svd import sorsvd, rsvd, tsrsvd, flop_count, recon_error_fro, eckart_young, orthonormality_defect  # noqa: F401
from .rpca import rpca_alm, shrink  # noqa: F401
