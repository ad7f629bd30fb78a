"""SOR-SVD (subspace-orbit randomized SVD, Kaloorazi & de Lamare) on GB300.

``native``  binding of the CUDA library's C ABI (include/sorsvd.h)
``inputs``  seeded synthetic test matrices shaped like the paper's workloads
"""
__all__ = ["native", "inputs"]
