"""GB300-native cell-list force evaluation under Kraynik-Reinelt boundary conditions.

Dobson, Fox & Saracino, "Cell List Algorithms for Nonequilibrium Molecular
Dynamics" (arXiv:1412.3784): the dynamic size and dynamic offset cell lists
(Sec. 4.1, 4.2) evaluated by hand-written CUDA kernels for sm_103a behind a
C-ABI library (include/nemd.h).  The CUDA binding lives in
``paper_1412_3784_gb300.nemd``; importing this package does not load it.
"""
__all__ = ["workloads"]
