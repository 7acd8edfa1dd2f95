"""GB300-native over-decomposed Jacobi relaxation (CUDA, sm_103a).

The CUDA library is loaded lazily by :mod:`paper_2303_02543_gb300.jacobi`;
importing the package itself loads nothing.
"""
__all__ = ["jacobi", "inputs"]
