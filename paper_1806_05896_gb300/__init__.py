"""GB300-native interior point method for L1-sparse, box-constrained PDE control.

The compute path is the CUDA library ``libipm`` (C ABI in include/ipm.h);
``paper_1806_05896_gb300.ipm`` is its Python binding and
``paper_1806_05896_gb300.build`` compiles it for sm_103a.
"""
__all__ = ["ipm", "build"]
