"""GB300-native selected inversion (SI) fused with the selected quadratic solve (SQ)
for complex block-tridiagonal-with-arrowhead (BTA) matrices.

The compute path is the C-ABI library ``libqsi.so`` (CUDA, sm_103a) built from
``csrc/``; ``qsi`` is its thin ctypes binding.  Importing this package does not
load the library; ``paper_2601_04904_gb300.qsi`` does, and raises if it is missing.
"""
__all__ = ["inputs", "metrics", "qsi"]
