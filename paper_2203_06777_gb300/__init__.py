"""GB300-native 5D domain-wall fermion operator (Shamir), after Grid (arXiv:2203.06777).

The compute path is a C-ABI CUDA library (``libgrid_dwf.so``, built for sm_103a from
``csrc/``) reached through the ctypes binding in :mod:`paper_2203_06777_gb300.dwf`.
Importing this package does not load the library; :func:`paper_2203_06777_gb300.dwf.load`
does, and fails loudly if it is missing.
"""

__all__ = ["synth"]
