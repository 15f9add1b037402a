"""GB300-native SparStencil hot path: stencil time steps as 2:4 sparse tensor-core MMAs.

The compute path is a C-ABI shared library (``include/sparstencil.h``) built from
``csrc/`` for sm_103a; :mod:`paper_2506_22969_gb300.binding` marshals arguments to it.
Importing this package does not load the library; the first call into
:mod:`~paper_2506_22969_gb300.binding` does, and raises if it is missing.
"""
__all__ = ["binding", "inputs"]
