"""GB300-native hybrid interior-point / column-generation solver for discrete optimal transport.

Method: Zanetti & Gondzio, arXiv:2206.11009.  The compute path is the CUDA library built from
``csrc/`` (C ABI in ``include/ot_ipm.h``); this package marshals arguments to it.  Importing
the package does not load the library; the first call that needs it does, and fails loudly if
it has not been built (``paper_2206_11009_gb300.build.build()``).
"""
from .api import Result, Solver, default_options, kernel_launches, kernel_timing, price_topk  # noqa: F401
