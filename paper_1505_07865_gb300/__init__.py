"""GB300-native constrained rigid-body immersed-boundary Stokes solver.

The compute path is the CUDA library ``libibrigid.so`` (C ABI in
``include/ibrigid.h``); ``paper_1505_07865_gb300.abi`` is its ctypes binding
(``from paper_1505_07865_gb300 import abi``).  Build the library with
``python -m paper_1505_07865_gb300.build``.
"""
