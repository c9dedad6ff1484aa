"""GB300 (sm_103a) library for the right-hand side and explicit stage update of the reacting
compressible Navier-Stokes equations for air in chemical nonequilibrium (arXiv 2210.05547).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``) behind the C ABI of
``include/hyp.h``; ``abi`` is its Python binding. Importing this package loads nothing: the
library is opened on the first call through ``abi``.
"""
