"""GB300-native GFMC hot path for the 3D double-exchange model (arXiv:1303.6016).

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI, declared
in ``include/gfmc.h``); ``gfmc.py`` is the thin ctypes binding.  Import
``paper_1303_6016_gb300.gfmc`` for the API; importing the package itself loads
nothing.
"""
