"""GB300-native (sm_103a CUDA) hot path of the coupled colour-gradient LBM / DEM
method for droplet-particle interactions on solid surfaces (arXiv 2505.10171).

The compute lives in ``csrc/`` behind the C-ABI declared in ``include/lbm.h``;
``lbm`` is the thin ctypes binding with the same entry-point names.
"""
