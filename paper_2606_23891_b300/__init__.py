"""B300-native SPH cell-pair offload pipeline (pack -> launch -> unpack).

The compute path is the in-tree CUDA library ``libsph.so`` (C-ABI in
``include/sph.h``); :mod:`.sph` is its thin ctypes binding and
:mod:`.pipeline` drives it over PyTorch-owned device memory.
"""
