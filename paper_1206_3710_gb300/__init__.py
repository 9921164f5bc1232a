"""GB300-native Monte Carlo radiative transfer on hierarchical (octree) grids.

The compute path lives in the CUDA library ``librt.so`` (sources under
``csrc/``, C-ABI declared in ``include/rt.h``); ``rt`` is its thin ctypes
binding and ``synth`` holds the seeded synthetic model generators.
"""
