"""GB300-native incremental octree LOD update (SimLOD, Schuetz, Herzberger and
Wimmer, 2023): count -> split -> voxel claim -> scatter into chunked leaves.

The compute path is the CUDA library ``libsimlod.so`` behind the C ABI in
``include/simlod.h``; :mod:`.simlod` is its ctypes binding.
"""
