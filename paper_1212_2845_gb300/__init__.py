"""GB300-native voxel lattice soft-body simulator (Hiller & Lipson, arXiv 1212.2845).

The hot path lives in hand-written sm_103a CUDA kernels behind a C ABI
(``include/vx.h``); this package only marshals arguments to it.
"""
