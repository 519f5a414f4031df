"""GB300-native (sm_103a) implementation of the data-parallel hot path of
SE(2,N) hypoelliptic-diffusion inpainting: lift to N directions, per-plane
2-D DFT, fused Crank-Nicolson integration of the decoupled Mathieu-type
systems, inverse DFT, static restoration and projection.

The compute path is the CUDA library libse2n.so (C ABI in include/se2n.h);
``paper_1304_2062_gb300.se2n`` is its Python binding and
``paper_1304_2062_gb300.build`` compiles it.
"""
