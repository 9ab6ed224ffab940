// cm_blocks_gauss_euler.cu -- block-level kernels (b >= 2) for curvature kind KIND_GAUSS_EULER.
#include "cm_phase_blocks.cuh"

CM_BLOCKS_INSTANTIATE(cm::KIND_GAUSS_EULER)
