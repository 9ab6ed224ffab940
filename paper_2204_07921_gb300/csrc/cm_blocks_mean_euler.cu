// cm_blocks_mean_euler.cu -- block-level kernels (b >= 2) for curvature kind KIND_MEAN_EULER.
#include "cm_phase_blocks.cuh"

CM_BLOCKS_INSTANTIATE(cm::KIND_MEAN_EULER)
