// cm_blocks_mean.cu -- block-level kernels (b >= 2) for curvature kind KIND_MEAN.
#include "cm_phase_blocks.cuh"

CM_BLOCKS_INSTANTIATE(cm::KIND_MEAN)
