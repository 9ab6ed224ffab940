// cm_blocks_gauss.cu -- block-level kernels (b >= 2) for curvature kind KIND_GAUSS.
#include "cm_phase_blocks.cuh"

CM_BLOCKS_INSTANTIATE(cm::KIND_GAUSS)
