// cm_blocks_mean_euler_odd.cu -- block-level kernels for the paper's block sides 2^j - 1
// (Sec. 2.2), curvature kind KIND_MEAN_EULER.
#include "cm_phase_blocks.cuh"

CM_BLOCKS_ODD_INSTANTIATE(cm::KIND_MEAN_EULER)
