// cm_phase_kinds.h -- per-curvature-kind entry points of the block levels.
//
// The kernels of the levels with block side b >= 2 are templates on the
// curvature kind; each kind is instantiated in its own translation unit
// (cm_blocks_<kind>.cu), so the four kinds compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "cm_kernels.h"

namespace cm {

constexpr int TILE = 32;       // tile of the coarse path's block sums
constexpr int COARSE_LB = 6;   // first level on the coarse path (b = 1 << COARSE_LB)

// One colour phase of a level with b in 2 .. 2048 (the per-phase kernels).
template <int KIND>
cudaError_t blocks_phase_kind(const PhaseArgs& A, cudaStream_t st);
// One colour phase of a level with the paper's block side A.bs = 2^j - 1 >= 3
// (A.lb = j: the shapes of side 1 << j).
template <int KIND>
cudaError_t blocks_phase_odd_kind(const PhaseArgs& A, cudaStream_t st);
// One colour's search on the coarse path (b >= 1 << COARSE_LB).
template <int KIND>
cudaError_t coarse_phase_kind(const PhaseArgs& A, const float* partials, float* cj,
                              cudaStream_t st);
// Allow the non-portable cluster sizes of this kind's coarse kernels.
template <int KIND>
cudaError_t coarse_setup_kind();

}  // namespace cm
