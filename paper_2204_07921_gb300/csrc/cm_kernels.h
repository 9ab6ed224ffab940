// cm_kernels.h -- host-side launchers of the sweep and energy kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace cm {

// Launch `kern` on st, as a grid of thread-block clusters of cluster_x CTAs
// when cluster_x > 1.
template <class... KArgs, class... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                            unsigned cluster_x, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster_x;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cluster_x > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Blocks per colour slot on a level with nbi x nbj blocks (an upper bound
// for every colour; active_block maps a slot to a block or rejects it).
inline int active_slots(int nbi, int nbj, int ncol) {
    if (ncol == 2) return nbi * ((nbj + 1) / 2);
    const int p = ncol == 16 ? 4 : (ncol == 9 ? 3 : (ncol == 1 ? 1 : 2));
    return ((nbi + p - 1) / p) * ((nbj + p - 1) / p);
}

// Colours of the level with block side b: coarse_ncolors when it is set and
// b >= 64; else ncolors, or for ncolors = 0 the decoupled colouring (the
// smallest p >= 2 with (p - 1) b >= 3, p^2 colours), under which a colour's
// blocks share no stencil.
inline int level_colours(int ncolors, int b, int coarse_ncolors = 0) {
    if (coarse_ncolors != 0 && b >= 64) return coarse_ncolors;
    if (ncolors != 0) return ncolors;
    int p = 2;
    while ((p - 1) * b < 3) ++p;
    return p * p;
}

// Block side of level j = 0, 1, ...: 1 << j, or with the paper's sides
// (sides = 1, Sec. 2.2) 2^(j+1) - 1.
inline int level_side(int j, int sides) { return sides ? (2 << j) - 1 : 1 << j; }

// Kernel shape class of block side b: the smallest lb with b <= 1 << lb.
inline int side_class(int b) {
    int lb = 0;
    while ((1 << lb) < b) ++lb;
    return lb;
}

// Default level count: the coarsest block side is the largest one <= half
// the shorter image side.
inline int auto_levels(int H, int W, int sides) {
    const int m = H < W ? H : W;
    int L = 1;
    while (level_side(L, sides) <= m / 2) ++L;
    return L;
}

struct PhaseArgs {
    const float* S;   // state at the start of the level
    float* R;         // blocks already updated on this level (and the output)
    const float* f;
    int H, W;
    float alpha;
    int kind;
    int lb;           // kernel shape class: block side bs <= 1 << lb
    int bs;           // block side: 1 << lb, or the paper's 2^lb - 1
    int ncolors;      // 2 or 4
    int colour;
    int G, K;         // block-search budget
    int use_paper;    // paper's one-step candidate on the finest level
    int one_step = 0; // the paper's single step per block instead of the search
    int coarse_spec = -1;   // coarse levels: first-pair speculation (-1: the level's default)
    int coarse_dmax = 0;    // coarse levels: golden steps per reduction (0: the level's default)
    int shapes = 0;         // bit lb - 1: the alternative kernel shape of level b = 1 << lb (2 .. 32)
    float* c_out;     // nullable: per-block corrections
    const int* active = nullptr;   // nullable: kernels return at once when *active == 0
    // Levels b >= 2 (not the coarse path): reads take R for the blocks of
    // colours below read_colour (-1: the phase's colour).  0 with R == S runs
    // the level in place, valid when no block's read window (the block and
    // 2 pixels around it) reaches another block of its colour:
    // in_place_ok(b, ncolors).
    int read_colour = -1;
};

// A level of block side b >= 2 with p x p colours can run in place: blocks of
// one colour are (p - 1) b >= 2 pixels apart, beyond each other's 2-pixel
// read window (two colours: diagonal neighbours touch).
inline bool in_place_ok(int b, int ncolors) {
    const int p = ncolors == 4 ? 2 : ncolors == 9 ? 3 : ncolors == 16 ? 4 : 0;
    return b >= 2 && p >= 2 && (p - 1) * b >= 2;
}

cudaError_t launch_energy(const float* u, const float* f, int H, int W, float alpha, int kind,
                          double* partials, unsigned int* ticket, double* E_out,
                          cudaStream_t st, const int* active = nullptr);
size_t energy_partials_needed(int H, int W);
cudaError_t launch_curvature(const float* u, int H, int W, int kind, float* out,
                             cudaStream_t st);
cudaError_t launch_phase(const PhaseArgs& a, cudaStream_t st);          // dispatch by level
cudaError_t launch_phase_b1(const PhaseArgs& a, cudaStream_t st);       // b = 1
cudaError_t launch_phase_blocks(const PhaseArgs& a, cudaStream_t st);   // b >= 2
int max_level_log2();

// Coarse path (block side >= 1 << coarse_level_log2()): a whole level at once.
// partials: coarse_partials_needed() floats; cj: coarse_c_needed() floats.
int coarse_level_log2();
size_t coarse_partials_needed(int H, int W);
size_t coarse_c_needed(int H, int W);
// sums_ready: `partials` already holds the tile sums of S - f (written by the
// previous coarse level's apply, which leaves those of its output).
cudaError_t launch_level_coarse(const PhaseArgs& a, float* partials, float* cj, cudaStream_t st,
                                bool sums_ready = false);
// Per-process kernel attributes of the coarse path (cluster sizes above 8);
// call before the first launch, outside stream capture.
cudaError_t coarse_setup();

}  // namespace cm
