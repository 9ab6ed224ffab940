// cm_recon.h -- reconstruction extension (Sec. 5): host side of cm_recon.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cm {

struct ReconWork;   // device buffers, the FFT plan and the captured cycle

ReconWork* recon_work_create();
void recon_work_destroy(ReconWork* w);

struct ReconArgs {
    const float2* kspace;     // b, device, H x W complex (zero off the mask)
    const uint8_t* mask;      // device, H x W, 0 or 1
    int H, W;
    float alpha;
    int kind;
    int levels;               // >= 1
    int sides;                // block sides: 0 powers of two, 1 the paper's 2^j - 1
    int ncolors;              // 2, 4, 9, 16 or 0 (decoupled)
    int cycles;
    int cg_iters;
    const float* u0;          // device, nullable (zero-filled Re(A^H b))
    float* u;                 // device, H x W: the result
    double* trace_host;       // nullable, cycles + 1 entries: J before and after each cycle
};

// Runs the reconstruction on `st` and synchronises it.  Returns 0, or
// 3 when out of memory, 2 for a CUDA or cuFFT failure (with *msg set).
int recon_run(ReconWork* w, const ReconArgs& a, cudaStream_t st, const char** msg);

}  // namespace cm
