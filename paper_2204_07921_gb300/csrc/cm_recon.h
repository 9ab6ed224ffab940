// cm_recon.h -- reconstruction extension (Sec. 5): host side of cm_recon.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cm {

struct ReconWork;   // device buffers, the FFT tables and the captured cycle

ReconWork* recon_work_create();
void recon_work_destroy(ReconWork* w);

enum { RECON_MRI = 0, RECON_CT = 1 };

// CT detector: D = 2 ceil(hypot(H - 1, W - 1) / 2) + 3 unit bins.
int radon_bins(int H, int W);

struct ReconArgs {
    int op = RECON_MRI;       // the operator A
    const float2* kspace;     // MRI: b, device, H x W complex (zero off the mask)
    const uint8_t* mask;      // MRI: device, H x W, 0 or 1
    const float* sino;        // CT: b, device, n_angles x radon_bins(H, W)
    int n_angles;             // CT: angles pi a / n_angles
    int H, W;
    float alpha;
    int kind;
    int levels;               // >= 1
    int sides;                // block sides: 0 powers of two, 1 the paper's 2^j - 1
    int ncolors;              // 2, 4, 9, 16 or 0 (decoupled)
    int cycles;
    int cg_iters;
    const float* u0;          // device, nullable (MRI: zero-filled Re(A^H b); CT: FBP)
    float* u;                 // device, H x W: the result
    double* trace_host;       // nullable, cycles + 1 entries: J before and after each cycle
};

// Runs the reconstruction on `st` and synchronises it.  Returns 0, 1 for an
// MRI image size beyond the transform's limits (fft_length_ok), 3 when out of
// memory, 2 for a CUDA failure (with *msg set).
int recon_run(ReconWork* w, const ReconArgs& a, cudaStream_t st, const char** msg);

// The CT operator pair alone (device buffers; allocates temporaries;
// synchronises st): sino = R u, and u = R^T sino.
int radon_forward(const float* u, int H, int W, int n_angles, float* sino, cudaStream_t st,
                  const char** msg);
int radon_adjoint(const float* sino, int n_angles, int H, int W, float* u, cudaStream_t st,
                  const char** msg);

}  // namespace cm
