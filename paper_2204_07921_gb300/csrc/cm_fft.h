// cm_fft.h -- the 2-D discrete Fourier transform of the MRI-like operator
// A = M F of the reconstruction extension (Sec. 5): host side of cm_fft.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cm {

// Largest transform held in shared memory by one CTA (complex points).  A
// line of power-of-two length n <= FFT_MAX_M is transformed directly; any
// other n uses a transform of the power of two M >= 2n - 1 (Bluestein), so
// n <= FFT_MAX_M / 2.
constexpr int FFT_MAX_M = 16384;

// True when lines of length n can be transformed.
bool fft_length_ok(int n);

struct FftAxis;   // device tables of one axis (twiddles, chirp, chirp spectrum)

struct FftPlan {
    int H = 0, W = 0;
    FftAxis* rows = nullptr;   // transforms of length W along the rows
    FftAxis* cols = nullptr;   // transforms of length H along the columns
};

// Builds the tables of an H x W plan (computed in FP64 on the host, stored
// as FP32 on the device; synchronous).  Returns 0, 1 for a length that
// fft_length_ok rejects, 2 for a CUDA failure, 3 when out of memory.
int fft_plan_make(FftPlan* p, int H, int W);
void fft_plan_free(FftPlan* p);

// In place, on `st`: X (H x W complex, row-major) <- its unnormalised 2-D
// DFT, X[k, l] = sum_{r, c} X[r, c] exp(-+2 pi i (k r / H + l c / W)), the
// minus sign for the forward transform, the plus sign for the inverse.  With
// mask (H x W, nullable) every output entry is then multiplied by mscale
// where mask is nonzero and set to 0 elsewhere, in the last pass's store
// (H W > 1: a 1 x 1 image has no pass, and a mask is then refused).
// No allocation; the launches can be captured in a CUDA graph.
cudaError_t fft2d(const FftPlan& p, float2* X, bool inverse, cudaStream_t st,
                  const uint8_t* mask = nullptr, float mscale = 1.0f);

// Dynamic shared memory of the line kernels above 48 KB (once per process).
cudaError_t fft_setup();

}  // namespace cm
