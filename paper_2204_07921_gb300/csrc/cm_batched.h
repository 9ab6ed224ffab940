// cm_batched.h -- device-side pieces of the batched solve (cm_batched.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace cm {

struct ImgDev;   // per-image stopping state (opaque to the host runtime)

size_t batch_state_bytes();    // bytes of one image's state
size_t batch_active_offset();  // offset of its int `active` flag
cudaError_t launch_batch_init(ImgDev* st, const double* E0, int n, int cycles, cudaStream_t s);
cudaError_t launch_batch_stop(ImgDev* st, const double* E_now, double tol, int cap,
                              double* trace, int trace_cap, cudaStream_t s);
// Single-image solve graph: initial state from the energy E0 (and the loop
// condition h), and the stopping test after a cycle (sets h to `active`).
cudaError_t launch_solve_init(ImgDev* st, const double* E0, int cycles, double* trace,
                              cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_solve_stop(ImgDev* st, const double* E_now, double tol, int cap, double* trace,
                              int trace_cap, cudaGraphConditionalHandle h, cudaStream_t s);
// Batched solve graph: sets the loop condition to "some image is active".
cudaError_t launch_batch_any(const ImgDev* st, int n, cudaGraphConditionalHandle h,
                             cudaStream_t s);
cudaError_t launch_batch_copy(const float* src, float* dst, size_t n, const int* active,
                              cudaStream_t s);
// Unpack one image's state copied to the host.
void batch_read_state(const void* host_state, int* cycles, int* converged, int* viol,
                      double* E, int* numeric_error, int* active);

}  // namespace cm
