// cm_batched.cu -- many images of uneven sizes solved together.
//
// One CUDA graph holds one cycle of every image: an independent chain per
// image (all its levels and colours, its FP64 energy and its stopping test),
// forked from and joined to one capture stream.  The graph executor runs the
// chains of different images concurrently, so the fine levels of one image
// overlap the latency-bound coarse levels of another and the GPU stays full.
// Ordering inside an image comes from the graph's edges, never from a kernel
// waiting on another, so no kernel spins.  Each image's stopping test (Eq.
// reerr) runs on the device and clears the image's `active` flag; every kernel
// of a retired image returns at entry.  The cycle is the body of a
// conditional WHILE node whose condition batch_any_kernel sets to "some image
// is active" after each cycle, so the whole batch is one graph launch; the
// loop is finite because every image retires at its cycle cap.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/cm.h"
#include "cm_batched.h"
#include "cm_kernels.h"

namespace cm {

struct ImgDev {
    double E_prev;
    double E;
    int active;
    int cycles;
    int viol;
    int converged;
    int numeric_error;
    int pad;
};

__global__ void batch_init_kernel(ImgDev* st, const double* E0, int n, int cycles) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    st[i].E_prev = E0[i];
    st[i].E = E0[i];
    st[i].active = cycles > 0 ? 1 : 0;
    st[i].cycles = 0;
    st[i].viol = 0;
    st[i].converged = 0;
    st[i].numeric_error = isfinite(E0[i]) ? 0 : 1;
    if (!isfinite(E0[i])) st[i].active = 0;
}

// Stopping test of one image after a cycle (Eq. reerr), on the device.
__device__ void stop_test(ImgDev* st, double E, double tol, int cap, double* trace, int trace_cap) {
    const int l = st->cycles + 1;
    st->cycles = l;
    st->E = E;
    if (l <= trace_cap) trace[l] = E;
    if (!isfinite(E)) {
        st->numeric_error = 1;
        st->active = 0;
        return;
    }
    if (E > st->E_prev) st->viol += 1;
    const bool stop = tol > 0.0 && fabs(E - st->E_prev) <= tol * fabs(E);
    st->E_prev = E;
    if (stop) {
        st->converged = 1;
        st->active = 0;
    } else if (l >= cap) {
        st->active = 0;
    }
}

__global__ void batch_stop_kernel(ImgDev* st, const double* E_now, double tol, int cap,
                                  double* trace, int trace_cap) {
    if (threadIdx.x != 0 || st->active == 0) return;
    stop_test(st, *E_now, tol, cap, trace, trace_cap);
}

// Single-image solve as one graph: the loop of cycles is a conditional WHILE
// node whose condition these kernels set from the image's state.
__global__ void solve_init_kernel(ImgDev* st, const double* E0, int cycles, double* trace,
                                  cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    const double E = *E0;
    st->E_prev = E;
    st->E = E;
    st->cycles = 0;
    st->viol = 0;
    st->converged = 0;
    st->numeric_error = isfinite(E) ? 0 : 1;
    st->active = (cycles > 0 && isfinite(E)) ? 1 : 0;
    trace[0] = E;
    cudaGraphSetConditional(h, (unsigned)st->active);
}

__global__ void solve_stop_kernel(ImgDev* st, const double* E_now, double tol, int cap,
                                  double* trace, int trace_cap, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    if (st->active) stop_test(st, *E_now, tol, cap, trace, trace_cap);
    cudaGraphSetConditional(h, (unsigned)st->active);
}

__global__ void batch_copy_kernel(const float* __restrict__ src, float* __restrict__ dst, size_t n,
                                  const int* __restrict__ active) {
    if (active && *active == 0) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t launch_batch_init(ImgDev* st, const double* E0, int n, int cycles, cudaStream_t s) {
    batch_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, E0, n, cycles);
    return cudaGetLastError();
}

cudaError_t launch_batch_stop(ImgDev* st, const double* E_now, double tol, int cap,
                              double* trace, int trace_cap, cudaStream_t s) {
    batch_stop_kernel<<<1, 32, 0, s>>>(st, E_now, tol, cap, trace, trace_cap);
    return cudaGetLastError();
}

// Loop condition of the batched solve graph: 1 while any image is active.
__global__ void batch_any_kernel(const ImgDev* st, int n, cudaGraphConditionalHandle h) {
    int any = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) any |= st[i].active;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

cudaError_t launch_batch_any(const ImgDev* st, int n, cudaGraphConditionalHandle h,
                             cudaStream_t s) {
    batch_any_kernel<<<1, 256, 0, s>>>(st, n, h);
    return cudaGetLastError();
}

cudaError_t launch_solve_init(ImgDev* st, const double* E0, int cycles, double* trace,
                              cudaGraphConditionalHandle h, cudaStream_t s) {
    solve_init_kernel<<<1, 32, 0, s>>>(st, E0, cycles, trace, h);
    return cudaGetLastError();
}

cudaError_t launch_solve_stop(ImgDev* st, const double* E_now, double tol, int cap, double* trace,
                              int trace_cap, cudaGraphConditionalHandle h, cudaStream_t s) {
    solve_stop_kernel<<<1, 32, 0, s>>>(st, E_now, tol, cap, trace, trace_cap, h);
    return cudaGetLastError();
}

cudaError_t launch_batch_copy(const float* src, float* dst, size_t n, const int* active,
                              cudaStream_t s) {
    int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    batch_copy_kernel<<<grid, 256, 0, s>>>(src, dst, n, active);
    return cudaGetLastError();
}

size_t batch_state_bytes() { return sizeof(ImgDev); }
size_t batch_active_offset() { return offsetof(ImgDev, active); }

void batch_read_state(const void* host_state, int* cycles, int* converged, int* viol,
                      double* E, int* numeric_error, int* active) {
    const ImgDev* s = static_cast<const ImgDev*>(host_state);
    *cycles = s->cycles;
    *converged = s->converged;
    *viol = s->viol;
    *E = s->E;
    *numeric_error = s->numeric_error;
    *active = s->active;
}

}  // namespace cm
