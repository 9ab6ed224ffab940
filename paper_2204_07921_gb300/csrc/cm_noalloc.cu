// cm_noalloc.cu -- energy evaluation that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc: a host whose caching
// allocator has already reserved (nearly) all device memory, code that must
// not take the implicit device-wide synchronisation that cudaMalloc and
// cudaFree bring, and pipelines with a hard no-allocation rule after start-up
// (real-time and embedded deployments).  cm_energy_noalloc serves them: it
// launches the same energy kernel as cm_energy, but its scratch -- the FP64
// per-CTA partial sums and the arrival counter of the deterministic finish --
// lives in the file-scope array below, which every GPU that loads the library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cm.h"
#include "cm_kernels.h"

namespace {

// Capacity: one FP64 partial per 32 x 32 tile of the image, for up to
// CM_NOALLOC_MAX_TILES tiles, then the 32-bit arrival counter.
constexpr size_t kPartialBytes = (size_t)CM_NOALLOC_MAX_TILES * sizeof(double);
constexpr size_t kScratchBytes = kPartialBytes + 256;

static __device__ __align__(256) unsigned char g_energy_scratch[kScratchBytes];

// Device address of g_energy_scratch, looked up once per device (the name is
// only a host-side stand-in in host code) and kept for the life of the
// process.  cudaDeviceReset destroys the module that holds the array, so the
// kept address is stale afterwards: a process that resets a device must not
// call cm_energy_noalloc on it again.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) return CM_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CM_OK;
}

}  // namespace

extern "C" int cm_energy_noalloc(const float* u, const float* f, int H, int W, float alpha,
                                 int kind, double* E_dev, void* stream) {
    if (!u || !f || !E_dev || H < 1 || W < 1 || !(alpha > 0.0f) || alpha != alpha ||
        alpha > 3.0e38f || kind < 0 || kind > 3)
        return CM_ERR_INVALID;
    // the image limits of every entry point first (the tile count below is
    // computed in int), then the energy kernel's grid: one CTA per 32 x 32 tile
    if (H > CM_MAX_SIDE || W > CM_MAX_SIDE || (long long)H * W > CM_MAX_PIXELS)
        return CM_ERR_INVALID;
    if (cm::energy_partials_needed(H, W) > (size_t)CM_NOALLOC_MAX_TILES) return CM_ERR_INVALID;
    void* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc != CM_OK) return rc;
    double* partials = static_cast<double*>(base);
    unsigned int* ticket =
        reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(base) + kPartialBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero whatever the last call left
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return CM_ERR_CUDA;
    if (cm::launch_energy(u, f, H, W, alpha, kind, partials, ticket, E_dev, st) != cudaSuccess)
        return CM_ERR_CUDA;
    return CM_OK;
}
