// cm_cnn.h -- the warm-start network as seen by the runtime (cm_api.cu).
#pragma once
#include <cuda_runtime.h>

namespace cm {
namespace cnn {

struct Net;
// u0 = f + net(f) for N images of H x W (device pointers), on stream st.
int net_forward(Net* net, const float* f, int N, int H, int W, float* u0, cudaStream_t st);
const char* net_error(const Net* net);
// After a synchronisation: CM_ERR_CUDA if a tensor-core wait timed out.
int net_status(Net* net);

}  // namespace cnn
}  // namespace cm
