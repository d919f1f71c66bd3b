// Dense leftover block (placeholder until the dense kernels land).
#include "common.cuh"
namespace tnvan {
cudaError_t launch_dense(const InstDev*, const LaunchInfo&, int, const int8_t*, double*, double*,
                         double*, cudaStream_t) {
  return cudaSuccess;
}
}  // namespace tnvan
