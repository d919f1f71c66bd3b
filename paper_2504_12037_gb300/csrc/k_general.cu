// General leftover components (placeholder until the elimination kernels land).
#include "common.cuh"
namespace tnvan {
cudaError_t launch_general(const InstDev*, const LaunchInfo&, int, const int8_t*, double*, double*,
                           double*, cudaStream_t) {
  return cudaSuccess;
}
}  // namespace tnvan
