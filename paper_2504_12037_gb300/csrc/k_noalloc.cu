// Allocation-free variant of the free-energy reduction.
//
// Some callers cannot call cudaMalloc at all: code running under an external
// memory manager that forbids device allocations, plugins that must not grow
// the process's device footprint, or launch paths where an allocation would
// synchronise the device.  tnvan_free_energy_noalloc serves them: it takes no
// context, allocates nothing, and keeps its scratch (the per-block partial
// tuples and per-instance statistics of the two-pass reduction) in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.
#include <mutex>

#include "common.cuh"

namespace tnvan {

// The two-pass FP64 reduction kernels (k_train.cu).
__global__ void reduce_part_kernel(const LaunchInfo li, int n_part, const double* __restrict__ logZR,
                                   const float* __restrict__ logq, double* __restrict__ part);
__global__ void reduce_final_kernel(const LaunchInfo li, int n_part, const double* __restrict__ part,
                                    double* __restrict__ stats);

#define NOALLOC_MAX_INST 128
#define NOALLOC_TUPLES 2048  // partial tuples (6 doubles each) shared by all instances
#define NOALLOC_DOUBLES (8 * NOALLOC_MAX_INST + 6 * NOALLOC_TUPLES)

// 106,496 bytes per device.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

__global__ void noalloc_out_kernel(int n_inst, const double* __restrict__ stats, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_inst) return;
  for (int j = 0; j < 4; ++j) out[5 * k + j] = stats[8 * k + j];
  out[5 * k + 4] = stats[8 * k + 5];
}

namespace {
std::mutex g_mu;
double* g_ptr[256] = {nullptr};
thread_local char g_err[256] = "";

int set_err(int code, const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return code;
}
}  // namespace

}  // namespace tnvan

using namespace tnvan;

extern "C" {

const char* tnvan_noalloc_last_error(void) { return g_err; }

int tnvan_free_energy_noalloc(int n_inst, int batch, const double* betas, const double* d_logZR,
                              const float* d_logq, double* d_out, void* stream) {
  if (n_inst < 1 || n_inst > NOALLOC_MAX_INST)
    return set_err(TNVAN_E_ARG, "n_inst must be in [1, 128]");
  if (batch < 1) return set_err(TNVAN_E_ARG, "batch must be >= 1");
  if (!betas || !d_logZR || !d_logq || !d_out) return set_err(TNVAN_E_ARG, "NULL pointer");
  LaunchInfo li;
  memset(&li, 0, sizeof li);
  li.n_inst = n_inst;
  li.batch = batch;
  li.tile = 1;
  for (int k = 0; k < n_inst; ++k) {
    if (!(betas[k] > 0.0) || !isfinite(betas[k])) return set_err(TNVAN_E_ARG, "betas must be finite and > 0");
    li.beta[k] = betas[k];
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return set_err(TNVAN_E_CUDA, "cudaGetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  {
    // The host-side symbol is only a stand-in: the kernels need the device
    // address of this device's copy of the array.  It is looked up on every
    // call made outside stream capture (so a device reset, which reloads the
    // module, cannot leave a stale address behind) and cached per device for
    // calls made while `stream` is being captured, where the lookup may not
    // run; the first call on a device must therefore come before any capture.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return set_err(TNVAN_E_CUDA, "cudaStreamIsCapturing failed");
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return set_err(TNVAN_E_CUDA, cudaGetErrorString(e));
      g_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_ptr[dev];
  }
  int n_part = (batch + 1023) / 1024;
  if (n_part > 64) n_part = 64;
  if (n_part > NOALLOC_TUPLES / n_inst) n_part = NOALLOC_TUPLES / n_inst;
  if (n_part < 1) n_part = 1;
  double* stats = scratch;
  double* part = scratch + 8 * NOALLOC_MAX_INST;
  // every tuple and statistic read below is written first: nothing to clear
  reduce_part_kernel<<<dim3(n_part, n_inst), 256, 0, s>>>(li, n_part, d_logZR, d_logq, part);
  reduce_final_kernel<<<n_inst, 32, 0, s>>>(li, n_part, part, stats);
  noalloc_out_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(n_inst, stats, d_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(TNVAN_E_CUDA, cudaGetErrorString(e));
  return TNVAN_OK;
}

}  // extern "C"
