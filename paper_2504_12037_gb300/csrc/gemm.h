// Problem descriptors of the batched tcgen05 GEMM (k_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnvan {

enum { GT_F32 = 0, GT_I8 = 1, GT_BF16 = 2 };
enum { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_DX = 2, EPI_MASK = 3 };

// Operand element (row r, k) is ptr[r * sr + k * sk] of type `type`.
struct GemmOperand {
  const void* ptr;
  long long sr, sk;
  int type;
};

// C[M x N] = A[M x K] * B[N x K]^T followed by the epilogue `epi`:
//   EPI_STORE      C[z * split_stride + m * ldc + n] = acc (z = K split)
//   EPI_BIAS_RELU  C[m * ldc + n] = max(acc + bias[n], 0)
//   EPI_DX         x = acc + bias[n]; s = spins[m * ld_spins + n];
//                  C[m * ldc + n] = row_w[m] * s / (1 + exp(s x))
//   EPI_MASK       C[m * ldc + n] = mask[m * ld_mask + n] > 0 ? acc : 0
// ones_col >= 0 appends a B row of ones at that column index; its result
// (the row sums of A) goes to bias_out[z * split_stride + m].
// In BF16 launches C and mask of EPI_BIAS_RELU, EPI_DX and EPI_MASK are BF16
// arrays (the next product's operands), C of EPI_STORE stays FP32.
struct GemmProblem {
  int M, N, K;
  GemmOperand A, B;
  int ones_col;
  int epi;
  void* C;  // float, or BF16 (see above)
  long long ldc, split_stride;
  float* bias_out;
  const float* bias;
  const int8_t* spins;
  long long ld_spins;
  const float* row_w;
  const void* mask;  // float, or BF16 (see above)
  long long ld_mask;
};

#define GEMM_MAX_PROB 40

struct GemmLaunch {
  int* status;
  int ncb;  // column blocks per M tile (set by launch_gemm)
  GemmProblem prob[GEMM_MAX_PROB];
};

cudaError_t launch_gemm(const GemmLaunch& L, int n_prob, int max_m, int splits, bool bf16,
                        cudaStream_t s);
int gemm_smem_bytes(bool bf16);

}  // namespace tnvan
