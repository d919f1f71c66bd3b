// Batched tensor-core GEMM on tcgen05 (sm_103a) with fused epilogues, used by
// the TF32 / BF16 backward of the network (Eq. 10).
//
// One CTA (128 threads) computes a 128-row tile of C[M x N] = A[M x K] B[N x K]^T
// (N <= 256) for one problem of the launch.  A and B are read from global
// memory through arbitrary (row, k) strides -- so transposed operands cost
// nothing extra -- into the canonical no-swizzle shared-memory layouts (K- or
// MN-major).  BF16 operands in aligned rows (the chain's intermediates and
// the BF16 copy of the weights) arrive by 16-byte asynchronous copies through
// a ring of four K stages of 32 elements, three in flight while the tensor
// core works on the fourth; FP32 and int8 operands are converted by the
// threads when their stage is filled (TF32: two stages).  One elected thread
// issues tcgen05.mma into a TMEM accumulator and commits each stage to an
// mbarrier, which frees the stage's slot for the stage NS - 1 ahead.  The
// epilogue reads the accumulator row per thread (tcgen05.ld), applies the
// fused operation and writes the next product's operand in BF16 (TF32: FP32).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gemm.h"
#include "tc.cuh"

namespace tnvan {

#define GM 128
#define GN 64  // columns per CTA
#define GK 32
#define GNS_BF16 4  // BF16: K stages in flight (asynchronous copies)

template <int TYPE>
__device__ __forceinline__ float load_elem(const void* p, long long idx) {
  if (TYPE == GT_F32) return static_cast<const float*>(p)[idx];
  if (TYPE == GT_I8) return (float)static_cast<const int8_t*>(p)[idx];
  return 0.f;
}

__device__ __forceinline__ float load_any(int type, const void* p, long long idx) {
  if (type == GT_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
  return type == GT_F32 ? static_cast<const float*>(p)[idx]
                        : (float)static_cast<const int8_t*>(p)[idx];
}

// Store 4 consecutive-k values of row r (k multiple of 4) into the K-major stage.
template <bool BF16>
__device__ __forceinline__ void st4k(unsigned char* s, int r, int k, float4 v) {
  constexpr int EL = BF16 ? 2 : 4;
  const uint32_t o = tc::kmajor_off(r, k, GK * EL, EL);
  if (BF16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(s + o) = u;
  } else {
    *reinterpret_cast<float4*>(s + o) = v;
  }
}

template <bool BF16>
__device__ __forceinline__ void st1(unsigned char* s, int r, int k, float v) {
  constexpr int EL = BF16 ? 2 : 4;
  const uint32_t o = tc::kmajor_off(r, k, GK * EL, EL);
  if (BF16) *reinterpret_cast<__nv_bfloat16*>(s + o) = __float2bfloat16(v);
  else *reinterpret_cast<float*>(s + o) = v;
}

// BF16 operands contiguous along their rows (transposed: the weight-gradient
// operands, the transposed weights) are staged MN-major instead: element
// (r, k) at (r >> 3) * MN_SBO + (k >> 3) * 128 + (k & 7) * 16 + (r & 7) * 2, so
// four consecutive rows at one k are one 8-byte store; the MMA reads them
// with the operand's major bit set.  MN_SBO pads each 8-row group by 16 bytes.
#define MN_SBO (GK * 2 / 16 * 128 + 16)
#define GSTAGE_BF16 (16 * MN_SBO)  // bytes of one BF16 A stage (either layout, 128 rows)
#define GSTAGE_B_BF16 (GN / 8 * MN_SBO)  // the same for B (GN rows)
__device__ __forceinline__ uint32_t mn_off(int r, int k) {
  return (uint32_t)((r >> 3) * MN_SBO + (k >> 3) * 128 + (k & 7) * 16 + (r & 7) * 2);
}
__device__ __forceinline__ void st4r_bf16(unsigned char* s, int r, int k, float a, float b, float c, float d) {
  __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t*>(&x);
  u.y = *reinterpret_cast<uint32_t*>(&y);
  *reinterpret_cast<uint2*>(s + mn_off(r, k)) = u;
}

// Whether fill_stage stages this operand MN-major (BF16 only; the transposed
// FP32 or int8 paths, and BF16 operands read in 16-byte granules along rows).
__device__ __forceinline__ bool operand_mn(const GemmOperand& op, int r0, int nrows) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(op.ptr);
  if (op.sr != 1 || op.sk == 1 || (op.sk & 3) != 0 || (r0 & 3) != 0 || (nrows & 3) != 0) return false;
  if (op.type == GT_F32) return (a & 15) == 0;
  if (op.type == GT_I8) return (a & 3) == 0;
  if (op.type == GT_BF16) return (a & 15) == 0 && (op.sk & 7) == 0 && (r0 & 7) == 0 && (nrows & 7) == 0;
  return false;
}

// Whether a BF16 operand's stages are fetched with 16-byte asynchronous copies
// (granules of 8 elements along the operand's contiguous index, aligned).
__device__ __forceinline__ bool operand_async(const GemmOperand& op, bool mn) {
  if (op.type != GT_BF16 || (reinterpret_cast<uintptr_t>(op.ptr) & 15) != 0) return false;
  return mn || (op.sk == 1 && (op.sr & 7) == 0);
}

// One 16-byte asynchronous copy global -> shared; src_bytes < 16 zero-fills
// the rest (0: nothing is read).
__device__ __forceinline__ void cp16(unsigned char* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Asynchronous fill of one BF16 stage: rows [r0, r0 + nrows), k in [k0, k0 +
// GK); rows >= rlim or k >= klim zero.  The granule that holds the ones row
// (the bias column) is written by the thread instead (a plain store).
__device__ void fill_stage_async(unsigned char* s, int nrows, const GemmOperand& op, int r0, int rlim, int k0,
                                 int klim, int ones_row, int t, bool mn) {
  const uint16_t* p = static_cast<const uint16_t*>(op.ptr);
  const uint16_t one = 0x3F80u;  // 1.0 in BF16
  if (!mn) {  // K-major: granule = row r, k .. k + 7
    const int units = nrows * (GK / 8);
    for (int u = t; u < units; u += 128) {
      const int r = u >> 2, kq = (u & 3) * 8;
      const int gr = r0 + r, gk = k0 + kq;
      unsigned char* dst = s + tc::kmajor_off(r, kq, GK * 2, 2);
      if (gr == ones_row) {
        uint16_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = gk + j < klim ? one : (uint16_t)0;
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
      } else {
        const int nv = gr < rlim ? max(0, min(8, klim - gk)) : 0;
        cp16(dst, nv ? static_cast<const void*>(p + (long long)gr * op.sr + gk) : op.ptr, 2u * (uint32_t)nv);
      }
    }
  } else {  // MN-major: granule = rows r .. r + 7 at one k
    const int rg = nrows >> 3;
    const int units = rg * GK;
    for (int u = t; u < units; u += 128) {
      const int r = (u % rg) * 8, k = u / rg;
      const int gr = r0 + r, gk = k0 + k;
      unsigned char* dst = s + mn_off(r, k);
      if (ones_row >= gr && ones_row < gr + 8) {
        uint16_t h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          h[i] = 0;
          if (gk < klim) h[i] = gr + i == ones_row ? one : (gr + i < rlim ? p[(long long)gk * op.sk + gr + i] : (uint16_t)0);
        }
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
      } else {
        const int nv = gk < klim ? max(0, min(8, rlim - gr)) : 0;
        cp16(dst, nv ? static_cast<const void*>(p + (long long)gk * op.sk + gr) : op.ptr, 2u * (uint32_t)nv);
      }
    }
  }
}

// Fill one K stage: rows [r0, r0 + nrows) of an operand, k in [k0, k0 + GK).
// Rows >= rlim or k >= klim are zero; row == ones_row reads 1 (bias column).
// Loads are issued in batches (registers first, stores after) so that each
// thread keeps many global loads in flight; FP32 operands whose contiguous
// index is k (or the row) are read as float4.
template <bool BF16>
__device__ __forceinline__ void fill_stage(unsigned char* s, int nrows, const GemmOperand& op,
                                           int r0, int rlim, int k0, int klim, int ones_row, int t, bool mn) {
  const bool full_k = k0 + GK <= klim;
  const bool f32 = op.type == GT_F32;
  const bool aligned = ((reinterpret_cast<uintptr_t>(op.ptr) & 15) == 0);
  if (!mn && f32 && aligned && full_k && op.sk == 1 && (op.sr & 3) == 0) {
    // row-major along k: units of (row, 4 k)
    const float* p = static_cast<const float*>(op.ptr);
    const int units = nrows * (GK / 4);
    for (int u0 = 0; u0 < units; u0 += 128 * 8) {
      float4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        const int r = u >> 3, kq = (u & 7) * 4;
        const int gr = r0 + r;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u < units) {
          if (gr == ones_row) v[j] = make_float4(1.f, 1.f, 1.f, 1.f);
          else if (gr < rlim)
            v[j] = __ldg(reinterpret_cast<const float4*>(p + (long long)gr * op.sr + k0 + kq));
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        if (u < units) st4k<BF16>(s, u >> 3, (u & 7) * 4, v[j]);
      }
    }
    return;
  }
  if (f32 && aligned && op.sr == 1 && (op.sk & 3) == 0 && (r0 & 3) == 0 && (nrows & 3) == 0) {
    // contiguous along rows (transposed operand): units of (4 rows, k)
    const float* p = static_cast<const float*>(op.ptr);
    const int rq = nrows / 4;
    const int units = rq * GK;
    for (int u0 = 0; u0 < units; u0 += 128 * 8) {
      float4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        const int r = (u % rq) * 4, k = u / rq;
        const int gr = r0 + r, gk = k0 + k;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (u < units && gk < klim) {
          if (gr + 3 < rlim) v[j] = __ldg(reinterpret_cast<const float4*>(p + (long long)gk * op.sk + gr));
          else {
            float e[4] = {0.f, 0.f, 0.f, 0.f};
            for (int i = 0; i < 4; ++i)
              if (gr + i < rlim) e[i] = p[(long long)gk * op.sk + gr + i];
            v[j] = make_float4(e[0], e[1], e[2], e[3]);
          }
          if (ones_row >= gr && ones_row < gr + 4) {
            float* f = reinterpret_cast<float*>(&v[j]);
            f[ones_row - gr] = 1.f;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        if (u < units) {
          const int r = (u % rq) * 4, k = u / rq;
          if (BF16 && mn) {
            st4r_bf16(s, r, k, v[j].x, v[j].y, v[j].z, v[j].w);
          } else {
            st1<BF16>(s, r, k, v[j].x);
            st1<BF16>(s, r + 1, k, v[j].y);
            st1<BF16>(s, r + 2, k, v[j].z);
            st1<BF16>(s, r + 3, k, v[j].w);
          }
        }
      }
    }
    return;
  }
  const bool i8 = op.type == GT_I8;
  const bool aligned4 = ((reinterpret_cast<uintptr_t>(op.ptr) & 3) == 0);
  if (!mn && i8 && aligned4 && full_k && op.sk == 1 && (op.sr & 3) == 0) {
    // int8 rows along k (spins): units of (row, 4 k), four bytes per load
    const int8_t* p = static_cast<const int8_t*>(op.ptr);
    const int units = nrows * (GK / 4);
    for (int u0 = 0; u0 < units; u0 += 128 * 8) {
      char4 c[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        const int gr = r0 + (u >> 3), kq = (u & 7) * 4;
        c[j] = make_char4(0, 0, 0, 0);
        if (u < units && gr != ones_row && gr < rlim)
          c[j] = __ldg(reinterpret_cast<const char4*>(p + (long long)gr * op.sr + k0 + kq));
        if (u < units && gr == ones_row) c[j] = make_char4(1, 1, 1, 1);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        if (u < units)
          st4k<BF16>(s, u >> 3, (u & 7) * 4, make_float4((float)c[j].x, (float)c[j].y, (float)c[j].z, (float)c[j].w));
      }
    }
    return;
  }
  if (i8 && aligned4 && op.sr == 1 && (op.sk & 3) == 0 && (r0 & 3) == 0 && (nrows & 3) == 0) {
    // int8 contiguous along rows (transposed spins): units of (4 rows, k)
    const int8_t* p = static_cast<const int8_t*>(op.ptr);
    const int rq = nrows / 4;
    const int units = rq * GK;
    for (int u0 = 0; u0 < units; u0 += 128 * 8) {
      char4 c[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        const int gr = r0 + (u % rq) * 4, gk = k0 + u / rq;
        c[j] = make_char4(0, 0, 0, 0);
        if (u < units && gk < klim) {
          if (gr + 3 < rlim && (ones_row < gr || ones_row > gr + 3)) {
            c[j] = __ldg(reinterpret_cast<const char4*>(p + (long long)gk * op.sk + gr));
          } else {
            signed char e[4] = {0, 0, 0, 0};
            for (int i = 0; i < 4; ++i) {
              if (gr + i == ones_row) e[i] = 1;
              else if (gr + i < rlim) e[i] = p[(long long)gk * op.sk + gr + i];
            }
            c[j] = make_char4(e[0], e[1], e[2], e[3]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = u0 + t + 128 * j;
        if (u < units) {
          const int r = (u % rq) * 4, k = u / rq;
          if (BF16 && mn) {
            st4r_bf16(s, r, k, (float)c[j].x, (float)c[j].y, (float)c[j].z, (float)c[j].w);
          } else {
            st1<BF16>(s, r, k, (float)c[j].x);
            st1<BF16>(s, r + 1, k, (float)c[j].y);
            st1<BF16>(s, r + 2, k, (float)c[j].z);
            st1<BF16>(s, r + 3, k, (float)c[j].w);
          }
        }
      }
    }
    return;
  }
  // generic: element by element, loads batched 16 at a time
  const bool kfast = op.sk == 1;
  const int total = nrows * GK;
  for (int e0 = 0; e0 < total; e0 += 128 * 16) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = e0 + t + 128 * j;
      int r, k;
      if (kfast) {
        r = e / GK;
        k = e % GK;
      } else {
        r = e % nrows;
        k = e / nrows;
      }
      const int gr = r0 + r, gk = k0 + k;
      float x = 0.f;
      if (e < total) {
        if (gr == ones_row) x = gk < klim ? 1.f : 0.f;
        else if (gr < rlim && gk < klim)
          x = load_any(op.type, op.ptr, (long long)gr * op.sr + (long long)gk * op.sk);
      }
      v[j] = x;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = e0 + t + 128 * j;
      if (e < total) {
        int r, k;
        if (kfast) {
          r = e / GK;
          k = e % GK;
        } else {
          r = e % nrows;
          k = e / nrows;
        }
        st1<BF16>(s, r, k, v[j]);
      }
    }
  }
}

// Out of line: both operands share one copy of the paths, which keeps the
// kernels with the larger epilogues within the instruction cache.
template <bool BF16>
__device__ __noinline__ void fill_stage_call(unsigned char* s, int nrows, const GemmOperand& op, int r0, int rlim,
                                             int k0, int klim, int ones_row, int t, bool mn) {
  fill_stage<BF16>(s, nrows, op, r0, rlim, k0, klim, ones_row, t, mn);
}

// EPI: the epilogue of every problem of the launch (one compiled per case).
template <bool BF16, int EPI>
__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmLaunch L) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int EL = BF16 ? 2 : 4;
  constexpr int KB = GK * EL;
  const GemmProblem& P = L.prob[blockIdx.y];
  // blockIdx.x = M tile * L.ncb + column block: this CTA computes columns
  // [n_lo, n_lo + Nc) of the padded N
  const int cb = blockIdx.x % L.ncb;
  const int m0 = (blockIdx.x / L.ncb) * GM;
  if (m0 >= P.M) return;
  const int t = threadIdx.x;
  const int Npad = (P.N + (P.ones_col >= 0 ? 1 : 0) + 15) & ~15;  // padded N (multiple of 16)
  const int n_lo = cb * GN;
  if (n_lo >= Npad) return;
  const int Np = min(GN, Npad - n_lo);
  const int stageA = BF16 ? GSTAGE_BF16 : GM * KB, stageB = BF16 ? GSTAGE_B_BF16 : GN * KB;
  constexpr int NS = BF16 ? GNS_BF16 : 2;  // K stages in the ring
  const bool amn = BF16 && operand_mn(P.A, m0, GM), bmn = BF16 && operand_mn(P.B, n_lo, Np);
  // BF16 operands in aligned 16-byte granules arrive by asynchronous copies,
  // the others are converted by the threads when their stage is filled
  const bool aas = BF16 && operand_async(P.A, amn), bas = BF16 && operand_async(P.B, bmn);
  auto sA = [&](int st) { return smem + st * (stageA + stageB); };
  auto sB = [&](int st) { return smem + st * (stageA + stageB) + stageA; };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * (stageA + stageB));
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + NS);
  // split K
  const int kchunk = (((P.K + gridDim.z - 1) / gridDim.z) + GK - 1) / GK * GK;
  const int kbeg = blockIdx.z * kchunk, kend = min(P.K, kbeg + kchunk);
  if (t == 0)
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
  if (t < 32) {
    tc::tmem_alloc(slot, GN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t id = tc::idesc(GM, Np, BF16 ? 1u : 2u) | (amn ? 1u << 15 : 0u) | (bmn ? 1u << 16 : 0u);
  const int nk = kend > kbeg ? (kend - kbeg + GK - 1) / GK : 0;
  // stage ks into ring slot ks % NS (every thread commits one copy group per
  // stage, empty past the last)
  auto fill = [&](int ks) {
    if (ks < nk) {
      const int st = ks % NS, k0 = kbeg + ks * GK;
      if (aas) fill_stage_async(sA(st), GM, P.A, m0, P.M, k0, kend, -1, t, amn);
      else if (EPI == EPI_STORE) fill_stage<BF16>(sA(st), GM, P.A, m0, P.M, k0, kend, -1, t, amn);
      else fill_stage_call<BF16>(sA(st), GM, P.A, m0, P.M, k0, kend, -1, t, amn);
      if (bas) fill_stage_async(sB(st), Np, P.B, n_lo, P.N, k0, kend, P.ones_col, t, bmn);
      else if (EPI == EPI_STORE) fill_stage<BF16>(sB(st), Np, P.B, n_lo, P.N, k0, kend, P.ones_col, t, bmn);
      else fill_stage_call<BF16>(sB(st), Np, P.B, n_lo, P.N, k0, kend, P.ones_col, t, bmn);
    }
    if (BF16) cp_commit();
  };
  for (int ks = 0; ks < NS - 1; ++ks) fill(ks);
  bool ok = true;
  for (int ks = 0; ks < nk; ++ks) {
    const int st = ks % NS;
    if (BF16) cp_wait<NS - 2>();  // this thread's copies of stage ks have landed
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int kk = 0; kk < KB / 32; ++kk) {
        const uint64_t a = tc::smem_desc(smem_u32(sA(st)) + kk * 256, 128, amn ? MN_SBO : KB / 16 * 128);
        const uint64_t b = tc::smem_desc(smem_u32(sB(st)) + kk * 256, 128, bmn ? MN_SBO : KB / 16 * 128);
        if (BF16) tc::mma_bf16(tmem, a, b, id, (ks > 0 || kk > 0) ? 1u : 0u);
        else tc::mma_tf32(tmem, a, b, id, (ks > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[st]);
    }
    // stage ks + NS - 1 reuses the slot of stage ks - 1: its MMAs first
    if (ks >= 1 && !mbar_wait(&bar[(ks - 1) % NS], (uint32_t)(((ks - 1) / NS) & 1))) {
      ok = false;
      break;
    }
    fill(ks + NS - 1);
  }
  if (ok && nk > 0) ok = mbar_wait(&bar[(nk - 1) % NS], (uint32_t)(((nk - 1) / NS) & 1));
  if (BF16) cp_wait<0>();  // no copy still in flight when the epilogue reuses the stages
  if (!ok && t == 0) atomicExch(L.status, 2);
  tc::fence_after_sync();
  // epilogue: TMEM lane t holds row m0 + t.  Each warp stages its 32 rows x
  // 16 columns in shared memory (the operand stages are free: the last MMA
  // has completed) and applies the epilogue with half a warp per row, so
  // that every global access of a warp covers two 64-byte row segments; the
  // chunk's epilogue inputs are loaded before any of them is used
  const int w = t >> 5, lane = t & 31;
  float* stg = reinterpret_cast<float*>(smem) + w * 32 * 17;
  if (ok) {
    const int cc = lane & 15;
    for (int c = 0; c < Np; c += 16) {
      float v[16];
      if (nk > 0) tc::tmem_ld16(tmem + ((uint32_t)(w * 32) << 16) + (uint32_t)c, v);
      else
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) stg[lane * 17 + i] = v[i];
      __syncwarp();
      const int n = n_lo + c + cc;
      const bool ncol = n < P.N;
      float a[16], in[16];
      bool ok_r[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int r = 2 * j + (lane >> 4);
        const int m = m0 + w * 32 + r;
        ok_r[j] = m < P.M;
        a[j] = stg[r * 17 + cc];
        in[j] = 0.f;
        if (ok_r[j] && ncol) {
          if (EPI == EPI_MASK)
            in[j] = BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(P.mask)[(long long)m * P.ld_mask + n])
                         : static_cast<const float*>(P.mask)[(long long)m * P.ld_mask + n];
          else if (EPI == EPI_DX) in[j] = (float)P.spins[(long long)m * P.ld_spins + n];
        }
      }
      const float bn = (ncol && (EPI == EPI_BIAS_RELU || EPI == EPI_DX)) ? P.bias[n] : 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int m = m0 + w * 32 + 2 * j + (lane >> 4);
        if (!ok_r[j]) continue;
        if (n == P.ones_col) {
          if (P.bias_out) P.bias_out[(long long)blockIdx.z * P.split_stride + m] = a[j];
          continue;
        }
        if (!ncol) continue;
        const long long o = (long long)m * P.ldc + n;
        float r = 0.f;
        switch (EPI) {
          case EPI_STORE:
            static_cast<float*>(P.C)[(long long)blockIdx.z * P.split_stride + o] = a[j];
            break;
          case EPI_BIAS_RELU:
            r = fmaxf(a[j] + bn, 0.f);
            break;
          case EPI_DX: {
            const float x = a[j] + bn, sp = in[j];
            r = P.row_w[m] * sp / (1.f + expf(sp * x));
            break;
          }
          case EPI_MASK:
            r = in[j] > 0.f ? a[j] : 0.f;
            break;
        }
        if (EPI != EPI_STORE) {  // the next product's operand
          if (BF16) static_cast<__nv_bfloat16*>(P.C)[o] = __float2bfloat16(r);
          else static_cast<float*>(P.C)[o] = r;
        }
      }
      __syncwarp();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, GN);
}

int gemm_smem_bytes(bool bf16) {
  return bf16 ? GNS_BF16 * (GSTAGE_BF16 + GSTAGE_B_BF16) + 8 * GNS_BF16 + 16 : 2 * (GM * GK * 4 + GN * GK * 4) + 32;
}

cudaError_t launch_gemm(const GemmLaunch& L, int n_prob, int max_m, int splits, bool bf16,
                        cudaStream_t s) {
  if (n_prob == 0 || max_m == 0) return cudaSuccess;
  const int smem = gemm_smem_bytes(bf16);
  // column blocks of GN: the widest padded N of the launch's problems
  int max_np = 16;
  for (int i = 0; i < n_prob; ++i) {
    const GemmProblem& P = L.prob[i];
    max_np = std::max(max_np, (P.N + (P.ones_col >= 0 ? 1 : 0) + 15) & ~15);
  }
  GemmLaunch Lm = L;
  Lm.ncb = (max_np + GN - 1) / GN;
  dim3 grid(((max_m + GM - 1) / GM) * Lm.ncb, n_prob, splits);
  const int epi = L.prob[0].epi;
  for (int i = 1; i < n_prob; ++i)
    if (L.prob[i].epi != epi) return cudaErrorInvalidValue;  // one epilogue per launch
  void (*kern)(const GemmLaunch) = nullptr;
#define TNVAN_GEMM_KERN(B, E) \
  if (bf16 == B && epi == E) kern = gemm_tc_kernel<B, E>;
  TNVAN_GEMM_KERN(true, EPI_STORE)
  TNVAN_GEMM_KERN(true, EPI_BIAS_RELU)
  TNVAN_GEMM_KERN(true, EPI_DX)
  TNVAN_GEMM_KERN(true, EPI_MASK)
  TNVAN_GEMM_KERN(false, EPI_STORE)
  TNVAN_GEMM_KERN(false, EPI_BIAS_RELU)
  TNVAN_GEMM_KERN(false, EPI_DX)
  TNVAN_GEMM_KERN(false, EPI_MASK)
#undef TNVAN_GEMM_KERN
  if (!kern) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 128, smem, s>>>(Lm);
  return cudaGetLastError();
}

}  // namespace tnvan
