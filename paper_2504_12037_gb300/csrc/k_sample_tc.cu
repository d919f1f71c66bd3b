// BF16 ancestral sampler on tcgen05 (Eq. 6-8) for networks with two hidden
// layers of at most 128 units and at most 128 inputs.
//
// One CTA (128 threads, thread = sample = TMEM lane) draws 128 samples.
// TMEM holds, for every unit not yet evaluated, its pre-activation from all
// inputs fixed so far: P1 [128 x H1], P2 [128 x H2], PO [128 x D].  The steps
// are processed in the host's step groups; inside a group, each step adds the
// few in-group contributions on the CUDA cores (FP32 triangle tiles of the
// group, bulk-copied into shared memory), evaluates the units that complete at
// that step and draws s_i = +1 iff u < sigmoid(x_i).  After the group, its
// new spins and hidden values (BF16 tiles, zero outside the group) are folded
// into every accumulator at once:
//   P1 += S_g W1_g^T,   P2 += H1_g W2_g^T,   PO += H2_g Wo_g^T
// -- three short tcgen05.mma chains whose K windows are the group's spins and
// units rounded out to multiples of 16, against BF16 weight tiles that were
// laid out once per call in the canonical K-major form and bulk-copied in.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tnvan {

namespace {

__device__ __forceinline__ uint32_t koff(int r, int c, uint32_t rowbytes) {
  return (uint32_t)(r >> 3) * (rowbytes / 16u) * 128u + (uint32_t)(c >> 3) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(c & 7) * 2u;
}
__device__ __forceinline__ void stb(unsigned char* base, uint32_t o, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + o) = __float2bfloat16(v);
}

}  // namespace

#define STC_WIN 64  // widest K window of a fold (units)
#define STC_UG 32   // most units of one layer completing inside a group
#define STC_GI 16   // most steps in a group

__host__ __device__ inline int sample_tc_smem(int D, int H1, int H2, int wmax) {
  const int weights = 2 * (H1 * D + H2 * H1 + D * H2);
  const int folds = 2 * 128 * (32 + STC_WIN + STC_WIN);           // S_g, H1_g, H2_g (BF16)
  const int pre = 4 * 128 * (STC_UG + STC_UG + STC_GI);           // P1, P2, PO of the group's units
  const int vals = 4 * 128 * (STC_GI + STC_UG + STC_UG);          // in-group s, h1, h2 (FP32)
  const int tri = 4 * ((wmax + 3) & ~3);                          // triangle tiles of a group
  const int sp = 128 * D;
  const int small = 4 * (STC_UG + STC_UG + STC_GI + 2 * (STC_GI + 1));
  return weights + folds + pre + vals + tri + sp + small + 64;
}

__global__ void __launch_bounds__(128, 1) sample_tc_kernel(const InstDev* __restrict__ inst,
                                                           const LaunchInfo li, int8_t* __restrict__ spins,
                                                           float* __restrict__ logq,
                                                           const int8_t* __restrict__ given) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const int D = md.D, H1 = md.H1, H2 = md.H2;
  const int t = threadIdx.x, w = t >> 5;
  const int b = (blockIdx.x - li.tile_begin[k]) * 128 + t;
  const bool valid = b < li.batch;
  const int wbytes = 2 * (H1 * D + H2 * H1 + D * H2);
  unsigned char* p = smem;
  unsigned char* sW1 = p;
  unsigned char* sW2 = sW1 + 2 * H1 * D;
  unsigned char* sWo = sW2 + 2 * H2 * H1;
  p += (wbytes + 127) & ~127;
  unsigned char* sS = p; p += 2 * 128 * 32;
  unsigned char* sH1 = p; p += 2 * 128 * STC_WIN;
  unsigned char* sH2 = p; p += 2 * 128 * STC_WIN;
  float* P1 = reinterpret_cast<float*>(p); p += 4 * 128 * STC_UG;
  float* P2 = reinterpret_cast<float*>(p); p += 4 * 128 * STC_UG;
  float* PO = reinterpret_cast<float*>(p); p += 4 * 128 * STC_GI;
  float* Sf = reinterpret_cast<float*>(p); p += 4 * 128 * STC_GI;
  float* H1f = reinterpret_cast<float*>(p); p += 4 * 128 * STC_UG;
  float* H2f = reinterpret_cast<float*>(p); p += 4 * 128 * STC_UG;
  float* TW = reinterpret_cast<float*>(p); p += 4 * ((md.wmax + 3) & ~3);
  float* gb1 = reinterpret_cast<float*>(p); p += 4 * STC_UG;   // biases of the group's units
  float* gb2 = reinterpret_cast<float*>(p); p += 4 * STC_UG;
  float* gbo = reinterpret_cast<float*>(p); p += 4 * STC_GI;
  int* gc1 = reinterpret_cast<int*>(p); p += 4 * (STC_GI + 1);  // c1[i], c2[i] for i = i0-1 .. i1-1
  int* gc2 = reinterpret_cast<int*>(p); p += 4 * (STC_GI + 1);
  int8_t* sp = reinterpret_cast<int8_t*>(p); p += 128 * D;
  p = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 7) & ~uintptr_t(7));
  uint64_t* bar = reinterpret_cast<uint64_t*>(p);   // MMA completion
  uint64_t* cbar = bar + 1;                         // bulk copies
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t rbW1 = 2u * D, rbW2 = 2u * H1, rbWo = 2u * H2;
  const float* b1 = md.packed + md.layer[0].dst_off + (long long)H1 * D;
  const float* b2 = md.packed + md.layer[1].dst_off + (long long)H2 * H1;
  const float* bo = md.packed + md.layer[2].dst_off + (long long)D * H2;
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  if (w == 0) {
    tc::tmem_alloc(slot, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  uint32_t cphase = 0;
  if (t == 0) {
    mbar_expect_tx(cbar, (uint32_t)wbytes);
    bulk_g2s(sW1, md.wtiles, (uint32_t)wbytes, cbar);
  }
  bool ok = mbar_wait(cbar, cphase);
  cphase ^= 1u;
  const uint32_t tmem = *slot;
  const uint32_t tP1 = tmem, tP2 = tmem + 128, tPO = tmem + 256;
  const uint32_t lane_off = (uint32_t)(w * 32) << 16;
  const uint32_t id1 = tc::idesc(128, H1, 1u), id2 = tc::idesc(128, H2, 1u), ido = tc::idesc(128, D, 1u);
  const uint2 key = make_uint2((uint32_t)li.seed, (uint32_t)(li.seed >> 32));
  const uint32_t step32 = launch_step(li);
  const int8_t* gv = given ? given + I.spin_units * li.batch + (long long)b * D : nullptr;
  uint32_t phase = 0;
  bool init1 = false, init2 = false, inito = false;  // accumulator written by a fold yet
  float lq = 0.f;
  uint4 rnd = make_uint4(0, 0, 0, 0);
  for (int g = 0; g < md.n_groups && ok; ++g) {
    const int* G = md.groups + GROUP_INTS * g;
    const int i0 = G[0], i1 = G[1], u1lo = G[2], u1hi = G[3], u2lo = G[4], u2hi = G[5];
    const int gi = i1 - i0, n1g = u1hi - u1lo, n2g = u2hi - u2lo;
    const int s0 = i0 & ~15, w1 = u1lo & ~15, w2 = u2lo & ~15;
    const int sN = ((i1 + 15) & ~15) - s0, n1 = ((u1hi + 15) & ~15) - w1, n2 = ((u2hi + 15) & ~15) - w2;
    // previous fold done (its operand tiles are free, the accumulators final)
    if (g > 0) {
      ok = mbar_wait(bar, phase);
      phase ^= 1u;
      tc::fence_after_sync();
      if (!ok) break;
    }
    __syncthreads();  // everyone is done with the previous triangle tiles and group tables
    if (t < n1g) gb1[t] = __ldg(b1 + u1lo + t);
    if (t >= 32 && t - 32 < n2g) gb2[t - 32] = __ldg(b2 + u2lo + t - 32);
    if (t >= 64 && t - 64 < gi) gbo[t - 64] = __ldg(bo + i0 + t - 64);
    if (t >= 96 && t - 96 <= gi) {
      const int i = i0 - 1 + (t - 96);
      gc1[t - 96] = i >= 0 ? md.c1[i] : 0;
      gc2[t - 96] = i >= 0 ? md.c2[i] : 0;
    }
    const int tstart = G[12];
    const uint32_t tbytes = (uint32_t)(G[10] - tstart) * 4u;
    if (t == 0 && tbytes) {
      fence_proxy_async_smem();
      mbar_expect_tx(cbar, tbytes);
      bulk_g2s(TW, md.blocks + G[9] + tstart, tbytes, cbar);
    }
    // accumulated pre-activations of the group's units -> FP32 [unit][T];
    // TMEM loads go in statically indexed pairs, one wait per pair
    auto take = [&](const uint32_t (&r)[16], int c0, int lo, int hi, float* dst) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = c0 + i;
        if (c >= lo && c < hi) dst[(c - lo) * 128 + t] = __uint_as_float(r[i]);
      }
    };
    auto load_window = [&](uint32_t tbase, int wlo, int wn, int lo, int hi, float* dst) {
      for (int c = 0; c < wn; c += 32) {
        uint32_t ra[16], rb[16];
        tc::tmem_ld16_nowait(tbase + lane_off + (uint32_t)(wlo + c), ra);
        const bool two = c + 16 < wn;
        if (two) tc::tmem_ld16_nowait(tbase + lane_off + (uint32_t)(wlo + c + 16), rb);
        tc::tmem_wait_ld();
        take(ra, wlo + c, lo, hi, dst);
        if (two) take(rb, wlo + c + 16, lo, hi, dst);
      }
    };
    if (init1) load_window(tP1, w1, n1, u1lo, u1hi, P1);
    else for (int u = 0; u < n1g; ++u) P1[u * 128 + t] = 0.f;
    if (init2) load_window(tP2, w2, n2, u2lo, u2hi, P2);
    else for (int u = 0; u < n2g; ++u) P2[u * 128 + t] = 0.f;
    if (inito) load_window(tPO, s0, sN, i0, i1, PO);
    else for (int i = 0; i < gi; ++i) PO[i * 128 + t] = 0.f;
    // zero this thread's rows of the fold tiles
    for (int c = 0; c < 32; c += 8) *reinterpret_cast<uint4*>(sS + koff(t, c, 64u)) = make_uint4(0, 0, 0, 0);
    for (int c = 0; c < STC_WIN; c += 8) {
      *reinterpret_cast<uint4*>(sH1 + koff(t, c, 2u * STC_WIN)) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(sH2 + koff(t, c, 2u * STC_WIN)) = make_uint4(0, 0, 0, 0);
    }
    if (tbytes) {
      ok = mbar_wait(cbar, cphase);
      cphase ^= 1u;
      if (!ok) break;
    }
    const float* TW1 = TW;
    const float* TW2 = TW + (G[13] - tstart);
    const float* TWo = TW + (G[14] - tstart);
    __syncthreads();  // group tables visible
    // in-group steps
    for (int i = i0; i < i1; ++i) {
      if ((i & 3) == 0)
        rnd = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(i >> 2), step32, (uint32_t)k), key);
      const int q = i - i0;  // gc*[q] = c*[i-1], gc*[q+1] = c*[i]
      if (i >= 1) {
        const int ua = gc1[q], ub = gc1[q + 1];
        for (int u = ua; u < ub; ++u) {
          const float* wr = TW1 + (u - u1lo) * gi;
          float a0 = P1[(u - u1lo) * 128 + t] + gb1[u - u1lo], a1 = 0.f;
          int j = 0;
          for (; j + 2 <= q; j += 2) {
            a0 = fmaf(wr[j], Sf[j * 128 + t], a0);
            a1 = fmaf(wr[j + 1], Sf[(j + 1) * 128 + t], a1);
          }
          if (j < q) a0 = fmaf(wr[j], Sf[j * 128 + t], a0);
          const float a = fmaxf(a0 + a1, 0.f);
          H1f[(u - u1lo) * 128 + t] = a;
          stb(sH1, koff(t, u - w1, 2u * STC_WIN), a);
        }
        const int n1i = ub - u1lo;
        for (int v = gc2[q]; v < gc2[q + 1]; ++v) {
          const float* wr = TW2 + (v - u2lo) * n1g;
          float a0 = P2[(v - u2lo) * 128 + t] + gb2[v - u2lo], a1 = 0.f, a2 = 0.f, a3 = 0.f;
          int u = 0;
          for (; u + 4 <= n1i; u += 4) {
            a0 = fmaf(wr[u], H1f[u * 128 + t], a0);
            a1 = fmaf(wr[u + 1], H1f[(u + 1) * 128 + t], a1);
            a2 = fmaf(wr[u + 2], H1f[(u + 2) * 128 + t], a2);
            a3 = fmaf(wr[u + 3], H1f[(u + 3) * 128 + t], a3);
          }
          for (; u < n1i; ++u) a0 = fmaf(wr[u], H1f[u * 128 + t], a0);
          const float a = fmaxf((a0 + a1) + (a2 + a3), 0.f);
          H2f[(v - u2lo) * 128 + t] = a;
          stb(sH2, koff(t, v - w2, 2u * STC_WIN), a);
        }
      }
      float x;
      {
        const float* wr = TWo + q * n2g;
        const int n2i = gc2[q + 1] - u2lo;
        float a0 = PO[q * 128 + t] + gbo[q], a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int v = 0;
        for (; v + 4 <= n2i; v += 4) {
          a0 = fmaf(wr[v], H2f[v * 128 + t], a0);
          a1 = fmaf(wr[v + 1], H2f[(v + 1) * 128 + t], a1);
          a2 = fmaf(wr[v + 2], H2f[(v + 2) * 128 + t], a2);
          a3 = fmaf(wr[v + 3], H2f[(v + 3) * 128 + t], a3);
        }
        for (; v < n2i; ++v) a0 = fmaf(wr[v], H2f[v * 128 + t], a0);
        x = (a0 + a1) + (a2 + a3);
      }
      const float pr = 1.f / (1.f + expf(-x));
      const uint32_t word = (i & 3) == 0 ? rnd.x : (i & 3) == 1 ? rnd.y : (i & 3) == 2 ? rnd.z : rnd.w;
      const float u = (float)(word >> 8) * 5.9604644775390625e-08f;
      float s = u < pr ? 1.f : -1.f;
      if (gv) s = valid ? (float)gv[i] : 1.f;
      Sf[q * 128 + t] = s;
      stb(sS, koff(t, i - s0, 64u), s);
      sp[t * D + i] = (int8_t)s;
      lq -= softplusf(-s * x);
    }
    // fold the group into every accumulator
    if (g + 1 < md.n_groups) {
      fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (t == 0) {
        const uint32_t aS = smem_u32(sS), aH1 = smem_u32(sH1), aH2 = smem_u32(sH2);
        for (int kk = 0; kk < sN / 16; ++kk)
          tc::mma_bf16(tP1, tc::smem_desc(aS + kk * 256u, 128u, 4u * 128u),
                       tc::smem_desc(smem_u32(sW1) + (uint32_t)((s0 >> 4) + kk) * 256u, 128u, rbW1 / 16u * 128u), id1,
                       (init1 || kk > 0) ? 1u : 0u);
        for (int kk = 0; kk < n1 / 16; ++kk)
          tc::mma_bf16(tP2, tc::smem_desc(aH1 + kk * 256u, 128u, (2u * STC_WIN) / 16u * 128u),
                       tc::smem_desc(smem_u32(sW2) + (uint32_t)((w1 >> 4) + kk) * 256u, 128u, rbW2 / 16u * 128u), id2,
                       (init2 || kk > 0) ? 1u : 0u);
        for (int kk = 0; kk < n2 / 16; ++kk)
          tc::mma_bf16(tPO, tc::smem_desc(aH2 + kk * 256u, 128u, (2u * STC_WIN) / 16u * 128u),
                       tc::smem_desc(smem_u32(sWo) + (uint32_t)((w2 >> 4) + kk) * 256u, 128u, rbWo / 16u * 128u), ido,
                       (inito || kk > 0) ? 1u : 0u);
        tc::mma_commit(bar);
      }
      init1 = init1 || sN > 0;
      init2 = init2 || n1 > 0;
      inito = inito || n2 > 0;
    }
  }
  if (!ok && t == 0) atomicExch(li.status, 4);
  __syncthreads();
  if (ok && valid) {
    if (spins) {
      int8_t* out = spins + I.spin_units * li.batch + (long long)b * D;
      for (int i = 0; i < D; ++i) out[i] = sp[t * D + i];
    }
    logq[(long long)k * li.batch + b] = lq;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 512);
}

int sample_tc_smem_bytes(int D, int H1, int H2, int wmax) { return sample_tc_smem(D, H1, H2, wmax); }

cudaError_t launch_sample_tc(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int8_t* spins,
                             float* logq, const int8_t* given, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  sample_tc_kernel<<<nblk, 128, smem_bytes, s>>>(d_inst, li, spins, logq, given);
  return cudaGetLastError();
}

}  // namespace tnvan
