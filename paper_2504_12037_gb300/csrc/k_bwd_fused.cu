// Fused BF16 backward of the MADE network on tcgen05 (Eq. 10), for networks
// with two hidden layers of at most 128 units (multiples of 16) and at most
// 128 inputs (padded to Dp, a multiple of 16: the padded inputs and outputs
// are zero and carry no gradient).
//
// One CTA (BWD_WG warpgroups, each thread one sample = TMEM lane and every
// BWD_WG-th 16-column chunk of each epilogue) walks the 128-sample
// tiles of its chunk.  Per tile, everything stays on chip:
//   A1 = relu(S W1^T + b1), A2 = relu(A1 W2^T + b2), X = A2 Wo^T + bo,
//   dX = w_b s sigmoid(-s x), dA2 = (dX Wo) 1[A2 > 0], dA1 = (dA2 W2) 1[A1 > 0],
// each product one chain of tcgen05.mma into a TMEM scratch accumulator whose
// epilogue (tcgen05.ld, one row per thread) writes the next BF16 operand tile
// into shared memory.  The weight gradients
//   GWo += dX^T [A2 | 1],  GW2 += dA2^T [A1 | 1],  GW1 += dA1^T [S | 1]
// reuse the same tiles read transposed (MN-major descriptors) and accumulate
// in TMEM across all tiles of the chunk; the column of ones yields the bias
// gradients.  At the end each CTA writes its partial gradient slice (packed,
// degree-sorted layout) for the deterministic chunk reduction.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tnvan {

namespace {

// Row-major-in-K tile geometry: rows of `kel` bf16 (a multiple of 16).
struct Tile {
  uint32_t base;  // shared address
  int kel;        // elements per row
  __device__ uint32_t rowbytes() const { return (uint32_t)kel * 2u; }
  // K-major operand descriptor for MMA k-step kk (16 elements of K)
  __device__ uint64_t kdesc(int kk) const {
    return tc::smem_desc(base + (uint32_t)kk * 256u, 128u, rowbytes() / 16u * 128u);
  }
  // MN-major view (MN = the row's elements, K = the rows), k-step kk covers rows 16kk..16kk+15
  __device__ uint64_t mndesc(int kk) const {
    const uint32_t kstride = rowbytes() * 8u;  // 8 rows
    return tc::smem_desc(base + (uint32_t)kk * 2u * kstride, kstride, 128u);
  }
};

__device__ __forceinline__ void store8(unsigned char* sm_base, uint32_t rowbytes, int r, int c,
                                       const float* v) {
  // 8 consecutive elements (c multiple of 8) of row r, canonical K-major layout
  const uint32_t o = (uint32_t)(r >> 3) * (rowbytes / 16u) * 128u + (uint32_t)(c >> 3) * 128u + (uint32_t)(r & 7) * 16u;
  __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
  uint4 u;
  u.x = *reinterpret_cast<uint32_t*>(&p0);
  u.y = *reinterpret_cast<uint32_t*>(&p1);
  u.z = *reinterpret_cast<uint32_t*>(&p2);
  u.w = *reinterpret_cast<uint32_t*>(&p3);
  *reinterpret_cast<uint4*>(sm_base + o) = u;
}

// Per-thread bit masks of up to 128 columns (4 words): set / get 16 bits
// at a column c that is a multiple of 16.
struct Mask128 {
  uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
  __device__ __forceinline__ void put16(int c, uint32_t m16) {
    const uint32_t v = m16 << (c & 16);
    const int j = c >> 5;
    w0 |= j == 0 ? v : 0u;
    w1 |= j == 1 ? v : 0u;
    w2 |= j == 2 ? v : 0u;
    w3 |= j == 3 ? v : 0u;
  }
  __device__ __forceinline__ uint32_t get16(int c) const {
    const int j = c >> 5;
    const uint32_t w = j == 0 ? w0 : (j == 1 ? w1 : (j == 2 ? w2 : w3));
    return (w >> (c & 16)) & 0xFFFFu;
  }
};

}  // namespace

// Warpgroups per CTA: thread (g, r) owns TMEM lane / sample row r and the
// 16-column chunks c with (c / 16) % BWD_WG == g of every epilogue.
#define BWD_WG 4

struct FusedBwdArgs {
  const int8_t* spins;
  const double* logZR;
  const float* logq;
  const double* stats;
  float* partials;
  long long part_stride;
  int* status;
};

// Bytes of the buffer dX and then dA2 share (D padded): dA2 is written once
// the products reading dX are done.  The MN-major view of dX (M = 128 of its
// D columns) reads up to 2 KB past the dX tile when D < 128; the buffer
// covers that.
__host__ __device__ inline int fused_bwd_xbuf(int D, int H2) {
  const int a = 256 * D + 2048, b = 256 * H2;
  return a > b ? a : b;
}

// Shared memory bytes for (D, H1, H2).
__host__ __device__ inline int fused_bwd_smem(int D0, int H1, int H2) {
  const int D = (D0 + 15) & ~15;
  const int w = H1 * D + H2 * H1 + D * H2;              // weights
  const int a = 128 * ((D + 16) + (H1 + 16) + (H2 + 16));  // S, A1, A2/dA1
  return 2 * (w + a) + fused_bwd_xbuf(D, H2) + 4 * (H1 + H2 + D) + 64;  // + dX/dA2, biases, barriers, TMEM slot
}

__global__ void __launch_bounds__(128 * BWD_WG, 1) bwd_fused_kernel(const InstDev* __restrict__ inst,
                                                           const LaunchInfo li, FusedBwdArgs args) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int gblk = blockIdx.x + li.blk0;  // a launch may cover a sub-range of the blocks
  const int k = find_inst(li, gblk);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  if (!md.fused_ok) return;
  const int D = md.D, Dp = (D + 15) & ~15, H1 = md.H1, H2 = md.H2;
  const int tid = threadIdx.x, w = tid >> 5, t = tid & 127, g = tid >> 7;
  const int B = li.batch;
  const int tiles_total = (B + 127) / 128;
  const int c_idx = gblk - li.tile_begin[k];
  // tiles per CTA: this instance's tiles over its CTAs (instances may differ)
  const int nblk_k = li.tile_begin[k + 1] - li.tile_begin[k];
  const int per = (tiles_total + nblk_k - 1) / nblk_k;
  const int tile0 = c_idx * per, tile1 = min(tiles_total, tile0 + per);
  // ---- shared memory carve ----
  unsigned char* p = smem;
  unsigned char* sW1 = p; p += H1 * Dp * 2;
  unsigned char* sW2 = p; p += H2 * H1 * 2;
  unsigned char* sWo = p; p += Dp * H2 * 2;
  unsigned char* sS = p; p += 128 * (Dp + 16) * 2;
  unsigned char* sA1 = p; p += 128 * (H1 + 16) * 2;
  unsigned char* sA2 = p; p += 128 * (H2 + 16) * 2;  // later dA1 (128 x H1)
  unsigned char* sdX = p;                             // dX, then dA2 in the same buffer
  unsigned char* sdA2 = p; p += fused_bwd_xbuf(Dp, H2);
  float* sb1 = reinterpret_cast<float*>(p); p += 4 * H1;  // biases
  float* sb2 = reinterpret_cast<float*>(p); p += 4 * H2;
  float* sbo = reinterpret_cast<float*>(p); p += 4 * Dp;  // padded: the barriers below stay 8-byte aligned
  uint64_t* bar = reinterpret_cast<uint64_t*>(p);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);  // cbar is bar + 2
  const Tile tW1{smem_u32(sW1), Dp}, tW2{smem_u32(sW2), H1}, tWo{smem_u32(sWo), H2};
  const Tile tS{smem_u32(sS), Dp + 16}, tA1{smem_u32(sA1), H1 + 16}, tA2{smem_u32(sA2), H2 + 16};
  const Tile tdX{smem_u32(sdX), Dp}, tdA2{smem_u32(sdA2), H2}, tdA1{smem_u32(sA2), H1};
  // ---- weights: packed FP32 (masked, degree-sorted) -> BF16 K-major tiles ----
  const float* W1 = md.packed + md.layer[0].dst_off;
  const float* b1 = W1 + (long long)H1 * D;
  const float* W2 = md.packed + md.layer[1].dst_off;
  const float* b2 = W2 + (long long)H2 * H1;
  const float* Wo = md.packed + md.layer[2].dst_off;
  const float* bo = Wo + (long long)D * H2;  // the packed layer is [D][H2] then b [D]
  // BF16 weight tiles (laid out once per call in the canonical K-major form)
  // arrive with one bulk copy; W1, W2, Wo are contiguous in both places
  uint64_t* cbar = bar + 2;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  if (w == 0) {
    tc::tmem_alloc(slot, 512);
    tc::tmem_relinquish();
  }
  for (int u = tid; u < H1; u += blockDim.x) sb1[u] = __ldg(b1 + u);
  for (int u = tid; u < H2; u += blockDim.x) sb2[u] = __ldg(b2 + u);
  for (int u = tid; u < D; u += blockDim.x) sbo[u] = __ldg(bo + u);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 0) {
    const uint32_t wbytes = 2u * (uint32_t)(H1 * Dp + H2 * H1 + Dp * H2);
    mbar_expect_tx(cbar, wbytes);
    bulk_g2s(sW1, md.wtiles, wbytes, cbar);
  }
  const bool weights_ok = mbar_wait(cbar, 0);
  const uint32_t tmem = *slot;
  // the ones column of [S | 1] (layer-1 bias gradient): inside the padding at
  // column D when D is not a multiple of 16 (W1's padded columns are zero, so
  // the forward product ignores it), else a 16-column block of its own at Dp
  const int oc1 = (D & 15) ? D : Dp, g1n = (D & 15) ? Dp : Dp + 16;
  const uint32_t tScr = tmem, tG1 = tmem + 128, tG2 = tG1 + (uint32_t)g1n, tGo = tG2 + (uint32_t)(H1 + 16);
  const uint32_t lane_off = (uint32_t)((w & 3) * 32) << 16;
  const uint32_t id_fwd1 = tc::idesc(128, H1, 1u), id_fwd2 = tc::idesc(128, H2, 1u), id_fwd3 = tc::idesc(128, Dp, 1u);
  const uint32_t id_d2 = tc::idesc(128, H2, 1u) | (1u << 16);         // B MN-major
  const uint32_t id_d1 = tc::idesc(128, H1, 1u) | (1u << 16);
  const uint32_t id_go = tc::idesc(128, H2 + 16, 1u) | (1u << 15) | (1u << 16);  // A, B MN-major
  const uint32_t id_g2 = tc::idesc(128, H1 + 16, 1u) | (1u << 15) | (1u << 16);
  const uint32_t id_g1 = tc::idesc(128, g1n, 1u) | (1u << 15) | (1u << 16);
  const double mean = args.stats[8 * k + 4];
  const double wsc = -1.0 / (li.beta[k] * stats_batch(args.stats + 8 * k));
  const int8_t* Sg = args.spins + I.spin_units * (long long)B;
  uint32_t phase = 0;
  bool ok = weights_ok;
  auto mma_wait = [&]() -> bool {
    if (tid == 0) tc::mma_commit(bar);
    const bool r = mbar_wait(bar, phase);
    phase ^= 1u;
    tc::fence_after_sync();
    return r;
  };
  auto sync_for_mma = [&]() {
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  bool first = true;
  for (int tile = tile0; tile < tile1 && ok; ++tile) {
    const int b = tile * 128 + t;
    const bool valid = b < B;
    const float vf = valid ? 1.f : 0.f;
    // spins -> S tile (+ ones column), 16 per vector load; mS bit f = (s_f > 0)
    Mask128 mS, m1, m2;
    for (int c = 16 * g; c < Dp; c += 16 * BWD_WG) {
      float sp[16];
      uint32_t m16 = 0;
      if ((D & 15) == 0 && (reinterpret_cast<uintptr_t>(Sg) & 15) == 0) {  // 16 spins per vector load
        uint4 raw = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
        if (valid) raw = *reinterpret_cast<const uint4*>(Sg + (long long)b * D + c);
        const uint32_t wv[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int8_t sv = (int8_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu);
          sp[i] = valid ? (float)sv : 0.f;
          m16 |= (sv > 0 ? 1u : 0u) << i;
        }
      } else {  // rows not 16-byte aligned: byte loads; padded spins are 0
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int f = c + i;
          const int8_t sv = (valid && f < D) ? Sg[(long long)b * D + f] : (int8_t)0;
          sp[i] = f == oc1 ? vf : (float)sv;  // oc1 < Dp only when D is not a multiple of 16
          m16 |= (sv > 0 ? 1u : 0u) << i;
        }
      }
      mS.put16(c, m16);
      store8(sS, tS.rowbytes(), t, c, sp);
      store8(sS, tS.rowbytes(), t, c + 8, sp + 8);
    }
    if (oc1 == Dp && ((Dp >> 4) % BWD_WG) == g) {
      float sp[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) sp[i] = i == 0 ? vf : 0.f;
      store8(sS, tS.rowbytes(), t, Dp, sp);
      store8(sS, tS.rowbytes(), t, Dp + 8, sp + 8);
    }
    const float wb = valid ? (float)(wsc * (args.logZR[(long long)k * B + b] - (double)args.logq[(long long)k * B + b] - mean)) : 0.f;
    sync_for_mma();
    // fwd1: scratch = S W1^T
    if (tid == 0)
      for (int kk = 0; kk < Dp / 16; ++kk) tc::mma_bf16(tScr, tS.kdesc(kk), tW1.kdesc(kk), id_fwd1, kk > 0);
    if (!(ok = mma_wait())) break;
    for (int c = 16 * g; c < H1 + 16; c += 16 * BWD_WG) {
      float v[16];
      if (c < H1) tc::tmem_ld16(tScr + lane_off + (uint32_t)c, v);
      uint32_t m16 = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int u = c + i;
        v[i] = u < H1 ? fmaxf(v[i] + sb1[u], 0.f) * vf : (u == H1 ? vf : 0.f);
        m16 |= (u < H1 && v[i] > 0.f ? 1u : 0u) << i;
      }
      if (c < H1) m1.put16(c, m16);
      store8(sA1, tA1.rowbytes(), t, c, v);
      store8(sA1, tA1.rowbytes(), t, c + 8, v + 8);
    }
    sync_for_mma();
    // fwd2: scratch = A1 W2^T
    if (tid == 0)
      for (int kk = 0; kk < H1 / 16; ++kk) tc::mma_bf16(tScr, tA1.kdesc(kk), tW2.kdesc(kk), id_fwd2, kk > 0);
    if (!(ok = mma_wait())) break;
    for (int c = 16 * g; c < H2 + 16; c += 16 * BWD_WG) {
      float v[16];
      if (c < H2) tc::tmem_ld16(tScr + lane_off + (uint32_t)c, v);
      uint32_t m16 = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int u = c + i;
        v[i] = u < H2 ? fmaxf(v[i] + sb2[u], 0.f) * vf : (u == H2 ? vf : 0.f);
        m16 |= (u < H2 && v[i] > 0.f ? 1u : 0u) << i;
      }
      if (c < H2) m2.put16(c, m16);
      store8(sA2, tA2.rowbytes(), t, c, v);
      store8(sA2, tA2.rowbytes(), t, c + 8, v + 8);
    }
    sync_for_mma();
    // fwd3: scratch = A2 Wo^T ; epilogue dX
    if (tid == 0)
      for (int kk = 0; kk < H2 / 16; ++kk) tc::mma_bf16(tScr, tA2.kdesc(kk), tWo.kdesc(kk), id_fwd3, kk > 0);
    if (!(ok = mma_wait())) break;
    for (int c = 16 * g; c < Dp; c += 16 * BWD_WG) {
      float v[16];
      tc::tmem_ld16(tScr + lane_off + (uint32_t)c, v);
      const uint32_t ms = mS.get16(c);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int f = c + i;
        const float x = v[i] + (f < D ? sbo[f] : 0.f);
        const float s = ((ms >> i) & 1u) ? 1.f : -1.f;
        v[i] = f < D ? wb * s * __frcp_rn(1.f + __expf(s * x)) : 0.f;  // padded outputs carry no gradient
      }
      store8(sdX, tdX.rowbytes(), t, c, v);
      store8(sdX, tdX.rowbytes(), t, c + 8, v + 8);
    }
    sync_for_mma();
    // scratch = dX Wo (B = Wo read MN-major);  GWo += dX^T [A2 | 1]
    if (tid == 0) {
      for (int kk = 0; kk < Dp / 16; ++kk) tc::mma_bf16(tScr, tdX.kdesc(kk), tWo.mndesc(kk), id_d2, kk > 0);
      for (int kk = 0; kk < 8; ++kk)
        tc::mma_bf16(tGo, tdX.mndesc(kk), tA2.mndesc(kk), id_go, (!first || kk > 0) ? 1u : 0u);
    }
    if (!(ok = mma_wait())) break;
    for (int c = 16 * g; c < H2; c += 16 * BWD_WG) {
      float v[16];
      tc::tmem_ld16(tScr + lane_off + (uint32_t)c, v);
      const uint32_t mk = m2.get16(c);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = ((mk >> i) & 1u) ? v[i] : 0.f;
      store8(sdA2, tdA2.rowbytes(), t, c, v);
      store8(sdA2, tdA2.rowbytes(), t, c + 8, v + 8);
    }
    sync_for_mma();
    // scratch = dA2 W2 (B = W2 read MN-major);  GW2 += dA2^T [A1 | 1]
    if (tid == 0) {
      for (int kk = 0; kk < H2 / 16; ++kk) tc::mma_bf16(tScr, tdA2.kdesc(kk), tW2.mndesc(kk), id_d1, kk > 0);
      for (int kk = 0; kk < 8; ++kk)
        tc::mma_bf16(tG2, tdA2.mndesc(kk), tA1.mndesc(kk), id_g2, (!first || kk > 0) ? 1u : 0u);
    }
    if (!(ok = mma_wait())) break;
    for (int c = 16 * g; c < H1; c += 16 * BWD_WG) {
      float v[16];
      tc::tmem_ld16(tScr + lane_off + (uint32_t)c, v);
      const uint32_t mk = m1.get16(c);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = ((mk >> i) & 1u) ? v[i] : 0.f;
      // dA1 overwrites A2 (GWo and the dA2 mask have consumed it)
      store8(sA2, tdA1.rowbytes(), t, c, v);
      store8(sA2, tdA1.rowbytes(), t, c + 8, v + 8);
    }
    sync_for_mma();
    // GW1 += dA1^T [S | 1]
    if (tid == 0)
      for (int kk = 0; kk < 8; ++kk)
        tc::mma_bf16(tG1, tdA1.mndesc(kk), tS.mndesc(kk), id_g1, (!first || kk > 0) ? 1u : 0u);
    if (!(ok = mma_wait())) break;
    first = false;
    tc::fence_before_sync();
    __syncthreads();
  }
  if (!ok && tid == 0) atomicExch(args.status, 3);
  // ---- flush the gradient partials of this CTA ----
  // Each layer's accumulator (TMEM lane = packed output unit, column =
  // packed input, the last column the bias) goes out in the packed layout:
  // every thread writes its 16 columns of a row as four 16-byte stores (the
  // row-major layer blocks need no transpose), the bias column as one float.
  float* G = args.partials + (long long)gblk * args.part_stride;
  if (ok && !first) {
    // ncol: the accumulator's input columns (a multiple of 16; the bias
    // column follows), nin <= ncol of them real
    // accumulator columns [0, ncols): the nin weight-gradient columns, and
    // the bias gradient at column bcol
    auto flush = [&](uint32_t tacc, int nin, int ncols, int bcol, int nout, long long off) {
      for (int c = 16 * g; c < ncols; c += 16 * BWD_WG) {
        float v[16];
        tc::tmem_ld16(tacc + lane_off + (uint32_t)c, v);
        if (t < nout) {
          if (c < nin) {
            float* row = G + off + (long long)t * nin + c;
            if ((nin & 3) == 0 && c + 16 <= nin) {
              float4* row4 = reinterpret_cast<float4*>(row);
#pragma unroll
              for (int q = 0; q < 4; ++q) row4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (c + q < nin) row[q] = v[q];
            }
          }
          if (bcol >= c && bcol < c + 16) {
            float bv = v[0];
#pragma unroll
            for (int q = 1; q < 16; ++q) bv = q == bcol - c ? v[q] : bv;
            G[off + (long long)nout * nin + t] = bv;
          }
        }
      }
    };
    flush(tG1, D, g1n, oc1, H1, md.layer[0].dst_off);
    flush(tG2, H1, H1 + 16, H1, H2, md.layer[1].dst_off);
    flush(tGo, H2, H2 + 16, H2, D, md.layer[2].dst_off);
  } else {
    for (long long e = tid; e < md.n_params; e += blockDim.x) G[e] = 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 512);
}

cudaError_t launch_bwd_fused(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                             const int8_t* spins, const double* logZR, const float* logq,
                             const double* stats, float* partials, long long part_stride, int* status,
                             cudaStream_t s, int blk_begin, int blk_end) {
  if (blk_end < 0) blk_end = li.tile_begin[li.n_inst];
  const int nblk = blk_end - blk_begin;
  if (nblk <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(bwd_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  LaunchInfo lc = li;
  lc.blk0 = blk_begin;
  FusedBwdArgs a{spins, logZR, logq, stats, partials, part_stride, status};
  bwd_fused_kernel<<<nblk, 128 * BWD_WG, smem_bytes, s>>>(d_inst, lc, a);
  return cudaGetLastError();
}

int fused_bwd_smem_bytes(int D, int H1, int H2) { return fused_bwd_smem(D, H1, H2); }

}  // namespace tnvan
