// MADE network kernels: parameter packing and ancestral sampling (Eq. 6-8).
#include <algorithm>

#include "common.cuh"

namespace tnvan {

// Value of the packed network at flat index j: each layer's [nout][nin]
// block with the MADE masks applied and hidden units sorted by degree, then
// its biases in the same order (layer offsets dst_off), read from the
// caller's natural layout.
__device__ __forceinline__ float packed_value(const MadeDev& md, long long jj) {
  int j = (int)jj;  // a network's parameter count fits in 32 bits (checked at set-up)
  for (int l = 0; l < md.n_layers; ++l) {
    const LayerDev& L = md.layer[l];
    const int nw = L.nout * L.nin;
    if (j < nw) {
      const int o = j / L.nin, i = j - o * L.nin;
      const int no = L.perm_out ? L.perm_out[o] : o;
      const int ni = L.perm_in ? L.perm_in[i] : i;
      const int dout = L.deg_out[o], din = L.deg_in[i];
      const bool conn = L.strict ? (dout > din) : (dout >= din);
      return conn ? md.raw[L.src_off + (long long)no * L.nin + ni] : 0.f;
    }
    j -= nw;
    if (j < L.nout) return md.raw[L.src_off + nw + (L.perm_out ? L.perm_out[j] : j)];
    j -= L.nout;
  }
  return 0.f;
}

// Weights the tiles hold (the padding excluded).
__host__ __device__ inline long long tile_elems(const MadeDev& md) {
  return md.wtiles ? (long long)md.H1 * md.D + (long long)md.H2 * md.H1 + (long long)md.D * md.H2 : 0;
}

// The tensor-core sampler plan a mask selects (bits 8 and up hold plan + 1;
// 0 = every plan).
__host__ __device__ inline int pack_tc_plan(int mask) { return (mask >> 8) - 1; }

// BF16 copy of packed weight (r, c) of layer l (l < 3) into the tensor cores'
// canonical K-major tiles: W1 [H1 x Dp], W2 [H2 x H1], Wo [Dp x H2], no
// swizzle, Dp = D rounded up to 16 (the padding stays zero).
__device__ __forceinline__ void store_tile(const MadeDev& md, int l, int r, int c, float v) {
  const int Dp = (md.D + 15) & ~15, H1 = md.H1, H2 = md.H2;
  const long long n1 = (long long)H1 * Dp, n2 = (long long)H2 * H1;
  const int cols = l == 0 ? Dp : (l == 1 ? H1 : H2);
  const long long base = l == 0 ? 0 : (l == 1 ? n1 : n1 + n2);
  const long long o = base + (long long)(r >> 3) * (cols / 8) * 64 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7);
  uint32_t u = __float_as_uint(v);
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
  md.wtiles[o] = (uint16_t)(u >> 16);
}

// Everything the kernels read from the network, rebuilt from the caller's
// parameters in one launch (grid = (ceil(max_total / 256), n_inst)); the
// segments selected by `mask`, back to back in a flat index:
//   PACK_FLAT  the packed copy (FP32, natural order of packed_value); with
//              PACK_TILES too, the same thread writes each weight's BF16 tile
//              entry, so the tiles need no segment of their own
//   PACK_TILES BF16 tiles in the tensor cores' canonical K-major layout (no
//              swizzle): W1 [H1 x D], W2 [H2 x H1], Wo [D x H2]
//   PACK_SIMT  the blocked SIMT sampler's weight blocks
//   PACK_TCG   the grouped tensor-core sampler plans' triangle tiles (one
//              plan, or all, per pack_tc_plan)
//   PACK_TC    the per-step tensor-core sampler plans' BF16 chunk weight
//              blobs and FP32 in-step weight tables (likewise)
__device__ __forceinline__ void pack_one(const MadeDev& md, int mask, long long e) {
  const bool tiles = (mask & PACK_TILES) && md.wtiles && md.n_layers == 3;
  if (mask & PACK_FLAT) {
    if (e < md.n_params) {
      const float v = packed_value(md, e);
      md.packed[e] = v;
      if (md.packed16) {
        uint32_t u = __float_as_uint(v);
        u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
        md.packed16[e] = (uint16_t)(u >> 16);
      }
      if (tiles) {  // weights of layer l at [dst_off, dst_off + nout * nin), row-major
        int j = (int)e;
        for (int l = 0; l < 3; ++l) {
          const LayerDev& L = md.layer[l];
          const int nw = L.nout * L.nin;
          if (j < nw) {
            const int r = j / L.nin;
            store_tile(md, l, r, j - r * L.nin, v);
            break;
          }
          j -= nw + L.nout;
          if (j < 0) break;  // a bias
        }
      }
      return;
    }
    e -= md.n_params;
  }
  if (tiles && !(mask & PACK_FLAT)) {
    const long long nt = tile_elems(md);
    if (e < nt) {
      const int D = md.D, H1 = md.H1, H2 = md.H2;
      const long long n1 = (long long)H1 * D, n2 = (long long)H2 * H1;
      int l, cols;
      long long base;
      if (e < n1) {
        l = 0, cols = D, base = 0;
      } else if (e < n1 + n2) {
        l = 1, cols = H1, base = n1;
      } else {
        l = 2, cols = H2, base = n1 + n2;
      }
      const int le = (int)(e - base);
      const int r = le / cols, c = le - r * cols;
      store_tile(md, l, r, c, packed_value(md, md.layer[l].dst_off + le));
      return;
    }
    e -= nt;
  }
  if (mask & PACK_SIMT) {
    if (e < md.n_blk) {
      const int j = md.blk_src[e];
      md.blocks[e] = j >= 0 ? packed_value(md, j) : 0.f;
      return;
    }
    e -= md.n_blk;
  }
  if (mask & PACK_TCG) {
    const int only = pack_tc_plan(mask);
    for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
      if (only >= 0 && p != only) continue;
      const MadeDev::TcGroupPlan& P = md.tcg[p];
      if (e < P.n_blk) {
        const int j = P.src[e];
        P.blocks[e] = j >= 0 ? packed_value(md, j) : 0.f;
        return;
      }
      e -= P.n_blk;
      if (e < P.n_wblob) {  // streamed group blobs' live elements (BF16, round to nearest even)
        uint32_t u = __float_as_uint(packed_value(md, P.wsrc[e]));
        u += 0x7fffu + ((u >> 16) & 1u);
        P.wblob[P.wdst[e]] = (uint16_t)(u >> 16);
        return;
      }
      e -= P.n_wblob;
    }
  }
  if (mask & PACK_TC) {
    const int only = pack_tc_plan(mask);
    for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
      if (only >= 0 && p != only) continue;
      const MadeDev::TcPlan& P = md.tc[p];
      if (e < P.n_wblob) {  // the chunk blobs' live elements
        uint32_t u = __float_as_uint(packed_value(md, P.wsrc[e]));
        u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
        P.wblob[P.wdst[e]] = (uint16_t)(u >> 16);
        return;
      }
      e -= P.n_wblob;
      if (e < P.n_steptab) {
        P.steptab[e] = packed_value(md, P.stepsrc[e]);
        return;
      }
      e -= P.n_steptab;
    }
  }
}

// CTAs [cta_begin[j], cta_begin[j + 1]) pack instance k0 + j, striding over
// its elements; the host shares the CTAs out in proportion to the instances'
// element counts, so a launch of mixed sizes ends with its largest instance.
struct PackGrid {
  int n, k0;
  int cta_begin[TNVAN_MAX_INST + 1];
};

__global__ void pack_all_kernel(const InstDev* __restrict__ inst, int mask, const PackGrid pg) {
  int j = 0;
  while (j + 1 < pg.n && pg.cta_begin[j + 1] <= (int)blockIdx.x) ++j;
  const MadeDev& md = inst[pg.k0 + j].made;
  const long long n = pack_elems(md, mask);
  const int c0 = pg.cta_begin[j], nc = pg.cta_begin[j + 1] - c0;
  for (long long e = (long long)(blockIdx.x - c0) * blockDim.x + threadIdx.x; e < n; e += (long long)nc * blockDim.x)
    pack_one(md, mask, e);
}

__host__ __device__ long long pack_elems(const MadeDev& md, int mask) {
  long long n = 0;
  const bool tiles = (mask & PACK_TILES) && md.wtiles && md.n_layers == 3;
  if (mask & PACK_FLAT) n += md.n_params;
  if (tiles && !(mask & PACK_FLAT)) n += tile_elems(md);
  if (mask & PACK_SIMT) n += md.n_blk;
  if (mask & PACK_TCG) {
    const int only = pack_tc_plan(mask);
    for (int p = 0; p < TNVAN_TC_PLANS; ++p)
      if (only < 0 || p == only) n += md.tcg[p].n_blk + md.tcg[p].n_wblob;
  }
  if (mask & PACK_TC) {
    const int only = pack_tc_plan(mask);
    for (int p = 0; p < TNVAN_TC_PLANS; ++p)
      if (only < 0 || p == only) n += md.tc[p].n_wblob + md.tc[p].n_steptab;
  }
  return n;
}

cudaError_t launch_pack_all(const InstDev* d_inst, int n_inst, const long long* counts, int mask, cudaStream_t s) {
  for (int k0 = 0; k0 < n_inst; k0 += TNVAN_MAX_INST) {
    const int n = std::min(TNVAN_MAX_INST, n_inst - k0);
    long long tot = 0;
    for (int j = 0; j < n; ++j) tot += counts[k0 + j];
    if (tot == 0) continue;
    // about sixteen CTAs per SM in all (152 SMs), at least one per instance,
    // none without 256 elements of its own
    const long long budget = 2432;
    PackGrid pg;
    pg.n = n;
    pg.k0 = k0;
    int acc = 0;
    for (int j = 0; j < n; ++j) {
      pg.cta_begin[j] = acc;
      const long long c = counts[k0 + j];
      const long long share = std::max(1LL, std::min((c + 255) / 256, (budget * c + tot - 1) / tot));
      acc += (int)share;
    }
    pg.cta_begin[n] = acc;
    pack_all_kernel<<<(unsigned)acc, 256, 0, s>>>(d_inst, mask, pg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Dot product of a warp-uniform weight row with this thread's activation
// column (layout [unit][T]) over entries [j0, j1).
__device__ __forceinline__ float dot_col(const float* __restrict__ w, const float* col, int T,
                                         int j0, int j1) {
  float a0 = 0.f, a1 = 0.f;
  int j = j0;
  for (; j + 2 <= j1; j += 2) {
    a0 = fmaf(__ldg(w + j), col[j * T], a0);
    a1 = fmaf(__ldg(w + j + 1), col[(j + 1) * T], a1);
  }
  if (j < j1) a0 = fmaf(__ldg(w + j), col[j * T], a0);
  return a0 + a1;
}

// Pre-activations of up to 16 units from n_in inputs: acc[q] = bias[q] +
// sum_j blk[j][q] * act[j], one activation load per 16 FMAs, weights as
// warp-uniform float4 loads.  Results go to pre[q][T] (q < nu).
__device__ __forceinline__ void block_preact(const float* blk, const float* act, int T,
                                             int n_in, const float* __restrict__ bias, int nu,
                                             float* pre) {
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = q < nu ? __ldg(bias + q) : 0.f;
  const float4* w4 = reinterpret_cast<const float4*>(blk);
#pragma unroll 2
  for (int j = 0; j < n_in; ++j) {
    const float x = act[j * T];
    const float4 a = w4[4 * j], b = w4[4 * j + 1], c = w4[4 * j + 2], d = w4[4 * j + 3];
    acc[0] = fmaf(a.x, x, acc[0]);
    acc[1] = fmaf(a.y, x, acc[1]);
    acc[2] = fmaf(a.z, x, acc[2]);
    acc[3] = fmaf(a.w, x, acc[3]);
    acc[4] = fmaf(b.x, x, acc[4]);
    acc[5] = fmaf(b.y, x, acc[5]);
    acc[6] = fmaf(b.z, x, acc[6]);
    acc[7] = fmaf(b.w, x, acc[7]);
    acc[8] = fmaf(c.x, x, acc[8]);
    acc[9] = fmaf(c.y, x, acc[9]);
    acc[10] = fmaf(c.z, x, acc[10]);
    acc[11] = fmaf(c.w, x, acc[11]);
    acc[12] = fmaf(d.x, x, acc[12]);
    acc[13] = fmaf(d.y, x, acc[13]);
    acc[14] = fmaf(d.z, x, acc[14]);
    acc[15] = fmaf(d.w, x, acc[15]);
  }
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (q < nu) pre[q * T] = acc[q];
}

// Pre-activations of the units [lo, hi) of one layer for the current group.
__device__ __forceinline__ void layer_preact(const float* blocks, int off, int n_in,
                                             int lo, int hi, const float* __restrict__ bias,
                                             const float* act, int T, float* pre) {
  for (int c = lo; c < hi; c += 16) {
    const int nu = min(16, hi - c);
    block_preact(blocks + off + (long long)(c - lo) * n_in, act, T, n_in, bias + c, nu,
                 pre + (c - lo) * T);
  }
}

// Ancestral sampling (Eq. 8), one thread per sample, T samples per CTA.
// Hidden units are degree-sorted, so output i (degree i+1) needs exactly the
// inputs 0..i-1, the layer-1 units of degree <= i and the layer-2 units of
// degree <= i, each evaluated once: one masked forward pass in total.
// The steps are processed in groups (host table `groups`, GROUP_INTS ints:
// i0, i1, u1lo, u1hi, u2lo, u2hi, off1, off2, offo, gstart, gsize, -, t1, t2, to):
//   the group's weight block is bulk-copied (TMA 1-D) into shared memory;
//   phase A: for the units completing inside the group, the contribution of
//            every input known before the group (register tiled, 16 units);
//   phase B: the group's steps one by one, adding the in-group contributions
//            and drawing s_i = +1 iff u < sigmoid(x_i).
// With `given` non-null the spins are read from it (teacher forcing).
// Shared memory: [unit][T] S [D], A1 [H1], A2 [H2], P1 [ug1], P2 [ug2],
// PO [ugo]; then the weight block [wmax] and one mbarrier.
__global__ void __launch_bounds__(64) sample_kernel(const InstDev* __restrict__ inst,
                                                    const LaunchInfo li,
                                                    int8_t* __restrict__ spins,
                                                    float* __restrict__ logq,
                                                    const int8_t* __restrict__ given) {
  extern __shared__ __align__(16) float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const int T = li.tile, t = threadIdx.x;
  const int b = (blockIdx.x - li.tile_begin[k]) * T + t;
  const int D = md.D, nh = md.nh, H1 = md.H1, H2 = md.H2;
  float* S = sm;
  float* A1 = S + D * T;
  float* A2 = A1 + H1 * T;
  float* P1 = A2 + H2 * T;
  float* P2 = P1 + md.ug1 * T;
  float* PO = P2 + md.ug2 * T;
  float* Wsm = PO + md.ugo * T;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Wsm + ((md.wmax + 3) & ~3));
  const float* src = nh == 0 ? S : (nh == 1 ? A1 : A2);
  const float* bias1 = md.packed + md.layer[0].dst_off + (long long)H1 * D;
  const float* bias2 = nh >= 2 ? md.packed + md.layer[1].dst_off + (long long)H2 * H1 : nullptr;
  const float* biaso = md.packed + md.layer[nh].dst_off + (long long)D * md.Hl;
  const int* cL = nh == 1 ? md.c1 : md.c2;
  const uint2 key = make_uint2((uint32_t)li.seed, (uint32_t)(li.seed >> 32));
  const uint32_t step32 = launch_step(li);
  const int8_t* gv = given ? given + I.spin_units * li.batch + (long long)b * D : nullptr;
  const bool valid = b < li.batch;
  if (t == 0) mbar_init(bar, 1);
  __syncthreads();
  float lq = 0.f;
  uint4 rnd = make_uint4(0, 0, 0, 0);
  for (int g = 0; g < md.n_groups; ++g) {
    const int* G = md.groups + GROUP_INTS * g;
    const int i0 = G[0], i1 = G[1], u1lo = G[2], u1hi = G[3], u2lo = G[4], u2hi = G[5];
    const int gsize = G[10];
    __syncthreads();  // every thread is done with the previous block
    if (t == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar, (uint32_t)gsize * 4u);
      bulk_g2s(Wsm, md.blocks + G[9], (uint32_t)gsize * 4u, bar);
    }
    if (!mbar_wait(bar, (uint32_t)(g & 1))) {
      if (t == 0) atomicExch(li.status, 1);
      return;
    }
    // phase A
    if (nh >= 1) layer_preact(Wsm, G[6], i0, u1lo, u1hi, bias1, S + t, T, P1 + t);
    if (nh >= 2) layer_preact(Wsm, G[7], u1lo, u2lo, u2hi, bias2, A1 + t, T, P2 + t);
    {
      const int n_in = nh == 0 ? i0 : (nh == 1 ? u1lo : u2lo);
      layer_preact(Wsm, G[8], n_in, i0, i1, biaso, src + t, T, PO + t);
    }
    // phase B
    const int gi = i1 - i0, n1 = u1hi - u1lo;
    const int clo = nh == 0 ? i0 : (nh == 1 ? u1lo : u2lo);
    const int nL = nh == 0 ? gi : (nh == 1 ? n1 : u2hi - u2lo);
    const float* TW1 = Wsm + G[12];
    const float* TW2 = Wsm + G[13];
    const float* TWo = Wsm + G[14];
    for (int i = i0; i < i1; ++i) {
      if ((i & 3) == 0)
        rnd = philox4x32_10(
            make_uint4((uint32_t)b, (uint32_t)(i >> 2), step32, (uint32_t)k), key);
      if (nh >= 1 && i >= 1) {
        for (int u = md.c1[i - 1]; u < md.c1[i]; ++u) {
          const float* w = TW1 + (u - u1lo) * gi;
          float a = P1[(u - u1lo) * T + t];
          for (int j = i0; j < i; ++j) a = fmaf(w[j - i0], S[j * T + t], a);
          A1[u * T + t] = fmaxf(a, 0.f);
        }
      }
      if (nh >= 2 && i >= 1) {
        const int n1i = md.c1[i];
        for (int v = md.c2[i - 1]; v < md.c2[i]; ++v) {
          const float* w = TW2 + (v - u2lo) * n1;
          float a = P2[(v - u2lo) * T + t];
          for (int u = u1lo; u < n1i; ++u) a = fmaf(w[u - u1lo], A1[u * T + t], a);
          A2[v * T + t] = fmaxf(a, 0.f);
        }
      }
      float x = PO[(i - i0) * T + t];
      {
        const float* w = TWo + (i - i0) * nL;
        const int chi = nh == 0 ? i : cL[i];
        for (int c = clo; c < chi; ++c) x = fmaf(w[c - clo], src[c * T + t], x);
      }
      const float p = 1.f / (1.f + expf(-x));
      const uint32_t word =
          (i & 3) == 0 ? rnd.x : (i & 3) == 1 ? rnd.y : (i & 3) == 2 ? rnd.z : rnd.w;
      const float u = (float)(word >> 8) * 5.9604644775390625e-08f;  // 2^-24
      float s = u < p ? 1.f : -1.f;
      if (gv) s = valid ? (float)gv[i] : 1.f;
      S[i * T + t] = s;
      lq -= softplusf(-s * x);
    }
  }
  if (valid) {
    if (spins) {
      int8_t* out = spins + I.spin_units * li.batch + (long long)b * D;
      for (int i = 0; i < D; ++i) out[i] = (int8_t)S[i * T + t];
    }
    logq[(long long)k * li.batch + b] = lq;
  }
}

int sample_smem_bytes(const Instance& in, int tile) {
  const MadeDev& md = in.dev.made;
  return (int)((in.W.size() + in.H[0] + in.H[1] + md.ug1 + md.ug2 + md.ugo) * tile * sizeof(float) +
               ((md.wmax + 3) & ~3) * sizeof(float) + 16);
}

cudaError_t launch_sample(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                          int8_t* spins, float* logq, const int8_t* given, cudaStream_t s) {
  int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes);
  if (e != cudaSuccess) return e;
  sample_kernel<<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, spins, logq, given);
  return cudaGetLastError();
}

}  // namespace tnvan
