// Dense leftover block (fully connected remainder, e.g. the SK model):
// exact sum over all 2^|R| states of R (Eq. 4), |R| <= 16, without SVD.
//
// R is split into halves A (8 spins) and B (8 spins); spins missing from a
// half are free phantoms that each double the sum (removed as ln 2 terms).
// With fields h(s) = J_RW s from the width set,
//   sum_r exp(beta[E'_RR(r) + h.r]) = g_A^T C g_B * exp(beta c_hat + beta |h|_1)
//   C(a,b)   = exp(beta[E'_AA(a) + E'_BB(b) + a^T J_AB b] - beta c_hat)   (per beta)
//   g_X(x)   = exp(beta h_X . x - beta |h_X|_1)                            (per sample)
// where E'_RR(r) = sum_{i<j in R} J_ij r_i r_j and c_hat = sum |J_ij| (so C <= 1).
// This is an exact regrouping of the 65536-term sum into a 256 x 256 bilinear
// form, i.e. a batched dense contraction [samples x 256] x [256 x 256].
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tnvan {

__device__ __forceinline__ float sgn_bit(int x, int i) { return ((x >> i) & 1) ? -1.f : 1.f; }

// C and dC/dbeta for every dense instance.  grid = (256 rows a, n_inst), 256 threads (b).
__global__ void __launch_bounds__(256) dense_table_kernel(const InstDev* __restrict__ inst,
                                                          const LaunchInfo li) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 1) return;
  __shared__ float J[256];
  J[threadIdx.x] = I.dense.JRR[threadIdx.x];
  __syncthreads();
  const int a = blockIdx.x, b = threadIdx.x;
  const int x = a | (b << 8);
  float E = 0.f;
#pragma unroll 4
  for (int i = 0; i < 16; ++i) {
    const float si = sgn_bit(x, i);
    float row = 0.f;
    for (int j = i + 1; j < 16; ++j) row = fmaf(J[i * 16 + j], sgn_bit(x, j), row);
    E = fmaf(si, row, E);
  }
  const float beta = (float)li.beta[k];
  const float ch = (float)I.dense.c_hat;
  const float c = expf(beta * (E - ch));
  I.dense.C32[a * 256 + b] = c;
  I.dense.dC32[a * 256 + b] = c * (E - ch);
  // bf16 copy (round to nearest even) in the tensor cores' canonical K-major
  // layout: row a, K index b, core matrices of 8 rows x 8 elements
  uint32_t u = __float_as_uint(c);
  u += 0x7fffu + ((u >> 16) & 1u);
  I.dense.C16[(a >> 3) * 2048 + (b >> 3) * 64 + (a & 7) * 8 + (b & 7)] = (uint16_t)(u >> 16);
}

#define DN_T 16  // samples per CTA (forward)

// Fields h[t][r] = sum_w J_RW[r][w] s_w and the W-W term for a tile of samples.
__device__ void dense_fields(const InstDev& I, const int8_t* sp, int D, int nv, float* h,
                             float* e1, int t) {
  {
    const int tt = t >> 4, r = t & 15;
    float acc = 0.f;
    if (tt < nv) {
      const float* jr = I.dense.JRW + r * D;
      const int8_t* st = sp + tt * D;
      for (int w = 0; w < D; ++w) acc = fmaf(__ldg(jr + w), (float)st[w], acc);
    }
    h[tt * 16 + r] = acc;
  }
  // W-W bonds: every thread takes a slice of the edge list for all samples
  float part[DN_T];
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) part[tt] = 0.f;
  for (int e = t; e < I.n_ww; e += blockDim.x) {
    const EdgeWW q = I.ww[e];
#pragma unroll
    for (int tt = 0; tt < DN_T; ++tt)
      if (tt < nv) part[tt] = fmaf(q.J, (float)(sp[tt * D + q.a] * sp[tt * D + q.b]), part[tt]);
  }
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) {
    const float v = warp_sum(part[tt]);
    if ((t & 31) == 0) e1[(t >> 5) * DN_T + tt] = v;
  }
}

template <bool DB>
__global__ void __launch_bounds__(256) dense_kernel(const InstDev* __restrict__ inst,
                                                    const LaunchInfo li,
                                                    const int8_t* __restrict__ spins,
                                                    double* __restrict__ logZR,
                                                    double* __restrict__ dbeta) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 1) return;
  const int t = threadIdx.x, D = I.D;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * DN_T;
  const int nv = min(DN_T, li.batch - b0);
  const float beta = (float)li.beta[k];
  float* gA = sm;                    // [T][256]
  float* gB = gA + DN_T * 256;       // [T][256]
  float* dgA = gB + DN_T * 256;      // [T][256] (DB)
  float* dgB = dgA + DN_T * 256;     // [T][256] (DB)
  float* h = dgB + DN_T * 256;       // [T][16]
  float* e1 = h + DN_T * 16;         // [8 warps][T]
  float* red = e1 + 8 * DN_T;        // [8 warps][T][2]
  int8_t* sp = reinterpret_cast<int8_t*>(red + 8 * DN_T * 2);  // [T][D]
  const int8_t* g = spins + I.spin_units * li.batch + (long long)b0 * D;
  for (int e = t; e < nv * D; e += blockDim.x) sp[e] = g[e];
  __syncthreads();
  dense_fields(I, sp, D, nv, h, e1, t);
  __syncthreads();
  for (int tt = 0; tt < DN_T; ++tt) {
    float sa = 0.f, aa = 0.f, sb = 0.f, ab = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float ha = h[tt * 16 + i], hb = h[tt * 16 + 8 + i];
      sa = fmaf(ha, sgn_bit(t, i), sa);
      aa += fabsf(ha);
      sb = fmaf(hb, sgn_bit(t, i), sb);
      ab += fabsf(hb);
    }
    const float ga = expf(beta * (sa - aa)), gb = expf(beta * (sb - ab));
    gA[tt * 256 + t] = ga;
    gB[tt * 256 + t] = gb;
    if (DB) {
      dgA[tt * 256 + t] = ga * (sa - aa);
      dgB[tt * 256 + t] = gb * (sb - ab);
    }
  }
  __syncthreads();
  // y0 = C gB, y1 = dC gB, y2 = C dgB for row a = t
  float y0[DN_T], y1[DN_T], y2[DN_T];
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) y0[tt] = y1[tt] = y2[tt] = 0.f;
  const float4* crow = reinterpret_cast<const float4*>(I.dense.C32 + t * 256);
  const float4* dcrow = reinterpret_cast<const float4*>(I.dense.dC32 + t * 256);
  for (int b4 = 0; b4 < 64; ++b4) {
    const float4 c = __ldg(crow + b4);
    float4 dc = make_float4(0, 0, 0, 0);
    if (DB) dc = __ldg(dcrow + b4);
#pragma unroll
    for (int tt = 0; tt < DN_T; ++tt) {
      const float4 v = reinterpret_cast<const float4*>(gB + tt * 256)[b4];
      y0[tt] = fmaf(c.x, v.x, fmaf(c.y, v.y, fmaf(c.z, v.z, fmaf(c.w, v.w, y0[tt]))));
      if (DB) {
        const float4 dv = reinterpret_cast<const float4*>(dgB + tt * 256)[b4];
        y1[tt] = fmaf(dc.x, v.x, fmaf(dc.y, v.y, fmaf(dc.z, v.z, fmaf(dc.w, v.w, y1[tt]))));
        y2[tt] = fmaf(c.x, dv.x, fmaf(c.y, dv.y, fmaf(c.z, dv.z, fmaf(c.w, dv.w, y2[tt]))));
      }
    }
  }
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) {
    const float ga = gA[tt * 256 + t];
    float z = warp_sum(ga * y0[tt]);
    float dz = 0.f;
    if (DB) dz = warp_sum(dgA[tt * 256 + t] * y0[tt] + ga * (y1[tt] + y2[tt]));
    if ((t & 31) == 0) {
      red[((t >> 5) * DN_T + tt) * 2] = z;
      red[((t >> 5) * DN_T + tt) * 2 + 1] = dz;
    }
  }
  __syncthreads();
  if (t < nv) {
    float z = 0.f, dz = 0.f, ew = 0.f;
    for (int w = 0; w < 8; ++w) {
      z += red[(w * DN_T + t) * 2];
      dz += red[(w * DN_T + t) * 2 + 1];
      ew += e1[w * DN_T + t];
    }
    double habs = 0.0;
    for (int r = 0; r < 16; ++r) habs += fabs((double)h[t * 16 + r]);
    const double chf = (double)(float)I.dense.c_hat;
    const double bd = li.beta[k];
    const double phantom = (16 - I.dense.nR) * 0.69314718055994530942;
    const long long o = (long long)k * li.batch + b0 + t;
    if (logZR) logZR[o] = bd * ((double)ew + chf + habs) + (double)logf(z) - phantom;
    if (DB) dbeta[o] = (double)ew + chf + habs + (double)(dz / z);
  }
}

// ---------------------------------------------------------------------------
// Reverse mode: d ln Z_R / d J = beta <r_i r_j> (R-R) or beta s_w <r_i> (R-W),
// batch mean accumulated into dJ (each sample weighted by li.wmul when given).  Marginals of the factored form:
//   P(a, b) = g_A(a) C(a,b) g_B(b) / z
// needs Y_j = C (g_B * sigma_j) for the 8 B spins, Y_0 = C g_B and U = C^T g_A.
// ---------------------------------------------------------------------------
#define DJ_T 4

__device__ __forceinline__ float block_sum256(float v, float* scratch, int t) {
  v = warp_sum(v);
  __syncthreads();
  if ((t & 31) == 0) scratch[t >> 5] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) s += scratch[w];
  return s;
}

__global__ void __launch_bounds__(256) dense_dJ_kernel(const InstDev* __restrict__ inst,
                                                       const LaunchInfo li,
                                                       const int8_t* __restrict__ spins,
                                                       double* __restrict__ dJ) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 1) return;
  const int t = threadIdx.x, D = I.D;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * DJ_T;
  const int nv = min(DJ_T, li.batch - b0);
  const float beta = (float)li.beta[k];
  float* gA = sm;                 // [T][256]
  float* gB = gA + DJ_T * 256;    // [T][256]
  float* h = gB + DJ_T * 256;     // [T][16]
  float* scratch = h + DJ_T * 16; // [8]
  int8_t* sp = reinterpret_cast<int8_t*>(scratch + 8);
  const int8_t* g = spins + I.spin_units * li.batch + (long long)b0 * D;
  for (int e = t; e < nv * D; e += blockDim.x) sp[e] = g[e];
  __syncthreads();
  if (t < DJ_T * 16) {
    const int tt = t >> 4, r = t & 15;
    float acc = 0.f;
    if (tt < nv)
      for (int w = 0; w < D; ++w) acc = fmaf(I.dense.JRW[r * D + w], (float)sp[tt * D + w], acc);
    h[tt * 16 + r] = acc;
  }
  __syncthreads();
  for (int tt = 0; tt < DJ_T; ++tt) {
    float sa = 0.f, aa = 0.f, sb = 0.f, ab = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float ha = h[tt * 16 + i], hb = h[tt * 16 + 8 + i];
      sa = fmaf(ha, sgn_bit(t, i), sa);
      aa += fabsf(ha);
      sb = fmaf(hb, sgn_bit(t, i), sb);
      ab += fabsf(hb);
    }
    gA[tt * 256 + t] = expf(beta * (sa - aa));
    gB[tt * 256 + t] = expf(beta * (sb - ab));
  }
  __syncthreads();
  // thread t as row a: y[tt][j] = sum_b C[a][b] gB[b] (sigma_j(b) for j >= 1)
  // thread t as column b: u[tt] = sum_a C[a][b] gA[a]
  float y[DJ_T][9], u[DJ_T];
#pragma unroll
  for (int tt = 0; tt < DJ_T; ++tt) {
    u[tt] = 0.f;
#pragma unroll
    for (int j = 0; j < 9; ++j) y[tt][j] = 0.f;
  }
  const float* C = I.dense.C32;
  for (int b = 0; b < 256; ++b) {
    const float c = __ldg(C + t * 256 + b);
    const float cc = __ldg(C + b * 256 + t);
#pragma unroll
    for (int tt = 0; tt < DJ_T; ++tt) {
      const float v = c * gB[tt * 256 + b];
      y[tt][0] += v;
#pragma unroll
      for (int j = 0; j < 8; ++j) y[tt][j + 1] = fmaf(v, sgn_bit(b, j), y[tt][j + 1]);
      u[tt] = fmaf(cc, gA[tt * 256 + b], u[tt]);
    }
  }
  const float scale = beta / (float)li.batch;
  for (int tt = 0; tt < DJ_T; ++tt) {
    if (tt >= nv) break;  // uniform across the block
    const float ga = gA[tt * 256 + t];
    const float z = block_sum256(ga * y[tt][0], scratch, t);
    // per-sample weight of the bond sums (importance multipliers when given)
    const float wv = li.wmul ? li.wmul[(long long)k * li.batch + b0 + tt] : 1.f;
    const float iz = scale * wv / z;
    const int8_t* st = sp + tt * D;
    // single-spin marginals -> R-W bonds
    for (int r = 0; r < 16; ++r) {
      float m;
      if (r < 8) m = block_sum256(ga * sgn_bit(t, r) * y[tt][0], scratch, t);
      else m = block_sum256(ga * y[tt][r - 8 + 1], scratch, t);
      for (int w = t; w < D; w += blockDim.x) {
        const int e = I.dense.eRW[r * D + w];
        if (e >= 0) atomicAdd(dJ + I.edge_off + e, (double)(m * iz * (float)st[w]));
      }
    }
    // pair marginals -> R-R bonds
    for (int i = 0; i < 16; ++i)
      for (int j = i + 1; j < 16; ++j) {
        const int e = I.dense.eRR[i * 16 + j];
        if (e < 0) continue;  // uniform: same table for every thread
        float v;
        if (j < 8) v = ga * sgn_bit(t, i) * sgn_bit(t, j) * y[tt][0];
        else if (i < 8) v = ga * sgn_bit(t, i) * y[tt][j - 8 + 1];
        else v = gB[tt * 256 + t] * sgn_bit(t, i - 8) * sgn_bit(t, j - 8) * u[tt];
        const float m = block_sum256(v, scratch, t);
        if (t == 0) atomicAdd(dJ + I.edge_off + e, (double)(m * iz));
      }
  }
}

// ---------------------------------------------------------------------------
// BF16 tensor-core form (precision TNVAN_BF16): per CTA a persistent walk over
// 128-sample tiles of one instance.  C (256 x 256, BF16, canonical layout) is
// bulk-copied into shared memory once; per tile every thread builds its
// sample's g_B row (256 BF16 values from 2 x 16 partial products), one
// elected thread issues the [128 x 256] x [256 x 256] product into TMEM
// (16 tcgen05.mma of K = 16), and each thread finishes z = g_A . (C g_B) from
// its TMEM lane, with g_A again from 2 x 16 partial products.
// ---------------------------------------------------------------------------
#define DTC_TILES_PER_CTA 8

__device__ __forceinline__ void half_products(const float* h, float beta, float* lo, float* hi) {
  // g(x) = exp(beta h.sigma(x) - beta |h|_1) over 8 spins = lo[x & 15] * hi[x >> 4]
#pragma unroll
  for (int x = 0; x < 16; ++x) {
    float a = 0.f, c = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a += h[i] * sgn_bit(x, i) - fabsf(h[i]);
      c += h[4 + i] * sgn_bit(x, i) - fabsf(h[4 + i]);
    }
    lo[x] = expf(beta * a);
    hi[x] = expf(beta * c);
  }
}

// The W-side terms of a tile (Eq. 4: the fields h = J_RW s on R and the W-W
// energy E_1(s)) are computed from the sample's spins held as 64 bits, with
// the couplings in shared memory (J_RW transposed [DMAX][16], J_WW as a dense
// upper triangle [DMAX][DMAX]) and every loop unrolled to DMAX >= D, so that
// no global load sits on the per-sample chain.  DMAX = 0: D > 64, the same
// sums straight from global memory.
template <int DMAX>
__global__ void __launch_bounds__(128, 1) dense_tc_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                          const int8_t* __restrict__ spins,
                                                          double* __restrict__ logZR) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 1) return;
  const int t = threadIdx.x, w = t >> 5, D = I.D;
  const int tiles = (li.batch + 127) / 128;
  const int per_cta = li.tile;  // tiles of this instance per CTA
  const int tile0 = (blockIdx.x - li.tile_begin[k]) * per_cta;
  const int tile1 = min(tiles, tile0 + per_cta);
  unsigned char* sC = smem;                   // 128 KB
  unsigned char* sG = smem + 131072;          // [128 x 256] BF16, 64 KB
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 131072 + 65536);
  uint64_t* cbar = bar + 1;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  float* sJ1 = reinterpret_cast<float*>(smem + 131072 + 65536 + 64);  // [DMAX][16] J_RW^T
  float* sJ2 = sJ1 + DMAX * 16;                                        // [DMAX][DMAX] J_WW, i < j
  if (DMAX > 0) {
    for (int e = t; e < DMAX * 16; e += 128) {
      const int wp = e >> 4, r = e & 15;
      sJ1[e] = wp < D ? I.dense.JRW[r * D + wp] : 0.f;
    }
    for (int e = t; e < DMAX * DMAX; e += 128) sJ2[e] = 0.f;
    __syncthreads();
    for (int e = t; e < I.n_ww; e += 128) {
      const EdgeWW q = I.ww[e];
      sJ2[min(q.a, q.b) * DMAX + max(q.a, q.b)] = q.J;
    }
  }
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  if (w == 0) {
    tc::tmem_alloc(slot, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (t == 0) {
    mbar_expect_tx(cbar, 131072u);
    bulk_g2s(sC, I.dense.C16, 131072u, cbar);
  }
  bool ok = mbar_wait(cbar, 0);
  const uint32_t tmem = *slot;
  const uint32_t lane_off = (uint32_t)(w * 32) << 16;
  const uint32_t id = tc::idesc(128, 256, 1u);
  const float beta = (float)li.beta[k];
  const double bd = li.beta[k];
  const double chf = (double)(float)I.dense.c_hat;
  const double phantom = (16 - I.dense.nR) * 0.69314718055994530942;
  uint32_t phase = 0;
  for (int tile = tile0; tile < tile1 && ok; ++tile) {
    const int b = tile * 128 + t;
    const bool valid = b < li.batch;
    const int8_t* st = spins + I.spin_units * li.batch + (long long)(valid ? b : 0) * D;
    float h[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) h[r] = 0.f;
    float e1 = 0.f;
    if (DMAX > 0) {
      unsigned long long m = 0ull;  // bit w: spin w is +1
      if ((D & 15) == 0 && (reinterpret_cast<uintptr_t>(spins + I.spin_units * li.batch) & 15) == 0) {
        for (int c = 0; c < D; c += 16) {
          const uint4 raw = *reinterpret_cast<const uint4*>(st + c);
          const uint32_t wv[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int i = 0; i < 16; ++i)
            m |= (unsigned long long)((int8_t)((wv[i >> 2] >> (8 * (i & 3))) & 0xFFu) > 0) << (c + i);
        }
      } else {
        for (int w = 0; w < D; ++w) m |= (unsigned long long)(st[w] > 0) << w;
      }
      float sv[DMAX > 0 ? DMAX : 1];
#pragma unroll
      for (int w = 0; w < DMAX; ++w) sv[w] = w < D ? (((m >> w) & 1ull) ? 1.f : -1.f) : 0.f;
#pragma unroll
      for (int w = 0; w < DMAX; ++w) {
        const float4* j4 = reinterpret_cast<const float4*>(sJ1 + w * 16);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 jq = j4[q];
          h[4 * q + 0] = fmaf(jq.x, sv[w], h[4 * q + 0]);
          h[4 * q + 1] = fmaf(jq.y, sv[w], h[4 * q + 1]);
          h[4 * q + 2] = fmaf(jq.z, sv[w], h[4 * q + 2]);
          h[4 * q + 3] = fmaf(jq.w, sv[w], h[4 * q + 3]);
        }
      }
#pragma unroll
      for (int i = 0; i + 1 < DMAX; ++i) {  // sum_{i<j} J_ij s_i s_j, rows of the upper triangle
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int j = i + 1; j < DMAX; j += 2) {
          a0 = fmaf(sJ2[i * DMAX + j], sv[j], a0);
          if (j + 1 < DMAX) a1 = fmaf(sJ2[i * DMAX + j + 1], sv[j + 1], a1);
        }
        e1 = fmaf(sv[i], a0 + a1, e1);
      }
    } else {
      for (int wpos = 0; wpos < D; ++wpos) {
        const float sw = (float)st[wpos];
#pragma unroll
        for (int r = 0; r < 16; ++r) h[r] = fmaf(__ldg(I.dense.JRW + r * D + wpos), sw, h[r]);
      }
      for (int e = 0; e < I.n_ww; ++e) {
        const EdgeWW q = I.ww[e];
        e1 = fmaf(q.J, (float)(st[q.a] * st[q.b]), e1);
      }
    }
    float lo[16], hi[16];
    half_products(h + 8, beta, lo, hi);  // g_B over the B half
    for (int c = 0; c < 256; c += 8) {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(lo[(c + 0) & 15] * hi[c >> 4], lo[(c + 1) & 15] * hi[c >> 4]);
      __nv_bfloat162 p1 = __floats2bfloat162_rn(lo[(c + 2) & 15] * hi[c >> 4], lo[(c + 3) & 15] * hi[c >> 4]);
      __nv_bfloat162 p2 = __floats2bfloat162_rn(lo[(c + 4) & 15] * hi[c >> 4], lo[(c + 5) & 15] * hi[c >> 4]);
      __nv_bfloat162 p3 = __floats2bfloat162_rn(lo[(c + 6) & 15] * hi[c >> 4], lo[(c + 7) & 15] * hi[c >> 4]);
      uint4 u;
      u.x = *reinterpret_cast<uint32_t*>(&p0);
      u.y = *reinterpret_cast<uint32_t*>(&p1);
      u.z = *reinterpret_cast<uint32_t*>(&p2);
      u.w = *reinterpret_cast<uint32_t*>(&p3);
      *reinterpret_cast<uint4*>(sG + (t >> 3) * 4096 + (c >> 3) * 128 + (t & 7) * 16) = u;
    }
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      for (int kk = 0; kk < 16; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc(smem_u32(sG) + kk * 256u, 128u, 4096u),
                     tc::smem_desc(smem_u32(sC) + kk * 256u, 128u, 4096u), id, kk > 0 ? 1u : 0u);
      tc::mma_commit(bar);
    }
    ok = mbar_wait(bar, phase);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) break;
    half_products(h, beta, lo, hi);  // g_A over the A half
    float z = 0.f;
    for (int c = 0; c < 256; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + lane_off + (uint32_t)c, v);
      float part = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) part = fmaf(lo[i], v[i], part);
      z = fmaf(hi[c >> 4], part, z);
    }
    if (valid) {
      double habs = 0.0;
      for (int r = 0; r < 16; ++r) habs += fabs((double)h[r]);
      logZR[(long long)k * li.batch + b] = bd * ((double)e1 + chf + habs) + (double)logf(z) - phantom;
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM read and G tile consumed before the next tile overwrites them
    tc::fence_after_sync();
  }
  if (!ok && t == 0) atomicExch(li.status, 5);
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, 256);
}

cudaError_t launch_dense(const InstDev* d_inst, const LaunchInfo& li_in, int precision,
                         const int8_t* spins, double* logZR, double* dbeta, double* dJ,
                         cudaStream_t s, int max_D) {
  (void)precision;
  if (li_in.n_inst == 0 || li_in.batch == 0) return cudaSuccess;
  int max_d = 0;
  LaunchInfo li = li_in;
  const int T = dJ ? DJ_T : DN_T;
  int acc = 0;
  for (int k = 0; k < li.n_inst; ++k) {
    li.tile_begin[k] = acc;
    acc += (li.batch + T - 1) / T;
  }
  li.tile_begin[li.n_inst] = acc;
  li.tile = T;
  // the table depends on beta: rebuilt on every call (65536 entries per instance)
  dense_table_kernel<<<dim3(256, li.n_inst), 256, 0, s>>>(d_inst, li);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (precision == TNVAN_BF16 && !dJ && !dbeta && logZR) {
    LaunchInfo lt = li_in;
    const int tiles = (li.batch + 127) / 128;
    // tiles per CTA: enough CTAs to cover the SMs, at most DTC_TILES_PER_CTA
    // (each CTA copies the 128 KB table once)
    int n_sm = 148;
    {
      int dev = 0;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    const int want = (tiles * lt.n_inst + n_sm - 1) / n_sm;
    const int per_cta = want < 1 ? 1 : (want > DTC_TILES_PER_CTA ? DTC_TILES_PER_CTA : want);
    const int per = (tiles + per_cta - 1) / per_cta;
    for (int k = 0; k <= lt.n_inst; ++k) lt.tile_begin[k] = k * per;
    lt.tile = per_cta;
    const int dmax = max_D;  // the largest width set of the dense instances
    auto go = [&](auto kern, int DM) -> cudaError_t {
      const int smem = 131072 + 65536 + 64 + 4 * (DM * 16 + DM * DM);
      cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e2 != cudaSuccess) return e2;
      kern<<<lt.tile_begin[lt.n_inst], 128, smem, s>>>(d_inst, lt, spins, logZR);
      return cudaGetLastError();
    };
    if (dmax <= 16) return go(dense_tc_kernel<16>, 16);
    if (dmax <= 32) return go(dense_tc_kernel<32>, 32);
    if (dmax <= 48) return go(dense_tc_kernel<48>, 48);
    if (dmax <= 64) return go(dense_tc_kernel<64>, 64);
    return go(dense_tc_kernel<0>, 0);
  }
  max_d = TNVAN_MAX_D;
  if (dJ) {
    const int smem = (DJ_T * 256 * 2 + DJ_T * 16 + 8) * 4 + DJ_T * max_d;
    e = cudaFuncSetAttribute(dense_dJ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dense_dJ_kernel<<<acc, 256, smem, s>>>(d_inst, li, spins, dJ);
    return cudaGetLastError();
  }
  const int smem = (DN_T * 256 * 4 + DN_T * 16 + 8 * DN_T + 8 * DN_T * 2) * 4 + DN_T * max_d;
  if (dbeta) {
    e = cudaFuncSetAttribute(dense_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dense_kernel<true><<<acc, 256, smem, s>>>(d_inst, li, spins, logZR, dbeta);
  } else {
    e = cudaFuncSetAttribute(dense_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dense_kernel<false><<<acc, 256, smem, s>>>(d_inst, li, spins, logZR, dbeta);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Magnetisation moments of the dense block (observables from samples, Sec. 3):
// the conditional mean and variance of M_R = sum of the real R spins given
// the width set, from the same factored sum.  With P(a, b) = g_A(a) C(a,b)
// g_B(b) / z and M_R = M_A(a) + M_B(b) (phantom spins excluded):
//   pass 1:  m = sum_a g_A(a) [M_A(a) (C g_B)(a) + (C (g_B M_B))(a)] / z;
//   pass 2:  var = sum_a g_A(a) [al^2 (C g_B) + 2 al (C (g_B be)) + C (g_B be^2)](a) / z
// with al = M_A - m/2 and be = M_B - m/2, so the variance is a sum of
// non-negative centred terms.  FP32, DN_T samples per CTA, thread t = row a
// of C.  Output E[M | s] = M_W(s) + m and Var(M | s) = var.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float half_mag(int x, int n) {
  return (float)(n - 2 * __popc(x & ((1 << n) - 1)));
}

__global__ void __launch_bounds__(256) dense_mom_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                        const int8_t* __restrict__ spins,
                                                        double* __restrict__ mag_mean, double* __restrict__ mag_var) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 1) return;
  const int t = threadIdx.x, D = I.D;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * DN_T;
  const int nv = min(DN_T, li.batch - b0);
  const float beta = (float)li.beta[k];
  const int nA = I.dense.nA, nB = I.dense.nB;
  float* gA = sm;                    // [T][256]
  float* gB = gA + DN_T * 256;       // [T][256]
  float* h = gB + DN_T * 256;        // [T][16]
  float* e1 = h + DN_T * 16;         // [8 warps][T] (fields helper scratch)
  float* red = e1 + 8 * DN_T;        // [8 warps][T][2]
  float* cen = red + 8 * DN_T * 2;   // [T] m / 2
  float* zs = cen + DN_T;            // [T] z
  int8_t* sp = reinterpret_cast<int8_t*>(zs + DN_T);  // [T][D]
  const int8_t* g = spins + I.spin_units * li.batch + (long long)b0 * D;
  for (int e = t; e < nv * D; e += blockDim.x) sp[e] = g[e];
  __syncthreads();
  dense_fields(I, sp, D, nv, h, e1, t);
  __syncthreads();
  for (int tt = 0; tt < DN_T; ++tt) {
    float sa = 0.f, aa = 0.f, sb = 0.f, ab = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float ha = h[tt * 16 + i], hb = h[tt * 16 + 8 + i];
      sa = fmaf(ha, sgn_bit(t, i), sa);
      aa += fabsf(ha);
      sb = fmaf(hb, sgn_bit(t, i), sb);
      ab += fabsf(hb);
    }
    gA[tt * 256 + t] = expf(beta * (sa - aa));
    gB[tt * 256 + t] = expf(beta * (sb - ab));
  }
  __syncthreads();
  const float4* crow = reinterpret_cast<const float4*>(I.dense.C32 + t * 256);
  const float ma = half_mag(t, nA);
  float y0[DN_T], y1[DN_T];
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) y0[tt] = y1[tt] = 0.f;
  // pass 1: C g_B and C (g_B M_B)
  for (int b4 = 0; b4 < 64; ++b4) {
    const float4 c = __ldg(crow + b4);
    const float m0 = half_mag(4 * b4, nB), m1 = half_mag(4 * b4 + 1, nB), m2 = half_mag(4 * b4 + 2, nB),
                m3 = half_mag(4 * b4 + 3, nB);
#pragma unroll
    for (int tt = 0; tt < DN_T; ++tt) {
      const float4 v = reinterpret_cast<const float4*>(gB + tt * 256)[b4];
      const float p0 = c.x * v.x, p1 = c.y * v.y, p2 = c.z * v.z, p3 = c.w * v.w;
      y0[tt] += (p0 + p1) + (p2 + p3);
      y1[tt] = fmaf(p0, m0, fmaf(p1, m1, fmaf(p2, m2, fmaf(p3, m3, y1[tt]))));
    }
  }
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) {
    const float ga = gA[tt * 256 + t];
    const float z = warp_sum(ga * y0[tt]);
    const float s1 = warp_sum(ga * fmaf(ma, y0[tt], y1[tt]));
    if ((t & 31) == 0) {
      red[((t >> 5) * DN_T + tt) * 2] = z;
      red[((t >> 5) * DN_T + tt) * 2 + 1] = s1;
    }
  }
  __syncthreads();
  if (t < DN_T) {
    float z = 0.f, s1 = 0.f;
    for (int w = 0; w < 8; ++w) {
      z += red[(w * DN_T + t) * 2];
      s1 += red[(w * DN_T + t) * 2 + 1];
    }
    cen[t] = t < nv ? 0.5f * s1 / z : 0.f;
    zs[t] = z;
  }
  __syncthreads();
  // pass 2: centred second moment
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) y1[tt] = 0.f;
  float y2[DN_T];
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) y2[tt] = 0.f;
  for (int b4 = 0; b4 < 64; ++b4) {
    const float4 c = __ldg(crow + b4);
    const float m0 = half_mag(4 * b4, nB), m1 = half_mag(4 * b4 + 1, nB), m2 = half_mag(4 * b4 + 2, nB),
                m3 = half_mag(4 * b4 + 3, nB);
#pragma unroll
    for (int tt = 0; tt < DN_T; ++tt) {
      const float4 v = reinterpret_cast<const float4*>(gB + tt * 256)[b4];
      const float ct = cen[tt];
      const float d0 = m0 - ct, d1 = m1 - ct, d2 = m2 - ct, d3 = m3 - ct;
      const float p0 = c.x * v.x * d0, p1 = c.y * v.y * d1, p2 = c.z * v.z * d2, p3 = c.w * v.w * d3;
      y1[tt] += (p0 + p1) + (p2 + p3);
      y2[tt] = fmaf(p0, d0, fmaf(p1, d1, fmaf(p2, d2, fmaf(p3, d3, y2[tt]))));
    }
  }
  __syncthreads();  // red is reused
#pragma unroll
  for (int tt = 0; tt < DN_T; ++tt) {
    const float ga = gA[tt * 256 + t];
    const float al = ma - cen[tt];
    const float q = warp_sum(ga * fmaf(al * al, y0[tt], fmaf(2.f * al, y1[tt], y2[tt])));
    if ((t & 31) == 0) red[((t >> 5) * DN_T + tt) * 2] = q;
  }
  __syncthreads();
  if (t < nv) {
    float q = 0.f;
    for (int w = 0; w < 8; ++w) q += red[(w * DN_T + t) * 2];
    int mw = 0;
    for (int j = 0; j < D; ++j) mw += sp[t * D + j];
    const long long o = (long long)k * li.batch + b0 + t;
    mag_mean[o] = (double)mw + 2.0 * (double)cen[t];
    mag_var[o] = (double)(q / zs[t]);
  }
}

int dense_mom_smem_bytes(int D) {
  return (2 * DN_T * 256 + DN_T * 16 + 8 * DN_T + 8 * DN_T * 2 + 2 * DN_T) * 4 + DN_T * D;
}

cudaError_t launch_dense_mom(const InstDev* d_inst, const LaunchInfo& li_in, int max_D, const int8_t* spins,
                             double* mag_mean, double* mag_var, cudaStream_t s) {
  if (li_in.n_inst == 0 || li_in.batch == 0) return cudaSuccess;
  LaunchInfo li = li_in;
  int acc = 0;
  for (int k = 0; k < li.n_inst; ++k) {
    li.tile_begin[k] = acc;
    acc += (li.batch + DN_T - 1) / DN_T;
  }
  li.tile_begin[li.n_inst] = acc;
  li.tile = DN_T;
  dense_table_kernel<<<dim3(256, li.n_inst), 256, 0, s>>>(d_inst, li);  // C at this call's betas
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int smem = dense_mom_smem_bytes(max_D);
  e = cudaFuncSetAttribute(dense_mom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dense_mom_kernel<<<acc, 256, smem, s>>>(d_inst, li, spins, mag_mean, mag_var);
  return cudaGetLastError();
}

}  // namespace tnvan
