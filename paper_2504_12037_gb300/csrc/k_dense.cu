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
#include "common.cuh"

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
  // bf16 copy, round to nearest even
  uint32_t u = __float_as_uint(c);
  u += 0x7fffu + ((u >> 16) & 1u);
  I.dense.C16[a * 256 + b] = (uint16_t)(u >> 16);
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
// batch mean accumulated into dJ.  Marginals of the factored form:
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
    const float iz = scale / z;
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

cudaError_t launch_dense(const InstDev* d_inst, const LaunchInfo& li_in, int precision,
                         const int8_t* spins, double* logZR, double* dbeta, double* dJ,
                         cudaStream_t s) {
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

}  // namespace tnvan
