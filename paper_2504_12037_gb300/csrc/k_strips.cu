// Lattice strips: exact row transfer-matrix contraction of the leftover
// sub-systems (Eq. 2-4 with W = whole columns), SVD-free, with power-of-two
// renormalisation after every row.
//
// A strip of w columns and L rows is contracted as
//   Z_strip(s) = 1^T D_0(s) V_0 D_1(s) V_1 ... D_{L-1}(s) 1,
// where D_y is diagonal over the 2^w states of row y (horizontal bonds of the
// row plus the fields J_L s_L, J_R s_R of the W neighbours left and right) and
// V_y is the Kronecker product of the w vertical 2x2 Boltzmann matrices
// B(+,+) = B(-,-) = e^{beta J}, B(+,-) = e^{-beta J} (Eq. 2).  Each factor is
// stored normalised (largest entry 1) and the removed constant
// beta * c_hat is added back in FP64 at the end.
#include "common.cuh"

namespace tnvan {

// Per-strip table layout in shared memory (floats, offset tab_off):
//   vert  [L][w] float4 (a, b, da/dbeta, db/dbeta): 2x2 factor [[a,b],[b,a]]
//   diag  [L][4][2^w]   D_y for the 4 combinations of (s_L, s_R) signs
//   ddiag [L][4][2^w]   d D_y / d beta
//   pos   [L][2] int    AR positions of the left / right W neighbours (-1 none)
__host__ __device__ inline int strip_tab_floats(int w, int L) {
  int n = L * w * 4 + 2 * L * 4 * (1 << w) + 2 * L;
  return (n + 3) & ~3;
}

__device__ __forceinline__ float spin_of(int x, int c) { return ((x >> c) & 1) ? -1.f : 1.f; }

__device__ void build_strip_tables(const InstDev& I, float beta, float* sm, int t, int T) {
  for (int st = 0; st < I.n_strips; ++st) {
    const StripDev sd = I.strips[st];
    const int w = sd.w, L = sd.L, nx = 1 << w;
    float* tab = sm + sd.tab_off;
    float4* vert = reinterpret_cast<float4*>(tab);
    float* diag = tab + L * w * 4;
    float* ddiag = diag + L * 4 * nx;
    int* pos = reinterpret_cast<int*>(ddiag + L * 4 * nx);
    const StripRow* rows = I.rows + sd.row0;
    for (int e = t; e < L * 4 * nx; e += T) {
      const int x = e % nx, idx = (e / nx) & 3, y = e / (4 * nx);
      const StripRow& R = rows[y];
      float ex = 0.f, ch = 0.f;
      for (int c = 0; c + 1 < w; ++c) {
        ex += R.Jh[c] * spin_of(x, c) * spin_of(x, c + 1);
        ch += fabsf(R.Jh[c]);
      }
      if (R.posL >= 0) {
        ex += R.JL * ((idx & 1) ? -1.f : 1.f) * spin_of(x, 0);
        ch += fabsf(R.JL);
      }
      if (R.posR >= 0) {
        ex += R.JR * ((idx & 2) ? -1.f : 1.f) * spin_of(x, w - 1);
        ch += fabsf(R.JR);
      }
      const float d = expf(beta * (ex - ch));
      diag[e] = d;
      ddiag[e] = d * (ex - ch);
    }
    for (int e = t; e < L * w; e += T) {
      const int y = e / w, c = e % w;
      const float J = rows[y].Jv[c], aj = fabsf(J);
      const float tt = (y + 1 < L) ? expf(-2.f * beta * aj) : 1.f;
      const float dt = -2.f * aj * tt;
      vert[e] = J >= 0.f ? make_float4(1.f, tt, 0.f, dt) : make_float4(tt, 1.f, dt, 0.f);
    }
    for (int y = t; y < L; y += T) {
      pos[2 * y] = rows[y].posL;
      pos[2 * y + 1] = rows[y].posR;
    }
  }
}

// Apply [[a,b],[b,a]] on bit c of the state index (and its beta-derivative).
template <int W, bool DB>
__device__ __forceinline__ void apply_pair(float (&v)[1 << W], float (&g)[1 << W], int c, float4 q) {
#pragma unroll
  for (int x = 0; x < (1 << W); ++x) {
    if ((x >> c) & 1) continue;
    const int x1 = x | (1 << c);
    const float v0 = v[x], v1 = v[x1];
    if (DB) {
      const float g0 = g[x], g1 = g[x1];
      g[x] = fmaf(q.x, g0, fmaf(q.y, g1, fmaf(q.z, v0, q.w * v1)));
      g[x1] = fmaf(q.y, g0, fmaf(q.x, g1, fmaf(q.w, v0, q.z * v1)));
    }
    v[x] = fmaf(q.x, v0, q.y * v1);
    v[x1] = fmaf(q.y, v0, q.x * v1);
  }
}

__device__ __forceinline__ int row_index(const int* pos, int y, const int8_t* srow) {
  const int pL = pos[2 * y], pR = pos[2 * y + 1];
  const int bl = (pL >= 0) ? (srow[pL] < 0) : 0;
  const int br = (pR >= 0) ? (srow[pR] < 0) : 0;
  return bl | (br << 1);
}

// Contract one strip for one sample.  Returns ln Z_strip - beta*c_hat as
// (float mantissa part, integer power-of-two exponent) and d/dbeta of it.
template <int W, bool DB>
__device__ void strip_chain(const float* tab, int L, const int8_t* srow, double& lnz, float& dl) {
  constexpr int NX = 1 << W;
  const float4* vert = reinterpret_cast<const float4*>(tab);
  const float* diag = tab + L * W * 4;
  const float* ddiag = diag + L * 4 * NX;
  const int* pos = reinterpret_cast<const int*>(ddiag + L * 4 * NX);
  float v[NX], g[NX];
  int e2 = 0;
  for (int y = 0; y < L; ++y) {
    const int idx = row_index(pos, y, srow);
    const float* dy = diag + (y * 4 + idx) * NX;
    const float* gy = ddiag + (y * 4 + idx) * NX;
    if (y == 0) {
#pragma unroll
      for (int x = 0; x < NX; ++x) {
        v[x] = dy[x];
        g[x] = DB ? gy[x] : 0.f;
      }
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) apply_pair<W, DB>(v, g, c, vert[(y - 1) * W + c]);
#pragma unroll
      for (int x = 0; x < NX; ++x) {
        if (DB) g[x] = fmaf(dy[x], g[x], gy[x] * v[x]);
        v[x] *= dy[x];
      }
    }
    float m = v[0];
#pragma unroll
    for (int x = 1; x < NX; ++x) m = fmaxf(m, v[x]);
    const int e = exponent_of(m);
    const float sc = pow2i(-e);
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      v[x] *= sc;
      if (DB) g[x] *= sc;
    }
    e2 += e;
  }
  float sv = 0.f, sg = 0.f;
#pragma unroll
  for (int x = 0; x < NX; ++x) {
    sv += v[x];
    sg += g[x];
  }
  lnz = (double)logf(sv) + (double)e2 * 0.69314718055994530942;
  dl = DB ? sg / sv : 0.f;
}

__device__ __forceinline__ int padded_row_bytes(int D) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return 4 * w4;
}

// Stage the tile's spins [T][D] (int8) into shared memory rows of Dp bytes.
__device__ void stage_spins(const int8_t* __restrict__ g, int n_valid, int D, int Dp, int8_t* s,
                            int t, int T) {
  for (int e = t; e < n_valid * D; e += T) s[(e / D) * Dp + (e % D)] = g[e];
}

template <bool DB>
__global__ void __launch_bounds__(128) strips_kernel(const InstDev* __restrict__ inst,
                                                     const LaunchInfo li,
                                                     const int8_t* __restrict__ spins,
                                                     double* __restrict__ logZR,
                                                     double* __restrict__ dbeta) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 0) return;  // another contraction kernel owns this instance
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_row_bytes(D);
  build_strip_tables(I, beta, sm, t, T);
  int8_t* ssp = reinterpret_cast<int8_t*>(sm + I.strip_tab_floats);
  const int n_valid = min(T, li.batch - b0);
  stage_spins(spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, D, Dp, ssp, t, T);
  __syncthreads();
  if (b >= li.batch) return;
  const int8_t* srow = ssp + t * Dp;
  double lz = 0.0, dl = 0.0, chat = 0.0;
  for (int st = 0; st < I.n_strips; ++st) {
    const StripDev& sd = I.strips[st];
    const float* tab = sm + sd.tab_off;
    double l = 0.0;
    float d = 0.f;
    switch (sd.w) {
      case 1: strip_chain<1, DB>(tab, sd.L, srow, l, d); break;
      case 2: strip_chain<2, DB>(tab, sd.L, srow, l, d); break;
      case 3: strip_chain<3, DB>(tab, sd.L, srow, l, d); break;
      default: strip_chain<4, DB>(tab, sd.L, srow, l, d); break;
    }
    lz += l;
    dl += d;
    chat += sd.c_hat;
  }
  // W-W bonds: -beta E_1(s) = beta sum J s_a s_b.
  float e1 = 0.f;
  for (int e = 0; e < I.n_ww; ++e) {
    const EdgeWW q = I.ww[e];
    e1 = fmaf(q.J, (float)(srow[q.a] * srow[q.b]), e1);
  }
  const double bd = li.beta[k];
  if (logZR) logZR[(long long)k * li.batch + b] = lz + bd * (chat + (double)e1);
  if (DB) dbeta[(long long)k * li.batch + b] = dl + chat + (double)e1;
}

int strip_smem_bytes(const Instance& in, int tile) {
  int D = (int)in.W.size();
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return in.dev.strip_tab_floats * 4 + tile * 4 * w4;
}

cudaError_t launch_strips(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                          const int8_t* spins, double* logZR, double* dbeta, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e;
  if (dbeta) {
    e = cudaFuncSetAttribute(strips_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    strips_kernel<true><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, spins, logZR, dbeta);
  } else {
    e = cudaFuncSetAttribute(strips_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    strips_kernel<false><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, spins, logZR, dbeta);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reverse mode: d ln Z_strip / d J_e = beta <s_i s_j> (bonds inside the strip)
// or beta s_W <s_i> (bonds to a W neighbour), from stored left vectors and a
// backward sweep of right vectors.  Accumulates (beta / batch) * value into
// dJ[edge] (batch mean), one atomic per bond per warp.
// ---------------------------------------------------------------------------
#define STRIP_DJ_LMAX 64

// Warp-sum a bond contribution and add it to the CTA's shared accumulator.
__device__ __forceinline__ void acc_bond(float* acc, int e, float val, bool lane0) {
  const float s = warp_sum(val);
  if (lane0 && e >= 0) atomicAdd(acc + e, s);
}

template <int W>
__device__ void strip_dJ(const float* tab, const StripRow* __restrict__ rows, int L,
                         const int8_t* srow, bool valid, float scale, float* dJ, bool lane0) {
  constexpr int NX = 1 << W;
  const float4* vert = reinterpret_cast<const float4*>(tab);
  const float* diag = tab + L * W * 4;
  const int* pos = reinterpret_cast<const int*>(diag + 2 * L * 4 * NX);
  float lv[STRIP_DJ_LMAX][NX];
  float v[NX], dummy[NX];
  for (int y = 0; y < L; ++y) {
    const float* dy = diag + (y * 4 + row_index(pos, y, srow)) * NX;
    if (y == 0) {
#pragma unroll
      for (int x = 0; x < NX; ++x) v[x] = dy[x];
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) apply_pair<W, false>(v, dummy, c, vert[(y - 1) * W + c]);
#pragma unroll
      for (int x = 0; x < NX; ++x) v[x] *= dy[x];
    }
    float m = v[0];
#pragma unroll
    for (int x = 1; x < NX; ++x) m = fmaxf(m, v[x]);
    const float sc = pow2i(-exponent_of(m));
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      v[x] *= sc;
      lv[y][x] = v[x];
    }
  }
  float r[NX];  // r_{y+1}
  for (int y = L - 1; y >= 0; --y) {
    float msg[NX];
    if (y == L - 1) {
#pragma unroll
      for (int x = 0; x < NX; ++x) msg[x] = 1.f;
    } else {
#pragma unroll
      for (int x = 0; x < NX; ++x) msg[x] = r[x];
#pragma unroll
      for (int c = 0; c < W; ++c) apply_pair<W, false>(msg, dummy, c, vert[y * W + c]);
    }
    float Z = 0.f, P[NX];
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      P[x] = lv[y][x] * msg[x];
      Z += P[x];
    }
    const float iz = valid ? scale / Z : 0.f;
    const StripRow& R = rows[y];
#pragma unroll
    for (int c = 0; c + 1 < W; ++c) {
      float a = 0.f;
#pragma unroll
      for (int x = 0; x < NX; ++x) a += P[x] * spin_of(x, c) * spin_of(x, c + 1);
      acc_bond(dJ, R.eh[c], a * iz, lane0);
    }
    if (R.posL >= 0) {
      float a = 0.f;
#pragma unroll
      for (int x = 0; x < NX; ++x) a += P[x] * spin_of(x, 0);
      acc_bond(dJ, R.eL, a * iz * (float)srow[R.posL], lane0);
    }
    if (R.posR >= 0) {
      float a = 0.f;
#pragma unroll
      for (int x = 0; x < NX; ++x) a += P[x] * spin_of(x, W - 1);
      acc_bond(dJ, R.eR, a * iz * (float)srow[R.posR], lane0);
    }
    if (y + 1 < L) {
#pragma unroll
      for (int c = 0; c < W; ++c) {
        float u[NX];
#pragma unroll
        for (int x = 0; x < NX; ++x) u[x] = r[x];
#pragma unroll
        for (int c2 = 0; c2 < W; ++c2) {
          float4 q = vert[y * W + c2];
          if (c2 == c) q = make_float4(q.x, -q.y, q.z, -q.w);
          apply_pair<W, false>(u, dummy, c2, q);
        }
        float a = 0.f;
#pragma unroll
        for (int x = 0; x < NX; ++x) a += lv[y][x] * u[x];
        acc_bond(dJ, R.ev[c], a * iz, lane0);
      }
    }
    // r_y = D_y * msg, renormalised
    const float* dy = diag + (y * 4 + row_index(pos, y, srow)) * NX;
    float m = 0.f;
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      r[x] = dy[x] * msg[x];
      m = fmaxf(m, r[x]);
    }
    const float sc = pow2i(-exponent_of(m));
#pragma unroll
    for (int x = 0; x < NX; ++x) r[x] *= sc;
  }
}

// One CTA per tile of samples: bond sums accumulate in shared memory (FP32,
// n_edges floats), then the CTA writes its row of `part` [CTA][max edges];
// strips_dJ_reduce_kernel adds the rows of each instance in a fixed order.
__global__ void __launch_bounds__(128) strips_dJ_kernel(const InstDev* __restrict__ inst,
                                                        const LaunchInfo li,
                                                        const int8_t* __restrict__ spins,
                                                        float* __restrict__ part, int part_stride) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_row_bytes(D);
  build_strip_tables(I, beta, sm, t, T);
  int8_t* ssp = reinterpret_cast<int8_t*>(sm + I.strip_tab_floats);
  float* acc = reinterpret_cast<float*>(ssp + T * Dp);  // [n_edges]
  for (int e = t; e < I.n_edges; e += T) acc[e] = 0.f;
  const int n_valid = min(T, li.batch - b0);
  stage_spins(spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, D, Dp, ssp, t, T);
  for (int e = n_valid * Dp + t; e < T * Dp; e += T) ssp[e] = 1;  // padding rows
  __syncthreads();
  const bool valid = b < li.batch;
  const int8_t* srow = ssp + t * Dp;
  const float scale = beta / (float)li.batch;
  const bool lane0 = (t & 31) == 0;
  for (int st = 0; st < I.n_strips; ++st) {
    const StripDev& sd = I.strips[st];
    const float* tab = sm + sd.tab_off;
    const StripRow* rows = I.rows + sd.row0;
    switch (sd.w) {
      case 1: strip_dJ<1>(tab, rows, sd.L, srow, valid, scale, acc, lane0); break;
      case 2: strip_dJ<2>(tab, rows, sd.L, srow, valid, scale, acc, lane0); break;
      case 3: strip_dJ<3>(tab, rows, sd.L, srow, valid, scale, acc, lane0); break;
      default: strip_dJ<4>(tab, rows, sd.L, srow, valid, scale, acc, lane0); break;
    }
  }
  __syncthreads();
  float* row = part + (long long)blockIdx.x * part_stride;
  for (int e = t; e < I.n_edges; e += T) row[e] = acc[e];
}

// dJ[edge] += sum over the instance's CTA rows, in CTA order (deterministic).
__global__ void strips_dJ_reduce_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                        const float* __restrict__ part, int part_stride,
                                        double* __restrict__ dJ) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.n_edges; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = li.tile_begin[k]; c < li.tile_begin[k + 1]; ++c) s += (double)part[(long long)c * part_stride + e];
    dJ[I.edge_off + e] += s;
  }
}

cudaError_t launch_strips_dJ(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                             const int8_t* spins, float* part, int part_stride, double* dJ, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(strips_dJ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes);
  if (e != cudaSuccess) return e;
  strips_dJ_kernel<<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, spins, part, part_stride);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  strips_dJ_reduce_kernel<<<dim3(4, li.n_inst), 256, 0, s>>>(d_inst, li, part, part_stride, dJ);
  return cudaGetLastError();
}

// W-W bonds: d(-beta E_1)/d J_e = beta s_a s_b, batch mean.  One CTA per
// (instance, bond chunk); threads stride over samples.
__global__ void ww_dJ_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                             const int8_t* __restrict__ spins, double* __restrict__ dJ) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  const int8_t* sp = spins + I.spin_units * li.batch;
  __shared__ int red[32];
  for (int e = blockIdx.x; e < I.n_ww; e += gridDim.x) {
    const EdgeWW q = I.ww[e];
    int acc = 0;
    for (int b = threadIdx.x; b < li.batch; b += blockDim.x)
      acc += sp[(long long)b * I.D + q.a] * sp[(long long)b * I.D + q.b];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      int v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0;
      v = warp_sum(v);
      if (threadIdx.x == 0) dJ[I.edge_off + q.e] += li.beta[k] * (double)v / (double)li.batch;
    }
    __syncthreads();
  }
}

cudaError_t launch_ww(const InstDev* d_inst, const LaunchInfo& li, const int8_t* spins,
                      double* dJ, cudaStream_t s) {
  if (li.n_inst == 0 || li.batch == 0) return cudaSuccess;
  ww_dJ_kernel<<<dim3(64, li.n_inst), 256, 0, s>>>(d_inst, li, spins, dJ);
  return cudaGetLastError();
}

}  // namespace tnvan
