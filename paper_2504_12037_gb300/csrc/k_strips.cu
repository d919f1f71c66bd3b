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
// beta * c_hat is added back in FP64 at the end.  The planner hands over the
// strip in a gauge where every vertical coupling is >= 0 (spins flipped
// column by column, the horizontal and W-neighbour couplings carrying the
// signs), so every normalised vertical factor is [[1, t], [t, 1]] with
// t = e^{-2 beta |J|}; bond expectations come back to the model's spins
// through the per-edge sign (I.edge_sign).
#include "common.cuh"

namespace tnvan {

// Per-strip table layout in shared memory (floats, offset tab_off):
//   vert  [L][w] float4 (1, t, 0, dt/dbeta): 2x2 factor [[1,t],[t,1]]
//   diag  [L][4][2^w]   D_y for the 4 combinations of (s_L, s_R) signs
//   ddiag [L][4][2^w]   d D_y / d beta
//   pos   [L][2] int    AR positions of the left / right W neighbours (-1 none)
// The adjoint kernel stores the same tables without ddiag, strip after strip.
__host__ __device__ inline int strip_tab_floats(int w, int L) {
  int n = L * w * 4 + 2 * L * 4 * (1 << w) + 2 * L;
  return (n + 3) & ~3;
}
// The adjoint's tables carry no ddiag.
__host__ __device__ inline int strip_tab_floats_adj(int w, int L) {
  int n = L * w * 4 + L * 4 * (1 << w) + 2 * L;
  return (n + 3) & ~3;
}

struct StripTab {
  const float4* vert;
  const float* diag;
  const float* ddiag;  // nullptr in the adjoint's layout
  const int* pos;
};

__device__ __forceinline__ StripTab strip_tab_at(const float* tab, int w, int L, bool with_ddiag) {
  StripTab s;
  const int nd = L * 4 * (1 << w);
  s.vert = reinterpret_cast<const float4*>(tab);
  s.diag = tab + L * w * 4;
  s.ddiag = with_ddiag ? s.diag + nd : nullptr;
  s.pos = reinterpret_cast<const int*>(s.diag + (with_ddiag ? 2 * nd : nd));
  return s;
}

// Float offset of strip st's tables: the host-planned offset, or (adjoint
// layout) the running sum of strip_tab_floats_adj over the earlier strips.
__device__ __forceinline__ int strip_tab_offset(const InstDev& I, int st, bool with_ddiag) {
  if (with_ddiag) return I.strips[st].tab_off;
  int off = 0;
  for (int j = 0; j < st; ++j) off += strip_tab_floats_adj(I.strips[j].w, I.strips[j].L);
  return off;
}

__device__ __forceinline__ float spin_of(int x, int c) { return ((x >> c) & 1) ? -1.f : 1.f; }

__device__ void build_strip_tables(const InstDev& I, float beta, float* sm, int t, int T, bool with_ddiag = true) {
  for (int st = 0; st < I.n_strips; ++st) {
    const StripDev sd = I.strips[st];
    const int w = sd.w, L = sd.L;
    float* tab = sm + strip_tab_offset(I, st, with_ddiag);
    const StripTab tb = strip_tab_at(tab, w, L, with_ddiag);
    float4* vert = const_cast<float4*>(tb.vert);
    float* diag = const_cast<float*>(tb.diag);
    float* ddiag = const_cast<float*>(tb.ddiag);
    int* pos = const_cast<int*>(tb.pos);
    const StripRow* rows = I.rows + sd.row0;
    const int nx = 1 << w;
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
      if (ddiag) ddiag[e] = d * (ex - ch);
    }
    for (int e = t; e < L * w; e += T) {
      const int y = e / w, c = e % w;
      const float aj = rows[y].Jv[c];  // >= 0 in the planner's gauge
      const float tt = (y + 1 < L) ? expf(-2.f * beta * aj) : 1.f;
      const float dt = -2.f * aj * tt;
      vert[e] = make_float4(1.f, tt, 0.f, dt);
    }
    for (int y = t; y < L; y += T) {
      pos[2 * y] = rows[y].posL;
      pos[2 * y + 1] = rows[y].posR;
    }
  }
}

// The adjoint's tables of instance I (built by strips_tab_kernel for this
// launch's beta) into shared memory: n floats, a multiple of 4.
__device__ __forceinline__ void copy_strip_tables(const InstDev& I, float* sm, int n, int t, int T) {
  const float4* src = reinterpret_cast<const float4*>(I.adj_tab);
  float4* dst = reinterpret_cast<float4*>(sm);
  for (int e = t; e < n / 4; e += T) dst[e] = __ldg(src + e);
}

// One CTA per instance of [k0, k1): the adjoint's strip tables at the
// instance's beta, into I.adj_tab (the layout the adjoint kernels use).
__global__ void strips_tab_kernel(const InstDev* __restrict__ inst, const LaunchInfo li, int k0) {
  const int k = blockIdx.x + k0;
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  build_strip_tables(I, (float)li.beta[k], I.adj_tab, threadIdx.x, blockDim.x, false);
}

cudaError_t launch_strip_tables(const InstDev* d_inst, const LaunchInfo& li, int k0, int k1, cudaStream_t s) {
  if (k1 <= k0) return cudaSuccess;
  strips_tab_kernel<<<k1 - k0, 256, 0, s>>>(d_inst, li, k0);
  return cudaGetLastError();
}

// Apply [[1,t],[t,1]] (t = q.y) on bit c of the state index, and its
// beta-derivative (dt/dbeta = q.w).
template <int W, bool DB>
__device__ __forceinline__ void apply_pair(float (&v)[1 << W], float (&g)[1 << W], int c, float4 q) {
#pragma unroll
  for (int x = 0; x < (1 << W); ++x) {
    if ((x >> c) & 1) continue;
    const int x1 = x | (1 << c);
    const float v0 = v[x], v1 = v[x1];
    if (DB) {
      const float g0 = g[x], g1 = g[x1];
      g[x] = fmaf(q.y, g1, fmaf(q.w, v1, g0));
      g[x1] = fmaf(q.y, g0, fmaf(q.w, v0, g1));
    }
    v[x] = fmaf(q.y, v1, v0);
    v[x1] = fmaf(q.y, v0, v1);
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
// With SAVE, the renormalised left vector of every even row y is also
// written to lvs[((y / 2) * 2^W + x) * T + t] (the adjoint's backward sweep
// reads it and recomputes the odd rows from it).
template <int W, bool DB, bool SAVE = false>
__device__ void strip_chain(const StripTab& tb, int L, const int8_t* srow, double& lnz, float& dl,
                            float* lvs = nullptr, int t = 0, int T = 0) {
  constexpr int NX = 1 << W;
  const float4* vert = tb.vert;
  const float* diag = tb.diag;
  const float* ddiag = tb.ddiag;
  const int* pos = tb.pos;
  float v[NX], g[NX];
  int e2 = 0;
  for (int y = 0; y < L; ++y) {
    const int idx = row_index(pos, y, srow);
    const float* dy = diag + (y * 4 + idx) * NX;
    const float* gy = DB ? ddiag + (y * 4 + idx) * NX : dy;
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
      if (SAVE && !(y & 1)) lvs[((y >> 1) * NX + x) * T + t] = v[x];
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
    const StripTab tb = strip_tab_at(sm + sd.tab_off, sd.w, sd.L, true);
    double l = 0.0;
    float d = 0.f;
    switch (sd.w) {
      case 1: strip_chain<1, DB>(tb, sd.L, srow, l, d); break;
      case 2: strip_chain<2, DB>(tb, sd.L, srow, l, d); break;
      case 3: strip_chain<3, DB>(tb, sd.L, srow, l, d); break;
      default: strip_chain<4, DB>(tb, sd.L, srow, l, d); break;
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
// Strip adjoint, fused.  For every sample, one forward sweep (the chain of
// strips_kernel) keeps each row's renormalised left vector in shared
// memory; one backward sweep of right vectors then gives every bond's local
// expectation:
//   d ln Z_strip / d J_e = beta <s_i s_j>   (bonds inside the strip)
//                        = beta s_W <s_i>   (bonds to a W neighbour),
// and the W-W bonds add d(-beta E_1)/d J_e = beta s_a s_b (Eq. 4
// differentiated), and d log Z_R / d beta = sum_e J_e <.>_e - E_1(s) per
// sample; optionally log Z_R itself (the forward sweep's value, as
// strips_kernel computes it).  Batch sums are formed per CTA in shared memory, one row
// of accumulators per warp so that the order of additions is fixed, and
// strips_dJ_reduce_kernel adds the CTA rows in CTA order.
// ---------------------------------------------------------------------------

// Sum NV per-lane values (NV a power of two, at most 32) over the warp by a
// transpose reduction: NV - 1 exchanges halve the values each lane holds,
// then log2(32 / NV) exchanges finish the sums.  On return the lanes with
// lane % (32 / NV) == 0 each hold the warp total of value number `idx`.
template <int NV>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[NV], int lane, int& idx) {
  idx = 0;
#pragma unroll
  for (int h = NV / 2, m = 16; h >= 1; h >>= 1, m >>= 1) {
    const bool up = (lane & m) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? v[j] : v[j + h];
      const float keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
    if (up) idx += h;
  }
  float s = v[0];
#pragma unroll
  for (int m = 16 / NV; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  return s;
}

// Edge id of bond slot j of a strip row: W-1 horizontal, left, right, W vertical.
__device__ __forceinline__ int row_edge(const StripRow& R, int W, int j) {
  if (j < W - 1) return R.eh[j];
  if (j == W - 1) return R.eL;
  if (j == W) return R.eR;
  return R.ev[j - W - 1];
}

// Bond slot whose warp total this lane holds after warp_transpose_sum<NV>
// (a function of the lane only).
template <int NV>
__device__ __forceinline__ int transpose_slot(int lane) {
  int idx = 0;
#pragma unroll
  for (int h = NV / 2, m = 16; h >= 1; h >>= 1, m >>= 1)
    if (lane & m) idx += h;
  return idx;
}

// Backward sweep of one strip for one sample (all 32 lanes of the warp take
// part; the sample's bond values enter the sums times wv: 1, a caller's
// weight, or 0 for padding samples).  Adds each
// bond's local expectation to the warp's accumulators and returns
// d ln Z_strip / d beta = sum_e J_e <.>_e: every Boltzmann weight depends on
// beta only through beta J_e, so the same expectations give the beta
// derivative.
//
// Row y, with left vector l (rows 0..y, D_y included) and right vector
// r = r_{y+1}: the message m = V_y r, P = l * m, Z = sum P; the horizontal
// and W-neighbour bonds are signed sums of P.  For the vertical bond of
// column c, with L_c = V_0..V_{c-1} l and R_c = V_{c+1}..V_{W-1} r and the
// factor on bit c being I + t X,
//   Z = L_c^T R_c + t L_c^T X R_c,  Z <s_c s'_c> = L_c^T R_c - t L_c^T X R_c,
// so Z <s_c s'_c> = 2 L_c^T R_c - Z, and the W vertical bonds share 2W - 1
// Kronecker-factor applications and one dot product each.  The row's bonds
// are read by slot (StripRow::Js, es), absent bonds carrying J = 0.  Only the
// even rows' left vectors are stored: an odd row's is recomputed from the
// row before it as D_y V_{y-1} l_{y-1}, without the renormalisation (a power
// of two that every ratio below cancels exactly), and that stored row is
// kept in registers for the next iteration.
template <int W>
__device__ float strip_backsweep(const StripTab& tb, const StripRow* __restrict__ rows, int L,
                                 const int8_t* srow, const float* lvs, int t, int T, float wv, float* accw,
                                 int lane) {
  constexpr int NX = 1 << W;
  constexpr int NB = 2 * W + 1;
  constexpr int NV = NB <= 4 ? 4 : (NB <= 8 ? 8 : 16);
  const float4* vert = tb.vert;
  const float* diag = tb.diag;
  const int* pos = tb.pos;
  const bool own = (lane & (32 / NV - 1)) == 0;
  const int slot = transpose_slot<NV>(lane);
  const bool has_slot = own && slot < NB;
  float r[NX];  // r_{y+1}, renormalised
  float lkeep[NX];  // l_{y} of an even row, loaded while recomputing row y + 1
  float dlog = 0.f;
  for (int y = L - 1; y >= 0; --y) {
    float Js[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) Js[j] = rows[y].Js[j];
    const int ecur = has_slot ? rows[y].es[slot] : -1;
    const int idx = row_index(pos, y, srow);
    float lv[NX], msg[NX], dummy[NX];
    if (y & 1) {
#pragma unroll
      for (int x = 0; x < NX; ++x) lkeep[x] = lvs[(((y - 1) >> 1) * NX + x) * T + t];
#pragma unroll
      for (int x = 0; x < NX; ++x) lv[x] = lkeep[x];
#pragma unroll
      for (int c = 0; c < W; ++c) apply_pair<W, false>(lv, dummy, c, vert[(y - 1) * W + c]);
      const float* dyl = diag + (y * 4 + idx) * NX;
#pragma unroll
      for (int x = 0; x < NX; ++x) lv[x] *= dyl[x];
    } else if (y == L - 1) {
#pragma unroll
      for (int x = 0; x < NX; ++x) lv[x] = lvs[((y >> 1) * NX + x) * T + t];
    } else {
#pragma unroll
      for (int x = 0; x < NX; ++x) lv[x] = lkeep[x];
    }
    float val[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) val[j] = 0.f;
    float d0[W];  // L_c^T R_c of the vertical bonds
    if (y == L - 1) {
#pragma unroll
      for (int x = 0; x < NX; ++x) msg[x] = 1.f;
    } else {
      float4 q[W];
#pragma unroll
      for (int c = 0; c < W; ++c) q[c] = vert[y * W + c];
      // suffix products R_c (R_{W-1} = r)
      float Rc[W][NX];
#pragma unroll
      for (int x = 0; x < NX; ++x) Rc[W - 1][x] = r[x];
#pragma unroll
      for (int c = W - 2; c >= 0; --c) {
#pragma unroll
        for (int x = 0; x < NX; ++x) Rc[c][x] = Rc[c + 1][x];
        apply_pair<W, false>(Rc[c], dummy, c + 1, q[c + 1]);
      }
#pragma unroll
      for (int x = 0; x < NX; ++x) msg[x] = Rc[0][x];
      apply_pair<W, false>(msg, dummy, 0, q[0]);
      // prefix products L_c (L_0 = l)
      float Lc[NX];
#pragma unroll
      for (int x = 0; x < NX; ++x) Lc[x] = lv[x];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (c > 0) apply_pair<W, false>(Lc, dummy, c - 1, q[c - 1]);
        float d = 0.f;
#pragma unroll
        for (int x = 0; x < NX; ++x) d = fmaf(Lc[x], Rc[c][x], d);
        d0[c] = d;
      }
    }
    float P[NX];
    float Z = 0.f;
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      P[x] = lv[x] * msg[x];
      Z = fmaf(lv[x], msg[x], Z);
    }
#pragma unroll
    for (int c = 0; c + 1 < W; ++c) {
      float a = 0.f;
#pragma unroll
      for (int x = 0; x < NX; ++x) a += P[x] * spin_of(x, c) * spin_of(x, c + 1);
      val[c] = a;
    }
    {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int x = 0; x < NX; ++x) {
        a += P[x] * spin_of(x, 0);
        b += P[x] * spin_of(x, W - 1);
      }
      val[W - 1] = (idx & 1) ? -a : a;  // s_L s_0
      val[W] = (idx & 2) ? -b : b;      // s_R s_{W-1}
    }
    if (y + 1 < L) {
#pragma unroll
      for (int c = 0; c < W; ++c) val[W + 1 + c] = fmaf(2.f, d0[c], -Z);
    }
    // the beta-weighted sum (absent bonds carry J = 0), then the masked
    // values for d/dJ
    const float iz = __fdividef(1.f, Z);  // Z is a normal number well inside the fast path's range
    float dJb = 0.f;
#pragma unroll
    for (int j = 0; j < NB; ++j) dJb = fmaf(Js[j], val[j], dJb);
    dlog = fmaf(dJb, iz, dlog);
    const float vz = wv * iz;
#pragma unroll
    for (int j = 0; j < NB; ++j) val[j] *= vz;
    int vi;
    const float sum = warp_transpose_sum<NV>(val, lane, vi);
    if (has_slot && ecur >= 0) accw[ecur] += sum;
    // r_y = D_y * msg, renormalised
    const float* dy = diag + (y * 4 + idx) * NX;
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
  return dlog;
}

// Shared memory of strips_adj_kernel: strip tables, the tile's spins, the
// left vectors of one strip's even rows [ceil(L/2)][2^w][T] and (T/32) rows of n_edges
// accumulators.
__host__ __device__ inline int strip_adj_lv_offset(int tab_floats, int T, int Dp) {
  return tab_floats + ((T * Dp + 15) & ~15) / 4;
}

// TT: samples per CTA (= li.tile), a compile-time constant so that the
// left-vector addressing folds into immediate offsets.
template <int TT>
__global__ void __launch_bounds__(128, 3) strips_adj_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                         int lv_floats, const int8_t* __restrict__ spins,
                                                         double* __restrict__ logZR, double* __restrict__ dbeta,
                                                         float* __restrict__ part, int part_stride) {
  extern __shared__ float sm[];
  const int gblk = blockIdx.x + li.blk0;
  const int k = find_inst(li, gblk);
  const InstDev& I = inst[k];
  if (I.kind != 0) return;  // another adjoint kernel owns this instance
  constexpr int T = TT;
  const int t = threadIdx.x, lane = t & 31;
  const int b0 = (gblk - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_row_bytes(D);
  const int tabn = strip_tab_offset(I, I.n_strips, false);
  copy_strip_tables(I, sm, tabn, t, T);
  int8_t* ssp = reinterpret_cast<int8_t*>(sm + tabn);
  float* lvs = sm + strip_adj_lv_offset(tabn, T, Dp);
  float* acc = lvs + lv_floats;
  const int ne = I.n_edges;
  for (int e = t; e < (T >> 5) * ne; e += T) acc[e] = 0.f;
  const int n_valid = min(T, li.batch - b0);
  stage_spins(spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, D, Dp, ssp, t, T);
  for (int e = n_valid * Dp + t; e < T * Dp; e += T) ssp[e] = 1;  // padding rows
  __syncthreads();
  const bool valid = b < li.batch;
  // the backward sweep only when d/dbeta or the bond sums are wanted
  const bool back = dbeta != nullptr || part != nullptr;
  // this sample's weight in the bond sums: 1, or the caller's multiplier
  // (importance weights of tnvan_observables); 0 for padding samples
  const float wv = !valid ? 0.f : (li.wmul ? li.wmul[(long long)k * li.batch + b] : 1.f);
  const int8_t* srow = ssp + t * Dp;
  float* accw = acc + (t >> 5) * ne;
  double dl = 0.0, lz = 0.0, chat = 0.0;
  for (int st = 0, off = 0; st < I.n_strips; ++st) {
    const StripDev& sd = I.strips[st];
    const StripTab tab = strip_tab_at(sm + off, sd.w, sd.L, false);
    off += strip_tab_floats_adj(sd.w, sd.L);
    const StripRow* rows = I.rows + sd.row0;
    double l = 0.0;
    float d = 0.f;
    if (!back) {  // log Z_R only: the forward chain, no left vectors kept
      switch (sd.w) {
        case 1: strip_chain<1, false>(tab, sd.L, srow, l, d); break;
        case 2: strip_chain<2, false>(tab, sd.L, srow, l, d); break;
        case 3: strip_chain<3, false>(tab, sd.L, srow, l, d); break;
        default: strip_chain<4, false>(tab, sd.L, srow, l, d); break;
      }
    } else {
      switch (sd.w) {
        case 1:
          strip_chain<1, false, true>(tab, sd.L, srow, l, d, lvs, t, T);
          d = strip_backsweep<1>(tab, rows, sd.L, srow, lvs, t, T, wv, accw, lane);
          break;
        case 2:
          strip_chain<2, false, true>(tab, sd.L, srow, l, d, lvs, t, T);
          d = strip_backsweep<2>(tab, rows, sd.L, srow, lvs, t, T, wv, accw, lane);
          break;
        case 3:
          strip_chain<3, false, true>(tab, sd.L, srow, l, d, lvs, t, T);
          d = strip_backsweep<3>(tab, rows, sd.L, srow, lvs, t, T, wv, accw, lane);
          break;
        default:
          strip_chain<4, false, true>(tab, sd.L, srow, l, d, lvs, t, T);
          d = strip_backsweep<4>(tab, rows, sd.L, srow, lvs, t, T, wv, accw, lane);
          break;
      }
    }
    dl += d;
    lz += l;
    chat += sd.c_hat;
  }
  // W-W bonds: -beta E_1 for log Z_R and d/dbeta, s_a s_b for d/dJ (eight bonds per warp reduction)
  float e1 = 0.f;
  for (int e0 = 0; e0 < I.n_ww; e0 += 8) {
    float val[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      val[j] = 0.f;
      if (e0 + j < I.n_ww) {
        const EdgeWW q = I.ww[e0 + j];
        const float ss = (float)(srow[q.a] * srow[q.b]);
        e1 = fmaf(q.J, ss, e1);
        val[j] = ss * wv;
      }
    }
    int vi;
    const float sum = warp_transpose_sum<8>(val, lane, vi);
    if ((lane & 3) == 0 && e0 + vi < I.n_ww) accw[I.ww[e0 + vi].e] += sum;
  }
  if (dbeta && valid) dbeta[(long long)k * li.batch + b] = dl + (double)e1;
  if (logZR && valid) logZR[(long long)k * li.batch + b] = lz + li.beta[k] * (chat + (double)e1);
  __syncthreads();
  if (!part) return;  // d/dbeta only: no bond sums wanted
  const float scale = beta / (float)li.batch;
  float* row = part + (long long)gblk * part_stride;
  for (int e = t; e < ne; e += T) {
    float s = 0.f;
    for (int w = 0; w < (T >> 5); ++w) s += acc[w * ne + e];
    row[e] = s * scale;
  }
}

// The same pass with one warp per strip (at most 8 strips): a CTA takes 32 samples, warp st
// contracts strip st for all of them (thread = (strip, sample)), so a CTA
// lasts one strip's sweeps instead of all strips' -- a short CTA that fills
// the tail of a launch and the gaps beside other kernels.  log Z_R and d/dbeta
// are assembled by warp 0 from the per-strip partials in strip order (the same
// arithmetic as strips_adj_kernel); W-W bond chunks are spread over the warps.
// Shared memory: tables | spins | even-row left vectors [ceil(L/2)][2^w][blockDim] | one row
// of n_edges accumulators per warp | per-(strip, sample) partials.
__global__ void __launch_bounds__(256) strips_adj_ws_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                             int lv_floats, const int8_t* __restrict__ spins,
                                                             double* __restrict__ logZR, double* __restrict__ dbeta,
                                                             float* __restrict__ part, int part_stride) {
  extern __shared__ float sm[];
  const int gblk = blockIdx.x + li.blk0;
  const int k = find_inst(li, gblk);
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  const int NT = blockDim.x, NW = NT >> 5, tid = threadIdx.x, lane = tid & 31, st = tid >> 5;
  const int b0 = (gblk - li.tile_begin[k]) * 32, b = b0 + lane;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_row_bytes(D);
  const int tabn = strip_tab_offset(I, I.n_strips, false);
  copy_strip_tables(I, sm, tabn, tid, NT);
  int8_t* ssp = reinterpret_cast<int8_t*>(sm + tabn);
  float* lvs = sm + strip_adj_lv_offset(tabn, 32, Dp);
  float* acc = lvs + lv_floats;
  const int ne = I.n_edges;
  double* pl = reinterpret_cast<double*>(acc + ((NW * ne + 1) & ~1));
  float* pd = reinterpret_cast<float*>(pl + NW * 32);
  for (int e = tid; e < NW * ne; e += NT) acc[e] = 0.f;
  const int n_valid = min(32, li.batch - b0);
  stage_spins(spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, D, Dp, ssp, tid, NT);
  for (int e = n_valid * Dp + tid; e < 32 * Dp; e += NT) ssp[e] = 1;  // padding rows
  __syncthreads();
  const bool valid = b < li.batch;
  // the backward sweep only when d/dbeta or the bond sums are wanted
  const bool back = dbeta != nullptr || part != nullptr;
  // this sample's weight in the bond sums: 1, or the caller's multiplier
  // (importance weights of tnvan_observables); 0 for padding samples
  const float wv = !valid ? 0.f : (li.wmul ? li.wmul[(long long)k * li.batch + b] : 1.f);
  const int8_t* srow = ssp + lane * Dp;
  float* accw = acc + st * ne;
  if (st < I.n_strips) {
    const StripDev& sd = I.strips[st];
    const StripTab tab = strip_tab_at(sm + strip_tab_offset(I, st, false), sd.w, sd.L, false);
    const StripRow* rows = I.rows + sd.row0;
    double l = 0.0;
    float d = 0.f;
    if (!back) {  // log Z_R only: the forward chain, no left vectors kept
      switch (sd.w) {
        case 1: strip_chain<1, false>(tab, sd.L, srow, l, d); break;
        case 2: strip_chain<2, false>(tab, sd.L, srow, l, d); break;
        case 3: strip_chain<3, false>(tab, sd.L, srow, l, d); break;
        default: strip_chain<4, false>(tab, sd.L, srow, l, d); break;
      }
    } else {
      switch (sd.w) {
        case 1:
          strip_chain<1, false, true>(tab, sd.L, srow, l, d, lvs, tid, NT);
          d = strip_backsweep<1>(tab, rows, sd.L, srow, lvs, tid, NT, wv, accw, lane);
          break;
        case 2:
          strip_chain<2, false, true>(tab, sd.L, srow, l, d, lvs, tid, NT);
          d = strip_backsweep<2>(tab, rows, sd.L, srow, lvs, tid, NT, wv, accw, lane);
          break;
        case 3:
          strip_chain<3, false, true>(tab, sd.L, srow, l, d, lvs, tid, NT);
          d = strip_backsweep<3>(tab, rows, sd.L, srow, lvs, tid, NT, wv, accw, lane);
          break;
        default:
          strip_chain<4, false, true>(tab, sd.L, srow, l, d, lvs, tid, NT);
          d = strip_backsweep<4>(tab, rows, sd.L, srow, lvs, tid, NT, wv, accw, lane);
          break;
      }
    }
    pl[st * 32 + lane] = l;
    pd[st * 32 + lane] = d;
  }
  // W-W bonds for d/dJ: chunks of eight bonds, one warp per chunk
  for (int e0 = st * 8; e0 < I.n_ww; e0 += NW * 8) {
    float val[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      val[j] = 0.f;
      if (valid && e0 + j < I.n_ww) {
        const EdgeWW q = I.ww[e0 + j];
        val[j] = (float)(srow[q.a] * srow[q.b]) * wv;
      }
    }
    int vi;
    const float sum = warp_transpose_sum<8>(val, lane, vi);
    if ((lane & 3) == 0 && e0 + vi < I.n_ww) accw[I.ww[e0 + vi].e] += sum;
  }
  __syncthreads();
  if (st == 0 && valid) {  // strips in order, then -beta E_1 (as strips_adj_kernel)
    double dl = 0.0, lz = 0.0, chat = 0.0;
    for (int j = 0; j < I.n_strips; ++j) {
      dl += pd[j * 32 + lane];
      lz += pl[j * 32 + lane];
      chat += I.strips[j].c_hat;
    }
    float e1 = 0.f;
    for (int e = 0; e < I.n_ww; ++e) {
      const EdgeWW q = I.ww[e];
      e1 = fmaf(q.J, (float)(srow[q.a] * srow[q.b]), e1);
    }
    if (dbeta) dbeta[(long long)k * li.batch + b] = dl + (double)e1;
    if (logZR) logZR[(long long)k * li.batch + b] = lz + li.beta[k] * (chat + (double)e1);
  }
  if (!part) return;  // d/dbeta only: no bond sums wanted
  const float scale = beta / (float)li.batch;
  float* row = part + (long long)gblk * part_stride;
  for (int e = tid; e < ne; e += NT) {
    float s = 0.f;
    for (int w = 0; w < NW; ++w) s += acc[w * ne + e];
    row[e] = s * scale;
  }
}

// dJ[edge] (+)= sum over the instance's CTA rows: one warp per edge, lane l
// adding rows l, l+32, ... in FP64, then a fixed xor tree (deterministic).
// With `assign` the sum overwrites dJ (every edge of a strip instance has a
// column in the rows, W-W bonds included).
__global__ void strips_dJ_reduce_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                        const float* __restrict__ part, int part_stride,
                                        double* __restrict__ dJ, bool assign) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (e >= I.n_edges) return;
  double s = 0.0;
  for (int c = li.tile_begin[k] + lane; c < li.tile_begin[k + 1]; c += 32) s += (double)part[(long long)c * part_stride + e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double v = (double)I.edge_sign[e] * s;
    dJ[I.edge_off + e] = assign ? v : dJ[I.edge_off + e] + v;
  }
}

int strip_adj_lv_floats(const Instance& in, int tile) {
  int lv = 0;
  for (const StripDev& sd : in.strip.strips) lv = std::max(lv, ((sd.L + 1) / 2) << sd.w);  // even rows
  return lv * tile;
}

// lv_floats: the launch-wide left-vector region (the maximum over instances)
int strip_adj_smem_bytes(const Instance& in, int tile, int lv_floats) {
  const int D = (int)in.W.size();
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  int tabn = 0;
  for (const StripDev& sd : in.strip.strips) tabn += strip_tab_floats_adj(sd.w, sd.L);
  return 4 * strip_adj_lv_offset(tabn, tile, 4 * w4) + 4 * lv_floats + 4 * (tile / 32) * in.m;
}

// Warp-per-strip variant: threads per CTA (32 x the most strips of an
// instance), left-vector floats per launch and shared memory per instance.
int strip_adj_ws_threads(const tnvan_ctx* ctx) {
  int nw = 0;
  for (const Instance& in : ctx->inst)
    if (in.kind == 0) nw = std::max(nw, (int)in.strip.strips.size());
  return 32 * nw;
}
int strip_adj_ws_lv_floats(const Instance& in, int threads) {
  int lv = 0;
  for (const StripDev& sd : in.strip.strips) lv = std::max(lv, ((sd.L + 1) / 2) << sd.w);  // even rows
  return lv * threads;
}
int strip_adj_ws_smem_bytes(const Instance& in, int threads, int lv_floats) {
  const int D = (int)in.W.size();
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  int tabn = 0;
  for (const StripDev& sd : in.strip.strips) tabn += strip_tab_floats_adj(sd.w, sd.L);
  const int nw = threads / 32;
  return 4 * strip_adj_lv_offset(tabn, 32, 4 * w4) + 4 * lv_floats + 4 * ((nw * in.m + 1) & ~1) + 12 * nw * 32;
}
int strips_adj_ws_occupancy(int threads, int smem_bytes) {
  if (cudaFuncSetAttribute(strips_adj_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, strips_adj_ws_kernel, threads, smem_bytes) != cudaSuccess)
    return 0;
  return nb;
}

// The instance of strips_adj_kernel for `tile` samples per CTA (nullptr if none).
static void (*strips_adj_for(int tile))(const InstDev*, const LaunchInfo, int, const int8_t*, double*, double*, float*,
                                        int) {
  switch (tile) {
    case 32: return strips_adj_kernel<32>;
    case 64: return strips_adj_kernel<64>;
    case 96: return strips_adj_kernel<96>;
    case 128: return strips_adj_kernel<128>;
    default: return nullptr;
  }
}

// CTAs of `tile` threads with `smem_bytes` of shared memory resident per SM.
int strips_adj_occupancy(int tile, int smem_bytes) {
  auto kern = strips_adj_for(tile);
  if (!kern || cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, tile, smem_bytes) != cudaSuccess) return 0;
  return nb;
}

// Blocks [blk_begin, blk_end) of the launch (blk_end < 0: all, followed by
// the d/dJ reduction when dJ is given; a partial launch leaves the reduction
// to launch_strips_dJ_reduce once every block has run).
cudaError_t launch_strips_adj(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int lv_floats,
                              const int8_t* spins, double* logZR, double* dbeta, float* part, int part_stride,
                              double* dJ, cudaStream_t s, int blk_begin, int blk_end, int ws_threads) {
  const bool whole = blk_end < 0;
  if (whole) blk_end = li.tile_begin[li.n_inst];
  const int nblk = blk_end - blk_begin;
  if (nblk <= 0) return cudaSuccess;
  LaunchInfo lc = li;
  lc.blk0 = blk_begin;
  cudaError_t e;
  if (ws_threads > 0) {
    if (li.tile != 32 || ws_threads % 32 != 0 || ws_threads > 256) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(strips_adj_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    strips_adj_ws_kernel<<<nblk, ws_threads, smem_bytes, s>>>(d_inst, lc, lv_floats, spins, logZR, dbeta, part,
                                                              part_stride);
  } else {
    auto kern = strips_adj_for(li.tile);
    if (!kern) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<nblk, li.tile, smem_bytes, s>>>(d_inst, lc, lv_floats, spins, logZR, dbeta, part, part_stride);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !dJ || !whole) return e;
  return launch_strips_dJ_reduce(d_inst, li, part, part_stride, dJ, s, false);
}

cudaError_t launch_strips_dJ_reduce(const InstDev* d_inst, const LaunchInfo& li, const float* part, int part_stride,
                                    double* dJ, cudaStream_t s, bool assign) {
  strips_dJ_reduce_kernel<<<dim3((unsigned)((part_stride + 7) / 8), li.n_inst), 256, 0, s>>>(d_inst, li, part,
                                                                                            part_stride, dJ, assign);
  return cudaGetLastError();
}

// W-W bonds of dense and elimination instances: d(-beta E_1)/d J_e =
// beta s_a s_b, batch mean (with li.wmul, each sample b weighted by
// wmul[b]).  One CTA per (instance, bond chunk); threads stride over samples;
// the sums are exact integers, or FP64 in a fixed order when weighted.
__global__ void ww_dJ_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                             const int8_t* __restrict__ spins, double* __restrict__ dJ) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind == 0) return;  // strips_adj_kernel covers the W-W bonds of strip instances
  const int8_t* sp = spins + I.spin_units * li.batch;
  const float* wm = li.wmul ? li.wmul + (long long)k * li.batch : nullptr;
  __shared__ double red[32];
  for (int e = blockIdx.x; e < I.n_ww; e += gridDim.x) {
    const EdgeWW q = I.ww[e];
    double acc = 0.0;
    if (wm) {
      for (int b = threadIdx.x; b < li.batch; b += blockDim.x)
        acc += (double)wm[b] * (double)(sp[(long long)b * I.D + q.a] * sp[(long long)b * I.D + q.b]);
    } else {
      int ia = 0;
      for (int b = threadIdx.x; b < li.batch; b += blockDim.x)
        ia += sp[(long long)b * I.D + q.a] * sp[(long long)b * I.D + q.b];
      acc = (double)ia;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0) dJ[I.edge_off + q.e] += li.beta[k] * v / (double)li.batch;
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

// ---------------------------------------------------------------------------
// Magnetisation moments of the strips (observables from samples, Sec. 3).
// For one sample, the conditional mean and variance of M_strip = sum of the
// strip's model spins given the width set, by the row chain in the moment
// form: each state x of the current row carries the chain's weight v(x) and
// the mean mu(x) and variance q(x) of the rows' magnetisation so far given
// that the current row is in x.  A vertical factor I + t X on bit c mixes x
// with x ^ (1 << c) at weight t (moment_mix), the diagonal D_y scales v and adds the
// row's magnetisation to mu (q unchanged: it is fixed given x), and the end
// sums the states the same way.  Model spin = tau * strip spin (the planner's
// gauge): the row's magnetisation of state x is w - 2 popc((x ^ tau_mask) & (2^w - 1)).
// ---------------------------------------------------------------------------
template <int W>
__device__ void strip_moments(const StripTab& tb, const StripRow* __restrict__ rows, int L, const int8_t* srow,
                              float& mean, float& var) {
  constexpr int NX = 1 << W;
  float v[NX], mu[NX], q[NX];
  for (int y = 0; y < L; ++y) {
    const int idx = row_index(tb.pos, y, srow);
    const float* dy = tb.diag + (y * 4 + idx) * NX;
    const int tm = rows[y].tau_mask;
    if (y > 0) {
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float t = tb.vert[(y - 1) * W + c].y;
#pragma unroll
        for (int x = 0; x < NX; ++x) {
          if ((x >> c) & 1) continue;
          const int x1 = x | (1 << c);
          const float v0 = v[x], m0 = mu[x], q0 = q[x], v1 = v[x1], m1 = mu[x1], q1 = q[x1];
          moment_mix(v0, m0, q0, t * v1, m1, q1, v[x], mu[x], q[x]);
          moment_mix(v1, m1, q1, t * v0, m0, q0, v[x1], mu[x1], q[x1]);
        }
      }
    }
    float mx = 0.f;
#pragma unroll
    for (int x = 0; x < NX; ++x) {
      const float a = (float)(W - 2 * __popc((x ^ tm) & (NX - 1)));
      if (y == 0) {
        v[x] = dy[x];
        mu[x] = a;
        q[x] = 0.f;
      } else {
        v[x] *= dy[x];
        mu[x] += a;
      }
      mx = fmaxf(mx, v[x]);
    }
    const float sc = pow2i(-exponent_of(mx));
#pragma unroll
    for (int x = 0; x < NX; ++x) v[x] *= sc;
  }
  float Z = 0.f, m = 0.f;
#pragma unroll
  for (int x = 0; x < NX; ++x) Z += v[x];
#pragma unroll
  for (int x = 0; x < NX; ++x) m = fmaf(v[x] / Z, mu[x], m);
  float qq = 0.f;
#pragma unroll
  for (int x = 0; x < NX; ++x) {
    const float d = mu[x] - m;
    qq = fmaf(v[x] / Z, fmaf(d, d, q[x]), qq);
  }
  mean = m;
  var = qq;
}

// One thread per sample: E[M | s] = M_W(s) + sum over strips of the strip
// means, Var(M | s) = sum of the strip variances (the strips are independent
// given the width set), both FP64 sums of the FP32 per-strip values.
__global__ void __launch_bounds__(128) strips_mom_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                         const int8_t* __restrict__ spins,
                                                         double* __restrict__ mag_mean, double* __restrict__ mag_var) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 0) return;
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const int D = I.D, Dp = padded_row_bytes(D);
  build_strip_tables(I, (float)li.beta[k], sm, t, T, false);  // tables without ddiag (adjoint layout)
  int8_t* ssp = reinterpret_cast<int8_t*>(sm + I.strip_tab_floats);
  const int n_valid = min(T, li.batch - b0);
  stage_spins(spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, D, Dp, ssp, t, T);
  __syncthreads();
  if (b >= li.batch) return;
  const int8_t* srow = ssp + t * Dp;
  int mw = 0;
  for (int j = 0; j < D; ++j) mw += srow[j];
  double mean = (double)mw, var = 0.0;
  for (int st = 0; st < I.n_strips; ++st) {
    const StripDev& sd = I.strips[st];
    const StripTab tb = strip_tab_at(sm + strip_tab_offset(I, st, false), sd.w, sd.L, false);
    const StripRow* rows = I.rows + sd.row0;
    float m = 0.f, q = 0.f;
    switch (sd.w) {
      case 1: strip_moments<1>(tb, rows, sd.L, srow, m, q); break;
      case 2: strip_moments<2>(tb, rows, sd.L, srow, m, q); break;
      case 3: strip_moments<3>(tb, rows, sd.L, srow, m, q); break;
      default: strip_moments<4>(tb, rows, sd.L, srow, m, q); break;
    }
    mean += (double)m;
    var += (double)q;
  }
  const long long o = (long long)k * li.batch + b;
  mag_mean[o] = mean;
  mag_var[o] = var;
}

cudaError_t launch_strips_mom(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, const int8_t* spins,
                              double* mag_mean, double* mag_var, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(strips_mom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  strips_mom_kernel<<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, spins, mag_mean, mag_var);
  return cudaGetLastError();
}

}  // namespace tnvan
