// General leftover components (e.g. random regular graphs): exact
// contraction of every connected component of R by variable elimination
// (Eq. 4), one program per component compiled by the host planner.
//
// Eliminating spin v multiplies every factor that contains v -- its field
// factor exp(beta h_v(s) r_v) from the width set, the Boltzmann matrices of its
// remaining bonds (Eq. 2) and the intermediate tables that contain it -- and
// sums v out, giving a table over its remaining neighbours (at most 2^8
// entries).  Tables live in a per-sample arena in shared memory, laid out
// [entry][sample] so that the threads of a warp (one sample each) touch
// consecutive words; the forward passes run the program with reused offsets
// (a table's space is free once the step that consumes it has run), the
// reverse sweep keeps every table.  Every new table is renormalised by a power of two.
// Factors are stored normalised (largest entry 1); the removed constants
// (beta |h_v| per field, beta |J| per bond) are added back in FP64.
// With DB, every table entry carries its beta-derivative (forward mode).
#include <algorithm>

#include "common.cuh"

namespace tnvan {

__device__ __forceinline__ int padded_bytes(int D) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return 4 * w4;
}

// One component's program (starting at its header P[ip]) for this thread's
// spin row s: adds its log Z_c (and with DB its beta-derivative) to lz / dl
// and returns the offset just past the program.
template <bool DB>
__device__ __forceinline__ int run_component(const GenDev& G, const int* P, int ip, const int8_t* s, float* A,
                                             float* dA, const float4* pt, int T, int t, float beta, double& lz,
                                             double& dl) {
  const int nsteps = P[ip], fin = P[ip + 2];
  ip += 3;
  for (int st = 0; st < nsteps; ++st) {
    const int fb = P[ip + 1], fc = P[ip + 2], m = P[ip + 3], out = P[ip + 4];
    const int nin = P[ip + 5], npair = P[ip + 6];
    ip += 7;
    const int in0 = ip;
    int q = ip;
    for (int i = 0; i < nin; ++i) q += 2 + P[q + 1];
    const int pq = q;
    ip = q + 2 * npair;
    float h = 0.f;
    for (int f = fb; f < fb + fc; ++f) h = fmaf(G.fldJ[f], (float)s[G.fld[2 * f]], h);
    const float ah = fabsf(h);
    lz += (double)beta * (double)ah;
    if (DB) dl += (double)ah;
    const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
    const float fr[2] = {h - ah, -h - ah};
    float mx = 0.f;
    for (int x = 0; x < (1 << m); ++x) {
      float acc = 0.f, dacc = 0.f;
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        float p = fv[sg], r = fr[sg];
        const int ext = x | (sg << m);
        for (int j = 0; j < npair; ++j) {
          const float4 ab = pt[P[pq + 2 * j]];
          const bool same = ((x >> P[pq + 2 * j + 1]) & 1) == sg;
          p *= same ? ab.x : ab.y;
          r += same ? ab.z : ab.w;
        }
        int qq = in0;
        for (int i = 0; i < nin; ++i) {
          const int off = P[qq], kk = P[qq + 1];
          int idx = 0;
          for (int j = 0; j < kk; ++j) idx |= ((ext >> P[qq + 2 + j]) & 1) << j;
          const float val = A[(off + idx) * T + t];
          p *= val;
          if (DB) r += dA[(off + idx) * T + t] / val;
          qq += 2 + kk;
        }
        acc += p;
        if (DB) dacc = fmaf(p, r, dacc);
      }
      A[(out + x) * T + t] = acc;
      if (DB) dA[(out + x) * T + t] = dacc;
      mx = fmaxf(mx, acc);
    }
    const int e = exponent_of(mx);
    const float sc = pow2i(-e);
    for (int x = 0; x < (1 << m); ++x) {
      A[(out + x) * T + t] *= sc;
      if (DB) dA[(out + x) * T + t] *= sc;
    }
    lz += (double)e * 0.69314718055994530942;
  }
  const float z = A[fin * T + t];
  lz += (double)logf(z);
  if (DB) dl += (double)(dA[fin * T + t] / z);
  return ip;
}

// Boundary index of component c for spin row s: bit j set iff its j-th
// width-set neighbour (ctab boundary list) is -1.
__device__ __forceinline__ int boundary_index(const GenDev& G, const int* cr, const int8_t* s) {
  int idx = 0;
  for (int j = 0; j < cr[2]; ++j) idx |= (s[G.bpos[cr[3] + j]] < 0 ? 1 : 0) << j;
  return idx;
}

template <bool DB>
__global__ void __launch_bounds__(64) general_kernel(const InstDev* __restrict__ inst,
                                                     const LaunchInfo li, int arena_floats,
                                                     int max_pairs,
                                                     const int8_t* __restrict__ spins,
                                                     double* __restrict__ logZR,
                                                     double* __restrict__ dbeta, float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  // tables [arena][T] (and their beta-derivatives) in shared memory, or for
  // large arenas in this CTA's slice of a global scratch buffer
  const size_t cta_floats = (size_t)arena_floats * T * (DB ? 2 : 1);
  float* A = garena ? garena + (size_t)blockIdx.x * cta_floats : sm;
  float* dA = A + arena_floats * T;
  float4* pt = reinterpret_cast<float4*>(garena ? sm : sm + cta_floats);  // [pairs]
  int8_t* ssp = reinterpret_cast<int8_t*>(pt + max_pairs);
  const GenDev& G = I.gen;
  for (int p = t; p < G.n_pairs; p += T) {
    const float J = G.pairJ[p], aj = fabsf(J);
    const float tt = expf(-2.f * beta * aj);
    // (a, b, d ln a / d beta, d ln b / d beta) of [[a,b],[b,a]] = e^{-beta|J|} B
    pt[p] = J >= 0.f ? make_float4(1.f, tt, 0.f, -2.f * aj) : make_float4(tt, 1.f, -2.f * aj, 0.f);
  }
  const int n_valid = min(T, li.batch - b0);
  const int8_t* gsp = spins + I.spin_units * li.batch + (long long)b0 * D;
  for (int e = t; e < n_valid * D; e += T) ssp[(e / D) * Dp + (e % D)] = gsp[e];
  __syncthreads();
  if (b >= li.batch) return;
  const int8_t* s = ssp + t * Dp;
  const int* P = G.prog_fwd;
  const bool tab = li.gen_tab && G.n_tab > 0 && G.n_tab <= li.batch;  // tables built for this call
  double lz = 0.0, dl = 0.0;
  const int ncomp = P[0];
  int ip = 1;
  for (int c = 0; c < ncomp; ++c) {
    const int* cr = G.ctab + 5 * c;
    if (tab && cr[4] >= 0) {  // a tabulated component: one lookup
      const int x = boundary_index(G, cr, s);
      lz += G.tab_lz[cr[4] + x];
      if (DB) dl += G.tab_db[cr[4] + x];
      ip = cr[1];
    } else {
      ip = run_component<DB>(G, P, ip, s, A, dA, pt, T, t, beta, lz, dl);
    }
  }
  float e1 = 0.f;
  for (int e = 0; e < I.n_ww; ++e) {
    const EdgeWW q = I.ww[e];
    e1 = fmaf(q.J, (float)(s[q.a] * s[q.b]), e1);
  }
  const double chf = G.c_hat;
  const long long o = (long long)k * li.batch + b;
  if (logZR) logZR[o] = lz + li.beta[k] * (chf + (double)e1);
  if (DB) dbeta[o] = dl + chf + (double)e1;
}

// The tables of the tabulated components (at most TNVAN_TAB_MAX_K width-set
// neighbours, f1 of the build's next rows): thread g of instance k takes
// entry g of the concatenated tables, i.e. one component c and one boundary
// configuration x, sets the boundary spins of a spin row from the bits of x
// (the other spins do not enter c) and runs c's program alone, so that
// tab_lz[toff_c + x] = log Z_c and tab_db[..] its beta-derivative.  Built
// per call (they depend on beta) when they are smaller than the batch.
template <bool DB>
__global__ void __launch_bounds__(64) general_tab_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                         int arena_floats, int max_pairs,
                                                         float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const GenDev& G = I.gen;
  if (G.n_tab == 0 || G.n_tab > li.batch) return;
  const int T = blockDim.x, t = threadIdx.x;
  const int g = blockIdx.x * T + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  const size_t cta_floats = (size_t)arena_floats * T * (DB ? 2 : 1);
  float* A = garena ? garena + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * cta_floats : sm;
  float* dA = A + arena_floats * T;
  float4* pt = reinterpret_cast<float4*>(garena ? sm : sm + cta_floats);
  int8_t* ssp = reinterpret_cast<int8_t*>(pt + max_pairs);
  for (int p = t; p < G.n_pairs; p += T) {
    const float J = G.pairJ[p], aj = fabsf(J);
    const float tt = expf(-2.f * beta * aj);
    pt[p] = J >= 0.f ? make_float4(1.f, tt, 0.f, -2.f * aj) : make_float4(tt, 1.f, -2.f * aj, 0.f);
  }
  int8_t* s = ssp + t * Dp;
  for (int j = 0; j < D; ++j) s[j] = 1;
  __syncthreads();
  if (blockIdx.x * T >= G.n_tab || g >= G.n_tab) return;
  // which tabulated component and configuration
  int c = -1, x = 0;
  for (int j = 0; j < G.n_tabc; ++j) {
    const int* cr = G.ctab + 5 * G.tabc[j];
    if (g >= cr[4] && g < cr[4] + (1 << cr[2])) {
      c = G.tabc[j];
      x = g - cr[4];
      break;
    }
  }
  if (c < 0) return;
  const int* cr = G.ctab + 5 * c;
  for (int j = 0; j < cr[2]; ++j) s[G.bpos[cr[3] + j]] = ((x >> j) & 1) ? -1 : 1;
  double lz = 0.0, dl = 0.0;
  run_component<DB>(G, G.prog_fwd, cr[0], s, A, dA, pt, T, t, beta, lz, dl);
  G.tab_lz[g] = lz;
  if (DB) G.tab_db[g] = dl;
}

// ---------------------------------------------------------------------------
// Reverse mode: d ln Z_c / d J_e for the bonds inside a component (beta <r r'>)
// and its bonds to the width set (beta s_w <r>).  Per component the program
// runs forward storing every (renormalised) table A_t and its scale 2^-e_t;
// then the steps run backwards carrying adjoints Abar = d ln Z / d A of each
// table entry, starting from 1 / A_final.  For step t with product terms
// term(x, sigma) (field factor, bond factors, input tables):
//   g(x, sigma)       = Abar_t[x] 2^-e_t term(x, sigma)
//   Abar_in[idx]     += g / A_in[idx]
//   d lnZ / d J_bond += beta sum g sigma sigma_u,  d lnZ / d J_field += beta s_w sum g sigma.
// Bond sums are warp-reduced into per-CTA shared accumulators, written as one
// row per CTA and added per instance in a fixed order.
// ---------------------------------------------------------------------------
// (blocks of fewer than 32 threads -- large tables -- have one partial warp:
// no shuffles there, every thread adds its own term)
__device__ __forceinline__ void acc_edge(float* acc, int e, float v, bool lane0) {
  if (blockDim.x >= 32) {
    v = warp_sum(v);
    if (lane0 && e >= 0) atomicAdd(acc + e, v);
  } else if (e >= 0) {
    atomicAdd(acc + e, v);
  }
}

__global__ void __launch_bounds__(64) general_dJ_kernel(const InstDev* __restrict__ inst,
                                                        const LaunchInfo li, int arena_floats,
                                                        int max_pairs, int max_steps,
                                                        const int8_t* __restrict__ spins,
                                                        float* __restrict__ part, int part_stride,
                                                        float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  // tables, adjoints and scales in shared memory, or for large arenas in this
  // CTA's slice of a global scratch buffer
  const size_t cta_floats = (size_t)(2 * arena_floats + max_steps) * T;
  float* A = garena ? garena + (size_t)blockIdx.x * cta_floats : sm;  // [arena][T]
  float* Ab = A + arena_floats * T;       // [arena][T] adjoints
  float* sc = Ab + arena_floats * T;      // [max_steps][T] scales 2^-e
  float2* pt = reinterpret_cast<float2*>(garena ? sm : sm + cta_floats);  // [pairs] (a, b)
  float* acc = reinterpret_cast<float*>(pt + max_pairs);       // [n_edges]
  int8_t* ssp = reinterpret_cast<int8_t*>(acc + ((I.n_edges + 3) & ~3));
  const GenDev& G = I.gen;
  for (int p = t; p < G.n_pairs; p += T) {
    const float J = G.pairJ[p], tt = expf(-2.f * beta * fabsf(J));
    pt[p] = J >= 0.f ? make_float2(1.f, tt) : make_float2(tt, 1.f);
  }
  for (int e = t; e < I.n_edges; e += T) acc[e] = 0.f;
  const int n_valid = min(T, li.batch - b0);
  const int8_t* gsp = spins + I.spin_units * li.batch + (long long)b0 * D;
  for (int e = t; e < n_valid * D; e += T) ssp[(e / D) * Dp + (e % D)] = gsp[e];
  for (int e = n_valid * Dp + t; e < T * Dp; e += T) ssp[e] = 1;
  __syncthreads();
  const bool valid = b < li.batch;
  const bool lane0 = (t & 31) == 0;
  const int8_t* s = ssp + t * Dp;
  const float wscale = valid ? beta / (float)li.batch : 0.f;
  const int* P = G.prog;
  int ip = 1;
  for (int c = 0; c < G.n_comp; ++c) {
    const int nsteps = P[ip], arena = P[ip + 1], fin = P[ip + 2];
    ip += 3;
    const int st0 = G.comp_step0[c];
    // forward: tables and their scales
    for (int st = 0; st < nsteps; ++st) {
      const int r = G.step_off[st0 + st];
      const int fb = P[r + 1], fc = P[r + 2], m = P[r + 3], out = P[r + 4], nin = P[r + 5], npair = P[r + 6];
      int q = r + 7;
      const int in0 = q;
      for (int i = 0; i < nin; ++i) q += 2 + P[q + 1];
      const int pq = q;
      float h = 0.f;
      for (int f = fb; f < fb + fc; ++f) h = fmaf(G.fldJ[f], (float)s[G.fld[2 * f]], h);
      const float ah = fabsf(h);
      const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
      float mx = 0.f;
      for (int x = 0; x < (1 << m); ++x) {
        float accv = 0.f;
        for (int sg = 0; sg < 2; ++sg) {
          float pr = fv[sg];
          const int ext = x | (sg << m);
          for (int j = 0; j < npair; ++j) {
            const float2 ab = pt[P[pq + 2 * j]];
            pr *= (((x >> P[pq + 2 * j + 1]) & 1) == sg) ? ab.x : ab.y;
          }
          int qq = in0;
          for (int i = 0; i < nin; ++i) {
            const int off = P[qq], kk = P[qq + 1];
            int idx = 0;
            for (int j = 0; j < kk; ++j) idx |= ((ext >> P[qq + 2 + j]) & 1) << j;
            pr *= A[(off + idx) * T + t];
            qq += 2 + kk;
          }
          accv += pr;
        }
        A[(out + x) * T + t] = accv;
        Ab[(out + x) * T + t] = 0.f;
        mx = fmaxf(mx, accv);
      }
      const float scl = pow2i(-exponent_of(mx));
      for (int x = 0; x < (1 << m); ++x) A[(out + x) * T + t] *= scl;
      sc[st * T + t] = scl;
    }
    (void)arena;
    Ab[fin * T + t] = 1.f / A[fin * T + t];
    // backward
    for (int st = nsteps - 1; st >= 0; --st) {
      const int r = G.step_off[st0 + st];
      const int fb = P[r + 1], fc = P[r + 2], m = P[r + 3], out = P[r + 4], nin = P[r + 5], npair = P[r + 6];
      int q = r + 7;
      const int in0 = q;
      for (int i = 0; i < nin; ++i) q += 2 + P[q + 1];
      const int pq = q;
      float h = 0.f;
      for (int f = fb; f < fb + fc; ++f) h = fmaf(G.fldJ[f], (float)s[G.fld[2 * f]], h);
      const float ah = fabsf(h);
      const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
      const float scl = sc[st * T + t];
      float gs = 0.f;       // sum g sigma_v
      float gp[8];          // sum g sigma_v sigma_u per pair (at most 8 neighbours)
      for (int j = 0; j < 8; ++j) gp[j] = 0.f;
      for (int x = 0; x < (1 << m); ++x) {
        const float abx = Ab[(out + x) * T + t] * scl;
        for (int sg = 0; sg < 2; ++sg) {
          float pr = fv[sg];
          const int ext = x | (sg << m);
          for (int j = 0; j < npair; ++j) {
            const float2 ab = pt[P[pq + 2 * j]];
            pr *= (((x >> P[pq + 2 * j + 1]) & 1) == sg) ? ab.x : ab.y;
          }
          int qq = in0;
          for (int i = 0; i < nin; ++i) {
            const int off = P[qq], kk = P[qq + 1];
            int idx = 0;
            for (int j = 0; j < kk; ++j) idx |= ((ext >> P[qq + 2 + j]) & 1) << j;
            pr *= A[(off + idx) * T + t];
            qq += 2 + kk;
          }
          const float g = abx * pr;
          const float sv = sg ? -1.f : 1.f;
          gs = fmaf(g, sv, gs);
          for (int j = 0; j < npair && j < 8; ++j)
            gp[j] = fmaf(g, ((((x >> P[pq + 2 * j + 1]) & 1) == sg) ? 1.f : -1.f), gp[j]);
          qq = in0;
          for (int i = 0; i < nin; ++i) {
            const int off = P[qq], kk = P[qq + 1];
            int idx = 0;
            for (int j = 0; j < kk; ++j) idx |= ((ext >> P[qq + 2 + j]) & 1) << j;
            const float a = A[(off + idx) * T + t];
            if (a > 0.f) Ab[(off + idx) * T + t] += g / a;
            qq += 2 + kk;
          }
        }
      }
      for (int f = fb; f < fb + fc; ++f)
        acc_edge(acc, G.fld[2 * f + 1], wscale * gs * (float)s[G.fld[2 * f]], lane0);
      for (int j = 0; j < npair && j < 8; ++j) acc_edge(acc, G.pairE[P[pq + 2 * j]], wscale * gp[j], lane0);
    }
    ip = G.step_off[st0 + nsteps - 1];
    {
      // advance ip past the last step record of this component
      const int r = ip;
      int q = r + 7;
      for (int i = 0; i < P[r + 5]; ++i) q += 2 + P[q + 1];
      ip = q + 2 * P[r + 6];
    }
  }
  __syncthreads();
  float* row = part + (long long)blockIdx.x * part_stride;
  for (int e = t; e < I.n_edges; e += T) row[e] = acc[e];
}

__global__ void general_dJ_reduce_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                         const float* __restrict__ part, int part_stride,
                                         double* __restrict__ dJ) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.n_edges; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = li.tile_begin[k]; c < li.tile_begin[k + 1]; ++c) s += (double)part[(long long)c * part_stride + e];
    dJ[I.edge_off + e] += s;
  }
}

int general_dJ_smem_bytes(int arena, int pairs, int steps, int D, int n_edges, int T, bool glob) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return (glob ? 0 : (2 * arena + steps) * T * 4) + pairs * 8 + ((n_edges + 3) & ~3) * 4 + T * 4 * w4;
}

size_t general_dJ_scratch_floats(int arena, int steps, int T, int nblk) {
  return (size_t)(2 * arena + steps) * T * nblk;
}

cudaError_t launch_general_dJ(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int arena,
                              int pairs, int steps, const int8_t* spins, float* part, int part_stride,
                              double* dJ, float* garena, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(general_dJ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  general_dJ_kernel<<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, steps, spins, part, part_stride,
                                                      garena);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  general_dJ_reduce_kernel<<<dim3(4, li.n_inst), 256, 0, s>>>(d_inst, li, part, part_stride, dJ);
  return cudaGetLastError();
}

// The components' tables at this call's betas (li.gen_tab: the largest
// table; general_kernel then looks them up).
cudaError_t launch_general_tables(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, bool db,
                                  float* garena, cudaStream_t s) {
  if (li.gen_tab <= 0) return cudaSuccess;
  const int arena = (int)(li.seed & 0xffffffffull), pairs = (int)(li.seed >> 32);
  const dim3 tg((unsigned)((li.gen_tab + li.tile - 1) / li.tile), li.n_inst);
  cudaError_t e;
  if (db) {
    e = cudaFuncSetAttribute(general_tab_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_tab_kernel<true><<<tg, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, garena);
  } else {
    e = cudaFuncSetAttribute(general_tab_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_tab_kernel<false><<<tg, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, garena);
  }
  return cudaGetLastError();
}

int general_smem_bytes(int arena, int pairs, int D, int T, bool db, bool glob) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return (glob ? 0 : arena * T * 4 * (db ? 2 : 1)) + pairs * 16 + T * 4 * w4;
}

// Scratch of the global-table mode: one [arena][T] slice (two with d/dbeta)
// per CTA of the contraction and of the tables kernel.
size_t general_scratch_floats(const LaunchInfo& li, int arena, bool db) {
  const size_t per = (size_t)arena * li.tile * (db ? 2 : 1);
  size_t ctas = (size_t)li.tile_begin[li.n_inst];
  if (li.gen_tab > 0) ctas = std::max(ctas, (size_t)((li.gen_tab + li.tile - 1) / li.tile) * li.n_inst);
  return per * ctas;
}

cudaError_t launch_general(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                           const int8_t* spins, double* logZR, double* dbeta, float* garena,
                           cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  // li.seed carries (arena floats, max pairs) for this launch
  const int arena = (int)(li.seed & 0xffffffffull), pairs = (int)(li.seed >> 32);
  cudaError_t e;
  if (dbeta) {
    e = cudaFuncSetAttribute(general_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<true><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, spins, logZR, dbeta, garena);
  } else {
    e = cudaFuncSetAttribute(general_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<false><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, spins, logZR, dbeta,
                                                            garena);
  }
  return cudaGetLastError();
}

}  // namespace tnvan
