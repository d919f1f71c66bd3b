// General leftover components (e.g. random regular graphs): exact
// contraction of every connected component of R by variable elimination
// (Eq. 4), one program per component compiled by the host planner.
//
// Eliminating spin v multiplies every factor that contains v -- its field
// factor exp(beta h_v(s) r_v) from the width set, the Boltzmann matrices of its
// remaining bonds (Eq. 2) and the intermediate tables that contain it -- and
// sums v out, giving a table over its remaining neighbours (at most
// 2^TNVAN_MAX_ELIM_W entries).  The host compiles each step into a record and, per input table,
// an index map from the step's extended index (its out-scope spins and v) to
// the input's entry; the product of a step's bond factors depends only on
// that index and beta and is tabulated once per call (general_pp_kernel), so
// a table entry costs one field factor, one bond product and one load per
// input.  A group of lanes shares one sample and splits each table's entries;
// tables are laid out [entry][sample] per CTA (consecutive samples in
// consecutive words), in shared memory, or for large arenas in a per-CTA
// slice of global scratch.  Forward
// passes use reused offsets (a table's space is free once the step that
// consumes it has run); the reverse sweep keeps every table.  Every new table
// is renormalised by a power of two.  Factors are stored normalised (largest
// entry 1); the removed constants (beta |h_v| per field, beta |J| per bond)
// are added back in FP64.  With DB, every table entry carries its
// beta-derivative (forward mode).
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace tnvan {

__device__ __forceinline__ int padded_bytes(int D) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return 4 * w4;
}

// One compiled elimination step (layout in GenDev).
struct StepRec {
  int m, fb, fc, nin, npair, ppo, mo, out_live, out_full;
  const int* io;  // n_in x (live offset, full offset, spins of the input)
  const int* pr;  // n_pair x (pair id, position of the neighbour in the out scope)
};

__device__ __forceinline__ StepRec step_at(const GenDev& G, int g) {
  const int* F = G.fprog + G.fstep[g];
  StepRec r;
  r.m = F[0];
  r.fb = F[1];
  r.fc = F[2];
  r.nin = F[3];
  r.npair = F[4];
  r.ppo = F[5];
  r.mo = F[6];
  r.out_live = F[7];
  r.out_full = F[8];
  r.io = F + 9;
  r.pr = F + 9 + 3 * r.nin;
  return r;
}

// Width-set field on the eliminated spin: h = sum_w J_vw s_w.
__device__ __forceinline__ float field_of(const GenDev& G, int fb, int fc, const int8_t* s) {
  float h = 0.f;
  for (int f = fb; f < fb + fc; ++f) h = fmaf(G.fldJ[f], (float)s[G.fld[2 * f]], h);
  return h;
}

// Bond products of every step at this call's beta: one CTA per (step,
// instance), one thread per extended index.  A bond [[a,b],[b,a]] scaled by
// e^{-beta |J|} has entries 1 and e^{-2 beta |J|} (the latter where the two
// spins disagree for J >= 0, agree for J < 0).
__global__ void __launch_bounds__(256) general_pp_kernel(const InstDev* __restrict__ inst, const LaunchInfo li) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const GenDev& G = I.gen;
  const int g = blockIdx.x;
  if (g >= G.n_steps) return;
  const StepRec r = step_at(G, g);
  const int E = 2 << r.m;
  const float beta = (float)li.beta[k];
  for (int ext = threadIdx.x; ext < E; ext += blockDim.x) {
    const int x = ext & ((1 << r.m) - 1), sg = ext >> r.m;
    float p = 1.f, d = 0.f;
    for (int j = 0; j < r.npair; ++j) {
      const float J = G.pairJ[r.pr[2 * j]], aj = fabsf(J);
      const bool same = ((x >> r.pr[2 * j + 1]) & 1) == sg;
      if (same != (J >= 0.f)) {
        p *= expf(-2.f * beta * aj);
        d -= 2.f * aj;
      }
    }
    G.pp[r.ppo + ext] = p;
    G.pp[G.n_pp + r.ppo + ext] = d;
  }
}

// Lanes per sample: a group of GL consecutive lanes (a power of two, at most
// 32, so that a group lies inside one warp) shares one sample; lane l of the
// group computes the table entries x = l, l + GL, ...  Every lane of a block
// runs the same program (invalid samples run on a dummy row), so the
// group-wide maximum and __syncwarp between steps see full warps.
// Row stride of the [entry][sample] tables: S samples plus 32 / GL floats,
// so that the GL consecutive entries written by a group and the 32 / GL
// samples of a warp fall in 32 different shared-memory banks.
__host__ __device__ __forceinline__ int gen_row_stride(int S, int GL) { return S + 32 / GL; }

__device__ __forceinline__ float group_max(float v, int GL) {
  for (int o = GL >> 1; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Component c for the sample whose tables start at A (entry e at A[e * RS];
// with DB the beta-derivatives at dA[e * RS]); forward, live offsets.
// Adds log Z_c (and with DB its beta-derivative) to lz / dl on lane 0 of the
// group.
template <bool DB>
__device__ __forceinline__ void run_component(const GenDev& G, int c, const int8_t* s, float* A, float* dA, int RS,
                                              int lane, int GL, float beta, double& lz, double& dl) {
  const int* H = G.fprog + G.fhdr[c];
  const int nsteps = H[0], fin = H[1];
  const int g0 = G.comp_step0[c];
  // log-scale terms of the component: the power-of-two scales add up exactly
  // as an integer, the field offsets |h_v| in a compensated FP32 sum (Kahan),
  // both added to the FP64 result once per component
  int esum = 0;
  float hs = 0.f, hc = 0.f;
  for (int st = 0; st < nsteps; ++st) {
    const StepRec r = step_at(G, g0 + st);
    const float h = field_of(G, r.fb, r.fc, s);
    const float ah = fabsf(h);
    {
      const float y = ah - hc;
      const float t2 = hs + y;
      hc = (t2 - hs) - y;
      hs = t2;
    }
    const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
    const float fr[2] = {h - ah, -h - ah};
    const int M = 1 << r.m, E = 2 * M;
    const float* pp = G.pp + r.ppo;
    const float* pd = G.pp + G.n_pp + r.ppo;
    const unsigned short* mp = G.map + r.mo;
    const int out = r.out_live;
    float mx = 0.f;
    for (int x = lane; x < M; x += GL) {
      float acc = 0.f, dacc = 0.f;
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const int ext = x | (sg << r.m);
        float p = fv[sg] * pp[ext];
        float rr = DB ? fr[sg] + pd[ext] : 0.f;
        for (int i = 0; i < r.nin; ++i) {
          const int a = (r.io[3 * i] + mp[i * E + ext]) * RS;
          const float val = A[a];
          p *= val;
          if (DB) rr += dA[a] / val;
        }
        acc += p;
        if (DB) dacc = fmaf(p, rr, dacc);
      }
      A[(out + x) * RS] = acc;
      if (DB) dA[(out + x) * RS] = dacc;
      mx = fmaxf(mx, acc);
    }
    mx = group_max(mx, GL);
    const int e = exponent_of(mx);
    const float sc = pow2i(-e);
    for (int x = lane; x < M; x += GL) {
      A[(out + x) * RS] *= sc;
      if (DB) dA[(out + x) * RS] *= sc;
    }
    esum += e;
    __syncwarp();
  }
  if (lane == 0) {
    const double hsum = (double)hs - (double)hc;
    const float z = A[fin * RS];
    lz += (double)beta * hsum + (double)esum * 0.69314718055994530942 + (double)logf(z);
    if (DB) dl += hsum + (double)(dA[fin * RS] / z);
  }
}

// Boundary index of component c for spin row s: bit j set iff its j-th
// width-set neighbour (ctab boundary list) is -1.
__device__ __forceinline__ int boundary_index(const GenDev& G, const int* cr, const int8_t* s) {
  int idx = 0;
  for (int j = 0; j < cr[2]; ++j) idx |= (s[G.bpos[cr[3] + j]] < 0 ? 1 : 0) << j;
  return idx;
}

// Stage the spin rows of this CTA's samples in shared memory (rows of
// samples past the batch set to +1).
__device__ __forceinline__ void stage_spins(int8_t* ssp, const int8_t* gsp, int n_valid, int S, int D, int Dp) {
  for (int e = threadIdx.x; e < n_valid * D; e += blockDim.x) ssp[(e / D) * Dp + (e % D)] = gsp[e];
  for (int e = n_valid * Dp + threadIdx.x; e < S * Dp; e += blockDim.x) ssp[e] = 1;
}

// li.tile = samples per CTA (S); blockDim.x = S * GL.
template <bool DB>
__global__ void __launch_bounds__(128) general_kernel(const InstDev* __restrict__ inst,
                                                      const LaunchInfo li, int arena_floats, int GL,
                                                      const int8_t* __restrict__ spins,
                                                      double* __restrict__ logZR,
                                                      double* __restrict__ dbeta, float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int S = li.tile, slot = threadIdx.x / GL, lane = threadIdx.x % GL;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * S, b = b0 + slot;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  // tables [entry][sample] (rows of RS floats; then their beta-derivatives)
  // in shared memory, or for large arenas in this CTA's slice of a global
  // scratch buffer
  const int RS = gen_row_stride(S, GL);
  const size_t cta_floats = (size_t)arena_floats * RS * (DB ? 2 : 1);
  float* base = garena ? garena + (size_t)blockIdx.x * cta_floats : sm;
  float* A = base + slot;
  float* dA = A + (size_t)arena_floats * RS;
  int8_t* ssp = reinterpret_cast<int8_t*>(garena ? sm : sm + cta_floats);
  const GenDev& G = I.gen;
  const int n_valid = min(S, li.batch - b0);
  stage_spins(ssp, spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, S, D, Dp);
  __syncthreads();
  const int8_t* s = ssp + slot * Dp;
  const bool tab = li.gen_tab && G.n_tab > 0 && G.n_tab <= li.batch;  // tables built for this call
  double lz = 0.0, dl = 0.0;
  for (int c = 0; c < G.n_comp; ++c) {
    const int* cr = G.ctab + 5 * c;
    if (tab && cr[4] >= 0) {  // a tabulated component: one lookup
      const int x = boundary_index(G, cr, s);
      lz += G.tab_lz[cr[4] + x];
      if (DB) dl += G.tab_db[cr[4] + x];
    } else {
      run_component<DB>(G, c, s, A, dA, RS, lane, GL, beta, lz, dl);
    }
  }
  if (lane != 0 || b >= li.batch) return;
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
// neighbours): group g of instance k takes entry g of the concatenated
// tables, i.e. one component c and one boundary configuration x, sets the
// boundary spins of a spin row from the bits of x (the other spins do not
// enter c) and runs c's program alone, so that tab_lz[toff_c + x] = log Z_c
// and tab_db[..] its beta-derivative.  Built per call (they depend on beta)
// when they are smaller than the batch.
template <bool DB>
__global__ void __launch_bounds__(128) general_tab_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                          int arena_floats, int GL, float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const GenDev& G = I.gen;
  if (G.n_tab == 0 || G.n_tab > li.batch) return;
  const int S = li.tile, slot = threadIdx.x / GL, lane = threadIdx.x % GL;
  const int g = blockIdx.x * S + slot;
  if (blockIdx.x * S >= G.n_tab) return;  // whole CTA idle (uniform)
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  const int RS = gen_row_stride(S, GL);
  const size_t cta_floats = (size_t)arena_floats * RS * (DB ? 2 : 1);
  float* base = garena ? garena + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * cta_floats : sm;
  float* A = base + slot;
  float* dA = A + (size_t)arena_floats * RS;
  int8_t* ssp = reinterpret_cast<int8_t*>(garena ? sm : sm + cta_floats);
  int8_t* s = ssp + slot * Dp;
  for (int j = lane; j < D; j += GL) s[j] = 1;
  __syncwarp();
  // which tabulated component and configuration (entries past the tables
  // run the first tabulated component on the all-up row, unwritten)
  int c = -1, x = 0;
  for (int j = 0; j < G.n_tabc; ++j) {
    const int* cr = G.ctab + 5 * G.tabc[j];
    if (g >= cr[4] && g < cr[4] + (1 << cr[2])) {
      c = G.tabc[j];
      x = g - cr[4];
      break;
    }
  }
  const bool live = c >= 0;
  // every group of a warp must run the same component (shuffles, syncwarp):
  // the components of one warp's entries may differ, so a warp walks the
  // distinct components of its groups in turn
  const unsigned wmask = 0xffffffffu;
  int cc = live ? c : G.tabc[0];
  __syncwarp();
  for (;;) {
    // the smallest component index still to run in this warp
    int want = cc;
    for (int o = 16; o > 0; o >>= 1) want = min(want, __shfl_xor_sync(wmask, want, o));
    if (want == INT_MAX) break;
    const bool mine = cc == want;
    const int* cr = G.ctab + 5 * want;
    if (mine && live && lane == 0)
      for (int j = 0; j < cr[2]; ++j) s[G.bpos[cr[3] + j]] = ((x >> j) & 1) ? -1 : 1;
    __syncwarp();
    double lz = 0.0, dl = 0.0;
    run_component<DB>(G, want, s, A, dA, RS, lane, GL, beta, lz, dl);
    if (mine && live && lane == 0) {
      G.tab_lz[g] = lz;
      if (DB) G.tab_db[g] = dl;
    }
    if (mine) cc = INT_MAX;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Reverse mode: d ln Z_c / d J_e for the bonds inside a component (beta <r r'>)
// and its bonds to the width set (beta s_w <r>).  Per component the steps run
// forward storing every (renormalised) table A_t and its scale 2^-e_t (full
// offsets); then backwards carrying adjoints Abar = d ln Z / d A of each table
// entry, starting from 1 / A_final.  For step t with product terms
// term(x, sigma) (field factor, bond factors, input tables):
//   g(x, sigma)       = Abar_t[x] 2^-e_t term(x, sigma)
//   Abar_in[idx]     += g / A_in[idx]
//   d lnZ / d J_bond += beta sum g sigma sigma_u,  d lnZ / d J_field += beta s_w sum g sigma.
// The input adjoints are gathered per input entry (inverse maps) from the
// step's stored g values, in a fixed order.  Bond sums are warp-reduced (over
// samples and lanes) into per-warp shared rows, added in warp order into one
// row per CTA, and the rows added per instance in a fixed order: the result
// does not depend on scheduling.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void acc_edge(float* acc_w, int e, float v, bool lane0) {
  v = warp_sum(v);
  if (lane0 && e >= 0) acc_w[e] += v;
}

__global__ void __launch_bounds__(128) general_dJ_kernel(const InstDev* __restrict__ inst,
                                                         const LaunchInfo li, int arena_floats, int max_steps,
                                                         int gmax, int GL, const int8_t* __restrict__ spins,
                                                         float* __restrict__ part, int part_stride,
                                                         float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int S = li.tile, slot = threadIdx.x / GL, lane = threadIdx.x % GL;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * S, b = b0 + slot;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  // tables, adjoints, scales and the step's g values, each [entry][sample]
  // (rows of RS floats), in shared memory or for large arenas in this CTA's
  // slice of a global scratch buffer
  const int RS = gen_row_stride(S, GL);
  const size_t cta_floats = (size_t)(2 * arena_floats + max_steps + gmax) * RS;
  float* base = garena ? garena + (size_t)blockIdx.x * cta_floats : sm;
  float* A = base + slot;                          // [arena]
  float* Ab = A + (size_t)arena_floats * RS;       // [arena] adjoints
  float* sc = Ab + (size_t)arena_floats * RS;      // [max_steps] scales 2^-e
  float* gb = sc + (size_t)max_steps * RS;         // [gmax] g of the current step
  const int ne4 = (I.n_edges + 3) & ~3, nw = blockDim.x >> 5;
  float* acc = garena ? sm : sm + cta_floats;  // [warps][n_edges]
  float* acc_w = acc + (threadIdx.x >> 5) * ne4;
  int8_t* ssp = reinterpret_cast<int8_t*>(acc + nw * ne4);
  const GenDev& G = I.gen;
  for (int e = threadIdx.x; e < nw * ne4; e += blockDim.x) acc[e] = 0.f;
  const int n_valid = min(S, li.batch - b0);
  stage_spins(ssp, spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, S, D, Dp);
  __syncthreads();
  const bool valid = b < li.batch;
  const bool lane0 = (threadIdx.x & 31) == 0;
  const int8_t* s = ssp + slot * Dp;
  // per-sample weight of the bond sums (importance multipliers when given)
  const float wscale =
      valid ? beta / (float)li.batch * (li.wmul ? li.wmul[(long long)k * li.batch + b] : 1.f) : 0.f;
  for (int c = 0; c < G.n_comp; ++c) {
    const int* H = G.fprog + G.fhdr[c];
    const int nsteps = H[0], fin = H[2];
    const int g0 = G.comp_step0[c];
    // forward: tables and their scales
    for (int st = 0; st < nsteps; ++st) {
      const StepRec r = step_at(G, g0 + st);
      const float h = field_of(G, r.fb, r.fc, s);
      const float ah = fabsf(h);
      const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
      const int M = 1 << r.m, E = 2 * M;
      const float* pp = G.pp + r.ppo;
      const unsigned short* mp = G.map + r.mo;
      const int out = r.out_full;
      float mx = 0.f;
      for (int x = lane; x < M; x += GL) {
        float accv = 0.f;
        for (int sg = 0; sg < 2; ++sg) {
          const int ext = x | (sg << r.m);
          float pr = fv[sg] * pp[ext];
          for (int i = 0; i < r.nin; ++i) pr *= A[(r.io[3 * i + 1] + mp[i * E + ext]) * RS];
          accv += pr;
        }
        A[(out + x) * RS] = accv;
        Ab[(out + x) * RS] = 0.f;
        mx = fmaxf(mx, accv);
      }
      mx = group_max(mx, GL);
      const float scl = pow2i(-exponent_of(mx));
      for (int x = lane; x < M; x += GL) A[(out + x) * RS] *= scl;
      if (lane == 0) sc[st * RS] = scl;
      __syncwarp();
    }
    if (lane == 0) Ab[fin * RS] = 1.f / A[fin * RS];
    __syncwarp();
    // backward
    for (int st = nsteps - 1; st >= 0; --st) {
      const StepRec r = step_at(G, g0 + st);
      const float h = field_of(G, r.fb, r.fc, s);
      const float ah = fabsf(h);
      const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
      const int M = 1 << r.m, E = 2 * M;
      const float* pp = G.pp + r.ppo;
      const unsigned short* mp = G.map + r.mo;
      const int out = r.out_full;
      const float scl = sc[st * RS];
      constexpr int MW = TNVAN_MAX_ELIM_W;
      const int np = min(r.npair, MW);  // at most MW neighbours remain
      int pos[MW];
#pragma unroll
      for (int j = 0; j < MW; ++j) pos[j] = j < np ? r.pr[2 * j + 1] : 0;
      float gs = 0.f;       // sum g sigma_v
      float gp[MW];         // sum g sigma_v sigma_u per pair
#pragma unroll
      for (int j = 0; j < MW; ++j) gp[j] = 0.f;
      for (int x = lane; x < M; x += GL) {
        const float abx = Ab[(out + x) * RS] * scl;
        for (int sg = 0; sg < 2; ++sg) {
          const int ext = x | (sg << r.m);
          float pr = fv[sg] * pp[ext];
          for (int i = 0; i < r.nin; ++i) pr *= A[(r.io[3 * i + 1] + mp[i * E + ext]) * RS];
          const float g = abx * pr;
          gb[ext * RS] = g;
          gs = fmaf(g, sg ? -1.f : 1.f, gs);
#pragma unroll
          for (int j = 0; j < MW; ++j)
            if (j < np) gp[j] = fmaf(g, (((x >> pos[j]) & 1) == sg) ? 1.f : -1.f, gp[j]);
        }
      }
      __syncwarp();
      // input adjoints: each entry gathers the g of the extended indices that
      // read it (inverse map), lanes split the entries
      for (int i = 0; i < r.nin; ++i) {
        const int in = r.io[3 * i + 1], kk = r.io[3 * i + 2];
        const int R = E >> kk;
        const unsigned short* inv = mp + (r.nin + i) * E;
        for (int e = lane; e < (1 << kk); e += GL) {
          const float av = A[(in + e) * RS];
          if (av > 0.f) {
            float sum = 0.f;
            for (int f = 0; f < R; ++f) sum += gb[inv[e * R + f] * RS];
            Ab[(in + e) * RS] += sum / av;
          }
        }
      }
      for (int f = r.fb; f < r.fb + r.fc; ++f)
        acc_edge(acc_w, G.fld[2 * f + 1], wscale * gs * (float)s[G.fld[2 * f]], lane0);
      for (int j = 0; j < np; ++j) acc_edge(acc_w, G.pairE[r.pr[2 * j]], wscale * gp[j], lane0);
      __syncwarp();
    }
  }
  __syncthreads();
  float* row = part + (long long)blockIdx.x * part_stride;
  for (int e = threadIdx.x; e < I.n_edges; e += blockDim.x) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += acc[w * ne4 + e];
    row[e] = v;
  }
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

cudaError_t launch_general_pp(const InstDev* d_inst, const LaunchInfo& li, int max_steps, cudaStream_t s) {
  if (max_steps <= 0) return cudaSuccess;
  general_pp_kernel<<<dim3(max_steps, li.n_inst), 256, 0, s>>>(d_inst, li);
  return cudaGetLastError();
}

// per-sample floats: 2 * arena + steps + gmax (tables, adjoints, scales, g)
int general_dJ_smem_bytes(int per_sample, int D, int n_edges, int T, int GL, bool glob) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return (glob ? 0 : per_sample * gen_row_stride(T, GL) * 4) + (T * GL / 32) * ((n_edges + 3) & ~3) * 4 +
         T * 4 * w4;
}

size_t general_dJ_scratch_floats(int per_sample, int T, int GL, int nblk) {
  return (size_t)per_sample * gen_row_stride(T, GL) * nblk;
}

cudaError_t launch_general_dJ(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int arena, int steps,
                              int gmax, int GL, const int8_t* spins, float* part, int part_stride, double* dJ,
                              float* garena, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(general_dJ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  general_dJ_kernel<<<nblk, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, steps, gmax, GL, spins, part,
                                                           part_stride, garena);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  general_dJ_reduce_kernel<<<dim3(4, li.n_inst), 256, 0, s>>>(d_inst, li, part, part_stride, dJ);
  return cudaGetLastError();
}

// The components' tables at this call's betas (li.gen_tab: the largest
// table; general_kernel then looks them up).
cudaError_t launch_general_tables(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, bool db, int GL,
                                  float* garena, cudaStream_t s) {
  if (li.gen_tab <= 0) return cudaSuccess;
  const int arena = (int)(li.seed & 0xffffffffull);
  const dim3 tg((unsigned)((li.gen_tab + li.tile - 1) / li.tile), li.n_inst);
  cudaError_t e;
  if (db) {
    e = cudaFuncSetAttribute(general_tab_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_tab_kernel<true><<<tg, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, GL, garena);
  } else {
    e = cudaFuncSetAttribute(general_tab_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_tab_kernel<false><<<tg, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, GL, garena);
  }
  return cudaGetLastError();
}

int general_smem_bytes(int arena, int D, int T, int GL, bool db, bool glob) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return (glob ? 0 : arena * gen_row_stride(T, GL) * 4 * (db ? 2 : 1)) + T * 4 * w4;
}

// Scratch of the global-table mode: one [arena][row stride] slice (two with
// d/dbeta) per CTA of the contraction and of the tables kernel.
size_t general_scratch_floats(const LaunchInfo& li, int arena, int GL, bool db) {
  const size_t per = (size_t)arena * gen_row_stride(li.tile, GL) * (db ? 2 : 1);
  size_t ctas = (size_t)li.tile_begin[li.n_inst];
  if (li.gen_tab > 0) ctas = std::max(ctas, (size_t)((li.gen_tab + li.tile - 1) / li.tile) * li.n_inst);
  return per * ctas;
}

cudaError_t launch_general(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int GL,
                           const int8_t* spins, double* logZR, double* dbeta, float* garena,
                           cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  // li.seed carries the arena size (floats) for this launch
  const int arena = (int)(li.seed & 0xffffffffull);
  cudaError_t e;
  if (dbeta) {
    e = cudaFuncSetAttribute(general_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<true><<<nblk, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, GL, spins, logZR, dbeta, garena);
  } else {
    e = cudaFuncSetAttribute(general_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<false><<<nblk, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, GL, spins, logZR, dbeta,
                                                                 garena);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Magnetisation moments of the elimination components (observables from
// samples, Sec. 3).  The forward program run in the moment form: every table
// entry carries, besides its weight, the conditional mean and variance of the
// magnetisation of the spins already summed into it given its scope.  A
// step's product term at (x, sigma) has mean sigma + sum of its inputs' means
// and variance the sum of their variances (the inputs cover disjoint
// eliminated spins, independent given the scope), and summing sigma out
// merges the two terms (moment_mix).  A component's final entry gives the
// conditional mean and variance of its magnetisation; components are
// independent given the width set.  Tabulated components run their programs
// here too.  Tables: weights, means, variances, each [entry][sample].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void run_component_mom(const GenDev& G, int c, const int8_t* s, float* A, float* Mu,
                                                  float* Q, int RS, int lane, int GL, float beta, double& mean,
                                                  double& var) {
  const int* H = G.fprog + G.fhdr[c];
  const int nsteps = H[0], fin = H[1];
  const int g0 = G.comp_step0[c];
  for (int st = 0; st < nsteps; ++st) {
    const StepRec r = step_at(G, g0 + st);
    const float h = field_of(G, r.fb, r.fc, s);
    const float ah = fabsf(h);
    const float fv[2] = {expf(beta * (h - ah)), expf(beta * (-h - ah))};
    const int M = 1 << r.m, E = 2 * M;
    const float* pp = G.pp + r.ppo;
    const unsigned short* mp = G.map + r.mo;
    const int out = r.out_live;
    float mx = 0.f;
    for (int x = lane; x < M; x += GL) {
      float tv[2], tm[2], tq[2];
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const int ext = x | (sg << r.m);
        float p = fv[sg] * pp[ext], m = sg ? -1.f : 1.f, q = 0.f;
        for (int i = 0; i < r.nin; ++i) {
          const int a = (r.io[3 * i] + mp[i * E + ext]) * RS;
          p *= A[a];
          m += Mu[a];
          q += Q[a];
        }
        tv[sg] = p;
        tm[sg] = m;
        tq[sg] = q;
      }
      float v, m, q;
      moment_mix(tv[0], tm[0], tq[0], tv[1], tm[1], tq[1], v, m, q);
      A[(out + x) * RS] = v;
      Mu[(out + x) * RS] = m;
      Q[(out + x) * RS] = q;
      mx = fmaxf(mx, v);
    }
    mx = group_max(mx, GL);
    const float sc = pow2i(-exponent_of(mx));
    for (int x = lane; x < M; x += GL) A[(out + x) * RS] *= sc;
    __syncwarp();
  }
  if (lane == 0) {
    mean += (double)Mu[fin * RS];
    var += (double)Q[fin * RS];
  }
}

__global__ void __launch_bounds__(128) general_mom_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                          int arena_floats, int GL, const int8_t* __restrict__ spins,
                                                          double* __restrict__ mag_mean, double* __restrict__ mag_var,
                                                          float* __restrict__ garena) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int S = li.tile, slot = threadIdx.x / GL, lane = threadIdx.x % GL;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * S, b = b0 + slot;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  const int RS = gen_row_stride(S, GL);
  const size_t cta_floats = (size_t)arena_floats * RS * 3;
  float* base = garena ? garena + (size_t)blockIdx.x * cta_floats : sm;
  float* A = base + slot;
  float* Mu = A + (size_t)arena_floats * RS;
  float* Q = Mu + (size_t)arena_floats * RS;
  int8_t* ssp = reinterpret_cast<int8_t*>(garena ? sm : sm + cta_floats);
  const GenDev& G = I.gen;
  const int n_valid = min(S, li.batch - b0);
  stage_spins(ssp, spins + I.spin_units * li.batch + (long long)b0 * D, n_valid, S, D, Dp);
  __syncthreads();
  const int8_t* s = ssp + slot * Dp;
  double mean = 0.0, var = 0.0;
  for (int c = 0; c < G.n_comp; ++c) run_component_mom(G, c, s, A, Mu, Q, RS, lane, GL, beta, mean, var);
  if (lane != 0 || b >= li.batch) return;
  int mw = 0;
  for (int j = 0; j < D; ++j) mw += s[j];
  const long long o = (long long)k * li.batch + b;
  mag_mean[o] = (double)mw + mean;
  mag_var[o] = var;
}

int general_mom_smem_bytes(int arena, int D, int T, int GL, bool glob) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return (glob ? 0 : arena * gen_row_stride(T, GL) * 4 * 3) + T * 4 * w4;
}

size_t general_mom_scratch_floats(const LaunchInfo& li, int arena, int GL) {
  return (size_t)arena * gen_row_stride(li.tile, GL) * 3 * (size_t)li.tile_begin[li.n_inst];
}

cudaError_t launch_general_mom(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int arena, int GL,
                               const int8_t* spins, double* mag_mean, double* mag_var, float* garena,
                               cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(general_mom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  general_mom_kernel<<<nblk, li.tile * GL, smem_bytes, s>>>(d_inst, li, arena, GL, spins, mag_mean, mag_var, garena);
  return cudaGetLastError();
}

}  // namespace tnvan
