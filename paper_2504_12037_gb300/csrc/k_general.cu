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
// consecutive words.  Every new table is renormalised by a power of two.
// Factors are stored normalised (largest entry 1); the removed constants
// (beta |h_v| per field, beta |J| per bond) are added back in FP64.
// With DB, every table entry carries its beta-derivative (forward mode).
#include "common.cuh"

namespace tnvan {

__device__ __forceinline__ int padded_bytes(int D) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return 4 * w4;
}

template <bool DB>
__global__ void __launch_bounds__(64) general_kernel(const InstDev* __restrict__ inst,
                                                     const LaunchInfo li, int arena_floats,
                                                     int max_pairs,
                                                     const int8_t* __restrict__ spins,
                                                     double* __restrict__ logZR,
                                                     double* __restrict__ dbeta) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.kind != 2) return;
  const int T = li.tile, t = threadIdx.x;
  const int b0 = (blockIdx.x - li.tile_begin[k]) * T, b = b0 + t;
  const float beta = (float)li.beta[k];
  const int D = I.D, Dp = padded_bytes(D);
  float* A = sm;                                   // [arena][T]
  float* dA = A + arena_floats * T;                // [arena][T] (DB)
  float4* pt = reinterpret_cast<float4*>(dA + (DB ? arena_floats * T : 0));  // [pairs]
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
  const int* P = G.prog;
  int ip = 1;
  double lz = 0.0, dl = 0.0;
  const int ncomp = P[0];
  for (int c = 0; c < ncomp; ++c) {
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

int general_smem_bytes(int arena, int pairs, int D, int T, bool db) {
  int w4 = (D + 3) / 4;
  if ((w4 & 1) == 0) ++w4;
  return arena * T * 4 * (db ? 2 : 1) + pairs * 16 + T * 4 * w4;
}

cudaError_t launch_general(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                           const int8_t* spins, double* logZR, double* dbeta, double*,
                           cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  // li.seed carries (arena floats, max pairs) for this launch
  const int arena = (int)(li.seed & 0xffffffffull), pairs = (int)(li.seed >> 32);
  cudaError_t e;
  if (dbeta) {
    e = cudaFuncSetAttribute(general_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<true><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, spins, logZR, dbeta);
  } else {
    e = cudaFuncSetAttribute(general_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    general_kernel<false><<<nblk, li.tile, smem_bytes, s>>>(d_inst, li, arena, pairs, spins, logZR, dbeta);
  }
  return cudaGetLastError();
}

}  // namespace tnvan
