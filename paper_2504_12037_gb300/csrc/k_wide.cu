// Wide lattice strips: exact row transfer-matrix contraction (Eq. 2-4 with W
// = whole columns) of strips of up to TNVAN_WIDE_MAX_W columns, for lattice
// instances whose plan is an elimination plan (their strips are wider than
// the per-thread strip kernels hold in registers).  Forward log Z_R only.
//
// One CTA per sample, one warp per strip.  The 2^w states of a strip row are
// spread over the warp: state x = lane | (j << 5), lane holding j = 0 ..
// 2^(w-5) - 1 in registers (strips narrower than 5 columns use lanes < 2^w).
// Per row y (same gauge as the strip planner: every vertical coupling >= 0):
//   v <- V_{y-1} v   with V the Kronecker product of [[1, t_c], [t_c, 1]],
//                    t_c = exp(-2 beta Jv_c): a shuffle for column bits < 5,
//                    a register pair for the others;
//   v <- D_y v       D_y(x) = product over the row's bonds that x leaves
//                    unsatisfied (J s s' < 0, W neighbours included) of
//                    exp(-2 beta |J|): every factor is at most 1;
//   v <- v / 2^e     e the exponent of the row's largest entry.
// ln Z_strip = ln sum_x v(x) + ln 2 sum e + beta sum |J| over the strip's
// bonds; log Z_R adds beta sum over W-W bonds J s s' (Eq. 4).
#include "common.cuh"

namespace tnvan {

namespace {

// Factor of a bond of coupling J that a state leaves unsatisfied.
__device__ __forceinline__ float unsat_factor(float J, float beta) { return expf(-2.f * beta * fabsf(J)); }

// One strip for one sample; NPL = states per lane (2^(w-5), or 1 for w <= 5).
// Returns ln of the normalised sum and the power-of-two exponent count.
template <int NPL>
__device__ void wide_chain(const WideStripDev& sd, const WideRow* __restrict__ rows, const int8_t* srow, float beta,
                           int lane, float& lnz, int& e2) {
  const int w = sd.w;
  const bool active = NPL > 1 || lane < (1 << w);
  float v[NPL];
  e2 = 0;
  for (int y = 0; y < sd.L; ++y) {
    const WideRow& R = rows[y];
    // the row's factors, one per lane: lanes 0..10 horizontal bonds, 16..27
    // vertical factors from row y - 1, 30 / 31 the W neighbours
    float f = 1.f;
    if (lane < w - 1) f = unsat_factor(R.Jh[lane], beta);
    else if (lane >= 16 && lane < 16 + w && y > 0) f = expf(-2.f * beta * rows[y - 1].Jv[lane - 16]);
    else if (lane == 30 && R.posL >= 0) f = unsat_factor(R.JL, beta);
    else if (lane == 31 && R.posR >= 0) f = unsat_factor(R.JR, beta);
    // negative-coupling bits of the horizontal bonds and the W-neighbour terms
    uint32_t neg = 0;
    for (int c = 0; c + 1 < w; ++c) neg |= (R.Jh[c] < 0.f ? 1u : 0u) << c;
    // a W-neighbour bond J s_W s_0 is satisfied iff bit 0 == (J s_W < 0)
    const float sL = R.posL >= 0 ? (float)srow[R.posL] : 0.f, sR = R.posR >= 0 ? (float)srow[R.posR] : 0.f;
    const uint32_t wantL = (R.JL * sL < 0.f) ? 1u : 0u, wantR = (R.JR * sR < 0.f) ? 1u : 0u;
    const float uL = __shfl_sync(0xffffffffu, f, 30), uR = __shfl_sync(0xffffffffu, f, 31);
    if (y > 0) {
      // vertical factors: column bits below 5 across lanes, the rest in registers
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float t = __shfl_sync(0xffffffffu, f, 16 + c);
        if (c < w) {
#pragma unroll
          for (int j = 0; j < NPL; ++j) v[j] = fmaf(t, __shfl_xor_sync(0xffffffffu, v[j], 1 << c), v[j]);
        }
      }
#pragma unroll
      for (int c = 5; c < 5 + 7; ++c) {
        if ((1 << (c - 5)) < NPL) {
          const float t = __shfl_sync(0xffffffffu, f, 16 + c);
#pragma unroll
          for (int j = 0; j < NPL; ++j) {
            if ((j >> (c - 5)) & 1) continue;
            const int j1 = j | (1 << (c - 5));
            const float a = v[j], b = v[j1];
            v[j] = fmaf(t, b, a);
            v[j1] = fmaf(t, a, b);
          }
        }
      }
    }
    // diagonal: the lane part (bonds among bits 0..4, the left neighbour, and
    // the right one when w <= 5), then per register the bonds among its bits
    const uint32_t x0 = (uint32_t)lane;
    float pl = 1.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float u = __shfl_sync(0xffffffffu, f, c);
      if (c + 1 < w && ((((x0 >> c) ^ (x0 >> (c + 1))) & 1u) != ((neg >> c) & 1u))) pl *= u;
    }
    if (R.posL >= 0 && ((x0 & 1u) != wantL)) pl *= uL;
    if (w <= 5 && R.posR >= 0 && (((x0 >> (w - 1)) & 1u) != wantR)) pl *= uR;
    // bond 4 (bits 4, 5) and bonds 5 .. w-2, the right neighbour on bit w-1
    const float u4 = __shfl_sync(0xffffffffu, f, 4);
    float ub[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) ub[i] = __shfl_sync(0xffffffffu, f, (5 + i) & 31);
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      float d = pl;
      if (NPL > 1) {
        const uint32_t x = x0 | ((uint32_t)j << 5);
        if (((((x >> 4) ^ (x >> 5)) & 1u) != ((neg >> 4) & 1u))) d *= u4;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
          const int c = 5 + i;
          if ((2 << i) < NPL && ((((x >> c) ^ (x >> (c + 1))) & 1u) != ((neg >> c) & 1u))) d *= ub[i];
        }
        if (R.posR >= 0 && (((x >> (w - 1)) & 1u) != wantR)) d *= uR;
      }
      const float vv = y == 0 ? d : v[j] * d;
      v[j] = active ? vv : 0.f;
      mx = fmaxf(mx, v[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exponent_of(mx);
    const float sc = pow2i(-e);
#pragma unroll
    for (int j = 0; j < NPL; ++j) v[j] *= sc;
    e2 += e;
  }
  float z = 0.f;
#pragma unroll
  for (int j = 0; j < NPL; ++j) z += v[j];
  z = warp_sum(z);
  lnz = logf(z);
}

}  // namespace

// States per lane of a strip of w columns.
__host__ __device__ __forceinline__ int wide_npl(int w) { return w <= 5 ? 1 : 1 << (w - 5); }

// The strips of one state-count class (wide_npl(w) == NPL): CTA = sample,
// warps over the instance's strips of that class; per-strip results to
// part[(k * batch + b) * li.tile_aux + strip].
template <int NPL>
__global__ void __launch_bounds__(256) wide_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                                    const int8_t* __restrict__ spins, double* __restrict__ part) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  if (I.n_wide == 0) return;
  const int b = blockIdx.x - li.tile_begin[k];
  const int t = threadIdx.x, wp = t >> 5, lane = t & 31;
  const int D = I.D;
  const int nw = blockDim.x >> 5;
  int8_t* srow = reinterpret_cast<int8_t*>(sm);
  const int8_t* g = spins + I.spin_units * li.batch + (long long)b * D;
  for (int e = t; e < D; e += blockDim.x) srow[e] = g[e];
  __syncthreads();
  const float beta = (float)li.beta[k];
  double* out = part + ((long long)k * li.batch + b) * li.tile_aux;
  int nth = 0;  // index of the strip among this class's strips
  for (int st = 0; st < I.n_wide; ++st) {
    const WideStripDev sd = I.wide[st];
    if (wide_npl(sd.w) != NPL) continue;
    if (nth++ % nw != wp) continue;
    float lnz = 0.f;
    int e2 = 0;
    wide_chain<NPL>(sd, I.wrows + sd.row0, srow, beta, lane, lnz, e2);
    if (lane == 0) out[st] = (double)lnz + (double)e2 * 0.69314718055994530942 + li.beta[k] * sd.c_hat;
  }
}

// log Z_R per sample: the strips' results in strip order plus the W-W term.
__global__ void wide_sum_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                const int8_t* __restrict__ spins, const double* __restrict__ part,
                                double* __restrict__ logZR) {
  const int k = blockIdx.y;
  const InstDev& I = inst[k];
  if (I.n_wide == 0 || li.tile_begin[k + 1] == li.tile_begin[k]) return;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < li.batch; b += gridDim.x * blockDim.x) {
    const double* p = part + ((long long)k * li.batch + b) * li.tile_aux;
    double lz = 0.0;
    for (int st = 0; st < I.n_wide; ++st) lz += p[st];
    const int8_t* srow = spins + I.spin_units * li.batch + (long long)b * I.D;
    float e1 = 0.f;
    for (int e = 0; e < I.n_ww; ++e) {
      const EdgeWW q = I.ww[e];
      e1 = fmaf(q.J, (float)(srow[q.a] * srow[q.b]), e1);
    }
    logZR[(long long)k * li.batch + b] = lz + li.beta[k] * (double)e1;
  }
}

cudaError_t launch_wide(const InstDev* d_inst, const LaunchInfo& li, const int* strips_per_class, int max_strips,
                        int max_D, const int8_t* spins, double* part, double* logZR, cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0 || max_strips == 0) return cudaSuccess;
  LaunchInfo lw = li;
  lw.tile_aux = max_strips;
  const int smem = max_D + 16;
  for (int c = 0; c < 8; ++c) {
    const int n = strips_per_class[c];  // most strips of class c in one instance
    if (n == 0) continue;
    const int warps = n < 8 ? n : 8;
    switch (c) {
      case 0: wide_kernel<1><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 1: wide_kernel<2><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 2: wide_kernel<4><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 3: wide_kernel<8><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 4: wide_kernel<16><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 5: wide_kernel<32><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      case 6: wide_kernel<64><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
      default: wide_kernel<128><<<nblk, 32 * warps, smem, s>>>(d_inst, lw, spins, part); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  wide_sum_kernel<<<dim3((unsigned)((li.batch + 255) / 256), li.n_inst), 256, 0, s>>>(d_inst, lw, spins, part, logZR);
  return cudaGetLastError();
}

}  // namespace tnvan
