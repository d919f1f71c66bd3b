// MADE network kernels: parameter packing and ancestral sampling (Eq. 6-8).
#include "common.cuh"

namespace tnvan {

// Build the packed copy of every instance's network: each layer's [nout][nin]
// block with MADE masks applied and hidden units sorted by degree, then the
// biases in the same order.  grid = (ceil(max_elems / 256), n_inst).
__global__ void pack_kernel(const InstDev* __restrict__ inst) {
  const MadeDev& md = inst[blockIdx.y].made;
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int l = 0; l < md.n_layers; ++l) {
    const LayerDev& L = md.layer[l];
    long long nw = (long long)L.nout * L.nin;
    if (e < nw) {
      int o = (int)(e / L.nin), i = (int)(e % L.nin);
      int no = L.perm_out ? L.perm_out[o] : o;
      int ni = L.perm_in ? L.perm_in[i] : i;
      int dout = L.deg_out[o], din = L.deg_in[i];
      bool conn = L.strict ? (dout > din) : (dout >= din);
      md.packed[L.dst_off + e] = conn ? md.raw[L.src_off + (long long)no * L.nin + ni] : 0.f;
      return;
    }
    e -= nw;
    if (e < L.nout) {
      int no = L.perm_out ? L.perm_out[e] : (int)e;
      md.packed[L.dst_off + nw + e] = md.raw[L.src_off + nw + no];
      return;
    }
    e -= L.nout;
  }
}

cudaError_t launch_pack(const InstDev* d_inst, int n_inst, long long max_elems, cudaStream_t s) {
  if (n_inst == 0 || max_elems == 0) return cudaSuccess;
  dim3 grid((unsigned)((max_elems + 255) / 256), n_inst);
  pack_kernel<<<grid, 256, 0, s>>>(d_inst);
  return cudaGetLastError();
}

// Dot product of a warp-uniform weight row with this thread's activation
// column (layout [unit][T]), four partial sums for instruction-level parallelism.
__device__ __forceinline__ float dot_col(const float* __restrict__ w, const float* col, int T,
                                         int n) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int j = 0;
  for (; j + 4 <= n; j += 4) {
    a0 = fmaf(__ldg(w + j), col[(j)*T], a0);
    a1 = fmaf(__ldg(w + j + 1), col[(j + 1) * T], a1);
    a2 = fmaf(__ldg(w + j + 2), col[(j + 2) * T], a2);
    a3 = fmaf(__ldg(w + j + 3), col[(j + 3) * T], a3);
  }
  for (; j < n; ++j) a0 = fmaf(__ldg(w + j), col[j * T], a0);
  return (a0 + a1) + (a2 + a3);
}

// Ancestral sampling, one thread per sample, tile of T samples per CTA.
// Hidden units are degree-sorted, so at step i (output i, degree i+1):
//   layer-1 units of degree i need inputs 0..i-1 (all drawn),
//   layer-2 units of degree i need the layer-1 prefix c1[i],
//   output i needs the last hidden prefix c_L[i].
// Every unit is therefore evaluated exactly once: one masked forward pass.
// With `given` non-null the spins are read from it instead of drawn (teacher
// forcing), which evaluates log q of caller-supplied configurations.
// Shared memory (per CTA): S [D][T] spins as +-1 floats, A1 [H1][T], A2 [H2][T].
__global__ void __launch_bounds__(128) sample_kernel(const InstDev* __restrict__ inst,
                                                     const LaunchInfo li,
                                                     int8_t* __restrict__ spins,
                                                     float* __restrict__ logq,
                                                     const int8_t* __restrict__ given) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const int T = li.tile, t = threadIdx.x;
  const int b = (blockIdx.x - li.tile_begin[k]) * T + t;
  const int D = md.D, nh = md.nh, H1 = md.H1, H2 = md.H2, Hl = md.Hl;
  float* S = sm;
  float* A1 = S + D * T;
  float* A2 = A1 + H1 * T;
  const float* W1 = md.packed + md.layer[0].dst_off;
  const float* b1 = W1 + (long long)H1 * D;
  const float* W2 = nh >= 2 ? md.packed + md.layer[1].dst_off : nullptr;
  const float* b2 = nh >= 2 ? W2 + (long long)H2 * H1 : nullptr;
  const float* Wo = md.packed + md.layer[nh].dst_off;
  const float* bo = Wo + (long long)D * Hl;
  const float* src = nh == 0 ? S : (nh == 1 ? A1 : A2);
  const int* cL = nh == 1 ? md.c1 : md.c2;
  const uint2 key = make_uint2((uint32_t)li.seed, (uint32_t)(li.seed >> 32));
  float lq = 0.f;
  uint4 rnd = make_uint4(0, 0, 0, 0);
  for (int i = 0; i < D; ++i) {
    if ((i & 3) == 0)
      rnd = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(i >> 2), (uint32_t)li.step, (uint32_t)k),
                          key);
    if (nh >= 1 && i >= 1) {
      const int u0 = md.c1[i - 1], u1 = md.c1[i];
      for (int u = u0; u < u1; ++u)
        A1[u * T + t] = fmaxf(__ldg(b1 + u) + dot_col(W1 + (long long)u * D, S + t, T, i), 0.f);
    }
    if (nh >= 2 && i >= 1) {
      const int u0 = md.c2[i - 1], u1 = md.c2[i], n1 = md.c1[i];
      for (int u = u0; u < u1; ++u)
        A2[u * T + t] = fmaxf(__ldg(b2 + u) + dot_col(W2 + (long long)u * H1, A1 + t, T, n1), 0.f);
    }
    const int nin = nh == 0 ? i : cL[i];
    const float x = __ldg(bo + i) + dot_col(Wo + (long long)i * Hl, src + t, T, nin);
    const float p = 1.f / (1.f + expf(-x));
    const uint32_t word = (i & 3) == 0 ? rnd.x : (i & 3) == 1 ? rnd.y : (i & 3) == 2 ? rnd.z : rnd.w;
    const float u = (float)(word >> 8) * 5.9604644775390625e-08f;  // 2^-24
    float s = u < p ? 1.f : -1.f;
    if (given) s = (b < li.batch) ? (float)given[I.spin_units * li.batch + (long long)b * D + i] : 1.f;
    S[i * T + t] = s;
    lq -= softplusf(-s * x);
  }
  if (b < li.batch) {
    if (spins) {
      int8_t* out = spins + I.spin_units * li.batch + (long long)b * D;
      for (int i = 0; i < D; ++i) out[i] = (int8_t)S[i * T + t];
    }
    logq[(long long)k * li.batch + b] = lq;
  }
}

int sample_smem_bytes(const Instance& in, int tile) {
  return (int)((in.W.size() + in.H[0] + in.H[1]) * tile * sizeof(float));
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
