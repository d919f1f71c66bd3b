// BF16 ancestral sampler on tcgen05 (Eq. 6-8), grouped form, for networks
// with two hidden layers of at most 256 units (multiples of 16) and at most
// 256 inputs (padded to a multiple of 16): the fast path where it applies;
// k_sample_tc.cu holds the general per-step form.
//
// One CTA (128 threads, thread = sample = TMEM lane) draws 128 samples; its
// TMEM footprint is at most 256 columns and its shared memory about 100 KB
// for the 64-128-128-64 network, so two CTAs share an SM.  Width sets of more
// than 128 spins, layers of more than 128 units (or weight tiles too large
// for shared memory) stream the
// weights instead: each step group carries one BF16 blob (its W2 and Wo
// windows, and W1's rows of its layer-1 units) that is bulk-copied one group
// ahead into one of two buffers; 512 TMEM columns, one CTA per SM.  TMEM holds
//   P1g [128 x w1]  layer-1 pre-activations of the current step group's units
//                   from every spin before the group, recomputed per group as
//                   S W1_g^T (S = the spin tile so far, zero beyond);
//   P2  [128 x H2]  layer-2 pre-activations, accumulated over the groups;
//   PO  [128 x D]   output pre-activations, accumulated over the groups.
// Steps are processed in the host's step groups.  Inside a group, each step
// reads the pre-activations of the units completing at that step straight
// from TMEM (tcgen05.ld), adds the in-group contributions on the CUDA cores
// (FP32 triangle tiles of the group, bulk-copied into shared memory; in-group
// spins from a register bitmask, in-group hidden values from the BF16 fold
// tiles), and draws s_i = +1 iff u < sigmoid(x_i).  After the group one
// tcgen05.mma chain folds its hidden values into the accumulators and
// recomputes P1g for the next group:
//   P2 += H1_g W2_g^T,  PO += H2_g Wo_g^T,  P1g' = S W1_g'^T.
// Every hidden value enters every later product as BF16 with FP32
// accumulation; in-group arithmetic is FP32 on the same BF16 values.
//
// When at most 4 units of a layer complete at any step (the host's slot
// layout, U slots per layer and step), the in-group steps run in the slot
// form: the group's accumulated pre-activations come from TMEM in one batch
// of loads at the group's start, and its hidden values stay in registers at
// compile-time indices (the group's 8 steps unrolled), so a step's dependency
// chain is register arithmetic only; the per-unit form reads them back from
// the fold tiles.
//
// The spin tile S and the fold tiles H1_g, H2_g are MN-major MMA operands in
// which consecutive 8-sample core-matrix groups are 16 bytes apart modulo
// 128, so the per-sample stores and loads (one 2-byte element per thread)
// are free of bank conflicts.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tnvan {

namespace {

// MN-major operand tile of 128 rows (samples) and kw columns (K, a multiple
// of 16): element (m, k) at (m >> 3) * sbo + (k >> 3) * 128 + (k & 7) * 16 +
// (m & 7) * 2 = (m >> 3) * sbo + (m & 7) * 2 + 16 k.
__host__ __device__ __forceinline__ uint32_t mn_sbo(int kw) { return (uint32_t)kw * 16u + 16u; }
__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t o, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + o) = __float2bfloat16(v);
}
__device__ __forceinline__ float ld_bf16(const unsigned char* base, uint32_t o) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + o));
}

// One TMEM column of the warp's 32 lanes into a register, without waiting;
// tmem_wait9 / tmem_wait1 order every later use of the destinations after
// the wait.
__device__ __forceinline__ void tmem_ld1_nowait(uint32_t taddr, uint32_t& r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait9(uint32_t (&a)[4], uint32_t (&b)[4], uint32_t& c) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(c)::"memory");
}
__device__ __forceinline__ void tmem_wait1(uint32_t& c) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(c)::"memory");
}
__device__ __forceinline__ float pick4(const uint32_t (&r)[4], int j) {
  const uint32_t v = j == 0 ? r[0] : (j == 1 ? r[1] : (j == 2 ? r[2] : r[3]));
  return __uint_as_float(v);
}

}  // namespace

#define STC_GI 8   // most steps in a group

const int kTcGroupMaxG[TNVAN_TC_PLANS] = {4, 6, 8};

struct SampleTcgLayout {
  int wbytes, oS, oH1, oH2, oBuf, buf, oBar, total;
};

// D is padded to a multiple of 16 (the weight tiles' padding: zero rows and
// columns, spins beyond D never drawn).
// wbmax > 0: streamed weights, two group blobs of wbmax bytes in place of the
// resident tiles.
__host__ __device__ inline SampleTcgLayout sample_tcg_layout(int D, int H1, int H2, int tcw1, int tcw2, int twmax,
                                                             int wbmax = 0) {
  D = (D + 15) & ~15;
  SampleTcgLayout L;
  L.wbytes = wbmax > 0 ? 2 * ((wbmax + 127) & ~127) : 2 * (H1 * D + H2 * H1 + D * H2);
  int p = (L.wbytes + 127) & ~127;
  L.oS = p;
  p += 16 * (int)mn_sbo(D);
  L.oH1 = p;
  p += 16 * (int)mn_sbo(tcw1) + 64;  // + zeroed tail read by the 4-wide in-group loops
  L.oH2 = p;
  p += 16 * (int)mn_sbo(tcw2) + 64;
  // two group buffers (this group's, the next group's): the record then the
  // triangles and biases
  L.oBuf = p;
  L.buf = 4 * TNVAN_TCGG_INTS + 4 * ((twmax + 3) & ~3);
  p += 2 * L.buf;
  p = (p + 15) & ~15;
  L.oBar = p;
  p += 32;
  L.total = p;
  return L;
}

__device__ __forceinline__ void tmem_wait_all() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Orders later uses of r after the preceding tcgen05.wait::ld.
__device__ __forceinline__ void tie(uint32_t& r) { asm volatile("" : "+r"(r)); }
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16(v)); }

// Dot product of a weight row (shared memory, 16-byte aligned) with the first
// N register values, four accumulators; N is a compile-time constant.
template <int N, int S>
__device__ __forceinline__ float slot_dot(const float* __restrict__ w, const float (&h)[S], float a0) {
  float a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int c4 = 0; c4 < (N + 3) / 4; ++c4) {
    const float4 x = reinterpret_cast<const float4*>(w)[c4];
    if (4 * c4 + 0 < N) a0 = fmaf(x.x, h[4 * c4 + 0], a0);
    if (4 * c4 + 1 < N) a1 = fmaf(x.y, h[4 * c4 + 1], a1);
    if (4 * c4 + 2 < N) a2 = fmaf(x.z, h[4 * c4 + 2], a2);
    if (4 * c4 + 3 < N) a3 = fmaf(x.w, h[4 * c4 + 3], a3);
  }
  return (a0 + a1) + (a2 + a3);
}

// Per-sample state the in-group steps update.
struct SlotState {
  uint4 rnd;
  uint32_t gbits;  // bit q set iff the group's step q drew +1
  float lq;
};

// The steps of one group in the slot form (U slots per layer and step, the
// host's slot layout): the accumulated pre-activations of every slot come
// from TMEM at once, the group's hidden values stay in registers at
// compile-time indices (q U + a), and only the fold tiles and the spin tile
// are written to shared memory.  Same arithmetic as the per-unit form: BF16
// hidden values, FP32 sums.
template <int U, int Q>
__device__ __forceinline__ void slot_step(const int* G, const float* TWb, int i0, const uint32_t (&a1)[8],
                                          const uint32_t (&a2)[8], uint32_t m1, uint32_t m2,
                                          const uint32_t (&r1)[8 * U], const uint32_t (&r2)[8 * U],
                                          const uint32_t (&ro)[8], float (&h1)[8 * U], float (&h2)[8 * U],
                                          float (&sg)[8], unsigned char* sH1, unsigned char* sH2, unsigned char* sS,
                                          uint32_t rbS, int b, uint32_t step32, int k, uint2 key, const int8_t* gv,
                                          bool valid, SlotState& st) {
  constexpr int S = 8 * U;
  const int i = i0 + Q;
  if ((i & 3) == 0) st.rnd = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(i >> 2), step32, (uint32_t)k), key);
  const float* TW1 = TWb;
  const float* TW2 = TWb + G[8];
  const float* TWo = TWb + G[9];
  const float* B1 = TWb + G[10];
  const float* B2 = TWb + G[11];
  const float* BO = TWb + G[12];
  // layer 1: + in-group spins j < Q (slot (Q, a) stores at a1[Q] + 16 a when it holds a unit)
#pragma unroll
  for (int a = 0; a < U; ++a) {
    const int r = Q * U + a;
    const float x = slot_dot<Q, 8>(TW1 + r * 8, sg, __uint_as_float(r1[r]) + B1[r]);
    const __nv_bfloat16 hb = __float2bfloat16(fmaxf(x, 0.f));
    h1[r] = __bfloat162float(hb);
    if ((m1 >> r) & 1u) *reinterpret_cast<__nv_bfloat16*>(sH1 + a1[Q] + 16u * a) = hb;
  }
  // layer 2: + in-group layer-1 slots of steps <= Q
#pragma unroll
  for (int a = 0; a < U; ++a) {
    const int r = Q * U + a;
    const float x = slot_dot<(Q + 1) * U, S>(TW2 + r * S, h1, __uint_as_float(r2[r]) + B2[r]);
    const __nv_bfloat16 hb = __float2bfloat16(fmaxf(x, 0.f));
    h2[r] = __bfloat162float(hb);
    if ((m2 >> r) & 1u) *reinterpret_cast<__nv_bfloat16*>(sH2 + a2[Q] + 16u * a) = hb;
  }
  // output i: + in-group layer-2 slots of steps <= Q
  const float x = slot_dot<(Q + 1) * U, S>(TWo + Q * S, h2, __uint_as_float(ro[Q]) + BO[Q]);
  // one exponential for both sigmoid(x) and softplus(-s x) (fast-math forms)
  const float ex = __expf(-fabsf(x));
  const float rcp = __frcp_rn(1.f + ex);
  const float pr = x >= 0.f ? rcp : ex * rcp;
  const uint32_t word = (i & 3) == 0 ? st.rnd.x : (i & 3) == 1 ? st.rnd.y : (i & 3) == 2 ? st.rnd.z : st.rnd.w;
  const float u = (float)(word >> 8) * 5.9604644775390625e-08f;
  bool up = u < pr;
  if (gv) up = valid ? gv[i] > 0 : true;
  const float s = up ? 1.f : -1.f;
  sg[Q] = s;
  st.gbits |= (up ? 1u : 0u) << Q;
  st_bf16(sS, rbS + 16u * (uint32_t)i, s);
  st.lq -= fmaxf(-s * x, 0.f) + __logf(1.f + ex);
}

template <int U>
__device__ __forceinline__ void slot_group(const int* G, const float* TWb, int gi, int i0, int w1, int w2, uint32_t tP1,
                                           uint32_t tP2, uint32_t tPO, bool p1ok, bool init2, bool inito,
                                           unsigned char* sH1, unsigned char* sH2, unsigned char* sS, uint32_t rb1,
                                           uint32_t rb2, uint32_t rbS, int b, uint32_t step32, int k, uint2 key,
                                           const int8_t* gv, bool valid, SlotState& st) {
  constexpr int S = 8 * U;
  uint32_t r1[S], r2[S], ro[8];
  // fold-tile addresses of each step's first unit, and which slots hold units
  uint32_t a1[8], a2[8], m1 = 0u, m2 = 0u;
#pragma unroll
  for (int j = 0; j < S; ++j) r1[j] = r2[j] = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) ro[q] = 0u;
  // every slot's accumulated pre-activations (warp-uniform conditions)
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    a1[q] = a2[q] = 0u;
    if (q < gi) {
      const int ua = G[13 + q], nu = G[14 + q] - ua, va = G[22 + q], nv = G[23 + q] - va;
      a1[q] = rb1 + 16u * (uint32_t)(ua - w1);
      a2[q] = rb2 + 16u * (uint32_t)(va - w2);
#pragma unroll
      for (int a = 0; a < U; ++a) {
        if (a < nu) m1 |= 1u << (q * U + a);
        if (a < nv) m2 |= 1u << (q * U + a);
        if (p1ok && a < nu) tmem_ld1_nowait(tP1 + (uint32_t)(ua + a - w1), r1[q * U + a]);
        if (init2 && a < nv) tmem_ld1_nowait(tP2 + (uint32_t)(va + a), r2[q * U + a]);
      }
      if (inito) tmem_ld1_nowait(tPO + (uint32_t)(i0 + q), ro[q]);
    }
  }
  tmem_wait_all();
#pragma unroll
  for (int j = 0; j < S; ++j) {
    tie(r1[j]);
    tie(r2[j]);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) tie(ro[q]);
  float h1[S], h2[S], sg[8];
#define TNVAN_SLOT_STEP(QQ)                                                                                     \
  if (QQ < gi)                                                                                                  \
    slot_step<U, QQ>(G, TWb, i0, a1, a2, m1, m2, r1, r2, ro, h1, h2, sg, sH1, sH2, sS, rbS, b, step32, k, key, gv, \
                     valid, st);
  TNVAN_SLOT_STEP(0)
  TNVAN_SLOT_STEP(1)
  TNVAN_SLOT_STEP(2)
  TNVAN_SLOT_STEP(3)
  TNVAN_SLOT_STEP(4)
  TNVAN_SLOT_STEP(5)
  TNVAN_SLOT_STEP(6)
  TNVAN_SLOT_STEP(7)
#undef TNVAN_SLOT_STEP
}

__host__ __device__ inline int sample_tcg_tmem_cols(int D, int H2, int tcw1) {
  D = (D + 15) & ~15;
  return tcw1 + H2 + D <= 256 ? 256 : 512;
}

// ANY_STREAMED: some instance of the launch streams its weights (the
// resident-only instantiation carries none of that code).
template <bool ANY_STREAMED>
__global__ void __launch_bounds__(128, 2) sample_tcg_kernel(const InstDev* __restrict__ inst,
                                                           const LaunchInfo li, const TcgOrder ord, int plan,
                                                           int8_t* __restrict__ spins, float* __restrict__ logq,
                                                           const int8_t* __restrict__ given) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int gblk = blockIdx.x + li.blk0;
  int k, tile;
  if (ord.n > 0) {
    int j = 0;
    while (j + 1 < ord.n && ord.begin[j + 1] <= gblk) ++j;
    k = ord.inst[j];
    tile = gblk - ord.begin[j];
  } else {
    k = find_inst(li, gblk);
    tile = gblk - li.tile_begin[k];
  }
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const MadeDev::TcGroupPlan& P = md.tcg[plan];
  const int D = md.D, H1 = md.H1, H2 = md.H2;
  const int t = threadIdx.x, w = t >> 5;
  const int b = tile * 128 + t;
  const bool valid = b < li.batch;
  const bool streamed = ANY_STREAMED && P.streamed != 0;
  const SampleTcgLayout LY = sample_tcg_layout(D, H1, H2, P.tcw1, P.tcw2, P.twmax, streamed ? P.wbmax : 0);
  const uint32_t wbuf = (uint32_t)((P.wbmax + 127) & ~127);  // one streamed blob buffer
  unsigned char* sW1 = smem;
  const int Dp = (D + 15) & ~15;  // the tiles' padded width set
  unsigned char* sW2 = sW1 + 2 * H1 * Dp;
  unsigned char* sWo = sW2 + 2 * H2 * H1;
  unsigned char* sS = smem + LY.oS;
  unsigned char* sH1 = smem + LY.oH1;
  unsigned char* sH2 = smem + LY.oH2;
  unsigned char* gbuf0 = smem + LY.oBuf;
  unsigned char* gbuf1 = gbuf0 + LY.buf;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + LY.oBar);  // MMA completion
  uint64_t* cbar = bar + 1;                                     // bulk copies
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t sboS = mn_sbo(Dp), sbo1 = mn_sbo(P.tcw1), sbo2 = mn_sbo(P.tcw2);
  // this thread's row in the MN-major tiles: element k at row base + 16 k
  const uint32_t rowb = (uint32_t)(t & 7) * 2u;
  const uint32_t rbS = (uint32_t)(t >> 3) * sboS + rowb, rb1 = (uint32_t)(t >> 3) * sbo1 + rowb,
                 rb2 = (uint32_t)(t >> 3) * sbo2 + rowb;
  const uint32_t kbW1 = 2u * Dp / 16u * 128u, kbW2 = 2u * H1 / 16u * 128u, kbWo = 2u * H2 / 16u * 128u;
  const int ncols = sample_tcg_tmem_cols(D, H2, P.tcw1);
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  if (w == 0) {
    tc::tmem_alloc(slot, (uint32_t)ncols);
    tc::tmem_relinquish();
  }
  // the spin tile starts at zero (spins not drawn yet contribute nothing);
  // the fold tiles too (later groups zero only the columns they do not write)
  for (int o = t * 16; o < 16 * (int)sboS; o += 128 * 16)
    *reinterpret_cast<uint4*>(sS + o) = make_uint4(0, 0, 0, 0);
  for (int o = t * 16; o < 16 * (int)sbo1 + 64; o += 128 * 16)
    *reinterpret_cast<uint4*>(sH1 + o) = make_uint4(0, 0, 0, 0);
  for (int o = t * 16; o < 16 * (int)sbo2 + 64; o += 128 * 16)
    *reinterpret_cast<uint4*>(sH2 + o) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  uint32_t cphase = 0;
  bool copy_pending = false, mma_pending = false;
  // group gg's record and block into a group buffer (one thread; the caller
  // has armed cbar for `extra` more bytes)
  // streamed blob of group gg (its record r): bytes of the W2 window, the Wo
  // window and the W1 rows
  auto blob_parts = [&](const int* r, uint32_t& a, uint32_t& bb, uint32_t& c) {
    const int u1lo = r[2], u1hi = r[3], u2lo = r[4], u2hi = r[5];
    const int n1 = ((u1hi + 15) & ~15) - (u1lo & ~15), n2 = ((u2hi + 15) & ~15) - (u2lo & ~15);
    a = 2u * (uint32_t)(H2 * n1);
    bb = 2u * (uint32_t)(Dp * n2);
    c = 2u * (uint32_t)(n1 * ((r[0] + 15) & ~15));
  };
  auto copy_group = [&](int gg, unsigned char* dst, uint32_t extra) {
    const int* Gg = P.groups + TNVAN_TCGG_INTS * gg;
    const uint32_t nb = (uint32_t)__ldg(Gg + 7) * 4u;
    uint32_t wa = 0, wb = 0, wc = 0;
    if (streamed) {
      const int r[6] = {__ldg(Gg), 0, __ldg(Gg + 2), __ldg(Gg + 3), __ldg(Gg + 4), __ldg(Gg + 5)};
      blob_parts(r, wa, wb, wc);
    }
    const uint32_t wt = wa + wb + wc;
    mbar_expect_tx(cbar, extra + 4u * TNVAN_TCGG_INTS + nb + wt);
    bulk_g2s(dst, Gg, 4u * TNVAN_TCGG_INTS, cbar);
    if (nb) bulk_g2s(dst + 4 * TNVAN_TCGG_INTS, P.blocks + __ldg(Gg + 6), nb, cbar);
    if (wt) bulk_g2s(smem + (gg & 1) * wbuf, P.wblob + __ldg(Gg + 31), wt, cbar);
  };
  if (t == 0) {
    copy_group(0, gbuf0, streamed ? 0u : (uint32_t)LY.wbytes);
    if (!streamed) bulk_g2s(sW1, md.wtiles, (uint32_t)LY.wbytes, cbar);
  }
  copy_pending = true;
  const uint32_t tmem = *slot;
  const uint32_t lane_off = (uint32_t)(w * 32) << 16;
  const uint32_t tP1 = tmem + lane_off, tP2 = tP1 + (uint32_t)P.tcw1, tPO = tP2 + (uint32_t)H2;
  const uint32_t idA = 1u << 15;  // A operand MN-major
  const uint32_t id2 = tc::idesc(128, H2, 1u) | idA, ido = tc::idesc(128, Dp, 1u) | idA;
  const uint2 key = make_uint2((uint32_t)li.seed, (uint32_t)(li.seed >> 32));
  const uint32_t step32 = launch_step(li);
  const int8_t* gv = given ? given + I.spin_units * li.batch + (long long)b * D : nullptr;
  uint32_t phase = 0;
  bool ok = true;
  bool p1ok = false, init2 = false, inito = false;  // accumulator holds data
  float lq = 0.f;
  uint4 rnd = make_uint4(0, 0, 0, 0);
  unsigned long long sb0 = 0ull, sb1 = 0ull;  // spin i is +1 iff bit i is set
  for (int g = 0; g < P.n_groups; ++g) {
    unsigned char* gb = (g & 1) ? gbuf1 : gbuf0;      // this group's buffer
    unsigned char* gbn = (g & 1) ? gbuf0 : gbuf1;     // the next group's
    if (copy_pending) {  // group 0 (with the weights); later groups arrived during the previous group
      if (mbar_wait(cbar, cphase)) {
        cphase ^= 1u;
        copy_pending = false;
      } else {
        ok = false;
      }
    }
    const int* G = reinterpret_cast<const int*>(gb);
    const float* TWb = reinterpret_cast<const float*>(gb + 4 * TNVAN_TCGG_INTS);
    const int i0 = G[0], i1 = G[1], u1lo = G[2], u1hi = G[3], u2lo = G[4], u2hi = G[5];
    const int gi = i1 - i0, n1g = u1hi - u1lo, n2g = u2hi - u2lo;
    const int w1 = u1lo & ~15, w2 = u2lo & ~15;
    const int n1 = ((u1hi + 15) & ~15) - w1, n2 = ((u2hi + 15) & ~15) - w2;
    // the previous MMA chain is done: fold tiles free, accumulators and P1g final
    if (mma_pending) {
      if (mbar_wait(bar, phase)) {
        phase ^= 1u;
        mma_pending = false;
      } else {
        ok = false;
      }
      tc::fence_after_sync();
    }
    // the fold's K windows must be zero outside the units this group writes:
    // columns [0, u_lo - w) and [u_hi - w, n) of every 8-sample row group
    {
      const int lo1 = u1lo - w1, hi1 = u1hi - w1, p1 = lo1 + (n1 - hi1);
      const int lo2 = u2lo - w2, hi2 = u2hi - w2, p2 = lo2 + (n2 - hi2);
      // f / pn by a multiply and a shift: f < 16 pn <= 512 and r = ceil(2^16 / pn)
      // give floor(f r / 2^16) = floor(f / pn) exactly
      const uint32_t r1 = p1 ? (65535u + (uint32_t)p1) / (uint32_t)p1 : 0u;
      const uint32_t r2 = p2 ? (65535u + (uint32_t)p2) / (uint32_t)p2 : 0u;
      for (int e = t; e < 16 * (p1 + p2); e += 128) {
        const bool l1 = e < 16 * p1;
        const int f = l1 ? e : e - 16 * p1, pn = l1 ? p1 : p2, lo = l1 ? lo1 : lo2, hi = l1 ? hi1 : hi2;
        const int rg = (int)(((uint32_t)f * (l1 ? r1 : r2)) >> 16), j = f - rg * pn;
        const int col = j < lo ? j : hi + (j - lo);
        *reinterpret_cast<uint4*>((l1 ? sH1 : sH2) + rg * (l1 ? sbo1 : sbo2) + 16 * col) = make_uint4(0, 0, 0, 0);
      }
    }
    ok = __syncthreads_and(ok) != 0;  // zeroed fold tiles visible; one agreed flag
    if (!ok) break;
    if (t == 0 && g + 1 < P.n_groups) {  // the next group's data, while this group runs
      copy_group(g + 1, gbn, 0u);
    }
    if (g + 1 < P.n_groups) copy_pending = true;
    if (P.slot_u == 0) {
      const float* TW1 = TWb;
      const float* TW2 = TWb + G[8];
      const float* TWo = TWb + G[9];
      const float* gb1 = TWb + G[10];  // biases of the group's units
      const float* gb2 = TWb + G[11];
      const float* gbo = TWb + G[12];
      const int* gc1 = G + 13;  // c1[i], c2[i] for i = i0-1 .. i1-1
      const int* gc2 = G + 22;
      const int s1 = (gi + 3) & ~3, s2 = (n1g + 3) & ~3, so = (n2g + 3) & ~3;  // triangle row strides
      float sg[STC_GI];  // in-group spins (0 until drawn)
  #pragma unroll
      for (int j = 0; j < STC_GI; ++j) sg[j] = 0.f;
      for (int i = i0; i < i1; ++i) {
        if ((i & 3) == 0)
          rnd = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(i >> 2), step32, (uint32_t)k), key);
        const int q = i - i0;  // gc*[q] = c*[i-1], gc*[q+1] = c*[i]
        const int ua = gc1[q], ub = gc1[q + 1], va = gc2[q], vb = gc2[q + 1];
        // pre-activations of the units completing at step i (up to four per layer at once)
        uint32_t ra[4] = {0u, 0u, 0u, 0u}, rb[4] = {0u, 0u, 0u, 0u}, rc = 0u;
        if (p1ok) {
  #pragma unroll
          for (int j = 0; j < 4; ++j)
            if (ua + j < ub) tmem_ld1_nowait(tP1 + (uint32_t)(ua + j - w1), ra[j]);
        }
        if (init2) {
  #pragma unroll
          for (int j = 0; j < 4; ++j)
            if (va + j < vb) tmem_ld1_nowait(tP2 + (uint32_t)(va + j), rb[j]);
        }
        if (inito) tmem_ld1_nowait(tPO + (uint32_t)i, rc);
        tmem_wait9(ra, rb, rc);
        // layer 1: + in-group spins (q <= 7 of them; sg is 0 for the rest)
        for (int u = ua; u < ub; ++u) {
          float a0;
          if (u - ua < 4) {
            a0 = pick4(ra, u - ua);
          } else {  // more than four units at one step
            uint32_t rx = 0u;
            if (p1ok) tmem_ld1_nowait(tP1 + (uint32_t)(u - w1), rx);
            tmem_wait1(rx);
            a0 = __uint_as_float(rx);
          }
          a0 += gb1[u - u1lo];
          const float4* wr = reinterpret_cast<const float4*>(TW1 + (u - u1lo) * s1);
          const float4 wa = wr[0];
          const float4 wb = s1 > 4 ? wr[1] : make_float4(0.f, 0.f, 0.f, 0.f);
          float a1 = wa.y * sg[1];
          a0 = fmaf(wa.x, sg[0], a0);
          a0 = fmaf(wa.z, sg[2], a0);
          a1 = fmaf(wa.w, sg[3], a1);
          a0 = fmaf(wb.x, sg[4], a0);
          a1 = fmaf(wb.y, sg[5], a1);
          a0 = fmaf(wb.z, sg[6], a0);
          a1 = fmaf(wb.w, sg[7], a1);
          st_bf16(sH1, rb1 + 16u * (uint32_t)(u - w1), fmaxf(a0 + a1, 0.f));
        }
        // layer 2: + in-group layer-1 units completed so far (BF16 values, 4 at a time;
        // units not computed yet read as 0 and carry masked weights)
        const uint32_t o1 = rb1 + 16u * (uint32_t)(u1lo - w1);
        auto pre2 = [&](int v) -> float {  // accumulated pre-activation + bias of layer-2 unit v
          float a;
          if (v - va < 4) {
            a = pick4(rb, v - va);
          } else {
            uint32_t rx = 0u;
            if (init2) tmem_ld1_nowait(tP2 + (uint32_t)v, rx);
            tmem_wait1(rx);
            a = __uint_as_float(rx);
          }
          return a + gb2[v - u2lo];
        };
        int v = va;
        for (; v + 2 <= vb; v += 2) {  // two units of one step share the in-group H1 values
          float a0 = pre2(v), b0 = pre2(v + 1);
          const float* wr = TW2 + (v - u2lo) * s2;
          const float* wq = wr + s2;
          float a1 = 0.f, b1 = 0.f;
          for (int c = 0; c < ub - u1lo; c += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wr + c);
            const float4 q4 = *reinterpret_cast<const float4*>(wq + c);
            const uint32_t o = o1 + 16u * (uint32_t)c;
            const float h0 = ld_bf16(sH1, o), h1 = ld_bf16(sH1, o + 16u), h2 = ld_bf16(sH1, o + 32u),
                        h3 = ld_bf16(sH1, o + 48u);
            a0 = fmaf(w4.x, h0, a0);
            b0 = fmaf(q4.x, h0, b0);
            a1 = fmaf(w4.y, h1, a1);
            b1 = fmaf(q4.y, h1, b1);
            a0 = fmaf(w4.z, h2, a0);
            b0 = fmaf(q4.z, h2, b0);
            a1 = fmaf(w4.w, h3, a1);
            b1 = fmaf(q4.w, h3, b1);
          }
          st_bf16(sH2, rb2 + 16u * (uint32_t)(v - w2), fmaxf(a0 + a1, 0.f));
          st_bf16(sH2, rb2 + 16u * (uint32_t)(v + 1 - w2), fmaxf(b0 + b1, 0.f));
        }
        if (v < vb) {
          float a0 = pre2(v);
          const float* wr = TW2 + (v - u2lo) * s2;
          float a1 = 0.f, a2 = 0.f, a3 = 0.f;
          for (int c = 0; c < ub - u1lo; c += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wr + c);
            const uint32_t o = o1 + 16u * (uint32_t)c;
            a0 = fmaf(w4.x, ld_bf16(sH1, o), a0);
            a1 = fmaf(w4.y, ld_bf16(sH1, o + 16u), a1);
            a2 = fmaf(w4.z, ld_bf16(sH1, o + 32u), a2);
            a3 = fmaf(w4.w, ld_bf16(sH1, o + 48u), a3);
          }
          st_bf16(sH2, rb2 + 16u * (uint32_t)(v - w2), fmaxf((a0 + a1) + (a2 + a3), 0.f));
        }
        float x;
        {
          const float* wr = TWo + q * so;
          const uint32_t o2 = rb2 + 16u * (uint32_t)(u2lo - w2);
          float a0 = __uint_as_float(rc) + gbo[q], a1 = 0.f, a2 = 0.f, a3 = 0.f;
          for (int c = 0; c < vb - u2lo; c += 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wr + c);
            const uint32_t o = o2 + 16u * (uint32_t)c;
            a0 = fmaf(w4.x, ld_bf16(sH2, o), a0);
            a1 = fmaf(w4.y, ld_bf16(sH2, o + 16u), a1);
            a2 = fmaf(w4.z, ld_bf16(sH2, o + 32u), a2);
            a3 = fmaf(w4.w, ld_bf16(sH2, o + 48u), a3);
          }
          x = (a0 + a1) + (a2 + a3);
        }
        // one exponential for both sigmoid(x) and softplus(-s x) (fast-math forms:
        // this kernel is the reduced-precision mode)
        const float ex = __expf(-fabsf(x));  // in (0, 1]
        const float rcp = __frcp_rn(1.f + ex);
        const float pr = x >= 0.f ? rcp : ex * rcp;
        const uint32_t word = (i & 3) == 0 ? rnd.x : (i & 3) == 1 ? rnd.y : (i & 3) == 2 ? rnd.z : rnd.w;
        const float u = (float)(word >> 8) * 5.9604644775390625e-08f;
        bool up = u < pr;
        if (gv) up = valid ? gv[i] > 0 : true;
        const float s = up ? 1.f : -1.f;
  #pragma unroll
        for (int j = 0; j < STC_GI; ++j) sg[j] = j == q ? s : sg[j];
        if (up) {
          if (i < 64) sb0 |= 1ull << i;
          else if (i < 128) sb1 |= 1ull << (i - 64);  // wider rows are written from the spin tile
        }
        st_bf16(sS, rbS + 16u * (uint32_t)i, s);
        lq -= fmaxf(-s * x, 0.f) + __logf(1.f + ex);
      }
    } else {
      SlotState st{rnd, 0u, lq};
      if (P.slot_u == 2)
        slot_group<2>(G, TWb, gi, i0, w1, w2, tP1, tP2, tPO, p1ok, init2, inito, sH1, sH2, sS, rb1, rb2, rbS, b,
                      step32, k, key, gv, valid, st);
      else if (P.slot_u == 3)
        slot_group<3>(G, TWb, gi, i0, w1, w2, tP1, tP2, tPO, p1ok, init2, inito, sH1, sH2, sS, rb1, rb2, rbS, b,
                      step32, k, key, gv, valid, st);
      else
        slot_group<4>(G, TWb, gi, i0, w1, w2, tP1, tP2, tPO, p1ok, init2, inito, sH1, sH2, sS, rb1, rb2, rbS, b,
                      step32, k, key, gv, valid, st);
      rnd = st.rnd;
      lq = st.lq;
      // the group's spin bits (at most 8, from bit i0) into the 128-bit mask
      const unsigned long long gb64 = st.gbits;
      if (i0 < 64) {
        sb0 |= gb64 << i0;
        if (i0 > 56) sb1 |= gb64 >> (64 - i0);
      } else if (i0 < 128) {  // wider rows are written from the spin tile
        sb1 |= gb64 << (i0 - 64);
      }
    }
    // fold the group; recompute P1g for the next group
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (g + 1 < P.n_groups) {
      if (mbar_wait(cbar, cphase)) {  // the next group's record (issued at this group's start)
        cphase ^= 1u;
        copy_pending = false;
      } else {
        ok = false;
      }
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      const int* Gn = reinterpret_cast<const int*>(gbn);
      const int w1n = Gn[2] & ~15, n1n = ((Gn[3] + 15) & ~15) - w1n;
      const int kS = (i1 + 15) & ~15;  // spins 0 .. i1-1 (zero beyond)
      if (t == 0) {
        const uint32_t aS = smem_u32(sS), aH1 = smem_u32(sH1), aH2 = smem_u32(sH2);
        // the B operands: windows of the resident tiles, or this group's blob
        // (W2 window, Wo window) and the next group's (W1 rows)
        const uint32_t aB = smem_u32(smem + (g & 1) * wbuf), aBn = smem_u32(smem + ((g + 1) & 1) * wbuf);
        uint32_t pa = 0, pb = 0, pc = 0, na = 0, nbn = 0, nc = 0;
        if (streamed) {
          blob_parts(G, pa, pb, pc);
          blob_parts(Gn, na, nbn, nc);
        }
        for (int kk = 0; kk < n1 / 16; ++kk)
          tc::mma_bf16(tmem + (uint32_t)P.tcw1, tc::smem_desc(aH1 + kk * 256u, 128u, sbo1),
                       streamed ? tc::smem_desc(aB + (uint32_t)kk * 256u, 128u, (uint32_t)n1 * 16u)
                                : tc::smem_desc(smem_u32(sW2) + (uint32_t)((w1 >> 4) + kk) * 256u, 128u, kbW2),
                       id2, (init2 || kk > 0) ? 1u : 0u);
        for (int kk = 0; kk < n2 / 16; ++kk)
          tc::mma_bf16(tmem + (uint32_t)(P.tcw1 + H2), tc::smem_desc(aH2 + kk * 256u, 128u, sbo2),
                       streamed ? tc::smem_desc(aB + pa + (uint32_t)kk * 256u, 128u, (uint32_t)n2 * 16u)
                                : tc::smem_desc(smem_u32(sWo) + (uint32_t)((w2 >> 4) + kk) * 256u, 128u, kbWo),
                       ido, (inito || kk > 0) ? 1u : 0u);
        if (n1n > 0) {
          const uint32_t id1 = tc::idesc(128, n1n, 1u) | idA;
          for (int kk = 0; kk < kS / 16; ++kk)
            tc::mma_bf16(tmem,
                         tc::smem_desc(aS + kk * 256u, 128u, sboS),
                         streamed ? tc::smem_desc(aBn + na + nbn + (uint32_t)kk * 256u, 128u, (uint32_t)kS * 16u)
                                  : tc::smem_desc(smem_u32(sW1) + (uint32_t)(w1n >> 3) * kbW1 + (uint32_t)kk * 256u,
                                                  128u, kbW1),
                         id1, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
      }
      mma_pending = true;
      init2 = init2 || n1 > 0;
      inito = inito || n2 > 0;
      p1ok = n1n > 0;
    }
  }
  if (!ok) {
    // give the work still in flight a bounded time to finish before TMEM is freed
    if (mma_pending) mbar_wait(bar, phase);
    if (copy_pending) mbar_wait(cbar, cphase);
    if (t == 0) atomicExch(li.status, 4);
  }
  if (ok && valid) {
    if (spins) {
      int8_t* row = spins + I.spin_units * li.batch + (long long)b * D;
      // rows of more than 128 spins: from the spin tile
      auto up_at = [&](int ii) {
        if (ANY_STREAMED && D > 128) return ld_bf16(sS, rbS + 16u * (uint32_t)ii) > 0.f;
        return ii < 64 ? ((sb0 >> ii) & 1ull) != 0 : ((sb1 >> (ii - 64)) & 1ull) != 0;
      };
      if ((D & 3) == 0 && (reinterpret_cast<uintptr_t>(row) & 3) == 0) {  // four spins per store
        uint32_t* out = reinterpret_cast<uint32_t*>(row);
        for (int i = 0; i < D; i += 4) {
          uint32_t v = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) v |= (up_at(i + j) ? 0x01u : 0xFFu) << (8 * j);
          out[i >> 2] = v;
        }
      } else {  // rows of other lengths or offsets: one byte per spin, none past the row
        for (int i = 0; i < D; ++i) row[i] = up_at(i) ? 1 : -1;
      }
    }
    logq[(long long)k * li.batch + b] = lq;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, (uint32_t)ncols);
}

int sample_tcg_smem_bytes(int D, int H1, int H2, int tcw1, int tcw2, int twmax, int wbmax) {
  const int need = sample_tcg_layout(D, H1, H2, tcw1, tcw2, twmax, wbmax).total;
  // never more resident CTAs per SM than the TMEM columns allow (228 KB of
  // shared memory per SM, 1 KB of it reserved per CTA)
  const int per_sm = sample_tcg_tmem_cols(D, H2, tcw1) <= 256 ? 2 : 1;
  const int floor_bytes = 228 * 1024 / (per_sm + 1) - 1024 + 16;
  return need > floor_bytes ? need : floor_bytes;
}

// Blocks [blk_begin, blk_end) of the launch (blk_end < 0: all).
cudaError_t launch_sample_tcg(const InstDev* d_inst, const LaunchInfo& li, const TcgOrder& ord, int plan,
                              int smem_bytes, bool streamed, int8_t* spins, float* logq, const int8_t* given,
                              cudaStream_t s, int blk_begin, int blk_end) {
  if (blk_end < 0) blk_end = li.tile_begin[li.n_inst];
  const int nblk = blk_end - blk_begin;
  if (nblk <= 0) return cudaSuccess;
  auto kern = streamed ? sample_tcg_kernel<true> : sample_tcg_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  LaunchInfo lc = li;
  lc.blk0 = blk_begin;
  kern<<<nblk, 128, smem_bytes, s>>>(d_inst, lc, ord, plan, spins, logq, given);
  return cudaGetLastError();
}

}  // namespace tnvan
