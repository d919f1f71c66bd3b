// BF16 ancestral sampler on tcgen05 (Eq. 6-8) for MADE networks with one or
// two hidden layers of at most 256 units (multiples of 16) and at most 256
// width-set spins (padded to Dp, a multiple of 16).
//
// One CTA (128 threads, thread = sample = TMEM lane) draws 128 samples, one
// step i (spin i) at a time, with one round trip to the tensor cores per
// step.  Hidden units are sorted by degree, so the units a step completes are
// a contiguous range of each layer.  At step i
//   L1:  layer-1 units [c1(i-1), c1(i)): pre-activations from TMEM (P1c: every
//        spin before i) + bias, rectified, written as BF16 into a delta tile
//        that holds only this step's units;
//   L2:  layer-2 units [c2(i-1), c2(i)): P2 from TMEM (every layer-1 unit of
//        an earlier step) + bias + this step's layer-1 units on the CUDA cores
//        (a per-step FP32 weight table), rectified, into a second delta tile;
//   out: x_i = PO[:, i] (every layer-2 unit of an earlier step) + b_i + this
//        step's layer-2 units on the CUDA cores; s_i = +1 iff u < sigmoid(x_i),
//        written into the spin tile S and a one-column spin delta tile;
//   then one MMA batch folds the step into the TMEM accumulators for the
//   steps after it: P2 += H1delta W2win^T, PO += H2delta Wowin^T and
//   P1c += Sdelta W1win^T (at a chunk's last step P1c is instead recomputed
//   for the next chunk's layer-1 units from every spin so far, P1c = S W1c'^T).
// With one hidden layer the output takes layer 1's place (PO += H1delta
// Wowin^T).  TMEM holds P1c [128 x tcw1] (the chunk's layer-1 units, <= 64),
// P2 [128 x H2] and PO [128 x Dp]: <= 256 columns gives two CTAs per SM.
// Steps are grouped into chunks; the weights a chunk's MMAs read -- the
// K-windows of W2 and Wo over the chunk's units and W1's rows of the chunk's
// layer-1 units -- are one BF16 blob per chunk in the MMA's K-major canonical
// layout, bulk-copied (TMA 1-D) one chunk ahead into a double buffer, so the
// shared-memory footprint does not grow with the network.
// Every hidden value and spin enters every product as BF16 with FP32
// accumulation (the reduced-precision mode); biases, the in-step products and
// the sigmoid are FP32.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tnvan {

namespace {

// MN-major spin tile of 128 rows (samples) and Dp columns: element (m, k) at
// (m >> 3) * sbo + (m & 7) * 2 + 16 k, sbo = 16 Dp + 16 (8-sample groups 16
// bytes apart modulo 128: one-element-per-thread stores are conflict free).
__host__ __device__ __forceinline__ uint32_t mn_sbo(int kw) { return (uint32_t)kw * 16u + 16u; }
__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t o, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + o) = __float2bfloat16(v);
}
__device__ __forceinline__ float ld_bf16(const unsigned char* base, uint32_t o) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + o));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// 16 consecutive TMEM columns of this thread's lane, waited.
__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])::"memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ float tmem_ld1w(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r)::"memory");
  return __uint_as_float(r);
}

// One 16-unit slice of a delta tile: units w16 .. w16+15 of a layer, of which
// those in [ua, ub) are this step's; value = ReLU(pre + bias), the rest 0;
// written as this thread's 32-byte row slice of the K-major tile.
__device__ __forceinline__ void delta_slice(const float (&pre)[16], const float* bias, int w16, int ua,
                                            int ub, unsigned char* row) {
  uint32_t pk[8];
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const int u0 = w16 + j, u1 = u0 + 1;
    const float h0 = (u0 >= ua && u0 < ub) ? fmaxf(pre[j] + bias[u0], 0.f) : 0.f;
    const float h1 = (u1 >= ua && u1 < ub) ? fmaxf(pre[j + 1] + bias[u1], 0.f) : 0.f;
    pk[j >> 1] = pack_bf16x2(h0, h1);
  }
  *reinterpret_cast<uint4*>(row) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  *reinterpret_cast<uint4*>(row + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

}  // namespace

const int kTcGroupMax[TNVAN_TC_PLANS] = {12, 16, 32};

struct SampleTcLayout {
  int oS, oSd, oD1, oD2, oBuf, buf, oStat, oBar, total;
};

// Shared memory of one CTA: S [16 x sbo(Dp)], the spin delta tile (K-major
// 128 x 16), the layer delta tiles (K-major 128 x dw1, 128 x dw2), two chunk
// weight buffers, the per-step tables (c1, c2, step table offsets [Dp + 1]
// ints; biases b1 [H1], b2 [H2], bo [Dp] floats; chunk records; the in-step
// weight tables [n_steptab] floats), the barriers.
__host__ __device__ inline SampleTcLayout sample_tc_layout(int Dp, int dw1, int dw2, int wbmax, int H1, int H2,
                                                           int n_chunks, int n_steptab) {
  SampleTcLayout L;
  int p = 0;
  L.oS = p;
  p += 16 * (int)mn_sbo(Dp);
  p = (p + 127) & ~127;
  L.oSd = p;
  p += 128 * 16 * 2;
  L.oD1 = p;
  p += 128 * dw1 * 2;
  L.oD2 = p;
  p += 128 * dw2 * 2;
  L.oBuf = p;
  L.buf = (wbmax + 127) & ~127;
  p += 2 * L.buf;
  L.oStat = p;
  p += 4 * (3 * (Dp + 1) + H1 + H2 + Dp + TNVAN_TCG_INTS * n_chunks + n_steptab);
  p = (p + 15) & ~15;
  L.oBar = p;
  p += 32;
  L.total = p;
  return L;
}

template <int NH>
__global__ void __launch_bounds__(128, 2) sample_tc_kernel(const InstDev* __restrict__ inst,
                                                           const LaunchInfo li, int plan,
                                                           int8_t* __restrict__ spins, float* __restrict__ logq,
                                                           const int8_t* __restrict__ given) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int gblk = blockIdx.x + li.blk0;
  const int k = find_inst(li, gblk);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const MadeDev::TcPlan& P = md.tc[plan];
  const int D = md.D, Dp = P.dp, H1 = md.H1, H2 = NH == 2 ? md.H2 : 0;
  const int t = threadIdx.x, w = t >> 5;
  const int b = (gblk - li.tile_begin[k]) * 128 + t;
  const bool valid = b < li.batch;
  const SampleTcLayout LY = sample_tc_layout(Dp, P.dw1, NH == 2 ? P.dw2 : 0, P.wbmax, H1, H2, P.n_chunks, P.n_steptab);
  unsigned char* sS = smem + LY.oS;
  unsigned char* sSd = smem + LY.oSd;
  unsigned char* sD1 = smem + LY.oD1;
  unsigned char* sD2 = smem + LY.oD2;
  unsigned char* wbuf0 = smem + LY.oBuf;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + LY.oBar);  // MMA completion
  uint64_t* cbar = bar + 1;                                     // bulk copies
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 2);
  const uint32_t sboS = mn_sbo(Dp);
  const uint32_t rbS = (uint32_t)(t >> 3) * sboS + (uint32_t)(t & 7) * 2u;  // element k of this row at rbS + 16 k
  // this thread's row in a K-major tile of width dw: (t >> 3) * 16 dw + (t & 7) * 16
  unsigned char* rowSd = sSd + (t >> 3) * 256 + (t & 7) * 16;
  unsigned char* rowD1 = sD1 + (t >> 3) * 16 * P.dw1 + (t & 7) * 16;
  unsigned char* rowD2 = sD2 + (t >> 3) * 16 * (NH == 2 ? P.dw2 : 0) + (t & 7) * 16;
  const int ncols = P.tmem_cols;
  // per-step tables in shared memory: units of degree <= d (c1, c2), the
  // degree-sorted biases, the chunk records
  int* c1 = reinterpret_cast<int*>(smem + LY.oStat);
  int* c2 = c1 + Dp + 1;
  float* b1 = reinterpret_cast<float*>(c2 + Dp + 1);
  float* b2 = b1 + H1;
  float* bo = b2 + H2;
  int* chunks = reinterpret_cast<int*>(bo + Dp);
  int* soff = chunks + TNVAN_TCG_INTS * P.n_chunks;  // step i's in-step table at stab + soff[i]
  float* stab = reinterpret_cast<float*>(soff + Dp + 1);
  {
    const float* gb1 = md.packed + md.layer[0].dst_off + (long long)H1 * D;
    const float* gb2 = NH == 2 ? md.packed + md.layer[1].dst_off + (long long)H2 * H1 : nullptr;
    const float* gbo = md.packed + md.layer[NH].dst_off + (long long)D * (NH == 2 ? H2 : H1);
    for (int j = t; j <= D; j += 128) {
      c1[j] = md.c1[j];
      c2[j] = NH == 2 ? md.c2[j] : 0;
    }
    for (int j = t; j < H1; j += 128) b1[j] = gb1[j];
    for (int j = t; j < H2; j += 128) b2[j] = gb2[j];
    for (int j = t; j < D; j += 128) bo[j] = gbo[j];
    for (int j = t; j < TNVAN_TCG_INTS * P.n_chunks; j += 128) chunks[j] = P.chunks[j];
    for (int j = t; j <= D; j += 128) soff[j] = P.stepoff[j];
    for (int j = t; j < P.n_steptab; j += 128) stab[j] = P.steptab[j];
  }
  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  if (w == 0) {
    tc::tmem_alloc(slot, (uint32_t)ncols);
    tc::tmem_relinquish();
  }
  // spin tile and delta tiles start at zero
  for (int o = t * 16; o < LY.oBuf; o += 128 * 16) *reinterpret_cast<uint4*>(smem + o) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // chunk cc's weight blob into its buffer (one thread)
  auto copy_chunk = [&](int cc) {
    const int* R = P.chunks + TNVAN_TCG_INTS * cc;
    const uint32_t wb = (uint32_t)(__ldg(R + 8) + __ldg(R + 9) + __ldg(R + 10));
    mbar_expect_tx(cbar, wb);
    bulk_g2s(wbuf0 + (cc & 1) * LY.buf, P.wblob + __ldg(R + 7), wb, cbar);
  };
  const uint32_t tmem = *slot;
  const uint32_t lane_off = (uint32_t)(w * 32) << 16;
  const uint32_t tP1 = tmem + lane_off, tP2 = tP1 + (uint32_t)P.tcw1, tPO = tP2 + (uint32_t)H2;
  const uint32_t colP2 = (uint32_t)P.tcw1, colPO = (uint32_t)(P.tcw1 + H2);
  const uint32_t idP2 = NH == 2 ? tc::idesc(128, H2, 1u) : 0u, idPO = tc::idesc(128, Dp, 1u);
  const uint2 key = make_uint2((uint32_t)li.seed, (uint32_t)(li.seed >> 32));
  const uint32_t step32 = launch_step(li);
  const int8_t* gv = given ? given + I.spin_units * li.batch + (long long)b * D : nullptr;
  uint32_t phase = 0, cphase = 0;
  bool ok = true, mma_pending = false, copy_pending = false;
  bool p1ok = false, init2 = false, inito = false;  // accumulators hold data
  float lq = 0.f;
  uint4 rnd = make_uint4(0, 0, 0, 0);
  // every phase starts once the MMAs queued so far have completed
  auto wait_mma = [&]() {
    if (mma_pending) {
      if (mbar_wait(bar, phase)) {
        phase ^= 1u;
      } else {
        ok = false;
      }
      mma_pending = false;
      tc::fence_after_sync();
    }
  };
  // the threads' shared-memory writes visible to the tensor core
  auto sync_for_mma = [&]() {
    fence_proxy_async_smem();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
  };
  if (t == 0) copy_chunk(0);
  copy_pending = true;
  int cidx = 0;
  const int* R = chunks;
  int ci0 = R[0], ci1 = R[1], w1c = R[2], w2c = R[4];
  uint32_t aW = 0, aWo = 0, aW1 = 0;  // this chunk's blob: W2 window | Wo window | W1 rows
  int kSc = R[6];
  for (int i = 0; i < D && ok; ++i) {
    if (i == ci0) {  // a new chunk: its blob has arrived; the one after it goes to the other buffer
      if (copy_pending) {
        if (mbar_wait(cbar, cphase)) cphase ^= 1u;
        else ok = false;
        copy_pending = false;
      }
      aW = smem_u32(wbuf0 + (cidx & 1) * LY.buf);
      aWo = aW + (uint32_t)R[8];
      aW1 = aWo + (uint32_t)R[9];
      if (cidx + 1 < P.n_chunks) {
        wait_mma();  // the previous chunk's MMAs (the other buffer) are done
        if (t == 0) copy_chunk(cidx + 1);
        copy_pending = true;
      }
    }
    if ((i & 3) == 0) rnd = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(i >> 2), step32, (uint32_t)k), key);
    wait_mma();  // the previous step's fold: P1c, P2 and PO include every earlier step
    const float* T = stab + soff[i];  // this step's in-step weights
    // ---- layer 1: units [ua, ub) ----
    const int ua = i > 0 ? c1[i - 1] : 0, ub = c1[i];
    const int w1s = ua & ~15, n1s = ub > ua ? ((ub + 15) & ~15) - w1s : 0;
    for (int s = 0; s < n1s; s += 16) {
      float pre[16];
      if (p1ok) {
        tmem_ld16w(tP1 + (uint32_t)(w1s + s - w1c), pre);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) pre[j] = 0.f;
      }
      delta_slice(pre, b1, w1s + s, ua, ub, rowD1 + s * 16);
    }
    // h1 of this step's unit u, as written (BF16) into the delta tile
    auto h1_of = [&](int u) {
      const int kk = u - w1s;
      return ld_bf16(rowD1, (uint32_t)((kk >> 3) * 128 + (kk & 7) * 2));
    };
    // ---- layer 2: units [va, vb) ----
    int va = 0, vb = 0, w2s = 0, n2s = 0;
    if (NH == 2) {
      va = i > 0 ? c2[i - 1] : 0;
      vb = c2[i];
      w2s = va & ~15;
      n2s = vb > va ? ((vb + 15) & ~15) - w2s : 0;
      const int nu = ub - ua;
      for (int s = 0; s < n2s; s += 16) {
        float pre[16];
        if (init2) {
          tmem_ld16w(tP2 + (uint32_t)(w2s + s), pre);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) pre[j] = 0.f;
        }
        // + this step's layer-1 units (T: [vb - va][nu]), for the units of
        // this slice: one dot product per unit, added into its register
        const int v0 = max(va, w2s + s), v1 = min(vb, w2s + s + 16);
        for (int v = v0; v < v1; ++v) {
          const float* tr = T + (v - va) * nu;
          float acc = 0.f;
          for (int u = ua; u < ub; ++u) acc = fmaf(tr[u - ua], h1_of(u), acc);
          const int jv = v - (w2s + s);
#pragma unroll
          for (int j = 0; j < 16; ++j) pre[j] += j == jv ? acc : 0.f;
        }
        delta_slice(pre, b2, w2s + s, va, vb, rowD2 + s * 16);
      }
    }
    // ---- output i and the draw ----
    float x = (inito ? tmem_ld1w(tPO + (uint32_t)i) : 0.f) + bo[i];
    if (NH == 2) {  // + this step's layer-2 units (T after the layer-2 block: [vb - va])
      const float* to = T + (vb - va) * (ub - ua);
      for (int v = va; v < vb; ++v) {
        const int kk = v - w2s;
        x = fmaf(to[v - va], ld_bf16(rowD2, (uint32_t)((kk >> 3) * 128 + (kk & 7) * 2)), x);
      }
    } else {  // + this step's layer-1 units (T: [ub - ua])
      for (int u = ua; u < ub; ++u) x = fmaf(T[u - ua], h1_of(u), x);
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
    const float sv = up ? 1.f : -1.f;
    lq -= fmaxf(-sv * x, 0.f) + __logf(1.f + ex);
    st_bf16(sS, rbS + 16u * (uint32_t)i, sv);
    if (i + 1 >= D) break;
    // ---- fold step i for the steps after it: one MMA batch, one commit ----
    const bool last_of_chunk = i + 1 == ci1;
    int n1c_next = 0;
    if (last_of_chunk) {
      ++cidx;
      R = chunks + TNVAN_TCG_INTS * cidx;
      n1c_next = R[3];
      if (copy_pending) {  // the next chunk's blob (issued at this chunk's start)
        if (mbar_wait(cbar, cphase)) cphase ^= 1u;
        else ok = false;
        copy_pending = false;
      }
    } else {  // spin i alone in the spin delta tile
      const int j = i & 15;
      uint32_t pk[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) pk[q] = pack_bf16x2((2 * q == j) ? sv : 0.f, (2 * q + 1 == j) ? sv : 0.f);
      *reinterpret_cast<uint4*>(rowSd) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      *reinterpret_cast<uint4*>(rowSd + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    sync_for_mma();
    if (!ok) break;
    const int n1c = R[3];  // after a chunk change: the next chunk's
    if (t == 0) {
      const uint32_t aD1 = smem_u32(sD1), aD2 = smem_u32(sD2);
      if (n1s > 0) {  // this step's layer-1 units -> P2 (or PO)
        for (int kk = 0; kk < n1s / 16; ++kk) {
          if (NH == 2)
            tc::mma_bf16(tmem + colP2, tc::smem_desc(aD1 + kk * 256u, 128u, (uint32_t)P.dw1 * 16u),
                         tc::smem_desc(aW + (uint32_t)((w1s - w1c) / 16 + kk) * (uint32_t)(H2 * 32), 128u, 256u),
                         idP2, (init2 || kk > 0) ? 1u : 0u);
          else
            tc::mma_bf16(tmem + colPO, tc::smem_desc(aD1 + kk * 256u, 128u, (uint32_t)P.dw1 * 16u),
                         tc::smem_desc(aWo + (uint32_t)((w1s - w1c) / 16 + kk) * (uint32_t)(Dp * 32), 128u, 256u),
                         idPO, (inito || kk > 0) ? 1u : 0u);
        }
      }
      if (NH == 2 && n2s > 0) {  // this step's layer-2 units -> PO
        for (int kk = 0; kk < n2s / 16; ++kk)
          tc::mma_bf16(tmem + colPO, tc::smem_desc(aD2 + kk * 256u, 128u, (uint32_t)P.dw2 * 16u),
                       tc::smem_desc(aWo + (uint32_t)((w2s - w2c) / 16 + kk) * (uint32_t)(Dp * 32), 128u, 256u),
                       idPO, (inito || kk > 0) ? 1u : 0u);
      }
      if (last_of_chunk) {  // P1c of the next chunk's units from every spin so far
        if (n1c_next > 0) {
          const uint32_t aS = smem_u32(sS);
          const uint32_t aW1n = smem_u32(wbuf0 + (cidx & 1) * LY.buf) + (uint32_t)(R[8] + R[9]);
          const uint32_t id1 = tc::idesc(128, n1c_next, 1u) | (1u << 15);  // A (spin tile) MN-major
          for (int kk = 0; kk < (i + 1 + 15) / 16; ++kk)  // the spins drawn so far (zero beyond)
            tc::mma_bf16(tmem, tc::smem_desc(aS + kk * 256u, 128u, sboS),
                         tc::smem_desc(aW1n + (uint32_t)kk * 256u, 128u, (uint32_t)R[6] * 16u), id1, kk > 0 ? 1u : 0u);
        }
      } else if (n1c > 0) {  // spin i -> the chunk's layer-1 pre-activations
        tc::mma_bf16(tmem, tc::smem_desc(smem_u32(sSd), 128u, 256u),
                     tc::smem_desc(aW1 + (uint32_t)(i >> 4) * 256u, 128u, (uint32_t)kSc * 16u),
                     tc::idesc(128, n1c, 1u), p1ok ? 1u : 0u);
      }
      tc::mma_commit(bar);
    }
    mma_pending = true;
    if (n1s > 0) {
      if (NH == 2) init2 = true;
      else inito = true;
    }
    if (NH == 2 && n2s > 0) inito = true;
    if (last_of_chunk) {
      ci0 = R[0], ci1 = R[1], w1c = R[2], w2c = R[4], kSc = R[6];
      p1ok = n1c_next > 0;
    } else if (n1c > 0) {
      p1ok = true;
    }
  }
  wait_mma();
  if (!ok) {
    // give the copy still in flight a bounded time to finish before returning
    if (copy_pending) mbar_wait(cbar, cphase);
    if (t == 0) atomicExch(li.status, 4);
  }
  if (ok && valid) {
    if (spins) {  // the drawn spins, from the spin tile
      int8_t* out = spins + I.spin_units * li.batch + (long long)b * D;
      if ((D & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 3) == 0) {
        for (int i = 0; i < D; i += 4) {
          uint32_t v = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) v |= (ld_bf16(sS, rbS + 16u * (uint32_t)(i + j)) > 0.f ? 0x01u : 0xFFu) << (8 * j);
          *reinterpret_cast<uint32_t*>(out + i) = v;
        }
      } else {
        for (int i = 0; i < D; ++i) out[i] = ld_bf16(sS, rbS + 16u * (uint32_t)i) > 0.f ? 1 : -1;
      }
    }
    logq[(long long)k * li.batch + b] = lq;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, (uint32_t)ncols);
}

// Shared memory of the plan's CTAs: at least the layout, and never more
// resident CTAs per SM than the TMEM columns allow (228 KB of shared memory
// per SM, 1 KB of it reserved per CTA).
int sample_tc_smem_bytes(const MadeDev& md, int plan) {
  const MadeDev::TcPlan& P = md.tc[plan];
  const int need =
      sample_tc_layout(P.dp, P.dw1, md.nh == 2 ? P.dw2 : 0, P.wbmax, md.H1, md.nh == 2 ? md.H2 : 0, P.n_chunks,
                       P.n_steptab).total;
  const int per_sm = P.tmem_cols <= 128 ? 4 : (P.tmem_cols <= 256 ? 2 : 1);
  const int floor_bytes = 228 * 1024 / (per_sm + 1) - 1024 + 16;
  return need > floor_bytes ? need : floor_bytes;
}

// Blocks [blk_begin, blk_end) of the launch (blk_end < 0: all); nh = the
// instances' number of hidden layers (1 or 2, the same for every instance).
cudaError_t launch_sample_tc(const InstDev* d_inst, const LaunchInfo& li, int plan, int nh, int smem_bytes,
                             int8_t* spins, float* logq, const int8_t* given, cudaStream_t s, int blk_begin,
                             int blk_end) {
  if (blk_end < 0) blk_end = li.tile_begin[li.n_inst];
  const int nblk = blk_end - blk_begin;
  if (nblk <= 0) return cudaSuccess;
  LaunchInfo lc = li;
  lc.blk0 = blk_begin;
  cudaError_t e;
  if (nh == 2) {
    e = cudaFuncSetAttribute(sample_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    sample_tc_kernel<2><<<nblk, 128, smem_bytes, s>>>(d_inst, lc, plan, spins, logq, given);
  } else {
    e = cudaFuncSetAttribute(sample_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    sample_tc_kernel<1><<<nblk, 128, smem_bytes, s>>>(d_inst, lc, plan, spins, logq, given);
  }
  return cudaGetLastError();
}

}  // namespace tnvan
