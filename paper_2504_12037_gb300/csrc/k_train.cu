// Reduction to F_q / log Z_IS (Eq. 9), REINFORCE backward of the network
// (Eq. 10) and the Adam update (Algorithm 1 step (d)).
#include <math.h>

#include "common.cuh"

namespace tnvan {

// ---------------------------------------------------------------------------
// K7, two-pass FP64 form (the allocation-free entry point's reduction): per
// instance, over l_b = log Z_R(s_b) - log q(s_b).
// Pass 1 (grid n_part x n_inst): each CTA reduces a contiguous chunk to the
// mergeable tuple (n, mean, M2, max l, sum exp(l - max), #non-finite):
// Welford's update per sample, the pairwise update of Chan, Golub and
// LeVeque to merge (no shift taken from any one sample, so a non-finite
// first sample cannot spoil the sums).
// Pass 2 (grid n_inst): merges the n_part tuples in order and writes
//   stats[8k + 0..7] = F_q, F_IS, stderr, logZ_IS, mean l, #non-finite, var l, n;
// with no finite l_b every statistic is NaN and n = 0.
// Non-finite l_b are counted and left out.  FP64 throughout.
// ---------------------------------------------------------------------------
struct Tuple {
  double n, mean, M2, m, se, bad;
};

__device__ __forceinline__ Tuple merge(Tuple a, Tuple b) {
  if (a.n == 0.0) {
    b.bad += a.bad;
    return b;
  }
  if (b.n == 0.0) {
    a.bad += b.bad;
    return a;
  }
  Tuple r;
  r.n = a.n + b.n;
  const double d = b.mean - a.mean;
  r.mean = a.mean + d * (b.n / r.n);
  r.M2 = a.M2 + b.M2 + d * d * (a.n * b.n / r.n);
  r.bad = a.bad + b.bad;
  r.m = fmax(a.m, b.m);
  r.se = a.se * exp(a.m - r.m) + b.se * exp(b.m - r.m);
  return r;
}

__device__ __forceinline__ Tuple shfl_tuple(Tuple t, int o) {
  Tuple r;
  r.n = __shfl_xor_sync(0xffffffffu, t.n, o);
  r.mean = __shfl_xor_sync(0xffffffffu, t.mean, o);
  r.M2 = __shfl_xor_sync(0xffffffffu, t.M2, o);
  r.m = __shfl_xor_sync(0xffffffffu, t.m, o);
  r.se = __shfl_xor_sync(0xffffffffu, t.se, o);
  r.bad = __shfl_xor_sync(0xffffffffu, t.bad, o);
  return r;
}

__global__ void __launch_bounds__(256) reduce_part_kernel(const LaunchInfo li, int n_part,
                                                          const double* __restrict__ logZR,
                                                          const float* __restrict__ logq,
                                                          double* __restrict__ part) {
  const int k = blockIdx.y, p = blockIdx.x, B = li.batch;
  const long long base = (long long)k * B;
  const int chunk = (B + n_part - 1) / n_part;
  const int lo = p * chunk, hi = min(B, lo + chunk);
  Tuple acc = {0, 0, 0, 0, 0, 0};
  for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
    const double l = logZR[base + b] - (double)logq[base + b];
    if (!isfinite(l)) {
      acc.bad += 1.0;
      continue;
    }
    acc.n += 1.0;
    const double d = l - acc.mean;
    acc.mean += d / acc.n;
    acc.M2 += d * (l - acc.mean);
    if (acc.n == 1.0) {
      acc.m = l;
      acc.se = 1.0;
    } else if (l > acc.m) {
      acc.se = acc.se * exp(acc.m - l) + 1.0;
      acc.m = l;
    } else {
      acc.se += exp(l - acc.m);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc = merge(acc, shfl_tuple(acc, o));
  __shared__ Tuple red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    Tuple r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = merge(r, red[w]);
    double* o = part + ((long long)k * n_part + p) * 6;
    o[0] = r.n;
    o[1] = r.mean;
    o[2] = r.M2;
    o[3] = r.m;
    o[4] = r.se;
    o[5] = r.bad;
  }
}

__global__ void reduce_final_kernel(const LaunchInfo li, int n_part, const double* __restrict__ part,
                                    double* __restrict__ stats) {
  const int k = blockIdx.x;
  if (threadIdx.x != 0) return;
  Tuple r = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < n_part; ++p) {
    const double* o = part + ((long long)k * n_part + p) * 6;
    Tuple t = {o[0], o[1], o[2], o[3], o[4], o[5]};
    r = merge(r, t);
  }
  double* s = stats + 8 * k;
  s[5] = r.bad;
  s[7] = r.n;
  if (r.n == 0.0) {  // no finite l_b: nothing to estimate
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    s[0] = s[1] = s[2] = s[3] = s[4] = s[6] = nan;
    return;
  }
  const double beta = li.beta[k];
  const double n = r.n;
  const double var = n > 1.0 ? r.M2 / (n - 1.0) : 0.0;
  const double lz = r.m + log(r.se) - log(n);
  s[0] = -r.mean / beta;
  s[1] = -lz / beta;
  s[2] = sqrt(var) / (beta * sqrt(n));
  s[3] = lz;
  s[4] = r.mean;
  s[6] = var;
}

// ---------------------------------------------------------------------------
// The same reduction in one launch (the context's form): the moment sums of
// l - K in float-float arithmetic -- each value an unevaluated sum hi + lo of
// two floats (error-free transforms: Knuth's TwoSum, Dekker's FastTwoSum, the
// FMA product error), about 48 significant bits, because FP64 is a narrow
// unit on this part -- and the logsumexp of the importance weights (log Z_IS)
// in FP64, about one FP64 exp per sample; the final statistics in FP64.
// Every CTA reduces its chunk and counts itself done on counters[k]; the
// last CTA of an instance merges the instance's n_part (<= 64) tuples with
// one warp -- a fixed tree over the chunk index, so the result does not
// depend on which CTA finishes last -- writes the statistics and re-arms the
// counter.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  FF s = ff_two_sum(x.hi, y.hi);
  const FF t = ff_two_sum(x.lo, y.lo);
  s = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ bool ff_gt(FF a, FF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// double -> float-float with integer operations: hi = the top 24 significand
// bits (truncated, exact), lo = the next 29 bits rounded to a float.
__device__ __forceinline__ FF ff_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const int E = (int)((u >> 52) & 0x7FFull);
  const int fe = E - 1023 + 127;
  if (E == 0x7FF) return FF{x != x ? __int_as_float(0x7FC00000) : __int_as_float((int)(sign | 0x7F800000u)), 0.f};
  if (fe <= 0 || fe >= 255) return FF{(float)x, 0.f};  // zero, tiny or huge: not met by log-likelihoods
  const unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | (unsigned)(M >> 29)));
  const int le = E - 1075 + 127;  // 2^(E - 1023 - 52)
  const float lo = le > 0 ? __uint2float_rn((unsigned)(M & 0x1FFFFFFFull)) * __int_as_float(le << 23) : 0.f;
  return FF{hi, sign ? -lo : lo};
}
__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

// s1, s2: float-float sums of l - K and (l - K)^2; m, se: the maximum of the
// importance weights' logs and the sum of exp(l - m), in FP64 (Eq. 9's log Z_IS
// is a logsumexp of the l_b, kept in FP64 throughout).
struct TupleFF {
  int n, bad;
  FF s1, s2;
  double m, se;
};
__device__ __forceinline__ FF shfl_ff(FF x, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}
// partial tuples in a 6-double slot: n, bad, s1, s2 in words 0..5, m and se
// in doubles 3 and 4
__device__ __forceinline__ void st_tuple_ff(double* slot, const TupleFF& t) {
  float* f = reinterpret_cast<float*>(slot);
  reinterpret_cast<int*>(f)[0] = t.n;
  reinterpret_cast<int*>(f)[1] = t.bad;
  f[2] = t.s1.hi, f[3] = t.s1.lo, f[4] = t.s2.hi, f[5] = t.s2.lo;
  slot[3] = t.m;
  slot[4] = t.se;
}
__device__ __forceinline__ TupleFF ld_tuple_ff(const double* slot) {
  const float* f = reinterpret_cast<const float*>(slot);
  const int* q = reinterpret_cast<const int*>(slot);
  return TupleFF{__ldcg(q), __ldcg(q + 1), FF{__ldcg(f + 2), __ldcg(f + 3)}, FF{__ldcg(f + 4), __ldcg(f + 5)},
                 __ldcg(slot + 3), __ldcg(slot + 4)};
}
// Block-wide reductions over the 256 threads (8 warps); `red` holds 8 values.
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < 8; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// Each CTA reduces a chunk in two passes over its samples: the chunk's
// largest l first (compares only), then per sample one FP64 exp(l - max) and
// the float-float moment sums; the CTA's warps are summed in a fixed order.
// The last CTA of an instance rescales the n_part (<= 64) chunk sums to the
// instance's largest l, one FP64 exp per chunk in parallel lanes, and adds
// them in a fixed tree, so the result does not depend on which CTA finishes
// last.  Only two exps lie on any thread's path: FP64 is a narrow unit on
// this part, and a running maximum with a rescale at every merge would put
// one exp per merge level on the critical path.
__global__ void __launch_bounds__(256) reduce_kernel(const LaunchInfo li, int n_part, const double* __restrict__ logZR,
                                                     const float* __restrict__ logq, double* __restrict__ part,
                                                     double* __restrict__ stats, int* __restrict__ counters,
                                                     int k0) {
  const int k = blockIdx.y + k0, p = blockIdx.x, B = li.batch;
  const long long base = (long long)k * B;
  // the shift of the moment sums: l_0 when finite (else 0)
  FF K = ff_add(ff_from_double(logZR[base]), FF{-logq[base], 0.f});
  if (!isfinite(K.hi) || !isfinite(K.lo)) K = FF{0.f, 0.f};
  const FF negK = ff_neg(K);
  const int chunk = (B + n_part - 1) / n_part;
  const int lo = p * chunk, hi = min(B, lo + chunk);
  __shared__ double redd[8];
  __shared__ TupleFF red[8];
  __shared__ int last;
  // pass 1: the chunk's largest finite l
  double mx = -INFINITY;
  for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
    const double ld = logZR[base + b] - (double)logq[base + b];
    if (isfinite(ld)) mx = fmax(mx, ld);
  }
  mx = block_max(mx, redd);
  // pass 2: exp sums against that maximum, moment sums, counts
  TupleFF acc = {0, 0, {0.f, 0.f}, {0.f, 0.f}, mx, 0.0};
  for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) {
    const double z = logZR[base + b];
    const float q = logq[base + b];
    const double ld = z - (double)q;
    if (!isfinite(ld)) {
      acc.bad += 1;
      continue;
    }
    const FF d = ff_add(ff_add(ff_from_double(z), FF{-q, 0.f}), negK);
    acc.s1 = ff_add(acc.s1, d);
    acc.s2 = ff_add(acc.s2, ff_mul(d, d));
    acc.se += exp(ld - mx);
    acc.n += 1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.n += __shfl_xor_sync(0xffffffffu, acc.n, o);
    acc.bad += __shfl_xor_sync(0xffffffffu, acc.bad, o);
    acc.s1 = ff_add(acc.s1, shfl_ff(acc.s1, o));
    acc.s2 = ff_add(acc.s2, shfl_ff(acc.s2, o));
    acc.se += __shfl_xor_sync(0xffffffffu, acc.se, o);
  }
  const int l = threadIdx.x & 31;
  if (l == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {  // the CTA's warps in order
    TupleFF r = red[0];
    for (int w = 1; w < 8; ++w) {
      r.n += red[w].n;
      r.bad += red[w].bad;
      r.s1 = ff_add(r.s1, red[w].s1);
      r.s2 = ff_add(r.s2, red[w].s2);
      r.se += red[w].se;
    }
    st_tuple_ff(part + ((long long)k * n_part + p) * 6, r);
    __threadfence();
    last = atomicAdd(counters + k, 1) == n_part - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // the instance's chunks: lane l holds chunks l and l + 32
  TupleFF r = {0, 0, {0.f, 0.f}, {0.f, 0.f}, -INFINITY, 0.0};
  TupleFF r2 = r;
  if (l < n_part) r = ld_tuple_ff(part + ((long long)k * n_part + l) * 6);
  if (l + 32 < n_part) r2 = ld_tuple_ff(part + ((long long)k * n_part + l + 32) * 6);
  double M = fmax(r.n ? r.m : -INFINITY, r2.n ? r2.m : -INFINITY);
  for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xffffffffu, M, o));
  double se = (r.n ? r.se * exp(r.m - M) : 0.0) + (r2.n ? r2.se * exp(r2.m - M) : 0.0);
  int n_ = r.n + r2.n, bad_ = r.bad + r2.bad;
  FF s1 = ff_add(r.s1, r2.s1), s2 = ff_add(r.s2, r2.s2);
  for (int o = 16; o > 0; o >>= 1) {
    n_ += __shfl_xor_sync(0xffffffffu, n_, o);
    bad_ += __shfl_xor_sync(0xffffffffu, bad_, o);
    s1 = ff_add(s1, shfl_ff(s1, o));
    s2 = ff_add(s2, shfl_ff(s2, o));
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  // FP64 statistics; the transcendental tails in parallel lanes
  const double beta = li.beta[k];
  const double n = (double)n_;
  const double s1d = ff_to_double(s1), s2d = ff_to_double(s2);
  const double mean_d = s1d / n;
  const double var = n_ > 1 ? fmax(s2d - s1d * mean_d, 0.0) / (n - 1.0) : 0.0;
  double f = 0.0;
  if (l == 1) f = log(se);
  else if (l == 2) f = log(n);
  else if (l == 3) f = sqrt(var);
  else if (l == 4) f = sqrt(n);
  const double lse = __shfl_sync(0xffffffffu, f, 1), ln_n = __shfl_sync(0xffffffffu, f, 2);
  const double sd = __shfl_sync(0xffffffffu, f, 3), sn = __shfl_sync(0xffffffffu, f, 4);
  if (l != 0) return;
  const double mean = ff_to_double(K) + mean_d;
  const double lz = M + lse - ln_n;
  double* st = stats + 8 * k;
  st[0] = -mean / beta;
  st[1] = -lz / beta;
  st[2] = sd / (beta * sn);
  st[3] = lz;
  st[4] = mean;
  st[5] = (double)bad_;
  st[6] = var;
  st[7] = n;
  counters[k] = 0;
}

cudaError_t launch_reduce(const InstDev*, const LaunchInfo& li, const double* logZR,
                          const float* logq, double* stats, int* counters, cudaStream_t s, int k0, int k1) {
  if (k1 < 0) k1 = li.n_inst;
  if (k1 <= k0) return cudaSuccess;
  // n_part: chunks of >= 256 samples, at most 64 per instance
  int n_part = (li.batch + 255) / 256;
  if (n_part > 64) n_part = 64;
  if (n_part < 1) n_part = 1;
  // partial tuples live right after the stats block
  double* part = stats + 8 * TNVAN_MAX_INST;
  reduce_kernel<<<dim3(n_part, k1 - k0), 256, 0, s>>>(li, n_part, logZR, logq, part, stats, counters, k0);
  return cudaGetLastError();
}

// Merge of Eq. 9 statistics rows computed on disjoint parts of one batch
// (data-parallel ranks), parts[(p * n_inst + k) * 8 + 0..7] in the layout of
// the reduction, into stats[8k + 0..7] for the union of the parts.  Each row
// is taken as the mergeable tuple (n, mean l, M2 = var (n - 1), log sum e^l =
// logZ_IS + ln n) and the parts are combined in index order by the pairwise
// update of Chan, Golub and LeVeque (1979) for the mean and M2 and a
// logaddexp for the log-sum; one thread per instance, so the result does not
// depend on the launch.  One part is copied unchanged.
__global__ void merge_stats_kernel(const LaunchInfo li, int n_parts, const double* __restrict__ parts,
                                   double* __restrict__ stats) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= li.n_inst) return;
  const double* p0 = parts + 8 * k;
  double* st = stats + 8 * k;
  if (n_parts == 1) {
    for (int j = 0; j < 8; ++j) st[j] = p0[j];
    return;
  }
  double n = 0.0, mean = 0.0, M2 = 0.0, lse = 0.0, bad = 0.0;
  for (int p = 0; p < n_parts; ++p) {
    const double* q = parts + ((long long)p * li.n_inst + k) * 8;
    const double nb = q[7];
    bad += q[5];
    if (!(nb > 0.0)) continue;
    const double mb = q[4], M2b = nb > 1.0 ? q[6] * (nb - 1.0) : 0.0, lb = q[3] + log(nb);
    if (n == 0.0) {
      n = nb, mean = mb, M2 = M2b, lse = lb;
      continue;
    }
    const double N = n + nb, d = mb - mean;
    mean += d * (nb / N);
    M2 += M2b + d * d * (n * nb / N);
    lse = fmax(lse, lb) + log1p(exp(-fabs(lse - lb)));
    n = N;
  }
  const double beta = li.beta[k];
  const double var = n > 1.0 ? M2 / (n - 1.0) : 0.0;
  const double lz = lse - log(n);
  st[0] = -mean / beta;
  st[1] = -lz / beta;
  st[2] = sqrt(var) / (beta * sqrt(n));
  st[3] = lz;
  st[4] = mean;
  st[5] = bad;
  st[6] = var;
  st[7] = n;
}

cudaError_t launch_merge_stats(const LaunchInfo& li, int n_parts, const double* parts, double* stats,
                               cudaStream_t s) {
  merge_stats_kernel<<<(li.n_inst + 127) / 128, 128, 0, s>>>(li, n_parts, parts, stats);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K2 + K3: teacher-forced forward and hand-written backward of
//   sum_b w_b log q(s_b),   w_b = -(l_b - mean l) / (beta B)       (Eq. 10)
// for a chunk of samples per CTA, 32 samples at a time (FP32 SIMT).
//   d log q / d x_i = s_i sigmoid(-s_i x_i)
// Shared memory, layout [unit][TP] with TP = 33:
//   S [D], A1 [H1], A2 [H2], X/dX [D], dA2 [H2], dA1 [H1].
// Weight-gradient partial sums of the chunk are accumulated in this CTA's
// slice of `partials` (packed, degree-sorted layout, n_params floats).
// ---------------------------------------------------------------------------
#define BW_TS 32
#define BW_TP 33

// G[M][N] (+)= sum_t A[m][t] Bm[n][t];  gb[M] (+)= sum_t A[m][t].
__device__ void outer_acc(float* __restrict__ G, float* __restrict__ gb, const float* A,
                          const float* Bm, int M, int N, int TS, bool first, int tid, int nth) {
  const int mb = (M + 3) >> 2, nb = (N + 3) >> 2;
  for (int blk = tid; blk < mb * nb; blk += nth) {
    const int i0 = (blk / nb) << 2, j0 = (blk % nb) << 2;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int t = 0; t < TS; ++t) {
      float a[4], bb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = (i0 + r < M) ? A[(i0 + r) * BW_TP + t] : 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) bb[c] = (j0 + c < N) ? Bm[(j0 + c) * BW_TP + t] : 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bb[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (i0 + r < M && j0 + c < N) {
          float* g = G + (long long)(i0 + r) * N + j0 + c;
          *g = first ? acc[r][c] : *g + acc[r][c];
        }
  }
  for (int m = tid; m < M; m += nth) {
    float s = 0.f;
    for (int t = 0; t < TS; ++t) s += A[m * BW_TP + t];
    gb[m] = first ? s : gb[m] + s;
  }
}

__device__ __forceinline__ float dot_row(const float* __restrict__ w, const float* col, int n) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int j = 0;
  for (; j + 4 <= n; j += 4) {
    a0 = fmaf(__ldg(w + j), col[j * BW_TP], a0);
    a1 = fmaf(__ldg(w + j + 1), col[(j + 1) * BW_TP], a1);
    a2 = fmaf(__ldg(w + j + 2), col[(j + 2) * BW_TP], a2);
    a3 = fmaf(__ldg(w + j + 3), col[(j + 3) * BW_TP], a3);
  }
  for (; j < n; ++j) a0 = fmaf(__ldg(w + j), col[j * BW_TP], a0);
  return (a0 + a1) + (a2 + a3);
}

// sum_{i = i0}^{n-1} col[i] * w[i * stride]
__device__ __forceinline__ float dot_strided(const float* __restrict__ w, long long stride,
                                             const float* col, int i0, int n) {
  float a0 = 0.f, a1 = 0.f;
  int i = i0;
  for (; i + 2 <= n; i += 2) {
    a0 = fmaf(__ldg(w + i * stride), col[i * BW_TP], a0);
    a1 = fmaf(__ldg(w + (i + 1) * stride), col[(i + 1) * BW_TP], a1);
  }
  if (i < n) a0 = fmaf(__ldg(w + i * stride), col[i * BW_TP], a0);
  return a0 + a1;
}

__global__ void __launch_bounds__(256) backward_kernel(const InstDev* __restrict__ inst,
                                                       const LaunchInfo li,
                                                       const int8_t* __restrict__ spins,
                                                       const double* __restrict__ logZR,
                                                       const float* __restrict__ logq,
                                                       const double* __restrict__ stats,
                                                       float* __restrict__ partials,
                                                       long long part_stride) {
  extern __shared__ float sm[];
  const int k = find_inst(li, blockIdx.x);
  const InstDev& I = inst[k];
  const MadeDev& md = I.made;
  const int D = md.D, nh = md.nh, H1 = md.H1, H2 = md.H2, Hl = md.Hl;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int t = tid & 31, q = tid >> 5, nq = nth >> 5;
  const int chunk = li.tile;
  const int c_idx = blockIdx.x - li.tile_begin[k];
  const int b_lo = c_idx * chunk, b_hi = min(li.batch, b_lo + chunk);
  float* S = sm;
  float* A1 = S + D * BW_TP;
  float* A2 = A1 + H1 * BW_TP;
  float* X = A2 + H2 * BW_TP;
  float* dA2 = X + D * BW_TP;
  float* dA1 = dA2 + H2 * BW_TP;
  const float* W1 = md.packed + md.layer[0].dst_off;
  const float* b1 = W1 + (long long)H1 * D;
  const float* W2 = nh >= 2 ? md.packed + md.layer[1].dst_off : nullptr;
  const float* b2 = nh >= 2 ? W2 + (long long)H2 * H1 : nullptr;
  const float* Wo = md.packed + md.layer[nh].dst_off;
  const float* bo = Wo + (long long)D * Hl;
  const float* src = nh == 0 ? S : (nh == 1 ? A1 : A2);
  const int* deg1 = nh >= 1 ? md.layer[0].deg_out : nullptr;
  const int* deg2 = nh >= 2 ? md.layer[1].deg_out : nullptr;
  const int* cL = nh == 1 ? md.c1 : md.c2;
  const double mean = stats[8 * k + 4];
  const double beta = li.beta[k];
  const double wscale = -1.0 / (beta * stats_batch(stats + 8 * k));
  float* Gk = partials + (long long)blockIdx.x * part_stride;
  const int8_t* sp = spins + I.spin_units * li.batch;
  bool first = true;
  for (int b0 = b_lo; b0 < b_hi; b0 += BW_TS) {
    const int nv = min(BW_TS, b_hi - b0);
    __syncthreads();
    for (int e = tid; e < BW_TS * D; e += nth) {
      const int tt = e / D, i = e % D;
      S[i * BW_TP + tt] = tt < nv ? (float)sp[(long long)(b0 + tt) * D + i] : 0.f;
    }
    __syncthreads();
    if (nh >= 1) {
      for (int o = q; o < H1; o += nq)
        A1[o * BW_TP + t] = fmaxf(__ldg(b1 + o) + dot_row(W1 + (long long)o * D, S + t, deg1[o]), 0.f);
      __syncthreads();
    }
    if (nh >= 2) {
      for (int o = q; o < H2; o += nq)
        A2[o * BW_TP + t] =
            fmaxf(__ldg(b2 + o) + dot_row(W2 + (long long)o * H1, A1 + t, md.c1[deg2[o]]), 0.f);
      __syncthreads();
    }
    // output logits -> dX = w_b s_i sigmoid(-s_i x_i)
    const bool valid = t < nv;
    const float wb =
        valid ? (float)(wscale * (logZR[(long long)k * li.batch + b0 + t] -
                                  (double)logq[(long long)k * li.batch + b0 + t] - mean))
              : 0.f;
    for (int i = q; i < D; i += nq) {
      const int nin = nh == 0 ? i : cL[i];
      const float x = __ldg(bo + i) + dot_row(Wo + (long long)i * Hl, src + t, nin);
      const float s = S[i * BW_TP + t];
      X[i * BW_TP + t] = wb * s / (1.f + expf(s * x));
    }
    __syncthreads();
    if (nh == 2) {
      // dA2[o] = 1[h2 > 0] sum_{i >= deg2(o)} dX[i] Wo[i][o]
      for (int o = q; o < H2; o += nq) {
        const float h = A2[o * BW_TP + t];
        dA2[o * BW_TP + t] = h > 0.f ? dot_strided(Wo + o, Hl, X + t, deg2[o], D) : 0.f;
      }
      __syncthreads();
      // dA1[j] = 1[h1 > 0] sum_{o: deg2(o) >= deg1(j)} dA2[o] W2[o][j]
      for (int j = q; j < H1; j += nq) {
        const float h = A1[j * BW_TP + t];
        const int o0 = md.c2[deg1[j] - 1];
        dA1[j * BW_TP + t] = h > 0.f ? dot_strided(W2 + j, H1, dA2 + t, o0, H2) : 0.f;
      }
      __syncthreads();
    } else if (nh == 1) {
      for (int j = q; j < H1; j += nq) {
        const float h = A1[j * BW_TP + t];
        dA1[j * BW_TP + t] = h > 0.f ? dot_strided(Wo + j, Hl, X + t, deg1[j], D) : 0.f;
      }
      __syncthreads();
    }
    // weight gradients of this sub-tile
    float* Go = Gk + md.layer[nh].dst_off;
    outer_acc(Go, Go + (long long)D * Hl, X, src, D, Hl, BW_TS, first, tid, nth);
    if (nh == 2) {
      float* G2 = Gk + md.layer[1].dst_off;
      outer_acc(G2, G2 + (long long)H2 * H1, dA2, A1, H2, H1, BW_TS, first, tid, nth);
    }
    if (nh >= 1) {
      float* G1 = Gk + md.layer[0].dst_off;
      outer_acc(G1, G1 + (long long)H1 * D, dA1, S, H1, D, BW_TS, first, tid, nth);
    }
    first = false;
  }
  if (first) {  // empty chunk: zero the slice
    for (long long e = tid; e < md.n_params; e += nth) Gk[e] = 0.f;
  }
}

cudaError_t launch_backward(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int,
                            const int8_t* spins, const double* logZR, const float* logq,
                            const double* stats, float* partials, int part_stride,
                            cudaStream_t s) {
  const int nblk = li.tile_begin[li.n_inst];
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes);
  if (e != cudaSuccess) return e;
  backward_kernel<<<nblk, 256, smem_bytes, s>>>(d_inst, li, spins, logZR, logq, stats, partials,
                                                part_stride);
  return cudaGetLastError();
}

// Adam (Kingma & Ba 2015) on one entry, bias corrections bc1 = 1 - b1^t,
// bc2 = 1 - b2^t.  The one definition both Adam kernels use.
__device__ __forceinline__ void adam_entry(float& p, float& m, float& v, float g, const AdamArgs& a, float bc1,
                                           float bc2) {
  const float mi = a.b1 * m + (1.f - a.b1) * g;
  const float vi = a.b2 * v + (1.f - a.b2) * g * g;
  m = mi;
  v = vi;
  p -= a.lr * (mi / bc1) / (sqrtf(vi / bc2) + a.eps);
}

// The bias corrections of this launch: the host's, or (device step counter)
// formed by one thread of the CTA in FP64 (a narrow unit here) from
// t = t_base + *t_dev.
__device__ __forceinline__ void adam_corrections(const AdamArgs& a, float& bc1, float& bc2) {
  bc1 = a.bc1;
  bc2 = a.bc2;
  if (a.t_dev) {
    __shared__ float bc[2];
    if (threadIdx.x == 0) {
      const double t = (double)(a.t_base + (long long)*a.t_dev);
      bc[0] = (float)(1.0 - exp(t * log((double)a.b1)));
      bc[1] = (float)(1.0 - exp(t * log((double)a.b2)));
    }
    __syncthreads();
    bc1 = bc[0];
    bc2 = bc[1];
  }
}

// Sum the chunk partials of every instance (fixed order: deterministic) and
// scatter from the packed, degree-sorted layout to the caller's natural
// layout; entries outside the MADE masks get 0.  With ADAM the same thread
// then applies Adam to that entry of the instance's own parameters
// (tnvan_set_made's pointer) with the moments at the gradient's offset, so a
// training step needs no separate optimizer pass over the gradient.
template <bool ADAM>
__global__ void grad_reduce_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                   const float* __restrict__ partials, long long part_stride,
                                   float* __restrict__ grad, const AdamArgs adam, int k0) {
  const int k = blockIdx.y + k0;
  if ((li.skip[k >> 5] >> (k & 31)) & 1u) return;  // reduced by another backward form
  const MadeDev& md = inst[k].made;
  float bc1 = 1.f, bc2 = 1.f;
  if (ADAM) adam_corrections(adam, bc1, bc2);
  const int p0 = li.tile_begin[k], p1 = li.tile_begin[k + 1];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < md.n_params;
       e += (long long)gridDim.x * blockDim.x) {
    // eight independent partial sums keep eight loads in flight; fixed order
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int p = p0;
    for (; p + 8 <= p1; p += 8)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] += partials[(long long)(p + j) * part_stride + e];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (p + j < p1) a[j] += partials[(long long)(p + j) * part_stride + e];
    const float s = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    int r = (int)e;  // a network's parameter count fits in 32 bits (checked at set-up)
    long long nat = -1;
    float gv = s;
    for (int l = 0; l < md.n_layers; ++l) {
      const LayerDev& L = md.layer[l];
      const int nw = L.nout * L.nin;
      if (r < nw) {
        const int o = r / L.nin, i = r - o * L.nin;
        const int no = L.perm_out ? L.perm_out[o] : o;
        const int ni = L.perm_in ? L.perm_in[i] : i;
        const bool conn = L.strict ? (L.deg_out[o] > L.deg_in[i]) : (L.deg_out[o] >= L.deg_in[i]);
        nat = L.src_off + (long long)no * L.nin + ni;
        gv = conn ? s : 0.f;
        break;
      }
      r -= nw;
      if (r < L.nout) {
        nat = L.src_off + nw + (L.perm_out ? L.perm_out[r] : r);
        break;
      }
      r -= L.nout;
    }
    if (nat < 0) continue;
    const long long o = md.param_off + nat;
    grad[o] = gv;
    if (ADAM) adam_entry(md.raw[nat], adam.m[o], adam.v[o], gv, adam, bc1, bc2);
  }
}

cudaError_t launch_grad_reduce(const InstDev* d_inst, const LaunchInfo& li, const float* partials,
                               int part_stride, float* grad, cudaStream_t s, const AdamArgs* adam, int k0, int k1) {
  if (k1 < 0) k1 = li.n_inst;
  if (k1 <= k0) return cudaSuccess;
  // one parameter per thread (the row stride bounds every instance's count),
  // at most 256 CTAs per instance and about 4096 per launch (a launch over
  // many instances strides instead)
  const int cap = 4096 / (k1 - k0) > 16 ? 4096 / (k1 - k0) : 16;
  int gx = (int)((part_stride + 255) / 256);
  gx = gx < cap ? gx : cap;
  gx = gx < 256 ? gx : 256;
  const dim3 grid((unsigned)(gx > 1 ? gx : 1), k1 - k0);
  if (adam)
    grad_reduce_kernel<true><<<grid, 256, 0, s>>>(d_inst, li, partials, part_stride, grad, *adam, k0);
  else
    grad_reduce_kernel<false><<<grid, 256, 0, s>>>(d_inst, li, partials, part_stride, grad, AdamArgs{}, k0);
  return cudaGetLastError();
}

// Importance weights of tnvan_observables as multipliers B w_b =
// exp(l_b - logZ_IS), w_b = exp(l_b) / sum_b' exp(l_b') (self-normalised;
// logZ_IS = logsumexp_b l_b - ln B from the F_q reduction's statistics).
__global__ void obs_weights_kernel(const LaunchInfo li, const double* __restrict__ logZR,
                                   const float* __restrict__ logq, const double* __restrict__ stats,
                                   float* __restrict__ wmul) {
  const int k = blockIdx.y;
  const double lz = stats[8 * k + 3];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < li.batch; b += gridDim.x * blockDim.x) {
    const long long o = (long long)k * li.batch + b;
    wmul[o] = (float)exp(logZR[o] - (double)logq[o] - lz);
  }
}

// Per instance (one CTA each): sum_b m_b E_b, sum_b E_b and sum_b m_b^2 with
// E_b = -dbeta_b and m_b the multipliers above, in a fixed order (FP64).
__global__ void obs_energy_kernel(const LaunchInfo li, const double* __restrict__ dbeta,
                                  const float* __restrict__ wmul, double* __restrict__ out) {
  const int k = blockIdx.x;
  double a = 0.0, e = 0.0, q = 0.0;
  for (int b = threadIdx.x; b < li.batch; b += blockDim.x) {
    const long long o = (long long)k * li.batch + b;
    const double E = -dbeta[o], m = (double)wmul[o];
    a += m * E;
    e += E;
    q += m * m;
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = e;
  red[2][threadIdx.x] = q;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int j = 0; j < 3; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double B = (double)li.batch;
    out[3 * k + 0] = red[0][0] / B;      // U  = sum_b w_b E_b
    out[3 * k + 1] = red[1][0] / B;      // U_q = mean_b E_b
    out[3 * k + 2] = B * B / red[2][0];  // effective sample size 1 / sum_b w_b^2
  }
}

cudaError_t launch_observables(const LaunchInfo& li, const double* logZR, const float* logq, const double* stats,
                               const double* dbeta, float* wmul, double* out, bool energies, cudaStream_t s) {
  if (li.n_inst == 0 || li.batch == 0) return cudaSuccess;
  if (!energies) {
    obs_weights_kernel<<<dim3(32, li.n_inst), 256, 0, s>>>(li, logZR, logq, stats, wmul);
    return cudaGetLastError();
  }
  obs_energy_kernel<<<li.n_inst, 256, 0, s>>>(li, dbeta, wmul, out);
  return cudaGetLastError();
}

// Per instance (one CTA each), in a fixed order (FP64), with m_b the
// multipliers B w_b above, mu_b = E[M | s_b] and v_b = Var(M | s_b):
//   out[5k+0] = sum_b m_b mu_b / B                 (<M>, importance-weighted)
//   out[5k+1] = sum_b m_b (mu_b^2 + v_b) / B       (<M^2>)
//   out[5k+2] = mean_b mu_b,  out[5k+3] = mean_b (mu_b^2 + v_b)   (the same under q)
//   out[5k+4] = B^2 / sum_b m_b^2                  (effective sample size)
__global__ void obs_mag_kernel(const LaunchInfo li, const double* __restrict__ mean, const double* __restrict__ var,
                               const float* __restrict__ wmul, double* __restrict__ out) {
  const int k = blockIdx.x;
  double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < li.batch; b += blockDim.x) {
    const long long o = (long long)k * li.batch + b;
    const double mu = mean[o], m2 = mu * mu + var[o], w = (double)wmul[o];
    a[0] += w * mu;
    a[1] += w * m2;
    a[2] += mu;
    a[3] += m2;
    a[4] += w * w;
  }
  __shared__ double red[5][256];
  for (int j = 0; j < 5; ++j) red[j][threadIdx.x] = a[j];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int j = 0; j < 5; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double B = (double)li.batch;
    for (int j = 0; j < 4; ++j) out[5 * k + j] = red[j][0] / B;
    out[5 * k + 4] = B * B / red[4][0];
  }
}

cudaError_t launch_obs_mag(const LaunchInfo& li, const double* mean, const double* var, const float* wmul,
                           double* out, cudaStream_t s) {
  if (li.n_inst == 0 || li.batch == 0) return cudaSuccess;
  obs_mag_kernel<<<li.n_inst, 256, 0, s>>>(li, mean, var, wmul, out);
  return cudaGetLastError();
}

// REINFORCE weights w_b = -(l_b - mean_b l) / (beta B) per instance (Eq. 10
// with the batch-mean baseline), FP32 copy for the tensor-core backward.
// Eq. 10's per-sample weights w[k][b]; with s16, also the spins of every
// instance not marked in li.skip as BF16 rows of D rounded up to 8 (zeros
// beyond D), instance k at sum_{j<k} batch * r8(D_j): the GEMM chain's spin
// operands.
__global__ void reinforce_w_kernel(const InstDev* __restrict__ inst, const LaunchInfo li,
                                   const double* __restrict__ logZR, const float* __restrict__ logq,
                                   const double* __restrict__ stats, float* __restrict__ w,
                                   const int8_t* __restrict__ spins, uint16_t* __restrict__ s16) {
  const int k = blockIdx.y;
  const double mean = stats[8 * k + 4];
  const double sc = -1.0 / (li.beta[k] * stats_batch(stats + 8 * k));
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < li.batch; b += gridDim.x * blockDim.x) {
    const long long o = (long long)k * li.batch + b;
    w[o] = (float)(sc * (logZR[o] - (double)logq[o] - mean));
  }
  if (!s16 || ((li.skip[k >> 5] >> (k & 31)) & 1u)) return;  // skipped: another backward form reads the spins
  long long off = 0;
  for (int j = 0; j < k; ++j) off += (long long)li.batch * ((inst[j].D + 7) & ~7);
  const int D = inst[k].D, G8 = (D + 7) >> 3;  // 8-spin groups per row
  const int8_t* src = spins + inst[k].spin_units * li.batch;
  const long long n = (long long)li.batch * G8;
  uint4* dst = reinterpret_cast<uint4*>(s16 + off);  // 16-byte aligned: off is a multiple of 8
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / G8;
    const int i0 = (int)(e - b * G8) * 8;
    uint32_t h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t v = 0;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = i0 + 2 * q + j;
        const uint32_t x = i < D ? (src[b * D + i] > 0 ? 0x3F80u : 0xBF80u) : 0u;
        v |= x << (16 * j);
      }
      h[q] = v;
    }
    dst[e] = make_uint4(h[0], h[1], h[2], h[3]);
  }
}

cudaError_t launch_reinforce_w(const InstDev* d_inst, const LaunchInfo& li, const double* logZR, const float* logq,
                               const double* stats, float* w, const int8_t* spins, uint16_t* s16, cudaStream_t s) {
  if (li.n_inst == 0 || li.batch == 0) return cudaSuccess;
  reinforce_w_kernel<<<dim3(32, li.n_inst), 256, 0, s>>>(d_inst, li, logZR, logq, stats, w, spins, s16);
  return cudaGetLastError();
}

// Adam over a flat array (tnvan_adam).  With t_dev, the step is
// t_base + *t_dev (a device step counter, for replayed CUDA graphs).
__global__ void adam_kernel(long long n, float* __restrict__ p, const float* __restrict__ g, const AdamArgs a) {
  float bc1, bc2;
  adam_corrections(a, bc1, bc2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    adam_entry(p[i], a.m[i], a.v[i], g[i], a, bc1, bc2);
}

cudaError_t launch_adam(long long n, float* p, const float* g, const AdamArgs& a, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 1216) nb = 1216;
  adam_kernel<<<(int)nb, 256, 0, s>>>(n, p, g, a);
  return cudaGetLastError();
}

}  // namespace tnvan
