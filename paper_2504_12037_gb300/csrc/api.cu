// C-ABI of the TNVAN GB300 library: context, host planner, launch sequencing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <set>
#include <utility>

#include "gemm.h"
#include "internal.h"

using namespace tnvan;

namespace {

thread_local std::string g_create_err;

int fail(tnvan_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_create_err = buf;
  return code;
}

int cuda_fail(tnvan_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, TNVAN_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                              \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Brackets one kernel launch with CUDA events when profiling is on.
struct Prof {
  tnvan_ctx* ctx;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  size_t idx = 0;
  static cudaEvent_t take(tnvan_ctx* c) {
    if (!c->event_pool.empty()) {
      cudaEvent_t e = c->event_pool.back();
      c->event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  Prof(tnvan_ctx* c, const char* name, cudaStream_t st) : ctx(c), s(st) {
    if (!ctx->prof_on) return;
    for (idx = 0; idx < ctx->prof.size(); ++idx)
      if (ctx->prof[idx].name == name) break;
    if (idx == ctx->prof.size()) {
      ctx->prof.emplace_back();
      ctx->prof.back().name = name;
    }
    a = take(ctx);
    b = take(ctx);
    if (!ctx->prof_ref_set) {
      if (!ctx->prof_ref) cudaEventCreate(&ctx->prof_ref);
      if (ctx->prof_ref) cudaEventRecord(ctx->prof_ref, s);
      ctx->prof_ref_set = ctx->prof_ref != nullptr;
    }
    if (a) cudaEventRecord(a, s);
  }
  ~Prof() {
    if (!a || !b) return;
    cudaEventRecord(b, s);
    ctx->prof[idx].pending.emplace_back(a, b);
  }
};

#define PROF(name, stream) Prof _prof_guard(ctx, name, stream)

template <typename T>
int upload(tnvan_ctx* ctx, Instance& in, const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return TNVAN_OK;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(%zu): %s", v.size() * sizeof(T), cudaGetErrorString(e));
  in.dev_allocs.push_back(p);
  e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy (plan upload)");
  *out = static_cast<T*>(p);
  return TNVAN_OK;
}

void free_instance(Instance& in) {
  for (void* p : in.dev_allocs) cudaFree(p);
  in.dev_allocs.clear();
}

// A BF16 weight blob of full.size() elements whose element e is packed
// weight full[e] (-1: zero).  The blob is zeroed once here; the pack kernel
// rewrites only the live elements, from the lists *src / *dst (*n_live long).
int upload_blob(tnvan_ctx* ctx, Instance& in, const std::vector<int>& full, uint16_t** blob, const int** src,
                const int** dst, long long* n_live) {
  std::vector<int> s, d;
  for (size_t e = 0; e < full.size(); ++e)
    if (full[e] >= 0) {
      s.push_back(full[e]);
      d.push_back((int)e);
    }
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(full.size(), 8) * sizeof(uint16_t);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(sampler blobs): %s", cudaGetErrorString(e));
  in.dev_allocs.push_back(p);
  if ((e = cudaMemset(p, 0, bytes)) != cudaSuccess) return cuda_fail(ctx, e, "cudaMemset (sampler blobs)");
  int rc;
  int *ds = nullptr, *dd = nullptr;
  if ((rc = upload(ctx, in, s, &ds)) || (rc = upload(ctx, in, d, &dd))) return rc;
  *blob = static_cast<uint16_t*>(p);
  *src = ds;
  *dst = dd;
  *n_live = (long long)s.size();
  return TNVAN_OK;
}

// Drop the device plan + network of an instance (keeps the graph).
void reset_plan(Instance& in) {
  free_instance(in);
  in.has_ws = false;
  in.has_made = false;
  in.dev = InstDev{};
}

int check_inst(tnvan_ctx* ctx, int instance, bool allow_append) {
  if (!ctx) return TNVAN_E_ARG;
  const int n = (int)ctx->inst.size();
  if (instance < 0 || instance > n || (!allow_append && instance == n) || instance >= TNVAN_MAX_INST)
    return fail(ctx, TNVAN_E_ARG, "instance %d out of range (have %d, max %d)", instance, n, TNVAN_MAX_INST);
  return TNVAN_OK;
}

// strip_tab_floats_adj of the kernels: tables without d/dbeta rows.
int strip_tab_floats_adj_host(int w, int L) {
  int n = L * w * 4 + L * 4 * (1 << w) + 2 * L;
  return (n + 3) & ~3;
}

int host_strip_tab_floats(int w, int L) {
  int n = L * w * 4 + 2 * L * 4 * (1 << w) + 2 * L;
  return (n + 3) & ~3;
}

// ---------------------------------------------------------------------------
// Planner: lattice strips.
// ---------------------------------------------------------------------------
int plan_strips(tnvan_ctx* ctx, Instance& in, const std::map<std::pair<int, int>, int>& edge_of,
                const std::vector<int>& pos) {
  const int Lx = in.Lx, Ly = in.Ly;
  std::vector<int> colW(Lx, 0);
  for (int w : in.W) colW[w % Lx]++;
  for (int x = 0; x < Lx; ++x)
    if (colW[x] != 0 && colW[x] != Ly) return TNVAN_E_UNSUPPORTED;  // not whole columns
  auto eid = [&](int a, int b) {
    auto it = edge_of.find({std::min(a, b), std::max(a, b)});
    return it == edge_of.end() ? -1 : it->second;
  };
  std::vector<char> used(in.m, 0);
  HostStripPlan plan;
  plan.edge_sign.assign(in.m, 1.f);
  int tab = 0;
  for (int x = 0; x < Lx;) {
    if (colW[x]) {
      ++x;
      continue;
    }
    int x0 = x;
    while (x < Lx && !colW[x]) ++x;
    const int w = x - x0;
    if (w > TNVAN_MAX_STRIP_W)
      return fail(ctx, TNVAN_E_UNSUPPORTED, "strip of %d columns (max %d)", w, TNVAN_MAX_STRIP_W);
    StripDev sd{};
    sd.w = w;
    sd.L = Ly;
    sd.row0 = (int)plan.rows.size();
    sd.tab_off = tab;
    double chat = 0;
    // Gauge: spin (y, c) of the strip is replaced by tau_c(y) * spin with
    // tau_c(0) = 1 and tau_c(y+1) = tau_c(y) * sign(Jv(y, c)), which makes every
    // vertical bond ferromagnetic (its normalised factor is [[1, t], [t, 1]]) and
    // leaves Z_strip unchanged; the other couplings of the row take the signs.
    float tau[TNVAN_MAX_STRIP_W];
    for (int c = 0; c < TNVAN_MAX_STRIP_W; ++c) tau[c] = 1.f;
    for (int y = 0; y < Ly; ++y) {
      StripRow R{};
      for (int c = 0; c < TNVAN_MAX_STRIP_W - 1; ++c) R.eh[c] = -1;
      for (int c = 0; c < TNVAN_MAX_STRIP_W; ++c) R.ev[c] = -1;
      R.eL = R.eR = -1;
      R.posL = R.posR = -1;
      R.tau_mask = 0;
      for (int c = 0; c < w; ++c)
        if (tau[c] < 0.f) R.tau_mask |= 1 << c;
      for (int c = 0; c + 1 < w; ++c) {
        int e = eid(y * Lx + x0 + c, y * Lx + x0 + c + 1);
        if (e >= 0) {
          R.Jh[c] = (float)in.J[e] * tau[c] * tau[c + 1];
          plan.edge_sign[e] = tau[c] * tau[c + 1];
          R.eh[c] = e;
          used[e] = 1;
          chat += fabs((double)R.Jh[c]);
        }
      }
      if (x0 > 0) {
        int e = eid(y * Lx + x0 - 1, y * Lx + x0);
        if (e >= 0) {
          R.JL = (float)in.J[e] * tau[0];
          plan.edge_sign[e] = tau[0];
          R.posL = pos[y * Lx + x0 - 1];
          R.eL = e;
          used[e] = 1;
          chat += fabs((double)R.JL);
        }
      }
      if (x0 + w < Lx) {
        int e = eid(y * Lx + x0 + w - 1, y * Lx + x0 + w);
        if (e >= 0) {
          R.JR = (float)in.J[e] * tau[w - 1];
          plan.edge_sign[e] = tau[w - 1];
          R.posR = pos[y * Lx + x0 + w];
          R.eR = e;
          used[e] = 1;
          chat += fabs((double)R.JR);
        }
      }
      if (y + 1 < Ly) {
        for (int c = 0; c < w; ++c) {
          int e = eid(y * Lx + x0 + c, (y + 1) * Lx + x0 + c);
          if (e >= 0) {
            const float sg = in.J[e] < 0 ? -1.f : 1.f;
            R.Jv[c] = (float)fabs(in.J[e]);
            plan.edge_sign[e] = sg;
            tau[c] *= sg;
            R.ev[c] = e;
            used[e] = 1;
            chat += fabs((double)R.Jv[c]);
          }
        }
      }
      for (int j = 0; j < TNVAN_STRIP_SLOTS; ++j) {
        R.Js[j] = 0.f;
        R.es[j] = -1;
      }
      for (int c = 0; c + 1 < w; ++c) {
        R.Js[c] = R.Jh[c];
        R.es[c] = R.eh[c];
      }
      R.Js[w - 1] = R.JL;
      R.es[w - 1] = R.eL;
      R.Js[w] = R.JR;
      R.es[w] = R.eR;
      for (int c = 0; c < w; ++c) {
        R.Js[w + 1 + c] = R.Jv[c];
        R.es[w + 1 + c] = R.ev[c];
      }
      plan.rows.push_back(R);
    }
    sd.c_hat = chat;
    plan.strips.push_back(sd);
    tab += host_strip_tab_floats(w, Ly);
  }
  for (int e = 0; e < in.m; ++e) {
    const bool wa = pos[in.ei[e]] >= 0, wb = pos[in.ej[e]] >= 0;
    if (wa && wb) used[e] = 1;
    if (!used[e]) return TNVAN_E_UNSUPPORTED;  // a bond the strip form cannot carry
  }
  in.strip = std::move(plan);
  in.dev.strip_tab_floats = tab;
  in.kind = 0;
  return TNVAN_OK;
}

// Wide strips: a lattice whose width set is whole columns, leaving strips of
// at most TNVAN_WIDE_MAX_W columns, gets (besides its elimination plan) the
// rows of every strip for the wide-strip forward contraction, in the same
// gauge as plan_strips.  Leaves in.wide empty when the instance does not
// qualify (then the elimination plan does everything).
void plan_wide_strips(Instance& in, const std::map<std::pair<int, int>, int>& edge_of, const std::vector<int>& pos) {
  in.wide = HostWidePlan{};
  if (in.topology != TNVAN_LATTICE2D) return;
  const int Lx = in.Lx, Ly = in.Ly;
  std::vector<int> colW(Lx, 0);
  for (int w : in.W) colW[w % Lx]++;
  for (int x = 0; x < Lx; ++x)
    if (colW[x] != 0 && colW[x] != Ly) return;
  auto eid = [&](int a, int b) {
    auto it = edge_of.find({std::min(a, b), std::max(a, b)});
    return it == edge_of.end() ? -1 : it->second;
  };
  std::vector<char> used(in.m, 0);
  HostWidePlan plan;
  for (int x = 0; x < Lx;) {
    if (colW[x]) {
      ++x;
      continue;
    }
    const int x0 = x;
    while (x < Lx && !colW[x]) ++x;
    const int w = x - x0;
    if (w > TNVAN_WIDE_MAX_W) return;
    WideStripDev sd{};
    sd.w = w;
    sd.L = Ly;
    sd.row0 = (int)plan.rows.size();
    double chat = 0;
    // gauge: tau_c(y + 1) = tau_c(y) sign(Jv(y, c)) makes every vertical bond ferromagnetic
    float tau[TNVAN_WIDE_MAX_W];
    for (int c = 0; c < TNVAN_WIDE_MAX_W; ++c) tau[c] = 1.f;
    for (int y = 0; y < Ly; ++y) {
      WideRow R{};
      R.posL = R.posR = -1;
      for (int c = 0; c + 1 < w; ++c) {
        const int e = eid(y * Lx + x0 + c, y * Lx + x0 + c + 1);
        if (e >= 0) {
          R.Jh[c] = (float)in.J[e] * tau[c] * tau[c + 1];
          used[e] = 1;
          chat += fabs((double)R.Jh[c]);
        }
      }
      if (x0 > 0) {
        const int e = eid(y * Lx + x0 - 1, y * Lx + x0);
        if (e >= 0) {
          R.JL = (float)in.J[e] * tau[0];
          R.posL = pos[y * Lx + x0 - 1];
          used[e] = 1;
          chat += fabs((double)R.JL);
        }
      }
      if (x0 + w < Lx) {
        const int e = eid(y * Lx + x0 + w - 1, y * Lx + x0 + w);
        if (e >= 0) {
          R.JR = (float)in.J[e] * tau[w - 1];
          R.posR = pos[y * Lx + x0 + w];
          used[e] = 1;
          chat += fabs((double)R.JR);
        }
      }
      if (y + 1 < Ly) {
        for (int c = 0; c < w; ++c) {
          const int e = eid(y * Lx + x0 + c, (y + 1) * Lx + x0 + c);
          if (e >= 0) {
            R.Jv[c] = (float)fabs(in.J[e]);
            if (in.J[e] < 0) tau[c] = -tau[c];
            used[e] = 1;
            chat += fabs((double)R.Jv[c]);
          }
        }
      }
      plan.rows.push_back(R);
    }
    sd.c_hat = chat;
    plan.strips.push_back(sd);
  }
  for (int e = 0; e < in.m; ++e) {
    const bool wa = pos[in.ei[e]] >= 0, wb = pos[in.ej[e]] >= 0;
    if (wa && wb) used[e] = 1;
    if (!used[e]) return;  // a bond the strips do not carry
  }
  in.wide = std::move(plan);
}

// Connected components of the graph induced on R.
std::vector<std::vector<int>> r_components(const Instance& in, const std::vector<int>& pos) {
  std::vector<std::vector<int>> adj(in.n);
  for (int e = 0; e < in.m; ++e) {
    adj[in.ei[e]].push_back(in.ej[e]);
    adj[in.ej[e]].push_back(in.ei[e]);
  }
  std::vector<char> seen(in.n, 0);
  std::vector<std::vector<int>> comps;
  for (int v = 0; v < in.n; ++v) {
    if (pos[v] >= 0 || seen[v]) continue;
    std::vector<int> c{v};
    seen[v] = 1;
    for (size_t h = 0; h < c.size(); ++h)
      for (int u : adj[c[h]])
        if (pos[u] < 0 && !seen[u]) {
          seen[u] = 1;
          c.push_back(u);
        }
    std::sort(c.begin(), c.end());
    comps.push_back(std::move(c));
  }
  return comps;
}

int plan_dense(tnvan_ctx* ctx, Instance& in, const std::vector<int>& pos);
int plan_general(tnvan_ctx* ctx, Instance& in, const std::vector<int>& pos, const std::vector<int>& rank);

int upload_plan(tnvan_ctx* ctx, Instance& in) {
  int rc;
  EdgeWW* dww = nullptr;
  if ((rc = upload(ctx, in, in.ww, &dww))) return rc;
  in.dev.ww = dww;
  in.dev.n_ww = (int)in.ww.size();
  in.dev.n_wide = 0;
  if (!in.wide.strips.empty()) {
    WideStripDev* dws = nullptr;
    WideRow* dwr = nullptr;
    if ((rc = upload(ctx, in, in.wide.strips, &dws))) return rc;
    if ((rc = upload(ctx, in, in.wide.rows, &dwr))) return rc;
    in.dev.wide = dws;
    in.dev.wrows = dwr;
    in.dev.n_wide = (int)in.wide.strips.size();
  }
  if (in.kind == 0) {
    StripDev* ds = nullptr;
    StripRow* dr = nullptr;
    float* dsg = nullptr;
    if ((rc = upload(ctx, in, in.strip.strips, &ds))) return rc;
    if ((rc = upload(ctx, in, in.strip.rows, &dr))) return rc;
    if ((rc = upload(ctx, in, in.strip.edge_sign, &dsg))) return rc;
    in.dev.strips = ds;
    in.dev.rows = dr;
    in.dev.edge_sign = dsg;
    int tabn = 0;
    for (const StripDev& sd : in.strip.strips) tabn += strip_tab_floats_adj_host(sd.w, sd.L);
    std::vector<float> zt((size_t)std::max(tabn, 4), 0.f);
    float* dt = nullptr;
    if ((rc = upload(ctx, in, zt, &dt))) return rc;
    in.dev.adj_tab = dt;
    in.dev.n_strips = (int)in.strip.strips.size();
  } else if (in.kind == 1) {
    float *jrw = nullptr, *jrr = nullptr;
    int *err = nullptr, *erw = nullptr;
    if ((rc = upload(ctx, in, in.JRW, &jrw))) return rc;
    if ((rc = upload(ctx, in, in.JRR, &jrr))) return rc;
    if ((rc = upload(ctx, in, in.eRR, &err))) return rc;
    if ((rc = upload(ctx, in, in.eRW, &erw))) return rc;
    DenseDev& dd = in.dev.dense;
    dd.nR = in.dense_nR;
    dd.nA = std::min(8, in.dense_nR);
    dd.nB = in.dense_nR - dd.nA;
    dd.JRW = jrw;
    dd.JRR = jrr;
    dd.eRR = err;
    dd.eRW = erw;
    dd.c_hat = in.dense_chat;
    std::vector<float> zc(256 * 256, 0.f);
    float* c32 = nullptr;
    if ((rc = upload(ctx, in, zc, &c32))) return rc;
    float* dc32 = nullptr;
    if ((rc = upload(ctx, in, zc, &dc32))) return rc;
    dd.dC32 = dc32;
    std::vector<uint16_t> zc16(256 * 256, 0);
    uint16_t* c16 = nullptr;
    if ((rc = upload(ctx, in, zc16, &c16))) return rc;
    std::vector<double> zc0(2, 0.0);
    double* c0 = nullptr;
    if ((rc = upload(ctx, in, zc0, &c0))) return rc;
    dd.C32 = c32;
    dd.C16 = c16;
    dd.c0 = c0;
  } else {
    int *fld = nullptr, *pe = nullptr, *cs = nullptr;
    float *pj = nullptr, *fj = nullptr;
    if ((rc = upload(ctx, in, in.gpairE, &pe))) return rc;
    if ((rc = upload(ctx, in, in.gcomp_step0, &cs))) return rc;
    if ((rc = upload(ctx, in, in.gfld, &fld))) return rc;
    if ((rc = upload(ctx, in, in.gpairJ, &pj))) return rc;
    if ((rc = upload(ctx, in, in.gfldJ, &fj))) return rc;
    GenDev& g = in.dev.gen;
    g.n_comp = in.g_ncomp;
    int *fp = nullptr, *fhd = nullptr, *fst = nullptr;
    unsigned short* mpd = nullptr;
    if ((rc = upload(ctx, in, in.gfprog, &fp))) return rc;
    if ((rc = upload(ctx, in, in.gfhdr, &fhd))) return rc;
    if ((rc = upload(ctx, in, in.gfstep, &fst))) return rc;
    if ((rc = upload(ctx, in, in.gmap, &mpd))) return rc;
    std::vector<float> zpp(2 * (size_t)std::max(in.g_npp, 1), 0.f);
    float* ppd = nullptr;
    if ((rc = upload(ctx, in, zpp, &ppd))) return rc;
    g.fprog = fp;
    g.fhdr = fhd;
    g.fstep = fst;
    g.map = mpd;
    g.pp = ppd;
    g.n_pp = in.g_npp;
    g.n_steps = (int)in.gfstep.size();
    g.pairJ = pj;
    g.pairE = pe;
    g.comp_step0 = cs;
    g.fld = fld;
    g.fldJ = fj;
    g.c_hat = in.g_chat;
    int *ct = nullptr, *bp = nullptr, *tc = nullptr;
    if ((rc = upload(ctx, in, in.gctab, &ct))) return rc;
    if ((rc = upload(ctx, in, in.gbpos, &bp))) return rc;
    if ((rc = upload(ctx, in, in.gtabc, &tc))) return rc;
    g.ctab = ct;
    g.bpos = bp;
    g.tabc = tc;
    g.n_tabc = (int)in.gtabc.size();
    g.n_tab = in.g_ntab;
    g.tab_lz = g.tab_db = nullptr;
    if (in.g_ntab > 0) {
      std::vector<double> zt((size_t)in.g_ntab, 0.0);
      if ((rc = upload(ctx, in, zt, &g.tab_lz))) return rc;
      if ((rc = upload(ctx, in, zt, &g.tab_db))) return rc;
    }
  }
  return TNVAN_OK;
}

// Make sure the device descriptor array matches the host instances.
int sync_descriptors(tnvan_ctx* ctx) {
  if (!ctx->dirty) return TNVAN_OK;
  const int n = (int)ctx->inst.size();
  long long su = 0, eo = 0, po = 0;
  std::vector<InstDev> h(n);
  for (int k = 0; k < n; ++k) {
    Instance& in = ctx->inst[k];
    in.dev.kind = in.kind;
    in.dev.n_spins = in.n;
    in.dev.n_edges = in.m;
    in.dev.D = (int)in.W.size();
    in.dev.spin_units = su;
    in.dev.edge_off = eo;
    in.dev.made.param_off = po;
    su += (long long)in.W.size();
    eo += in.m;
    po += in.n_params;
    h[k] = in.dev;
  }
  if (n > ctx->d_inst_cap) {
    if (ctx->d_inst) cudaFree(ctx->d_inst);
    ctx->d_inst = nullptr;
    CK(cudaMalloc(&ctx->d_inst, sizeof(InstDev) * TNVAN_MAX_INST), "cudaMalloc(descriptors)");
    ctx->d_inst_cap = TNVAN_MAX_INST;
  }
  if (n) CK(cudaMemcpy(ctx->d_inst, h.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice), "cudaMemcpy(descriptors)");
  ctx->dirty = false;
  return TNVAN_OK;
}

int check_ready(tnvan_ctx* ctx, bool need_made) {
  if (ctx->inst.empty()) return fail(ctx, TNVAN_E_STATE, "no instances");
  for (size_t k = 0; k < ctx->inst.size(); ++k) {
    const Instance& in = ctx->inst[k];
    if (!in.has_graph || !in.has_ws) return fail(ctx, TNVAN_E_STATE, "instance %zu has no graph/width set", k);
    if (need_made && !in.has_made) return fail(ctx, TNVAN_E_STATE, "instance %zu has no network", k);
  }
  return sync_descriptors(ctx);
}

int fill_launch(tnvan_ctx* ctx, const double* betas, int batch, int tile, LaunchInfo& li) {
  memset(&li, 0, sizeof li);
  li.status = ctx->d_status;
  li.step_dev = ctx->step_dev;
  li.n_inst = (int)ctx->inst.size();
  li.batch = batch;
  li.tile = tile;
  if (!betas) return fail(ctx, TNVAN_E_ARG, "betas is NULL");
  int acc = 0;
  for (int k = 0; k < li.n_inst; ++k) {
    if (!(betas[k] > 0.0) || !isfinite(betas[k])) return fail(ctx, TNVAN_E_ARG, "beta[%d] = %g must be finite and > 0", k, betas[k]);
    li.beta[k] = betas[k];
    li.tile_begin[k] = acc;
    acc += (batch + tile - 1) / tile;
  }
  li.tile_begin[li.n_inst] = acc;
  return TNVAN_OK;
}

int max_sample_smem(const tnvan_ctx* ctx, int tile) {
  int m = 0;
  for (const Instance& in : ctx->inst) m = std::max(m, sample_smem_bytes(in, tile));
  return m;
}

int pick_sample_tile(const tnvan_ctx* ctx) {
  if (ctx->tune_sample_tile && max_sample_smem(ctx, ctx->tune_sample_tile) <= 227 * 1024) return ctx->tune_sample_tile;
  // largest tile that keeps two CTAs per SM, else the largest that fits
  for (int T : {64, 32})
    if (max_sample_smem(ctx, T) <= 113 * 1024) return T;
  for (int T : {32, 16, 8})
    if (max_sample_smem(ctx, T) <= 227 * 1024) return T;
  return 8;
}


// Launch shape of the strip adjoint: one thread per sample with T in
// {128, 96, 64, 32} samples per CTA (all strips in turn), or one warp per
// strip over 32 samples per CTA (ws_threads = 32 x strips; tuning value 1).
// The left vectors of a strip's even rows take ceil(L/2) 2^w floats per thread of shared memory,
// so the shape sets the CTAs per SM; the default minimises (waves of CTAs) x
// (strips a thread sweeps) / (the SM's issue rate, taken as saturating at 8
// warps).  An autotuned shape (tnvan_autotune) takes precedence when it fits.
int plan_strip_adjoint(tnvan_ctx* ctx, int batch, int* tile, int* smem, int* lv_floats, int* ws_threads) {
  auto& c = ctx->adj_plan;
  if (c.valid && !ctx->dirty && c.batch == batch && c.tune == ctx->tune_adj_tile) {
    *tile = c.tile;
    *smem = c.smem;
    *lv_floats = c.lv;
    *ws_threads = c.ws;
    return TNVAN_OK;
  }
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (n_sm < 1) n_sm = 1;
  int max_strips = 0, n_strip_inst = 0;
  for (const Instance& in : ctx->inst)
    if (in.kind == 0) {
      max_strips = std::max(max_strips, (int)in.strip.strips.size());
      ++n_strip_inst;
    }
  double best = 1e300;
  *tile = 0;
  *ws_threads = 0;
  for (int T : {1, 128, 96, 64, 32}) {
    const bool ws = T == 1;
    const int threads = ws ? strip_adj_ws_threads(ctx) : T;
    const int spc = ws ? 32 : T;  // samples per CTA
    if (threads < 32 || threads > (ws ? 256 : 128)) continue;
    int sm = 0, lv = 0;
    for (const Instance& in : ctx->inst)
      if (in.kind == 0) lv = std::max(lv, ws ? strip_adj_ws_lv_floats(in, threads) : strip_adj_lv_floats(in, T));
    for (const Instance& in : ctx->inst)
      if (in.kind == 0)
        sm = std::max(sm, ws ? strip_adj_ws_smem_bytes(in, threads, lv) : strip_adj_smem_bytes(in, T, lv));
    if (sm > 227 * 1024) continue;
    const int nb = ws ? strips_adj_ws_occupancy(threads, sm) : strips_adj_occupancy(T, sm);
    if (nb < 1) continue;
    const long long ctas = (long long)n_strip_inst * ((batch + spc - 1) / spc);
    const double waves = ceil((double)ctas / ((double)nb * n_sm));
    const double warps = nb * threads / 32.0;
    const double cost = waves * (ws ? 1 : max_strips) / std::min(1.0, warps / 8.0);
    const bool forced = ctx->tune_adj_tile == T;
    if (forced || cost < best) {
      best = cost;
      *tile = spc;
      *smem = sm;
      *lv_floats = lv;
      *ws_threads = ws ? threads : 0;
    }
    if (forced) break;
  }
  if (!*tile) return fail(ctx, TNVAN_E_UNSUPPORTED, "strip adjoint needs more than 227 KB of shared memory");
  c.valid = !ctx->dirty;
  c.batch = batch;
  c.tune = ctx->tune_adj_tile;
  c.tile = *tile;
  c.smem = *smem;
  c.lv = *lv_floats;
  c.ws = *ws_threads;
  return TNVAN_OK;
}

int contract_all(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                 int precision, double* d_logZR, double* d_dbeta, cudaStream_t s, bool strips = true);
int run_adjoint(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins, int precision,
                double* d_logZR, double* d_dbeta, double* d_dJ, cudaStream_t s, const float* wmul = nullptr);
int plan_strip_adjoint(tnvan_ctx* ctx, int batch, int* tile, int* smem, int* lv_floats, int* ws_threads);
int pack_network(tnvan_ctx* ctx, int mask, cudaStream_t s);
int sampler_pack_mask(const tnvan_ctx* ctx, int precision);
int run_sampler(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step, int precision,
                int8_t* d_spins, float* d_logq, const int8_t* given, cudaStream_t s);
int pick_tc_plan(const tnvan_ctx* ctx);
// Every instance has a tensor-core sampler plan and all share one number of
// hidden layers (one kernel instantiation per launch).
bool tc_sampler_usable(const tnvan_ctx* ctx);
// Every instance fits the grouped form (the fast path).
bool tc_grouped_usable(const tnvan_ctx* ctx);
int tc_plan_value(const tnvan_ctx* ctx, int p);
int tc_sampler_smem(const tnvan_ctx* ctx, int plan, bool grouped);
// Some instance streams its weights in the grouped sampler's plan `plan`.
bool tc_any_streamed(const tnvan_ctx* ctx, int plan);
TcgOrder tcg_order(const tnvan_ctx* ctx, const LaunchInfo& li, int k0, int k1);
int backward_impl(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins, const double* d_logZR,
                  const float* d_logq, int precision, float* d_grad_params, double* d_dbeta, double* d_dJ,
                  cudaStream_t s, bool pack, const AdamArgs* adam, bool stats_ready = false);
AdamArgs adam_args(const tnvan_ctx* ctx, float* d_m, float* d_v, double lr, double beta1, double beta2, double eps,
                   int64_t t);
// The fused BF16 backward's launch shape: CTAs of `per` 128-sample tiles,
// about one CTA per SM overall; the gradient workspace holds one row per CTA.
struct FusedBwdPlan {
  LaunchInfo lf;
  int smem;
  long long max_elems;
};
int plan_fused_bwd(tnvan_ctx* ctx, const double* betas, int batch, FusedBwdPlan& p);
// Backward and Adam of each instance chunk, queued behind that chunk's
// adjoint and Eq. 9 reduction (whose mean is Eq. 10's baseline) in the
// overlapped schedule.
struct ChunkBackward {
  const FusedBwdPlan* plan;
  float* d_grad;
  const AdamArgs* adam;
};
int sample_contract_adjoint_impl(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step,
                                 int precision, int8_t* d_spins, float* d_logq, double* d_logZR, double* d_dbeta,
                                 double* d_dJ, cudaStream_t s, bool* dj_deferred = nullptr,
                                 bool* stats_done = nullptr, const ChunkBackward* cb = nullptr,
                                 bool* bwd_done = nullptr);

}  // namespace

int ensure_ws(tnvan_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return TNVAN_OK;
  if (ctx->d_ws) cudaFree(ctx->d_ws);
  ctx->d_ws = nullptr;
  ctx->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->d_ws, bytes);
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(workspace, %zu B): %s", bytes, cudaGetErrorString(e));
  ctx->ws_bytes = bytes;
  return TNVAN_OK;
}

// Floats of the tensor-core backward workspace for `batch` samples.
size_t tc_ws_floats(const tnvan_ctx* ctx, int batch) {
  // per instance: A1, A2, dX, dA2, dA1, w and the BF16 spins, each rounded up
  // to 16 floats by the carve; then the REINFORCE weights of all instances
  size_t tot = 0;
  for (const Instance& in : ctx->inst)
    tot += (size_t)batch * (2 * in.H[0] + 2 * in.H[1] + in.W.size() + 1) + 6 * 16 +
           ((size_t)batch * ((in.W.size() + 7) & ~size_t(7)) + 1) / 2 + 16;
  return tot + (size_t)ctx->inst.size() * batch + 16;
}

#define TC_SPLITS 16

// Backward of sum_b w_b log q(s_b) on the tensor cores (TF32 or BF16 operands,
// FP32 accumulation): forward chain, delta propagation, and split-K weight
// gradients (bias gradients ride along as an extra column of ones).
int backward_tc(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                const double* d_logZR, const float* d_logq, bool bf16, int part_stride,
                cudaStream_t s, bool skip_fused) {
  int rc;
  const int n = (int)ctx->inst.size();
  // instances the fused backward handles in the same call are left out
  auto skip = [&](int k) { return skip_fused && ctx->inst[k].dev.made.fused_ok; };
  if ((rc = ensure_ws(ctx, tc_ws_floats(ctx, batch) * sizeof(float)))) return rc;
  float* ws = static_cast<float*>(ctx->d_ws);
  struct Bufs { float *A1, *A2, *dX, *dA2, *dA1, *w; };
  std::vector<Bufs> bf(n);
  size_t off = 0;
  auto take = [&](size_t cnt) {
    float* p = ws + off;
    off += (cnt + 15) & ~size_t(15);
    return p;
  };
  for (int k = 0; k < n; ++k) {
    const Instance& in = ctx->inst[k];
    const size_t B = batch, D = in.W.size();
    bf[k].A1 = take(B * in.H[0]);
    bf[k].A2 = take(B * in.H[1]);
    bf[k].dX = take(B * D);
    bf[k].dA2 = take(B * in.H[1]);
    bf[k].dA1 = take(B * in.H[0]);
    bf[k].w = take(B);
  }
  // BF16 mode: the intermediates (A1 ... dA1) are stored in BF16 (the next
  // product's operands), the weights read from the packed BF16 copy and the
  // spins from a BF16 copy (rows of r8(D)) that the weights kernel writes; the
  // biases and the REINFORCE weights stay FP32
  const int IT = bf16 ? GT_BF16 : GT_F32;
  uint16_t* s16 = nullptr;
  std::vector<size_t> s16off(n, 0);
  if (bf16) {
    size_t tot16 = 0;
    for (int k = 0; k < n; ++k) {
      s16off[k] = tot16;
      tot16 += (size_t)batch * ((ctx->inst[k].W.size() + 7) & ~size_t(7));
    }
    s16 = reinterpret_cast<uint16_t*>(take((tot16 + 1) / 2));
  }
  auto wts = [&](const MadeDev& md, long long o) -> const void* {
    return bf16 ? static_cast<const void*>(md.packed16 + o) : static_cast<const void*>(md.packed + o);
  };
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  for (int k = 0; k < n; ++k)
    if (skip(k)) li.skip[k >> 5] |= 1u << (k & 31);  // no BF16 spins for the fused instances
  // per-instance REINFORCE weights laid out [k][batch] in one contiguous buffer
  float* wall = take((size_t)n * batch);
  {
    PROF("reinforce_w", s);
    CK(launch_reinforce_w(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats, wall, d_spins, s16, s), "weights kernel");
  }
  auto op = [](const void* p, long long sr, long long sk, int type) { return GemmOperand{p, sr, sk, type}; };
  auto spin_op = [&](int k, bool transposed) {
    const Instance& in = ctx->inst[k];
    const long long D = (long long)in.W.size(), D8 = (D + 7) & ~7LL;
    if (bf16) return transposed ? op(s16 + s16off[k], 1, D8, GT_BF16) : op(s16 + s16off[k], D8, 1, GT_BF16);
    const int8_t* S = d_spins + in.dev.spin_units * batch;
    return transposed ? op(S, 1, D, GT_I8) : op(S, D, 1, GT_I8);
  };
  std::vector<GemmProblem> probs;
  int max_m = 0, splits = 1;
  auto flush = [&](const char* name) -> int {
    for (size_t i = 0; i < probs.size(); i += GEMM_MAX_PROB) {
      GemmLaunch L;
      memset(&L, 0, sizeof L);
      L.status = ctx->d_status;
      const int cnt = (int)std::min<size_t>(GEMM_MAX_PROB, probs.size() - i);
      for (int j = 0; j < cnt; ++j) L.prob[j] = probs[i + j];
      PROF(name, s);
      CK(launch_gemm(L, cnt, max_m, splits, bf16, s), name);
    }
    probs.clear();
    max_m = 0;
    return TNVAN_OK;
  };
  auto base = [&](int M, int N, int K, GemmOperand A, GemmOperand Bo, int epi, float* C, long long ldc) {
    GemmProblem P;
    memset(&P, 0, sizeof P);
    P.M = M;
    P.N = N;
    P.K = K;
    P.A = A;
    P.B = Bo;
    P.ones_col = -1;
    P.epi = epi;
    P.C = C;
    P.ldc = ldc;
    return P;
  };
  const int B = batch;
  // stage 1: A1 = relu(S W1^T + b1)
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const Instance& in = ctx->inst[k];
    const MadeDev& md = in.dev.made;
    if (md.nh < 1) continue;
    const int D = md.D;
    const long long o1 = md.layer[0].dst_off;
    GemmProblem P = base(B, md.H1, D, spin_op(k, false), op(wts(md, o1), D, 1, IT), EPI_BIAS_RELU, bf[k].A1, md.H1);
    P.bias = md.packed + o1 + (long long)md.H1 * D;
    probs.push_back(P);
    max_m = std::max(max_m, B);
  }
  if ((rc = flush("gemm_fwd1"))) return rc;
  // stage 2: A2 = relu(A1 W2^T + b2)
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const MadeDev& md = ctx->inst[k].dev.made;
    if (md.nh < 2) continue;
    const long long o2 = md.layer[1].dst_off;
    GemmProblem P = base(B, md.H2, md.H1, op(bf[k].A1, md.H1, 1, IT), op(wts(md, o2), md.H1, 1, IT),
                         EPI_BIAS_RELU, bf[k].A2, md.H2);
    P.bias = md.packed + o2 + (long long)md.H2 * md.H1;
    probs.push_back(P);
    max_m = std::max(max_m, B);
  }
  if ((rc = flush("gemm_fwd2"))) return rc;
  // stage 3: dX = w_b s sigmoid(-s x), x = src Wo^T + bo
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const Instance& in = ctx->inst[k];
    const MadeDev& md = in.dev.made;
    const int D = md.D, Hl = md.Hl;
    const int8_t* S = d_spins + in.dev.spin_units * batch;
    const long long oo = md.layer[md.nh].dst_off;
    GemmOperand A = md.nh == 0 ? op(S, D, 1, GT_I8) : op(md.nh == 1 ? bf[k].A1 : bf[k].A2, Hl, 1, IT);
    GemmProblem P = base(B, D, Hl, A, op(wts(md, oo), Hl, 1, IT), EPI_DX, bf[k].dX, D);
    P.bias = md.packed + oo + (long long)D * Hl;
    P.spins = S;
    P.ld_spins = D;
    P.row_w = wall + (size_t)k * batch;
    probs.push_back(P);
    max_m = std::max(max_m, B);
  }
  if ((rc = flush("gemm_out_dx"))) return rc;
  // stage 4: delta of the last hidden layer = (dX Wo) * 1[h > 0]
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const MadeDev& md = ctx->inst[k].dev.made;
    if (md.nh < 1) continue;
    const int D = md.D, Hl = md.Hl;
    float* out = md.nh == 2 ? bf[k].dA2 : bf[k].dA1;
    const float* mask = md.nh == 2 ? bf[k].A2 : bf[k].A1;
    GemmProblem P = base(B, Hl, D, op(bf[k].dX, D, 1, IT), op(wts(md, md.layer[md.nh].dst_off), 1, Hl, IT), EPI_MASK,
                         out, Hl);
    P.mask = mask;
    P.ld_mask = Hl;
    probs.push_back(P);
    max_m = std::max(max_m, B);
  }
  if ((rc = flush("gemm_bwd_last"))) return rc;
  // stage 5: dA1 = (dA2 W2) * 1[h1 > 0]
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const MadeDev& md = ctx->inst[k].dev.made;
    if (md.nh < 2) continue;
    GemmProblem P = base(B, md.H1, md.H2, op(bf[k].dA2, md.H2, 1, IT), op(wts(md, md.layer[1].dst_off), 1, md.H1, IT),
                         EPI_MASK, bf[k].dA1, md.H1);
    P.mask = bf[k].A1;
    P.ld_mask = md.H1;
    probs.push_back(P);
    max_m = std::max(max_m, B);
  }
  if ((rc = flush("gemm_bwd_h1"))) return rc;
  // stage 6: weight gradients, split over the batch into TC_SPLITS partial slices
  splits = std::max(1, std::min(TC_SPLITS, (batch + 127) / 128));
  float* part = ctx->d_grad_packed;
  for (int k = 0; k < n; ++k) {
    if (skip(k)) continue;
    const Instance& in = ctx->inst[k];
    const MadeDev& md = in.dev.made;
    float* pk = part + (long long)k * splits * part_stride;
    for (int l = 0; l <= md.nh; ++l) {
      const LayerDev& L = md.layer[l];
      const float* delta = l == md.nh ? bf[k].dX : (l == 1 ? bf[k].dA2 : bf[k].dA1);
      GemmOperand act;
      if (l == 0) act = spin_op(k, true);
      else act = op(l == 1 ? bf[k].A1 : bf[k].A2, 1, L.nin, IT);
      for (int n0 = 0; n0 < L.nin; n0 += 128) {
        const bool last = n0 + 128 >= L.nin;
        const int nn = (L.nin + 1 <= 256) ? L.nin : std::min(128, L.nin - n0);
        GemmOperand actn = act;
        actn.ptr = static_cast<const char*>(act.ptr) + (size_t)n0 * (act.type == GT_F32 ? 4 : act.type == GT_BF16 ? 2 : 1);
        GemmProblem P = base(L.nout, nn, B, op(delta, 1, L.nout, IT), actn, EPI_STORE,
                             pk + L.dst_off + n0, L.nin);
        P.split_stride = part_stride;
        if (last || L.nin + 1 <= 256) {
          P.ones_col = nn;
          P.bias_out = pk + L.dst_off + (long long)L.nout * L.nin;
        }
        probs.push_back(P);
        max_m = std::max(max_m, L.nout);
        if (L.nin + 1 <= 256) break;
      }
    }
  }
  if ((rc = flush("gemm_wgrad"))) return rc;
  return TNVAN_OK;
}

// ===========================================================================
// Public API
// ===========================================================================
extern "C" {

int tnvan_version(void) { return 100; }

int tnvan_create(tnvan_ctx** out, int device) {
  if (!out) return fail(nullptr, TNVAN_E_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return fail(nullptr, TNVAN_E_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (device < 0 || device >= n) return fail(nullptr, TNVAN_E_ARG, "device %d out of range (%d devices)", device, n);
  tnvan_ctx* ctx = new (std::nothrow) tnvan_ctx();
  if (!ctx) return fail(nullptr, TNVAN_E_NOMEM, "host allocation failed");
  ctx->device = device;
  DeviceGuard g(device);
  // status words, then the reduction counters of the training path, then
  // those of tnvan_free_energy (its own, so that it may run beside a step)
  e = cudaMalloc(&ctx->d_status, (4 + 2 * TNVAN_MAX_INST) * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, (4 + 2 * TNVAN_MAX_INST) * sizeof(int));
  if (e != cudaSuccess) {
    delete ctx;
    return fail(nullptr, TNVAN_E_NOMEM, "cudaMalloc(status): %s", cudaGetErrorString(e));
  }
  const size_t stats_doubles = 8 * TNVAN_MAX_INST + (size_t)TNVAN_MAX_INST * 64 * 6;
  e = cudaMalloc(&ctx->d_stats, 2 * stats_doubles * sizeof(double));  // training path | tnvan_free_energy
  ctx->d_stats_fe = e == cudaSuccess ? ctx->d_stats + stats_doubles : nullptr;
  if (e != cudaSuccess) {
    delete ctx;
    return fail(nullptr, TNVAN_E_NOMEM, "cudaMalloc(stats): %s", cudaGetErrorString(e));
  }
  *out = ctx;
  return TNVAN_OK;
}

int tnvan_destroy(tnvan_ctx* ctx) {
  if (!ctx) return TNVAN_OK;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (Instance& in : ctx->inst) free_instance(in);
  for (auto& r : ctx->prof)
    for (auto& pr : r.pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (cudaStream_t st : ctx->side)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : ctx->side_lo)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : ctx->chunk_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->adj_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->dj_ev) cudaEventDestroy(ctx->dj_ev);
  for (cudaEvent_t e : ctx->join_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->d_inst) cudaFree(ctx->d_inst);
  if (ctx->d_stats) cudaFree(ctx->d_stats);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_grad_packed) cudaFree(ctx->d_grad_packed);
  if (ctx->d_ws) cudaFree(ctx->d_ws);
  if (ctx->d_obs) cudaFree(ctx->d_obs);
  if (ctx->d_dj_part) cudaFree(ctx->d_dj_part);
  if (ctx->d_wide_part) cudaFree(ctx->d_wide_part);
  if (ctx->prof_ref) cudaEventDestroy(ctx->prof_ref);
  for (float* p : ctx->d_gen_scratch)
    if (p) cudaFree(p);
  delete ctx;
  return TNVAN_OK;
}

const char* tnvan_last_error(const tnvan_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

int tnvan_init_graph(tnvan_ctx* ctx, int instance, int n_spins, int n_edges, const int32_t* ei,
                     const int32_t* ej, const double* J, int topology, int Lx, int Ly,
                     int periodic) {
  int rc = check_inst(ctx, instance, true);
  if (rc) return rc;
  if (n_spins < 1 || n_edges < 0 || (n_edges > 0 && (!ei || !ej || !J)))
    return fail(ctx, TNVAN_E_ARG, "bad graph sizes or NULL arrays");
  if (topology < 0 || topology > 2) return fail(ctx, TNVAN_E_ARG, "unknown topology %d", topology);
  if (topology == TNVAN_LATTICE2D) {
    if (periodic) return fail(ctx, TNVAN_E_UNSUPPORTED, "periodic lattices are not supported");
    if (Lx < 1 || Ly < 1 || (long long)Lx * Ly != n_spins)
      return fail(ctx, TNVAN_E_ARG, "lattice %d x %d does not match %d spins", Lx, Ly, n_spins);
  }
  std::map<std::pair<int, int>, int> seen;
  for (int e = 0; e < n_edges; ++e) {
    if (ei[e] < 0 || ej[e] < 0 || ei[e] >= n_spins || ej[e] >= n_spins || ei[e] == ej[e])
      return fail(ctx, TNVAN_E_ARG, "edge %d (%d,%d) invalid", e, ei[e], ej[e]);
    if (!isfinite(J[e])) return fail(ctx, TNVAN_E_ARG, "J[%d] is not finite", e);
    auto key = std::make_pair(std::min(ei[e], ej[e]), std::max(ei[e], ej[e]));
    if (!seen.emplace(key, e).second) return fail(ctx, TNVAN_E_ARG, "edge %d repeats a pair", e);
  }
  DeviceGuard g(ctx->device);
  if (instance == (int)ctx->inst.size()) ctx->inst.emplace_back();
  Instance& in = ctx->inst[instance];
  reset_plan(in);
  in.has_graph = true;
  in.n = n_spins;
  in.m = n_edges;
  in.topology = topology;
  in.Lx = Lx;
  in.Ly = Ly;
  in.ei.assign(ei, ei + n_edges);
  in.ej.assign(ej, ej + n_edges);
  in.J.assign(J, J + n_edges);
  in.W.clear();
  in.n_params = 0;
  ctx->dirty = true;
  ctx->adj_plan.valid = 0;
  return TNVAN_OK;
}

int tnvan_set_width_set(tnvan_ctx* ctx, int instance, int n_w, const int32_t* w) {
  return tnvan_set_width_set_ordered(ctx, instance, n_w, w, nullptr);
}

int tnvan_set_width_set_ordered(tnvan_ctx* ctx, int instance, int n_w, const int32_t* w,
                                const int32_t* r_order) {
  int rc = check_inst(ctx, instance, false);
  if (rc) return rc;
  Instance& in = ctx->inst[instance];
  if (!in.has_graph) return fail(ctx, TNVAN_E_STATE, "instance %d has no graph", instance);
  if (n_w < 1 || n_w > TNVAN_MAX_D || !w) return fail(ctx, TNVAN_E_ARG, "n_w = %d out of range [1, %d]", n_w, TNVAN_MAX_D);
  std::vector<int> pos(in.n, -1);
  for (int i = 0; i < n_w; ++i) {
    if (w[i] < 0 || w[i] >= in.n) return fail(ctx, TNVAN_E_ARG, "w[%d] = %d out of range", i, w[i]);
    if (pos[w[i]] >= 0) return fail(ctx, TNVAN_E_ARG, "w[%d] = %d repeated", i, w[i]);
    pos[w[i]] = i;
  }
  std::vector<int> rank;
  if (r_order) {
    rank.assign(in.n, -1);
    for (int k = 0; k < in.n - n_w; ++k) {
      const int v = r_order[k];
      if (v < 0 || v >= in.n || pos[v] >= 0 || rank[v] >= 0)
        return fail(ctx, TNVAN_E_ARG, "r_order[%d] = %d is not a spin of R or repeated", k, v);
      rank[v] = k;
    }
  }
  DeviceGuard g(ctx->device);
  reset_plan(in);
  in.W.assign(w, w + n_w);
  in.ww.clear();
  in.wide = HostWidePlan{};
  std::map<std::pair<int, int>, int> edge_of;
  for (int e = 0; e < in.m; ++e) {
    edge_of[{std::min(in.ei[e], in.ej[e]), std::max(in.ei[e], in.ej[e])}] = e;
    const int a = pos[in.ei[e]], b = pos[in.ej[e]];
    if (a >= 0 && b >= 0) in.ww.push_back(EdgeWW{a, b, (float)in.J[e], e});
  }
  auto comps = r_components(in, pos);
  in.n_comp = (int)comps.size();
  in.max_comp = 0;
  for (auto& c : comps) in.max_comp = std::max(in.max_comp, (int)c.size());
  in.max_width = 0;
  rc = TNVAN_E_UNSUPPORTED;
  if (in.topology == TNVAN_LATTICE2D) {
    rc = plan_strips(ctx, in, edge_of, pos);
    if (rc == TNVAN_OK) {
      int mw = 0;
      for (auto& sd : in.strip.strips) mw = std::max(mw, sd.w);
      in.max_width = mw;
    } else if (rc != TNVAN_E_UNSUPPORTED) {
      return rc;
    }
  } else if (in.topology == TNVAN_DENSE) {
    rc = plan_dense(ctx, in, pos);
    if (rc != TNVAN_OK && rc != TNVAN_E_UNSUPPORTED) return rc;
  }
  if (rc == TNVAN_OK && r_order) return fail(ctx, TNVAN_E_ARG, "r_order is only used by elimination plans");
  if (rc == TNVAN_E_UNSUPPORTED) {
    ctx->err.clear();
    if (in.topology == TNVAN_LATTICE2D && rank.empty()) {
      // a lattice whose strips are too wide for the strip kernels: eliminate
      // row by row (width = the widest strip), else by min-fill
      std::vector<int> rm(in.n, -1);
      int r = 0;
      for (int v = 0; v < in.n; ++v)
        if (pos[v] < 0) rm[v] = r++;
      rc = plan_general(ctx, in, pos, rm);
      if (rc == TNVAN_E_UNSUPPORTED) {
        ctx->err.clear();
        rc = plan_general(ctx, in, pos, rank);
      }
    } else {
      rc = plan_general(ctx, in, pos, rank);
    }
    if (rc) return rc;
    plan_wide_strips(in, edge_of, pos);
  }
  if ((rc = upload_plan(ctx, in))) return rc;
  in.has_ws = true;
  in.has_made = false;
  ctx->dirty = true;
  ctx->adj_plan.valid = 0;
  return TNVAN_OK;
}

int tnvan_set_made(tnvan_ctx* ctx, int instance, int n_hidden, const int32_t* widths,
                   float* d_params) {
  int rc = check_inst(ctx, instance, false);
  if (rc) return rc;
  Instance& in = ctx->inst[instance];
  if (!in.has_ws) return fail(ctx, TNVAN_E_STATE, "instance %d has no width set", instance);
  if (n_hidden < 0 || n_hidden > 2 || (n_hidden > 0 && !widths))
    return fail(ctx, TNVAN_E_ARG, "n_hidden = %d (0..2)", n_hidden);
  if (!d_params) return fail(ctx, TNVAN_E_ARG, "d_params is NULL");
  const int D = (int)in.W.size();
  int H[2] = {0, 0};
  for (int l = 0; l < n_hidden; ++l) {
    if (widths[l] < 1 || widths[l] > TNVAN_MAX_HIDDEN)
      return fail(ctx, TNVAN_E_ARG, "hidden width %d out of range [1, %d]", widths[l], TNVAN_MAX_HIDDEN);
    H[l] = widths[l];
  }
  DeviceGuard g(ctx->device);
  const int cyc = std::max(D - 1, 1);
  // integer buffer: degIO [D] | deg1s [H1] | deg2s [H2] | perm1 [H1] | perm2 [H2] | c1 [D+1] | c2 [D+1]
  std::vector<int> buf;
  std::vector<int> degIO(D), deg1(H[0]), deg2(H[1]), perm1(H[0]), perm2(H[1]);
  for (int i = 0; i < D; ++i) degIO[i] = i + 1;
  auto sorted = [&](int Hn, std::vector<int>& perm, std::vector<int>& deg) {
    std::vector<int> raw(Hn);
    for (int k = 0; k < Hn; ++k) raw[k] = k % cyc + 1;
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return raw[a] < raw[b]; });
    for (int k = 0; k < Hn; ++k) deg[k] = raw[perm[k]];
  };
  sorted(H[0], perm1, deg1);
  sorted(H[1], perm2, deg2);
  std::vector<int> c1(D + 1, 0), c2(D + 1, 0);
  for (int d = 0; d <= D; ++d) {
    c1[d] = (int)std::count_if(deg1.begin(), deg1.end(), [d](int x) { return x <= d; });
    c2[d] = (int)std::count_if(deg2.begin(), deg2.end(), [d](int x) { return x <= d; });
  }
  const int o_deg = 0, o_d1 = D, o_d2 = o_d1 + H[0], o_p1 = o_d2 + H[1], o_p2 = o_p1 + H[0],
            o_c1 = o_p2 + H[1], o_c2 = o_c1 + D + 1;
  buf.insert(buf.end(), degIO.begin(), degIO.end());
  buf.insert(buf.end(), deg1.begin(), deg1.end());
  buf.insert(buf.end(), deg2.begin(), deg2.end());
  buf.insert(buf.end(), perm1.begin(), perm1.end());
  buf.insert(buf.end(), perm2.begin(), perm2.end());
  buf.insert(buf.end(), c1.begin(), c1.end());
  buf.insert(buf.end(), c2.begin(), c2.end());
  (void)o_c2;
  int* dbuf = nullptr;
  if ((rc = upload(ctx, in, buf, &dbuf))) return rc;
  MadeDev md{};
  md.D = D;
  md.nh = n_hidden;
  md.H1 = H[0];
  md.H2 = H[1];
  md.Hl = n_hidden == 0 ? D : H[n_hidden - 1];
  md.n_layers = n_hidden + 1;
  const int sizes[4] = {D, H[0], H[1], D};
  int szl[4];
  int nl = 0;
  szl[nl++] = D;
  for (int l = 0; l < n_hidden; ++l) szl[nl++] = H[l];
  szl[nl++] = D;
  (void)sizes;
  const int* degp[4];
  const int* permp[4];
  degp[0] = dbuf + o_deg;
  permp[0] = nullptr;
  if (n_hidden >= 1) {
    degp[1] = dbuf + o_d1;
    permp[1] = dbuf + o_p1;
  }
  if (n_hidden >= 2) {
    degp[2] = dbuf + o_d2;
    permp[2] = dbuf + o_p2;
  }
  degp[n_hidden + 1] = dbuf + o_deg;
  permp[n_hidden + 1] = nullptr;
  long long off = 0;
  for (int l = 0; l <= n_hidden; ++l) {
    LayerDev& L = md.layer[l];
    L.nin = szl[l];
    L.nout = szl[l + 1];
    L.src_off = off;
    L.dst_off = off;
    L.perm_in = permp[l];
    L.perm_out = permp[l + 1];
    L.deg_in = degp[l];
    L.deg_out = degp[l + 1];
    L.strict = (l == n_hidden) ? 1 : 0;
    off += (long long)L.nout * L.nin + L.nout;
  }
  md.n_params = off;
  if (off >= (1LL << 30)) return fail(ctx, TNVAN_E_UNSUPPORTED, "network too large (%lld parameters)", off);
  const int Dp16 = (D + 15) & ~15;  // the fused backward pads D to a multiple of 16
  // TMEM of the fused kernel: 128 scratch columns, then the weight-gradient
  // accumulators [S | 1], [A1 | 1], [A2 | 1] (the ones column of S sits in
  // its padding when D is not a multiple of 16)
  const int g1n = (D % 16) ? Dp16 : Dp16 + 16;
  md.fused_ok = n_hidden == 2 && H[0] % 16 == 0 && H[1] % 16 == 0 && Dp16 <= 128 && H[0] <= 128 &&
                H[1] <= 128 && 128 + g1n + (H[0] + 16) + (H[1] + 16) <= 512 &&
                fused_bwd_smem_bytes(D, H[0], H[1]) <= 227 * 1024;
  md.sample_tc_ok = 0;  // decided once the step groups are known
  md.wtiles = nullptr;
  if (md.fused_ok || (n_hidden == 2 && H[0] % 16 == 0 && H[1] % 16 == 0 && Dp16 <= 128 && H[0] <= 128 &&
                      H[1] <= 128)) {
    void* wt = nullptr;
    const size_t n = (size_t)H[0] * Dp16 + (size_t)H[1] * H[0] + (size_t)Dp16 * H[1];
    cudaError_t e2 = cudaMalloc(&wt, n * sizeof(uint16_t));
    if (e2 == cudaSuccess) e2 = cudaMemset(wt, 0, n * sizeof(uint16_t));  // the padding stays zero
    if (e2 != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(weight tiles): %s", cudaGetErrorString(e2));
    in.dev_allocs.push_back(wt);
    md.wtiles = static_cast<uint16_t*>(wt);
  }
  md.c1 = dbuf + o_c1;
  md.c2 = dbuf + o_c2;
  md.raw = d_params;
  // Step groups of the blocked sampler: at most 8 steps and 32 units of each
  // hidden layer completing inside a group.  Per group, one contiguous weight
  // block (gathered from `packed` on every call) holds, in order:
  //   L1 / L2 / output pre-activation tiles: chunks of 16 units, [n_in][16];
  //   in-group triangles TW1 [n1][gi], TW2 [n2][n1], TWo [gi][nL]
  //   (n1, n2 = the group's layer units, gi = its steps, nL = the width feeding
  //   the output inside the group), each padded to a multiple of 4 floats.
  {
    const int GMAX = 8, UGMAX = 32;
    auto before = [](const std::vector<int>& c, int d) { return d >= 1 ? c[d - 1] : 0; };  // deg < d
    auto cnt = [&](const std::vector<int>& c, int a, int b) { return before(c, b) - before(c, a); };
    std::vector<int> grp, src;
    int ug1 = 0, ug2 = 0, ugo = 0, wmax = 0;
    const int Hl = md.Hl;
    auto pad4 = [&]() {
      while (src.size() % 4) src.push_back(-1);
    };
    auto add_blocks = [&](int n_in, int lo, int hi, long long wofs, int stride) {
      const int off = (int)src.size();
      for (int c = lo; c < hi; c += 16)
        for (int j = 0; j < n_in; ++j)
          for (int q = 0; q < 16; ++q) {
            const int u = c + q;
            src.push_back(u < hi ? (int)(wofs + (long long)u * stride + j) : -1);
          }
      return off;
    };
    auto add_tile = [&](int rlo, int rhi, int clo, int chi, long long wofs, int stride) {
      const int off = (int)src.size();
      for (int r = rlo; r < rhi; ++r)
        for (int c = clo; c < chi; ++c) src.push_back((int)(wofs + (long long)r * stride + c));
      pad4();
      return off;
    };
    for (int i0 = 0; i0 < D;) {
      int i1 = i0 + 1;
      while (i1 < D && i1 - i0 < GMAX && cnt(c1, i0, i1 + 1) <= UGMAX && cnt(c2, i0, i1 + 1) <= UGMAX) ++i1;
      const int u1lo = before(c1, i0), u1hi = before(c1, i1);
      const int u2lo = before(c2, i0), u2hi = before(c2, i1);
      ug1 = std::max(ug1, u1hi - u1lo);
      ug2 = std::max(ug2, u2hi - u2lo);
      ugo = std::max(ugo, i1 - i0);
      const int gstart = (int)src.size();
      int off1 = 0, off2 = 0, offo = 0, t1 = 0, t2 = 0, to = 0;
      if (n_hidden >= 1) off1 = add_blocks(i0, u1lo, u1hi, md.layer[0].dst_off, D);
      if (n_hidden >= 2) off2 = add_blocks(u1lo, u2lo, u2hi, md.layer[1].dst_off, H[0]);
      const int n_in_o = n_hidden == 0 ? i0 : (n_hidden == 1 ? u1lo : u2lo);
      offo = add_blocks(n_in_o, i0, i1, md.layer[n_hidden].dst_off, Hl);
      if (n_hidden >= 1) t1 = add_tile(u1lo, u1hi, i0, i1, md.layer[0].dst_off, D);
      if (n_hidden >= 2) t2 = add_tile(u2lo, u2hi, u1lo, u1hi, md.layer[1].dst_off, H[0]);
      {
        const int clo = n_hidden == 0 ? i0 : (n_hidden == 1 ? u1lo : u2lo);
        const int chi = n_hidden == 0 ? i1 : (n_hidden == 1 ? u1hi : u2hi);
        to = add_tile(i0, i1, clo, chi, md.layer[n_hidden].dst_off, Hl);
      }
      pad4();
      const int gsize = (int)src.size() - gstart;
      wmax = std::max(wmax, gsize);
      grp.insert(grp.end(), {i0, i1, u1lo, u1hi, u2lo, u2hi, n_hidden >= 1 ? off1 - gstart : 0,
                             n_hidden >= 2 ? off2 - gstart : 0, offo - gstart, gstart, gsize, 0,
                             n_hidden >= 1 ? t1 - gstart : 0, n_hidden >= 2 ? t2 - gstart : 0,
                             to - gstart});
      i0 = i1;
    }
    int* dgrp = nullptr;
    if ((rc = upload(ctx, in, grp, &dgrp))) return rc;
    int* dsrc = nullptr;
    if ((rc = upload(ctx, in, src, &dsrc))) return rc;
    void* blk = nullptr;
    if (!src.empty()) {
      cudaError_t e2 = cudaMalloc(&blk, src.size() * sizeof(float));
      if (e2 != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(sampler blocks): %s", cudaGetErrorString(e2));
      in.dev_allocs.push_back(blk);
    }
    md.n_groups = (int)grp.size() / GROUP_INTS;
    md.wmax = wmax;
    md.groups = dgrp;
    md.ug1 = ug1;
    md.ug2 = ug2;
    md.ugo = ugo;
    md.blocks = static_cast<float*>(blk);
    md.blk_src = dsrc;
    md.n_blk = (long long)src.size();
  }
  // Step chunks of the tensor-core sampler, one plan per chunk-size limit
  // (kTcGroupMax; the autotuner picks one): at most that many steps and 64
  // layer-1 units completing inside a chunk.  Per chunk a record of
  // TNVAN_TCG_INTS ints and one BF16 weight blob of three parts, each in the
  // MMA's K-major canonical layout (core matrices of 8 rows x 16 bytes):
  //   A  W2's columns [w1c, w1c + n1c) for every layer-2 row: n1c / 16 slabs of
  //      [H2 rows][16], element (r, kk) at (r >> 3) * 128 + (kk >> 3) * 64 +
  //      (r & 7) * 8 + (kk & 7) within its slab (two hidden layers only);
  //   B  Wo's columns over the chunk's last-layer units, [Dp rows][16] slabs;
  //   C  W1's rows [w1c, w1c + n1c) over the spins 0 .. kSc-1, row groups of
  //      8: element (r, k) at (r >> 3) * 8 kSc + (k >> 3) * 64 + (r & 7) * 8 + (k & 7).
  // Rows past the network (outputs >= D, spins >= D) are zero.
  {
    const int Dp = (D + 15) & ~15;
    const bool shape_ok = (n_hidden == 1 || n_hidden == 2) && Dp <= 256 && H[0] % 16 == 0 && H[0] <= 256 &&
                          (n_hidden == 1 || (H[1] % 16 == 0 && H[1] <= 256));
    const int Hl = n_hidden == 2 ? H[1] : H[0];
    const long long wofs = md.layer[n_hidden].dst_off;  // output layer
    auto before = [](const std::vector<int>& c, int i) { return i >= 1 ? c[i - 1] : 0; };  // degree < i
    for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
      MadeDev::TcPlan& P = md.tc[p];
      P = MadeDev::TcPlan{};
      if (!shape_ok) continue;
      const int CMAX = kTcGroupMax[p];
      std::vector<int> rec, src;
      int tcw1 = 16, dw1 = 16, dw2 = 16, wbmax = 0;
      bool fits = true;
      for (int i = 0; i < D; ++i) {  // per-step unit windows (the delta tiles)
        const int ua = before(c1, i), ub = before(c1, i + 1);
        if (ub > ua) dw1 = std::max(dw1, ((ub + 15) & ~15) - (ua & ~15));
        if (n_hidden == 2) {
          const int va = before(c2, i), vb = before(c2, i + 1);
          if (vb > va) dw2 = std::max(dw2, ((vb + 15) & ~15) - (va & ~15));
        }
      }
      fits = fits && dw1 <= 64 && dw2 <= 64;
      for (int i0 = 0; i0 < D && fits;) {
        // units completing at steps [i0, i1): degree in [i0, i1 - 1]
        auto win = [&](const std::vector<int>& c, int a, int b, int& w, int& n) {
          const int lo = before(c, a), hi = before(c, b);
          if (hi <= lo) {
            w = lo & ~15;
            n = 0;
          } else {
            w = lo & ~15;
            n = ((hi + 15) & ~15) - w;
          }
        };
        int i1 = i0 + 1;
        while (i1 < D && i1 - i0 < CMAX) {
          int w, n;
          win(c1, i0, i1 + 1, w, n);
          if (n > 64) break;
          ++i1;
        }
        int w1c, n1c, w2c = 0, n2c = 0;
        win(c1, i0, i1, w1c, n1c);
        if (n_hidden == 2) win(c2, i0, i1, w2c, n2c);
        if (n1c > 64) fits = false;
        const int kSc = std::min(Dp, std::max(16, (i1 + 15) & ~15));
        const int wL = n_hidden == 2 ? w2c : w1c, nL = n_hidden == 2 ? n2c : n1c;
        const int off = (int)src.size();
        const int nA = n_hidden == 2 ? H[1] * n1c : 0, nB = Dp * nL, nC = n1c * kSc;
        src.resize(src.size() + nA + nB + nC, -1);
        int* A = src.data() + off;
        int* Bp = A + nA;
        int* C = Bp + nB;
        for (int sl = 0; sl < n1c / 16 && n_hidden == 2; ++sl)  // W2 [H2][H1], column = layer-1 unit
          for (int r = 0; r < H[1]; ++r)
            for (int kk = 0; kk < 16; ++kk)
              A[sl * H[1] * 16 + (r >> 3) * 128 + (kk >> 3) * 64 + (r & 7) * 8 + (kk & 7)] =
                  (int)(md.layer[1].dst_off + (long long)r * H[0] + w1c + 16 * sl + kk);
        for (int sl = 0; sl < nL / 16; ++sl)  // Wo [D][Hl]
          for (int r = 0; r < D; ++r)
            for (int kk = 0; kk < 16; ++kk)
              Bp[sl * Dp * 16 + (r >> 3) * 128 + (kk >> 3) * 64 + (r & 7) * 8 + (kk & 7)] =
                  (int)(wofs + (long long)r * Hl + wL + 16 * sl + kk);
        for (int r = 0; r < n1c; ++r)  // W1 [H1][D]
          for (int k2 = 0; k2 < std::min(kSc, D); ++k2)
            C[(r >> 3) * 8 * kSc + (k2 >> 3) * 64 + (r & 7) * 8 + (k2 & 7)] =
                (int)(md.layer[0].dst_off + (long long)(w1c + r) * D + k2);
        const int bytes = 2 * (nA + nB + nC);
        wbmax = std::max(wbmax, bytes);
        tcw1 = std::max(tcw1, n1c);
        int r16[TNVAN_TCG_INTS] = {i0, i1, w1c, n1c, w2c, n2c, kSc, off, 2 * nA, 2 * nB, 2 * nC};
        rec.insert(rec.end(), r16, r16 + TNVAN_TCG_INTS);
        i0 = i1;
      }
      // in-step weights of every step (the layer-1 -> layer-2 block, then the
      // last hidden layer -> output i row)
      std::vector<int> soff(D + 1, 0), ssrc;
      for (int i = 0; i < D; ++i) {
        soff[i] = (int)ssrc.size();
        const int ua = before(c1, i), ub = before(c1, i + 1);
        if (n_hidden == 2) {
          const int va = before(c2, i), vb = before(c2, i + 1);
          for (int v = va; v < vb; ++v)
            for (int u = ua; u < ub; ++u) ssrc.push_back((int)(md.layer[1].dst_off + (long long)v * H[0] + u));
          for (int v = va; v < vb; ++v) ssrc.push_back((int)(wofs + (long long)i * Hl + v));
        } else {
          for (int u = ua; u < ub; ++u) ssrc.push_back((int)(wofs + (long long)i * Hl + u));
        }
      }
      soff[D] = (int)ssrc.size();
      const int need_cols = tcw1 + (n_hidden == 2 ? H[1] : 0) + Dp;
      int cols = 32;
      while (cols < need_cols) cols *= 2;
      fits = fits && cols <= 512;
      if (!fits) continue;
      int* drec = nullptr;
      if ((rc = upload(ctx, in, rec, &drec))) return rc;
      if ((rc = upload_blob(ctx, in, src, &P.wblob, &P.wsrc, &P.wdst, &P.n_wblob))) return rc;
      int* dsoff = nullptr;
      if ((rc = upload(ctx, in, soff, &dsoff))) return rc;
      int* dssrc = nullptr;
      if (!ssrc.empty() && (rc = upload(ctx, in, ssrc, &dssrc))) return rc;
      void* stab = nullptr;
      cudaError_t e2 = cudaMalloc(&stab, std::max<size_t>(ssrc.size(), 1) * sizeof(float));
      if (e2 != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(sampler step tables): %s", cudaGetErrorString(e2));
      in.dev_allocs.push_back(stab);
      P.steptab = static_cast<float*>(stab);
      P.stepsrc = dssrc;
      P.stepoff = dsoff;
      P.n_steptab = (int)ssrc.size();
      P.n_chunks = (int)rec.size() / TNVAN_TCG_INTS;
      P.chunks = drec;
      P.dp = Dp;
      P.tcw1 = tcw1;
      P.dw1 = dw1;
      P.dw2 = n_hidden == 2 ? dw2 : 0;
      P.wbmax = wbmax;
      P.tmem_cols = cols;
      MadeDev probe = md;
      probe.nh = n_hidden;
      probe.tc[p] = P;
      P.ok = sample_tc_smem_bytes(probe, p) <= 227 * 1024;
    }
  }
  // Step groups of the grouped tensor-core sampler (the fast path for two
  // hidden layers of <= 128 units and D <= 128, a multiple of 16), one plan
  // per group-size limit (kTcGroupMaxG): at most that many steps and 32 units
  // of each hidden layer completing inside a group.  Per group the in-group
  // triangles and the group's biases, each row padded to a multiple of 4
  // floats, and a record of TNVAN_TCGG_INTS ints (bounds, offsets and the
  // per-step unit counts) that the kernel bulk-copies one group ahead.
  for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
    MadeDev::TcGroupPlan& P = md.tcg[p];
    P = MadeDev::TcGroupPlan{};
    if (n_hidden != 2 || H[0] % 16 || H[1] % 16 || H[0] > 256 || H[1] > 256 || ((D + 15) & ~15) > 256) continue;
    const int GMAX = kTcGroupMaxG[p], UGMAX = 32;
    auto before = [](const std::vector<int>& c, int d) { return d >= 1 ? c[d - 1] : 0; };  // deg < d
    auto cnt = [&](const std::vector<int>& c, int a, int b) { return before(c, b) - before(c, a); };
    std::vector<int> grp, src;
    int twmax = 0, tcw1 = 16, tcw2 = 16;
    bool fits = true;
    // most units of one layer completing at one step: up to 4, the slot layout
    // (the kernel keeps the group's hidden values in registers)
    int umax = 1;
    for (int i = 0; i < D; ++i) umax = std::max({umax, cnt(c1, i, i + 1), cnt(c2, i, i + 1)});
    const int U = umax <= 4 ? std::max(umax, 2) : 0;
    P.slot_u = U;
    auto add_tile = [&](int rlo, int rhi, int clo, int chi, long long wofs, int stride) {
      const int off = (int)src.size();
      const int rw = (chi - clo + 3) & ~3;
      for (int r = rlo; r < rhi; ++r)
        for (int c = 0; c < rw; ++c) src.push_back(c < chi - clo ? (int)(wofs + (long long)r * stride + clo + c) : -1);
      return off;
    };
    for (int i0 = 0; i0 < D;) {
      int i1 = i0 + 1;
      while (i1 < D && i1 - i0 < GMAX && cnt(c1, i0, i1 + 1) <= UGMAX && cnt(c2, i0, i1 + 1) <= UGMAX) ++i1;
      const int u1lo = before(c1, i0), u1hi = before(c1, i1);
      const int u2lo = before(c2, i0), u2hi = before(c2, i1);
      fits = fits && u1hi - u1lo <= UGMAX && u2hi - u2lo <= UGMAX;
      const int gstart = (int)src.size();
      int t2, to, b1o, b2o, boo;
      if (U == 0) {
        add_tile(u1lo, u1hi, i0, i1, md.layer[0].dst_off, D);
        t2 = add_tile(u2lo, u2hi, u1lo, u1hi, md.layer[1].dst_off, H[0]);
        to = add_tile(i0, i1, u2lo, u2hi, md.layer[2].dst_off, H[1]);
        // the group's biases (gathered with the triangles)
        b1o = add_tile(0, 1, u1lo, u1hi, md.layer[0].dst_off + (long long)H[0] * D, 0);
        b2o = add_tile(0, 1, u2lo, u2hi, md.layer[1].dst_off + (long long)H[1] * H[0], 0);
        boo = add_tile(0, 1, i0, i1, md.layer[2].dst_off + (long long)D * H[1], 0);
      } else {
        // slot layout (strides for 8 steps whatever the group's length): slot
        // (q, a) is unit a of those completing at step i0 + q (empty: zeros)
        //   TW1 [8U][8]   layer-1 slot x in-group spin j < q
        //   TW2 [8U][8U]  layer-2 slot (q, b) x layer-1 slot (q', a'), q' <= q
        //   TWo [8][8U]   output i0 + q x layer-2 slot (q', b'), q' <= q
        //   b1 [8U], b2 [8U], bo [8]
        const int gi = i1 - i0, S = 8 * U;
        auto u_at = [&](const std::vector<int>& c, int q, int a) {  // unit of slot (q, a), -1 empty
          if (q >= gi) return -1;
          const int lo = before(c, i0 + q), hi = before(c, i0 + q + 1);
          return a < hi - lo ? lo + a : -1;
        };
        const long long o0 = md.layer[0].dst_off, o1 = md.layer[1].dst_off, o2 = md.layer[2].dst_off;
        for (int r = 0; r < S; ++r)
          for (int j = 0; j < 8; ++j) {
            const int u = u_at(c1, r / U, r % U);
            src.push_back(u >= 0 && j < r / U ? (int)(o0 + (long long)u * D + i0 + j) : -1);
          }
        t2 = (int)src.size();
        for (int r = 0; r < S; ++r)
          for (int c = 0; c < S; ++c) {
            const int v = u_at(c2, r / U, r % U), u = u_at(c1, c / U, c % U);
            src.push_back(v >= 0 && u >= 0 && c / U <= r / U ? (int)(o1 + (long long)v * H[0] + u) : -1);
          }
        to = (int)src.size();
        for (int q = 0; q < 8; ++q)
          for (int c = 0; c < S; ++c) {
            const int v = u_at(c2, c / U, c % U);
            src.push_back(q < gi && v >= 0 && c / U <= q ? (int)(o2 + (long long)(i0 + q) * H[1] + v) : -1);
          }
        b1o = (int)src.size();
        for (int r = 0; r < S; ++r) {
          const int u = u_at(c1, r / U, r % U);
          src.push_back(u >= 0 ? (int)(o0 + (long long)H[0] * D + u) : -1);
        }
        b2o = (int)src.size();
        for (int r = 0; r < S; ++r) {
          const int v = u_at(c2, r / U, r % U);
          src.push_back(v >= 0 ? (int)(o1 + (long long)H[1] * H[0] + v) : -1);
        }
        boo = (int)src.size();
        for (int q = 0; q < 8; ++q) src.push_back(q < gi ? (int)(o2 + (long long)D * H[1] + i0 + q) : -1);
      }
      const int gsize = (int)src.size() - gstart;
      twmax = std::max(twmax, gsize);
      tcw1 = std::max(tcw1, ((u1hi + 15) & ~15) - (u1lo & ~15));
      tcw2 = std::max(tcw2, ((u2hi + 15) & ~15) - (u2lo & ~15));
      int rec[TNVAN_TCGG_INTS] = {i0, i1, u1lo, u1hi, u2lo, u2hi, gstart, gsize, t2 - gstart, to - gstart,
                                  b1o - gstart, b2o - gstart, boo - gstart};
      for (int q = 0; q <= i1 - i0; ++q) {  // units with degree < i0 + q
        rec[13 + q] = before(c1, i0 + q);
        rec[22 + q] = before(c2, i0 + q);
      }
      grp.insert(grp.end(), rec, rec + TNVAN_TCGG_INTS);
      i0 = i1;
    }
    // the weight tiles resident in shared memory (D <= 128 and room for
    // them), else one streamed blob per group: the W2 window [H2 x n1] (the
    // fold of the group's layer-1 units), the Wo window [Dp x n2] (its
    // layer-2 units) and W1's rows of its layer-1 units [n1 x r16(i0)] (their
    // pre-activations, recomputed at the end of the group before), each in the
    // MMA's K-major canonical layout; record word 31 = the blob's offset
    const bool resident = md.wtiles != nullptr && D <= 128 &&
                          sample_tcg_smem_bytes(D, H[0], H[1], tcw1, tcw2, twmax) <= 227 * 1024;
    std::vector<int> wsrc;
    int wbmax = 0;
    if (!resident) {
      const int Dpg = (D + 15) & ~15;
      const long long o0 = md.layer[0].dst_off, o1 = md.layer[1].dst_off, o2 = md.layer[2].dst_off;
      auto kmaj = [](int r, int c, int kw) {
        return (size_t)(r >> 3) * (size_t)(kw / 8) * 64 + (size_t)(c >> 3) * 64 + (size_t)(r & 7) * 8 + (size_t)(c & 7);
      };
      const int ng = (int)grp.size() / TNVAN_TCGG_INTS;
      for (int g = 0; g < ng; ++g) {
        int* Gr = grp.data() + (size_t)g * TNVAN_TCGG_INTS;
        const int gi0 = Gr[0], u1lo = Gr[2], u1hi = Gr[3], u2lo = Gr[4], u2hi = Gr[5];
        // the fold windows as the kernel forms them
        const int w1 = u1lo & ~15, n1 = ((u1hi + 15) & ~15) - w1;
        const int w2 = u2lo & ~15, n2 = ((u2hi + 15) & ~15) - w2;
        const int kS = (gi0 + 15) & ~15;
        const size_t base = wsrc.size();
        Gr[31] = (int)base;
        const size_t nA = (size_t)H[1] * n1, nB = (size_t)Dpg * n2, nC = (size_t)n1 * kS;
        wsrc.resize(base + nA + nB + nC, -1);
        for (int v = 0; v < H[1]; ++v)
          for (int c = 0; c < n1; ++c)
            if (w1 + c < H[0]) wsrc[base + kmaj(v, c, n1)] = (int)(o1 + (long long)v * H[0] + w1 + c);
        for (int i = 0; i < D; ++i)
          for (int c = 0; c < n2; ++c)
            if (w2 + c < H[1]) wsrc[base + nA + kmaj(i, c, n2)] = (int)(o2 + (long long)i * H[1] + w2 + c);
        for (int r = 0; r < n1; ++r)
          for (int kk = 0; kk < kS && kk < D; ++kk)
            if (w1 + r < H[0]) wsrc[base + nA + nB + kmaj(r, kk, kS)] = (int)(o0 + (long long)(w1 + r) * D + kk);
        wbmax = std::max(wbmax, (int)(2 * (nA + nB + nC)));
      }
    }
    int* dgrp = nullptr;
    if ((rc = upload(ctx, in, grp, &dgrp))) return rc;
    int* dsrc = nullptr;
    if ((rc = upload(ctx, in, src, &dsrc))) return rc;
    void* blk = nullptr;
    if (!src.empty()) {
      cudaError_t e2 = cudaMalloc(&blk, src.size() * sizeof(float));
      if (e2 != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(sampler triangles): %s", cudaGetErrorString(e2));
      in.dev_allocs.push_back(blk);
    }
    P.streamed = resident ? 0 : 1;
    P.wbmax = wbmax;
    if (!resident && !wsrc.empty() &&
        (rc = upload_blob(ctx, in, wsrc, &P.wblob, &P.wsrc, &P.wdst, &P.n_wblob)))
      return rc;
    P.n_groups = (int)grp.size() / TNVAN_TCGG_INTS;
    P.groups = dgrp;
    P.blocks = static_cast<float*>(blk);
    P.src = dsrc;
    P.n_blk = (long long)src.size();
    P.twmax = twmax;
    P.tcw1 = tcw1;
    P.tcw2 = tcw2;
    P.ok = fits && (resident || sample_tcg_smem_bytes(D, H[0], H[1], tcw1, tcw2, twmax, wbmax) <= 227 * 1024);
  }
  md.sample_tcg_ok = 0;
  for (int p = 0; p < TNVAN_TC_PLANS; ++p) md.sample_tcg_ok = md.sample_tcg_ok || md.tcg[p].ok;
  md.sample_tc_ok = 0;
  for (int p = 0; p < TNVAN_TC_PLANS; ++p) md.sample_tc_ok = md.sample_tc_ok || md.tc[p].ok;
  // the FP32 copy, then (16-byte aligned) its BF16 twin
  const size_t f32_bytes = ((size_t)off * sizeof(float) + 15) & ~size_t(15);
  void* packed = nullptr;
  cudaError_t e = cudaMalloc(&packed, f32_bytes + (size_t)off * sizeof(uint16_t));
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(packed params): %s", cudaGetErrorString(e));
  in.dev_allocs.push_back(packed);
  md.packed = static_cast<float*>(packed);
  md.packed16 = reinterpret_cast<uint16_t*>(static_cast<char*>(packed) + f32_bytes);
  in.dev.made = md;
  in.nh = n_hidden;
  in.H[0] = H[0];
  in.H[1] = H[1];
  in.d_params = d_params;
  in.n_params = off;
  in.has_made = true;
  ctx->dirty = true;
  ctx->adj_plan.valid = 0;
  return TNVAN_OK;
}

int tnvan_n_params(const tnvan_ctx* ctx, int instance, int64_t* n_params, int64_t* offset) {
  if (!ctx || instance < 0 || instance >= (int)ctx->inst.size()) return TNVAN_E_ARG;
  long long off = 0;
  for (int k = 0; k < instance; ++k) off += ctx->inst[k].n_params;
  if (n_params) *n_params = ctx->inst[instance].n_params;
  if (offset) *offset = off;
  return TNVAN_OK;
}

int tnvan_instance_info(const tnvan_ctx* ctx, int instance, int32_t* info) {
  if (!ctx || !info || instance < 0 || instance >= (int)ctx->inst.size()) return TNVAN_E_ARG;
  const Instance& in = ctx->inst[instance];
  info[0] = in.n;
  info[1] = in.m;
  info[2] = (int)in.W.size();
  info[3] = in.kind;
  info[4] = in.n_comp;
  info[5] = in.max_comp;
  info[6] = in.max_width;
  info[7] = (int)in.ww.size();
  info[8] = in.kind == 2 ? in.g_max_entries : 0;
  info[9] = in.kind == 2 ? in.g_max_live : 0;
  const MadeDev& md = in.dev.made;
  info[10] = md.sample_tcg_ok ? md.tcg[TNVAN_TC_PLANS - 1].slot_u : -1;
  info[11] = md.fused_ok ? 1 : 0;
  info[12] = md.sample_tcg_ok ? md.tcg[TNVAN_TC_PLANS - 1].streamed : -1;
  return TNVAN_OK;
}

static int ensure_dj_part(tnvan_ctx* ctx, size_t floats) {
  if (floats <= ctx->dj_part_floats) return TNVAN_OK;
  if (ctx->d_dj_part) cudaFree(ctx->d_dj_part);
  ctx->d_dj_part = nullptr;
  ctx->dj_part_floats = 0;
  cudaError_t e = cudaMalloc(&ctx->d_dj_part, floats * sizeof(float));
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(d/dJ partials): %s", cudaGetErrorString(e));
  ctx->dj_part_floats = floats;
  return TNVAN_OK;
}

// Elimination launch shape: GL lanes share a sample and a CTA has 128
// threads, so 128 / GL samples.  GL is the largest power of two not above the
// instances' mean table size, doubled once when the batch alone would give
// fewer than 2^17 threads, at most `cap` (measured on random regular graphs,
// n = 1000: the forward pass gains up to 16 lanes, the reverse sweep up to
// 8).  The tables stay in shared memory when a CTA needs at most 100 KB of it
// (two CTAs per SM), else they go to a global scratch slice per CTA.
// smem(S, global) gives a launch's shared bytes.
extern "C++" {
int gen_lanes(const tnvan_ctx* ctx, int batch, int cap) {
  double mean = 1;
  for (const Instance& in : ctx->inst)
    if (in.kind == 2) mean = std::max(mean, in.g_mean_entries);
  int gl = 1;
  while (2 * gl <= cap && 2 * gl <= mean) gl *= 2;
  if ((long long)batch * gl < (1 << 17) && 2 * gl <= cap) gl *= 2;
  return gl;
}

template <class F>
bool gen_tables_global(int S, F smem) {
  return smem(S, false) > 100 * 1024;
}
}  // extern "C++"

// Global table scratch of the elimination kernels (which: 0 forward, 1
// reverse sweep); grows only, kept for the context's lifetime.
static int ensure_gen_scratch(tnvan_ctx* ctx, int which, size_t floats) {
  if (floats <= ctx->gen_scratch_floats[which]) return TNVAN_OK;
  if (ctx->d_gen_scratch[which]) cudaFree(ctx->d_gen_scratch[which]);
  ctx->d_gen_scratch[which] = nullptr;
  ctx->gen_scratch_floats[which] = 0;
  cudaError_t e = cudaMalloc(&ctx->d_gen_scratch[which], floats * sizeof(float));
  if (e != cudaSuccess)
    return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(elimination tables, %zu floats): %s", floats, cudaGetErrorString(e));
  ctx->gen_scratch_floats[which] = floats;
  return TNVAN_OK;
}

// Per-strip results of the wide-strip kernels [n_inst][batch][strips]; grows only.
static int ensure_wide_part(tnvan_ctx* ctx, size_t n) {
  if (n <= ctx->wide_part_n) return TNVAN_OK;
  if (ctx->d_wide_part) cudaFree(ctx->d_wide_part);
  ctx->d_wide_part = nullptr;
  ctx->wide_part_n = 0;
  cudaError_t e = cudaMalloc(&ctx->d_wide_part, n * sizeof(double));
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(wide strips, %zu): %s", n, cudaGetErrorString(e));
  ctx->wide_part_n = n;
  return TNVAN_OK;
}

static int wide_max_strips(const tnvan_ctx* ctx) {
  int ms = 0;
  for (const Instance& in : ctx->inst)
    if (in.kind == 2) ms = std::max(ms, in.dev.n_wide);
  return ms;
}

static int ensure_grad_ws(tnvan_ctx* ctx, size_t floats) {
  if (floats <= ctx->grad_packed_floats) return TNVAN_OK;
  if (ctx->d_grad_packed) cudaFree(ctx->d_grad_packed);
  ctx->d_grad_packed = nullptr;
  ctx->grad_packed_floats = 0;
  cudaError_t e = cudaMalloc(&ctx->d_grad_packed, floats * sizeof(float));
  if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(gradient partials, %zu floats): %s", floats, cudaGetErrorString(e));
  ctx->grad_packed_floats = floats;
  return TNVAN_OK;
}

// Backward chunking: about two CTAs per SM over all instances.
static int backward_chunk(const tnvan_ctx* ctx, int batch) {
  const int n = (int)ctx->inst.size();
  int per = std::max(1, 304 / std::max(n, 1));
  int chunk = (batch + per - 1) / per;
  chunk = ((chunk + 31) / 32) * 32;
  return std::max(chunk, 32);
}

static size_t grad_ws_floats(const tnvan_ctx* ctx, int batch) {
  const int chunk = backward_chunk(ctx, batch);
  const int parts = (batch + chunk - 1) / chunk;
  long long maxp = 0;
  for (const Instance& in : ctx->inst) maxp = std::max(maxp, in.n_params);
  return (size_t)parts * ctx->inst.size() * (size_t)maxp;
}

int tnvan_reserve(tnvan_ctx* ctx, int max_batch) {
  if (!ctx || max_batch < 0) return TNVAN_E_ARG;
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  rc = ensure_grad_ws(ctx, grad_ws_floats(ctx, std::max(max_batch, 1)));
  if (rc) return rc;
  {
    long long maxp = 0;
    for (const Instance& in : ctx->inst) maxp = std::max(maxp, in.n_params);
    const int splits = std::max(1, std::min(TC_SPLITS, (std::max(max_batch, 1) + 127) / 128));
    rc = ensure_grad_ws(ctx, std::max(grad_ws_floats(ctx, std::max(max_batch, 1)),
                                      (size_t)splits * ctx->inst.size() * (size_t)maxp));
    if (rc) return rc;
    rc = ensure_ws(ctx, tc_ws_floats(ctx, std::max(max_batch, 1)) * sizeof(float));
    if (rc) return rc;
    int max_edges = 0, ctas = 0;
    for (const Instance& in : ctx->inst) {
      max_edges = std::max(max_edges, in.m);
      ctas += (std::max(max_batch, 1) + 127) / 128;
    }
    rc = ensure_dj_part(ctx, (size_t)ctas * ((max_edges + 3) & ~3));
    if (rc) return rc;
    const int ms = wide_max_strips(ctx);
    if (ms > 0 && (rc = ensure_wide_part(ctx, ctx->inst.size() * (size_t)std::max(max_batch, 1) * ms))) return rc;
  }
  ctx->reserved_batch = std::max(ctx->reserved_batch, max_batch);
  CK(cudaDeviceSynchronize(), "reserve");
  return TNVAN_OK;
}

int tnvan_sample_and_contract(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed,
                              uint64_t step, int precision, int8_t* d_spins, float* d_logq,
                              double* d_logZR, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 0) return fail(ctx, TNVAN_E_ARG, "batch < 0");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (batch > 0 && (!d_spins || !d_logq || !d_logZR)) return fail(ctx, TNVAN_E_ARG, "NULL output");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (batch == 0) return TNVAN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = pack_network(ctx, sampler_pack_mask(ctx, precision), s))) return rc;
  if ((rc = run_sampler(ctx, betas, batch, seed, step, precision, d_spins, d_logq, nullptr, s))) return rc;
  return contract_all(ctx, betas, batch, d_spins, precision, d_logZR, nullptr, s);
}

// Side streams and events of the overlapped schedule (created once).
static int ensure_side_streams(tnvan_ctx* ctx) {
  if (ctx->side[0]) return TNVAN_OK;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  for (cudaStream_t& st : ctx->side)
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi);
  for (cudaStream_t& st : ctx->side_lo)
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->dj_ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : ctx->join_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : ctx->chunk_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : ctx->adj_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "side streams");
  return TNVAN_OK;
}

// Sampling and the strip adjoint as an overlapped schedule: the instances are
// cut into up to 8 chunks, each with its own side stream on which the chunk
// is sampled and then contracted (adjoint pass).  All samplers start at once
// (the same CTAs as one launch); the adjoint of a chunk starts as soon as its
// samples exist and shares the SMs with the samplers still running (a
// sampler CTA and an adjoint CTA fit on one SM together), filling the
// sampler's tail.  The caller's stream forks to the side streams and joins
// them again, so stream order (and CUDA graph capture) behave as for one
// launch.
// With defer_dj the d/dJ reduction runs on a side stream (beside whatever the
// caller queues next) and the caller waits on ctx->dj_ev before it is done;
// with chunk_stats each chunk's Eq. 9 reduction (F_q, F_IS, stderr, log Z_IS
// and the baseline of tnvan_backward) follows its adjoint on the chunk's
// stream.
// With cb (implies chunk_stats) each chunk's fused backward and gradient
// reduction with Adam follow too, so a chunk's whole training step runs as
// soon as its samples exist.
static int sample_adjoint_overlapped(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step,
                                     int plan, int8_t* d_spins, float* d_logq, double* d_logZR,
                                     double* d_dbeta, double* d_dJ, cudaStream_t s, bool defer_dj,
                                     bool chunk_stats, const ChunkBackward* cb) {
  int rc;
  int adj_tile = 0, adj_smem = 0, adj_lv = 0, adj_ws = 0;
  if ((rc = plan_strip_adjoint(ctx, batch, &adj_tile, &adj_smem, &adj_lv, &adj_ws))) return rc;
  LaunchInfo li, la;
  if ((rc = fill_launch(ctx, betas, batch, 128, li))) return rc;
  li.seed = seed;
  li.step = step;
  if ((rc = fill_launch(ctx, betas, batch, adj_tile, la))) return rc;
  const bool grouped = tc_grouped_usable(ctx);
  const int smem = tc_sampler_smem(ctx, plan, grouped);
  int max_edges = 0;
  for (const Instance& in : ctx->inst) {
    max_edges = std::max(max_edges, in.m);
  }
  const int stride = (max_edges + 3) & ~3;
  if (d_dJ && (rc = ensure_dj_part(ctx, (size_t)la.tile_begin[la.n_inst] * stride))) return rc;
  if ((rc = ensure_side_streams(ctx))) return rc;
  LaunchInfo lr;
  if (chunk_stats && (rc = fill_launch(ctx, betas, batch, 1, lr))) return rc;
  const int n = li.n_inst, nc = std::min(n, 8);
  CK(cudaEventRecord(ctx->fork_ev, s), "fork");
  for (int c = 0; c < nc; ++c) CK(cudaStreamWaitEvent(ctx->side[c], ctx->fork_ev, 0), "fork wait");
  for (int c = 0; c < nc; ++c) {  // samplers on high-priority streams, adjoints behind them
    const int k0 = c * n / nc, k1 = (c + 1) * n / nc;
    {
      PROF("sample_tc", ctx->side[c]);
      if (grouped)
        CK(launch_sample_tcg(ctx->d_inst, li, tcg_order(ctx, li, k0, k1), plan, smem, tc_any_streamed(ctx, plan),
                             d_spins, d_logq, nullptr, ctx->side[c], li.tile_begin[k0],
                             li.tile_begin[k1]),
           "tensor-core sample kernel");
      else
        CK(launch_sample_tc(ctx->d_inst, li, plan, ctx->inst[0].dev.made.nh, smem, d_spins, d_logq, nullptr,
                            ctx->side[c], li.tile_begin[k0], li.tile_begin[k1]),
           "tensor-core sample kernel");
    }
    CK(cudaEventRecord(ctx->chunk_ev[c], ctx->side[c]), "chunk event");
    // the chunk's strip tables need no samples: built while its sampler runs
    CK(cudaStreamWaitEvent(ctx->side_lo[c], ctx->fork_ev, 0), "fork wait");
    CK(launch_strip_tables(ctx->d_inst, la, k0, k1, ctx->side_lo[c]), "strip tables");
    CK(cudaStreamWaitEvent(ctx->side_lo[c], ctx->chunk_ev[c], 0), "chunk wait");
    {
      PROF("strips_adj", ctx->side_lo[c]);
      CK(launch_strips_adj(ctx->d_inst, la, adj_smem, adj_lv, d_spins, d_logZR, d_dbeta,
                           d_dJ ? ctx->d_dj_part : nullptr, stride, nullptr, ctx->side_lo[c], la.tile_begin[k0],
                           la.tile_begin[k1], adj_ws),
         "strip adjoint kernel");
    }
    CK(cudaEventRecord(ctx->adj_ev[c], ctx->side_lo[c]), "adjoint event");
    if (chunk_stats || cb) {
      PROF("reduce", ctx->side_lo[c]);
      CK(launch_reduce(ctx->d_inst, lr, d_logZR, d_logq, ctx->d_stats, ctx->d_status + 4, ctx->side_lo[c], k0, k1),
         "reduce kernel");
    }
    if (cb) {
      const FusedBwdPlan& fp = *cb->plan;
      {
        PROF("bwd_fused", ctx->side_lo[c]);
        CK(launch_bwd_fused(ctx->d_inst, fp.lf, fp.smem, d_spins, d_logZR, d_logq, ctx->d_stats, ctx->d_grad_packed,
                            fp.max_elems, ctx->d_status, ctx->side_lo[c], fp.lf.tile_begin[k0], fp.lf.tile_begin[k1]),
           "fused backward kernel");
      }
      PROF("grad_reduce", ctx->side_lo[c]);
      CK(launch_grad_reduce(ctx->d_inst, fp.lf, ctx->d_grad_packed, (int)fp.max_elems, cb->d_grad, ctx->side_lo[c],
                            cb->adam, k0, k1),
         "gradient reduce kernel");
    }
  }
  for (int c = 0; c < nc; ++c) {
    CK(cudaEventRecord(ctx->join_ev[c], ctx->side_lo[c]), "join");
    CK(cudaStreamWaitEvent(s, ctx->join_ev[c], 0), "join wait");
  }
  if (d_dJ) {  // every edge's sum overwrites d_dJ: no clearing pass
    cudaStream_t sr = s;
    if (defer_dj) {  // after every chunk's adjoint, beside what follows them
      sr = ctx->side[0];
      for (int c = 0; c < nc; ++c) CK(cudaStreamWaitEvent(sr, ctx->adj_ev[c], 0), "adjoint wait");
    }
    {
      PROF("strips_dJ_reduce", sr);
      CK(launch_strips_dJ_reduce(ctx->d_inst, la, ctx->d_dj_part, stride, d_dJ, sr, true), "d/dJ reduce");
    }
    if (defer_dj) CK(cudaEventRecord(ctx->dj_ev, sr), "d/dJ event");
  }
  return TNVAN_OK;
}

int tnvan_sample_contract_adjoint(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed,
                                  uint64_t step, int precision, int8_t* d_spins, float* d_logq,
                                  double* d_logZR, double* d_dbeta, double* d_dJ, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (!d_dbeta && !d_dJ)
    return tnvan_sample_and_contract(ctx, betas, batch, seed, step, precision, d_spins, d_logq, d_logZR, stream);
  if (batch < 0) return fail(ctx, TNVAN_E_ARG, "batch < 0");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (batch > 0 && (!d_spins || !d_logq || !d_logZR)) return fail(ctx, TNVAN_E_ARG, "NULL output");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (batch == 0) return TNVAN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = pack_network(ctx, sampler_pack_mask(ctx, precision), s))) return rc;
  return sample_contract_adjoint_impl(ctx, betas, batch, seed, step, precision, d_spins, d_logq, d_logZR, d_dbeta,
                                      d_dJ, s);
}

int tnvan_train_step(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step, int precision,
                     int8_t* d_spins, float* d_logq, double* d_logZR, double* d_dbeta, double* d_dJ,
                     float* d_grad_params, float* d_m, float* d_v, double lr, double beta1, double beta2,
                     double eps, int64_t t, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (!d_spins || !d_logq || !d_logZR || !d_grad_params || !d_m || !d_v)
    return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  if (t < 1 || !(beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps >= 0))
    return fail(ctx, TNVAN_E_ARG, "bad Adam arguments");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // one pack serves the sampler and the backward (the parameters change only
  // in the last kernel of the step)
  bool all_fused = precision == TNVAN_BF16, any_fused = false;
  for (const Instance& in : ctx->inst) {
    all_fused = all_fused && in.dev.made.fused_ok;
    any_fused = any_fused || in.dev.made.fused_ok;
  }
  any_fused = any_fused && precision == TNVAN_BF16;  // the fused backward reads the BF16 tiles
  if ((rc = pack_network(ctx, sampler_pack_mask(ctx, precision) | PACK_FLAT | (any_fused ? PACK_TILES : 0), s)))
    return rc;
  // the overlapped schedule runs each chunk's Eq. 9 reduction (statistics
  // and the backward's baseline) behind its adjoint, and the d/dJ reduction (it reads only the adjoint's partial
  // rows) beside the backward; the step ends after both.
  // With the fused BF16 backward the chunks' backward and Adam follow their
  // reductions too.
  bool dj_deferred = false, stats_done = false, bwd_done = false;
  const AdamArgs a = adam_args(ctx, d_m, d_v, lr, beta1, beta2, eps, t);
  FusedBwdPlan fp;
  ChunkBackward cb{&fp, d_grad_params, &a};
  if (all_fused && (rc = plan_fused_bwd(ctx, betas, batch, fp))) return rc;
  if (d_dbeta || d_dJ)
    rc = sample_contract_adjoint_impl(ctx, betas, batch, seed, step, precision, d_spins, d_logq, d_logZR, d_dbeta,
                                      d_dJ, s, &dj_deferred, &stats_done, all_fused ? &cb : nullptr, &bwd_done);
  else if (!(rc = run_sampler(ctx, betas, batch, seed, step, precision, d_spins, d_logq, nullptr, s)))
    rc = contract_all(ctx, betas, batch, d_spins, precision, d_logZR, nullptr, s);
  if (rc) return rc;
  if (!bwd_done)
    rc = backward_impl(ctx, betas, batch, d_spins, d_logZR, d_logq, precision, d_grad_params, nullptr, nullptr, s,
                       false, &a, stats_done);
  if (dj_deferred) CK(cudaStreamWaitEvent(s, ctx->dj_ev, 0), "d/dJ join");
  return rc;
}

}  // extern "C"

namespace {

// Sampling, then the contraction with its adjoint (overlapped on side
// streams where every instance is a strip instance and the tensor-core
// sampler runs), on a network the caller has packed.
int sample_contract_adjoint_impl(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step,
                                 int precision, int8_t* d_spins, float* d_logq, double* d_logZR, double* d_dbeta,
                                 double* d_dJ, cudaStream_t s, bool* dj_deferred, bool* stats_done,
                                 const ChunkBackward* cb, bool* bwd_done) {
  int rc;
  if (dj_deferred) *dj_deferred = false;
  if (stats_done) *stats_done = false;
  if (bwd_done) *bwd_done = false;
  bool strips_only = ctx->inst.size() >= 2;
  for (const Instance& in : ctx->inst) strips_only = strips_only && in.kind == 0;
  bool tc_all = precision == TNVAN_BF16;
  tc_all = tc_all && tc_sampler_usable(ctx);
  const int plan = tc_all ? pick_tc_plan(ctx) : -1;
  if (strips_only && plan >= 0 && ctx->tune_overlap) {
    const bool defer = dj_deferred && d_dJ;
    if ((rc = sample_adjoint_overlapped(ctx, betas, batch, seed, step, plan, d_spins, d_logq, d_logZR, d_dbeta, d_dJ,
                                        s, defer, stats_done != nullptr, cb)))
      return rc;
    if (defer) *dj_deferred = true;
    if (stats_done) *stats_done = true;
    if (bwd_done) *bwd_done = cb != nullptr;
    return TNVAN_OK;
  }
  if ((rc = run_sampler(ctx, betas, batch, seed, step, precision, d_spins, d_logq, nullptr, s))) return rc;
  return run_adjoint(ctx, betas, batch, d_spins, precision, d_logZR, d_dbeta, d_dJ, s);
}

}  // namespace

extern "C" {

int tnvan_log_prob(tnvan_ctx* ctx, int batch, const int8_t* d_spins, int precision, float* d_logq,
                   void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (batch < 0) return fail(ctx, TNVAN_E_ARG, "batch < 0");
  if (batch > 0 && (!d_spins || !d_logq)) return fail(ctx, TNVAN_E_ARG, "NULL spins or output");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (batch == 0) return TNVAN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = pack_network(ctx, sampler_pack_mask(ctx, precision), s))) return rc;
  std::vector<double> ones(ctx->inst.size(), 1.0);
  return run_sampler(ctx, ones.data(), batch, 0, 0, precision, nullptr, d_logq, d_spins, s);
}

int tnvan_contract(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                   int precision, double* d_logZR, double* d_dbeta, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 0) return fail(ctx, TNVAN_E_ARG, "batch < 0");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (batch > 0 && (!d_spins || !d_logZR)) return fail(ctx, TNVAN_E_ARG, "NULL spins or output");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  if (batch == 0) return TNVAN_OK;
  return contract_all(ctx, betas, batch, d_spins, precision, d_logZR, d_dbeta,
                      static_cast<cudaStream_t>(stream));
}

int tnvan_free_energy(tnvan_ctx* ctx, const double* betas, int batch, const double* d_logZR,
                      const float* d_logq, double* h_out, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (!d_logZR || !d_logq || !h_out) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    PROF("reduce", s);
    CK(launch_reduce(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats_fe, ctx->d_status + 4 + TNVAN_MAX_INST, s),
       "reduce kernels");
  }
  const int n = li.n_inst;
  std::vector<double> st(8 * n);
  CK(cudaMemcpyAsync(st.data(), ctx->d_stats_fe, st.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
     "stats copy");
  int status[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(status, ctx->d_status, sizeof status, cudaMemcpyDeviceToHost, s), "status copy");
  CK(cudaStreamSynchronize(s), "stream sync");
  if (status[0]) {
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof status, s), "status reset");
    CK(cudaStreamSynchronize(s), "stream sync");
    return fail(ctx, TNVAN_E_TIMEOUT, "a bounded device wait gave up (code %d); results of this batch are invalid", status[0]);
  }
  for (int k = 0; k < n; ++k) {
    if (st[8 * k + 5] > 0)
      return fail(ctx, TNVAN_E_OVERFLOW, "instance %d: %.0f non-finite l_b values", k, st[8 * k + 5]);
    for (int j = 0; j < 4; ++j) h_out[4 * k + j] = st[8 * k + j];
  }
  return TNVAN_OK;
}

int tnvan_reduce(tnvan_ctx* ctx, const double* betas, int batch, const double* d_logZR, const float* d_logq,
                 double* d_stats_out, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (!d_logZR || !d_logq) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    PROF("reduce", s);
    CK(launch_reduce(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats, ctx->d_status + 4, s), "reduce kernel");
  }
  if (d_stats_out)
    CK(cudaMemcpyAsync(d_stats_out, ctx->d_stats, 8 * (size_t)li.n_inst * sizeof(double), cudaMemcpyDeviceToDevice,
                       s),
       "statistics copy");
  return TNVAN_OK;
}

int tnvan_step_stats(tnvan_ctx* ctx, double* d_stats_out, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (!d_stats_out) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  if (ctx->inst.empty()) return fail(ctx, TNVAN_E_STATE, "no instances");
  DeviceGuard g(ctx->device);
  CK(cudaMemcpyAsync(d_stats_out, ctx->d_stats, 8 * ctx->inst.size() * sizeof(double), cudaMemcpyDeviceToDevice,
                     static_cast<cudaStream_t>(stream)),
     "statistics copy");
  return TNVAN_OK;
}

int tnvan_merge_stats(tnvan_ctx* ctx, const double* betas, int n_parts, const double* d_parts, double* d_stats_out,
                      void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (n_parts < 1) return fail(ctx, TNVAN_E_ARG, "n_parts must be >= 1");
  if (!d_parts) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, 1, 1, li))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    PROF("merge_stats", s);
    CK(launch_merge_stats(li, n_parts, d_parts, ctx->d_stats, s), "merge kernel");
  }
  if (d_stats_out)
    CK(cudaMemcpyAsync(d_stats_out, ctx->d_stats, 8 * (size_t)li.n_inst * sizeof(double), cudaMemcpyDeviceToDevice,
                       s),
       "statistics copy");
  return TNVAN_OK;
}

int tnvan_backward_stats(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                         const double* d_logZR, const float* d_logq, int precision, float* d_grad_params,
                         void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (!d_spins || !d_logZR || !d_logq || !d_grad_params) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  return backward_impl(ctx, betas, batch, d_spins, d_logZR, d_logq, precision, d_grad_params, nullptr, nullptr,
                       static_cast<cudaStream_t>(stream), true, nullptr, true);
}

int tnvan_observables(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                      const double* d_logZR, const float* d_logq, double* d_corr, double* h_out, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (!d_spins || !d_logZR || !d_logq || !h_out) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  const int n = (int)ctx->inst.size();
  const size_t nb = (size_t)n * batch;
  const size_t bytes = nb * sizeof(double) + nb * sizeof(float) + 3 * (size_t)n * sizeof(double) + 64;
  if (bytes > ctx->obs_bytes) {
    if (ctx->d_obs) cudaFree(ctx->d_obs);
    ctx->d_obs = nullptr;
    ctx->obs_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->d_obs, bytes);
    if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(observables): %s", cudaGetErrorString(e));
    ctx->obs_bytes = bytes;
  }
  double* d_db = static_cast<double*>(ctx->d_obs);
  double* d_sums = d_db + nb;
  float* d_w = reinterpret_cast<float*>(d_sums + 3 * n);
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the importance weights need logZ_IS: the F_q reduction in
  // tnvan_free_energy's own workspace
  CK(launch_reduce(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats_fe, ctx->d_status + 4 + TNVAN_MAX_INST, s),
     "reduce kernels");
  CK(launch_observables(li, d_logZR, d_logq, ctx->d_stats_fe, nullptr, d_w, nullptr, false, s), "weights kernel");
  // per-sample energies (d/dbeta) and the weighted bond sums
  if ((rc = run_adjoint(ctx, betas, batch, d_spins, TNVAN_FP32, nullptr, d_db, d_corr, s, d_w))) return rc;
  CK(launch_observables(li, d_logZR, d_logq, ctx->d_stats_fe, d_db, d_w, d_sums, true, s), "energy kernel");
  std::vector<double> sums(3 * n);
  CK(cudaMemcpyAsync(sums.data(), d_sums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "sums copy");
  CK(cudaStreamSynchronize(s), "stream sync");
  for (int k = 0; k < 3 * n; ++k) h_out[k] = sums[k];
  return TNVAN_OK;
}

int tnvan_magnetisation(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                        const double* d_logZR, const float* d_logq, double* d_mag_mean, double* d_mag_var,
                        double* h_out, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (!d_spins || !d_logZR || !d_logq || !h_out) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  const int n = (int)ctx->inst.size();
  const size_t nb = (size_t)n * batch;
  const size_t bytes = 2 * nb * sizeof(double) + 5 * (size_t)n * sizeof(double) + nb * sizeof(float) + 64;
  if (bytes > ctx->obs_bytes) {
    if (ctx->d_obs) cudaFree(ctx->d_obs);
    ctx->d_obs = nullptr;
    ctx->obs_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->d_obs, bytes);
    if (e != cudaSuccess) return fail(ctx, TNVAN_E_NOMEM, "cudaMalloc(observables): %s", cudaGetErrorString(e));
    ctx->obs_bytes = bytes;
  }
  double* mean = d_mag_mean ? d_mag_mean : static_cast<double*>(ctx->d_obs);
  double* var = d_mag_var ? d_mag_var : static_cast<double*>(ctx->d_obs) + nb;
  double* d_sums = static_cast<double*>(ctx->d_obs) + 2 * nb;
  float* d_w = reinterpret_cast<float*>(d_sums + 5 * n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  // importance weights (logZ_IS from the F_q reduction, in tnvan_free_energy's workspace)
  CK(launch_reduce(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats_fe, ctx->d_status + 4 + TNVAN_MAX_INST, s),
     "reduce kernels");
  CK(launch_observables(li, d_logZR, d_logq, ctx->d_stats_fe, nullptr, d_w, nullptr, false, s), "weights kernel");
  // per-sample moments, by contraction kind
  bool k0 = false, k1 = false, k2 = false;
  int max_D = 0, arena = 0, nsteps = 0;
  int strip_sm = 0;
  for (const Instance& in : ctx->inst) {
    max_D = std::max(max_D, (int)in.W.size());
    if (in.kind == 0) {
      k0 = true;
      strip_sm = std::max(strip_sm, strip_smem_bytes(in, 128));
    } else if (in.kind == 1) {
      k1 = true;
    } else {
      k2 = true;
      arena = std::max(arena, in.g_max_live);
      nsteps = std::max(nsteps, (int)in.gfstep.size());
    }
  }
  if (k0) {
    if (strip_sm > 227 * 1024) return fail(ctx, TNVAN_E_UNSUPPORTED, "strip tables need %d B of shared memory", strip_sm);
    LaunchInfo ls;
    if ((rc = fill_launch(ctx, betas, batch, 128, ls))) return rc;
    CK(launch_strips_mom(ctx->d_inst, ls, strip_sm, d_spins, mean, var, s), "strip moments kernel");
  }
  if (k1) CK(launch_dense_mom(ctx->d_inst, li, max_D, d_spins, mean, var, s), "dense moments kernel");
  if (k2) {
    const int GL = gen_lanes(ctx, batch, 16), T = 128 / GL;
    const bool glob = gen_tables_global(T, [&](int t, bool gg) { return general_mom_smem_bytes(arena, max_D, t, GL, gg); });
    const int sm = general_mom_smem_bytes(arena, max_D, T, GL, glob);
    if (sm > 227 * 1024) return fail(ctx, TNVAN_E_UNSUPPORTED, "elimination tables need %d B of shared memory", sm);
    LaunchInfo lg;
    if ((rc = fill_launch(ctx, betas, batch, T, lg))) return rc;
    CK(launch_general_pp(ctx->d_inst, lg, nsteps, s), "elimination bond products");
    float* gs = nullptr;
    if (glob) {
      if ((rc = ensure_gen_scratch(ctx, 0, general_mom_scratch_floats(lg, arena, GL)))) return rc;
      gs = ctx->d_gen_scratch[0];
    }
    CK(launch_general_mom(ctx->d_inst, lg, sm, arena, GL, d_spins, mean, var, gs, s), "elimination moments kernel");
  }
  CK(launch_obs_mag(li, mean, var, d_w, d_sums, s), "magnetisation reduction");
  std::vector<double> sums(5 * n);
  CK(cudaMemcpyAsync(sums.data(), d_sums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "sums copy");
  CK(cudaStreamSynchronize(s), "stream sync");
  for (int k = 0; k < n; ++k) {
    const double* a = sums.data() + 5 * k;
    h_out[6 * k + 0] = a[0];
    h_out[6 * k + 1] = a[1];
    h_out[6 * k + 2] = li.beta[k] * (a[1] - a[0] * a[0]) / (double)ctx->inst[k].n;
    h_out[6 * k + 3] = a[2];
    h_out[6 * k + 4] = a[3];
    h_out[6 * k + 5] = a[4];
  }
  return TNVAN_OK;
}

int tnvan_backward(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                   const double* d_logZR, const float* d_logq, int precision,
                   float* d_grad_params, double* d_dbeta, double* d_dJ, void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (batch < 1) return fail(ctx, TNVAN_E_ARG, "batch must be >= 1");
  if (precision < 0 || precision > 2) return fail(ctx, TNVAN_E_ARG, "unknown precision %d", precision);
  if (!d_spins || !d_logZR || !d_logq || !d_grad_params) return fail(ctx, TNVAN_E_ARG, "NULL pointer");
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  return backward_impl(ctx, betas, batch, d_spins, d_logZR, d_logq, precision, d_grad_params, d_dbeta, d_dJ,
                       static_cast<cudaStream_t>(stream), true, nullptr);
}

}  // extern "C"

namespace {

// Eq. 10 and (optionally) the contraction adjoint, after argument checks:
// with `pack` false the caller has packed the network for this call; with
// `adam` the gradient reduction also takes Adam's step on every instance's
// parameters.
int backward_impl(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins, const double* d_logZR,
                  const float* d_logq, int precision, float* d_grad_params, double* d_dbeta, double* d_dJ,
                  cudaStream_t s, bool pack, const AdamArgs* adam, bool stats_ready) {
  int rc;
  long long max_elems = 0;
  for (const Instance& in : ctx->inst) max_elems = std::max(max_elems, in.n_params);
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  bool all_fused = precision == TNVAN_BF16, any_fused = false;
  for (const Instance& in : ctx->inst) {
    all_fused = all_fused && in.dev.made.fused_ok;
    any_fused = any_fused || in.dev.made.fused_ok;
  }
  any_fused = any_fused && precision == TNVAN_BF16;
  if (pack && (rc = pack_network(ctx, PACK_FLAT | (any_fused ? PACK_TILES : 0), s))) return rc;
  if (!stats_ready) {
    PROF("reduce", s);
    CK(launch_reduce(ctx->d_inst, li, d_logZR, d_logq, ctx->d_stats, ctx->d_status + 4, s), "reduce kernel");
  }
  // instances the fused kernel takes (BF16): fused; the rest by the forms below
  unsigned int fused_bits[TNVAN_MAX_INST / 32] = {0u};
  for (int k = 0; k < (int)ctx->inst.size() && any_fused; ++k)
    if (ctx->inst[k].dev.made.fused_ok) fused_bits[k >> 5] |= 1u << (k & 31);
  if (any_fused) {
    FusedBwdPlan fp;
    if ((rc = plan_fused_bwd(ctx, betas, batch, fp))) return rc;
    {
      PROF("bwd_fused", s);
      CK(launch_bwd_fused(ctx->d_inst, fp.lf, fp.smem, d_spins, d_logZR, d_logq, ctx->d_stats, ctx->d_grad_packed,
                          fp.max_elems, ctx->d_status, s),
         "fused backward kernel");
    }
    {
      PROF("grad_reduce", s);
      CK(launch_grad_reduce(ctx->d_inst, fp.lf, ctx->d_grad_packed, (int)fp.max_elems, d_grad_params, s, adam),
         "gradient reduce kernel");
    }
  }
  // without the fused kernel, the reduced-precision modes take the tensor-core
  // GEMM chain or (tuned, where faster) the FP32 SIMT backward
  const bool simt = precision == TNVAN_FP32 || (!all_fused && ctx->tune_bwd_form == 2);
  if (!all_fused && !simt) {
    const int splits = std::max(1, std::min(TC_SPLITS, (batch + 127) / 128));
    if ((rc = ensure_grad_ws(ctx, (size_t)splits * ctx->inst.size() * (size_t)max_elems))) return rc;
    if ((rc = backward_tc(ctx, betas, batch, d_spins, d_logZR, d_logq, precision == TNVAN_BF16,
                          (int)max_elems, s, any_fused)))
      return rc;
    LaunchInfo lr;
    if ((rc = fill_launch(ctx, betas, batch, 1, lr))) return rc;
    for (int k = 0; k <= lr.n_inst; ++k) lr.tile_begin[k] = k * splits;
    for (int j = 0; j < TNVAN_MAX_INST / 32; ++j) lr.skip[j] = fused_bits[j];
    {
      PROF("grad_reduce", s);
      CK(launch_grad_reduce(ctx->d_inst, lr, ctx->d_grad_packed, (int)max_elems, d_grad_params, s, adam),
         "gradient reduce kernel");
    }
  }
  const int chunk = backward_chunk(ctx, batch);
  LaunchInfo lb;
  if ((rc = fill_launch(ctx, betas, batch, chunk, lb))) return rc;
  if (any_fused) {  // the SIMT backward leaves the fused instances out (no CTAs, not reduced)
    int acc = 0;
    for (int k = 0; k < lb.n_inst; ++k) {
      lb.tile_begin[k] = acc;
      if (!((fused_bits[k >> 5] >> (k & 31)) & 1u)) acc += (batch + chunk - 1) / chunk;
    }
    lb.tile_begin[lb.n_inst] = acc;
    for (int j = 0; j < TNVAN_MAX_INST / 32; ++j) lb.skip[j] = fused_bits[j];
  }
  if (simt && (rc = ensure_grad_ws(ctx, grad_ws_floats(ctx, batch)))) return rc;
  int smem = 0;
  for (const Instance& in : ctx->inst)
    smem = std::max(smem, (int)((2 * in.W.size() + 2 * in.H[0] + 2 * in.H[1]) * 33 * sizeof(float)));
  if (simt) {
    {
      PROF("backward", s);
      CK(launch_backward(ctx->d_inst, lb, smem, precision, d_spins, d_logZR, d_logq, ctx->d_stats,
                         ctx->d_grad_packed, (int)max_elems, s),
         "backward kernel");
    }
    {
      PROF("grad_reduce", s);
      CK(launch_grad_reduce(ctx->d_inst, lb, ctx->d_grad_packed, (int)max_elems, d_grad_params, s, adam),
         "gradient reduce kernel");
    }
  }
  if (d_dbeta || d_dJ) return run_adjoint(ctx, betas, batch, d_spins, precision, nullptr, d_dbeta, d_dJ, s);
  return TNVAN_OK;
}

int plan_fused_bwd(tnvan_ctx* ctx, const double* betas, int batch, FusedBwdPlan& p) {
  int rc;
  p.max_elems = 0;
  p.smem = 0;
  for (const Instance& in : ctx->inst) {
    // rows of a multiple of 4 floats: the flush writes 16-byte vectors
    p.max_elems = std::max(p.max_elems, (in.n_params + 3) & ~3LL);
    if (in.dev.made.fused_ok)
      p.smem = std::max(p.smem, fused_bwd_smem_bytes((int)in.W.size(), in.H[0], in.H[1]));
  }
  const int n_inst = (int)ctx->inst.size();
  const int tiles = (batch + 127) / 128;
  const int ctas = std::max(1, std::min(tiles, ctx->tune_bwd_ctas ? ctx->tune_bwd_ctas : (148 + n_inst - 1) / n_inst));
  const int per = (tiles + ctas - 1) / ctas;
  // the last instance (the overlapped schedule's last chunk, whose backward
  // runs on a GPU the other chunks have left) is cut finer: at most 2 tiles
  // per CTA (1 measured slower: more gradient rows to reduce)
  const int per_last = std::min(per, 2);
  if ((rc = fill_launch(ctx, betas, batch, per, p.lf))) return rc;
  int acc = 0;
  for (int k = 0; k < p.lf.n_inst; ++k) {
    p.lf.tile_begin[k] = acc;
    const int pk = (k == n_inst - 1 && n_inst > 1) ? per_last : per;
    if (ctx->inst[k].dev.made.fused_ok) acc += (tiles + pk - 1) / pk;
    else p.lf.skip[k >> 5] |= 1u << (k & 31);  // no CTAs; another backward form reduces it
  }
  p.lf.tile_begin[p.lf.n_inst] = acc;
  p.lf.tile = per;
  return ensure_grad_ws(ctx, (size_t)p.lf.tile_begin[p.lf.n_inst] * (size_t)p.max_elems);
}

AdamArgs adam_args(const tnvan_ctx* ctx, float* d_m, float* d_v, double lr, double beta1, double beta2, double eps,
                   int64_t t) {
  AdamArgs a;
  a.m = d_m;
  a.v = d_v;
  a.lr = (float)lr;
  a.b1 = (float)beta1;
  a.b2 = (float)beta2;
  a.eps = (float)eps;
  a.bc1 = (float)(1.0 - pow(beta1, (double)t));
  a.bc2 = (float)(1.0 - pow(beta2, (double)t));
  a.t_dev = ctx->step_dev;
  a.t_base = (long long)t;
  return a;
}

}  // namespace

extern "C" {

int tnvan_adam(tnvan_ctx* ctx, int64_t n, float* d_params, const float* d_grad, float* d_m,
               float* d_v, double lr, double beta1, double beta2, double eps, int64_t t,
               void* stream) {
  if (!ctx) return TNVAN_E_ARG;
  if (n < 0 || t < 1 || (n > 0 && (!d_params || !d_grad || !d_m || !d_v)))
    return fail(ctx, TNVAN_E_ARG, "bad Adam arguments");
  if (!(beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps >= 0))
    return fail(ctx, TNVAN_E_ARG, "bad Adam hyper-parameters");
  DeviceGuard g(ctx->device);
  const AdamArgs a = adam_args(ctx, d_m, d_v, lr, beta1, beta2, eps, t);
  PROF("adam", static_cast<cudaStream_t>(stream));
  CK(launch_adam(n, d_params, d_grad, a, static_cast<cudaStream_t>(stream)), "adam kernel");
  return TNVAN_OK;
}

int tnvan_autotune(tnvan_ctx* ctx, const double* betas, int batch, int precision, void* stream,
                   int32_t* out) {
  if (!ctx || batch < 1 || !betas) return ctx ? fail(ctx, TNVAN_E_ARG, "bad autotune arguments") : TNVAN_E_ARG;
  DeviceGuard g(ctx->device);
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long spins_n = 0, params_n = 0;
  for (const Instance& in : ctx->inst) {
    spins_n += (long long)batch * (long long)in.W.size();
    params_n += in.n_params;
  }
  const int n = (int)ctx->inst.size();
  int8_t* sp = nullptr;
  float *lq = nullptr, *gr = nullptr;
  double* lz = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (sp) cudaFree(sp);
    if (lq) cudaFree(lq);
    if (gr) cudaFree(gr);
    if (lz) cudaFree(lz);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&sp, spins_n) != cudaSuccess || cudaMalloc(&lq, sizeof(float) * n * batch) != cudaSuccess ||
      cudaMalloc(&lz, sizeof(double) * n * batch) != cudaSuccess ||
      cudaMalloc(&gr, sizeof(float) * params_n) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return fail(ctx, TNVAN_E_NOMEM, "autotune buffers");
  }
  // time fn: one warm-up call, then the mean of three
  auto time_it = [&](auto fn, float* ms) -> int {
    int r = fn();
    if (r) return r;
    cudaEventRecord(e0, s);
    for (int i = 0; i < 3; ++i)
      if ((r = fn())) return r;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return TNVAN_OK;
  };
  auto sample = [&]() { return tnvan_sample_and_contract(ctx, betas, batch, 1, 0, precision, sp, lq, lz, stream); };
  bool tc_sampler = precision == TNVAN_BF16;
  ctx->tune_tc_form = 0;
  tc_sampler = tc_sampler && tc_sampler_usable(ctx);
  if (tc_sampler) {  // every plan of both forms that fits every instance
    int best = -1, best_form = 0;
    float best_ms = 1e30f;
    for (int form = 1; form <= 2; ++form) {
      ctx->tune_tc_form = form;
      if (form == 1 && !tc_grouped_usable(ctx)) continue;
      if (form == 2 && !tc_sampler_usable(ctx)) continue;
      for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
        ctx->tune_tc_plan = p;
        if (pick_tc_plan(ctx) != p) continue;
        float ms = 0.f;
        if ((rc = time_it(sample, &ms))) {
          cleanup();
          return rc;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = p;
          best_form = form;
        }
      }
    }
    ctx->tune_tc_plan = best;
    ctx->tune_tc_form = best >= 0 ? best_form : 0;
  }
  if (!tc_sampler) {
    int best = 0;
    float best_ms = 1e30f;
    for (int T : {16, 32, 64}) {
      if (max_sample_smem(ctx, T) > 227 * 1024) continue;
      ctx->tune_sample_tile = T;
      float ms = 0.f;
      if ((rc = time_it(sample, &ms))) {
        cleanup();
        return rc;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = T;
      }
    }
    ctx->tune_sample_tile = best;
  }
  if ((rc = sample())) {  // spins for the contraction and backward candidates
    cleanup();
    return rc;
  }
  bool any_strip = false;
  for (const Instance& in : ctx->inst) any_strip = any_strip || in.kind == 0;
  if (any_strip) {
    int best = 0;
    float best_ms = 1e30f;
    for (int T : {32, 64, 128}) {
      ctx->tune_strip_tile = T;
      float ms = 0.f;
      auto contract = [&]() { return tnvan_contract(ctx, betas, batch, sp, precision, lz, nullptr, stream); };
      if ((rc = time_it(contract, &ms))) {
        cleanup();
        return rc;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = T;
      }
    }
    ctx->tune_strip_tile = best;
  }
  bool fused = precision == TNVAN_BF16;
  for (const Instance& in : ctx->inst) fused = fused && in.dev.made.fused_ok;
  if (fused) {
    int best = 0;
    float best_ms = 1e30f;
    const int base = (148 + n - 1) / n;
    for (int c : {base / 2, base, 2 * base, 4 * base}) {
      if (c < 1) continue;
      ctx->tune_bwd_ctas = c;
      float ms = 0.f;
      auto bwd = [&]() {
        return tnvan_backward(ctx, betas, batch, sp, lz, lq, precision, gr, nullptr, nullptr, stream);
      };
      if ((rc = time_it(bwd, &ms))) {
        cleanup();
        return rc;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    ctx->tune_bwd_ctas = best;
  }
  if (!fused && precision != TNVAN_FP32) {  // the tensor-core GEMM chain or the FP32 SIMT backward
    int best = 0;
    float best_ms = 1e30f;
    for (int f : {1, 2}) {
      ctx->tune_bwd_form = f;
      float ms = 0.f;
      auto bwd = [&]() {
        return tnvan_backward(ctx, betas, batch, sp, lz, lq, precision, gr, nullptr, nullptr, stream);
      };
      if ((rc = time_it(bwd, &ms))) {
        cleanup();
        return rc;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = f;
      }
    }
    ctx->tune_bwd_form = best;
  }
  if (any_strip) {
    // the strip adjoint's launch shape, and (tensor-core sampler) whether
    // sampling and the adjoint overlap on side streams: timed together on the
    // combined pass a training step runs
    long long ne = 0;
    for (const Instance& in : ctx->inst) ne += in.m;
    double *dj = nullptr, *db = nullptr;
    if (cudaMalloc(&dj, sizeof(double) * std::max(ne, 1LL)) != cudaSuccess ||
        cudaMalloc(&db, sizeof(double) * (size_t)n * batch) != cudaSuccess) {
      if (dj) cudaFree(dj);
      cleanup();
      return fail(ctx, TNVAN_E_NOMEM, "autotune buffers");
    }
    auto pass = [&]() {
      return tnvan_sample_contract_adjoint(ctx, betas, batch, 1, 0, precision, sp, lq, lz, db, dj, stream);
    };
    int best_t = 0, best_o = 1;
    float best_ms = 1e30f;
    for (int ov : {1, 0}) {
      if (ov == 0 && !tc_sampler) continue;
      for (int T : {1, 128, 96, 64, 32}) {
        ctx->tune_adj_tile = T;
        ctx->tune_overlap = ov;
        int t_used = 0, sm = 0, lv = 0, ws = 0;
        if (plan_strip_adjoint(ctx, batch, &t_used, &sm, &lv, &ws) || (ws ? 1 : t_used) != T) continue;
        float ms = 0.f;
        if ((rc = time_it(pass, &ms))) {
          cudaFree(dj);
          cudaFree(db);
          cleanup();
          return rc;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best_t = T;
          best_o = ov;
        }
      }
    }
    ctx->tune_adj_tile = best_t;
    ctx->tune_overlap = best_o;
    if (fused && tc_sampler && best_o) {
      // the overlapped training step runs each chunk's backward behind its
      // adjoint, so the backward's CTA count and the adjoint's shape are
      // re-timed together on whole training steps (learning rate 0 on
      // scratch moments: the networks do not move)
      float *m = nullptr, *v = nullptr;
      if (cudaMalloc(&m, sizeof(float) * params_n) != cudaSuccess ||
          cudaMalloc(&v, sizeof(float) * params_n) != cudaSuccess) {
        if (m) cudaFree(m);
        cudaFree(dj);
        cudaFree(db);
        cleanup();
        return fail(ctx, TNVAN_E_NOMEM, "autotune buffers");
      }
      cudaMemsetAsync(m, 0, sizeof(float) * params_n, s);
      cudaMemsetAsync(v, 0, sizeof(float) * params_n, s);
      cudaStreamSynchronize(s);
      // the step as it is meant to run: captured once in a CUDA graph on a
      // private stream (an eager call first sizes the workspaces), then
      // replayed; the time of one replay
      cudaStream_t sc = nullptr;
      if (cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(m);
        cudaFree(v);
        cudaFree(dj);
        cudaFree(db);
        cleanup();
        return fail(ctx, TNVAN_E_CUDA, "autotune stream");
      }
      auto step_on = [&](cudaStream_t st) {
        return tnvan_train_step(ctx, betas, batch, 1, 0, precision, sp, lq, lz, db, dj, gr, m, v, 0.0, 0.9, 0.999,
                                1.0, 1, st);
      };
      auto graph_time = [&](float* ms) -> int {
        int r = step_on(sc);
        if (r) return r;
        if (cudaStreamSynchronize(sc) != cudaSuccess) return fail(ctx, TNVAN_E_CUDA, "autotune step");
        cudaGraph_t gph = nullptr;
        cudaGraphExec_t ex = nullptr;
        if (cudaStreamBeginCapture(sc, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return fail(ctx, TNVAN_E_CUDA, "autotune capture");
        r = step_on(sc);
        const cudaError_t ec = cudaStreamEndCapture(sc, &gph);
        if (r || ec != cudaSuccess) {
          if (gph) cudaGraphDestroy(gph);
          return r ? r : fail(ctx, TNVAN_E_CUDA, "autotune capture: %s", cudaGetErrorString(ec));
        }
        if (cudaGraphInstantiate(&ex, gph, 0) != cudaSuccess) {
          cudaGraphDestroy(gph);
          return fail(ctx, TNVAN_E_CUDA, "autotune graph");
        }
        cudaGraphLaunch(ex, sc);
        cudaEventRecord(e0, sc);
        for (int i = 0; i < 5; ++i) cudaGraphLaunch(ex, sc);
        cudaEventRecord(e1, sc);
        const cudaError_t es = cudaEventSynchronize(e1);
        float tot = 0.f;
        cudaEventElapsedTime(&tot, e0, e1);
        *ms = tot / 5.f;
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(gph);
        return es == cudaSuccess ? TNVAN_OK : fail(ctx, TNVAN_E_CUDA, "autotune replay: %s", cudaGetErrorString(es));
      };
      const int tiles = (batch + 127) / 128;
      int best_c = ctx->tune_bwd_ctas, best_a = best_t;
      float best_step = 1e30f;
      for (int per : {2, 3, 4, 5, 6}) {
        const int c = (tiles + per - 1) / per;
        if (c < 1 || (per > 2 && c == (tiles + per - 2) / (per - 1))) continue;  // same launch as per - 1
        for (int T : {best_t, 1, 128, 96}) {
          ctx->tune_bwd_ctas = c;
          ctx->tune_adj_tile = T;
          int t_used = 0, sm = 0, lv = 0, ws = 0;
          if (plan_strip_adjoint(ctx, batch, &t_used, &sm, &lv, &ws) || (ws ? 1 : t_used) != T) continue;
          float ms = 0.f;
          if ((rc = graph_time(&ms))) {
            cudaStreamDestroy(sc);
            cudaFree(m);
            cudaFree(v);
            cudaFree(dj);
            cudaFree(db);
            cleanup();
            return rc;
          }
          if (ms < best_step) {
            best_step = ms;
            best_c = c;
            best_a = T;
          }
        }
      }
      cudaStreamSynchronize(sc);
      cudaStreamDestroy(sc);
      cudaFree(m);
      cudaFree(v);
      ctx->tune_bwd_ctas = best_c;
      ctx->tune_adj_tile = best_a;
    }
    cudaStreamSynchronize(s);
    cudaFree(dj);
    cudaFree(db);
  }
  if (out) {
    out[0] = ctx->tune_sample_tile;
    out[1] = ctx->tune_strip_tile;
    out[2] = ctx->tune_bwd_ctas;
    out[3] = ctx->tune_adj_tile;
    out[4] = tc_plan_value(ctx, ctx->tune_tc_plan);
    out[5] = ctx->tune_overlap ? 2 : 1;
    out[6] = ctx->tune_bwd_form;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
  return TNVAN_OK;
}

int tnvan_set_tuning(tnvan_ctx* ctx, const int32_t* c) {
  if (!ctx) return TNVAN_E_ARG;
  if (!c) return fail(ctx, TNVAN_E_ARG, "NULL tuning");
  auto in = [](int v, std::initializer_list<int> ok) {
    if (v == 0) return true;
    for (int o : ok)
      if (v == o) return true;
    return false;
  };
  // the plan value names the form: grouped 4, 6, 8 steps, per-step chunks 12, 16, 32
  int plan = -1, form = 0;
  for (int p = 0; p < TNVAN_TC_PLANS; ++p) {
    if (kTcGroupMaxG[p] == c[4]) plan = p, form = 1;
    if (kTcGroupMax[p] == c[4]) plan = p, form = 2;
  }
  if (!in(c[0], {16, 32, 64}) || !in(c[1], {32, 64, 128}) || c[2] < 0 || !in(c[3], {1, 32, 64, 96, 128}) ||
      (c[4] != 0 && plan < 0) || c[5] < 0 || c[5] > 2 || c[6] < 0 || c[6] > 2)
    return fail(ctx, TNVAN_E_ARG, "tuning value outside the autotuner's candidates");
  ctx->tune_sample_tile = c[0];
  ctx->tune_strip_tile = c[1];
  ctx->tune_bwd_ctas = c[2];
  ctx->tune_adj_tile = c[3];
  ctx->tune_tc_plan = plan;
  ctx->tune_tc_form = form;
  ctx->tune_overlap = c[5] != 1;  // 0 and 2 (default) on, 1 off
  ctx->tune_bwd_form = c[6];
  return TNVAN_OK;
}

int tnvan_set_step_counter(tnvan_ctx* ctx, const uint64_t* d_counter) {
  if (!ctx) return TNVAN_E_ARG;
  ctx->step_dev = reinterpret_cast<const unsigned long long*>(d_counter);
  return TNVAN_OK;
}

int tnvan_profile(tnvan_ctx* ctx, int enable) {
  if (!ctx) return TNVAN_E_ARG;
  DeviceGuard g(ctx->device);
  if (enable) {
    cudaDeviceSynchronize();
    for (auto& r : ctx->prof)
      for (auto& pr : r.pending) {
        ctx->event_pool.push_back(pr.first);
        ctx->event_pool.push_back(pr.second);
      }
    ctx->prof.clear();
    ctx->prof_ref_set = false;
  }
  ctx->prof_on = enable != 0;
  return TNVAN_OK;
}

int tnvan_profile_trace(tnvan_ctx* ctx, int64_t max_entries, int32_t* kernel, float* start_ms, float* end_ms,
                        int64_t* n_out) {
  if (!ctx || !n_out || max_entries < 0) return TNVAN_E_ARG;
  DeviceGuard g(ctx->device);
  int64_t n = 0;
  for (size_t i = 0; i < ctx->prof.size(); ++i)
    for (auto& pr : ctx->prof[i].pending) {
      if (n < max_entries && ctx->prof_ref_set) {
        CK(cudaEventSynchronize(pr.second), "trace event sync");
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, ctx->prof_ref, pr.first), "trace elapsed time");
        CK(cudaEventElapsedTime(&b, ctx->prof_ref, pr.second), "trace elapsed time");
        if (kernel) kernel[n] = (int32_t)i;
        if (start_ms) start_ms[n] = a;
        if (end_ms) end_ms[n] = b;
      }
      ++n;
    }
  *n_out = n;
  return TNVAN_OK;
}

int tnvan_profile_read(tnvan_ctx* ctx, int index, char* name, int name_len, double* total_ms,
                       int64_t* launches) {
  if (!ctx || index < 0 || index >= (int)ctx->prof.size()) return TNVAN_E_ARG;
  DeviceGuard g(ctx->device);
  tnvan_prof_rec& r = ctx->prof[index];
  for (auto& pr : r.pending) {
    CK(cudaEventSynchronize(pr.second), "profile event sync");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second), "profile elapsed time");
    r.total_ms += ms;
    r.launches += 1;
    ctx->event_pool.push_back(pr.first);
    ctx->event_pool.push_back(pr.second);
  }
  r.pending.clear();
  if (name && name_len > 0) {
    strncpy(name, r.name.c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (total_ms) *total_ms = r.total_ms;
  if (launches) *launches = r.launches;
  return TNVAN_OK;
}

}  // extern "C"

namespace {

// Rebuild what the kernels read from the networks (segments in `mask`).
int pack_network(tnvan_ctx* ctx, int mask, cudaStream_t s) {
  std::vector<long long> counts;
  for (const Instance& in : ctx->inst) counts.push_back(pack_elems(in.dev.made, mask));
  PROF("pack", s);
  CK(launch_pack_all(ctx->d_inst, (int)ctx->inst.size(), counts.data(), mask, s), "pack kernel");
  return TNVAN_OK;
}

// Segments the sampler of this precision reads.
int sampler_pack_mask(const tnvan_ctx* ctx, int precision) {
  bool tc_all = precision == TNVAN_BF16;
  tc_all = tc_all && tc_sampler_usable(ctx);
  const int plan = tc_all ? pick_tc_plan(ctx) : -1;
  if (plan >= 0)  // only the plan in use
    return tc_grouped_usable(ctx) ? (PACK_FLAT | PACK_TILES | PACK_TCG | ((plan + 1) << 8))
                                  : (PACK_FLAT | PACK_TC | ((plan + 1) << 8));
  return PACK_FLAT | PACK_SIMT;
}

bool tc_grouped_usable(const tnvan_ctx* ctx) {
  if (ctx->inst.empty() || ctx->tune_tc_form == 2) return false;
  for (const Instance& in : ctx->inst)
    if (!in.dev.made.sample_tcg_ok) return false;
  return true;
}

bool tc_sampler_usable(const tnvan_ctx* ctx) {
  if (ctx->inst.empty()) return false;
  if (tc_grouped_usable(ctx)) return true;
  const int nh = ctx->inst[0].dev.made.nh;
  for (const Instance& in : ctx->inst)
    if (!in.dev.made.sample_tc_ok || in.dev.made.nh != nh) return false;
  return true;
}

// The tuning value of plan p (its step limit) for the sampler form in use.
int tc_plan_value(const tnvan_ctx* ctx, int p) {
  if (p < 0 || p >= TNVAN_TC_PLANS) return 0;
  return tc_grouped_usable(ctx) ? kTcGroupMaxG[p] : kTcGroupMax[p];
}

// The grouped sampler's block order over instances [k0, k1) of a launch:
// widest width set first, ties in instance order.
TcgOrder tcg_order(const tnvan_ctx* ctx, const LaunchInfo& li, int k0, int k1) {
  TcgOrder o;
  o.n = k1 - k0;
  std::vector<int> ks;
  for (int k = k0; k < k1; ++k) ks.push_back(k);
  std::stable_sort(ks.begin(), ks.end(),
                   [&](int a, int b) { return ctx->inst[a].W.size() > ctx->inst[b].W.size(); });
  int acc = li.tile_begin[k0];
  for (int j = 0; j < o.n; ++j) {
    o.inst[j] = ks[j];
    o.begin[j] = acc;
    acc += li.tile_begin[ks[j] + 1] - li.tile_begin[ks[j]];
  }
  o.begin[o.n] = acc;
  return o;
}

bool tc_any_streamed(const tnvan_ctx* ctx, int plan) {
  for (const Instance& in : ctx->inst)
    if (in.dev.made.tcg[plan].streamed) return true;
  return false;
}

// Shared memory of a tensor-core sampler launch over every instance.
int tc_sampler_smem(const tnvan_ctx* ctx, int plan, bool grouped) {
  int smem = 0;
  for (const Instance& in : ctx->inst) {
    if (grouped) {
      const MadeDev::TcGroupPlan& P = in.dev.made.tcg[plan];
      smem = std::max(smem, sample_tcg_smem_bytes((int)in.W.size(), in.H[0], in.H[1], P.tcw1, P.tcw2, P.twmax,
                                                  P.streamed ? P.wbmax : 0));
    } else {
      smem = std::max(smem, sample_tc_smem_bytes(in.dev.made, plan));
    }
  }
  return smem;
}

// Tensor-core sampler plan usable by every instance: the autotuned one, else
// the largest group-size limit that fits, else -1 (SIMT sampler).
int pick_tc_plan(const tnvan_ctx* ctx) {
  const bool grouped = tc_grouped_usable(ctx);
  auto usable = [&](int p) {
    if (p < 0 || p >= TNVAN_TC_PLANS) return false;
    for (const Instance& in : ctx->inst)
      if (!(grouped ? in.dev.made.tcg[p].ok : in.dev.made.tc[p].ok)) return false;
    return true;
  };
  if (usable(ctx->tune_tc_plan)) return ctx->tune_tc_plan;
  for (int p = TNVAN_TC_PLANS - 1; p >= 0; --p)
    if (usable(p)) return p;
  return -1;
}

int run_sampler(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step, int precision,
                int8_t* d_spins, float* d_logq, const int8_t* given, cudaStream_t s) {
  int rc;
  bool tc_all = precision == TNVAN_BF16;
  tc_all = tc_all && tc_sampler_usable(ctx);
  int plan = -1;
  if (tc_all) plan = pick_tc_plan(ctx);
  if (plan >= 0) {
    LaunchInfo li;
    if ((rc = fill_launch(ctx, betas, batch, 128, li))) return rc;
    li.seed = seed;
    li.step = step;
    const bool grouped = tc_grouped_usable(ctx);
    PROF(given ? "log_prob_tc" : "sample_tc", s);
    if (grouped) {
      const int smem = tc_sampler_smem(ctx, plan, grouped);
      CK(launch_sample_tcg(ctx->d_inst, li, tcg_order(ctx, li, 0, li.n_inst), plan, smem,
                           tc_any_streamed(ctx, plan), d_spins, d_logq, given, s),
         "tensor-core sample kernel");
      return TNVAN_OK;
    }
    // per-step form: instances whose CTAs fit two per SM (<= 256 TMEM columns)
    // launch apart from those that need a whole SM, each launch with its own
    // shared memory (a launch's CTAs all take its largest instance's); the
    // other class's instances get no blocks (empty tile ranges)
    for (int cls = 0; cls < 2; ++cls) {
      LaunchInfo lc = li;
      int acc = 0, smem = 0;
      for (int k = 0; k < li.n_inst; ++k) {
        lc.tile_begin[k] = acc;
        const MadeDev& md = ctx->inst[k].dev.made;
        if ((md.tc[plan].tmem_cols > 256) == (cls == 1)) {
          acc += li.tile_begin[k + 1] - li.tile_begin[k];
          smem = std::max(smem, sample_tc_smem_bytes(md, plan));
        }
      }
      lc.tile_begin[li.n_inst] = acc;
      if (acc == 0) continue;
      CK(launch_sample_tc(ctx->d_inst, lc, plan, ctx->inst[0].dev.made.nh, smem, d_spins, d_logq, given, s),
         "tensor-core sample kernel");
    }
    return TNVAN_OK;
  }
  const int tile = pick_sample_tile(ctx);
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, tile, li))) return rc;
  li.seed = seed;
  li.step = step;
  PROF(given ? "log_prob" : "sample", s);
  CK(launch_sample(ctx->d_inst, li, max_sample_smem(ctx, tile), d_spins, d_logq, given, s), "sample kernel");
  return TNVAN_OK;
}

int contract_all(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                 int precision, double* d_logZR, double* d_dbeta, cudaStream_t s, bool strips) {
  int rc;
  bool k0 = false, k1 = false, k2 = false;
  for (const Instance& in : ctx->inst) {
    k0 |= in.kind == 0 && strips;
    k1 |= in.kind == 1;
    k2 |= in.kind == 2;
  }
  const int stile = ctx->tune_strip_tile ? ctx->tune_strip_tile : 128;
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, stile, li))) return rc;
  if (k0) {
    int sm = 0;
    for (const Instance& in : ctx->inst)
      if (in.kind == 0) sm = std::max(sm, strip_smem_bytes(in, stile));
    if (sm > 227 * 1024) return fail(ctx, TNVAN_E_UNSUPPORTED, "strip tables need %d B of shared memory", sm);
    PROF(d_dbeta ? (d_logZR ? "strips+dbeta" : "strips_dbeta") : "strips", s);
    CK(launch_strips(ctx->d_inst, li, sm, d_spins, d_logZR, d_dbeta, s), "strip kernel");
  }
  if (k1) {
    PROF(d_dbeta ? "dense_dbeta" : "dense", s);
    int max_D = 0;
    for (const Instance& in : ctx->inst)
      if (in.kind == 1) max_D = std::max(max_D, (int)in.W.size());
    CK(launch_dense(ctx->d_inst, li, precision, d_spins, d_logZR, d_dbeta, nullptr, s, max_D), "dense kernel");
  }
  // lattice instances with a wide-strip plan: log Z_R by the wide-strip
  // kernel (forward mode d/dbeta stays with their elimination plans)
  bool any_wide = false;
  for (const Instance& in : ctx->inst) any_wide = any_wide || (in.kind == 2 && in.dev.n_wide > 0 && !d_dbeta);
  if (any_wide) {
    LaunchInfo lw;
    if ((rc = fill_launch(ctx, betas, batch, 1, lw))) return rc;
    int acc = 0, ms = 0, Dm = 0;
    bool rest = false;
    for (int k = 0; k < lw.n_inst; ++k) {
      const Instance& in = ctx->inst[k];
      lw.tile_begin[k] = acc;
      if (in.kind == 2 && in.dev.n_wide > 0) {
        acc += batch;
        ms = std::max(ms, in.dev.n_wide);
        Dm = std::max(Dm, (int)in.W.size());
      } else if (in.kind == 2) {
        rest = true;
      }
    }
    lw.tile_begin[lw.n_inst] = acc;
    int per_class[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (const Instance& in : ctx->inst) {
      if (in.kind != 2 || in.dev.n_wide == 0) continue;
      int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (const WideStripDev& sd : in.wide.strips) ++cnt[sd.w <= 5 ? 0 : sd.w - 5];
      for (int c = 0; c < 8; ++c) per_class[c] = std::max(per_class[c], cnt[c]);
    }
    if ((rc = ensure_wide_part(ctx, (size_t)lw.n_inst * batch * ms))) return rc;
    PROF("wide_strips", s);
    CK(launch_wide(ctx->d_inst, lw, per_class, ms, Dm, d_spins, ctx->d_wide_part, d_logZR, s), "wide-strip kernels");
    k2 = rest;
  }
  if (k2) {
    int arena = 0, Dm = 0, nsteps = 0;
    for (const Instance& in : ctx->inst)
      if (in.kind == 2) {
        arena = std::max(arena, in.g_max_live);
        Dm = std::max(Dm, (int)in.W.size());
        nsteps = std::max(nsteps, (int)in.gfstep.size());
      }
    const bool db = d_dbeta != nullptr;
    const int GL = gen_lanes(ctx, batch, 16), T = 128 / GL;
    const bool glob =
        gen_tables_global(T, [&](int t, bool g) { return general_smem_bytes(arena, Dm, t, GL, db, g); });
    const int sm = general_smem_bytes(arena, Dm, T, GL, db, glob);
    if (sm > 227 * 1024) return fail(ctx, TNVAN_E_UNSUPPORTED, "elimination tables need %d B of shared memory", sm);
    LaunchInfo lg;
    if ((rc = fill_launch(ctx, betas, batch, T, lg))) return rc;
    lg.seed = (unsigned long long)arena;
    if (any_wide) {  // instances the wide-strip kernel has contracted get no tiles
      int acc = 0;
      for (int k = 0; k < lg.n_inst; ++k) {
        const int nt = lg.tile_begin[k + 1] - lg.tile_begin[k];
        lg.tile_begin[k] = acc;
        if (!(ctx->inst[k].kind == 2 && ctx->inst[k].dev.n_wide > 0)) acc += nt;
      }
      lg.tile_begin[lg.n_inst] = acc;
    }
    {
      PROF("general_pp", s);
      CK(launch_general_pp(ctx->d_inst, lg, nsteps, s), "elimination bond products");
    }
    // components with small boundaries: tables when they are smaller than the batch
    for (const Instance& in : ctx->inst)
      if (in.kind == 2 && in.g_ntab > 0 && in.g_ntab <= batch)
        lg.gen_tab = std::max(lg.gen_tab, in.g_ntab);
    float* gs = nullptr;
    if (glob) {
      if ((rc = ensure_gen_scratch(ctx, 0, general_scratch_floats(lg, arena, GL, db)))) return rc;
      gs = ctx->d_gen_scratch[0];
    }
    if (lg.gen_tab > 0) {
      PROF("general_tables", s);
      CK(launch_general_tables(ctx->d_inst, lg, sm, db, GL, gs, s), "general tables kernel");
    }
    PROF(d_dbeta ? "general_dbeta" : "general", s);
    CK(launch_general(ctx->d_inst, lg, sm, GL, d_spins, d_logZR, d_dbeta, gs, s), "general kernel");
  }
  return TNVAN_OK;
}

// Contraction adjoint (Eq. 4 differentiated): d log Z_R / d beta per sample
// and the batch-mean d log Z_R / d J, each optional; with d_logZR non-NULL
// also log Z_R itself (strip instances from the adjoint's own forward sweep,
// the other kinds from their contraction kernels).
int run_adjoint(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins, int precision,
                double* d_logZR, double* d_dbeta, double* d_dJ, cudaStream_t s, const float* wmul) {
  int rc;
  bool any_strip = false, other = false;
  for (const Instance& in : ctx->inst) {
    if (in.kind == 0) any_strip = true;
    else other = true;
  }
  // the strip adjoint keeps a strip's left vectors in shared memory: 128,
  // 96, 64 or 32 samples per CTA
  int adj_tile = 0, adj_smem = 0, adj_lv = 0, adj_ws = 0;
  if (any_strip && (rc = plan_strip_adjoint(ctx, batch, &adj_tile, &adj_smem, &adj_lv, &adj_ws))) return rc;
  LaunchInfo li;
  if ((rc = fill_launch(ctx, betas, batch, 1, li))) return rc;
  li.wmul = wmul;  // weighted bond sums (W-W bonds)
  if (d_dJ) {
    long long ne = 0;
    for (const Instance& in : ctx->inst) ne += in.m;
    CK(cudaMemsetAsync(d_dJ, 0, ne * sizeof(double), s), "dJ memset");
  }
  if (other && (d_logZR || d_dbeta)) {
    // dense and elimination instances: log Z_R and forward-mode d/dbeta
    if ((rc = contract_all(ctx, betas, batch, d_spins, precision, d_logZR, d_dbeta, s, false))) return rc;
  }
  if (adj_tile) {
    LaunchInfo la;
    if ((rc = fill_launch(ctx, betas, batch, adj_tile, la))) return rc;
    la.wmul = wmul;
    int max_edges = 0;
    for (const Instance& in : ctx->inst)
      if (in.kind == 0) max_edges = std::max(max_edges, in.m);
    const int stride = (max_edges + 3) & ~3;
    if (d_dJ && (rc = ensure_dj_part(ctx, (size_t)la.tile_begin[la.n_inst] * stride))) return rc;
    CK(launch_strip_tables(ctx->d_inst, la, 0, la.n_inst, s), "strip tables");
    PROF(d_dJ ? "strips_adj" : "strips_dbeta", s);
    CK(launch_strips_adj(ctx->d_inst, la, adj_smem, adj_lv, d_spins, d_logZR, d_dbeta,
                         d_dJ ? ctx->d_dj_part : nullptr, stride, d_dJ, s, 0, -1, adj_ws),
       "strip adjoint kernel");
  }
  if (d_dJ) {
    LaunchInfo lt;
    if ((rc = fill_launch(ctx, betas, batch, 128, lt))) return rc;
    lt.wmul = wmul;
    if (other) {
      {
        PROF("ww_dJ", s);
        CK(launch_ww(ctx->d_inst, li, d_spins, d_dJ, s), "W-W adjoint kernel");
      }
      {
        PROF("dense_dJ", s);
        CK(launch_dense(ctx->d_inst, lt, precision, d_spins, nullptr, nullptr, d_dJ, s), "dense adjoint kernel");
      }
      int arena = 0, steps = 0, Dm = 0, me = 0, nsteps = 0, mw = 0;
      bool any_gen = false;
      for (const Instance& in : ctx->inst)
        if (in.kind == 2) {
          any_gen = true;
          arena = std::max(arena, in.g_max_entries);
          steps = std::max(steps, in.g_max_steps);
          Dm = std::max(Dm, (int)in.W.size());
          me = std::max(me, in.m);
          nsteps = std::max(nsteps, (int)in.gfstep.size());
          mw = std::max(mw, in.max_width);
        }
      if (any_gen) {
        const int gmax = 2 << mw;  // g of one step: 2^(m+1) extended indices
        const int per = 2 * arena + steps + gmax;
        const int GL = gen_lanes(ctx, batch, 8), T = 128 / GL;
        const bool glob =
            gen_tables_global(T, [&](int t, bool g) { return general_dJ_smem_bytes(per, Dm, me, t, GL, g); });
        const int sm = general_dJ_smem_bytes(per, Dm, me, T, GL, glob);
        if (sm > 227 * 1024) return fail(ctx, TNVAN_E_UNSUPPORTED, "elimination adjoint needs %d B of shared memory", sm);
        LaunchInfo lg;
        if ((rc = fill_launch(ctx, betas, batch, T, lg))) return rc;
        lg.wmul = wmul;
        const int stride = (me + 3) & ~3;
        if ((rc = ensure_dj_part(ctx, (size_t)lg.tile_begin[lg.n_inst] * stride))) return rc;
        float* gs = nullptr;
        if (glob) {
          if ((rc = ensure_gen_scratch(ctx, 1, general_dJ_scratch_floats(per, T, GL, lg.tile_begin[lg.n_inst]))))
            return rc;
          gs = ctx->d_gen_scratch[1];
        }
        {
          PROF("general_pp", s);
          CK(launch_general_pp(ctx->d_inst, lg, nsteps, s), "elimination bond products");
        }
        PROF("general_dJ", s);
        CK(launch_general_dJ(ctx->d_inst, lg, sm, arena, steps, gmax, GL, d_spins, ctx->d_dj_part, stride, d_dJ, gs,
                             s),
           "general adjoint kernel");
      }
    }
  }
  return TNVAN_OK;
}


// Dense leftover block: R (|R| <= 16, in index order) split in halves A = R[0..7]
// and B = R[8..15]; missing spins are free phantoms (no couplings).
int plan_dense(tnvan_ctx* ctx, Instance& in, const std::vector<int>& pos) {
  std::vector<int> R;
  for (int v = 0; v < in.n; ++v)
    if (pos[v] < 0) R.push_back(v);
  if (R.size() > 16) return TNVAN_E_UNSUPPORTED;
  const int D = (int)in.W.size();
  std::vector<int> rpos(in.n, -1);
  for (size_t i = 0; i < R.size(); ++i) rpos[R[i]] = (int)i;
  in.dense_nR = (int)R.size();
  in.JRW.assign(16 * D, 0.f);
  in.JRR.assign(16 * 16, 0.f);
  in.eRR.assign(16 * 16, -1);
  in.eRW.assign(16 * D, -1);
  double chat = 0;
  for (int e = 0; e < in.m; ++e) {
    const int a = in.ei[e], b = in.ej[e];
    const int ra = rpos[a], rb = rpos[b];
    if (ra >= 0 && rb >= 0) {
      in.JRR[ra * 16 + rb] = in.JRR[rb * 16 + ra] = (float)in.J[e];
      in.eRR[ra * 16 + rb] = in.eRR[rb * 16 + ra] = e;
      chat += fabs((double)(float)in.J[e]);
    } else if (ra >= 0 || rb >= 0) {
      const int r = ra >= 0 ? ra : rb, w = ra >= 0 ? pos[b] : pos[a];
      in.JRW[r * D + w] = (float)in.J[e];
      in.eRW[r * D + w] = e;
    }
  }
  (void)ctx;
  in.dense_chat = chat;
  in.kind = 1;
  return TNVAN_OK;
}

// General leftover components: each connected component of R is compiled into
// a variable-elimination program (order: min-fill on the component graph, ties
// to the lowest local index; or, when `rank` is non-empty, the order of the
// component's spins by rank).  Program layout (ints), per component:
//   n_steps, arena_floats, final_offset, then per step:
//   v, fld_begin, fld_count, m, out_off, n_in, n_pair,
//   n_in x { in_off, k, pos_0 .. pos_{k-1} }  (pos in the extended scope out+{v})
//   n_pair x { pair_id, pos_u }                (pos of the neighbour in the out scope)
// fld: per W-neighbour bond of an R spin, (AR position, edge id); fldJ its coupling.
int plan_general(tnvan_ctx* ctx, Instance& in, const std::vector<int>& pos, const std::vector<int>& rank) {
  auto comps = r_components(in, pos);
  std::vector<std::vector<std::pair<int, int>>> adj(in.n);  // (neighbour, edge)
  for (int e = 0; e < in.m; ++e) {
    adj[in.ei[e]].push_back({in.ej[e], e});
    adj[in.ej[e]].push_back({in.ei[e], e});
  }
  std::vector<int> prog{(int)comps.size()};
  std::vector<int> fld, pairE, step_off, comp_step0, ctab, bpos, tabc;
  int n_tab = 0;
  std::vector<float> fldJ, pairJ;
  int max_steps = 0;
  double chat = 0;
  int arena_max = 0, width_max = 0;
  for (const auto& comp : comps) {
    const int n = (int)comp.size();
    std::map<int, int> loc;
    for (int i = 0; i < n; ++i) loc[comp[i]] = i;
    // local graph, pair ids, field lists
    std::vector<std::set<int>> g(n);
    std::map<std::pair<int, int>, int> pair_of;  // (lo, hi) local -> pair id
    std::vector<int> fb(n), fc(n);
    for (int i = 0; i < n; ++i) {
      fb[i] = (int)fld.size() / 2;
      for (auto [u, e] : adj[comp[i]]) {
        auto it = loc.find(u);
        if (it != loc.end()) {
          const int j = it->second;
          g[i].insert(j);
          if (i < j) {
            pair_of[{i, j}] = (int)pairJ.size();
            pairJ.push_back((float)in.J[e]);
            pairE.push_back(e);
            chat += fabs((double)(float)in.J[e]);
          }
        } else if (pos[u] >= 0) {
          fld.push_back(pos[u]);
          fld.push_back(e);
          fldJ.push_back((float)in.J[e]);
        }
      }
      fc[i] = (int)fld.size() / 2 - fb[i];
    }
    // min-fill elimination order
    std::vector<std::set<int>> h = g;
    std::vector<char> gone(n, 0);
    std::vector<int> order;
    if (!rank.empty()) {
      for (int i = 0; i < n; ++i) order.push_back(i);
      std::sort(order.begin(), order.end(), [&](int a, int b) { return rank[comp[a]] < rank[comp[b]]; });
    }
    for (int step = (int)order.size(); step < n; ++step) {
      int best = -1;
      long best_fill = -1;
      for (int v = 0; v < n; ++v) {
        if (gone[v]) continue;
        long fill = 0;
        for (auto a = h[v].begin(); a != h[v].end(); ++a)
          for (auto b = std::next(a); b != h[v].end(); ++b)
            if (!h[*a].count(*b)) ++fill;
        if (best < 0 || fill < best_fill) {
          best = v;
          best_fill = fill;
        }
      }
      order.push_back(best);
      gone[best] = 1;
      for (int a : h[best])
        for (int b : h[best])
          if (a != b) h[a].insert(b);
      for (int a : h[best]) h[a].erase(best);
      h[best].clear();
    }
    // simulate elimination to emit the program
    struct Fac { std::vector<int> scope; int off; };
    std::vector<Fac> active;
    std::set<std::pair<int, int>> edges_left;
    for (auto& kv : pair_of) edges_left.insert(kv.first);
    const size_t hdr = prog.size();
    // the component's width-set boundary; tabulated when small
    {
      std::set<int> bset;
      for (int i = 0; i < n; ++i)
        for (int f = fb[i]; f < fb[i] + fc[i]; ++f) bset.insert(fld[2 * f]);
      const int kb = (int)bset.size();
      const int toff = kb <= TNVAN_TAB_MAX_K ? n_tab : -1;
      if (toff >= 0) {
        n_tab += 1 << kb;
        tabc.push_back((int)ctab.size() / 5);
      }
      ctab.push_back((int)hdr);
      ctab.push_back(0);  // program end, patched below
      ctab.push_back(kb);
      ctab.push_back((int)bpos.size());
      ctab.push_back(toff);
      bpos.insert(bpos.end(), bset.begin(), bset.end());
    }
    comp_step0.push_back((int)step_off.size());
    max_steps = std::max(max_steps, n);
    prog.push_back(n);
    prog.push_back(0);  // arena size, patched below
    prog.push_back(0);  // final offset, patched below
    int arena = 0, last_off = 0;
    for (int v : order) {
      std::vector<Fac> use, keep;
      for (auto& f : active) (std::count(f.scope.begin(), f.scope.end(), v) ? use : keep).push_back(f);
      active.swap(keep);
      std::vector<std::pair<int, int>> pairs;  // (pair id, u)
      for (int u : g[v]) {
        auto key = std::make_pair(std::min(u, v), std::max(u, v));
        if (edges_left.count(key)) {
          pairs.push_back({pair_of[key], u});
          edges_left.erase(key);
        }
      }
      std::set<int> sc;
      for (auto& f : use) sc.insert(f.scope.begin(), f.scope.end());
      for (auto& p : pairs) sc.insert(p.second);
      sc.erase(v);
      std::vector<int> out(sc.begin(), sc.end());
      const int m = (int)out.size();
      if (m > TNVAN_MAX_ELIM_W)
        return fail(ctx, TNVAN_E_UNSUPPORTED, "component of %d spins needs elimination width %d (max %d)", n, m, TNVAN_MAX_ELIM_W);
      width_max = std::max(width_max, m);
      auto ext_pos = [&](int var) -> int {
        if (var == v) return m;
        return (int)(std::lower_bound(out.begin(), out.end(), var) - out.begin());
      };
      step_off.push_back((int)prog.size());
      prog.push_back(v);
      prog.push_back(fb[v]);
      prog.push_back(fc[v]);
      prog.push_back(m);
      prog.push_back(arena);
      prog.push_back((int)use.size());
      prog.push_back((int)pairs.size());
      for (auto& f : use) {
        prog.push_back(f.off);
        prog.push_back((int)f.scope.size());
        for (int var : f.scope) prog.push_back(ext_pos(var));
      }
      for (auto& p : pairs) {
        prog.push_back(p.first);
        prog.push_back(ext_pos(p.second));
      }
      active.push_back(Fac{out, arena});
      last_off = arena;
      arena += 1 << m;
    }
    prog[hdr + 1] = arena;
    prog[hdr + 2] = last_off;
    ctab[ctab.size() - 4] = (int)prog.size();
    arena_max = std::max(arena_max, (arena + 3) & ~3);  // keeps the float4 pair table aligned
  }
  comp_step0.push_back((int)step_off.size());
  // Forward-only passes keep a table only until the step that consumes it:
  // the same program with offsets from a first-fit allocator over the
  // arena (the new table is placed before its inputs are released).
  std::vector<int> fwd(prog);
  int live_max = 0;
  for (size_t c = 0; c < comps.size(); ++c) {
    std::map<int, int> free_;          // start -> length
    std::map<int, std::pair<int, int>> where;  // full offset -> (live offset, size)
    std::vector<int> owner;            // self-check: live entry -> step + 1
    int top = 0;
    auto alloc = [&](int sz) {
      for (auto it = free_.begin(); it != free_.end(); ++it)
        if (it->second >= sz) {
          const int off = it->first, len = it->second;
          free_.erase(it);
          if (len > sz) free_[off + sz] = len - sz;
          return off;
        }
      const int off = top;
      top += sz;
      return off;
    };
    auto release = [&](int off, int sz) {
      auto nx = free_.lower_bound(off);
      if (nx != free_.end() && nx->first == off + sz) {
        sz += nx->second;
        free_.erase(nx);
      }
      auto pv = free_.lower_bound(off);
      if (pv != free_.begin()) {
        --pv;
        if (pv->first + pv->second == off) {
          off = pv->first;
          sz += pv->second;
          free_.erase(pv);
        }
      }
      free_[off] = sz;
    };
    for (int st = comp_step0[c]; st < comp_step0[c + 1]; ++st) {
      const int r = step_off[st];
      const int m = prog[r + 3], out = prog[r + 4], nin = prog[r + 5];
      const int lo = alloc(1 << m);
      if ((int)owner.size() < top) owner.resize(top, 0);
      for (int x = 0; x < (1 << m); ++x) {
        if (owner[lo + x]) return fail(ctx, TNVAN_E_UNSUPPORTED, "internal: overlapping tables in the live layout");
        owner[lo + x] = st + 1;
      }
      where[out] = {lo, 1 << m};
      fwd[r + 4] = lo;
      int q = r + 7;
      for (int i = 0; i < nin; ++i) {
        auto it = where.find(prog[q]);
        if (it == where.end()) return fail(ctx, TNVAN_E_UNSUPPORTED, "internal: table consumed before it is made");
        fwd[q] = it->second.first;
        for (int x = 0; x < it->second.second; ++x) owner[it->second.first + x] = 0;
        release(it->second.first, it->second.second);
        where.erase(it);
        q += 2 + prog[q + 1];
      }
    }
    const int hdr = ctab[5 * c];
    auto it = where.find(prog[hdr + 2]);
    if (it == where.end()) return fail(ctx, TNVAN_E_UNSUPPORTED, "internal: no final table");
    fwd[hdr + 2] = it->second.first;
    live_max = std::max(live_max, (top + 3) & ~3);
  }
  // compiled step records and input index maps
  {
    std::vector<int> F, fh, fs(step_off.size());
    std::vector<unsigned short> mp;
    int npp = 0;
    for (size_t c = 0; c < comps.size(); ++c) {
      const int hdr = ctab[5 * c];
      fh.push_back((int)F.size());
      F.push_back(prog[hdr]);
      F.push_back(fwd[hdr + 2]);
      F.push_back(prog[hdr + 2]);
      for (int st = comp_step0[c]; st < comp_step0[c + 1]; ++st) {
        const int r = step_off[st];
        const int m = prog[r + 3], nin = prog[r + 5], npair = prog[r + 6], E = 2 << m;
        fs[st] = (int)F.size();
        F.push_back(m);
        F.push_back(prog[r + 1]);
        F.push_back(prog[r + 2]);
        F.push_back(nin);
        F.push_back(npair);
        F.push_back(npp);
        F.push_back((int)mp.size());
        F.push_back(fwd[r + 4]);
        F.push_back(prog[r + 4]);
        npp += E;
        int q = r + 7;
        std::vector<std::vector<int>> idx_of(nin, std::vector<int>(E));
        std::vector<int> kin(nin);
        for (int i = 0; i < nin; ++i) {
          const int k = prog[q + 1];
          kin[i] = k;
          F.push_back(fwd[q]);
          F.push_back(prog[q]);
          F.push_back(k);
          for (int ext = 0; ext < E; ++ext) {
            int idx = 0;
            for (int j = 0; j < k; ++j) idx |= ((ext >> prog[q + 2 + j]) & 1) << j;
            idx_of[i][ext] = idx;
            mp.push_back((unsigned short)idx);
          }
          q += 2 + k;
        }
        // inverse maps: per input, the extended indices of each entry (E >> k
        // of them, increasing), entry-major
        for (int i = 0; i < nin; ++i) {
          std::vector<unsigned short> inv(E);
          std::vector<int> fill_(1 << kin[i], 0);
          const int R = E >> kin[i];
          for (int ext = 0; ext < E; ++ext) {
            const int e = idx_of[i][ext];
            inv[e * R + fill_[e]++] = (unsigned short)ext;
          }
          mp.insert(mp.end(), inv.begin(), inv.end());
        }
        for (int j = 0; j < npair; ++j) {
          F.push_back(prog[q + 2 * j]);
          F.push_back(prog[q + 2 * j + 1]);
        }
      }
    }
    {
      double tot = 0;
      for (size_t st = 0; st < step_off.size(); ++st) tot += (double)(1 << prog[step_off[st] + 3]);
      in.g_mean_entries = step_off.empty() ? 1.0 : tot / (double)step_off.size();
    }
    in.gfprog.swap(F);
    in.gfhdr.swap(fh);
    in.gfstep.swap(fs);
    in.gmap.swap(mp);
    in.g_npp = npp;
  }
  in.gprog_fwd.swap(fwd);
  in.g_max_live = live_max;
  in.gprog.swap(prog);
  in.gfld.swap(fld);
  in.gpairE.swap(pairE);
  in.gstep_off.swap(step_off);
  in.gcomp_step0.swap(comp_step0);
  in.g_max_steps = max_steps;
  in.gfldJ.swap(fldJ);
  in.gpairJ.swap(pairJ);
  in.g_npairs = (int)in.gpairJ.size();
  in.g_ncomp = (int)comps.size();
  in.g_max_entries = arena_max;
  in.g_chat = chat;
  in.max_width = width_max;
  in.gctab.swap(ctab);
  in.gbpos.swap(bpos);
  in.gtabc.swap(tabc);
  in.g_ntab = n_tab;
  in.kind = 2;
  return TNVAN_OK;
}

}  // namespace
