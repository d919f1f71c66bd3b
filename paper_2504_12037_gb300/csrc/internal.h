// Internal declarations of the TNVAN GB300 library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tnvan.h"

#define TNVAN_MAX_INST 128
#define TNVAN_MAX_HIDDEN 512
#define TNVAN_MAX_D 1024
#define TNVAN_MAX_STRIP_W 4
#define TNVAN_MAX_ELIM_W 12
#define GROUP_INTS 15
#define TNVAN_TC_PLANS 3  // tensor-core sampler plans: grouped 4, 6, 8 steps; per-step chunks 12, 16, 32
// Tensor-core sampler chunk record: i0 i1 (steps), w1c n1c (16-aligned window
// of the chunk's layer-1 units), w2c n2c (layer 2), kSc (K width of the W1
// rows: spins 0 .. kSc-1), blob offset (BF16 elements, a multiple of 8), the
// blob's three part sizes in bytes (W2 window, Wo window, W1 rows), pad.
#define TNVAN_TCG_INTS 16
// Grouped tensor-core sampler group record: i0 i1 u1lo u1hi u2lo u2hi, block
// start and size (floats), offsets of TW2 TWo b1 b2 bo in the block, then c1
// and c2 at the group's steps (9 each: units with degree < i0 + q, q = 0..8),
// pad.
#define TNVAN_TCGG_INTS 32

namespace tnvan {

// ---------------------------------------------------------------------------
// Device-side descriptors (plain structs, pointers into context-owned memory).
// ---------------------------------------------------------------------------

// One layer of the packed network: units of hidden layers are stored sorted by
// MADE degree, so "all units of degree <= d" is a prefix.
struct LayerDev {
  int nin, nout;
  long long src_off;  // offset of W_l in the caller's natural parameter layout
  long long dst_off;  // offset of the packed [nout][nin] block in the packed buffer
  const int* perm_in;   // packed input index -> natural (nullptr = identity)
  const int* perm_out;  // packed output index -> natural (nullptr = identity)
  const int* deg_in;    // degree of each packed input
  const int* deg_out;   // degree of each packed output
  int strict;           // output layer: connect iff deg_out > deg_in, else >=
};

struct MadeDev {
  int D, nh, H1, H2, Hl;  // Hl = width feeding the output layer (D if nh == 0)
  int n_layers;
  LayerDev layer[3];
  float* raw;             // borrowed natural-layout parameters (written only by the fused Adam step)
  float* packed;          // packed, masked, degree-sorted copy (W then b per layer)
  uint16_t* packed16;     // the same in BF16 (round to nearest even): the GEMM chain's weight operands
  const int* c1;          // [D+1] number of layer-1 units with degree <= d
  const int* c2;          // [D+1] number of layer-2 units with degree <= d
  // Blocked sampler: steps are grouped; for each group and layer the weights
  // from all earlier inputs to the group's units are stored as chunks of 16
  // units, [n_in][16] floats each (see k_made.cu).
  int n_groups;
  const int* groups;      // [n_groups][GROUP_INTS], see k_made.cu
  int ug1, ug2, ugo;      // largest group unit counts per layer
  int wmax;               // largest per-group weight block (floats)
  // Tensor-core sampler: one step-chunk plan per chunk-size limit.  Per
  // chunk one BF16 weight blob in the MMA's K-major canonical layout (see
  // k_sample_tc.cu): the K-window of W2 over the chunk's layer-1 units, that
  // of Wo over its layer-2 (or, with one hidden layer, layer-1) units, and
  // W1's rows of its layer-1 units.
  struct TcPlan {
    int ok;               // eligible (sizes within the kernel's limits)
    int n_chunks;
    const int* chunks;    // [n_chunks][TNVAN_TCG_INTS], see TNVAN_TCG_INTS
    uint16_t* wblob;      // BF16 blobs (zero where no weight), gathered from the network on every call
    const int* wsrc;      // [n_wblob] the live elements: index into the packed network
    const int* wdst;      // [n_wblob] and element of wblob
    long long n_wblob;
    int dp;               // D padded to a multiple of 16
    int tcw1;             // TMEM columns of the chunk's layer-1 pre-activations
    int dw1, dw2;         // widest per-step unit window (delta tiles), layers 1 and 2
    int wbmax;            // largest chunk blob (bytes)
    int tmem_cols;        // TMEM allocation of a CTA
    // In-step weights of every step i (FP32, gathered on every call): from
    // its layer-1 units to its layer-2 units [nv][nu], then from its last
    // hidden layer's units to output i [nv] (one hidden layer: [nu]).
    float* steptab;
    const int* stepsrc;   // [n_steptab] index into the packed network
    const int* stepoff;   // [D + 1] offset of step i's table
    int n_steptab;
  } tc[TNVAN_TC_PLANS];
  // Grouped tensor-core sampler (the fast path for two hidden layers of
  // <= 128 units and D <= 128, a multiple of 16): one step-group plan per
  // group-size limit.  Per group only the in-group triangles: per unit, rows
  // padded to 4 floats, TW1 [n1g][r4(gi)], TW2 [n2g][r4(n1g)], TWo [gi][r4(n2g)];
  // or, when at most 4 units of a layer complete at any step, per slot (U
  // slots per layer and step, strides for 8 steps; see the host builder).
  struct TcGroupPlan {
    int ok;               // eligible (unit counts within the kernel's limits)
    int n_groups;
    const int* groups;    // [n_groups][TNVAN_TCGG_INTS]
    float* blocks;        // gathered from `packed` on every call
    const int* src;       // [n_blk] index into `packed`, -1 = zero
    long long n_blk;
    int twmax;            // largest group (floats)
    int tcw1, tcw2;       // widest 16-aligned unit window of a group, layers 1 and 2
    int slot_u;           // 0: per-unit triangles; 1..4: slot layout, U slots per layer and step
    // streamed weights (width sets the resident tiles do not fit: D up to 256):
    // per group one BF16 blob in the MMA's K-major layout, bulk-copied one
    // group ahead -- the W2 window [H2 x n1], the Wo window [Dp x n2] and W1's
    // rows of the group's layer-1 units [n1 x r16(i0)]; record word 31 = its
    // element offset
    int streamed;
    uint16_t* wblob;      // gathered from the network on every call (zero where no weight)
    const int* wsrc;      // [n_wblob] the live elements: index into the packed network
    const int* wdst;      // [n_wblob] and element of wblob
    long long n_wblob;
    int wbmax;            // largest blob (bytes)
  } tcg[TNVAN_TC_PLANS];
  int sample_tcg_ok;      // eligible for the grouped sampler
  float* blocks;          // blocked weights (gathered from `packed` every call)
  const int* blk_src;     // [n_blk] index into `packed`, -1 = zero
  long long n_blk;
  int fused_ok;           // eligible for the fused BF16 tcgen05 backward
  int sample_tc_ok;       // eligible for the BF16 tcgen05 sampler
  uint16_t* wtiles;       // BF16 K-major tiles W1 [H1 x D] | W2 [H2 x H1] | Wo [D x H2] (fused kernels)
  long long n_params;     // size of the natural layout
  long long param_off;    // offset in the all-instances packed gradient layout
};

// Lattice strip: w whole columns x0..x0+w-1, L rows.  Row y has horizontal
// bonds Jh[c] (c, c+1), left/right W neighbours at AR positions posL/posR
// (-1 = none), and vertical bonds Jv[c] to row y+1.  The same bonds by slot
// (w-1 horizontal, left, right, w vertical), as the adjoint reads them: Js the
// coupling (0 = no bond), es the edge id (-1 = none).
#define TNVAN_STRIP_SLOTS 12  // >= 2 * TNVAN_MAX_STRIP_W + 1, a multiple of 4
struct alignas(16) StripRow {
  float Js[TNVAN_STRIP_SLOTS];
  int es[TNVAN_STRIP_SLOTS];
  float Jh[TNVAN_MAX_STRIP_W - 1];
  float JL, JR;
  int posL, posR;
  float Jv[TNVAN_MAX_STRIP_W];
  int eh[TNVAN_MAX_STRIP_W - 1];  // edge ids (-1 none), for d/dJ
  int eL, eR;
  int ev[TNVAN_MAX_STRIP_W];
  int tau_mask;  // bit c set iff the gauge flips column c in this row (model spin = -strip spin)
};

// Wide lattice strip (5 to TNVAN_WIDE_MAX_W whole columns; forward
// contraction of elimination instances, see k_wide.cu): per row the
// gauge-signed horizontal couplings Jh[c] (c, c+1), the W-neighbour couplings
// JL, JR (0 = none) with their AR positions, and the vertical couplings
// Jv[c] >= 0 to the next row (the planner's gauge, as for StripRow).
#define TNVAN_WIDE_MAX_W 12
struct WideRow {
  float Jh[TNVAN_WIDE_MAX_W - 1];
  float JL, JR;
  float Jv[TNVAN_WIDE_MAX_W];
  int posL, posR;
};
struct WideStripDev {
  int w, L;
  int row0;      // first row in the instance's wide-row array
  int pad;
  double c_hat;  // sum of |J| over the strip's bonds (horizontal, vertical, W neighbours)
};

struct StripDev {
  int w, L;
  int row0;       // index of the first row in the instance's row array
  int tab_off;    // float offset of this strip's tables in shared memory
  double c_hat;   // sum_y (sum|Jh| + |JL| + |JR|) + sum |Jv|: constant log-offset / beta
};

struct EdgeWW {
  int a, b;  // AR positions
  float J;
  int e;     // edge id
};

// Dense block: R = 16 spins (padded), split in halves A (first 8) and B.
struct DenseDev {
  int nR;              // real leftover spins (<= 16)
  int nA, nB;          // real spins in each half (<= 8)
  const float* JRW;    // [16][D] couplings R -> W positions (zero rows for padding)
  const float* JRR;    // [16][16] symmetric, zero diagonal, zero padding
  float* C32;          // [256][256] exp(beta(E_AA+E_BB+a^T J_AB b) - c0), per call
  float* dC32;         // [256][256] d C / d beta
  uint16_t* C16;       // same in bf16
  double* c0;          // [1] log offset, written with C
  double c_hat;        // sum_{i<j in R} |J_ij| (c0 = beta * c_hat)
  const int* eRR;      // [16][16] edge ids (-1 none)
  const int* eRW;      // [16][D] edge ids (-1 none)
};

// General components: elimination programs (see k_general.cu).
struct GenDev {
  int n_comp;
  // Compiled elimination program (built by the host planner from its packed
  // per-component programs).  Per component c, at fhdr[c]:
  //   n_steps, final table (live offset), final table (full offset);
  // per step (global step index g, record at fstep[g]):
  //   m, fld_begin, fld_count, n_in, n_pair, pp_off, map_off, out_live, out_full,
  //   n_in x (in_live, in_full, k_in), n_pair x (pair_id, pos_u).
  // map[map_off + i * 2^(m+1) + ext]: entry of input i at extended index ext
  // (bit j of ext: out-scope spin j, bit m: the eliminated spin); then
  // map[map_off + (n_in + i) * 2^(m+1) + e * 2^(m+1-k_in) + f]: the f-th
  // extended index that reads entry e of input i (the inverse map).
  // pp[pp_off + ext]: product of the step's bond factors at ext (this
  // call's beta, general_pp_kernel); pp[n_pp + pp_off + ext] its d ln / d beta.
  const int* fprog;
  const int* fhdr;
  const int* fstep;
  const unsigned short* map;
  float* pp;
  int n_pp;
  int n_steps;           // steps of all components
  const float* pairJ;    // couplings of R-R bonds referenced by the program
  const int* pairE;      // edge id of each pair
  const int* comp_step0; // [n_comp + 1] first step index of each component
  const int* fld;        // per R spin: W-neighbour list (pos, edge id) packed
  const float* fldJ;
  double c_hat;          // constant log-offset / beta
  // components with at most TNVAN_TAB_MAX_K width-set neighbours can be
  // tabulated: log Z_c (and d/dbeta) over every boundary configuration
  const int* ctab;       // [n_comp][5]: program header, program end, k, boundary list offset,
                         // table offset (-1: not tabulated)
  const int* bpos;       // boundary lists (AR positions of the W neighbours), bit j of the index = spin j
  const int* tabc;       // the tabulated components
  int n_tabc;
  int n_tab;             // entries of all tables (sum of 2^k)
  double* tab_lz;        // [n_tab] log Z_c at the current call's beta (general_tab_kernel)
  double* tab_db;        // [n_tab] its beta-derivative
};
#define TNVAN_TAB_MAX_K 12

struct InstDev {
  int kind;  // 0 strips, 1 dense, 2 general
  int n_spins, n_edges, D;
  long long spin_units;  // sum_{j<k} D_j : spins offset = batch * spin_units
  long long edge_off;    // sum_{j<k} n_edges_j
  MadeDev made;
  int n_ww;
  const EdgeWW* ww;
  // strips
  int n_strips;
  const StripDev* strips;
  const StripRow* rows;
  const float* edge_sign;  // gauge sign per edge (see HostStripPlan)
  float* adj_tab;          // the adjoint's strip tables for the current beta (strips_tab_kernel)
  int strip_tab_floats;  // shared-memory floats for all strip tables
  // dense
  DenseDev dense;
  // general
  GenDev gen;
  // wide lattice strips of an elimination instance (forward log Z_R only;
  // n_wide = 0: none)
  int n_wide;
  const WideStripDev* wide;
  const WideRow* wrows;
};

// Per-launch parameters passed by value.
struct LaunchInfo {
  int n_inst;
  int batch;
  int tile;  // samples per CTA
  int blk0;  // launch-wide block offset: a launch may cover a sub-range of the blocks
  unsigned long long seed, step;
  int* status;  // device status word: nonzero after a bounded wait gave up
  const unsigned long long* step_dev;  // optional device step counter added to `step`
  const float* wmul;  // optional per-sample multipliers [n_inst * batch] of the adjoint's bond sums
  int gen_tab;        // elimination instances: > 0 = build and use the component tables (the largest n_tab)
  int tile_aux;       // wide-strip launches: the most strips of an instance (shared-memory rows)
  double beta[TNVAN_MAX_INST];
  int tile_begin[TNVAN_MAX_INST + 1];
  unsigned int skip[TNVAN_MAX_INST / 32];  // per-instance bits: 1 = a kernel that reads them leaves the instance out
};

// Block order of a grouped-sampler launch: the instances of the launch's
// range, longest width set first (a CTA's time grows with D), so that the
// longest CTAs start first.  Blocks [begin[j], begin[j + 1]) draw the tiles
// of instance inst[j]; n = 0 keeps the LaunchInfo order.
struct TcgOrder {
  int n;
  int inst[TNVAN_MAX_INST];
  int begin[TNVAN_MAX_INST + 1];
};

// ---------------------------------------------------------------------------
// Host-side instance state.
// ---------------------------------------------------------------------------
struct HostStripPlan {
  std::vector<StripDev> strips;
  std::vector<StripRow> rows;
  // Per edge, the gauge sign that maps an expectation of the strip rows (all
  // vertical bonds made ferromagnetic by flipping spins) back to the model's
  // variables: tau_i tau_j for R-R bonds, tau_r for R-W bonds, 1 for W-W.
  std::vector<float> edge_sign;
};

struct HostWidePlan {
  std::vector<WideStripDev> strips;
  std::vector<WideRow> rows;
};

struct Instance {
  bool has_graph = false, has_ws = false, has_made = false;
  int n = 0, m = 0, topology = 0, Lx = 0, Ly = 0;
  std::vector<int> ei, ej;
  std::vector<double> J;
  std::vector<int> W;   // AR order
  int kind = -1;
  // plan summary
  int n_comp = 0, max_comp = 0, max_width = 0;
  std::vector<EdgeWW> ww;
  HostStripPlan strip;
  HostWidePlan wide;  // lattice instances planned for elimination whose R is strips of <= 12 columns
  // dense
  int dense_nR = 0;
  std::vector<float> JRW, JRR;
  std::vector<int> eRR, eRW;
  double dense_chat = 0;
  // general
  std::vector<int> gprog, gprog_fwd, gfld, gpairE, gstep_off, gcomp_step0;
  std::vector<int> gfprog, gfhdr, gfstep;  // compiled step records (GenDev::fprog)
  std::vector<unsigned short> gmap;       // input index maps (GenDev::map)
  int g_npp = 0;
  double g_mean_entries = 1;  // mean table size (entries) of the elimination steps
  int g_max_steps = 0;
  std::vector<int> gctab, gbpos, gtabc;  // component tables (GenDev)
  int g_ntab = 0;
  std::vector<float> gpairJ, gfldJ;
  int g_ncomp = 0, g_max_entries = 0, g_max_live = 0, g_npairs = 0;
  double g_chat = 0;
  // network
  int nh = 0, H[2] = {0, 0};
  float* d_params = nullptr;
  long long n_params = 0;
  // device allocations owned by this instance
  std::vector<void*> dev_allocs;
  InstDev dev{};
};

}  // namespace tnvan

struct tnvan_prof_rec {
  std::string name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double total_ms = 0;
  long long launches = 0;
};

struct tnvan_ctx {
  int device = 0;
  const unsigned long long* step_dev = nullptr;  // tnvan_set_step_counter
  // autotuned launch shapes (0 = built-in heuristic)
  int tune_sample_tile = 0, tune_strip_tile = 0, tune_bwd_ctas = 0, tune_adj_tile = 0;
  int tune_tc_plan = -1;  // tensor-core sampler step-group plan (-1 = default)
  int tune_tc_form = 0;   // tensor-core sampler form: 0 automatic, 1 grouped, 2 per-step
  int tune_bwd_form = 0;  // backward without the fused kernel, BF16/TF32: 0/1 tensor-core GEMM chain, 2 FP32 SIMT
  int tune_overlap = 1;   // overlapped sampling + adjoint schedule (1 on, 0 off)
  // last strip-adjoint launch plan (valid while batch, tuning and instances are unchanged)
  struct {
    int valid = 0, batch = 0, tune = 0, tile = 0, smem = 0, lv = 0, ws = 0;
  } adj_plan;
  // side streams and events of the overlapped sampling + adjoint schedule
  cudaStream_t side[8] = {};  // samplers (highest stream priority)
  cudaStream_t side_lo[8] = {};  // adjoints (default priority)
  cudaEvent_t fork_ev = nullptr, join_ev[8] = {}, chunk_ev[8] = {}, adj_ev[8] = {}, dj_ev = nullptr;
  bool prof_on = false;
  std::vector<tnvan_prof_rec> prof;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t prof_ref = nullptr;  // recorded before the first launch of a profiled region (trace origin)
  bool prof_ref_set = false;
  std::string err;
  std::vector<tnvan::Instance> inst;
  tnvan::InstDev* d_inst = nullptr;  // device copy of the descriptors
  int d_inst_cap = 0;
  bool dirty = true;                 // descriptors changed since last upload
  // workspaces (grown on demand, or by tnvan_reserve)
  double* d_stats = nullptr;         // [n_inst][8] + partial tuples (training path)
  double* d_stats_fe = nullptr;      // the same for tnvan_free_energy (inside d_stats' allocation)
  int* d_status = nullptr;           // [4] device status words, then [TNVAN_MAX_INST] reduction counters
  size_t ws_bytes = 0;
  void* d_ws = nullptr;              // general workspace
  int reserved_batch = 0;
  float* d_grad_packed = nullptr;    // packed-layout gradient partials
  size_t grad_packed_floats = 0;
  float* d_dj_part = nullptr;        // d/dJ partial rows [CTA][max edges]
  size_t dj_part_floats = 0;
  float* d_gen_scratch[2] = {nullptr, nullptr};  // global elimination tables: forward, reverse sweep
  size_t gen_scratch_floats[2] = {0, 0};
  double* d_wide_part = nullptr;  // per-strip log Z of the wide-strip kernels
  size_t wide_part_n = 0;
  void* d_obs = nullptr;             // tnvan_observables: weights, d/dbeta, sums
  size_t obs_bytes = 0;
};

namespace tnvan {

// Kernel launchers (defined in the .cu files).  All return a cudaError_t.
enum { PACK_FLAT = 1, PACK_TILES = 2, PACK_SIMT = 4, PACK_TC = 8, PACK_TCG = 16 };
__host__ __device__ long long pack_elems(const MadeDev& md, int mask);
cudaError_t launch_pack_all(const InstDev* d_inst, int n_inst, const long long* counts, int mask, cudaStream_t s);
cudaError_t launch_sample(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                          int8_t* spins, float* logq, const int8_t* given, cudaStream_t s);
cudaError_t launch_strips(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                          const int8_t* spins, double* logZR, double* dbeta, cudaStream_t s);
cudaError_t launch_strips_adj(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int lv_floats,
                              const int8_t* spins, double* logZR, double* dbeta, float* part, int part_stride,
                              double* dJ, cudaStream_t s, int blk_begin = 0, int blk_end = -1, int ws_threads = 0);
cudaError_t launch_strips_dJ_reduce(const InstDev* d_inst, const LaunchInfo& li, const float* part, int part_stride,
                                    double* dJ, cudaStream_t s, bool assign);
cudaError_t launch_dense(const InstDev* d_inst, const LaunchInfo& li, int precision,
                         const int8_t* spins, double* logZR, double* dbeta, double* dJ,
                         cudaStream_t s, int max_D = 1024);
// Elimination kernels keep their tables in shared memory, or (garena
// non-NULL: arenas too large for 32 samples per CTA) in a global scratch
// buffer of general_scratch_floats / general_dJ_scratch_floats floats.
// li.tile = samples per CTA, GL lanes per sample (li.tile * GL threads, a
// multiple of 32).
cudaError_t launch_general(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int GL,
                           const int8_t* spins, double* logZR, double* dbeta, float* garena,
                           cudaStream_t s);
cudaError_t launch_general_dJ(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int arena, int steps,
                              int gmax, int GL, const int8_t* spins, float* part, int part_stride, double* dJ,
                              float* garena, cudaStream_t s);
// bond products of every elimination step at li.beta (before the kernels above)
cudaError_t launch_general_pp(const InstDev* d_inst, const LaunchInfo& li, int max_steps, cudaStream_t s);
int general_dJ_smem_bytes(int per_sample, int D, int n_edges, int T, int GL, bool glob);
size_t general_dJ_scratch_floats(int per_sample, int T, int GL, int nblk);
size_t general_scratch_floats(const LaunchInfo& li, int arena, int GL, bool db);
cudaError_t launch_ww(const InstDev* d_inst, const LaunchInfo& li, const int8_t* spins,
                      double* dJ, cudaStream_t s);
// The strip adjoint's tables (Boltzmann factors of every strip row at the
// launch's betas) of instances [k0, k1), into each instance's adj_tab; the
// adjoint kernels copy them instead of building them per CTA.
cudaError_t launch_strip_tables(const InstDev* d_inst, const LaunchInfo& li, int k0, int k1, cudaStream_t s);
// tnvan_observables: energies = false writes the importance-weight
// multipliers B w_b into wmul (from the statistics' logZ_IS); energies = true
// reduces dbeta and wmul to out[3k..3k+2] = U, U_q, effective sample size.
cudaError_t launch_observables(const LaunchInfo& li, const double* logZR, const float* logq, const double* stats,
                               const double* dbeta, float* wmul, double* out, bool energies, cudaStream_t s);
// Wide strips (k_wide.cu): log Z_R of the elimination instances that carry a
// wide-strip plan (li: one tile per sample of the instances to run, zero
// tiles for the others), one CTA per sample, one launch per class of states
// per lane (strips_per_class[c]: the most strips of 2^c states per lane in
// one instance, c = 0 for strips of <= 5 columns), per-strip results in
// part [n_inst][batch][max_strips], then their sum in strip order.
cudaError_t launch_wide(const InstDev* d_inst, const LaunchInfo& li, const int* strips_per_class, int max_strips,
                        int max_D, const int8_t* spins, double* part, double* logZR, cudaStream_t s);
// Magnetisation moments (tnvan_magnetisation): per sample E[M | s] and
// Var(M | s) of the whole system's magnetisation given the width set, by
// contraction kind (strips: li.tile samples per CTA, smem as strip_smem_bytes;
// dense: builds the block's table at li.beta; elimination: as launch_general,
// tables x 3, garena of general_mom_scratch_floats when too large).
cudaError_t launch_strips_mom(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, const int8_t* spins,
                              double* mag_mean, double* mag_var, cudaStream_t s);
cudaError_t launch_dense_mom(const InstDev* d_inst, const LaunchInfo& li, int max_D, const int8_t* spins,
                             double* mag_mean, double* mag_var, cudaStream_t s);
int general_mom_smem_bytes(int arena, int D, int T, int GL, bool glob);
size_t general_mom_scratch_floats(const LaunchInfo& li, int arena, int GL);
cudaError_t launch_general_mom(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, int arena, int GL,
                               const int8_t* spins, double* mag_mean, double* mag_var, float* garena,
                               cudaStream_t s);
// out[5k + 0..4] = <M>, <M^2> (importance-weighted), the same under q, and
// the effective sample size, from the moments and the multipliers B w_b.
cudaError_t launch_obs_mag(const LaunchInfo& li, const double* mean, const double* var, const float* wmul,
                           double* out, cudaStream_t s);
// Eq. 9 statistics of instances [k0, k1) (k1 < 0: all) of the launch into
// stats[8k + 0..7] = F_q, F_IS, stderr, logZ_IS, mean l, #non-finite, var l,
// n (the backward's baseline is [4], its sample count [5] + [7]).
cudaError_t launch_reduce(const InstDev* d_inst, const LaunchInfo& li, const double* logZR,
                          const float* logq, double* stats, int* counters, cudaStream_t s, int k0 = 0,
                          int k1 = -1);
// Statistics rows of n_parts disjoint parts of a batch ([n_parts][n_inst][8])
// merged into stats[8k + 0..7] for their union (fixed order).
cudaError_t launch_merge_stats(const LaunchInfo& li, int n_parts, const double* parts, double* stats,
                               cudaStream_t s);
cudaError_t launch_backward(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                            int precision, const int8_t* spins, const double* logZR,
                            const float* logq, const double* stats, float* partials,
                            int part_stride, cudaStream_t s);
// Adam's state and hyper-parameters for one launch (moments in the packed
// all-instances gradient layout).  With t_dev the step is t_base + *t_dev and
// bc1/bc2 are formed on the device.
struct AdamArgs {
  float* m;
  float* v;
  float lr, b1, b2, eps, bc1, bc2;
  const unsigned long long* t_dev;
  long long t_base;
};
// With adam non-NULL the reduction also applies Adam to every instance's own
// parameters (the fused optimizer step of tnvan_train_step).
cudaError_t launch_grad_reduce(const InstDev* d_inst, const LaunchInfo& li,
                               const float* partials, int part_stride, float* grad,
                               cudaStream_t s, const AdamArgs* adam = nullptr, int k0 = 0, int k1 = -1);
// s16 != nullptr: also the spins as BF16 rows of r8(D) (the GEMM chain's operand)
cudaError_t launch_reinforce_w(const InstDev* d_inst, const LaunchInfo& li, const double* logZR, const float* logq,
                               const double* stats, float* w, const int8_t* spins, uint16_t* s16, cudaStream_t s);
cudaError_t launch_bwd_fused(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes,
                             const int8_t* spins, const double* logZR, const float* logq,
                             const double* stats, float* partials, long long part_stride, int* status,
                             cudaStream_t s, int blk_begin = 0, int blk_end = -1);
int fused_bwd_smem_bytes(int D, int H1, int H2);
cudaError_t launch_sample_tc(const InstDev* d_inst, const LaunchInfo& li, int plan, int nh, int smem_bytes,
                             int8_t* spins, float* logq, const int8_t* given, cudaStream_t s, int blk_begin = 0,
                             int blk_end = -1);
int sample_tc_smem_bytes(const MadeDev& md, int plan);
extern const int kTcGroupMax[TNVAN_TC_PLANS];
// streamed: some instance of the launch streams its weights (plan `plan`).
cudaError_t launch_sample_tcg(const InstDev* d_inst, const LaunchInfo& li, const TcgOrder& ord, int plan,
                              int smem_bytes, bool streamed, int8_t* spins, float* logq, const int8_t* given,
                              cudaStream_t s, int blk_begin = 0, int blk_end = -1);
int sample_tcg_smem_bytes(int D, int H1, int H2, int tcw1, int tcw2, int twmax, int wbmax = 0);
extern const int kTcGroupMaxG[TNVAN_TC_PLANS];
cudaError_t launch_adam(long long n, float* p, const float* g, const AdamArgs& a, cudaStream_t s);

int sample_smem_bytes(const Instance& in, int tile);
int general_smem_bytes(int arena, int D, int T, int GL, bool db, bool glob);
cudaError_t launch_general_tables(const InstDev* d_inst, const LaunchInfo& li, int smem_bytes, bool db, int GL,
                                  float* garena, cudaStream_t s);
int strip_smem_bytes(const Instance& in, int tile);
int strip_adj_smem_bytes(const Instance& in, int tile, int lv_floats);
int strip_adj_lv_floats(const Instance& in, int tile);
int strips_adj_occupancy(int tile, int smem_bytes);
int strip_adj_ws_threads(const tnvan_ctx* ctx);
int strip_adj_ws_lv_floats(const Instance& in, int threads);
int strip_adj_ws_smem_bytes(const Instance& in, int threads, int lv_floats);
int strips_adj_ws_occupancy(int threads, int smem_bytes);

}  // namespace tnvan
