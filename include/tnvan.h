/*
 * tnvan.h -- C-ABI of the GB300 (sm_103a) TNVAN hot path.
 *
 * TNVAN (tensor-network-based variational autoregressive networks, arXiv
 * 2504.12037) splits the spins into a width set W and a remainder R (Sec. 2).
 * For every configuration s of W drawn from an autoregressive network q_theta
 * (Eq. 6-8) it contracts R exactly, giving the effective energy Etilde(s)
 * (Eq. 3-4), and reduces the batch to the variational free energy F_q (Eq. 9)
 * and its score-function gradient (Eq. 10).  This library runs those steps on
 * one GPU.
 *
 * Conventions shared by every call
 *   - Return value: TNVAN_OK (0) or a negative TNVAN_E_* code.  No exception,
 *     abort or exit crosses this boundary; the message of the last failure on a
 *     context is returned by tnvan_last_error().
 *   - "host" pointers are read during the call and copied; the caller keeps
 *     ownership.  "device" pointers are borrowed: they must stay valid until the
 *     work queued on `stream` has finished.  `stream` is a cudaStream_t (NULL =
 *     the legacy default stream).
 *   - Calls that launch work are asynchronous on `stream` unless stated.
 *   - Instances: a context holds instances 0..n-1 (graph + width set +
 *     network), registered in order.  Batched calls process all of them in one
 *     launch per stage.  For instance k with D_k width-set spins, per-sample
 *     outputs sit at:   spins  byte offset  batch * sum_{j<k} D_j, layout [batch][D_k]
 *                       logq / logZR / dbeta  element offset  k * batch.
 *   - Per-sample quantity: log Z_R(s) := -beta * Etilde(s)
 *       = -beta E_1(s) + ln sum_{r in R} exp(-beta E_2(s, r))     (Eq. 4)
 *     i.e. it includes the W-W energy E_1.  Energies follow Eq. 1:
 *     E(s) = - sum_<ij> J_ij s_i s_j.
 *   - Spins are int8 values +1 / -1.
 *   - Not thread-safe: one host thread drives a context at a time.
 */
#ifndef TNVAN_H
#define TNVAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define TNVAN_OK 0
#define TNVAN_E_ARG (-1)          /* invalid argument or inconsistent sizes        */
#define TNVAN_E_NOMEM (-2)        /* device or host allocation failed              */
#define TNVAN_E_CUDA (-3)         /* a CUDA runtime call or kernel launch failed   */
#define TNVAN_E_TIMEOUT (-4)      /* a bounded device wait gave up                 */
#define TNVAN_E_OVERFLOW (-5)     /* a non-finite value reached a reduction        */
#define TNVAN_E_STATE (-6)        /* call out of order (e.g. no graph yet)         */
#define TNVAN_E_UNSUPPORTED (-7)  /* shape outside what the kernels implement      */

/* Graph topologies (how the remainder R is contracted). */
#define TNVAN_LATTICE2D 0  /* Lx x Ly open lattice, spin = y*Lx + x; W = whole columns -> strips */
#define TNVAN_DENSE 1      /* fully connected; |R| <= 16 summed as a dense block              */
#define TNVAN_GENERAL 2    /* any graph; R components contracted by variable elimination       */

/* Arithmetic modes for the contractions and network GEMMs. */
#define TNVAN_FP32 0 /* FP32 everywhere (FP64 only for final log-norms and reductions)   */
#define TNVAN_TF32 1 /* TF32 tensor-core GEMMs, FP32 accumulate                         */
#define TNVAN_BF16 2 /* BF16 tensor-core GEMMs / dense block, FP32 accumulate           */

typedef struct tnvan_ctx tnvan_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int tnvan_version(void);

/* Create a context bound to CUDA device `device`.  *out receives the handle.
 * Errors: TNVAN_E_ARG (out NULL), TNVAN_E_CUDA (bad device). */
int tnvan_create(tnvan_ctx** out, int device);

/* Release every device buffer the context owns.  Borrowed pointers are not
 * touched.  Synchronises the device first.  NULL is accepted (no-op). */
int tnvan_destroy(tnvan_ctx* ctx);

/* Message of the last failed call on `ctx` ("" if none); for ctx == NULL the
 * last failure of tnvan_create on this thread.  Valid until the next call. */
const char* tnvan_last_error(const tnvan_ctx* ctx);

/* Define instance `instance` (must be 0..n, n = current count; n appends).
 * Sec. 2, Eq. 1-2: the Ising graph TN({B},{s}).
 *   n_spins, n_edges   sizes; edges are undirected, (ei[k], ej[k]) with
 *                      0 <= ei, ej < n_spins, ei != ej, no repeated pair.
 *   ei, ej, J          host arrays [n_edges] (copied).
 *   topology           TNVAN_LATTICE2D | TNVAN_DENSE | TNVAN_GENERAL.
 *   Lx, Ly, periodic   lattice shape (LATTICE2D only; periodic must be 0).
 * Redefining an instance drops its width set and network.
 * Errors: TNVAN_E_ARG, TNVAN_E_UNSUPPORTED (periodic lattice). */
int tnvan_init_graph(tnvan_ctx* ctx, int instance, int n_spins, int n_edges, const int32_t* ei,
                     const int32_t* ej, const double* J, int topology, int Lx, int Ly,
                     int periodic);

/* Set the width set W of `instance` (Sec. 2; Algorithm 1 step 1 takes it as
 * given).  w: host array [n_w] of distinct spin indices in autoregressive
 * order (Eq. 6's "predetermined order").  The host planner then builds the
 * contraction plan of R: lattice strips (W must then be whole columns),
 * a dense block (|R| <= 16), or per-component elimination programs
 * (elimination width <= 12).  Plans are independent of beta.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE (no graph), TNVAN_E_UNSUPPORTED. */
int tnvan_set_width_set(tnvan_ctx* ctx, int instance, int n_w, const int32_t* w);

/* As tnvan_set_width_set, with the elimination order of R given for GENERAL
 * instances (e.g. the order tnvan_find_width_set returns): r_order is a host
 * array [n_spins - n_w] listing every spin not in W exactly once; each
 * component is eliminated in the order its spins appear there (instead of
 * the planner's min-fill order).  r_order == NULL is tnvan_set_width_set.
 * Errors: as tnvan_set_width_set; TNVAN_E_ARG when r_order is not a
 * permutation of R, or is given for a LATTICE2D / DENSE plan;
 * TNVAN_E_UNSUPPORTED when the order needs elimination width > 12. */
int tnvan_set_width_set_ordered(tnvan_ctx* ctx, int instance, int n_w, const int32_t* w,
                                const int32_t* r_order);

/* Width-set finder (Sec. 2: a contraction order is searched, then spins are
 * sliced out of it -- "dynamic slicing" -- until the remaining network has
 * width <= w_u, and sliced spins are returned to R one at a time in random
 * order while the width stays <= w_u).  Width: eliminating a spin of R
 * creates a factor over its neighbours at that point (fill edges included);
 * the width of an order is the largest such factor.  w_u = 1 leaves a
 * forest, i.e. W is a feedback vertex set; the GPU elimination kernels accept
 * w_u <= 12.  Host only (no device work, no context, callable without a GPU).
 *   n_spins <= TNVAN_FIND_MAX_N; edges as in tnvan_init_graph.
 *   w_u        width bound (>= 0).
 *   restarts   number of randomised trials per search (>= 1);
 *   seed       seed of the trials' tie-breaking.
 *   mode       TNVAN_SLICE_FIXED: min-fill order of the whole graph, then
 *              slicing along it (the spin in the most maximum-width factors
 *              first); TNVAN_SLICE_GREEDY: order and slicing built together
 *              (eliminate the least-fill spin of degree <= w_u, else slice the
 *              spin of largest degree); TNVAN_SLICE_BEST: both, smaller W wins.
 *   anneal_iters  >= 0: moves of simulated annealing applied to the winner
 *              (one sliced spin returns to R, a greedy elimination with
 *              slicing repairs the width, Metropolis acceptance on |W| under a
 *              linearly falling temperature from 0.5; the smallest feasible
 *              set is kept); 0 = none.
 *   out_w      [n_spins] receives W (slicing order, or for annealed sets the
 *              order in which spins entered W; use it as the
 *              autoregressive order);
 *   out_order  [n_spins] receives R's elimination order (n_spins - n_w
 *              entries; pass it to tnvan_set_width_set_ordered);
 *   out_info   [3] receives n_w, the order's width, and the winning trial
 *              of the searches (2 * restart + (search == GREEDY)).
 * Deterministic for a given seed (integer arithmetic only).
 * Errors: TNVAN_E_ARG. */
#define TNVAN_FIND_MAX_N 16384
#define TNVAN_SLICE_FIXED 1
#define TNVAN_SLICE_GREEDY 2
#define TNVAN_SLICE_BEST 3
int tnvan_find_width_set(int n_spins, int n_edges, const int32_t* ei, const int32_t* ej, int w_u,
                         int restarts, uint64_t seed, int mode, int anneal_iters, int32_t* out_w,
                         int32_t* out_order, int32_t* out_info);

/* Attach the MADE network of `instance` (Eq. 7, Fig. 1(d)): D = n_w inputs and
 * outputs, n_hidden (0..2) ReLU hidden layers of widths[0..n_hidden-1]
 * (each <= 512).  d_params: borrowed device pointer to float32 parameters,
 * layer by layer W_l [out][in] row-major then b_l [out]; entries outside the
 * MADE masks are ignored (hidden unit k has degree (k mod max(D-1,1)) + 1,
 * input/output i has degree i+1).  Count with tnvan_n_params().
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE (no width set), TNVAN_E_NOMEM. */
int tnvan_set_made(tnvan_ctx* ctx, int instance, int n_hidden, const int32_t* widths,
                   float* d_params);

/* Number of float32 parameters of instance's network (after set_made), and
 * the offset of that instance in the packed all-instances gradient layout
 * used by tnvan_backward / tnvan_adam (sum of n_params of lower instances). */
int tnvan_n_params(const tnvan_ctx* ctx, int instance, int64_t* n_params, int64_t* offset);

/* Plan summary of `instance`: info[0] n_spins, [1] n_edges, [2] n_w (D),
 * [3] contraction kind (0 strips, 1 dense, 2 general), [4] number of R
 * components, [5] largest component (spins), [6] largest elimination width,
 * [7] number of W-W edges, [8] per-sample table arena of elimination plans
 * (floats, every table kept: reverse sweeps), [9] the same with consumed
 * tables' space reused (forward passes), [10] the grouped BF16 sampler's
 * in-group form (-1 not eligible or no network, 0 per unit, 2-4 slots per
 * layer and step: the register form), [11] 1 if the fused BF16 backward takes
 * the instance, [12] 1 if the grouped sampler streams the instance's weights
 * per step group (width sets of 129 to 256 spins, or tiles too large to stay
 * in shared memory), 0 if they stay resident, -1 not eligible.  info: host
 * array [13]. */
int tnvan_instance_info(const tnvan_ctx* ctx, int instance, int32_t* info);

/* Pre-allocate the context's internal workspaces for batches up to
 * max_batch so that later calls allocate nothing (needed before capturing
 * calls into a CUDA graph).  Synchronous. */
int tnvan_reserve(tnvan_ctx* ctx, int max_batch);

/* Algorithm 1 steps (a)-(b) for every instance, in one pass on `stream`:
 * ancestral sampling from q_theta (Eq. 8: s_i = +1 iff u < sigmoid(x_i), u a
 * 24-bit uniform from Philox4x32-10 with counter (b, i>>2, step mod 2^32,
 * instance) and key (seed mod 2^32, seed >> 32), word i & 3, u = (word >> 8)
 * * 2^-24), log q (Eq. 6, 8) and the exact conditional contraction log Z_R(s)
 * (Eq. 3-4).
 *   betas     host [n_instances] inverse temperatures.
 *   batch     samples per instance (>= 0).
 *   precision TNVAN_FP32 | TNVAN_TF32 | TNVAN_BF16.  With TNVAN_BF16 the
 *             network runs on the tensor cores in BF16 (FP32 accumulate) when
 *             every instance has one or two hidden layers of <= 256 units
 *             (multiples of 16) and D <= 256 and all share one number of
 *             hidden layers; the contractions stay FP32.
 *   d_spins   device int8 out, layout above.   d_logq  device float out.
 *   d_logZR   device double out.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE (an instance lacks network or width set),
 * TNVAN_E_CUDA. */
int tnvan_sample_and_contract(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed,
                              uint64_t step, int precision, int8_t* d_spins, float* d_logq,
                              double* d_logZR, void* stream);

/* tnvan_sample_and_contract plus the contraction adjoint of tnvan_backward
 * (Eq. 4 differentiated) in the same pass: for strip instances one kernel
 * sweeps each strip forward (log Z_R, identical to tnvan_contract's) and
 * backward (d log Z_R / d beta per sample, d log Z_R / d J_e as the batch
 * mean).  A training step then calls tnvan_backward with d_dbeta and d_dJ
 * NULL.  Not a separate step of the paper: the same quantities, computed
 * together.
 *   d_dbeta   device double out [n_instances * batch], or NULL.
 *   d_dJ      device double out [sum_k n_edges_k] (instances back to back,
 *             input edge order), or NULL.
 * Other arguments and errors as tnvan_sample_and_contract; TNVAN_E_UNSUPPORTED
 * if a strip's left vectors do not fit in shared memory. */
int tnvan_sample_contract_adjoint(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed,
                                  uint64_t step, int precision, int8_t* d_spins, float* d_logq,
                                  double* d_logZR, double* d_dbeta, double* d_dJ, void* stream);

/* Eq. 6 and 8 alone: log q_theta(s) for caller-given width-set
 * configurations d_spins (device int8 +-1, layout above), by the same
 * masked forward the sampler of that precision runs (teacher forcing).
 * d_logq: device float [n_inst * batch] out.  Asynchronous.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE (no network), TNVAN_E_CUDA. */
int tnvan_log_prob(tnvan_ctx* ctx, int batch, const int8_t* d_spins, int precision, float* d_logq,
                   void* stream);

/* Eq. 3-4 alone: log Z_R(s) for caller-given width-set configurations
 * d_spins (device int8, layout above) of every instance.  Optional
 * d_dlogZR_dbeta (device double [n_inst*batch], may be NULL) receives
 * d log Z_R / d beta = -E_1(s) - <E_2(s, r)>_{r|s}.  For elimination
 * instances, leftover components with at most 12 width-set neighbours are
 * tabulated over their boundary configurations at the call's beta when the
 * tables (sum of 2^k entries) are no larger than the batch, and looked up per
 * sample (the same values up to FP64 rounding).  Asynchronous. */
int tnvan_contract(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                   int precision, double* d_logZR, double* d_dlogZR_dbeta, void* stream);

/* Eq. 9 and the importance-sampled log Z over each instance's batch, with
 * l_b = log Z_R(s_b) - log q(s_b):
 *   h_out[4k+0] F_q      = -(1/beta) mean_b l_b
 *   h_out[4k+1] F_IS     = -(1/beta) (logsumexp_b l_b - ln batch)
 *   h_out[4k+2] stderr   = std_b(l_b) / (beta sqrt(batch))   (ddof 1)
 *   h_out[4k+3] logZ_IS  =  logsumexp_b l_b - ln batch
 * reduced in FP64 on the device.  h_out: host double [4 * n_instances].
 * Synchronises `stream`.  The reduction has a workspace of its own, so the
 * call may run on one stream while a training step of the same context runs
 * on another (e.g. the statistics of step i beside step i + 1, on separate
 * output buffers); two tnvan_free_energy calls on one context must not
 * overlap.  Errors: TNVAN_E_ARG (batch < 1), TNVAN_E_OVERFLOW (a non-finite
 * l_b), TNVAN_E_CUDA. */
int tnvan_free_energy(tnvan_ctx* ctx, const double* betas, int batch, const double* d_logZR,
                      const float* d_logq, double* h_out, void* stream);

/* Eq. 9 statistics of each instance's batch, asynchronous on `stream` (the
 * device-side counterpart of tnvan_free_energy, capturable in a CUDA graph):
 * with l_b = log Z_R(s_b) - log q(s_b), one statistics row per instance,
 *   row[0] F_q = -(1/beta) mean l,   row[1] F_IS = -(1/beta) logZ_IS,
 *   row[2] stderr = std(l) / (beta sqrt(n)) (ddof 1),
 *   row[3] logZ_IS = logsumexp l - ln n,   row[4] mean l,
 *   row[5] number of non-finite l_b (left out of every other entry),
 *   row[6] var l (ddof 1),   row[7] n = number of finite l_b.
 * The rows become the context's step statistics: the baseline (row[4]) and
 * sample count (row[5] + row[7]) of the next tnvan_backward_stats.
 *   d_stats_out  device double [8 * n_inst] (row k at 8k), or NULL.
 * Errors: TNVAN_E_ARG (batch < 1, NULL input), TNVAN_E_STATE, TNVAN_E_CUDA. */
int tnvan_reduce(tnvan_ctx* ctx, const double* betas, int batch, const double* d_logZR, const float* d_logq,
                 double* d_stats_out, void* stream);

/* The step statistics of the context (rows as tnvan_reduce) -- written by the
 * last tnvan_train_step, tnvan_reduce or tnvan_merge_stats queued on the
 * context -- copied to d_stats_out (device double [8 * n_inst]),
 * asynchronously on `stream`.  Eq. 9 for the batch a training step drew.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE (no instances), TNVAN_E_CUDA. */
int tnvan_step_stats(tnvan_ctx* ctx, double* d_stats_out, void* stream);

/* Data-parallel exchange (not in the paper; the samples of one batch split
 * over ranks, one exchange of statistics per step): merges the statistics rows of
 * n_parts disjoint parts of a batch, d_parts = device double
 * [n_parts][n_inst][8] (each part's tnvan_reduce rows, e.g. gathered from
 * every rank), into the rows of their union, in part order: counts add,
 * means and the second central moments by the pairwise update of Chan,
 * Golub and LeVeque, log sum e^l by logaddexp.  The result becomes the
 * context's step statistics (so tnvan_backward_stats then uses the global
 * baseline and batch size) and goes to d_stats_out (device double
 * [8 * n_inst]) unless NULL.  One part is copied unchanged.  Asynchronous.
 * Errors: TNVAN_E_ARG (n_parts < 1, NULL d_parts), TNVAN_E_STATE, TNVAN_E_CUDA. */
int tnvan_merge_stats(tnvan_ctx* ctx, const double* betas, int n_parts, const double* d_parts, double* d_stats_out,
                      void* stream);

/* Eq. 10 on this process's samples with the baseline and batch size of the
 * context's step statistics (tnvan_reduce or tnvan_merge_stats):
 *   grad = sum_{b local} -(l_b - mean) / (beta B) grad_theta log q(s_b),
 * mean = row[4], B = row[5] + row[7].  With merged statistics, summing grad
 * over the ranks (an all-reduce) gives tnvan_backward's gradient of the union
 * batch; with this process's own statistics it is tnvan_backward's gradient.
 * Arguments as tnvan_backward without the contraction adjoint.
 * Asynchronous.  Errors: TNVAN_E_ARG, TNVAN_E_STATE, TNVAN_E_CUDA. */
int tnvan_backward_stats(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                         const double* d_logZR, const float* d_logq, int precision, float* d_grad_params,
                         void* stream);

/* Observables from one batch (the paper notes that samples of the trained
 * network give magnetisation, correlations and susceptibility, Sec. 3, and
 * leaves correlation functions to future work, Sec. 4): with the
 * self-normalised importance weights w_b = exp(l_b) / sum_b' exp(l_b'),
 * l_b = log Z_R(s_b) - log q(s_b), which make averages over q estimates of
 * Boltzmann averages, and the exact conditional energy of each sample,
 * E_b = -d log Z_R(s_b) / d beta = E_1(s_b) + <E_2>_{r|s_b} (Eq. 4):
 *   h_out[3k+0] U    = sum_b w_b E_b   (internal energy, importance-weighted)
 *   h_out[3k+1] U_q  = mean_b E_b      (the same under q)
 *   h_out[3k+2] ESS  = 1 / sum_b w_b^2 (effective sample size of the weights)
 *   d_corr          device double [sum_k n_edges_k] out, or NULL: per edge
 *                   sum_b w_b d log Z_R(s_b) / d J_e = beta sum_b w_b <s_i s_j>_{r|s_b}
 *                   (instances back to back, input edge order); divide by
 *                   beta for the bond correlation.  Every contraction kind.
 * h_out: host double [3 * n_instances].  FP32 contraction.  Uses the
 * reduction workspace of tnvan_free_energy (do not overlap the two) and
 * allocates a workspace of its own on growth.  Synchronises `stream`.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE, TNVAN_E_NOMEM, TNVAN_E_CUDA. */
int tnvan_observables(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                      const double* d_logZR, const float* d_logq, double* d_corr, double* h_out,
                      void* stream);

/* Magnetisation and susceptibility from samples (Sec. 3: with the trained
 * network, samples give magnetisation and susceptibility).  For each sample
 * the exact conditional moments of the total magnetisation M = sum_i s_i
 * given its width-set spins,
 *   mu_b = E[M | s_b] = M_W(s_b) + <M_R>_{r|s_b},   v_b = Var(M | s_b) = Var(M_R | s_b),
 * by each contraction kind carried in moment form (every partial sum keeps its
 * weight, the conditional mean and the conditional variance of the
 * magnetisation summed into it; two branches merge by the law of total
 * variance), FP32 arithmetic with FP64 sums over strips and components.  With
 * the self-normalised importance weights w_b of tnvan_observables:
 *   h_out[6k+0] <M>    = sum_b w_b mu_b
 *   h_out[6k+1] <M^2>  = sum_b w_b (mu_b^2 + v_b)
 *   h_out[6k+2] chi    = beta (<M^2> - <M>^2) / N   (per spin)
 *   h_out[6k+3] <M>_q  = mean_b mu_b,  h_out[6k+4] <M^2>_q = mean_b (mu_b^2 + v_b)
 *   h_out[6k+5] ESS    = 1 / sum_b w_b^2
 *   d_mag_mean, d_mag_var  device double [n_inst*batch] out (mu_b, v_b), or
 *                  NULL (the context's workspace holds them).
 * h_out: host double [6 * n_instances].  Every contraction kind.  Shares the
 * workspace of tnvan_observables (do not overlap the two).  Synchronises
 * `stream`.  Errors: TNVAN_E_ARG, TNVAN_E_STATE, TNVAN_E_NOMEM,
 * TNVAN_E_UNSUPPORTED (tables beyond shared memory), TNVAN_E_CUDA. */
int tnvan_magnetisation(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                        const double* d_logZR, const float* d_logq, double* d_mag_mean, double* d_mag_var,
                        double* h_out, void* stream);

/* Eq. 10: REINFORCE gradient of F_q for every instance,
 *   grad = sum_b w_b grad_theta log q(s_b),  w_b = -(l_b - mean_b l) / (beta batch),
 * (the batch mean is the baseline; it leaves the expectation unchanged), by a
 * teacher-forced forward and hand-written backward of the network.  With
 * TNVAN_BF16, instances whose network has two hidden layers of <= 128 units
 * (multiples of 16) and a width set that fits the fused kernel's TMEM (D
 * padded to 16 as Dp; 128 + G + (H1 + 16) + (H2 + 16) <= 512 columns with
 * G = Dp when D is not a multiple of 16, else Dp + 16) and whose tiles fit
 * 227 KB of shared memory (every such width set does with H1 = H2 = 128) run
 * the fused tcgen05 backward; the other instances of the same call run the
 * tensor-core GEMM chain (TF32 / BF16 operands, FP32 accumulate) or, where the
 * autotuner found it faster, the FP32 SIMT backward.
 *   d_grad_params   device float [total params] out, packed layout of
 *                   tnvan_n_params (overwritten; masked entries are 0).
 * Contraction adjoint (optional, NULL to skip):
 *   d_dlogZR_dbeta  device double [n_inst*batch]: d log Z_R(s_b)/d beta.
 *   d_dlogZR_dJ     device double [sum_k n_edges_k] (instance k at offset
 *                   sum_{j<k} n_edges_j): (1/batch) sum_b d log Z_R(s_b)/d J_e
 *                   = beta * mean_b <s_i s_j>_{r|s_b}.
 * Asynchronous.  Errors: TNVAN_E_ARG, TNVAN_E_STATE, TNVAN_E_CUDA. */
int tnvan_backward(tnvan_ctx* ctx, const double* betas, int batch, const int8_t* d_spins,
                   const double* d_logZR, const float* d_logq, int precision,
                   float* d_grad_params, double* d_dlogZR_dbeta, double* d_dlogZR_dJ,
                   void* stream);

/* Algorithm 1 step (d) with Adam (Kingma & Ba 2015) over n float32 entries:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).  t >= 1.
 * All pointers are device float [n].  Asynchronous. */
int tnvan_adam(tnvan_ctx* ctx, int64_t n, float* d_params, const float* d_grad, float* d_m,
               float* d_v, double lr, double beta1, double beta2, double eps, int64_t t,
               void* stream);

/* One whole iteration of Algorithm 1 (a)-(d) in one call, asynchronous on
 * `stream`: tnvan_sample_contract_adjoint (tnvan_sample_and_contract when
 * d_dbeta and d_dJ are both NULL), the REINFORCE gradient of tnvan_backward
 * (Eq. 10) into d_grad_params, and Adam on every instance's own parameters
 * (the d_params pointers given to tnvan_set_made, which this call updates in
 * place).  Equal to those calls in sequence, with tnvan_adam run over the
 * packed gradient layout; here the network is packed once for the whole
 * step and the gradient reduction and Adam are one kernel.  The step's Eq. 9
 * statistics (F_q, F_IS, stderr, logZ_IS of the batch it drew; rows as
 * tnvan_reduce) are reduced inside the step; tnvan_step_stats copies them out.
 *   d_spins, d_logq, d_logZR, d_dbeta, d_dJ   as tnvan_sample_contract_adjoint.
 *   d_grad_params   device float [total params] out, layout of tnvan_n_params.
 *   d_m, d_v        device float [total params] Adam moments in that layout
 *                   (in/out).
 *   lr, beta1, beta2, eps, t   as tnvan_adam (t >= 1); with a step counter
 *                   (tnvan_set_step_counter) the Philox step is step +
 *                   *d_counter and Adam's step t + *d_counter.
 * Errors: TNVAN_E_ARG (batch < 1, NULL pointer, bad Adam arguments),
 * TNVAN_E_STATE, TNVAN_E_UNSUPPORTED, TNVAN_E_CUDA. */
int tnvan_train_step(tnvan_ctx* ctx, const double* betas, int batch, uint64_t seed, uint64_t step,
                     int precision, int8_t* d_spins, float* d_logq, double* d_logZR, double* d_dbeta,
                     double* d_dJ, float* d_grad_params, float* d_m, float* d_v, double lr,
                     double beta1, double beta2, double eps, int64_t t, void* stream);

/* Autotuner (not in the paper): times candidate launch shapes on a batch of
 * `batch` samples drawn from the current networks -- the SIMT sampler's
 * samples per CTA, the strip contraction's samples per CTA, the number of
 * CTAs per instance of the fused BF16 backward, the strip adjoint's samples
 * per CTA, the BF16 tensor-core sampler's form and plan (the grouped form,
 * two hidden layers of <= 128 units and D <= 128: step-group size limit 4, 6
 * or 8; the per-step form, any network the sampler takes: chunk size limit
 * 12, 16 or 32), whether tnvan_sample_contract_adjoint overlaps sampling
 * and the strip adjoint on side streams (2 = on, 1 = off), and, for networks
 * the fused BF16 backward does not take, whether the TF32 / BF16 backward
 * runs as the tensor-core GEMM chain (1) or as the FP32 SIMT backward (2,
 * exact to FP32 and faster for small networks) -- with CUDA events on
 * `stream`, and keeps
 * the fastest in the context for later calls.  With the overlapped schedule
 * and the fused backward, the backward's CTA count and the adjoint's shape
 * are finally re-timed together on whole tnvan_train_step calls, captured
 * in a CUDA graph on a private stream and replayed, with learning rate 0 and
 * scratch moments, so the networks are left as they were.  out (host
 * int32[7], may be NULL) receives the choices in that order (0 = heuristic,
 * not tuned).
 * Synchronous; allocates and frees temporary device buffers.
 * Errors: TNVAN_E_ARG, TNVAN_E_STATE, TNVAN_E_NOMEM, TNVAN_E_CUDA. */
int tnvan_autotune(tnvan_ctx* ctx, const double* betas, int batch, int precision, void* stream,
                   int32_t* out);

/* Sets the launch shapes that tnvan_autotune chooses, in the same order and
 * units as its `out` (host int32[7]: SIMT sampler samples per CTA, strip
 * samples per CTA, fused-backward CTAs per instance, strip-adjoint samples
 * per CTA (1 = one warp per strip over 32 samples), tensor-core sampler
 * form and plan as above, overlapped schedule 2 on / 1 off, backward form 1
 * tensor-core chain / 2 FP32 SIMT); 0 restores the
 * built-in default for that entry (the overlapped schedule is on by
 * default).  Lets a caller reuse an earlier tuning without re-timing.  Not in
 * the paper.
 * Errors: TNVAN_E_ARG (NULL, or a value outside the candidates the autotuner
 * tries: {16,32,64}, {32,64,128}, >= 1, {1,32,64,96,128}, {4,6,8,12,16,32}, {1,2},
 * {1,2}). */
int tnvan_set_tuning(tnvan_ctx* ctx, const int32_t* choices);

/* Optional device step counter (not in the paper; for CUDA-graph capture).
 * With d_counter non-NULL, every sampling launch uses the Philox step
 * `step + *d_counter`, read on the device when the kernel runs, so a graph
 * captured once draws fresh random numbers on each replay if the caller
 * advances *d_counter between replays (e.g. inside the graph).  tnvan_adam
 * then takes its step as t + *d_counter, with the bias corrections formed on
 * the device.  d_counter: borrowed device uint64; NULL restores host-only
 * steps. */
int tnvan_set_step_counter(tnvan_ctx* ctx, const uint64_t* d_counter);

/* Per-kernel timing, a tracing aid (not in the paper).  enable = 1 clears the
 * records and starts bracketing every kernel launch of this context with a
 * pair of CUDA events on the launch stream; enable = 0 stops recording.
 * Synchronous only in tnvan_profile_read, which waits for the recorded
 * events and reports, for kernel `index` (0-based, in first-launch order):
 * its name (NUL-terminated, truncated to name_len), summed elapsed ms and
 * number of launches.  Returns TNVAN_E_ARG when index is past the last kernel. */
int tnvan_profile(tnvan_ctx* ctx, int enable);
int tnvan_profile_read(tnvan_ctx* ctx, int index, char* name, int name_len, double* total_ms,
                       int64_t* launches);

/* Timeline of the launches recorded since profiling was enabled, a tracing
 * aid: for launch n (kernels in first-launch order, each kernel's launches in
 * recording order) kernel[n] = its kernel index (as for tnvan_profile_read)
 * and start_ms[n], end_ms[n] its bracketing events relative to an event
 * recorded before the first profiled launch, whatever streams the launches
 * ran on.  Writes at most max_entries (host arrays, any may be NULL); *n_out =
 * the number of recorded launches.  Call before tnvan_profile_read, which
 * consumes the records.  Synchronous.  Errors: TNVAN_E_ARG, TNVAN_E_CUDA. */
int tnvan_profile_trace(tnvan_ctx* ctx, int64_t max_entries, int32_t* kernel, float* start_ms, float* end_ms,
                        int64_t* n_out);

/* Allocation-free free-energy reduction.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory at all
 * (an external memory manager that owns every byte, a plugin that must not
 * grow the device footprint, a launch path on which cudaMalloc's implicit
 * synchronisation is not acceptable).  It needs no context and allocates
 * nothing: it computes, for n_inst instances of `batch` samples each (layout
 * of tnvan_free_energy), on `stream`, asynchronously,
 *   d_out[5k+0..4] = F_q, F_IS, stderr, logZ_IS, number of non-finite l_b
 * in FP64 (a two-pass reduction; its result equals tnvan_free_energy's to
 * FP64 rounding).  Non-finite l_b are left out of the sums instead of failing
 * the call, whichever samples they are: the statistics are those of the
 * finite l_b alone.  Check d_out[5k+4] < batch: when every l_b of an instance
 * is non-finite, its four statistics are NaN and d_out[5k+4] = batch.
 *   betas    host double [n_inst], finite and > 0 (read during the call).
 *   d_logZR  device double [n_inst*batch]; d_logq device float [n_inst*batch].
 *   d_out    device double [5*n_inst].
 * Its scratch is a fixed 104 KB array in this library's device image, held by
 * every GPU that loads the library until the process exits; hence the limit
 * n_inst <= 128 (larger counts fail with TNVAN_E_ARG).  All calls on a device
 * share that array: calls whose work may overlap on the GPU (different
 * streams, or different host threads) race and give wrong results; calls on
 * one stream are ordered and safe.  Each call made outside stream capture
 * looks up the array's device address (cudaGetSymbolAddress, with the
 * caller's current device) and remembers it for calls made during a
 * capture, so the first call on each device must come before any stream
 * capture.  Errors: TNVAN_E_ARG, TNVAN_E_CUDA; message from
 * tnvan_noalloc_last_error(). */
int tnvan_free_energy_noalloc(int n_inst, int batch, const double* betas, const double* d_logZR,
                              const float* d_logq, double* d_out, void* stream);
const char* tnvan_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TNVAN_H */
