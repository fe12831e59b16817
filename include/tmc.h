/*
 * tmc.h -- C ABI of the GB300 (sm_103a) Tensor Monte Carlo hot path.
 *
 * Tensor Monte Carlo (Aitchison, ICML 2019) estimates the marginal likelihood of a latent
 * variable model by drawing K_i proposal samples for each latent z_i and averaging the
 * importance ratio over all prod_i K_i combinations of samples (Eq. (is), Section 2.1).
 * For a tree-structured directed model the ratio is a product of factors, one per latent,
 * each indexed by the latent's own sample and its parent's (Eq. (fac), Section 2.2, and
 * the Appendix "Typical choice of factors"), so the sum is evaluated exactly by summing
 * out one index at a time from the leaves up: a chain of log-space K x K tensor
 * contractions (Section 2.2, Fig. 2; the log-domain product of the Appendix
 * "Numerically stable matrix (tensor) products").  This library evaluates log P_TMC and its
 * reparameterisation gradient (Section 2.2: gradient ascent on log P_TMC) for batches of
 * linear-Gaussian instances:
 *
 *   z_0 ~ N(bias_0, prior_var I)
 *   z_i | z_p ~ N(W_i z_p + bias_i, prior_var I),   i >= 1, p = parent[i] < i
 *   x_l | z_l ~ N(C z_l, obs_var I)                 for every leaf l of the tree
 *   Q_i(z_i) = N(m_i, diag(exp(2 logs_i))),  z_i^k = m_i + exp(logs_i) * eps_i^k
 *
 * Conventions for every entry point
 *   - Status codes are returned, never raised; no entry point aborts the process.
 *   - Memory: pointers named "host" are host memory, every tensor in tmc_inputs / tmc_grads
 *     and log_phat / grad_out are DEVICE memory owned by the caller; the plan owns its
 *     workspace (allocated once by tmc_plan_create, freed by tmc_plan_destroy).
 *   - Streams: `stream` is a cudaStream_t (0 = legacy default stream).  Calls enqueue work
 *     and return without synchronising; inputs must stay valid until the work completes.
 *   - A plan is not thread-safe; calls on one plan must be serialised by the caller.
 *   - After tmc_plan_create no call allocates device or host memory.
 */
#ifndef TMC_H
#define TMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TMC_OK = 0,
  TMC_ERR_INVALID_ARG = 1, /* malformed description / NULL required pointer / bad sizes */
  TMC_ERR_UNSUPPORTED = 2, /* valid problem outside what the kernels implement            */
  TMC_ERR_NOMEM = 3,       /* workspace allocation failed                                  */
  TMC_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed                  */
  TMC_ERR_NUMERIC = 5,     /* the device saw a non-finite input or result                  */
  TMC_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up                           */
  TMC_ERR_STATE = 7        /* call order violated (e.g. backward before forward)           */
} tmc_status;

/* Value 1 is reserved and rejected (TMC_ERR_INVALID_ARG): single bf16 operands cannot hold the
 * pairwise exponent to the reduced-precision tolerance (errors of 0.2-1.3 nats at K = 1024,
 * d = 128), and a bf16 hi/lo split keeps fewer bits (16) than the fp16 split (22). */
typedef enum {
  TMC_PREC_FP32 = 0,    /* CUDA-core FP32 contractions                                     */
  TMC_PREC_FP16_TC = 2, /* tcgen05 tensor cores; every product feeding an exponent is formed
                           from split fp16 operands (x = hi + lo) as hi*hi + lo*hi + hi*lo
                           with FP32 accumulation (about 22 significant bits)             */
  TMC_PREC_FP32_UNFUSED = 3 /* FP32, every K x K log-factor written to device memory before a
                               separate row log-sum-exp pass (the materialised baseline of
                               Section 2.2's sums; adjoint as TMC_PREC_FP32)                  */
} tmc_precision;

typedef struct tmc_plan_s* tmc_plan;

/* Problem description; all arrays are HOST memory and are copied into the plan.
 * Section 2.1 fixes what a problem is: the graph (parents), K_i samples per latent (Eq. (is)
 * lets K_i differ from latent to latent), the generative model P and the proposal Q.
 * Sizes: with K_node == NULL every latent of instance b has K[b] samples, and with d_node ==
 * NULL dimension d[b]; otherwise K_node / d_node give K_i / d_i latent by latent (then W_i is
 * d_i x d_parent, and the leaves of an instance must share one dimension, the one C acts on). */
typedef struct {
  int32_t num_instances;  /* B >= 1                                                        */
  const int32_t* n;       /* [B]    latents per instance, n_b >= 1                          */
  const int32_t* parent;  /* [sum n_b] local parent index, parent[0] = -1, 0<=parent[i]<i   */
  const int32_t* K;       /* [B]    samples per latent (every latent of b; see K_node)      */
  const int32_t* d;       /* [B]    latent dimension (every latent of b; see d_node)        */
  const int32_t* obs_dim; /* [B]    observation dimension                                   */
  int32_t shared_params;  /* 1: all instances share W, bias, C (then n, parent, d_i,       */
                          /*    obs_dim must agree; K may differ); 0: each has its own      */
  double prior_var;       /* sigma_z^2 > 0                                                  */
  double obs_var;         /* sigma_x^2 > 0                                                  */
  int32_t precision;      /* tmc_precision                                                  */
  const int32_t* K_node;  /* [sum n_b] per-latent K_i, or NULL                               */
  const int32_t* d_node;  /* [sum n_b] per-latent d_i, or NULL                               */
  int32_t coupled_proposal; /* 0: factorised Q_i = N(m_i, diag(exp(2 logs_i))) (Section 2.1);
                               1: sample k of latent i is drawn given its parent's sample k,
                               Q_i = N(m_i + A_i (z_p^k - m_p), diag(exp(2 logs_i))) -- a
                               non-factorised proposal of Section 2.3 (needs K_i <= K_parent,
                               tmc_inputs.q_A, and not the materialised-factor baseline)      */
} tmc_problem_desc;

/* Device inputs: contiguous float32, instance b directly after instance b-1 and latent i
 * after latent i-1 within it (sizes K_i, d_i as described above; d_p = the parent's d):
 *   eps       [sum K_i*d_i]      [i][k][j]   proposal noise
 *   q_mean    [sum d_i]          [i][j]      proposal means m_i
 *   q_logstd  [sum d_i]          [i][j]      proposal log standard deviations
 *   W         [sum d_i*d_p]      [i][r][c]   W_i is d_i x d_p; the root's block is d_0 x d_0
 *                                            and ignored (one instance's blocks when shared)
 *   bias      [sum d_i]          bias_0 is the root prior mean (one instance's when shared)
 *   C         [obs*d_leaf] per instance (one when shared), [o][c]
 *   x         [sum leaves_b*obs_b]  one observation per leaf, leaves in node order */
typedef struct {
  const float *eps, *q_mean, *q_logstd, *W, *bias, *C, *x;
  const float* q_A;  /* coupled proposals: A_i, [sum d_i*d_p] per instance (layout of unshared W,
                        root blocks ignored); NULL otherwise                                 */
} tmc_inputs;

/* Device gradient outputs (same layouts as the inputs).  Every non-NULL buffer is
 * OVERWRITTEN with d(sum_b grad_out[b] * log P_TMC_b)/d(input) -- whatever it held before is
 * ignored, so the caller need not zero it; NULL skips that output.  (Overwriting rather than
 * adding into the buffer lets a training loop reuse one set of gradient buffers per step
 * without a memset; a caller that accumulates adds the result itself.)
 *   dz         gradient w.r.t. the samples z_i^k (proposal density evaluated at z, its
 *              parameters held fixed)
 *   dq_mean, dq_logstd   reparameterisation gradients w.r.t. m_i and logs_i
 *   dW, dbias, dC        model gradients (summed over instances when shared)
 *   deps       gradient w.r.t. the noise eps (= exp(logs) * dz), same layout as eps; after the
 *              others, so the fields before it keep the order dz, dq_mean, dq_logstd, dW,
 *              dbias, dC
 * With a coupled proposal the samples move with their parents' (eps held fixed), and dz is
 * defined as (d / d eps) / exp(logs) -- which is the factorised definition above when A = 0. */
typedef struct {
  float *dz, *dq_mean, *dq_logstd, *dW, *dbias, *dC, *deps;
  float* dq_A;  /* coupled proposals: gradient w.r.t. A_i (layout of q_A; root blocks zero)  */
} tmc_grads;

/* Builds a plan: validates the description (tree shape, sizes), derives the
 * leaves-to-root elimination schedule of Section 2.2 (one level of the tree at a time),
 * allocates the device workspace.  On success *out owns the plan.  Errors:
 * TMC_ERR_INVALID_ARG, TMC_ERR_UNSUPPORTED (e.g. a precision the kernels do not cover for these shapes,
 * d or obs_dim > 1024, K > 16384), TMC_ERR_NOMEM, TMC_ERR_CUDA. */
tmc_status tmc_plan_create(const tmc_problem_desc* desc, tmc_plan* out);

/* log P_TMC of Eq. (is) for every instance, evaluated by the elimination of Section 2.2:
 * for each edge (p -> i), lambda_i[k] = log (1/K_i) sum_k' exp(log f_i^{(k',k)} + beta_i[k'])
 * with f_i = P(z_i | z_p) / Q_i(z_i) (Appendix) and beta_i the log of everything indexed by
 * k_i alone (node terms and children's messages); the root closes the sum.
 * log_phat: DEVICE double[B], written.  Saves what tmc_backward needs in the plan. */
tmc_status tmc_log_marginal(tmc_plan plan, const tmc_inputs* in, double* log_phat,
                            void* stream);

/* Reparameterisation gradient of sum_b grad_out[b] * log P_TMC_b (Section 2.2, "gradient
 * ascent on log P_TMC"; Section 1, reparameterisation trick), computed by the adjoint of
 * the elimination: top-down marginal weights over samples, with the K x K factors
 * recomputed rather than stored.  grad_out: DEVICE double[B] or NULL (all ones).
 * Requires a preceding tmc_log_marginal on the same plan with the same inputs
 * (TMC_ERR_STATE otherwise).  Outputs are overwritten (see tmc_grads). */
tmc_status tmc_backward(tmc_plan plan, const tmc_inputs* in, const double* grad_out,
                        const tmc_grads* grads, void* stream);

/* log P_TMC per instance for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of tmc_log_marginal (FP32 path, forward only).
 * It is for code that must not call cudaMalloc -- running inside a real-time loop, under a
 * memory pool that owns the whole device, or in a host process whose allocator is not
 * CUDA's -- and so cannot hold a plan.  It takes no plan: the description (HOST memory, as
 * for tmc_plan_create, precision TMC_PREC_FP32) and the DEVICE inputs / output are passed
 * per call, and all scratch lives in one fixed-size file-scope device array of 10,330,368
 * bytes (~9.9 MiB) that every GPU running this call holds until the process exits.  Nothing
 * here calls cudaMalloc, cudaFree or any allocating routine.
 *   Limits of one call: at most 2048 latents and 1024 instances in total, sum of n_b*K_b <=
 *   65536, sum of n_b*K_b*d_b <= 1048576, 8192 64-sample tiles; beyond them the call returns
 *   TMC_ERR_UNSUPPORTED before any device work.
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress with
 *   that device current).
 *   A call on a stream that is being captured into a CUDA graph returns TMC_ERR_UNSUPPORTED
 *   and enqueues nothing: each call uploads its node and tile tables from static host arrays
 *   that the next call rewrites, so a captured upload would replay another call's tables.
 *   Every call reuses the same array, and its contents are left from the last call: calls
 *   whose GPU work overlaps (different streams or host threads) race and must be serialised.
 *   Device-side numeric errors are not reported; a non-finite input gives a non-finite result.
 * log_phat: DEVICE double[B], written on `stream`. */
tmc_status tmc_log_marginal_noalloc(const tmc_problem_desc* desc, const tmc_inputs* in,
                                    double* log_phat, void* stream);

/* Waits for the plan's outstanding work on `stream` and reports device-side errors recorded
 * since the last call (TMC_ERR_NUMERIC for non-finite values, TMC_ERR_TIMEOUT), clearing
 * them.  TMC_OK if none. */
tmc_status tmc_plan_sync_status(tmc_plan plan, void* stream);

/* Budget, in SM clock cycles, of every cross-CTA dependency wait of the persistent edge
 * launches (a tile waiting for the tiles whose messages or weights it reads).  Default 2^31
 * (about a second at 2 GHz); a wait that runs out makes the kernel record TMC_ERR_TIMEOUT and
 * return.  Takes effect from the next call.  TMC_ERR_INVALID_ARG for cycles < 1.
 *
 * Fault injection for tests of the error paths, read from the environment variable TMC_FAULT
 * when a plan is created (host side; nothing here makes a GPU fault, trap or hang):
 *   "alloc"   tmc_plan_create returns TMC_ERR_NOMEM before allocating anything;
 *   "launch"  tmc_log_marginal / tmc_backward return TMC_ERR_CUDA before enqueuing any work;
 *   "stall"   (tensor-core plans) the persistent forward edge launch leaves out the tiles of
 *             the deepest latent of instance 0, so its parent's tiles wait on a completion
 *             count that never arrives: the wait runs out after the wait limit, the kernel
 *             records the timeout and returns, and tmc_plan_sync_status reports
 *             TMC_ERR_TIMEOUT (the results of that call are meaningless). */
tmc_status tmc_plan_set_wait_limit(tmc_plan plan, long long cycles);

/* Bytes of device workspace owned by the plan. */
tmc_status tmc_plan_workspace_bytes(tmc_plan plan, size_t* bytes);

/* Releases the plan and its workspace (synchronises the device first).  NULL is a no-op. */
tmc_status tmc_plan_destroy(tmc_plan plan);

/* Static, human-readable name of a status code. */
const char* tmc_status_string(tmc_status s);

/* Work order of the persistent edge launches of a tensor-core plan (the tunable of the
 * autotuner in the Python binding).  Every order keeps each tile after all tiles it depends
 * on (the next tree level), so none can deadlock:
 *   0 (default) level by level, the tiles of one edge adjacent (instance by instance);
 *   1 level by level, tile index major (tile r of every edge, then tile r+1);
 *   2 level by level, instances with more edge work (sum of K^2 d) first.
 * set: synchronises the device and rewrites the plan's tile list (no allocation);
 * TMC_ERR_UNSUPPORTED on FP32 plans, TMC_ERR_INVALID_ARG for an unknown order. */
tmc_status tmc_plan_set_schedule(tmc_plan plan, int schedule);
tmc_status tmc_plan_get_schedule(tmc_plan plan, int* schedule);

/* Tuning knobs of a tensor-core plan (the autotuner in the Python binding sweeps them); none
 * changes the arithmetic of a tile, so every setting gives the same log P_TMC bit for bit:
 *   TMC_TUNE_SCHEDULE      the work order above (0, 1, 2)
 *   TMC_TUNE_PROLOGUE_LEAD chunks before the end of a forward item at which the next item's
 *                          prologue operands and mu~ product enter the ring / MMA order (1..3;
 *                          default 2): earlier overlaps more, later keeps more ring stages for
 *                          the item's own chunks
 *   TMC_TUNE_GRID          CTAs of each persistent edge launch: 0 (default) one per SM, else
 *                          that many (capped at the SM count and the item count)
 * set: no allocation; TMC_ERR_UNSUPPORTED on FP32 plans, TMC_ERR_INVALID_ARG for an unknown
 * knob or value. */
enum { TMC_TUNE_SCHEDULE = 0, TMC_TUNE_PROLOGUE_LEAD = 1, TMC_TUNE_GRID = 2 };
tmc_status tmc_plan_set_tuning(tmc_plan plan, int knob, int value);
tmc_status tmc_plan_get_tuning(tmc_plan plan, int knob, int* value);

/* Per-instance completion times of the last tmc_log_marginal / tmc_backward on a tensor-core
 * plan: the time (microseconds) from the first edge tile of the persistent edge launch to
 * the moment the instance's last edge tile finished, in each direction.  HOST double[B]
 * outputs (either may be NULL); synchronises the device.  TMC_ERR_UNSUPPORTED on the FP32
 * paths (their edge kernels run one launch per tree level). */
tmc_status tmc_plan_instance_times(tmc_plan plan, double* fwd_us, double* bwd_us);

/* ---- kernel timing (library-internal CUDA events on the launch stream) ----------------
 * Kernel classes, in the order of the hot path: */
enum {
  TMC_KC_SAMPLE = 0,  /* samples, node terms, observation residuals                         */
  TMC_KC_PROJECT = 1, /* conditional means mu_i = W_i z_p + bias_i                          */
  TMC_KC_EDGE_FWD = 2,/* fused pairwise factor + log-sum-exp message                        */
  TMC_KC_ROOT = 3,    /* root reduction to log P_TMC (FP64)                                 */
  TMC_KC_EDGE_BWD = 4,/* fused adjoint of the messages (factors recomputed)                 */
  TMC_KC_PARAM = 5,   /* parameter / proposal gradient assembly                             */
  TMC_KC_SAMPLE_GRAD = 6, /* per-sample gradients dz / deps beyond the above (tensor-core path) */
  TMC_KC_COUNT = 7
};
/* Turns event timing of every launch on (1) or off (0); resets the accumulators. */
tmc_status tmc_profile_enable(tmc_plan plan, int enable);
/* Synchronises, then returns the summed device time (ms) and launch count of a kernel
 * class since the last enable. */
tmc_status tmc_profile_read(tmc_plan plan, int kernel_class, double* total_ms,
                            long long* launches);

/* ---- the loopy graph of Fig. 1: matrix messages (Section 2.2) ---------------------------
 * Four latents of dimension d, K samples each, where z4 has two parents that share the parent
 * z1 (a loop in the undirected graph):
 *   z1 ~ N(bias_0, prior_var I),  z2 | z1 ~ N(W_1 z1 + bias_1, prior_var I),
 *   z3 | z1 ~ N(W_2 z1 + bias_2, prior_var I),  z4 | z2, z3 ~ N(W_3 z2 + W_4 z3 + bias_3, prior_var I),
 *   x | z4 ~ N(C z4, obs_var I);   Q_i = N(m_i, diag(exp(2 logs_i))) (factorised).
 * Summing out k4 and then k1 (Fig. 1 C, D) leaves two factors over (k2, k3), each a log-domain
 * matrix product of K x K factor matrices (the Appendix's "Numerically stable matrix (tensor)
 * products"); log P_TMC is the log-mean-exp of their sum with the (k2, k3) factor.
 * Inputs (tmc_inputs, DEVICE float32; q_A unused):
 *   eps [B][4][K][d], q_mean / q_logstd [B][4][d], W [5][d][d] per instance (W_0 unused),
 *   bias [4][d] per instance, C [obs][d] per instance (one instance's when shared), x [B][obs].
 * Arithmetic: factor matrices from split fp16 operands on tcgen05 tensor cores (as
 * TMC_PREC_FP16_TC), the matrix products exp(X - x) exp(Y - y)^T of the messages from bf16
 * exponentials on tcgen05 (split pairs or single, see message_precision; FP32 range), entries
 * whose sum underflows recomputed exactly; FP64 final reduction.
 * Limits: d <= 128, obs_dim <= 1024, K <= 16384 (TMC_ERR_UNSUPPORTED beyond). */
typedef struct tmc_loopy_plan_s* tmc_loopy_plan;
typedef struct {
  int32_t num_instances; /* B >= 1                                                         */
  int32_t K;             /* samples per latent                                             */
  int32_t d;             /* latent dimension                                               */
  int32_t obs_dim;       /* observation dimension                                          */
  int32_t shared_params; /* 1: one W, bias, C for all instances                            */
  double prior_var, obs_var;
  int32_t message_precision; /* operands exp(X - x), exp(Y - y) of the two message products:
                                0 split bf16 pairs (hi*hi + lo*hi + hi*lo, ~16 bits, 3 MMAs);
                                1 single bf16 (1 MMA; each product within 2^-8 relative, so
                                each message entry within 3.9e-3 nats, log P_TMC within
                                7.8e-3)                                                      */
} tmc_loopy_desc;

/* Allocates the plan and its device workspace (about B (10 K^2 + 24 K d) * 4 bytes).
 * Errors: TMC_ERR_INVALID_ARG, TMC_ERR_UNSUPPORTED, TMC_ERR_NOMEM, TMC_ERR_CUDA. */
tmc_status tmc_loopy_plan_create(const tmc_loopy_desc* desc, tmc_loopy_plan* out);
/* Enqueues log P_TMC[b] (DEVICE double[B]) on `stream`; returns without synchronising. */
tmc_status tmc_loopy_log_marginal(tmc_loopy_plan plan, const tmc_inputs* in, double* log_phat,
                                  void* stream);
/* Stages of tmc_loopy_log_marginal, in launch order. */
enum {
  TMC_LOOPY_PREP = 0,    /* samples, node terms, projections, split fp16 operands            */
  TMC_LOOPY_FACTOR = 1,  /* the five K x K factor matrices (one tensor-core launch)          */
  TMC_LOOPY_EXP = 2,     /* row maxima and bf16 exponentials of the message operands          */
  TMC_LOOPY_MESSAGE = 3, /* the two log-domain matrix products (one tensor-core launch)      */
  TMC_LOOPY_FINAL = 4,   /* the (k2, k3) sum, exact recomputation of underflowed entries     */
  TMC_LOOPY_STAGE_COUNT = 5
};
/* Synchronises; returns (HOST, each may be NULL) the summed device time (ms) of every stage
 * since the last call (stage_ms: double[TMC_LOOPY_STAGE_COUNT]), the forward calls timed, and
 * the number of message entries recomputed exactly; then turns stage timing on (enable = 1)
 * or off and resets the counters.  Timing synchronises each timed call.  TMC_ERR_TIMEOUT if a
 * bounded device wait gave up since the last call. */
tmc_status tmc_loopy_profile(tmc_loopy_plan plan, int enable, double* stage_ms, long long* calls,
                             int* exact_entries);
/* N tile of the message products: 128 or 256 columns per CTA tile (0: 256 when K > 128, the
 * default).  No allocation; the results are the same up to the order of the FP32 sums within
 * a tile.  TMC_ERR_INVALID_ARG for another value. */
tmc_status tmc_loopy_plan_set_tile(tmc_loopy_plan plan, int n_tile);
/* Releases the plan (synchronises the device first).  NULL is a no-op. */
tmc_status tmc_loopy_plan_destroy(tmc_loopy_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* TMC_H */
