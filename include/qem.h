/*
 * qem.h -- C ABI of libqem: the QEM E-step (massively parallel importance
 * weighting over a plated hierarchical model) and M-step on one GB300 GPU.
 *
 * Method: arXiv 2503.08264, "Massively Parallel Expectation Maximization For
 * Approximate Posteriors".  Every entry point below cites the passage that
 * defines the operation it performs.
 *
 * Conventions shared by every call
 *  - Plain pointers and sizes only.  A pointer documented DEVICE must point to
 *    memory of the CUDA device that was current when the plan was created; a
 *    pointer documented HOST must point to host memory.  The caller owns every
 *    buffer it passes; the plan owns only its internal workspace.
 *  - All device work is enqueued on the plan's stream (qem_plan_opts.stream,
 *    or the legacy default stream when NULL).  Calls are asynchronous unless
 *    documented otherwise; inputs must stay valid until the stream reaches
 *    the call's work.
 *  - Errors are returned as qem_status; nothing is thrown across the ABI and
 *    nothing aborts.  Argument errors are detected on the host before any
 *    launch.  Asynchronous CUDA faults surface as QEM_ERR_CUDA at a later
 *    call; numerical failures (non-finite log P_MP) as QEM_ERR_NUMERIC from
 *    qem_log_pmp; an expired bounded device wait as QEM_ERR_TIMEOUT.
 *  - Flat, level-major buffers.  A model has L levels; level l has n_l plate
 *    elements of latent dimension D_l.  A "per-element" buffer of E values per
 *    element stores level 0's n_0*E values, then level 1's, and so on;
 *    qem_layout() returns each level's offset (in elements of the buffer's
 *    type).
 *      q_params     float  [n_l][2][D_l]       proposal parameters
 *                                               Gaussian (loc, scale), Gamma (shape, rate), Beta (a, b)
 *      moments      double [n_l][2][D_l]       E_w[T(z)]: Gaussian (z, z^2), Gamma (z, log z),
 *                                               Beta (log z, log(1-z))
 *      mean_params  double [n_l][2][D_l]       EMA state m_t, same statistics
 *      eps          float  [n_l][K][nps_l]     supplied noise; nps = D (Gaussian),
 *                                               D*(2*QEM_GAMMA_TRIES+1) (Gamma), twice that (Beta)
 *      weights      float  [n_l][K]            marginal weight of every sample
 */
#ifndef QEM_H
#define QEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QEM_MAX_LEVELS 4
#define QEM_GAMMA_TRIES 8

typedef enum {
  QEM_OK = 0,
  QEM_ERR_INVALID_ARG = 1,  /* a size, pointer or descriptor field is invalid          */
  QEM_ERR_UNSUPPORTED = 2,  /* valid but not implemented (e.g. a dimension too large)   */
  QEM_ERR_OOM = 3,          /* workspace allocation failed                              */
  QEM_ERR_CUDA = 4,         /* a CUDA call or kernel failed                             */
  QEM_ERR_NUMERIC = 5,      /* non-finite log P_MP or weights                            */
  QEM_ERR_TIMEOUT = 6       /* a bounded device-side wait expired                       */
} qem_status;

/* How p(z_e | z_parent) is defined for the elements of a level (the model's
 * prior factor in Eq. rmp; App. F gives the models).                        */
enum {
  QEM_PRIOR_STD_NORMAL = 0,       /* N(0, prior_a I)                               (level 0 only) */
  QEM_PRIOR_NORMAL_FIXED_VAR = 1, /* N(z_parent, prior_a I), D_parent = D                         */
  QEM_PRIOR_NORMAL_MEAN_LOGVAR = 2,/* N(z_parent[0:D], diag exp(z_parent[D:2D])), D_parent = 2D    */
  QEM_PRIOR_GAMMA = 3,            /* Gamma(shape prior_a, rate prior_b)            (level 0 only) */
  QEM_PRIOR_BETA = 4              /* Beta(prior_a, prior_b)                         (level 0 only) */
};

/* Likelihood of the observations of one element; s_n = z . x_n.            */
enum {
  QEM_LIK_NONE = 0,
  QEM_LIK_GAUSS = 1,              /* y_n ~ N(s_n, lik_var)                      */
  QEM_LIK_BERNOULLI_LOGIT = 2,    /* y_n ~ Bernoulli(sigmoid(s_n))              */
  QEM_LIK_POISSON_LOG = 3,        /* y_n ~ Poisson(exp(s_n))                    */
  QEM_LIK_POISSON_RATE = 4,       /* y_n ~ Poisson(z), D = 1                    */
  QEM_LIK_BERNOULLI_PROB = 5      /* y_n ~ Bernoulli(z), D = 1                  */
};

/* Exponential-family proposal families with closed-form M-steps (Sec. 4).   */
enum { QEM_Q_GAUSS = 0, QEM_Q_GAMMA = 1, QEM_Q_BETA = 2 };

/* Arithmetic of the K x K log-factor contraction (the other steps are FP32
 * with FP64 plate sums, root and moments in every mode).                    */
enum {
  QEM_PREC_FP32 = 0,    /* FP32 CUDA-core contraction                                   */
  QEM_PREC_BF16 = 1,    /* tcgen05 BF16 operands, FP32 accumulation                      */
  QEM_PREC_BF16X3 = 2,  /* tcgen05 split BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulation */
  QEM_PREC_TF32 = 3     /* tcgen05 kind::tf32, operands rounded to TF32 (10-bit mantissa),
                         * one product per k-step, FP32 accumulation; the local factor h
                         * enters as three TF32 parts, so only the bilinear terms round  */
};

typedef struct {
  int64_t n;            /* plate elements at this level over all instances (n_0 = instances) */
  int dim;              /* latent dimension D (1..64)                                        */
  int prior;            /* QEM_PRIOR_*                                                        */
  double prior_a, prior_b;
  int lik;              /* QEM_LIK_*                                                          */
  double lik_var;       /* variance of QEM_LIK_GAUSS                                          */
  int n_obs;            /* observations per element (0 with QEM_LIK_NONE)                     */
  int qfam;             /* QEM_Q_*                                                            */
  const int64_t* parent;/* HOST [n]: parent element at level-1, non-decreasing; NULL at level 0 */
  const float* x;       /* DEVICE [n][n_obs][dim] covariates (read at every E-step)            */
  const float* y;       /* DEVICE [n][n_obs] observations                                      */
  int chain;            /* 0 or 1: plain plate.  T > 1: a chain plate (App. F's Covid model:
                         * a daily autoregressive timeseries per region): the level's elements
                         * are n / T regions of T consecutive days, element c*T + d, each day
                         * its own latent; the T elements of a region share its parent; day 0
                         * takes the level's prior given the parent, day d >= 1 the prior
                         * N(z_{c,d-1}, prior_b I).  n a multiple of T, prior_b > 0 and one
                         * parent per region (QEM_ERR_INVALID_ARG otherwise).  Only as level 1
                         * of a two-level model, with a FP32 plan, a Gaussian proposal,
                         * dim <= 8 and K <= 1024 (QEM_ERR_UNSUPPORTED otherwise).             */
  int qcond;            /* 0: factorised proposal.  1: parent-conditioned proposal (App. A.2's
                         * non-factorised Q_MP with the permutation copy scheme): copy k is
                         * drawn from N(z_parent^{s(k)}[0:D] + loc, diag scale^2), s a uniformly
                         * random permutation of the parent's K copies per element (counter-
                         * based, or supplied by qem_set_perm); moments of the level are then
                         * the residual's (E d, E d^2), d = z - z_parent[0:D], which the
                         * Gaussian M-step turns into (loc, scale).  Only as level 1 of a
                         * two-level model with a FP32 plan, a Gaussian proposal, a normal
                         * prior given the parent and dim <= 32 (QEM_ERR_UNSUPPORTED else).  */
} qem_level_desc;

typedef struct {
  int n_levels;                         /* 1..QEM_MAX_LEVELS */
  qem_level_desc levels[QEM_MAX_LEVELS];
} qem_model_desc;

typedef struct {
  int K;                /* samples per latent, 1..4096                                       */
  int precision;        /* QEM_PREC_*                                                        */
  int tile;             /* 0: default launch shapes; QEM_TILE_AUTO: autotuned (see qem_tune)  */
  void* stream;         /* cudaStream_t the plan's work is enqueued on (NULL: default stream) */
  double var_floor;     /* Gaussian M-step variance floor factor (0: 1e-10)                   */
  double timeout_s;     /* bound of every device-side wait of the tensor-core contraction (0: 2 s):
                         * an expired wait stops the launch and qem_log_pmp then reports
                         * QEM_ERR_TIMEOUT; a CTA's waits for its own copies and MMAs before it
                         * exits keep a bound of their own (at least ~2 s of SM cycles)      */
} qem_plan_opts;

typedef struct qem_plan_s* qem_plan_t;

#define QEM_TILE_AUTO (-1)
#define QEM_TUNE_FORCE 1

/* Human-readable name of a status code (static storage). */
const char* qem_status_string(qem_status s);

/* Build a plan for the E-step of Eq. mp_iw over the model's plate tree (the
 * plated Bayes net of Sec. 3.1, summed leaves to root as in Sec. 6) and the
 * M-step of Alg. 1: validate the model (parents non-decreasing and in range,
 * prior and dimension compatible with the parent level), copy its plate structure
 * to the device and allocate the workspace, the plan's only device-memory
 * allocation: qem_estep, qem_mstep and qem_log_pmp_fresh allocate nothing
 * (graph-capturable), except that a plan made with tile = QEM_TILE_AUTO tunes
 * on its first call outside a capture; qem_run creates its graph (and, on the
 * legacy stream, a private stream), qem_tune a scratch buffer, and the
 * profiler its events.
 * The model's x and y pointers are kept and read by every E-step.  *out is
 * set to NULL on failure.                                                   */
qem_status qem_plan(const qem_model_desc* desc, const qem_plan_opts* opts, qem_plan_t* out);

/* Test hook of the bounded device waits (no counterpart in the paper): with
 * on != 0, every tensor-core contraction launched afterwards first makes its
 * MMA-issuing thread wait on a barrier that nothing completes before the
 * kernel's teardown.  That wait runs out after the plan's timeout_s, the CTA
 * aborts as after any expired wait (each role stops at its next wait, the
 * CTA waits for its own copies and MMAs, frees TMEM and exits) and
 * qem_log_pmp then returns QEM_ERR_TIMEOUT, which stays set for the plan's
 * life.  Plans whose contraction runs on the CUDA cores (QEM_PREC_FP32, chain
 * levels) have no such wait and are not affected.  Invalidates qem_run's
 * cached graph.                                                             */
qem_status qem_test_expire_wait(qem_plan_t plan, int on);

/* Release the plan and its workspace (synchronises the plan's stream). NULL is a no-op. */
qem_status qem_plan_destroy(qem_plan_t plan);

/* Bytes of device workspace the plan holds. */
qem_status qem_workspace_size(const qem_plan_t plan, size_t* bytes);

/* Offsets of level `level` inside the flat buffers (see the file comment):
 * q_off (q_params, moments and mean_params), eps_off (eps), w_off (weights). */
qem_status qem_layout(const qem_plan_t plan, int level, int64_t* q_off, int64_t* eps_off, int64_t* w_off);

/* Total lengths of the flat buffers: q_len (q_params / moments / mean_params),
 * eps_len (eps), w_len (weights), n_inst (log_pmp).                          */
qem_status qem_sizes(const qem_plan_t plan, int64_t* q_len, int64_t* eps_len, int64_t* w_len, int64_t* n_inst);

/* E-step (Alg. 1 "z ~ Q_t; m = MPIW(z, Q_t)"; Eq. mp_iw; Sec. 6 for the
 * plate-tree recursion).  Draws K samples per latent from the proposal
 * q_params (DEVICE float, layout above), forms the K_parent x K_child
 * log-factor tiles, contracts them leaves-to-root in log space into
 * log P_MP, runs the adjoint of that contraction root-to-leaves for the
 * marginal weight of every sample, and writes
 *   moments  DEVICE double [q_len]  E_w[T(z)] per element and dimension
 *   log_pmp  DEVICE double [n_inst] log P_MP of every instance (nullable)
 * eps: DEVICE float [eps_len] supplied noise, or NULL to draw it in-kernel
 * from the counter-based stream keyed by (seed, iter).                     */
qem_status qem_estep(qem_plan_t plan, const float* q_params, const float* eps, uint64_t seed,
                     uint64_t iter, double* moments, double* log_pmp);

/* E-step with the root's two halves as separate latents (the paper's own
 * form of App. F's MovieLens model: the global mean mu and the global
 * log-variance psi each carry their own sample index, so a user's prior
 * factor N(z_m; mu^a, diag exp(psi^b)) takes two parent indices and is
 * summed into a K x K table per user -- the K^(number of parents) tables of
 * the Limitations section; qem_estep groups (mu, psi) into one latent with
 * one index instead).  Eq. mp_iw over all (a, b, k_1, ..., k_M):
 *   log P_MP = log (1/K^2) sum_{a,b} exp(f_mu[a] + f_psi[b] + sum_m L_m[a][b]).
 * The plan must have two levels: level 0 of dimension 2D with the
 * QEM_PRIOR_STD_NORMAL prior, a Gaussian proposal and no likelihood; level 1
 * with QEM_PRIOR_NORMAL_MEAN_LOGVAR (mu = dimensions [0, D), psi = [D, 2D)
 * of the root sample rows, the same samples as qem_estep draws), D <= 32
 * and K <= 1024; otherwise QEM_ERR_UNSUPPORTED.  The contraction runs on the
 * CUDA cores in FP32 whatever the plan's precision (FP64 root sums).
 * Arguments as qem_estep; moments of the root take the mu weights for
 * dimensions [0, D) and the psi weights for [D, 2D).  root_weights: DEVICE
 * float [n_inst][2][K] (nullable) receives (w_mu, w_psi); qem_weights then
 * returns w_mu at level 0 and the users' marginal weights at level 1.
 * Workspace: n_1 K^2 floats of per-user tables plus n_0 K^2 root values,
 * allocated by the first call (QEM_ERR_OOM when it does not fit; that call
 * must not be inside a stream capture, QEM_ERR_UNSUPPORTED otherwise) and
 * kept by the plan.                                                         */
qem_status qem_estep_split_root(qem_plan_t plan, const float* q_params, const float* eps, uint64_t seed,
                                uint64_t iter, double* moments, double* log_pmp, float* root_weights);

/* Parent-copy permutations of the qcond level for the following E-steps:
 * perm DEVICE int32 [n_1][K], row e a permutation of 0..K-1 (copy k of element
 * e is drawn from parent copy perm[e][k]); kept by pointer (the caller keeps
 * it valid); NULL returns to the counter-based draw: per element the K keys
 * word (k mod 4) of Philox4x32-10 (Salmon et al. 2011) with counter
 * (k div 4, e mod 2^32, (e div 2^32) | 2^30, iter) and key seed, the copies
 * ordered by (key, k) ascending.  Invalidates qem_run's cached graph.
 * QEM_ERR_INVALID_ARG when the plan has no qcond level.                     */
qem_status qem_set_perm(qem_plan_t plan, const int32_t* perm);

/* Sharding one instance's plate over several processes (one GPU each).
 * Sec. 6 sums each plate out given the parent's samples: the elements of the
 * root's child plate are independent given the root's K samples, and the
 * root only sees their plate sum G[i][k_p] = sum_c log mean_k exp S_c[k_p][k]
 * (Eq. Prmp).  A shard's plan holds every root of the model and a contiguous
 * range of the root's children (with all their descendants); each process
 *   1. qem_estep_shard_forward: samples and contracts its range into its own
 *      G_r (no root step);
 *   2. sums G over the processes (an all-reduce of n_inst x K doubles, by the
 *      caller's collective library);
 *   3. qem_estep_shard_finish: the root step on the summed G (identical on
 *      every shard, since the roots' samples are), then the adjoint and the
 *      moments of its own range (the adjoint needs no exchange: the root's
 *      weights are replicated).
 * Then log P_MP, the root's weights and moments equal those of one process
 * holding the whole plate, and each shard holds its range's weights and
 * moments; the M-step stays per shard (the root's on every shard alike).
 * The paper has no multi-process form of the method; this is the
 * distributive law of Sec. 6 cut at the root.                                 */

/* Index in the counter-based noise streams (qem_estep's in-kernel draws and
 * qem_set_perm's default permutations) of element 0 of each level:
 * base HOST int64 [n_levels], each >= 0 (a shard passes the index, in the
 * whole model, of the first element it holds at each level, so that a
 * sharded run draws the whole model's noise).  Default 0.  Invalidates
 * qem_run's cached graph.                                                    */
qem_status qem_set_elem_base(qem_plan_t plan, const int64_t* base);

/* Step 1 above: the E-step of qem_estep up to and including the plate sums
 * into the root, without the root step.  Arguments as qem_estep; root_G:
 * DEVICE double [n_inst][K] receives G_r (copied on the plan's stream).
 * QEM_ERR_UNSUPPORTED for a one-level plan.                                  */
qem_status qem_estep_shard_forward(qem_plan_t plan, const float* q_params, const float* eps, uint64_t seed,
                                   uint64_t iter, double* root_G);

/* Step 3 above: root_G DEVICE double [n_inst][K], the sum over all shards of
 * their G_r (read on the plan's stream); then as qem_estep: moments DEVICE
 * double [q_len] of this shard's elements, log_pmp DEVICE double [n_inst]
 * (nullable).  Must follow qem_estep_shard_forward on the same plan with no
 * other E-step in between (the samples and tables of step 1 are reused).    */
qem_status qem_estep_shard_finish(qem_plan_t plan, const double* root_G, double* moments, double* log_pmp);

/* log P_MP of q_params from a fresh draw of the samples (the noise stream
 * keyed by (seed, iter), which the caller chooses distinct from the E-step's):
 * the forward half of the E-step only (Eq. Prmp; no weights, no moments).
 * The self-normalised estimate of qem_estep reuses the samples that its
 * moments came from; an independent draw gives an unbiased estimate of P_MP
 * for the given q, and with qem_moments_rescale the second-sample moment
 * estimate of the remark after Theorem 1.  log_pmp: DEVICE
 * double [n_inst] (nullable: the plan keeps the values for qem_log_pmp).
 * Overwrites the plan's samples and local factors (qem_weights and
 * qem_samples then describe no E-step).                                      */
qem_status qem_log_pmp_fresh(qem_plan_t plan, const float* q_params, uint64_t seed, uint64_t iter,
                             double* log_pmp);

/* The moment estimate normalised by a second, distinct sample (the remark
 * after Theorem 1): moments of every element of instance i multiplied by
 * exp(log_pmp_same[i] - log_pmp_fresh[i]), where log_pmp_same is the E-step's
 * own log P_MP (the self-normalising one) and log_pmp_fresh that of an
 * independent draw (qem_log_pmp_fresh).  All DEVICE, double; moments
 * [q_len] in/out; asynchronous on the plan's stream.                         */
qem_status qem_moments_rescale(qem_plan_t plan, const double* log_pmp_same, const double* log_pmp_fresh,
                               double* moments);

/* Predictive log-likelihood of held-out observations of every element of
 * `level` (the paper's diagnostic on held-out data), from the samples and
 * marginal weights of the last E-step:
 *   out[e] = log sum_k w_e[k] prod_n p(y_new[e][n] | z_e^k, x_new[e][n])
 * with the level's likelihood.  x_new DEVICE float [n][n_obs_new][dim]
 * (NULL allowed for the Poisson-rate and Bernoulli-probability likelihoods),
 * y_new DEVICE float [n][n_obs_new], out DEVICE double [n]; asynchronous on
 * the plan's stream.  QEM_ERR_INVALID_ARG for a level without likelihood,
 * QEM_ERR_UNSUPPORTED when n_obs_new * (dim + 2) floats exceed 48 KB.  No
 * counterpart of this entry point's exact form in the paper's code.         */
qem_status qem_predictive(qem_plan_t plan, int level, const float* x_new, const float* y_new, int n_obs_new,
                          double* out);

/* M-step with EMA (Alg. 1 "m_t = lambda m_hat + (1-lambda) m_{t-1}" followed by
 * the next iteration's "Q = set_exp_family_params(m_t)"; Eq. ema; App. B).
 *   moments      DEVICE double [q_len]  this iteration's E-step estimate m_hat
 *   mean_params  DEVICE double [q_len]  in: m_{t-1}; out: m_t
 *   q_params     DEVICE float  [q_len]  out: parameters matched to m_t
 * lambda is the weight of the new estimate; with sched_p in (0,1) it is
 * replaced by t^-sched_p (the schedule of Thm. 1, 1-lambda(t) in its
 * notation); t >= 1 is the iteration number.  moments may be NULL to only set
 * q_params from mean_params (Alg. 1's initial M-step).  Gamma and Beta
 * statistics that no member of the family has (non-finite; E log z >= log E z
 * for the Gamma; e^{E log z} + e^{E log(1-z)} >= 1 for the Beta, which
 * rounding can produce when the weights collapse) keep that element's
 * previous q_params and raise QEM_ERR_NUMERIC at the next qem_log_pmp.      */
qem_status qem_mstep(qem_plan_t plan, const double* moments, double* mean_params, float* q_params,
                     double lambda, double sched_p, int64_t t);

/* Mean parameters of given proposal parameters (Alg. 1 "m_0 = initial values"):
 *   q_params DEVICE float [q_len] in, mean_params DEVICE double [q_len] out.  */
qem_status qem_mean_params(qem_plan_t plan, const float* q_params, double* mean_params);

/* Copy log P_MP of the last E-step (Eq. Prmp: the log of the massively
 * parallel importance-weighted estimate of the evidence P(x), the quantity
 * Sec. 5 reports as the ELBO of each method) to HOST double [n_inst].
 * Synchronises the plan's stream; returns QEM_ERR_NUMERIC if any value is not
 * finite or a Gamma/Beta M-step met statistics outside its family's domain,
 * and QEM_ERR_TIMEOUT if a device wait of that E-step expired.  Error states
 * are sticky for the plan's life.                                           */
qem_status qem_log_pmp(qem_plan_t plan, double* host_out);

/* Copy the marginal weights of the last E-step (the per-sample posterior
 * weights of Eq. mmp, each element's K weights sum to one) to DEVICE float
 * [w_len], asynchronously on the plan's stream.                              */
qem_status qem_weights(qem_plan_t plan, float* weights);

/* Copy the samples of the last E-step to DEVICE float [sum_l n_l*K*D_l]
 * (level-major, [n_l][K][D_l] per level), asynchronously.                   */
qem_status qem_samples(qem_plan_t plan, float* z);

/* Run iterations t0 .. t0 + T - 1 of QEM (Alg. 1) on the device in ONE graph
 * launch: a CUDA graph whose conditional (while) node repeats one iteration
 * (E-step, EMA + M-step) until T are done or an error bit is set, with no
 * host round trip between iterations.  The graph is built on the first call
 * and kept by the plan while the buffers, lambda and sched_p stay the same (a
 * call with others rebuilds it).  Asynchronous on the plan's stream (on the
 * legacy stream: a private stream, synchronised before returning):
 *   mean_params   DEVICE double [q_len]  in: m_{t0-1}; out: m_{t0+T-1}
 *   q_params      DEVICE float  [q_len]  out: parameters matched to the final m
 *   moments       DEVICE double [q_len]  scratch for each iteration's estimate
 *   log_pmp_trace DEVICE double [T][n_inst] log P_MP of every iteration (nullable)
 * Iteration t draws its noise from the stream keyed by (seed, t) and, with
 * sched_p > 0, takes the EMA weight t^-sched_p (Thm. 1), so the state of a run
 * is its mean parameters and its next t: a run of T1 iterations (t0 = 1)
 * followed by a run of T2 from t0 = T1 + 1 on the saved mean parameters gives
 * the same bits as one run of T1 + T2 (checkpoint and resume).  t0 >= 1.   */
qem_status qem_run(qem_plan_t plan, int64_t T, int64_t t0, double lambda, double sched_p, uint64_t seed,
                   double* mean_params, float* q_params, double* moments, double* log_pmp_trace);

/* Autotuning of the launch shapes (sampler and moments block sizes; FP32
 * contraction rows per block and staged child samples; the tensor-core
 * schedules of the forward and the adjoint): a coordinate search
 * timing whole E-steps on q_params (DEVICE float [q_len]) on the plan's
 * stream, keeping a candidate only when it is at least 3% faster; results do
 * not depend on the choice beyond rounding order of the FP32 contraction.
 * The choice is cached per shape signature for the process, and in the file
 * named by the environment variable QEM_TUNE_CACHE when set; a cached
 * choice is applied without timing unless flags has QEM_TUNE_FORCE.  Runs
 * E-steps and allocates q_len doubles of scratch; synchronises the stream;
 * QEM_ERR_INVALID_ARG while the stream is being captured.  Plans made with
 * tile = QEM_TILE_AUTO call it on their first qem_estep / qem_run outside a
 * capture.  No counterpart in the paper (launch configuration only).        */
qem_status qem_tune(qem_plan_t plan, const float* q_params, int flags);

/* Apply launch shapes without timing (HOST int [5], the layout qem_tune_get
 * returns; every value one of the tuner's candidates, QEM_ERR_INVALID_ARG
 * otherwise): results depend on the choice only through the rounding order
 * of the FP32 contraction.  Synchronises the plan's stream; drops qem_run's
 * cached graph.  No counterpart in the paper (launch configuration only).   */
qem_status qem_tune_set(qem_plan_t plan, const int* params);

/* The plan's launch shapes: HOST int [5] = sampler threads per block, moments
 * threads per block, FP32 contraction rows per block, FP32 staged child
 * samples, tensor-core schedules (bit 0: the forward keeps a whole element's
 * operand rows in shared memory while the parent's row blocks stream; bit 1:
 * the adjoint keeps the element's rows, four row blocks per pass, while the
 * parent's kept rows stream; each used when its operands fit; a clear bit:
 * one row block per CTA, the other operand streamed).  Default 1.           */
qem_status qem_tune_get(qem_plan_t plan, int* params);

/* ------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper: an amortised proposal
 * network, plain QEM continuing from its prediction).  For a user of the
 * hierarchical logistic model (dim = QEM_MLP_DIM) with items (x_n, y_n):
 *   features f = [sum_n x_n y_n (D), sum_n x_n (D), sum_n y_n]        (2D+1)
 *   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3        (2D)
 *   q = N(o[:D], diag exp(o[D:])^2)
 * trained on the KL divergence from the user's QEM proposal N(m, diag s^2)
 * to q (mean over users, summed over dimensions).  Matrix-product operands
 * are rounded to BF16, products accumulate in FP32.  Parameters: DEVICE
 * float [QEM_MLP_PARAMS], W1 [H][2D+1], b1 [H], W2 [H][H], b2 [H],
 * W3 [2D][H], b3 [2D] (row-major, rows = outputs).  All calls are
 * asynchronous on `stream` (a cudaStream_t, NULL = default stream).       */
#define QEM_MLP_DIM 18
#define QEM_MLP_HIDDEN 128
#define QEM_MLP_PARAMS 26020

/* Features of n users: x DEVICE float [n][n_obs][dim], y DEVICE float
 * [n][n_obs] -> feats DEVICE float [n][2 dim + 1].  dim must be QEM_MLP_DIM
 * (QEM_ERR_UNSUPPORTED otherwise).                                           */
qem_status qem_mlp_features(const float* x, const float* y, int64_t n, int n_obs, int dim, float* feats,
                            void* stream);

/* Network output of n users: feats DEVICE float [n][2D+1] -> out DEVICE
 * float [n][2D] (means, then log scales).                                    */
qem_status qem_mlp_forward(const float* params, const float* feats, int64_t n, float* out, void* stream);

/* Bytes of the caller-owned workspace qem_mlp_backward needs for n users
 * (per-block partial gradients).                                             */
qem_status qem_mlp_workspace_size(int64_t n, size_t* bytes);

/* Loss and gradient of a batch of n >= 1 users: target DEVICE float
 * [n][2][D] (the users' QEM proposal: means, then scales > 0, the plan's
 * q_params layout) -> grad DEVICE float [QEM_MLP_PARAMS], loss DEVICE double
 * [1] (nullable).  Deterministic: blocks' partial sums are added in order. */
qem_status qem_mlp_backward(const float* params, const float* feats, const float* target, int64_t n, float* grad,
                            double* loss, void* workspace, void* stream);

/* One Adam step t >= 1 (Kingma & Ba 2015) on params with FP32 moment
 * estimates m, v (DEVICE float [QEM_MLP_PARAMS] each, zero before t = 1). */
qem_status qem_mlp_step(float* params, const float* grad, float* m, float* v, int64_t t, double lr, double beta1,
                        double beta2, double eps, void* stream);

/* Proposal parameters from the network output: out DEVICE float [n][2D] ->
 * q_params DEVICE float [n][2][D] (means; scales = exp of the log scales,
 * clamped to [-12, 6]), ready to be copied into a plan's q_params.          */
qem_status qem_mlp_to_q(const float* out, int64_t n, float* q_params, void* stream);

/* Kernels of the plan's qem_run graph (tracing support; valid after a
 * qem_run call): per_iteration = kernel launches of one iteration inside the
 * device loop (the E-step, the M-step and the loop control), per_call = the
 * kernels each qem_run call launches outside the loop.                        */
qem_status qem_run_kernels(qem_plan_t plan, int64_t* per_iteration, int64_t* per_call);

/* Work of the last E-step's adjoint (tracing support, not part of the
 * method): the (kept parent sample, child sample) pairs over every element
 * below the root, where a parent keeps the samples whose weight is at least
 * 2^-40 (FP32 plans) or 2^-24 (mixed-precision plans) of its largest (the
 * adjoint's compaction); kept_tc counts those of parents keeping more than
 * four samples on a mixed-precision plan (the tensor-core adjoint's share).
 * Chain plates are not counted.  HOST doubles, either may be NULL;
 * synchronises the plan's stream.                                          */
qem_status qem_adjoint_pairs(qem_plan_t plan, double* kept_tc, double* kept_all);

/* Kernel classes of the per-kernel profiler. */
enum {
  QEM_K_SAMPLE = 0,      /* sampling and local factors                 */
  QEM_K_PARENT = 1,      /* conditional parameters of children         */
  QEM_K_FINALIZE = 2,    /* relative local factors of inner levels     */
  QEM_K_FORWARD = 3,     /* forward K x K contraction                  */
  QEM_K_PLATE_SUM = 4,   /* FP64 plate sums                            */
  QEM_K_ROOT = 5,        /* root log P_MP and weights                  */
  QEM_K_ADJOINT = 6,     /* adjoint K x K contraction (marginals)      */
  QEM_K_MOMENTS = 7,     /* moments                                    */
  QEM_K_MSTEP = 8,       /* EMA + M-step                               */
  QEM_K_OPERANDS = 9,    /* tensor-core operand features / compaction  */
  QEM_K_ADJ_SMALL = 10,  /* adjoint of parents keeping few samples (CUDA cores, mixed-precision plans) */
  QEM_K_COUNT = 11
};

/* Per-kernel timing (tracing support, not part of the method): while enabled,
 * every kernel the plan launches from qem_estep / qem_mstep is bracketed by
 * CUDA events on the plan's stream.  on = 1 clears previous records and
 * enables; on = 0 disables (records are kept).  qem_run is never profiled. */
qem_status qem_profile_enable(qem_plan_t plan, int on);

/* Accumulated device time (ms) and launch count of kernel class `kind`
 * (QEM_K_*) over the records since the last enable.  Synchronises the plan's
 * stream.  Either output pointer (HOST) may be NULL.                       */
qem_status qem_profile_read(qem_plan_t plan, int kind, double* ms, int64_t* launches);

/* Name of a kernel class (static storage), or NULL for an invalid class. */
const char* qem_profile_name(int kind);

/* Diagnostic (validation of the tensor-core operand path, not part of the
 * method): out = A * B^T computed by one tcgen05 MMA chain exactly as the
 * contraction kernels issue it.
 *   A    DEVICE bf16 [128 rows][fk] in the canonical K-major core-matrix
 *        layout (element (r, c) at ((r/8)*(fk/8) + c/8)*64 + (r%8)*8 + c%8)
 *   B    DEVICE bf16 [n rows][fk], same layout
 *   out  DEVICE float [128][n] row-major
 * fk in 16..128 and n in 16..256, both multiples of 16.  Synchronous on
 * `stream`; allocates and frees a small control block.                      */
qem_status qem_diag_tc_gemm(const void* A, const void* B, int fk, int n, float* out, void* stream);

/* Allocation-free E-step for single-level models (every instance has one
 * latent, no plate below it).  The paper has no counterpart of this entry
 * point.  It is for callers that cannot allocate device memory at the moment
 * they need an E-step: a runtime whose memory pool forbids allocations from
 * outside it, or a real-time loop that cannot afford an allocation's latency
 * and implicit device synchronisation.  It allocates nothing, on the device
 * or the host.
 *   level      HOST descriptor of the single level (parent must be NULL; x, y DEVICE)
 *   q_params   DEVICE float [n][2][D]; eps DEVICE float [n][K][nps] or NULL
 *   moments    DEVICE double [n][2][D] out; log_pmp DEVICE double [n] out (nullable)
 *   stream     cudaStream_t (NULL: legacy default stream), asynchronous
 * Scratch lives in one library-wide device array of 32 MiB, held by every GPU
 * that loads the library until the process exits: requests needing more
 * (about n*K*(D+2)*4 bytes) return QEM_ERR_UNSUPPORTED.  Every call shares
 * that array and it keeps the last call's contents (each call writes what it
 * reads first); calls whose GPU work overlaps (other streams, other host
 * threads) race on it.  The first call on a device looks the array's address
 * up (cudaGetSymbolAddress) with that device current and keeps it for the
 * process; make that first call before any stream capture, and make no call
 * after a cudaDeviceReset (the kept address then names released memory).
 * The call is asynchronous and cannot report a non-finite log P_MP: pass
 * log_pmp and check its values.  Moments and log P_MP equal qem_estep's on
 * the same single-level model and inputs.                                   */
qem_status qem_estep_single_noalloc(const qem_level_desc* level, int K, const float* q_params, const float* eps,
                                    uint64_t seed, uint64_t iter, double* moments, double* log_pmp, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QEM_H */
