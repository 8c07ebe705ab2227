/*
 * crl.h -- C ABI of libcrl, a GB300 (sm_103a) implementation of the
 * contrastive-RL (CRL) update step of arXiv 2408.11052 ("JaxGCRL").
 *
 * One update step (Algorithm 1, App. F, inner loop body) is:
 *   insert new time slices into the replay buffer,
 *   sample a batch with hindsight future-state goals (§3.1, §3.2),
 *   critic step: phi(s,a), psi(g) encoders, B x B energy matrix, InfoNCE +
 *                beta * logsumexp penalty, backward, Adam (§3.1, App. A.2),
 *   actor step:  tanh-Gaussian policy, DDPG-style objective with entropy term
 *                (Eq. 3, §5.1), backward, Adam.
 *
 * Conventions (all entry points)
 * ------------------------------
 * - Every call returns CRL_OK (0) or a negative CRL_E_* code.  Nothing aborts
 *   and no C++ exception crosses this boundary.  crl_last_error() gives a
 *   human-readable message for the last failing call on the same context (or,
 *   for calls without a context, on the calling thread).
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Calls are asynchronous on that stream unless stated otherwise.
 * - Pointers are device pointers unless the entry point says "host or
 *   device"; those accept pinned or pageable host memory as well, detected
 *   with cudaPointerGetAttributes, and the library stages the copy itself.
 * - Matrices are dense, row-major, with the leading dimension equal to the
 *   row length unless a separate ld argument is given.
 * - Device-side failures (a non-finite loss, an index outside the buffer)
 *   do not stop the stream; kernels set bits of a device status word that
 *   crl_sync_status() reads and clears.
 * - The library owns the replay buffer and its workspaces (allocated by
 *   crl_create, freed by crl_destroy).  The caller owns parameters, gradients,
 *   Adam moments and batch tensors, and keeps them alive while work that uses
 *   them is in flight.
 */
#ifndef CRL_H_
#define CRL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define CRL_OK 0
#define CRL_E_INVALID_ARG (-1)   /* null pointer, value outside its range    */
#define CRL_E_SHAPE (-2)         /* sizes inconsistent with the config       */
#define CRL_E_BUFFER_EMPTY (-3)  /* sampling from an empty replay buffer     */
#define CRL_E_CUDA (-4)          /* a CUDA runtime call failed               */
#define CRL_E_NONFINITE (-5)     /* device status: non-finite loss           */
#define CRL_E_TIMEOUT (-6)       /* device status: a bounded wait gave up    */
#define CRL_E_NOT_BOUND (-7)     /* step called before crl_bind_params       */
#define CRL_E_UNSUPPORTED (-8)   /* option combination not implemented       */

/* device status bits (crl_sync_status) */
#define CRL_STATUS_NONFINITE 1u
#define CRL_STATUS_BAD_INDEX 2u
#define CRL_STATUS_TIMEOUT 4u

/* ---- enumerations ---------------------------------------------------- */
/* Energy functions, App. A.2: f = <x,y>/(|x||y|), <x,y>, -|x-y|_1,
 * -|x-y|_2 (the sign of App. A.2), -|x-y|_2^2; all divided by temperature. */
#define CRL_ENERGY_L2 0
#define CRL_ENERGY_DOT 1
#define CRL_ENERGY_COS 2
#define CRL_ENERGY_L1 3
#define CRL_ENERGY_L2SQ 4
/* InfoNCE direction, App. A.2: forward (softmax over goals), backward
 * (softmax over state-actions), symmetric (both). */
#define CRL_LOSS_FWD 0
#define CRL_LOSS_BWD 1
#define CRL_LOSS_SYM 2
/* The other contrastive objectives of App. A.2 / §5.2, over F_ij = f(s_i, a_i,
 * g_j) / temperature with the positives on the diagonal; each also takes the
 * logsumexp penalty (§5.2 adds it to every objective).
 *   FLATNCE_FWD / _BWD: S_i = sum_j exp(F_ij - F_ii) over goals j (FWD) or
 *     S_i = sum_j exp(F_ji - F_ii) over state-actions j (BWD), j = i included;
 *     the loss log(S_i / detach S_i) has the value 0 and (reading: the printed
 *     leading minus is a sign slip) the gradient of mean_i log S_i, which equals
 *     InfoNCE's of the same direction.
 *   FB: Monte Carlo forward-backward, mean_i [-exp(F_ii) + sum_{j != i}
 *     exp(F_ij)^2 / (2 (B - 1))]; needs B >= 2 (CRL_E_SHAPE otherwise).
 *   DPO: mean over all B^2 pairs of -log sigma(F_ii - F_ij).
 *   IPO: mean over all pairs of (F_ii - F_ij - 1)^2.
 *   SPPO: mean over all pairs of (F_ii - 1)^2 + (F_ij + 1)^2.
 *   NCE_BINARY (named in §5.2, not defined there; reading: binary
 *     cross-entropy of sigma(F_ij) against the label [i = j], mean over pairs).
 * For these, loss4 = {objective + penalty, InfoNCE forward value, InfoNCE
 * backward value, penalty}: the InfoNCE values are diagnostics.  Every path
 * takes every objective. */
#define CRL_LOSS_FLATNCE_FWD 3
#define CRL_LOSS_FLATNCE_BWD 4
#define CRL_LOSS_FB 5
#define CRL_LOSS_DPO 6
#define CRL_LOSS_IPO 7
#define CRL_LOSS_SPPO 8
#define CRL_LOSS_NCE_BINARY 9
/* symmetric reduction: mean of the two directions, or their sum (App. A.2) */
#define CRL_SYM_MEAN 0
#define CRL_SYM_SUM 1
/* logsumexp penalty (Algorithm 1; not defined in the paper): beta times the
 * batch mean of the squared row logsumexp (ROW), column logsumexp (COL), or
 * the average of both (BOTH). */
#define CRL_PENALTY_ROW 0
#define CRL_PENALTY_COL 1
#define CRL_PENALTY_BOTH 2
/* arithmetic of the encoder / energy path */
#define CRL_PREC_FP32 0   /* FP32 SIMT kernels                                    */
#define CRL_PREC_BF16 1   /* BF16 tensor-core GEMMs (tcgen05), FP32 accumulate    */
#define CRL_PREC_FP64 2   /* FP64 SIMT kernels: the finite-difference check path */
/* kernel organisation */
#define CRL_PATH_PLAIN 0  /* one kernel per op; the B x B energy matrix in HBM */
#define CRL_PATH_FUSED 1  /* fused kernels; the B x B matrix is never written   */
                          /* (BF16 only; repr 64 / 128 / 192 / 256, B a multiple
                           * of 8; every energy: L1 on FP32 SIMT tiles over the
                           * FP32 representations, the others on tcgen05) */
/* networks */
#define CRL_NET_PHI 0     /* phi(s, a): input concat(s, a), output repr        */
#define CRL_NET_PSI 1     /* psi(g):    input g, output repr                   */
#define CRL_NET_PI 2      /* pi(s, g):  input concat(s, g), output 2A (mu, log std) */

#define CRL_STEP_AUTO UINT64_MAX  /* use (and advance) the context's step counter */
#define CRL_MAX_GOAL_DIMS 16
#define CRL_MAX_LAYERS 8

/* ---- configuration ----------------------------------------------------- */
/* Sizes and hyperparameters of one agent.  Names follow App. B.3 where the
 * paper has them.  All fields are read once by crl_create. */
typedef struct crl_config {
  int32_t E;            /* parallel environments (buffer rows), >= 1                  */
  int32_t T;            /* stored steps per environment (ring capacity), >= 1        */
  int32_t D;            /* observation dim, >= 1                                    */
  int32_t A;            /* action dim, >= 1                                         */
  int32_t G;            /* goal dim, 1..CRL_MAX_GOAL_DIMS                             */
  int32_t B;            /* maximum batch size, >= 1                                 */
  int32_t hidden;       /* hidden width of phi, psi and pi, >= 1                     */
  int32_t layers;       /* hidden layers, 1..CRL_MAX_LAYERS                           */
  int32_t repr;         /* representation dim R, >= 1                               */
  int32_t goal_idx[CRL_MAX_GOAL_DIMS]; /* goal = obs[goal_idx[0..G-1]], each in [0, D) */
  float gamma;          /* discount in [0, 1): offset ~ Geom(1 - gamma) (§3)          */
  float beta_lse;       /* logsumexp penalty weight (0.1 in App. B.3)                 */
  float temperature;    /* tau > 0; F = f / tau                                     */
  float alpha;          /* entropy coefficient of the actor objective, >= 0          */
  int32_t energy;       /* CRL_ENERGY_*                                             */
  int32_t loss;         /* CRL_LOSS_*                                               */
  int32_t sym_reduction;/* CRL_SYM_*                                                */
  int32_t penalty_axis; /* CRL_PENALTY_*                                            */
  int32_t layernorm;    /* 1: LayerNorm before every hidden ReLU (§5.4)              */
  int32_t precision;    /* CRL_PREC_*                                               */
  int32_t path;         /* CRL_PATH_*                                               */
  int32_t offset_min;   /* 1: goal offset k in {1..L} (strict future); 0: {0..L}     */
  float lr_critic;      /* 3e-4 in App. B.3                                          */
  float lr_actor;       /* 6e-4 in App. B.3                                          */
  float adam_beta1, adam_beta2, adam_eps;
  uint64_t seed;        /* Philox key word 0                                        */
  uint64_t agent;       /* Philox key word 1 (independent agents)                   */
  /* entropy-coefficient auto-tuning (§5.1 "a tuneable entropy coefficient";
   * the rule is a reading): with alpha_autotune = 1, log(alpha) starts at
   * log(alpha) and after every actor update takes one Adam step (lr_alpha,
   * adam_beta1/2, adam_eps) on  -log(alpha) * (mean log pi + target_entropy)
   * with log pi held fixed; the actor loss of a step uses alpha before that
   * step's update.  crl_get_alpha reads the current value. */
  int32_t alpha_autotune;
  float target_entropy; /* -A by convention (crl_config_default: -8)               */
  float lr_alpha;       /* crl_config_default: 6e-4 (the actor's rate)             */
  /* random-goal actor mix (App. D; 0, the paper's choice, by default): in
   * crl_update_step each sample's actor goal is, with probability alpha_rg,
   * the relabelled goal of sample (b + 1) mod B (a goal of another, independently
   * drawn transition), else its own; the choice is (word 2 of the sample's
   * relabel Philox block) >> 32 < floor(alpha_rg 2^32).  The critic always
   * takes the relabelled goals (single agents and every kind of sweep). */
  float alpha_rg;
} crl_config;

/* Fill *cfg with the paper's defaults (App. B.3: batch 256, gamma 0.99,
 * 2 x 256 hidden, repr 64, L2 energy, symmetric InfoNCE, penalty 0.1,
 * lr 3e-4 / 6e-4) and Ant-like sizes (E 1024, T 1000, D 29, A 8, G 2);
 * fixed alpha 0.1 (alpha_autotune 0). */
void crl_config_default(crl_config* cfg);

/* ---- parameter layout ---------------------------------------------------- */
/* Each network's parameters live in ONE caller-owned flat array (float for
 * FP32/BF16 contexts, double for FP64).  Tensor i of network `net`:
 *   hidden layer l (0..layers-1): W_l [out][in], b_l [out]
 *       and, with layernorm, ln_gain_l [out], ln_bias_l [out];
 *   then the output layer W_out [out][in], b_out [out].
 * W is stored like torch.nn.Linear.weight.  Each tensor starts at a multiple
 * of 64 elements.  Gradients and the two Adam moments use the same layout. */
typedef struct crl_tensor_info {
  int64_t offset;       /* in elements from the start of the flat array */
  int32_t rows, cols;   /* cols == 1 for vectors                         */
  int32_t kind;         /* 0 W, 1 b, 2 ln_gain, 3 ln_bias                */
  int32_t layer;        /* 0..layers (layers = output layer)             */
} crl_tensor_info;

/* Number of elements of network `net`'s flat array (padding included). */
int crl_param_count(const crl_config* cfg, int32_t net, int64_t* count);
/* Number of tensors of network `net`. */
int crl_param_tensors(const crl_config* cfg, int32_t net, int32_t* n);
/* Description of tensor i of network `net`; CRL_E_INVALID_ARG when i is out of range. */
int crl_param_tensor(const crl_config* cfg, int32_t net, int32_t i, crl_tensor_info* out);

/* ---- context ------------------------------------------------------------ */
typedef struct crl_ctx crl_ctx;

/* Validate cfg, allocate the replay buffer (E x T rows of roundup(D+A+1, 4)
 * floats) and all workspaces on the current device, build the discount table.
 * Synchronous.  *out is NULL on failure. */
int crl_create(const crl_config* cfg, crl_ctx** out);
/* Free everything crl_create allocated (synchronises the device first).  NULL is a no-op. */
int crl_destroy(crl_ctx* ctx);

/* Caller-owned parameter storage of one network: params, grads, Adam m and v,
 * each a flat array of crl_param_count elements (device pointers). */
typedef struct crl_net_ptrs {
  void* params;
  void* grads;
  void* adam_m;
  void* adam_v;
} crl_net_ptrs;
/* Bind the three networks (index CRL_NET_*).  Moments must start at zero for
 * a fresh optimiser.  Resets the Adam step counters to 0.  Every array must
 * start on a 16-byte boundary (CRL_E_INVALID_ARG otherwise). */
int crl_bind_params(crl_ctx* ctx, const crl_net_ptrs nets[3]);

/* ---- replay buffer (Algorithm 1 "store trajectory"; App. B.3 capacity) -----
 * Append n time slices for all E environments at once:
 *   obs [n][E][D] float, act [n][E][A] float, done [n][E] uint8 (nonzero: that
 *   step's observation is the last of its episode).  Host or device pointers:
 *   pinned (page-locked, mapped) host memory is read by the insert kernel in
 *   place over the CPU-GPU link; pageable host memory is copied to a staging
 *   buffer first.  Either way the call is asynchronous on `stream` and host
 *   inputs must stay valid and unchanged until the stream has passed it.
 * The ring keeps the newest T steps per environment.  n >= 1. */
int crl_buffer_insert(crl_ctx* ctx, const float* obs, const float* act, const uint8_t* done,
                      int32_t n, void* stream);
/* Host-side view of the ring fill: stored steps per env and steps ever inserted. */
int crl_buffer_size(const crl_ctx* ctx, int32_t* size, int64_t* total);

/* ---- sample + relabel (§3.1, §3.2, Algorithm 1 "sample with discount") -----
 * For b in [0, B): Philox4x64-10 block at counter (step, b, 0, 0) under key
 * (seed, agent); word 0 picks the stored transition (e, t) uniformly, the top
 * 32 bits of word 1 pick the goal offset k from the geometric distribution
 * with parameter 1 - gamma truncated to the episode (exact integer inverse
 * CDF).  Writes s [B][D] = obs[e][t], a [B][A] = act[e][t],
 * g [B][G] = obs[e][t+k][goal_idx] and, if idx != NULL, idx [B][3] = (e, t, k)
 * with t counted from the oldest stored step.  step == CRL_STEP_AUTO uses the
 * context's device step counter and advances it.  Device pointers.  B may
 * exceed cfg.B (the outputs are the caller's; B x D < 2^31).
 * CRL_E_BUFFER_EMPTY if nothing is stored; CRL_E_SHAPE if B < 1. */
int crl_sample_relabel(crl_ctx* ctx, uint64_t step, int32_t B, float* s, float* a, float* g,
                       int32_t* idx, void* stream);

/* ---- critic step (§3.1 critic objective, App. A.2, Algorithm 1) -----------
 * phi = phi(concat(s, a)), psi = psi(g); F_ij = f(phi_i, psi_j) / tau;
 * loss = InfoNCE(F) + beta * penalty.  Writes the gradient of every phi and
 * psi parameter into the bound grads arrays; with apply_update != 0 then
 * applies Adam (lr_critic) to phi and psi.
 * s [B][D], a [B][A], g [B][G] device.  loss_out: 4 floats {total,
 * InfoNCE-fwd, InfoNCE-bwd, penalty}, host or device, or NULL. */
int crl_critic_step(crl_ctx* ctx, const float* s, const float* a, const float* g, int32_t B,
                    int32_t apply_update, float* loss_out, void* stream);

/* ---- actor step (Eq. 3, §3.2; App. C with random-goal weight 0) -----------
 * (mu, l) = pi(concat(s, g)), l clipped to [-5, 2], a' = tanh(mu + exp(l) eps);
 * loss = mean(alpha * log pi(a'|s,g) - F(phi(s, a'), psi(g))) with the critic
 * as currently stored (the critic is not changed).  Writes the actor
 * gradient; with apply_update != 0 applies Adam (lr_actor).
 * eps [B][A] device, or NULL to draw N(0,1) noise from Philox at counter
 * (step, b, 1, 0) with the step counter of the last sample (Box-Muller).
 * loss_out: 2 floats {actor loss, mean log pi}, host or device, or NULL. */
int crl_actor_step(crl_ctx* ctx, const float* s, const float* g, const float* eps, int32_t B,
                   int32_t apply_update, float* loss_out, void* stream);

/* ---- one full update step ----------------------------------------------
 * insert (if n_insert > 0) -> sample_relabel (CRL_STEP_AUTO) -> critic step
 * -> actor step (Philox noise), with Adam for both; the batch lives in
 * library workspaces.  obs/act/done as crl_buffer_insert (host or device).
 * loss_out: 6 floats {critic total, fwd, bwd, penalty, actor loss,
 * mean log pi}, host or device, or NULL.  B = cfg.B.
 * From the second call on a non-default stream (and while tracing is off) the
 * relabel -> critic -> actor sequence is captured once as a CUDA graph and
 * replayed; crl_bind_params discards the graph.  Between crl_update_step
 * calls the library assumes it is the only writer of the parameters (the
 * BF16 weight shadows follow them through Adam); after changing parameters
 * from outside, call crl_bind_params again. */
int crl_update_step(crl_ctx* ctx, const float* obs, const float* act, const uint8_t* done,
                    int32_t n_insert, float* loss_out, void* stream);

/* Device step counter used by CRL_STEP_AUTO (readable / settable for resume). */
int crl_get_step(crl_ctx* ctx, uint64_t* step);
int crl_set_step(crl_ctx* ctx, uint64_t step);

/* Synchronise `stream`, read the device status word into *status (CRL_STATUS_*
 * bits) and clear it.  Returns CRL_E_NONFINITE / CRL_E_TIMEOUT when those bits
 * are set, CRL_OK otherwise. */
int crl_sync_status(crl_ctx* ctx, void* stream, uint32_t* status);
/* Bound of every device wait of the context's tensor-core kernels (GEMMs and
 * fused energy stage), in nanoseconds; 0 restores the default of one second
 * (library extension; the paper has no counterpart).  A wait that runs out
 * sets CRL_STATUS_TIMEOUT; the kernel then waits (at most a second more) for
 * its own copies and MMAs in flight, frees its tensor memory and returns, so
 * the context stays usable: the outputs of that step are undefined and
 * crl_sync_status reports CRL_E_TIMEOUT.  Limits below 100 us poll without
 * suspending the waiting thread, so even a limit of a few nanoseconds runs
 * out.  The limit lives in device memory next to the status word: captured
 * step graphs see a new value on their next replay.  Synchronises the device
 * (so not during stream capture: CRL_E_CUDA). */
int crl_set_wait_limit_ns(crl_ctx* ctx, uint32_t ns);
/* The entropy coefficient the next actor step will use: exp(log alpha) with
 * auto-tuning, else cfg.alpha.  Synchronous read. */
int crl_get_alpha(crl_ctx* ctx, float* alpha);

/* ---- collection stub (Algorithm 1's loop over environments) -------------
 * The simulator is outside this library; this call stands in for it with
 * synthetic dynamics so that the update-to-data loop (§5.6) runs end to end
 * on the device.  n_steps environment steps for all E environments, each:
 * a = tanh(mu + sigma eps) from the policy pi(s, g) (the actor's head, noise
 * from its own Philox stream), the slice (s, a, done) appended to the replay
 * buffer (done on an episode's last step, t = episode_length - 1), then
 * s' = s + 0.1 xi + 0.05 a[d mod A] (xi ~ N(0, I)), or after an episode's last
 * step a fresh s' ~ N(0, I) with a fresh commanded goal g' ~ N(0, I) [G].
 * The first call draws every environment's first state and goal.  All draws:
 * Box-Muller on Philox4x64-10 blocks (step, env, word, d / 4) keyed (seed,
 * agent), words 2 (action), 3 (dynamics), 4 (reset state), 5 (reset goal); the
 * collection counter starts at 0, the first states use 2^64 - 1.
 * obs_out [n_steps][E][D], act_out [n_steps][E][A], done_out [n_steps][E]
 * (device, optional): the slices inserted.  Async on `stream`. */
int crl_collect(crl_ctx* ctx, int32_t n_steps, int32_t episode_length, float* obs_out, float* act_out,
                uint8_t* done_out, void* stream);

/* ---- checkpoint / resume --------------------------------------------------
 * The library-owned training state of ctx as one host blob: the replay buffer
 * (rows, episode starts, fill and insert count), the device counters (the
 * CRL_STEP_AUTO step, the last sampled step, the Adam step counts of critic
 * and actor, the tuned log alpha with its Adam moments) and, once crl_collect
 * has run, the collection stub's environments (states, goals, episode steps,
 * collection counter).  Parameters, gradients and Adam moments are the
 * caller's memory and are saved by the caller.  Because every draw of the
 * method (relabel offsets, actor noise, goal mix, collection) is a
 * counter-based Philox block of (seed, agent, step), a context created with
 * the same config, bound to the saved parameters and moments and given this
 * blob continues bit-identically to the one that saved it.  (A library
 * extension: the paper describes no checkpoint format.)
 * crl_state_bytes: size of the blob now (it grows once crl_collect has run).
 * crl_save_state: synchronises the device, writes the blob to `host` (host
 *   memory, >= crl_state_bytes, else CRL_E_SHAPE).
 * crl_load_state: synchronises the device, checks the blob's magic and sizes
 *   (CRL_E_INVALID_ARG if it is not a blob of this library or is corrupt,
 *   CRL_E_SHAPE if it comes from a context of other sizes or is truncated),
 *   restores the state, drops the captured update graph and refreshes the
 *   BF16 weight shadows at the next step.  A blob carrying environments needs
 *   bound parameters (CRL_E_NOT_BOUND). */
int crl_state_bytes(crl_ctx* ctx, size_t* bytes);
int crl_save_state(crl_ctx* ctx, void* host, size_t bytes);
int crl_load_state(crl_ctx* ctx, const void* host, size_t bytes);

/* ---- logit statistics (library diagnostic) --------------------------------
 * With on != 0 every critic step of ctx (crl_critic_step, crl_update_step, a
 * sweep step) also computes, from the representations its energy was formed
 * from, the mean positive-pair logit (1/B) sum_i F_ii and the mean negative
 * logit (1/(B^2 - B)) sum_{i != j} F_ij (NaN for B = 1), F = f(phi_i, psi_j) /
 * tau with the configured energy (§3.1, App. A.2).  The representations are the
 * encoders' FP32 outputs (FP64 on the check path); on the fused BF16 path the
 * energy itself is formed from their BF16 rounding.  Cost: one extra pass over
 * the B x B pairs (two launches, deterministic FP64 sums); off by default.
 * crl_get_logit_stats synchronises the device and copies the values of the
 * last such step to out[2] (host memory; NaN before any). */
int crl_set_logit_stats(crl_ctx* ctx, int32_t on);
int crl_get_logit_stats(crl_ctx* ctx, float* out);

/* Message of the last failing call on ctx (ctx == NULL: on this thread). */
const char* crl_last_error(const crl_ctx* ctx);

/* ---- tracing: CUDA-event timing of one class of kernels ------------------
 * After crl_trace_start, every launch of the chosen class made by calls on
 * ctx (up to max_launches) is bracketed by two CUDA events on its stream, and
 * its algorithmic work is added up: flops for GEMM / ENERGY (2 M N K per
 * product), bytes moved for INSERT / RELABEL / ADAM / AUX.  crl_trace_stop
 * synchronises those events and returns the launch count, the summed kernel
 * time in milliseconds and the summed work, then disables tracing.  Launches
 * beyond max_launches are not counted. */
#define CRL_TRACE_INSERT 1   /* buffer insert + episode close                 */
#define CRL_TRACE_RELABEL 2  /* sample + relabel gather                       */
#define CRL_TRACE_GEMM 3     /* encoder / actor MLP products                  */
#define CRL_TRACE_ENERGY 4   /* energy matrix, InfoNCE and their backward      */
#define CRL_TRACE_ADAM 5     /* Adam updates                                  */
#define CRL_TRACE_AUX 6      /* LayerNorm, reductions, actor head, counters   */
int crl_trace_start(crl_ctx* ctx, int32_t kernel_class, int32_t max_launches);
int crl_trace_stop(crl_ctx* ctx, int32_t* launches, double* total_ms, double* work);

/* ---- batched sweep (library extension: the paper trains one agent per run;
 * its multi-seed experiments, §5, become one GPU program) -------------------
 * A sweep owns n independent agents (1 <= n <= 64), each a full context built
 * from cfgs[i] (its own replay buffer, networks and Philox key (seed, agent)).
 * The agents share precision, path, hidden width, depth and LayerNorm; batch,
 * obs / action / goal dims, buffer size, repr and hyperparameters may differ.
 * grouped = 1 (BF16 fused only): every kernel of the update step is one launch
 * over all agents (grouped tcgen05 GEMMs over every agent's networks of a
 * layer; block-offset tables for the other kernels).  grouped = 0 (any
 * precision): the agents' update steps one after another.  Each agent's
 * results are those of crl_update_step on that agent alone.
 * CRL_E_INVALID_ARG / CRL_E_UNSUPPORTED on mismatched or unsupported configs. */
typedef struct crl_sweep crl_sweep;
int crl_sweep_create(const crl_config* cfgs, int32_t n, int32_t grouped, crl_sweep** out);
int crl_sweep_destroy(crl_sweep* sw);     /* destroys the agents' contexts too */
/* Agent i's context, owned by the sweep (do not crl_destroy it): bind its
 * parameters, fill its buffer, read its state with the single-agent calls.
 * Re-binding an agent's parameters makes the next sweep step rebuild its
 * launch tables and graph. */
int crl_sweep_agent(crl_sweep* sw, int32_t i, crl_ctx** ctx);
/* One update step of every agent (crl_update_step per agent): insert n_insert
 * time slices into each agent's buffer (obs[i] [n][E_i][D_i], act[i], done[i]
 * as crl_buffer_insert; device pointers go into one launch, host pointers are
 * staged per agent; arrays may be NULL when n_insert = 0), then relabel,
 * critic + Adam, actor + Adam.  The step after the first is captured once as a
 * CUDA graph on `stream` (not the legacy default stream) and replayed.
 * loss_out: [n][6] floats (the crl_update_step layout per agent), host or
 * device, or NULL. */
int crl_sweep_update_step(crl_sweep* sw, const float* const* obs, const float* const* act,
                          const uint8_t* const* done, int32_t n_insert, float* loss_out, void* stream);
/* Tracing a sweep: crl_trace_start / crl_trace_stop on agent 0's context
 * record every launch of the sweep step (the step then runs eagerly). */
/* OR of the status words of the sweep's shared launches and of every agent
 * (read and cleared); the return code as crl_sync_status. */
int crl_sweep_sync_status(crl_sweep* sw, void* stream, uint32_t* status);
const char* crl_sweep_last_error(const crl_sweep* sw);

/* ---- launch overlap (library extension; the paper has no counterpart) -----
 * Process-wide.  enable = 1 (the default): every kernel of the library is
 * launched with programmatic stream serialisation, so it is scheduled while
 * its predecessor on the stream drains and waits on the device
 * (griddepcontrol.wait) before it touches memory; results are identical.
 * enable = 0: plain stream order.  Takes effect for launches made (and CUDA
 * graphs captured) after the call; a context whose update-step graph was
 * captured before keeps replaying it.  Returns the previous setting. */
int32_t crl_set_launch_overlap(int32_t enable);

/* ---- tile autotuning (library extension; the paper has no counterpart) ----
 * Process-wide.  enable = 1 (the default): the first eager launch of each
 * distinct grouped tensor-core GEMM (a problem list: sizes, operands,
 * epilogue) times the tile widths 64, 128 and 256 on the launch itself
 * (repeating it is harmless: its outputs are a pure function of inputs it
 * does not modify) and keeps the fastest for that context or sweep; outputs
 * do not depend on the pick.  (The weight gradients of batches of 4096 and
 * more split the batch over several CTAs; the split follows from the
 * problem's shape alone, and such a launch is tuned over the one-tile kernel
 * only, the one that splits.)  enable = 0: a fixed rule (128-wide tiles when
 * they fill the GPU, else 64).  Never tunes during graph capture or tracing.
 * Returns the previous setting. */
int32_t crl_set_autotune(int32_t enable);

/* Which tensor-core GEMM kernels the grouped launches may use (process-wide;
 * library extension): CRL_GEMM_ANY (the default; the autotuner picks among
 * all three), CRL_GEMM_ONE_TILE (one CTA per output tile), CRL_GEMM_PERSISTENT (one
 * CTA per SM walking the tiles, its epilogue overlapping the next tile's
 * main loop through a double-buffered TMEM accumulator), CRL_GEMM_CTA_PAIR
 * (the persistent schedule over 256-row tiles, each computed by a cluster of
 * two CTAs with tcgen05.mma.cta_group::2; every CTA loads its own half of the
 * operands, no multicast).  All kernels give identical outputs, except the
 * weight gradients of batches of 4096 and more, which only the one-tile kernel
 * splits over the batch (the other two sum them unsplit: the same values up
 * to FP32 rounding).  Without
 * autotuning the fixed rule picks the tile width and this setting the kernel
 * (ANY: one tile per CTA).  Returns the previous setting, or
 * CRL_E_INVALID_ARG for an unknown mode. */
#define CRL_GEMM_ANY 0
#define CRL_GEMM_ONE_TILE 1
#define CRL_GEMM_PERSISTENT 2
#define CRL_GEMM_CTA_PAIR 3
int32_t crl_set_gemm_kernel(int32_t mode);

/* What the tile autotuner measured (library extension; the paper has no
 * counterpart).  Writes a NUL-terminated JSON array with one object per
 * grouped GEMM problem list the context (or sweep) has tuned so far, in tuning
 * order: "problems" (the list's length), "first_mnk" (M, N, K of its first
 * problem), "gflop" (one launch's algorithmic work), "issued_gflop" (its
 * tensor work as launched: the forward layers multiply BF16 hi / lo pairs of
 * the input and the weights, two to four products per algorithmic one), "picked" (the kept
 * configuration: kernel, tile rows x columns, ring depth) and "us" (each
 * candidate's faster time per launch over the two timing rounds, in
 * microseconds; -1 where it could not be timed).  *needed receives the bytes
 * the report takes including the NUL; call with buf = NULL and len = 0 to ask
 * for it.  Returns CRL_E_SHAPE (nothing written) when 0 < len < *needed.
 * Host memory only; does not touch the device. */
int32_t crl_gemm_tuning_report(crl_ctx* ctx, char* buf, size_t len, size_t* needed);
int32_t crl_sweep_gemm_tuning_report(crl_sweep* sw, char* buf, size_t len, size_t* needed);


/* ---- op-level entry points (stateless; used by torch.autograd.Function) ---
 * Same kernels as the step calls.  dtype: CRL_PREC_FP32 (float) or
 * CRL_PREC_FP64 (double) for every floating pointer of the call; inputs x0/x1
 * are float for both. */
typedef struct crl_mlp_desc {
  int32_t in0;          /* columns taken from x0                             */
  int32_t in1;          /* columns taken from x1 (0: no second input)        */
  int32_t hidden, layers, out;
  int32_t layernorm;
  int32_t dtype;        /* CRL_PREC_FP32 or CRL_PREC_FP64                    */
} crl_mlp_desc;

/* Bytes of the activation workspace `saved` for M rows. */
int crl_mlp_saved_bytes(const crl_mlp_desc* d, int32_t M, size_t* bytes);
/* y [M][out] = MLP(concat(x0 [M][in0], x1 [M][in1])) with params in the flat
 * layout above; stores what backward needs in `saved`. */
int crl_mlp_forward(const crl_mlp_desc* d, const void* params, const float* x0, const float* x1,
                    int32_t M, void* y, void* saved, void* stream);
/* Given dy [M][out]: writes dparams (flat layout; overwritten) and, if not
 * NULL, dx0 [M][in0] / dx1 [M][in1].  dparams may be NULL (input gradient only). */
int crl_mlp_backward(const crl_mlp_desc* d, const void* params, const float* x0, const float* x1,
                     int32_t M, const void* saved, const void* dy, void* dparams, void* dx0,
                     void* dx1, void* stream);

typedef struct crl_loss_desc {
  int32_t energy, loss, sym_reduction, penalty_axis;
  float temperature, beta_lse;
  int32_t dtype;        /* CRL_PREC_FP32 or CRL_PREC_FP64 */
  int32_t path;         /* CRL_PATH_*                     */
} crl_loss_desc;

/* Bytes of the workspace of the InfoNCE calls for batch B, repr R. */
int crl_infonce_workspace_bytes(const crl_loss_desc* d, int32_t B, int32_t R, size_t* bytes);
/* loss4 (device, dtype) = {total, fwd, bwd, penalty}; row_lse [B], col_lse [B]
 * (device, dtype).  phi, psi [B][R].  ws: workspace of the size above. */
int crl_infonce_forward(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B, int32_t R,
                        void* loss4, void* row_lse, void* col_lse, void* ws, size_t ws_bytes,
                        void* stream);
/* dphi, dpsi [B][R] = dtotal * d loss4[0] / d(phi, psi), using the row/col
 * logsumexp of the forward call.  dtotal: scalar multiplier. */
int crl_infonce_backward(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B, int32_t R,
                         const void* row_lse, const void* col_lse, double dtotal, void* dphi,
                         void* dpsi, void* ws, size_t ws_bytes, void* stream);

/* Allocation-free variant of crl_infonce_forward (the paper has no
 * counterpart; this is a library service).  For callers that must not
 * allocate device memory when they evaluate the loss -- e.g. a host that
 * fixes its device memory at start-up and forbids allocation afterwards
 * (cudaMalloc can stall on a device-wide synchronisation and fragments
 * memory), or a plugin inside a runtime that owns the device allocator.
 * Same arguments and results as crl_infonce_forward, minus the workspace: the
 * scratch is a fixed 4 MiB array inside the library, held on every GPU that
 * loads it until the process exits; sizes whose scratch would exceed it
 * (crl_infonce_workspace_bytes > 4194304, e.g. B > ~900 at R = 64 in FP32)
 * are rejected with CRL_E_SHAPE.  Allocates nothing (no cudaMalloc/cudaFree).
 * The first call on each device does a one-time set-up (looks up the array's
 * device address); make that first call before any stream capture.  Every
 * call shares the one array: calls whose work may overlap on the GPU (other
 * streams or threads without ordering) race and give wrong results.  The
 * array's device address is cached per device: do not call this on a device
 * after cudaDeviceReset.  Descriptor checks and error codes are those of
 * crl_infonce_forward; dtype CRL_PREC_FP32 / CRL_PREC_FP64, path
 * CRL_PATH_PLAIN (else CRL_E_UNSUPPORTED). */
int crl_infonce_forward_noalloc(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B, int32_t R,
                                void* loss4, void* row_lse, void* col_lse, void* stream);

/* One Adam step on n elements at step number t (1-based), dtype as above. */
int crl_adam_update(int32_t dtype, void* params, const void* grads, void* m, void* v, int64_t n,
                    int32_t t, float lr, float beta1, float beta2, float eps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CRL_H_ */
