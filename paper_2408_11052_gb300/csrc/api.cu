// C ABI of libcrl (include/crl.h): context management, argument checking and
// the orchestration of one CRL update step (arXiv 2408.11052, Algorithm 1):
// buffer insert -> sample + relabel -> critic step (+ Adam) -> actor step (+ Adam).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "energy_tc.cuh"
#include "internal.h"
#include "mlp_bf16.cuh"
#include "ctx.h"
#include "trace.h"

using namespace crl;

namespace crl {
thread_local Tracer* g_tracer = nullptr;
int g_launch_overlap = 1;
int g_autotune = 1;
int g_gemm_kernel = CRL_GEMM_ANY;
}

namespace crl {

thread_local std::string g_thread_error;

// The device address of pinned, mapped host memory (a kernel may read it in
// place), or nullptr for device, pageable or unknown memory.
const void* host_device_alias(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

PointerKind classify_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return PointerKind{true, nullptr};
  }
  if (at.type == cudaMemoryTypeHost) return PointerKind{true, at.devicePointer};
  return PointerKind{at.type == cudaMemoryTypeUnregistered, nullptr};
}

bool is_host_pointer(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

size_t dtype_size(int precision) { return precision == CRL_PREC_FP64 ? sizeof(double) : sizeof(float); }

MlpShape net_shape(const crl_config& c, int net) {
  MlpShape s{};
  s.hidden = c.hidden;
  s.layers = c.layers;
  s.layernorm = c.layernorm ? 1 : 0;
  if (net == CRL_NET_PHI) {
    s.in0 = c.D;
    s.in1 = c.A;
    s.out = c.repr;
  } else if (net == CRL_NET_PSI) {
    s.in0 = c.G;
    s.in1 = 0;
    s.out = c.repr;
  } else {
    s.in0 = c.D;
    s.in1 = c.G;
    s.out = 2 * c.A;
  }
  return s;
}

void validate_config(const crl_config& c) {
  CRL_REQUIRE(c.E >= 1 && c.T >= 1 && c.D >= 1 && c.A >= 1 && c.B >= 1, CRL_E_INVALID_ARG,
              "E, T, D, A and B must be >= 1");
  CRL_REQUIRE(c.G >= 1 && c.G <= CRL_MAX_GOAL_DIMS, CRL_E_INVALID_ARG, "G must lie in [1, 16]");
  CRL_REQUIRE(c.hidden >= 1 && c.repr >= 1, CRL_E_INVALID_ARG, "hidden and repr must be >= 1");
  CRL_REQUIRE(c.layers >= 1 && c.layers <= CRL_MAX_LAYERS, CRL_E_INVALID_ARG, "layers must lie in [1, 8]");
  for (int i = 0; i < c.G; ++i)
    CRL_REQUIRE(c.goal_idx[i] >= 0 && c.goal_idx[i] < c.D, CRL_E_INVALID_ARG, "goal_idx entries must lie in [0, D)");
  CRL_REQUIRE(c.gamma >= 0.f && c.gamma < 1.f, CRL_E_INVALID_ARG, "gamma must lie in [0, 1)");
  CRL_REQUIRE(c.temperature > 0.f && std::isfinite(c.temperature), CRL_E_INVALID_ARG, "temperature must be > 0");
  CRL_REQUIRE(c.beta_lse >= 0.f && c.alpha >= 0.f, CRL_E_INVALID_ARG, "beta_lse and alpha must be >= 0");
  CRL_REQUIRE(c.alpha_autotune == 0 || c.alpha_autotune == 1, CRL_E_INVALID_ARG, "alpha_autotune must be 0 or 1");
  CRL_REQUIRE(c.alpha_rg >= 0.f && c.alpha_rg <= 1.f, CRL_E_INVALID_ARG, "alpha_rg must lie in [0, 1]");
  CRL_REQUIRE(!c.alpha_autotune || (c.alpha > 0.f && std::isfinite(c.target_entropy) && c.lr_alpha >= 0.f),
              CRL_E_INVALID_ARG, "alpha_autotune needs alpha > 0, a finite target_entropy and lr_alpha >= 0");
  CRL_REQUIRE(c.energy >= CRL_ENERGY_L2 && c.energy <= CRL_ENERGY_L2SQ, CRL_E_INVALID_ARG, "unknown energy");
  CRL_REQUIRE(c.loss >= CRL_LOSS_FWD && c.loss <= CRL_LOSS_NCE_BINARY, CRL_E_INVALID_ARG, "unknown loss");
  CRL_REQUIRE(c.loss != CRL_LOSS_FB || c.B >= 2, CRL_E_INVALID_ARG, "the forward-backward objective needs B >= 2");
  CRL_REQUIRE(c.sym_reduction == CRL_SYM_MEAN || c.sym_reduction == CRL_SYM_SUM, CRL_E_INVALID_ARG,
              "unknown sym_reduction");
  CRL_REQUIRE(c.penalty_axis >= CRL_PENALTY_ROW && c.penalty_axis <= CRL_PENALTY_BOTH, CRL_E_INVALID_ARG,
              "unknown penalty_axis");
  CRL_REQUIRE(c.offset_min == 0 || c.offset_min == 1, CRL_E_INVALID_ARG, "offset_min must be 0 or 1");
  CRL_REQUIRE(c.precision >= CRL_PREC_FP32 && c.precision <= CRL_PREC_FP64, CRL_E_INVALID_ARG, "unknown precision");
  CRL_REQUIRE(c.path == CRL_PATH_PLAIN || c.path == CRL_PATH_FUSED, CRL_E_INVALID_ARG, "unknown path");
  if (c.path == CRL_PATH_FUSED) {
    CRL_REQUIRE(c.precision == CRL_PREC_BF16, CRL_E_UNSUPPORTED, "the fused energy path runs in BF16 only");
    const char* why = nullptr;
    LossSpec ls{c.energy, c.loss, c.sym_reduction, c.penalty_axis, c.temperature, c.beta_lse};
    CRL_REQUIRE(energy_tc_supported(ls, c.B, c.repr, &why), CRL_E_UNSUPPORTED, why);
  }
  if (c.precision == CRL_PREC_BF16) {
    CRL_REQUIRE(c.B % 8 == 0 && c.hidden % 8 == 0, CRL_E_UNSUPPORTED,
                "the BF16 path needs B and hidden to be multiples of 8 (16-byte TMA rows)");
  }
  CRL_REQUIRE(c.lr_critic >= 0.f && c.lr_actor >= 0.f && c.adam_eps > 0.f && c.adam_beta1 >= 0.f &&
                  c.adam_beta1 < 1.f && c.adam_beta2 >= 0.f && c.adam_beta2 < 1.f,
              CRL_E_INVALID_ARG, "bad Adam hyperparameters");
  const int64_t W = round_up((int64_t)c.D + c.A + 1, 4);
  CRL_REQUIRE((int64_t)c.E * c.T * W < ((int64_t)1 << 40), CRL_E_INVALID_ARG, "replay buffer too large");
}

}  // namespace crl


namespace crl {
void set_thread_error(const std::string& msg) { g_thread_error = msg; }
}  // namespace crl

namespace crl {

int fail(crl_ctx* ctx, const Failure& f) {
  if (ctx) ctx->err = f.msg;
  g_thread_error = f.msg;
  return f.code;
}

LossSpec loss_spec(const crl_config& c) {
  LossSpec ls;
  ls.energy = c.energy;
  ls.loss = c.loss;
  ls.sym_reduction = c.sym_reduction;
  ls.penalty_axis = c.penalty_axis;
  ls.tau = c.temperature;
  ls.beta = c.beta_lse;
  return ls;
}

template <typename T>
__global__ void to_float_kernel(const T* __restrict__ src, float* __restrict__ dst, int n) {
  pdl_enter();
  const int i = threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// Copy n floats of the ctx's loss staging (already float) to a host or device destination.
void deliver_floats(float* dst, const float* src, int n, cudaStream_t st) {
  if (!dst) return;
  const cudaMemcpyKind kind = is_host_pointer(dst) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CRL_CHECK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(float), kind, st));
}

template <typename T>
void critic_impl(crl_ctx* c, const float* s, const float* a, const float* g, int B, int apply, cudaStream_t st) {
  const crl_config& cf = c->cfg;
  const T* pphi = static_cast<const T*>(c->nets[CRL_NET_PHI].params);
  const T* ppsi = static_cast<const T*>(c->nets[CRL_NET_PSI].params);
  T* phi = static_cast<T*>(c->phi);
  T* psi = static_cast<T*>(c->psi);
  T* dphi = static_cast<T*>(c->dphi);
  T* dpsi = static_cast<T*>(c->dpsi);
  T* rl = static_cast<T*>(c->row_lse);
  T* cl = static_cast<T*>(c->col_lse);
  T* loss = static_cast<T*>(c->loss);
  mlp_forward<T, float>(c->shapes[CRL_NET_PHI], pphi, s, a, B, phi, c->saved[CRL_NET_PHI], st);
  mlp_forward<T, float>(c->shapes[CRL_NET_PSI], ppsi, g, nullptr, B, psi, c->saved[CRL_NET_PSI], st);
  const LossSpec ls = loss_spec(cf);
  infonce_forward<T>(ls, phi, psi, B, cf.repr, loss, rl, cl, c->ws, cf.path, &c->ctr->status,
                     apply ? &c->ctr->t_critic : nullptr, st);
  logit_stats_launch(c, phi, psi, B, sizeof(T) == 8, st);
  infonce_backward<T>(ls, phi, psi, B, cf.repr, rl, cl, 1.0, dphi, dpsi, c->ws, cf.path, st);
  mlp_backward<T, float>(c->shapes[CRL_NET_PHI], pphi, s, a, B, c->saved[CRL_NET_PHI], dphi,
                         static_cast<T*>(c->nets[CRL_NET_PHI].grads), nullptr, nullptr, st);
  mlp_backward<T, float>(c->shapes[CRL_NET_PSI], ppsi, g, nullptr, B, c->saved[CRL_NET_PSI], dpsi,
                         static_cast<T*>(c->nets[CRL_NET_PSI].grads), nullptr, nullptr, st);
  if (apply) {
    for (int net : {CRL_NET_PHI, CRL_NET_PSI}) {
      const crl_net_ptrs& np = c->nets[net];
      adam_update<T>(static_cast<T*>(np.params), static_cast<const T*>(np.grads), static_cast<T*>(np.adam_m),
                     static_cast<T*>(np.adam_v), c->counts[net], &c->ctr->t_critic, 0, cf.lr_critic, cf.adam_beta1,
                     cf.adam_beta2, cf.adam_eps, st);
    }
  }
  if constexpr (sizeof(T) != sizeof(float)) {
    TraceLaunch tr(CRL_TRACE_AUX, st, 4.0 * (sizeof(T) + 4));
    launch_k(to_float_kernel<T>, dim3(1), dim3(32), 0, st, loss, c->loss_f, 4);
  }
  check_launch("critic step");
}

// bump_step: the loss kernel also advances the relabel step counter (update step).
template <typename T>
void actor_impl(crl_ctx* c, const float* s, const float* g, const float* eps, int B, int apply, cudaStream_t st,
                bool bump_step = false) {
  const crl_config& cf = c->cfg;
  const T* ppi = static_cast<const T*>(c->nets[CRL_NET_PI].params);
  const T* pphi = static_cast<const T*>(c->nets[CRL_NET_PHI].params);
  const T* ppsi = static_cast<const T*>(c->nets[CRL_NET_PSI].params);
  T* pi_out = static_cast<T*>(c->pi_out);
  T* a_new = static_cast<T*>(c->a_new);
  T* logpi = static_cast<T*>(c->logpi);
  T* eps_used = static_cast<T*>(c->eps_used);
  T* phi = static_cast<T*>(c->phi);
  T* psi = static_cast<T*>(c->psi);
  T* dphi = static_cast<T*>(c->dphi);
  T* da = static_cast<T*>(c->da);
  T* dout = static_cast<T*>(c->dout);
  T* loss = static_cast<T*>(c->loss) + 4;
  const ActorSpec as = actor_spec_of(c);
  mlp_forward<T, float>(c->shapes[CRL_NET_PI], ppi, s, g, B, pi_out, c->saved[CRL_NET_PI], st);
  actor_head_forward<T>(as, pi_out, eps, &c->ctr->last_step, cf.seed, cf.agent, B, a_new, logpi, eps_used, st);
  mlp_forward<T, T>(c->shapes[CRL_NET_PHI], pphi, s, a_new, B, phi, c->saved[CRL_NET_PHI], st);
  mlp_forward<T, float>(c->shapes[CRL_NET_PSI], ppsi, g, nullptr, B, psi, c->saved[CRL_NET_PSI], st);
  actor_energy_and_loss<T>(as, phi, psi, logpi, B, cf.repr, dphi, static_cast<T*>(c->fdiag), loss, c->actor_ws,
                           &c->ctr->ticket_actor, &c->ctr->status, apply ? &c->ctr->t_actor : nullptr,
                           bump_step ? &c->ctr->step : nullptr, &c->ctr->last_step, st);
  mlp_backward<T, T>(c->shapes[CRL_NET_PHI], pphi, s, a_new, B, c->saved[CRL_NET_PHI], dphi, nullptr, nullptr, da,
                     st);
  actor_head_backward<T>(as, pi_out, eps_used, da, B, dout, st);
  const crl_net_ptrs& np = c->nets[CRL_NET_PI];
  mlp_backward<T, float>(c->shapes[CRL_NET_PI], ppi, s, g, B, c->saved[CRL_NET_PI], dout, static_cast<T*>(np.grads),
                         nullptr, nullptr, st);
  if (apply) {
    adam_update<T>(static_cast<T*>(np.params), static_cast<const T*>(np.grads), static_cast<T*>(np.adam_m),
                   static_cast<T*>(np.adam_v), c->counts[CRL_NET_PI], &c->ctr->t_actor, 0, cf.lr_actor,
                   cf.adam_beta1, cf.adam_beta2, cf.adam_eps, st);
  }
  if constexpr (sizeof(T) != sizeof(float)) {
    TraceLaunch tr(CRL_TRACE_AUX, st, 2.0 * (sizeof(T) + 4));
    launch_k(to_float_kernel<T>, dim3(1), dim3(32), 0, st, loss, c->loss_f + 4, 2);
  }
  check_launch("actor step");
}

void* ctx_alloc(void* owner, size_t bytes) {
  try {
    return static_cast<crl_ctx*>(owner)->dalloc(bytes);
  } catch (...) {
    return nullptr;
  }
}

void bf_maps(crl_ctx* c, int net, int B) {
  const char* e = bf_net_maps(c->bf[net], B);
  if (e) throw Failure(CRL_E_CUDA, std::string("tensor map: ") + e);
}

void bf_check(const char* err) {
  if (err) throw Failure(CRL_E_CUDA, std::string("BF16 network pass: ") + err);
}

// Refresh the BF16 shadows of `net` unless they are known to match (refresh forces it).
void bf_refresh(crl_ctx* c, int net, bool refresh, cudaStream_t st) {
  if (refresh || !c->shadow_ok[net]) {
    bf_net_shadow(c->bf[net], static_cast<const float*>(c->nets[net].params), st);
    c->shadow_ok[net] = true;
  }
}

ActorSpec actor_spec_of(crl_ctx* c) {
  const crl_config& cf = c->cfg;
  ActorSpec as;
  std::memset(&as, 0, sizeof(as));   // member by member: zeroed padding keys the device tables
  as.A = cf.A;
  as.energy = cf.energy;
  as.tau = (double)cf.temperature;
  as.alpha = (double)cf.alpha;
  if (cf.alpha_autotune) {
    as.tune.state = c->ctr->alpha;
    as.tune.target_entropy = (double)cf.target_entropy;
    as.tune.lr = (double)cf.lr_alpha;
    as.tune.b1 = (double)cf.adam_beta1;
    as.tune.b2 = (double)cf.adam_beta2;
    as.tune.eps = (double)cf.adam_eps;
  }
  return as;
}

void reset_alpha(crl_ctx* c) {
  const double a = (double)c->cfg.alpha;
  const double init[4] = {std::log(a), 0.0, 0.0, a};
  CRL_CHECK_CUDA(cudaMemcpy(c->ctr->alpha, init, sizeof(init), cudaMemcpyHostToDevice));
}

AdamShadowNet adam_net_of(crl_ctx* c, int net, const int* t, float lr) {
  const crl_net_ptrs& np = c->nets[net];
  const crl_config& cf = c->cfg;
  return AdamShadowNet{static_cast<float*>(np.params),
                       static_cast<const float*>(np.grads),
                       static_cast<float*>(np.adam_m),
                       static_cast<float*>(np.adam_v),
                       c->counts[net],
                       t,
                       lr,
                       cf.adam_beta1,
                       cf.adam_beta2,
                       cf.adam_eps,
                       &c->bf[net]};
}

// Critic step with BF16 tensor-core encoders (FP32 master weights).  refresh:
// rebuild the BF16 weight shadows first (the caller may have changed the
// weights).  packed: the relabel kernel already wrote the split network inputs.
// phi and psi run side by side as grouped launches (one per layer).
// with_pi: the policy's forward (its parameters do not change before the
// actor step) joins the encoders' grouped launches; the actor step then
// reuses its output (update step only, where relabel packed its input).
// head: the actor head's forward, run by extra blocks of the Adam launch (update
// step only: it reads the policy output the with_pi forward wrote).
void critic_impl_bf16(crl_ctx* c, const float* s, const float* a, const float* g, int B, int apply, cudaStream_t st,
                      bool refresh = true, bool packed = false, bool with_pi = false,
                      const HeadFwdArgs<float>* head = nullptr) {
  const crl_config& cf = c->cfg;
  unsigned* status = &c->ctr->status;
  BfNet& P = c->bf[CRL_NET_PHI];
  BfNet& Q = c->bf[CRL_NET_PSI];
  const float* pphi = static_cast<const float*>(c->nets[CRL_NET_PHI].params);
  const float* ppsi = static_cast<const float*>(c->nets[CRL_NET_PSI].params);
  bf_maps(c, CRL_NET_PHI, B);
  bf_maps(c, CRL_NET_PSI, B);
  bf_refresh(c, CRL_NET_PHI, refresh, st);
  bf_refresh(c, CRL_NET_PSI, refresh, st);
  if (!packed) {
    bf_net_pack_input(P, s, a, B, st);
    bf_net_pack_input(Q, g, nullptr, B, st);
  }
  const BfPass pass[3] = {{&P, pphi, static_cast<float*>(c->nets[CRL_NET_PHI].grads), nullptr, B},
                          {&Q, ppsi, static_cast<float*>(c->nets[CRL_NET_PSI].grads), nullptr, B},
                          {&c->bf[CRL_NET_PI], static_cast<const float*>(c->nets[CRL_NET_PI].params), nullptr,
                           nullptr, B}};
  if (with_pi) {
    bf_maps(c, CRL_NET_PI, B);
    bf_refresh(c, CRL_NET_PI, refresh, st);
  }
  // fused path: the encoders' output layers also write the energy's BF16 operands
  const EnergyOut eo[2] = {{c->etc.X, c->etc.auxX, cf.energy}, {c->etc.Y, c->etc.auxY, cf.energy}};
  BfPass fpass[3] = {pass[0], pass[1], pass[2]};
  if (c->fused) {
    fpass[0].energy_out = &eo[0];
    fpass[1].energy_out = &eo[1];
  }
  bf_check(bf_forward(c->groups, fpass, with_pi ? 3 : 2, status, st));
  logit_stats_launch(c, P.y, Q.y, B, false, st);
  float* rl = static_cast<float*>(c->row_lse);
  float* cl = static_cast<float*>(c->col_lse);
  float* loss = static_cast<float*>(c->loss);
  float* dphi = static_cast<float*>(c->dphi);
  float* dpsi = static_cast<float*>(c->dpsi);
  const LossSpec ls = loss_spec(cf);
  if (c->fused) {
    // fused tcgen05 energy stage: no B x B matrix; the gradients land in the encoders' dy buffers
    const char* e = energy_tc_maps(c->etc, B);
    if (e) throw Failure(CRL_E_CUDA, std::string("tensor map: ") + e);
    energy_tc_forward(c->etc, ls, B, P.y, Q.y, loss, rl, cl, c->etc_ws, status, apply ? &c->ctr->t_critic : nullptr,
                      st);
    energy_tc_backward(c->etc, ls, B, P.y, Q.y, rl, cl, 1.0, P.dz[P.layers], Q.dz[Q.layers], c->etc_ws, status,
                       st);
  } else {
    infonce_forward<float>(ls, P.y, Q.y, B, cf.repr, loss, rl, cl, c->ws, CRL_PATH_PLAIN, status,
                           apply ? &c->ctr->t_critic : nullptr, st);
    infonce_backward<float>(ls, P.y, Q.y, B, cf.repr, rl, cl, 1.0, dphi, dpsi, c->ws, CRL_PATH_PLAIN, st);
    bf_net_load_dy(P, dphi, B, st);
    bf_net_load_dy(Q, dpsi, B, st);
  }
  bf_check(bf_backward(c->groups, pass, 2, status, st));
  if (apply) {
    // Adam for phi and psi in one launch, refreshing their BF16 shadows
    const AdamShadowNet an[2] = {adam_net_of(c, CRL_NET_PHI, &c->ctr->t_critic, cf.lr_critic),
                                 adam_net_of(c, CRL_NET_PSI, &c->ctr->t_critic, cf.lr_critic)};
    const std::vector<HeadFwdArgs<float>> heads(head ? 1 : 0, head ? *head : HeadFwdArgs<float>{});
    bf_check(adam_shadow_update(c->tables, an, 2, st, &heads));
  }
  check_launch("critic step (bf16)");
}

// Actor step with BF16 tensor-core networks: pi(s, g) (unless pi_ready), the
// head, phi(s, a') and psi(g) side by side, the diagonal energy with the loss,
// and the backward through phi (input gradient only) and pi.  packed: the
// relabel kernel wrote the split network inputs, so the head writes a' into
// phi's input directly.  bump_step: the loss kernel advances the relabel step.
// head_done: the head's forward already ran in the critic's Adam launch.
void actor_impl_bf16(crl_ctx* c, const float* s, const float* g, const float* eps, int B, int apply, cudaStream_t st,
                     bool refresh = true, bool packed = false, bool pi_ready = false, bool bump_step = false,
                     bool head_done = false) {
  const crl_config& cf = c->cfg;
  unsigned* status = &c->ctr->status;
  BfNet& PI = c->bf[CRL_NET_PI];
  BfNet& P = c->bf[CRL_NET_PHI];
  BfNet& Q = c->bf[CRL_NET_PSI];
  const float* ppi = static_cast<const float*>(c->nets[CRL_NET_PI].params);
  const float* pphi = static_cast<const float*>(c->nets[CRL_NET_PHI].params);
  const float* ppsi = static_cast<const float*>(c->nets[CRL_NET_PSI].params);
  for (int net = 0; net < 3; ++net) {
    bf_maps(c, net, B);
    bf_refresh(c, net, refresh, st);
  }
  float* a_new = static_cast<float*>(c->a_new);
  float* logpi = static_cast<float*>(c->logpi);
  float* eps_used = static_cast<float*>(c->eps_used);
  float* da = static_cast<float*>(c->da);
  float* loss = static_cast<float*>(c->loss) + 4;
  const ActorSpec as = actor_spec_of(c);
  if (!packed) {
    bf_net_pack_input(PI, s, g, B, st);
    bf_net_pack_input(Q, g, nullptr, B, st);
  }
  if (!pi_ready) {
    const BfPass pi_fwd[1] = {{&PI, ppi, nullptr, nullptr, B}};
    bf_check(bf_forward(c->groups, pi_fwd, 1, status, st));
  }
  if (!head_done)
    actor_head_forward<float>(as, PI.y, eps, &c->ctr->last_step, cf.seed, cf.agent, B, a_new, logpi, eps_used, st,
                              packed ? P.x0 : nullptr, bf_net_x0_ld(P), P.s.in0);
  if (!packed) bf_net_pack_input(P, s, a_new, B, st);
  // phi(s, a') and psi(g) with the critic's updated weights
  const BfPass fwd[2] = {{&P, pphi, nullptr, da, B}, {&Q, ppsi, nullptr, nullptr, B}};
  bf_check(bf_forward(c->groups, fwd, 2, status, st));
  actor_energy_and_loss<float>(as, P.y, Q.y, logpi, B, cf.repr, nullptr, static_cast<float*>(c->fdiag), loss,
                               c->actor_ws, &c->ctr->ticket_actor, status, apply ? &c->ctr->t_actor : nullptr,
                               bump_step ? &c->ctr->step : nullptr, &c->ctr->last_step, st, P.dz[P.layers],
                               P.L[P.layers].out_pad);
  bf_check(bf_backward(c->groups, fwd, 1, status, st));
  actor_head_backward<float>(as, PI.y, eps_used, da, B, nullptr, st, PI.dz[PI.layers], PI.L[PI.layers].out_pad);
  const BfPass pi_pass[1] = {{&PI, ppi, static_cast<float*>(c->nets[CRL_NET_PI].grads), nullptr, B}};
  bf_check(bf_backward(c->groups, pi_pass, 1, status, st));
  if (apply) {
    const AdamShadowNet an = adam_net_of(c, CRL_NET_PI, &c->ctr->t_actor, cf.lr_actor);
    bf_check(adam_shadow_update(c->tables, &an, 1, st));
  }
  check_launch("actor step (bf16)");
}

void insert_impl(crl_ctx* c, const float* obs, const float* act, const uint8_t* done, int n, cudaStream_t st) {
  const crl_config& cf = c->cfg;
  CRL_REQUIRE(obs && act && done, CRL_E_INVALID_ARG, "obs, act and done must be non-null");
  CRL_REQUIRE(n >= 1, CRL_E_INVALID_ARG, "n must be >= 1");
  CRL_REQUIRE(c->total_host + n < ((int64_t)1 << 31) - 1, CRL_E_INVALID_ARG,
              "more than 2^31 - 2 steps inserted per environment");
  const size_t nobs = (size_t)n * cf.E * cf.D * sizeof(float);
  const size_t nact = (size_t)n * cf.E * cf.A * sizeof(float);
  const size_t ndone = (size_t)n * cf.E;
  // pinned host inputs: the insert kernel reads them in place through their
  // device alias (no copy); pageable host inputs: staged through device memory
  const PointerKind k_obs = classify_pointer(obs), k_act = classify_pointer(act), k_done = classify_pointer(done);
  const void* d_obs = k_obs.alias;
  const void* d_act = k_act.alias;
  const void* d_done = k_done.alias;
  const bool h_obs = k_obs.host && !d_obs, h_act = k_act.host && !d_act, h_done = k_done.host && !d_done;
  if (d_obs) obs = static_cast<const float*>(d_obs);
  if (d_act) act = static_cast<const float*>(d_act);
  if (d_done) done = static_cast<const uint8_t*>(d_done);
  if (h_obs || h_act || h_done) {
    const size_t need = round_up(nobs, 256) + round_up(nact, 256) + round_up(ndone, 256);
    if (need > c->stage_bytes) {
      if (c->stage) {
        CRL_CHECK_CUDA(cudaStreamSynchronize(st));
        cudaFree(c->stage);
        c->stage = nullptr;
      }
      CRL_CHECK_CUDA(cudaMalloc(&c->stage, need));
      c->stage_bytes = need;
    }
    char* p = static_cast<char*>(c->stage);
    if (h_obs) {
      CRL_CHECK_CUDA(cudaMemcpyAsync(p, obs, nobs, cudaMemcpyHostToDevice, st));
      obs = reinterpret_cast<const float*>(p);
    }
    p += round_up(nobs, 256);
    if (h_act) {
      CRL_CHECK_CUDA(cudaMemcpyAsync(p, act, nact, cudaMemcpyHostToDevice, st));
      act = reinterpret_cast<const float*>(p);
    }
    p += round_up(nact, 256);
    if (h_done) {
      CRL_CHECK_CUDA(cudaMemcpyAsync(p, done, ndone, cudaMemcpyHostToDevice, st));
      done = reinterpret_cast<const uint8_t*>(p);
    }
  }
  launch_buffer_insert(c->bd, obs, act, done, n, c->total_host, st);
  check_launch("buffer insert");
  c->total_host += n;
  c->size_host = (int32_t)(c->total_host < cf.T ? c->total_host : cf.T);
}

// bump: advance the step counter after a CRL_STEP_AUTO draw (the update step
// leaves that to its actor-loss kernel, which runs once per step anyway).
// Checked relabel arguments (spw set for the batch).
RelabelArgs relabel_args(crl_ctx* c, uint64_t step, int B, float* s, float* a, float* g, int32_t* idx,
                         bool pack_bf16) {
  const crl_config& cf = c->cfg;
  CRL_REQUIRE(s && a && g, CRL_E_INVALID_ARG, "s, a and g must be non-null");
  CRL_REQUIRE(B >= 1, CRL_E_SHAPE, "B must be >= 1");
  CRL_REQUIRE(!pack_bf16 || B <= cf.B, CRL_E_SHAPE, "B must lie in [1, cfg.B]");
  CRL_REQUIRE((int64_t)B * cf.D < ((int64_t)1 << 31) && (int64_t)B * 3 < ((int64_t)1 << 31), CRL_E_SHAPE,
              "B x D must stay below 2^31");
  CRL_REQUIRE(c->size_host > 0, CRL_E_BUFFER_EMPTY, "the replay buffer is empty");
  RelabelArgs ra;
  std::memset(&ra, 0, sizeof(ra));   // zero padding: these arguments also key device tables
  ra.seed = cf.seed;
  ra.agent = cf.agent;
  ra.step = step;
  ra.step_dev = &c->ctr->step;
  ra.last_step_dev = &c->ctr->last_step;
  ra.B = B;
  ra.G = cf.G;
  ra.offset_min = cf.offset_min;
  for (int i = 0; i < cf.G; ++i) ra.goal_idx[i] = cf.goal_idx[i];
  ra.s = s;
  ra.a = a;
  ra.g = g;
  ra.idx = idx;
  ra.status = &c->ctr->status;
  if (pack_bf16) {
    for (int k = 0; k < 3; ++k) {
      BfNet& n = c->bf[k];
      ra.pack[k] = RelabelPack{n.x0, bf_net_x0_ld(n)};
    }
  }
  ra.spw = relabel_spw(B);
  return ra;
}

void relabel_impl(crl_ctx* c, uint64_t step, int B, float* s, float* a, float* g, int32_t* idx, cudaStream_t st,
                  bool pack_bf16, bool bump) {
  const RelabelArgs ra = relabel_args(c, step, B, s, a, g, idx, pack_bf16);
  launch_relabel(c->bd, ra, st);
  if (step == CRL_STEP_AUTO && bump) launch_bump_u64(&c->ctr->step, st);
  check_launch("sample relabel");
}

}  // namespace crl

// =============================================================================
extern "C" {

void crl_config_default(crl_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->E = 1024;
  c->T = 1000;
  c->D = 29;
  c->A = 8;
  c->G = 2;
  c->B = 256;
  c->hidden = 256;
  c->layers = 2;
  c->repr = 64;
  for (int i = 0; i < CRL_MAX_GOAL_DIMS; ++i) c->goal_idx[i] = i;
  c->gamma = 0.99f;
  c->beta_lse = 0.1f;
  c->temperature = 1.0f;
  c->alpha = 0.1f;
  c->energy = CRL_ENERGY_L2;
  c->loss = CRL_LOSS_SYM;
  c->sym_reduction = CRL_SYM_MEAN;
  c->penalty_axis = CRL_PENALTY_ROW;
  c->layernorm = 0;
  c->precision = CRL_PREC_FP32;
  c->path = CRL_PATH_PLAIN;
  c->offset_min = 1;
  c->lr_critic = 3e-4f;
  c->lr_actor = 6e-4f;
  c->adam_beta1 = 0.9f;
  c->adam_beta2 = 0.999f;
  c->adam_eps = 1e-8f;
  c->seed = 0;
  c->agent = 0;
  c->alpha_autotune = 0;
  c->target_entropy = -(float)c->A;
  c->lr_alpha = c->lr_actor;
}

int crl_param_count(const crl_config* cfg, int32_t net, int64_t* count) {
  return guarded(nullptr, [&] {
    CRL_REQUIRE(cfg && count, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(net >= 0 && net <= 2, CRL_E_INVALID_ARG, "net must be CRL_NET_PHI, _PSI or _PI");
    CRL_REQUIRE(cfg->layers >= 1 && cfg->layers <= CRL_MAX_LAYERS, CRL_E_INVALID_ARG, "layers must lie in [1, 8]");
    LayerOffsets lay[CRL_MAX_LAYERS + 1];
    *count = mlp_layout(net_shape(*cfg, net), lay);
  });
}

int crl_param_tensors(const crl_config* cfg, int32_t net, int32_t* n) {
  return guarded(nullptr, [&] {
    CRL_REQUIRE(cfg && n, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(net >= 0 && net <= 2, CRL_E_INVALID_ARG, "net must be CRL_NET_PHI, _PSI or _PI");
    *n = cfg->layers * (cfg->layernorm ? 4 : 2) + 2;
  });
}

int crl_param_tensor(const crl_config* cfg, int32_t net, int32_t i, crl_tensor_info* out) {
  return guarded(nullptr, [&] {
    CRL_REQUIRE(cfg && out, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(net >= 0 && net <= 2, CRL_E_INVALID_ARG, "net must be CRL_NET_PHI, _PSI or _PI");
    CRL_REQUIRE(cfg->layers >= 1 && cfg->layers <= CRL_MAX_LAYERS, CRL_E_INVALID_ARG, "layers must lie in [1, 8]");
    const MlpShape s = net_shape(*cfg, net);
    LayerOffsets lay[CRL_MAX_LAYERS + 1];
    mlp_layout(s, lay);
    const int per = s.layernorm ? 4 : 2;
    const int ntens = s.layers * per + 2;
    CRL_REQUIRE(i >= 0 && i < ntens, CRL_E_INVALID_ARG, "tensor index out of range");
    int layer = i / per, kind = i % per;
    if (layer >= s.layers) {
      layer = s.layers;
      kind = i - s.layers * per;
    }
    const LayerOffsets& L = lay[layer];
    out->layer = layer;
    out->kind = kind;
    if (kind == 0) {
      out->offset = L.W;
      out->rows = L.out;
      out->cols = L.in;
    } else {
      out->offset = (kind == 1) ? L.b : (kind == 2 ? L.g : L.beta);
      out->rows = L.out;
      out->cols = 1;
    }
  });
}

int crl_create(const crl_config* cfg, crl_ctx** out) {
  if (out) *out = nullptr;
  crl_ctx* c = nullptr;
  const int rc = guarded(nullptr, [&] {
    CRL_REQUIRE(cfg && out, CRL_E_INVALID_ARG, "null argument");
    validate_config(*cfg);
    c = new crl_ctx();
    c->cfg = *cfg;
    CRL_CHECK_CUDA(cudaGetDevice(&c->device));
    c->esz = dtype_size(cfg->precision);
    const crl_config& cf = c->cfg;
    const int W = (int)round_up((int64_t)cf.D + cf.A + 1, 4);
    c->rows = static_cast<float*>(c->dalloc((size_t)cf.E * cf.T * W * sizeof(float)));
    c->ep_start = static_cast<int32_t*>(c->dalloc((size_t)cf.E * sizeof(int32_t)));
    c->bstate = static_cast<int32_t*>(c->dalloc(2 * sizeof(int32_t)));
    c->gq = static_cast<unsigned long long*>(c->dalloc((size_t)(cf.T + 2) * sizeof(unsigned long long)));
    c->ctr = static_cast<Counters*>(c->dalloc(sizeof(Counters)));
    CRL_CHECK_CUDA(cudaMemset(c->ep_start, 0, (size_t)cf.E * sizeof(int32_t)));
    CRL_CHECK_CUDA(cudaMemset(c->bstate, 0, 2 * sizeof(int32_t)));
    CRL_CHECK_CUDA(cudaMemset(c->ctr, 0, sizeof(Counters)));
    reset_alpha(c);
    CRL_CHECK_CUDA(cudaMemset(c->rows, 0, (size_t)cf.E * cf.T * W * sizeof(float)));
    std::vector<unsigned long long> table(cf.T + 2);
    build_discount_table(cf.gamma, cf.T + 2, table.data());
    CRL_CHECK_CUDA(cudaMemcpy(c->gq, table.data(), table.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice));
    c->bd = BufferDev{c->rows, c->ep_start, c->bstate, c->gq, cf.E, cf.T, cf.D, cf.A, W};

    const int B = cf.B, R = cf.repr, A = cf.A;
    const size_t e = c->esz;
    for (int net = 0; net < 3; ++net) {
      c->shapes[net] = net_shape(cf, net);
      LayerOffsets lay[CRL_MAX_LAYERS + 1];
      c->counts[net] = mlp_layout(c->shapes[net], lay);
      c->saved[net] = c->dalloc(mlp_saved_bytes(c->shapes[net], B, e));
    }
    c->phi = c->dalloc((size_t)B * R * e);
    c->psi = c->dalloc((size_t)B * R * e);
    c->dphi = c->dalloc((size_t)B * R * e);
    c->dpsi = c->dalloc((size_t)B * R * e);
    c->row_lse = c->dalloc((size_t)B * e);
    c->col_lse = c->dalloc((size_t)B * e);
    c->loss = c->dalloc(8 * e);
    // the fused path keeps no B x B buffer (its energy stage has its own small workspace)
    c->ws_bytes = (cf.path == CRL_PATH_FUSED) ? 0 : infonce_ws_bytes(loss_spec(cf), B, R, e, cf.path);
    c->ws = c->dalloc(c->ws_bytes);
    c->pi_out = c->dalloc((size_t)B * 2 * A * e);
    c->a_new = c->dalloc((size_t)B * A * e);
    c->logpi = c->dalloc((size_t)B * e);
    c->eps_used = c->dalloc((size_t)B * A * e);
    c->fdiag = c->dalloc((size_t)B * e);
    c->da = c->dalloc((size_t)B * A * e);
    c->dout = c->dalloc((size_t)B * 2 * A * e);
    c->actor_ws = c->dalloc(actor_loss_ws_bytes(B, e));
    // FP32 / BF16: the loss parts are already float and land in the ABI's float buffer directly
    c->loss_f = (e == sizeof(float)) ? static_cast<float*>(c->loss) : static_cast<float*>(c->dalloc(8 * sizeof(float)));
    c->bs = static_cast<float*>(c->dalloc((size_t)B * cf.D * sizeof(float)));
    c->ba = static_cast<float*>(c->dalloc((size_t)B * cf.A * sizeof(float)));
    c->bg = static_cast<float*>(c->dalloc((size_t)B * cf.G * sizeof(float)));
    c->bg_act = static_cast<float*>(c->dalloc((size_t)B * cf.G * sizeof(float)));
    CRL_CHECK_CUDA(cudaMemset(c->loss, 0, 8 * e));
    CRL_CHECK_CUDA(cudaMemset(c->loss_f, 0, 8 * sizeof(float)));
    if (cf.precision == CRL_PREC_BF16) {
      c->bf16 = true;
      for (int net = 0; net < 3; ++net) {
        const char* e = bf_net_init(c->bf[net], c->shapes[net], B, ctx_alloc, c);
        if (e) throw Failure(CRL_E_CUDA, std::string("BF16 network set-up: ") + e);
      }
    }
    if (cf.path == CRL_PATH_FUSED) {
      c->fused = true;
      EnergyTc& e = c->etc;
      e.R = R;
      e.Bmax = B;
      e.ldt = B;
      e.X = static_cast<__nv_bfloat16*>(c->dalloc((size_t)B * R * 2));
      e.Y = static_cast<__nv_bfloat16*>(c->dalloc((size_t)B * R * 2));
      e.auxX = static_cast<float*>(c->dalloc((size_t)B * 4));
      e.auxY = static_cast<float*>(c->dalloc((size_t)B * 4));
      const size_t ews = energy_tc_ws_bytes(loss_spec(cf), B, R);
      c->etc_ws = c->dalloc(ews);
      CRL_CHECK_CUDA(cudaMemset(c->etc_ws, 0, ews));   // the finalize ticket starts at 0
    }
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
  });
  if (rc != CRL_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return CRL_OK;
}

int crl_destroy(crl_ctx* ctx) {
  if (!ctx) return CRL_OK;
  cudaDeviceSynchronize();
  delete ctx;
  return CRL_OK;
}

int crl_bind_params(crl_ctx* ctx, const crl_net_ptrs nets[3]) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && nets, CRL_E_INVALID_ARG, "null argument");
    for (int i = 0; i < 3; ++i)
      CRL_REQUIRE(nets[i].params && nets[i].grads && nets[i].adam_m && nets[i].adam_v, CRL_E_INVALID_ARG,
                  "every network needs params, grads, adam_m and adam_v");
    for (int i = 0; i < 3; ++i) {
      const void* p[4] = {nets[i].params, nets[i].grads, nets[i].adam_m, nets[i].adam_v};
      for (const void* q : p)
        CRL_REQUIRE((reinterpret_cast<uintptr_t>(q) & 15) == 0, CRL_E_INVALID_ARG,
                    "parameter, gradient and Adam arrays must be 16-byte aligned");
    }
    for (int i = 0; i < 3; ++i) {
      ctx->nets[i] = nets[i];
      // Padding between tensors never receives a gradient; keep it at zero.
      CRL_CHECK_CUDA(cudaMemset(nets[i].grads, 0, (size_t)ctx->counts[i] * ctx->esz));
    }
    CRL_CHECK_CUDA(cudaMemset(&ctx->ctr->t_critic, 0, 2 * sizeof(int)));
    reset_alpha(ctx);
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    ctx->drop_graph();
    ctx->groups.reset();   // tables hold parameter pointers
    ctx->tables.reset();
    ctx->update_calls = 0;
    for (int i = 0; i < 3; ++i) ctx->shadow_ok[i] = false;
    ctx->bound = true;
    ctx->bind_generation += 1;
  });
}

int crl_buffer_insert(crl_ctx* ctx, const float* obs, const float* act, const uint8_t* done, int32_t n,
                      void* stream) {
  NvtxRange nvtx("crl_buffer_insert");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    insert_impl(ctx, obs, act, done, n, static_cast<cudaStream_t>(stream));
  });
}

int crl_buffer_size(const crl_ctx* ctx, int32_t* size, int64_t* total) {
  if (!ctx) return CRL_E_INVALID_ARG;
  if (size) *size = ctx->size_host;
  if (total) *total = ctx->total_host;
  return CRL_OK;
}

int crl_sample_relabel(crl_ctx* ctx, uint64_t step, int32_t B, float* s, float* a, float* g, int32_t* idx,
                       void* stream) {
  NvtxRange nvtx("crl_sample_relabel");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    relabel_impl(ctx, step, B, s, a, g, idx, static_cast<cudaStream_t>(stream));
  });
}

int crl_critic_step(crl_ctx* ctx, const float* s, const float* a, const float* g, int32_t B, int32_t apply_update,
                    float* loss_out, void* stream) {
  NvtxRange nvtx("crl_critic_step");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(ctx->bound, CRL_E_NOT_BOUND, "crl_bind_params has not been called");
    CRL_REQUIRE(s && a && g, CRL_E_INVALID_ARG, "s, a and g must be non-null");
    CRL_REQUIRE(B >= 1 && B <= ctx->cfg.B, CRL_E_SHAPE, "B must lie in [1, cfg.B]");
    CRL_REQUIRE(ctx->cfg.loss != CRL_LOSS_FB || B >= 2, CRL_E_SHAPE, "the forward-backward objective needs B >= 2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ctx->cfg.precision == CRL_PREC_FP64) critic_impl<double>(ctx, s, a, g, B, apply_update, st);
    else if (ctx->bf16) critic_impl_bf16(ctx, s, a, g, B, apply_update, st);
    else critic_impl<float>(ctx, s, a, g, B, apply_update, st);
    deliver_floats(loss_out, ctx->loss_f, 4, st);
  });
}

int crl_actor_step(crl_ctx* ctx, const float* s, const float* g, const float* eps, int32_t B, int32_t apply_update,
                   float* loss_out, void* stream) {
  NvtxRange nvtx("crl_actor_step");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(ctx->bound, CRL_E_NOT_BOUND, "crl_bind_params has not been called");
    CRL_REQUIRE(s && g, CRL_E_INVALID_ARG, "s and g must be non-null");
    CRL_REQUIRE(B >= 1 && B <= ctx->cfg.B, CRL_E_SHAPE, "B must lie in [1, cfg.B]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ctx->cfg.precision == CRL_PREC_FP64) actor_impl<double>(ctx, s, g, eps, B, apply_update, st);
    else if (ctx->bf16) actor_impl_bf16(ctx, s, g, eps, B, apply_update, st);
    else actor_impl<float>(ctx, s, g, eps, B, apply_update, st);
    deliver_floats(loss_out, ctx->loss_f + 4, 2, st);
  });
}

}  // extern "C"

namespace crl {
// relabel (device step counter) -> critic + Adam -> actor + Adam on the batch workspaces
void update_body(crl_ctx* ctx, cudaStream_t st) {
  const int B = ctx->cfg.B;
  // the BF16 path has the relabel kernel pack the network inputs directly; the
  // actor-loss kernel advances the step counter
  relabel_impl(ctx, CRL_STEP_AUTO, B, ctx->bs, ctx->ba, ctx->bg, nullptr, st, ctx->bf16, false);
  // random-goal actor mix: the actor takes its own goals (and its own input packs)
  const bool mix = ctx->cfg.alpha_rg > 0.f;
  const float* g_actor = ctx->bg;
  if (mix) {
    launch_actor_goals(B, ctx->cfg.G, ctx->bg, ctx->bg_act, ctx->cfg.seed, ctx->cfg.agent, &ctx->ctr->last_step,
                       ctx->cfg.alpha_rg, st);
    g_actor = ctx->bg_act;
  }
  if (ctx->cfg.precision == CRL_PREC_FP64) {
    critic_impl<double>(ctx, ctx->bs, ctx->ba, ctx->bg, B, 1, st);
    actor_impl<double>(ctx, ctx->bs, g_actor, nullptr, B, 1, st, true);
  } else if (ctx->bf16) {
    // the shadows follow the weights through the fused Adam; only the first call refreshes.
    // Without the goal mix the actor's head forward (Philox noise at the last
    // sampled step, a' straight into phi's packed input) runs in the critic's Adam launch.
    BfNet& P = ctx->bf[CRL_NET_PHI];
    HeadFwdArgs<float> head;
    memset(&head, 0, sizeof(head));   // member by member: zeroed padding keys the device table
    head.B = B;
    head.A = ctx->cfg.A;
    head.out = ctx->bf[CRL_NET_PI].y;
    head.eps = nullptr;
    head.step_dev = &ctx->ctr->last_step;
    head.seed = ctx->cfg.seed;
    head.agent = ctx->cfg.agent;
    head.a_new = static_cast<float*>(ctx->a_new);
    head.logpi = static_cast<float*>(ctx->logpi);
    head.eps_used = static_cast<float*>(ctx->eps_used);
    head.x0 = P.x0;
    head.x0_ld = bf_net_x0_ld(P);
    head.x0_col = P.s.in0;
    critic_impl_bf16(ctx, ctx->bs, ctx->ba, ctx->bg, B, 1, st, false, true, !mix, mix ? nullptr : &head);
    actor_impl_bf16(ctx, ctx->bs, g_actor, nullptr, B, 1, st, false, !mix, !mix, true, !mix);
  } else {
    critic_impl<float>(ctx, ctx->bs, ctx->ba, ctx->bg, B, 1, st);
    actor_impl<float>(ctx, ctx->bs, g_actor, nullptr, B, 1, st, true);
  }
}
}  // namespace crl

extern "C" {

int crl_update_step(crl_ctx* ctx, const float* obs, const float* act, const uint8_t* done, int32_t n_insert,
                    float* loss_out, void* stream) {
  NvtxRange nvtx("crl_update_step");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(ctx->bound, CRL_E_NOT_BOUND, "crl_bind_params has not been called");
    CRL_REQUIRE(n_insert >= 0, CRL_E_INVALID_ARG, "n_insert must be >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_insert > 0) insert_impl(ctx, obs, act, done, n_insert, st);
    CRL_REQUIRE(ctx->size_host > 0, CRL_E_BUFFER_EMPTY, "the replay buffer is empty");
    // Every argument of the body is fixed (device counters, library workspaces,
    // bound parameters), so after one eager call it is captured once and
    // replayed.  The legacy default stream cannot be captured, and tracing needs
    // eager launches: those run eagerly.
    const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread &&
                            ctx->tracer.cls == 0;
    if (capturable && ctx->graph && ctx->graph_stream == st) {
      CRL_CHECK_CUDA(cudaGraphLaunch(ctx->graph, st));
    } else if (capturable && ctx->update_calls > 0) {
      ctx->drop_graph();
      cudaGraph_t g = nullptr;
      CRL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      try {
        update_body(ctx, st);
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      CRL_CHECK_CUDA(cudaStreamEndCapture(st, &g));
      const cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
      cudaGraphDestroy(g);
      CRL_CHECK_CUDA(e);
      ctx->graph_stream = st;
      CRL_CHECK_CUDA(cudaGraphLaunch(ctx->graph, st));
    } else {
      update_body(ctx, st);
    }
    ctx->update_calls += 1;
    deliver_floats(loss_out, ctx->loss_f, 6, st);
  });
}

int crl_get_step(crl_ctx* ctx, uint64_t* step) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && step, CRL_E_INVALID_ARG, "null argument");
    unsigned long long v = 0;
    CRL_CHECK_CUDA(cudaMemcpy(&v, &ctx->ctr->step, sizeof(v), cudaMemcpyDeviceToHost));
    *step = v;
  });
}

int crl_set_step(crl_ctx* ctx, uint64_t step) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(step != CRL_STEP_AUTO, CRL_E_INVALID_ARG, "CRL_STEP_AUTO is not a step value");
    unsigned long long v = step;
    CRL_CHECK_CUDA(cudaMemcpy(&ctx->ctr->step, &v, sizeof(v), cudaMemcpyHostToDevice));
  });
}

int crl_get_alpha(crl_ctx* ctx, float* alpha) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && alpha, CRL_E_INVALID_ARG, "null argument");
    if (!ctx->cfg.alpha_autotune) {
      *alpha = ctx->cfg.alpha;
      return;
    }
    double v[4];
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    CRL_CHECK_CUDA(cudaMemcpy(v, ctx->ctr->alpha, sizeof(v), cudaMemcpyDeviceToHost));
    *alpha = (float)std::exp(v[0]);
  });
}

int crl_sync_status(crl_ctx* ctx, void* stream, uint32_t* status) {
  unsigned v = 0;
  const int rc = guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CRL_CHECK_CUDA(cudaStreamSynchronize(st));
    CRL_CHECK_CUDA(cudaMemcpy(&v, &ctx->ctr->status, sizeof(v), cudaMemcpyDeviceToHost));
    CRL_CHECK_CUDA(cudaMemset(&ctx->ctr->status, 0, sizeof(unsigned)));
  });
  if (rc != CRL_OK) return rc;
  if (status) *status = v;
  if (v & CRL_STATUS_NONFINITE) return fail(ctx, Failure(CRL_E_NONFINITE, "a loss was not finite"));
  if (v & CRL_STATUS_TIMEOUT) return fail(ctx, Failure(CRL_E_TIMEOUT, "a bounded device wait gave up"));
  return CRL_OK;
}

int crl_set_wait_limit_ns(crl_ctx* ctx, uint32_t ns) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    CRL_CHECK_CUDA(cudaMemcpy(&ctx->ctr->wait_ns, &ns, sizeof(ns), cudaMemcpyHostToDevice));
    ctx->wait_ns = ns;
  });
}

const char* crl_last_error(const crl_ctx* ctx) { return ctx ? ctx->err.c_str() : g_thread_error.c_str(); }

int32_t crl_set_launch_overlap(int32_t enable) {
  const int32_t prev = g_launch_overlap;
  g_launch_overlap = enable ? 1 : 0;
  return prev;
}

int32_t crl_set_autotune(int32_t enable) {
  const int32_t prev = g_autotune;
  g_autotune = enable ? 1 : 0;
  return prev;
}

int32_t crl_set_gemm_kernel(int32_t mode) {
  if (mode < CRL_GEMM_ANY || mode > CRL_GEMM_CTA_PAIR) return CRL_E_INVALID_ARG;
  const int32_t prev = g_gemm_kernel;
  g_gemm_kernel = mode;
  return prev;
}

int32_t crl_gemm_tuning_report(crl_ctx* ctx, char* buf, size_t len, size_t* needed) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && needed, CRL_E_INVALID_ARG, "null argument");
    const std::string js = gemm_tuning_json(ctx->groups);
    *needed = js.size() + 1;
    CRL_REQUIRE(buf != nullptr || len == 0, CRL_E_INVALID_ARG, "null buffer with a nonzero length");
    if (len == 0) return;
    CRL_REQUIRE(len >= js.size() + 1, CRL_E_SHAPE, "the report needs " + std::to_string(js.size() + 1) + " bytes");
    memcpy(buf, js.c_str(), js.size() + 1);
  });
}

int crl_trace_start(crl_ctx* ctx, int32_t kernel_class, int32_t max_launches) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(kernel_class >= CRL_TRACE_INSERT && kernel_class <= CRL_TRACE_AUX, CRL_E_INVALID_ARG,
                "unknown kernel class");
    CRL_REQUIRE(max_launches >= 1 && max_launches <= (1 << 20), CRL_E_INVALID_ARG,
                "max_launches must lie in [1, 2^20]");
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    ctx->drop_trace_events();
    Tracer t;
    t.ev = new cudaEvent_t[2 * (size_t)max_launches];
    for (int i = 0; i < 2 * max_launches; ++i) {
      cudaError_t e = cudaEventCreate(&t.ev[i]);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(t.ev[j]);
        delete[] t.ev;
        throw Failure(CRL_E_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
      }
    }
    t.cap = max_launches;
    t.cls = kernel_class;
    ctx->tracer = t;
  });
}

int crl_trace_stop(crl_ctx* ctx, int32_t* launches, double* total_ms, double* work) {
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    Tracer& t = ctx->tracer;
    double ms = 0.0;
    for (int i = 0; i < t.n; ++i) {
      CRL_CHECK_CUDA(cudaEventSynchronize(t.ev[2 * i + 1]));
      float x = 0.f;
      CRL_CHECK_CUDA(cudaEventElapsedTime(&x, t.ev[2 * i], t.ev[2 * i + 1]));
      ms += x;
    }
    if (launches) *launches = t.n;
    if (total_ms) *total_ms = ms;
    if (work) *work = t.work;
    ctx->drop_trace_events();
  });
}

// ---- op-level entry points -------------------------------------------------
int crl_mlp_saved_bytes(const crl_mlp_desc* d, int32_t M, size_t* bytes) {
  return guarded(nullptr, [&] {
    CRL_REQUIRE(d && bytes && M >= 1, CRL_E_INVALID_ARG, "bad argument");
    CRL_REQUIRE(d->dtype == CRL_PREC_FP32 || d->dtype == CRL_PREC_FP64 || d->dtype == CRL_PREC_BF16,
                CRL_E_UNSUPPORTED, "dtype must be CRL_PREC_FP32, CRL_PREC_FP64 or CRL_PREC_BF16");
    MlpShape s{d->in0, d->in1, d->hidden, d->layers, d->out, d->layernorm ? 1 : 0};
    if (d->dtype == CRL_PREC_BF16) {
      *bytes = mlp_bf16_saved_bytes(s, M);
      CRL_REQUIRE(*bytes > 0, CRL_E_UNSUPPORTED, "this MLP shape has no BF16 buffer layout");
    } else {
      *bytes = mlp_saved_bytes(s, M, dtype_size(d->dtype));
    }
  });
}

namespace {
MlpShape checked_shape(const crl_mlp_desc* d) {
  CRL_REQUIRE(d, CRL_E_INVALID_ARG, "null descriptor");
  CRL_REQUIRE(d->in0 >= 1 && d->in1 >= 0 && d->hidden >= 1 && d->out >= 1, CRL_E_INVALID_ARG, "bad MLP sizes");
  CRL_REQUIRE(d->layers >= 1 && d->layers <= CRL_MAX_LAYERS, CRL_E_INVALID_ARG, "layers must lie in [1, 8]");
  CRL_REQUIRE(d->dtype == CRL_PREC_FP32 || d->dtype == CRL_PREC_FP64 || d->dtype == CRL_PREC_BF16,
              CRL_E_UNSUPPORTED, "dtype must be CRL_PREC_FP32, CRL_PREC_FP64 or CRL_PREC_BF16");
  return MlpShape{d->in0, d->in1, d->hidden, d->layers, d->out, d->layernorm ? 1 : 0};
}
}  // namespace

int crl_mlp_forward(const crl_mlp_desc* d, const void* params, const float* x0, const float* x1, int32_t M, void* y,
                    void* saved, void* stream) {
  return guarded(nullptr, [&] {
    const MlpShape s = checked_shape(d);
    CRL_REQUIRE(params && x0 && y && saved && M >= 1, CRL_E_INVALID_ARG, "bad argument");
    CRL_REQUIRE(s.in1 == 0 || x1, CRL_E_INVALID_ARG, "x1 is required when in1 > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->dtype == CRL_PREC_BF16)
      mlp_bf16_forward(s, static_cast<const float*>(params), x0, x1, M, static_cast<float*>(y), saved, st);
    else if (d->dtype == CRL_PREC_FP64)
      mlp_forward<double, float>(s, static_cast<const double*>(params), x0, x1, M, static_cast<double*>(y), saved, st);
    else
      mlp_forward<float, float>(s, static_cast<const float*>(params), x0, x1, M, static_cast<float*>(y), saved, st);
    check_launch("mlp forward");
  });
}

int crl_mlp_backward(const crl_mlp_desc* d, const void* params, const float* x0, const float* x1, int32_t M,
                     const void* saved, const void* dy, void* dparams, void* dx0, void* dx1, void* stream) {
  return guarded(nullptr, [&] {
    const MlpShape s = checked_shape(d);
    CRL_REQUIRE(params && x0 && saved && dy && M >= 1, CRL_E_INVALID_ARG, "bad argument");
    CRL_REQUIRE(s.in1 == 0 || x1, CRL_E_INVALID_ARG, "x1 is required when in1 > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->dtype == CRL_PREC_BF16)
      mlp_bf16_backward(s, static_cast<const float*>(params), M, saved, static_cast<const float*>(dy),
                        static_cast<float*>(dparams), static_cast<float*>(dx0), static_cast<float*>(dx1), st);
    else if (d->dtype == CRL_PREC_FP64)
      mlp_backward<double, float>(s, static_cast<const double*>(params), x0, x1, M, saved,
                                  static_cast<const double*>(dy), static_cast<double*>(dparams),
                                  static_cast<double*>(dx0), static_cast<double*>(dx1), st);
    else
      mlp_backward<float, float>(s, static_cast<const float*>(params), x0, x1, M, saved, static_cast<const float*>(dy),
                                 static_cast<float*>(dparams), static_cast<float*>(dx0), static_cast<float*>(dx1), st);
    check_launch("mlp backward");
  });
}

}  // extern "C"

namespace crl {
LossSpec checked_loss(const crl_loss_desc* d) {
  CRL_REQUIRE(d, CRL_E_INVALID_ARG, "null descriptor");
  CRL_REQUIRE(d->energy >= CRL_ENERGY_L2 && d->energy <= CRL_ENERGY_L2SQ, CRL_E_INVALID_ARG, "unknown energy");
  CRL_REQUIRE(d->loss >= CRL_LOSS_FWD && d->loss <= CRL_LOSS_NCE_BINARY, CRL_E_INVALID_ARG, "unknown loss");
  CRL_REQUIRE(d->sym_reduction == CRL_SYM_MEAN || d->sym_reduction == CRL_SYM_SUM, CRL_E_INVALID_ARG,
              "unknown sym_reduction");
  CRL_REQUIRE(d->penalty_axis >= CRL_PENALTY_ROW && d->penalty_axis <= CRL_PENALTY_BOTH, CRL_E_INVALID_ARG,
              "unknown penalty_axis");
  CRL_REQUIRE(d->temperature > 0.f && d->beta_lse >= 0.f, CRL_E_INVALID_ARG, "bad temperature or beta");
  CRL_REQUIRE(((d->dtype == CRL_PREC_FP32 || d->dtype == CRL_PREC_FP64) && d->path == CRL_PATH_PLAIN) ||
                  (d->dtype == CRL_PREC_BF16 && d->path == CRL_PATH_FUSED),
              CRL_E_UNSUPPORTED, "dtype / path must be FP32 or FP64 on the plain path, or BF16 on the fused path");
  LossSpec ls;
  ls.energy = d->energy;
  ls.loss = d->loss;
  ls.sym_reduction = d->sym_reduction;
  ls.penalty_axis = d->penalty_axis;
  ls.tau = d->temperature;
  ls.beta = d->beta_lse;
  return ls;
}
}  // namespace crl

extern "C" {

int crl_infonce_workspace_bytes(const crl_loss_desc* d, int32_t B, int32_t R, size_t* bytes) {
  return guarded(nullptr, [&] {
    const LossSpec ls = checked_loss(d);
    CRL_REQUIRE(bytes && B >= 1 && R >= 1, CRL_E_INVALID_ARG, "bad argument");
    *bytes = d->dtype == CRL_PREC_BF16 ? infonce_bf16_ws_bytes(ls, B, R)
                                       : infonce_ws_bytes(ls, B, R, dtype_size(d->dtype), d->path);
  });
}

int crl_infonce_forward(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B, int32_t R, void* loss4,
                        void* row_lse, void* col_lse, void* ws, size_t ws_bytes, void* stream) {
  return guarded(nullptr, [&] {
    const LossSpec ls = checked_loss(d);
    CRL_REQUIRE(phi && psi && loss4 && row_lse && col_lse && ws && B >= 1 && R >= 1, CRL_E_INVALID_ARG,
                "bad argument");
    CRL_REQUIRE(ws_bytes >= (d->dtype == CRL_PREC_BF16 ? infonce_bf16_ws_bytes(ls, B, R)
                                                       : infonce_ws_bytes(ls, B, R, dtype_size(d->dtype), d->path)),
                CRL_E_SHAPE, "workspace too small");
    CRL_REQUIRE(ls.loss != CRL_LOSS_FB || B >= 2, CRL_E_SHAPE, "the forward-backward objective needs B >= 2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->dtype == CRL_PREC_BF16)
      infonce_bf16_forward(ls, static_cast<const float*>(phi), static_cast<const float*>(psi), B, R,
                           static_cast<float*>(loss4), static_cast<float*>(row_lse), static_cast<float*>(col_lse), ws,
                           st);
    else if (d->dtype == CRL_PREC_FP64)
      infonce_forward<double>(ls, static_cast<const double*>(phi), static_cast<const double*>(psi), B, R,
                              static_cast<double*>(loss4), static_cast<double*>(row_lse),
                              static_cast<double*>(col_lse), ws, d->path, nullptr, nullptr, st);
    else
      infonce_forward<float>(ls, static_cast<const float*>(phi), static_cast<const float*>(psi), B, R,
                             static_cast<float*>(loss4), static_cast<float*>(row_lse), static_cast<float*>(col_lse),
                             ws, d->path, nullptr, nullptr, st);
    check_launch("infonce forward");
  });
}

int crl_infonce_backward(const crl_loss_desc* d, const void* phi, const void* psi, int32_t B, int32_t R,
                         const void* row_lse, const void* col_lse, double dtotal, void* dphi, void* dpsi, void* ws,
                         size_t ws_bytes, void* stream) {
  return guarded(nullptr, [&] {
    const LossSpec ls = checked_loss(d);
    CRL_REQUIRE(phi && psi && row_lse && col_lse && dphi && dpsi && ws && B >= 1 && R >= 1, CRL_E_INVALID_ARG,
                "bad argument");
    CRL_REQUIRE(ws_bytes >= (d->dtype == CRL_PREC_BF16 ? infonce_bf16_ws_bytes(ls, B, R)
                                                       : infonce_ws_bytes(ls, B, R, dtype_size(d->dtype), d->path)),
                CRL_E_SHAPE, "workspace too small");
    CRL_REQUIRE(ls.loss != CRL_LOSS_FB || B >= 2, CRL_E_SHAPE, "the forward-backward objective needs B >= 2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->dtype == CRL_PREC_BF16)
      infonce_bf16_backward(ls, static_cast<const float*>(phi), static_cast<const float*>(psi), B, R,
                            static_cast<const float*>(row_lse), static_cast<const float*>(col_lse), dtotal,
                            static_cast<float*>(dphi), static_cast<float*>(dpsi), ws, st);
    else if (d->dtype == CRL_PREC_FP64)
      infonce_backward<double>(ls, static_cast<const double*>(phi), static_cast<const double*>(psi), B, R,
                               static_cast<const double*>(row_lse), static_cast<const double*>(col_lse), dtotal,
                               static_cast<double*>(dphi), static_cast<double*>(dpsi), ws, d->path, st);
    else
      infonce_backward<float>(ls, static_cast<const float*>(phi), static_cast<const float*>(psi), B, R,
                              static_cast<const float*>(row_lse), static_cast<const float*>(col_lse), dtotal,
                              static_cast<float*>(dphi), static_cast<float*>(dpsi), ws, d->path, st);
    check_launch("infonce backward");
  });
}

int crl_adam_update(int32_t dtype, void* params, const void* grads, void* m, void* v, int64_t n, int32_t t, float lr,
                    float beta1, float beta2, float eps, void* stream) {
  return guarded(nullptr, [&] {
    CRL_REQUIRE(params && grads && m && v && n >= 0 && t >= 1, CRL_E_INVALID_ARG, "bad argument");
    CRL_REQUIRE(dtype == CRL_PREC_FP32 || dtype == CRL_PREC_FP64, CRL_E_UNSUPPORTED,
                "dtype must be CRL_PREC_FP32 or CRL_PREC_FP64");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == CRL_PREC_FP64)
      adam_update<double>(static_cast<double*>(params), static_cast<const double*>(grads), static_cast<double*>(m),
                          static_cast<double*>(v), n, nullptr, t, lr, beta1, beta2, eps, st);
    else
      adam_update<float>(static_cast<float*>(params), static_cast<const float*>(grads), static_cast<float*>(m),
                         static_cast<float*>(v), n, nullptr, t, lr, beta1, beta2, eps, st);
    check_launch("adam");
  });
}

}  // extern "C"
