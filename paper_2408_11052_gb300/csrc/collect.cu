// Collection side of Algorithm 1 (the loop over environments) with synthetic
// dynamics standing in for the simulator, which is outside this library: it
// lets the update-to-data loop run end to end on the device (§5.6 studies the
// ratio of gradient updates to environment steps; App. B.3 fixes 1024
// environments and 1000-step episodes for Ant).
//
// Per environment step, for all E environments at once:
//   1. (mu, l) = pi(concat(s, g)), a = tanh(mu + e^clip(l) eps)   (the actor's
//      policy head; eps from Philox stream word 2 at the collection step);
//   2. the slice (s, a, done) goes into the replay buffer, done = the episode's
//      last step (t = episode_length - 1);
//   3. s' = s + 0.1 xi + 0.05 a[d mod A] with xi ~ N(0, I) (stream word 3), or,
//      after the last step of an episode, a fresh state s' ~ N(0, I) (word 4)
//      and a fresh commanded goal g' ~ N(0, I) (word 5).
// The first call draws every environment's first state and goal as a reset at
// the counter value 2^64 - 1.  All draws are Box-Muller on Philox4x64-10 blocks
// (step, env, word, d / 4) keyed (seed, agent), the same construction as the
// actor's noise.
#include <cuda_bf16.h>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "philox.cuh"
#include "trace.h"

namespace crl {

namespace {

constexpr unsigned long long kInitStep = ~0ull;

// First states and goals of every environment.  One warp per environment.
__global__ void __launch_bounds__(256) env_init_kernel(int E, int D, int G, float* __restrict__ s,
                                                      float* __restrict__ g, int32_t* __restrict__ t,
                                                      unsigned long long seed, unsigned long long agent) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int e = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (e >= E) return;
  for (int d = lane; d < D; d += kWarp) s[(size_t)e * D + d] = philox_normal<float>(kInitStep, e, 4ull, d, seed, agent);
  for (int d = lane; d < G; d += kWarp) g[(size_t)e * G + d] = philox_normal<float>(kInitStep, e, 5ull, d, seed, agent);
  if (lane == 0) t[e] = 0;
}

// Steps 2 and 3 for one environment per warp; the last block's thread 0 does
// not advance the counter (a separate launch does, after every reader).
template <typename T>
__global__ void __launch_bounds__(256) env_step_kernel(int E, int D, int A, int G, int episode_length,
                                                      float* __restrict__ s, float* __restrict__ g,
                                                      int32_t* __restrict__ t, const T* __restrict__ a,
                                                      const unsigned long long* __restrict__ step_dev,
                                                      float* __restrict__ obs, float* __restrict__ act,
                                                      uint8_t* __restrict__ done, float* __restrict__ obs_out,
                                                      float* __restrict__ act_out, uint8_t* __restrict__ done_out,
                                                      unsigned long long seed, unsigned long long agent) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int e = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (e >= E) return;
  const unsigned long long k = *step_dev;
  const int te = t[e];
  const bool last = te >= episode_length - 1;
  float* se = s + (size_t)e * D;
  for (int c = lane; c < A; c += kWarp) {
    const float av = (float)a[(size_t)e * A + c];
    act[(size_t)e * A + c] = av;
    if (act_out) act_out[(size_t)e * A + c] = av;
  }
  for (int d = lane; d < D; d += kWarp) {
    const float x = se[d];
    obs[(size_t)e * D + d] = x;
    if (obs_out) obs_out[(size_t)e * D + d] = x;
    float nx;
    if (last) {
      nx = philox_normal<float>(k, e, 4ull, d, seed, agent);
    } else {
      const float xi = philox_normal<float>(k, e, 3ull, d, seed, agent);
      nx = x + 0.1f * xi + 0.05f * (float)a[(size_t)e * A + (d % A)];
    }
    se[d] = nx;
  }
  if (last)
    for (int d = lane; d < G; d += kWarp) g[(size_t)e * G + d] = philox_normal<float>(k, e, 5ull, d, seed, agent);
  if (lane == 0) {
    done[e] = last ? 1 : 0;
    if (done_out) done_out[e] = last ? 1 : 0;
    t[e] = last ? 0 : te + 1;
  }
}

template <typename T>
void collect_steps(crl_ctx* c, int n, int episode_length, float* obs_out, float* act_out, uint8_t* done_out,
                   cudaStream_t st) {
  const crl_config& cf = c->cfg;
  crl_ctx::Envs& v = c->env;
  const int E = cf.E;
  const T* params = static_cast<const T*>(c->nets[CRL_NET_PI].params);
  ActorSpec as;
  memset(&as, 0, sizeof(as));
  as.A = cf.A;
  as.energy = cf.energy;
  as.tau = cf.temperature;
  as.alpha = cf.alpha;
  for (int i = 0; i < n; ++i) {
    mlp_forward<T, float>(c->shapes[CRL_NET_PI], params, v.s, v.g, E, static_cast<T*>(v.pi_out), v.saved, st);
    actor_head_forward<T>(as, static_cast<const T*>(v.pi_out), nullptr, v.step, cf.seed, cf.agent, E,
                          static_cast<T*>(v.a), static_cast<T*>(v.logpi), static_cast<T*>(v.eps), st, nullptr, 0,
                          0, /*noise_extra=*/1);
    {
      TraceLaunch tr(CRL_TRACE_AUX, st, (double)E * (2.0 * cf.D * 4 + cf.A * (sizeof(T) + 4)));
      launch_k(env_step_kernel<T>, dim3(ceil_div(E, 8)), dim3(256), 0, st, E, cf.D, cf.A, cf.G, episode_length,
               v.s, v.g, v.t, static_cast<const T*>(v.a), (const unsigned long long*)v.step, v.obs, v.act, v.done,
               obs_out ? obs_out + (size_t)i * E * cf.D : nullptr, act_out ? act_out + (size_t)i * E * cf.A : nullptr,
               done_out ? done_out + (size_t)i * E : nullptr, (unsigned long long)cf.seed,
               (unsigned long long)cf.agent);
    }
    launch_bump_u64(v.step, st);
    insert_impl(c, v.obs, v.act, v.done, 1, st);
  }
}

}  // namespace

// Allocates the collection stub's environments and staging and resets every
// environment (episode starts drawn from the collection stream at step 0).
void collect_alloc(crl_ctx* ctx, cudaStream_t st) {
  const crl_config& cf = ctx->cfg;
  crl_ctx::Envs& v = ctx->env;
  const size_t es = ctx->esz;
  const int E = cf.E;
  v.s = static_cast<float*>(ctx->dalloc((size_t)E * cf.D * sizeof(float)));
  v.g = static_cast<float*>(ctx->dalloc((size_t)E * cf.G * sizeof(float)));
  v.t = static_cast<int32_t*>(ctx->dalloc((size_t)E * sizeof(int32_t)));
  v.step = static_cast<unsigned long long*>(ctx->dalloc(sizeof(unsigned long long)));
  v.pi_out = ctx->dalloc((size_t)E * 2 * cf.A * es);
  v.a = ctx->dalloc((size_t)E * cf.A * es);
  v.logpi = ctx->dalloc((size_t)E * es);
  v.eps = ctx->dalloc((size_t)E * cf.A * es);
  v.saved = ctx->dalloc(mlp_saved_bytes(ctx->shapes[CRL_NET_PI], E, es));
  v.obs = static_cast<float*>(ctx->dalloc((size_t)E * cf.D * sizeof(float)));
  v.act = static_cast<float*>(ctx->dalloc((size_t)E * cf.A * sizeof(float)));
  v.done = static_cast<uint8_t*>(ctx->dalloc((size_t)E));
  CRL_CHECK_CUDA(cudaMemsetAsync(v.step, 0, sizeof(unsigned long long), st));
  launch_k(env_init_kernel, dim3(ceil_div(E, 8)), dim3(256), 0, st, E, cf.D, cf.G, v.s, v.g, v.t,
           (unsigned long long)cf.seed, (unsigned long long)cf.agent);
  v.ready = true;
}

}  // namespace crl

extern "C" int crl_collect(crl_ctx* ctx, int32_t n_steps, int32_t episode_length, float* obs_out, float* act_out,
                           uint8_t* done_out, void* stream) {
  using namespace crl;
  NvtxRange nvtx("crl_collect");
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    CRL_REQUIRE(ctx->bound, CRL_E_NOT_BOUND, "crl_bind_params has not been called");
    CRL_REQUIRE(n_steps >= 1, CRL_E_INVALID_ARG, "n_steps must be >= 1");
    CRL_REQUIRE(episode_length >= 1, CRL_E_INVALID_ARG, "episode_length must be >= 1");
    CRL_REQUIRE(!obs_out || !is_host_pointer(obs_out), CRL_E_INVALID_ARG, "obs_out must be device memory");
    CRL_REQUIRE(!act_out || !is_host_pointer(act_out), CRL_E_INVALID_ARG, "act_out must be device memory");
    CRL_REQUIRE(!done_out || !is_host_pointer(done_out), CRL_E_INVALID_ARG, "done_out must be device memory");
    const crl_config& cf = ctx->cfg;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ctx->env.ready) collect_alloc(ctx, st);
    if (cf.precision == CRL_PREC_FP64)
      collect_steps<double>(ctx, n_steps, episode_length, obs_out, act_out, done_out, st);
    else
      collect_steps<float>(ctx, n_steps, episode_length, obs_out, act_out, done_out, st);
    check_launch("collect");
  });
}
