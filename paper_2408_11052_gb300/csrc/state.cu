// Checkpoint / resume of the state the library owns: the replay buffer (rows,
// episode starts, fill), the device counters (relabel step, Adam step counts,
// the tuned entropy coefficient and its moments) and the collection stub's
// environments.  Parameters, gradients and Adam moments belong to the caller
// and are saved by it.  Relabelling and the actor noise are counter-based
// Philox draws keyed by (seed, agent) and the step, so a resumed context draws
// exactly the batches the original would have drawn.
//
// Blob layout (host memory): a header {magic, version, the configuration's
// sizes E, T, W, D, A, G, fill}, then the counters, the episode starts [E],
// the buffer state [2], the rows [E][T][W], then (if the collection stub was
// used) its states [E][D], goals [E][G], steps [E] and counter.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "ctx.h"
#include "internal.h"

namespace crl {
namespace {

constexpr uint64_t kStateMagic = 0x3174617473726c63ull;  // "crlstat1"

struct StateHeader {
  uint64_t magic;
  int32_t version, E, T, W, D, A, G, env_ready;
  int64_t size_host, total_host;
};

size_t state_bytes(const crl_ctx* c) {
  const crl_config& cf = c->cfg;
  const size_t E = (size_t)cf.E;
  size_t n = sizeof(StateHeader) + sizeof(Counters) + E * 4 + 2 * 4 + E * cf.T * (size_t)c->bd.W * 4;
  if (c->env.ready) n += E * cf.D * 4 + E * cf.G * 4 + E * 4 + 8;
  return n;
}

}  // namespace
}  // namespace crl

extern "C" {

int crl_state_bytes(crl_ctx* ctx, size_t* bytes) {
  using namespace crl;
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && bytes, CRL_E_INVALID_ARG, "null argument");
    *bytes = state_bytes(ctx);
  });
}

int crl_save_state(crl_ctx* ctx, void* host, size_t bytes) {
  using namespace crl;
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && host, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(bytes >= state_bytes(ctx), CRL_E_SHAPE, "state buffer too small (see crl_state_bytes)");
    const crl_config& cf = ctx->cfg;
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    char* p = static_cast<char*>(host);
    StateHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kStateMagic;
    h.version = 2;
    h.E = cf.E;
    h.T = cf.T;
    h.W = ctx->bd.W;
    h.D = cf.D;
    h.A = cf.A;
    h.G = cf.G;
    h.env_ready = ctx->env.ready ? 1 : 0;
    h.size_host = ctx->size_host;
    h.total_host = ctx->total_host;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    auto d2h = [&](const void* src, size_t n) {
      CRL_CHECK_CUDA(cudaMemcpy(p, src, n, cudaMemcpyDeviceToHost));
      p += n;
    };
    d2h(ctx->ctr, sizeof(Counters));
    d2h(ctx->ep_start, (size_t)cf.E * 4);
    d2h(ctx->bstate, 2 * 4);
    d2h(ctx->rows, (size_t)cf.E * cf.T * ctx->bd.W * 4);
    if (ctx->env.ready) {
      d2h(ctx->env.s, (size_t)cf.E * cf.D * 4);
      d2h(ctx->env.g, (size_t)cf.E * cf.G * 4);
      d2h(ctx->env.t, (size_t)cf.E * 4);
      d2h(ctx->env.step, 8);
    }
  });
}

int crl_load_state(crl_ctx* ctx, const void* host, size_t bytes) {
  using namespace crl;
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && host, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(bytes >= sizeof(StateHeader), CRL_E_SHAPE, "state blob too small");
    const crl_config& cf = ctx->cfg;
    StateHeader h;
    memcpy(&h, host, sizeof(h));
    CRL_REQUIRE(h.magic == kStateMagic && h.version == 2, CRL_E_INVALID_ARG, "not a state blob of this library");
    CRL_REQUIRE(h.E == cf.E && h.T == cf.T && h.W == ctx->bd.W && h.D == cf.D && h.A == cf.A && h.G == cf.G,
                CRL_E_SHAPE, "the state blob was saved from a context of other sizes");
    // the fill is min(total, T) and the device keeps total as int32 (the insert kernel's counter)
    CRL_REQUIRE(h.total_host >= 0 && h.total_host <= INT32_MAX &&
                    h.size_host == (h.total_host < cf.T ? h.total_host : (int64_t)cf.T),
                CRL_E_INVALID_ARG, "corrupt buffer fill in the state blob");
    const bool env = h.env_ready != 0;
    const size_t E = (size_t)cf.E;
    size_t need = sizeof(StateHeader) + sizeof(Counters) + E * 4 + 8 + E * cf.T * (size_t)ctx->bd.W * 4;
    if (env) need += E * cf.D * 4 + E * cf.G * 4 + E * 4 + 8;
    CRL_REQUIRE(bytes >= need, CRL_E_SHAPE, "state blob truncated");
    {
      // the device copy of {size, total} must be the header's: the sampler turns
      // it into ring-row addresses without further checks
      int32_t dev_fill[2];
      memcpy(dev_fill, static_cast<const char*>(host) + sizeof(h) + sizeof(Counters) + E * 4, sizeof(dev_fill));
      CRL_REQUIRE(dev_fill[0] == (int32_t)h.size_host && dev_fill[1] == (int32_t)h.total_host, CRL_E_INVALID_ARG,
                  "corrupt buffer fill in the state blob");
    }
    if (env && !ctx->env.ready)  // the environments are allocated the way crl_collect's first call does
      CRL_REQUIRE(ctx->bound, CRL_E_NOT_BOUND, "bind the parameters before loading a state with environments");
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    const char* p = static_cast<const char*>(host) + sizeof(h);
    auto h2d = [&](void* dst, size_t n) {
      CRL_CHECK_CUDA(cudaMemcpy(dst, p, n, cudaMemcpyHostToDevice));
      p += n;
    };
    h2d(ctx->ctr, sizeof(Counters));
    // the wait limit is a setting of this context, not part of the saved state
    CRL_CHECK_CUDA(cudaMemcpy(&ctx->ctr->wait_ns, &ctx->wait_ns, sizeof(uint32_t), cudaMemcpyHostToDevice));
    h2d(ctx->ep_start, E * 4);
    h2d(ctx->bstate, 2 * 4);
    h2d(ctx->rows, E * cf.T * (size_t)ctx->bd.W * 4);
    if (env) {
      if (!ctx->env.ready) collect_alloc(ctx, nullptr);
      h2d(ctx->env.s, E * cf.D * 4);
      h2d(ctx->env.g, E * cf.G * 4);
      h2d(ctx->env.t, E * 4);
      h2d(ctx->env.step, 8);
    }
    ctx->size_host = (int32_t)h.size_host;
    ctx->total_host = h.total_host;
    // the captured step and the BF16 weight shadows may not match any more
    ctx->drop_graph();
    for (int i = 0; i < 3; ++i) ctx->shadow_ok[i] = false;
    ctx->update_calls = 0;
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
  });
}

}  // extern "C"
