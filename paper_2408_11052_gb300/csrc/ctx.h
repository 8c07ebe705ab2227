// Library-internal state of a context and the helpers shared by the C ABI
// translation units (api.cu: single-agent calls; sweep.cu: several agents).
#pragma once

#include <cuda_runtime.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/crl.h"
#include "energy_tc.cuh"
#include "internal.h"
#include "mlp_bf16.cuh"
#include "tables.h"
#include "trace.h"

namespace crl {

struct Counters {
  unsigned long long step;       // next Philox step for CRL_STEP_AUTO
  unsigned long long last_step;  // step of the last sample (actor noise)
  int t_critic;                  // Adam step counters (incremented by the loss kernels)
  int t_actor;
  unsigned status;               // CRL_STATUS_* bits
  unsigned wait_ns;              // bounded-wait limit of the kernels (0: 1 s); read as the word after status
  unsigned ticket_actor;         // last-block ticket of the actor loss kernel (zero between launches)
  unsigned pad_;
  double alpha[4];               // entropy-coefficient auto-tuning: log alpha, Adam m, v, alpha last used
};

class Failure {
 public:
  int code;
  std::string msg;
  Failure(int c, std::string m) : code(c), msg(std::move(m)) {}
};

#define CRL_CHECK_CUDA(expr)                                                                     \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) throw Failure(CRL_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CRL_REQUIRE(cond, code, msg) \
  do {                               \
    if (!(cond)) throw Failure((code), (msg)); \
  } while (0)

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Failure(CRL_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_host_pointer(const void* p);
// The device address of pinned, mapped host memory, or nullptr (device, pageable or unknown memory).
const void* host_device_alias(const void* p);
// Both answers from one driver query: host = is_host_pointer(p), alias =
// host_device_alias(p).
struct PointerKind {
  bool host;
  const void* alias;
};
PointerKind classify_pointer(const void* p);
size_t dtype_size(int precision);
MlpShape net_shape(const crl_config& c, int net);
void validate_config(const crl_config& c);

}  // namespace crl

using namespace crl;

struct crl_ctx {
  crl_config cfg{};
  int device = 0;
  size_t esz = 4;
  BufferDev bd{};
  float* rows = nullptr;
  int32_t* ep_start = nullptr;
  int32_t* bstate = nullptr;
  unsigned long long* gq = nullptr;
  int32_t size_host = 0;
  int64_t total_host = 0;
  Counters* ctr = nullptr;
  uint32_t wait_ns = 0;     // host copy of ctr->wait_ns (crl_set_wait_limit_ns)
  bool bound = false;
  int bind_generation = 0;  // incremented by crl_bind_params and crl_set_logit_stats (sweeps rebuild)
  crl_net_ptrs nets[3]{};
  MlpShape shapes[3]{};
  int64_t counts[3]{};
  // workspaces
  std::vector<void*> allocs;
  void* saved[3]{};
  void *phi = nullptr, *psi = nullptr, *dphi = nullptr, *dpsi = nullptr;
  void *row_lse = nullptr, *col_lse = nullptr, *loss = nullptr, *ws = nullptr;
  size_t ws_bytes = 0;
  void *pi_out = nullptr, *a_new = nullptr, *logpi = nullptr, *eps_used = nullptr, *fdiag = nullptr;
  void *da = nullptr, *dout = nullptr;
  void* actor_ws = nullptr;  // per-block partial sums of the actor loss
  float* loss_f = nullptr;  // 8 floats: float copy of the loss parts
  float *bs = nullptr, *ba = nullptr, *bg = nullptr;  // batch of crl_update_step
  float* bg_act = nullptr;                             // the actor's goals (random-goal mix)
  // collection stub (crl_collect): environment state and staging, allocated on first use
  struct Envs {
    bool ready = false;
    float* s = nullptr;                   // [E][D] current states
    float* g = nullptr;                   // [E][G] current commanded goals
    int32_t* t = nullptr;                 // [E] step within the episode
    unsigned long long* step = nullptr;   // next collection step (Philox counter)
    void *pi_out = nullptr, *a = nullptr, *logpi = nullptr, *eps = nullptr, *saved = nullptr;
    float *obs = nullptr, *act = nullptr;  // one time slice for the insert
    uint8_t* done = nullptr;
  } env;
  // logit statistics of the critic steps (crl_set_logit_stats): [2] floats and per-tile FP64 sums
  bool stats_on = false;
  float* stats = nullptr;
  double* stats_part = nullptr;
  // host-input staging for crl_buffer_insert
  void* stage = nullptr;
  size_t stage_bytes = 0;
  Tracer tracer;
  // BF16 tensor-core networks (precision CRL_PREC_BF16)
  bool bf16 = false;
  BfNet bf[3];
  bool shadow_ok[3] = {false, false, false};  // BF16 shadows match the FP32 master weights
  bool fused = false;
  EnergyTc etc;
  void* etc_ws = nullptr;
  // device problem tables of the grouped tensor-core GEMMs, and other launch tables
  GemmGroups groups;
  BlobCache tables;
  // CUDA graph of relabel -> critic -> actor, replayed by crl_update_step
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  int update_calls = 0;
  std::string err;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    CRL_CHECK_CUDA(cudaMalloc(&p, bytes > 0 ? bytes : 16));
    allocs.push_back(p);
    return p;
  }
  void drop_trace_events() {
    if (tracer.ev) {
      for (int i = 0; i < 2 * tracer.cap; ++i) cudaEventDestroy(tracer.ev[i]);
      delete[] tracer.ev;
    }
    tracer = Tracer();
  }
  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_stream = nullptr;
  }
  ~crl_ctx() {
    drop_graph();
    drop_trace_events();
    for (void* p : allocs) cudaFree(p);
    if (stage) cudaFree(stage);
  }
};

namespace crl {

int fail(crl_ctx* ctx, const Failure& f);
LossSpec loss_spec(const crl_config& c);
void deliver_floats(float* dst, const float* src, int n, cudaStream_t st);
void* ctx_alloc(void* owner, size_t bytes);
void bf_maps(crl_ctx* c, int net, int B);
void bf_check(const char* err);
void bf_refresh(crl_ctx* c, int net, bool refresh, cudaStream_t st);
AdamShadowNet adam_net_of(crl_ctx* c, int net, const int* t, float lr);
// The actor's sizes, energy, temperature, fixed alpha and (with alpha_autotune)
// the device state of the tuned alpha.
ActorSpec actor_spec_of(crl_ctx* c);
// Resets the tuned alpha to log(cfg.alpha) with zero Adam moments (synchronous).
void reset_alpha(crl_ctx* c);
void insert_impl(crl_ctx* c, const float* obs, const float* act, const uint8_t* done, int n, cudaStream_t st);
void relabel_impl(crl_ctx* c, uint64_t step, int B, float* s, float* a, float* g, int32_t* idx, cudaStream_t st,
                  bool pack_bf16 = false, bool bump = true);
RelabelArgs relabel_args(crl_ctx* c, uint64_t step, int B, float* s, float* a, float* g, int32_t* idx,
                         bool pack_bf16);
void update_body(crl_ctx* ctx, cudaStream_t st);
// Logit statistics of a critic step's representations phi, psi [B][R] (float,
// or double when fp64) into c->stats, when switched on (stats.cu).
void logit_stats_alloc(crl_ctx* c);
void logit_stats_launch(crl_ctx* c, const void* phi, const void* psi, int B, bool fp64, cudaStream_t st);
// Allocates and resets the collection stub's environments (crl_collect's first call).
void collect_alloc(crl_ctx* ctx, cudaStream_t st);

// The loss of a crl_loss_desc after validation (throws Failure: CRL_E_INVALID_ARG
// for an unknown energy, objective, reduction or penalty axis, or a bad
// temperature / beta; CRL_E_UNSUPPORTED for a dtype / path this build lacks).
LossSpec checked_loss(const crl_loss_desc* d);

// Runs one entry point: maps internal failures to status codes and makes the
// context's tracer visible to the launch sites for the duration of the call.
template <typename F>
int guarded(crl_ctx* ctx, F&& body) {
  struct TracerScope {
    explicit TracerScope(crl_ctx* c) { g_tracer = (c && c->tracer.cls) ? &c->tracer : nullptr; }
    ~TracerScope() { g_tracer = nullptr; }
  } scope(ctx);
  try {
    body();
    return CRL_OK;
  } catch (const Failure& f) {
    return fail(ctx, f);
  } catch (const std::bad_alloc&) {
    return fail(ctx, Failure(CRL_E_INVALID_ARG, "host allocation failed"));
  } catch (...) {
    return fail(ctx, Failure(CRL_E_INVALID_ARG, "unexpected internal error"));
  }
}

}  // namespace crl
