// Batched sweep: many independent agents (seeds or hyperparameter settings,
// each a full context with its own replay buffer, networks and Philox key)
// advanced by one update step together (the multi-seed experiments of arXiv
// 2408.11052, §5, as one GPU program).
//
// grouped = 1 (BF16): every kernel of the step is one launch over all agents --
// the grouped tcgen05 GEMMs take every agent's networks of one layer as one
// problem list, and the other kernels map blocks to agents through block-offset
// tables -- so the step is ~25 launches whatever the number of agents.
// grouped = 0 (any precision): the agents' own update steps one after another.
// Either way the step is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace crl;

struct crl_sweep {
  std::vector<crl_ctx*> agents;
  int grouped = 0;
  GemmGroups groups;
  BlobCache tables;
  unsigned* status = nullptr;   // device status word of the launches shared by all agents, then their wait limit
  float* loss_all = nullptr;    // [n][6] float losses of the last step
  std::vector<int> generation;  // agents' bind generations the tables were built for
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  int calls = 0;
  std::string err;

  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_stream = nullptr;
  }
  ~crl_sweep() {
    drop_graph();
    for (crl_ctx* c : agents) crl_destroy(c);
    if (status) cudaFree(status);
    if (loss_all) cudaFree(loss_all);
  }
};

namespace {

int sweep_fail(crl_sweep* sw, const Failure& f) {
  if (sw) sw->err = f.msg;
  return fail(nullptr, f);
}

// Runs one sweep entry point; launches are traced by agent 0's tracer when it is on.
template <typename F>
int sweep_guarded(crl_sweep* sw, F&& body) {
  struct TracerScope {
    explicit TracerScope(crl_sweep* s) {
      crl_ctx* c = (s && !s->agents.empty()) ? s->agents[0] : nullptr;
      g_tracer = (c && c->tracer.cls) ? &c->tracer : nullptr;
    }
    ~TracerScope() { g_tracer = nullptr; }
  } scope(sw);
  try {
    body();
    return CRL_OK;
  } catch (const Failure& f) {
    return sweep_fail(sw, f);
  } catch (const std::bad_alloc&) {
    return sweep_fail(sw, Failure(CRL_E_INVALID_ARG, "host allocation failed"));
  } catch (...) {
    return sweep_fail(sw, Failure(CRL_E_INVALID_ARG, "unexpected internal error"));
  }
}

__global__ void gather_losses_kernel(const float* const* __restrict__ src, float* __restrict__ dst, int n) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 6 * n) dst[i] = src[i / 6][i % 6];
}

void sweep_check(const char* err) {
  if (err) throw Failure(CRL_E_CUDA, std::string("sweep: ") + err);
}

// One update step of every agent with one launch per kernel (BF16).
void body_grouped(crl_sweep* sw, cudaStream_t st) {
  const int na = (int)sw->agents.size();
  unsigned* status = sw->status;
  // ---- relabel (packs every network input in BF16)
  {
    std::vector<RelabelTask> tasks(na);
    std::vector<int> begin(na + 1, 0);
    double bytes = 0.0;
    for (int i = 0; i < na; ++i) {
      crl_ctx* c = sw->agents[i];
      const crl_config& cf = c->cfg;
      CRL_REQUIRE(c->size_host > 0, CRL_E_BUFFER_EMPTY, "an agent's replay buffer is empty");
      memset(&tasks[i], 0, sizeof(RelabelTask));
      tasks[i].bd = c->bd;
      tasks[i].ra = relabel_args(c, CRL_STEP_AUTO, cf.B, c->bs, c->ba, c->bg, nullptr, true);
      begin[i + 1] = begin[i] + relabel_blocks(tasks[i].ra);
      bytes += cf.B * ((cf.D + cf.A + 1 + cf.G) * 4.0 + (cf.D + cf.A + cf.G) * 4.0);
    }
    const char* err = nullptr;
    const RelabelTask* dt = sw->tables.get(tasks, st, &err);
    sweep_check(dt ? nullptr : err);
    const int* db = sw->tables.get(begin, st, &err);
    sweep_check(db ? nullptr : err);
    launch_relabel_multi(dt, db, na, begin[na], bytes, true, 0, st);
  }
  // random-goal actor mix: the agents with alpha_rg > 0 draw their actors' goals
  // now and take the single-agent path's unfused actor head (below)
  for (crl_ctx* c : sw->agents)
    if (c->cfg.alpha_rg > 0.f)
      launch_actor_goals(c->cfg.B, c->cfg.G, c->bg, c->bg_act, c->cfg.seed, c->cfg.agent, &c->ctr->last_step,
                         c->cfg.alpha_rg, st);
  // ---- critic: phi, psi and pi forward (pi's parameters do not change before the actor step)
  std::vector<BfPass> fwd, bwd;
  std::vector<EnergyOut> eo(2 * na);
  for (int i = 0; i < na; ++i) {
    crl_ctx* c = sw->agents[i];
    eo[2 * i] = EnergyOut{c->etc.X, c->etc.auxX, c->cfg.energy};
    eo[2 * i + 1] = EnergyOut{c->etc.Y, c->etc.auxY, c->cfg.energy};
  }
  for (int i = 0; i < na; ++i) {
    crl_ctx* c = sw->agents[i];
    const int B = c->cfg.B;
    for (int net = 0; net < 3; ++net) {
      bf_maps(c, net, B);
      bf_refresh(c, net, false, st);
    }
    const crl_net_ptrs* np = c->nets;
    fwd.push_back({&c->bf[CRL_NET_PHI], static_cast<const float*>(np[CRL_NET_PHI].params),
                   static_cast<float*>(np[CRL_NET_PHI].grads), nullptr, B, &eo[2 * i]});
    fwd.push_back({&c->bf[CRL_NET_PSI], static_cast<const float*>(np[CRL_NET_PSI].params),
                   static_cast<float*>(np[CRL_NET_PSI].grads), nullptr, B, &eo[2 * i + 1]});
    bwd.push_back(fwd[fwd.size() - 2]);
    bwd.push_back(fwd.back());
    bwd[bwd.size() - 2].energy_out = nullptr;
    bwd.back().energy_out = nullptr;
    fwd.push_back({&c->bf[CRL_NET_PI], static_cast<const float*>(np[CRL_NET_PI].params), nullptr, nullptr, B});
  }
  sweep_check(bf_forward(sw->groups, fwd.data(), (int)fwd.size(), status, st));
  for (crl_ctx* c : sw->agents)
    logit_stats_launch(c, c->bf[CRL_NET_PHI].y, c->bf[CRL_NET_PSI].y, c->cfg.B, false, st);
  // ---- fused energy + InfoNCE + penalty, forward and backward
  std::vector<EnergyAgent> ea;
  for (crl_ctx* c : sw->agents) {
    const int B = c->cfg.B;
    BfNet& P = c->bf[CRL_NET_PHI];
    BfNet& Q = c->bf[CRL_NET_PSI];
    sweep_check(energy_tc_maps(c->etc, B));
    ea.push_back(EnergyAgent{&c->etc, loss_spec(c->cfg), B, P.y, Q.y, static_cast<float*>(c->loss),
                             static_cast<float*>(c->row_lse), static_cast<float*>(c->col_lse), c->etc_ws,
                             &c->ctr->t_critic, P.dz[P.layers], Q.dz[Q.layers], &c->ctr->status});
  }
  // (the operands were written by the encoders' output layers: no prepare stage)
  for (int stage = 1; stage < 3; ++stage) sweep_check(energy_tc_multi(sw->tables, ea, stage, st));
  sweep_check(bf_backward(sw->groups, bwd.data(), (int)bwd.size(), status, st));
  // Adam for every phi and psi; the actors' head forwards (a' into phi's input:
  // they read only the policies' outputs) run as extra blocks of the same launch
  {
    std::vector<HeadFwdArgs<float>> hf;
    for (crl_ctx* c : sw->agents) {
      const crl_config& cf = c->cfg;
      if (cf.alpha_rg > 0.f) continue;   // its head runs with the actor's own goals below
      BfNet& P = c->bf[CRL_NET_PHI];
      HeadFwdArgs<float> h;
      memset(&h, 0, sizeof(h));   // member by member: zeroed padding keys the device table
      h.B = cf.B;
      h.A = cf.A;
      h.out = c->bf[CRL_NET_PI].y;
      h.eps = nullptr;
      h.step_dev = &c->ctr->last_step;
      h.seed = cf.seed;
      h.agent = cf.agent;
      h.a_new = static_cast<float*>(c->a_new);
      h.logpi = static_cast<float*>(c->logpi);
      h.eps_used = static_cast<float*>(c->eps_used);
      h.x0 = P.x0;
      h.x0_ld = bf_net_x0_ld(P);
      h.x0_col = P.s.in0;
      hf.push_back(h);
    }
    std::vector<AdamShadowNet> an;
    for (crl_ctx* c : sw->agents) {
      an.push_back(adam_net_of(c, CRL_NET_PHI, &c->ctr->t_critic, c->cfg.lr_critic));
      an.push_back(adam_net_of(c, CRL_NET_PSI, &c->ctr->t_critic, c->cfg.lr_critic));
    }
    sweep_check(adam_shadow_update(sw->tables, an.data(), (int)an.size(), st, &hf));
  }
  // ---- actor, goal-mixing agents first: pi(s, g_actor) and psi(g_actor)
  // inputs, pi's forward, the head's forward and phi's input (s, a')
  {
    std::vector<BfPass> pis;
    for (crl_ctx* c : sw->agents) {
      if (c->cfg.alpha_rg <= 0.f) continue;
      const int B = c->cfg.B;
      bf_net_pack_input(c->bf[CRL_NET_PI], c->bs, c->bg_act, B, st);
      bf_net_pack_input(c->bf[CRL_NET_PSI], c->bg_act, nullptr, B, st);
      pis.push_back({&c->bf[CRL_NET_PI], static_cast<const float*>(c->nets[CRL_NET_PI].params), nullptr, nullptr, B});
    }
    if (!pis.empty()) {
      sweep_check(bf_forward(sw->groups, pis.data(), (int)pis.size(), status, st));
      for (crl_ctx* c : sw->agents) {
        if (c->cfg.alpha_rg <= 0.f) continue;
        const crl_config& cf = c->cfg;
        float* a_new = static_cast<float*>(c->a_new);
        actor_head_forward<float>(actor_spec_of(c), c->bf[CRL_NET_PI].y, nullptr, &c->ctr->last_step, cf.seed,
                                  cf.agent, cf.B, a_new, static_cast<float*>(c->logpi),
                                  static_cast<float*>(c->eps_used), st);
        bf_net_pack_input(c->bf[CRL_NET_PHI], c->bs, a_new, cf.B, st);
      }
    }
  }
  // ---- actor: phi and psi forward with the updated critic, diagonal energy +
  // loss, phi's input gradient, head backward, pi backward
  std::vector<BfPass> afwd, phi_b, pi_b;
  for (crl_ctx* c : sw->agents) {
    const int B = c->cfg.B;
    const crl_net_ptrs* np = c->nets;
    afwd.push_back({&c->bf[CRL_NET_PHI], static_cast<const float*>(np[CRL_NET_PHI].params), nullptr,
                    static_cast<float*>(c->da), B});
    phi_b.push_back(afwd.back());
    afwd.push_back({&c->bf[CRL_NET_PSI], static_cast<const float*>(np[CRL_NET_PSI].params), nullptr, nullptr, B});
    pi_b.push_back({&c->bf[CRL_NET_PI], static_cast<const float*>(np[CRL_NET_PI].params),
                    static_cast<float*>(np[CRL_NET_PI].grads), nullptr, B});
  }
  sweep_check(bf_forward(sw->groups, afwd.data(), (int)afwd.size(), status, st));
  {
    std::vector<ActorLossArgs<float>> al;
    for (crl_ctx* c : sw->agents) {
      const crl_config& cf = c->cfg;
      BfNet& P = c->bf[CRL_NET_PHI];
      BfNet& Q = c->bf[CRL_NET_PSI];
      ActorLossArgs<float> t;
      memset(&t, 0, sizeof(t));
      t.B = cf.B;
      t.R = cf.repr;
      t.energy = cf.energy;
      t.tau = (double)cf.temperature;
      t.alpha = (double)cf.alpha;
      t.phi = P.y;
      t.psi = Q.y;
      t.logpi = static_cast<const float*>(c->logpi);
      t.fdiag = static_cast<float*>(c->fdiag);
      t.dphi = nullptr;
      t.dz = P.dz[P.layers];
      t.ldz = P.L[P.layers].out_pad;
      t.partial = static_cast<float*>(c->actor_ws);
      t.ticket = &c->ctr->ticket_actor;
      t.loss2 = static_cast<float*>(c->loss) + 4;
      t.status = &c->ctr->status;
      t.t_bump = &c->ctr->t_actor;
      t.step_bump = &c->ctr->step;
      t.last_step = &c->ctr->last_step;
      t.tune = actor_spec_of(c).tune;
      al.push_back(t);
    }
    sweep_check(actor_loss_multi(sw->tables, al, st));
  }
  sweep_check(bf_backward(sw->groups, phi_b.data(), (int)phi_b.size(), status, st));
  {
    std::vector<HeadBwdArgs<float>> hb;
    for (crl_ctx* c : sw->agents) {
      const crl_config& cf = c->cfg;
      BfNet& PI = c->bf[CRL_NET_PI];
      HeadBwdArgs<float> h;
      memset(&h, 0, sizeof(h));
      h.B = cf.B;
      h.A = cf.A;
      h.alpha = (double)cf.alpha;
      h.out = PI.y;
      h.eps_used = static_cast<const float*>(c->eps_used);
      h.da = static_cast<const float*>(c->da);
      h.dout = nullptr;
      h.dz = PI.dz[PI.layers];
      h.ldz = PI.L[PI.layers].out_pad;
      h.alpha_used = cf.alpha_autotune ? c->ctr->alpha + 3 : nullptr;
      hb.push_back(h);
    }
    sweep_check(actor_head_backward_multi(sw->tables, hb, st));
  }
  sweep_check(bf_backward(sw->groups, pi_b.data(), (int)pi_b.size(), status, st));
  {
    std::vector<AdamShadowNet> an;
    for (crl_ctx* c : sw->agents) an.push_back(adam_net_of(c, CRL_NET_PI, &c->ctr->t_actor, c->cfg.lr_actor));
    sweep_check(adam_shadow_update(sw->tables, an.data(), (int)an.size(), st));
  }
  check_launch("sweep step");
}

void sweep_body(crl_sweep* sw, cudaStream_t st) {
  if (sw->grouped) {
    body_grouped(sw, st);
  } else {
    for (crl_ctx* c : sw->agents) {
      CRL_REQUIRE(c->size_host > 0, CRL_E_BUFFER_EMPTY, "an agent's replay buffer is empty");
      update_body(c, st);
    }
  }
  // every agent's six loss values into one buffer
  std::vector<const float*> src;
  for (crl_ctx* c : sw->agents) src.push_back(c->loss_f);
  const char* err = nullptr;
  const float* const* dsrc = sw->tables.get(src, st, &err);
  sweep_check(dsrc ? nullptr : err);
  const int n = (int)sw->agents.size();
  TraceLaunch tr(CRL_TRACE_AUX, st, 48.0 * n);
  launch_k(gather_losses_kernel, dim3(ceil_div(6 * n, 256)), dim3(256), 0, st, dsrc, sw->loss_all, n);
  check_launch("sweep loss gather");
}

}  // namespace

extern "C" {

int crl_sweep_create(const crl_config* cfgs, int32_t n, int32_t grouped, crl_sweep** out) {
  if (out) *out = nullptr;
  crl_sweep* sw = nullptr;
  const int rc = sweep_guarded(nullptr, [&] {
    CRL_REQUIRE(cfgs && out, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(n >= 1 && n <= kMaxAgents, CRL_E_INVALID_ARG, "a sweep holds 1 to 64 agents");
    const crl_config& c0 = cfgs[0];
    for (int i = 0; i < n; ++i) {
      const crl_config& c = cfgs[i];
      CRL_REQUIRE(c.precision == c0.precision && c.path == c0.path && c.hidden == c0.hidden &&
                      c.layers == c0.layers && (c.layernorm != 0) == (c0.layernorm != 0),
                  CRL_E_INVALID_ARG, "the agents of a sweep share precision, path, hidden width, depth and LayerNorm");
    }
    if (grouped) {
      CRL_REQUIRE(c0.precision == CRL_PREC_BF16 && c0.path == CRL_PATH_FUSED, CRL_E_UNSUPPORTED,
                  "the grouped sweep runs the BF16 fused path");
    }
    sw = new crl_sweep();
    sw->grouped = grouped ? 1 : 0;
    for (int i = 0; i < n; ++i) {
      crl_ctx* c = nullptr;
      const int r = crl_create(&cfgs[i], &c);
      if (r != CRL_OK) throw Failure(r, std::string("agent ") + std::to_string(i) + ": " + crl_last_error(nullptr));
      sw->agents.push_back(c);
    }
    // the status word and, after it, the wait limit of the launches (0: the default)
    CRL_CHECK_CUDA(cudaMalloc(&sw->status, 2 * sizeof(unsigned)));
    CRL_CHECK_CUDA(cudaMemset(sw->status, 0, 2 * sizeof(unsigned)));
    CRL_CHECK_CUDA(cudaMalloc(&sw->loss_all, (size_t)6 * n * sizeof(float)));
    CRL_CHECK_CUDA(cudaMemset(sw->loss_all, 0, (size_t)6 * n * sizeof(float)));
  });
  if (rc != CRL_OK) {
    delete sw;
    return rc;
  }
  *out = sw;
  return CRL_OK;
}

int crl_sweep_destroy(crl_sweep* sw) {
  if (!sw) return CRL_OK;
  cudaDeviceSynchronize();
  delete sw;
  return CRL_OK;
}

int crl_sweep_agent(crl_sweep* sw, int32_t i, crl_ctx** ctx) {
  return sweep_guarded(sw, [&] {
    CRL_REQUIRE(sw && ctx, CRL_E_INVALID_ARG, "null argument");
    CRL_REQUIRE(i >= 0 && i < (int)sw->agents.size(), CRL_E_INVALID_ARG, "agent index out of range");
    *ctx = sw->agents[i];
  });
}

int crl_sweep_update_step(crl_sweep* sw, const float* const* obs, const float* const* act,
                          const uint8_t* const* done, int32_t n_insert, float* loss_out, void* stream) {
  NvtxRange nvtx("crl_sweep_update_step");
  return sweep_guarded(sw, [&] {
    CRL_REQUIRE(sw, CRL_E_INVALID_ARG, "null sweep");
    CRL_REQUIRE(n_insert >= 0, CRL_E_INVALID_ARG, "n_insert must be >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int na = (int)sw->agents.size();
    for (crl_ctx* c : sw->agents) CRL_REQUIRE(c->bound, CRL_E_NOT_BOUND, "an agent's parameters are not bound");
    // a re-bound agent invalidates the tables (they hold parameter pointers) and the graph
    std::vector<int> gen;
    for (crl_ctx* c : sw->agents) gen.push_back(c->bind_generation);
    if (gen != sw->generation) {
      CRL_CHECK_CUDA(cudaStreamSynchronize(st));
      sw->drop_graph();
      sw->groups.reset();
      sw->tables.reset();
      sw->generation = gen;
      sw->calls = 0;
    }
    if (n_insert > 0) {
      CRL_REQUIRE(obs && act && done, CRL_E_INVALID_ARG, "obs, act and done must be non-null");
      // device pointers, or the device aliases of pinned host inputs (read in place)
      bool device = true;
      std::vector<const void*> in(3 * (size_t)na);
      for (int i = 0; i < na; ++i) {
        CRL_REQUIRE(obs[i] && act[i] && done[i], CRL_E_INVALID_ARG, "obs, act and done must be non-null");
        const void* ptrs[3] = {obs[i], act[i], done[i]};
        for (int j = 0; j < 3; ++j) {
          const PointerKind k = classify_pointer(ptrs[j]);
          const void* q = k.host ? k.alias : ptrs[j];
          device = device && q != nullptr;
          in[3 * i + j] = q;
        }
      }
      if (device && na <= kMaxAgents) {
        // one launch over every agent's buffer (arguments by value: they change every step)
        InsertMulti m;
        memset(&m, 0, sizeof(m));
        m.n = na;
        for (int i = 0; i < na; ++i) {
          crl_ctx* c = sw->agents[i];
          CRL_REQUIRE(c->total_host + n_insert < ((int64_t)1 << 31) - 1, CRL_E_INVALID_ARG,
                      "more than 2^31 - 2 steps inserted per environment");
          const int i0 = n_insert > c->cfg.T ? n_insert - c->cfg.T : 0;
          m.a[i] = InsertArgs{c->bd, static_cast<const float*>(in[3 * i]), static_cast<const float*>(in[3 * i + 1]),
                              static_cast<const uint8_t*>(in[3 * i + 2]), n_insert, i0, (long long)c->total_host};
          m.begin[i + 1] = m.begin[i] + insert_blocks(c->bd);
        }
        launch_buffer_insert_multi(m, st);
        check_launch("sweep insert");
        for (crl_ctx* c : sw->agents) {
          c->total_host += n_insert;
          c->size_host = (int32_t)std::min<int64_t>(c->total_host, c->cfg.T);
        }
      } else {
        for (int i = 0; i < na; ++i) insert_impl(sw->agents[i], obs[i], act[i], done[i], n_insert, st);
      }
    }
    const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    bool tracing = false;
    for (crl_ctx* c : sw->agents) tracing = tracing || c->tracer.cls != 0;
    if (capturable && !tracing && sw->graph && sw->graph_stream == st) {
      CRL_CHECK_CUDA(cudaGraphLaunch(sw->graph, st));
    } else if (capturable && !tracing && sw->calls > 0) {
      sw->drop_graph();
      cudaGraph_t g = nullptr;
      CRL_CHECK_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      try {
        sweep_body(sw, st);
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      CRL_CHECK_CUDA(cudaStreamEndCapture(st, &g));
      const cudaError_t e = cudaGraphInstantiate(&sw->graph, g, 0);
      cudaGraphDestroy(g);
      CRL_CHECK_CUDA(e);
      sw->graph_stream = st;
      CRL_CHECK_CUDA(cudaGraphLaunch(sw->graph, st));
    } else {
      sweep_body(sw, st);
    }
    sw->calls += 1;
    for (crl_ctx* c : sw->agents) c->update_calls += 1;
    deliver_floats(loss_out, sw->loss_all, 6 * na, st);
  });
}

int crl_sweep_sync_status(crl_sweep* sw, void* stream, uint32_t* status) {
  return sweep_guarded(sw, [&] {
    CRL_REQUIRE(sw && status, CRL_E_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned v = 0;
    CRL_CHECK_CUDA(cudaMemcpyAsync(&v, sw->status, sizeof(v), cudaMemcpyDeviceToHost, st));
    CRL_CHECK_CUDA(cudaStreamSynchronize(st));
    CRL_CHECK_CUDA(cudaMemsetAsync(sw->status, 0, sizeof(unsigned), st));
    uint32_t all = v;
    int worst = CRL_OK;
    for (crl_ctx* c : sw->agents) {
      uint32_t s = 0;
      const int r = crl_sync_status(c, stream, &s);
      all |= s;
      if (r != CRL_OK && worst == CRL_OK) worst = r;
    }
    *status = all;
    if (all & CRL_STATUS_NONFINITE) throw Failure(CRL_E_NONFINITE, "a loss was not finite");
    if (all & CRL_STATUS_TIMEOUT) throw Failure(CRL_E_TIMEOUT, "a bounded device wait gave up");
    if (worst != CRL_OK) throw Failure(worst, "agent status");
  });
}

int32_t crl_sweep_gemm_tuning_report(crl_sweep* sw, char* buf, size_t len, size_t* needed) {
  return sweep_guarded(sw, [&] {
    CRL_REQUIRE(sw && needed, CRL_E_INVALID_ARG, "null argument");
    const std::string js = gemm_tuning_json(sw->groups);
    *needed = js.size() + 1;
    CRL_REQUIRE(buf != nullptr || len == 0, CRL_E_INVALID_ARG, "null buffer with a nonzero length");
    if (len == 0) return;
    CRL_REQUIRE(len >= js.size() + 1, CRL_E_SHAPE, "the report needs " + std::to_string(js.size() + 1) + " bytes");
    memcpy(buf, js.c_str(), js.size() + 1);
  });
}

const char* crl_sweep_last_error(const crl_sweep* sw) { return sw ? sw->err.c_str() : crl_last_error(nullptr); }

}  // extern "C"
