// Internal interfaces between the translation units of libcrl (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/crl.h"

namespace crl {

// ---------------------------------------------------------------- replay buffer
// Row layout of the ring: [obs (D) | act (A) | ep_end (1, int32 bits) | pad] with
// W = roundup(D + A + 1, 4) floats, so every row starts on a 16-byte boundary.
// ep_end holds the absolute insertion index of the last step of the row's
// episode, or -1 while that episode is open.
struct BufferDev {
  float* rows;                      // [E][T][W]
  int32_t* ep_start;                // [E] absolute index of each env's open episode start
  int32_t* state;                   // [2] device copy of {size, total}
  const unsigned long long* gq;     // [T + 2] fixed-point discount table (see relabel)
  int E, T, D, A, W;
  int pad_;                         // explicit (zero): no implicit padding (descriptors key device tables)
};

// Optional BF16 packing of a network input by the relabel kernel: the split
// (hi, lo) interleaved row-major copy x0 [Mmax][ld] (see mlp_bf16.cuh).
// Source columns: kind 0 = concat(s, a), 1 = g, 2 = concat(s, g).
struct RelabelPack {
  void* x0;
  int ld;
};

struct RelabelArgs {
  uint64_t seed, agent;
  uint64_t step;                    // CRL_STEP_AUTO: read *step_dev
  unsigned long long* step_dev;     // device step counter
  unsigned long long* last_step_dev;  // receives the step used (read by the actor's Philox noise)
  int B, G, offset_min;
  int goal_idx[CRL_MAX_GOAL_DIMS];
  float *s, *a, *g;                 // [B][D], [B][A], [B][G]
  int32_t* idx;                     // [B][3] or null
  unsigned* status;                 // device status word
  RelabelPack pack[3];              // phi (s, a), psi (g), pi (s, g); x0 == null: not written
  int spw;                          // samples per warp (set by launch_relabel)
};

void launch_buffer_insert(const BufferDev& bd, const float* obs, const float* act, const uint8_t* done,
                          int n, int64_t total_before, cudaStream_t st);
void launch_relabel(const BufferDev& bd, const RelabelArgs& ra, cudaStream_t st);

// ---------------------------------------------------------------- multi-agent launches
constexpr int kMaxAgents = 64;
struct InsertArgs {
  BufferDev bd;
  const float* obs;
  const float* act;
  const uint8_t* done;
  int n, i0;                        // slices given, first slice written (n - T when n > T)
  long long total_before;
};
// Insert into several buffers in one launch: buffer s owns blocks [begin[s], begin[s+1]).
struct InsertMulti {
  InsertArgs a[kMaxAgents];
  int begin[kMaxAgents + 1];
  int n;
};
int insert_blocks(const BufferDev& bd);
void launch_buffer_insert_multi(const InsertMulti& m, cudaStream_t st);
struct RelabelTask {
  BufferDev bd;
  RelabelArgs ra;                   // ra.spw set (relabel_spw)
};
int relabel_spw(int B);
bool relabel_packs(const RelabelArgs& ra);
int relabel_blocks(const RelabelArgs& ra);
// tasks / begin: device tables (n tasks, n + 1 block offsets).  packs: every
// task writes the BF16 input packs (smem: the largest task's relabel_pack_smem).
void launch_relabel_multi(const RelabelTask* tasks, const int* begin, int n, int blocks, double bytes, bool packs,
                          size_t smem, cudaStream_t st);
void build_discount_table(float gamma, int n, unsigned long long* out);  // host

// ---------------------------------------------------------------- MLPs
struct MlpShape {
  int in0, in1, hidden, layers, out, layernorm;
  int in() const { return in0 + in1; }
};
struct LayerOffsets {
  int64_t W, b, g, beta;            // g/beta = -1 without LayerNorm
  int in, out;
};
// Layout of the flat parameter array; returns the element count (64-element aligned tensors).
int64_t mlp_layout(const MlpShape& s, LayerOffsets* lay /* layers + 1 entries */);
size_t mlp_saved_bytes(const MlpShape& s, int M, size_t elem);

template <typename T, typename TX1>
void mlp_forward(const MlpShape& s, const T* params, const float* x0, const TX1* x1, int M, T* y,
                 void* saved, cudaStream_t st);
// dparams / dx0 / dx1 may be null.
template <typename T, typename TX1>
void mlp_backward(const MlpShape& s, const T* params, const float* x0, const TX1* x1, int M,
                  const void* saved, const T* dy, T* dparams, T* dx0, T* dx1, cudaStream_t st);

// ---------------------------------------------------------------- energy + InfoNCE
struct LossSpec {
  int energy, loss, sym_reduction, penalty_axis;
  double tau, beta;
};
size_t infonce_ws_bytes(const LossSpec& ls, int B, int R, size_t elem, int path);
// loss4 = {total, fwd, bwd, penalty}.  t_bump: if non-null, ++*t_bump (Adam step counter).
template <typename T>
void infonce_forward(const LossSpec& ls, const T* phi, const T* psi, int B, int R, T* loss4, T* row_lse,
                     T* col_lse, void* ws, int path, unsigned* status, int* t_bump, cudaStream_t st);
template <typename T>
void infonce_backward(const LossSpec& ls, const T* phi, const T* psi, int B, int R, const T* row_lse,
                      const T* col_lse, double dtotal, T* dphi, T* dpsi, void* ws, int path,
                      cudaStream_t st);

// ---------------------------------------------------------------- op-level BF16 (ops_bf16.cu)
// One encoder on the tensor-core path: params FP32 (flat layout), x0 / x1 /
// y / dy / dparams / dx0 / dx1 FP32; `saved` (mlp_bf16_saved_bytes) holds the
// BF16 shadows and activations between a forward and its backward.  Failures throw.
size_t mlp_bf16_saved_bytes(const MlpShape& s, int M);
void mlp_bf16_forward(const MlpShape& s, const float* params, const float* x0, const float* x1, int M, float* y,
                      void* saved, cudaStream_t st);
void mlp_bf16_backward(const MlpShape& s, const float* params, int M, const void* saved, const float* dy,
                       float* dparams, float* dx0, float* dx1, cudaStream_t st);
// The fused energy stage on FP32 representations phi, psi [B][R]; ws
// (infonce_bf16_ws_bytes) carries the BF16 operands from a forward to its backward.
size_t infonce_bf16_ws_bytes(const LossSpec& ls, int B, int R);
void infonce_bf16_forward(const LossSpec& ls, const float* phi, const float* psi, int B, int R, float* loss4,
                          float* row_lse, float* col_lse, void* ws, cudaStream_t st);
void infonce_bf16_backward(const LossSpec& ls, const float* phi, const float* psi, int B, int R, const float* row_lse,
                           const float* col_lse, double dtotal, float* dphi, float* dpsi, void* ws, cudaStream_t st);

// ---------------------------------------------------------------- actor head
// Entropy-coefficient auto-tuning (the rule is a reading; the paper only says the
// coefficient is tuneable): state == null keeps the fixed alpha.  state[4] =
// {log alpha, Adam m, Adam v, alpha used by the last actor loss}, in FP64 for every
// precision.  After the actor loss of an applied step, log alpha takes one Adam step
// on  -log alpha * (mean log pi + target_entropy)  at the actor's step number.
struct AlphaTune {
  double* state;
  double target_entropy, lr, b1, b2, eps;
};
struct ActorSpec {
  int A, energy;
  double tau, alpha;
  AlphaTune tune;
};
// eps: explicit [B][A] (may be float for a T = double path) or null -> Philox noise.
// x0 != null: a' is also written, split into BF16 (hi, lo), into columns
// [x0_col, x0_col + A) of the BF16 network input x0 (row stride x0_ld).
template <typename T>
void actor_head_forward(const ActorSpec& as, const T* pi_out, const float* eps,
                        const unsigned long long* step_dev, uint64_t seed, uint64_t agent, int B,
                        T* a_new, T* logpi, T* eps_used, cudaStream_t st, __nv_bfloat16* x0 = nullptr,
                        int x0_ld = 0, int x0_col = 0, int noise_extra = 0);
template <typename T>
struct ActorLossArgs {
  int B, R, energy;
  double tau, alpha;
  const T* phi;
  const T* psi;
  const T* logpi;
  T* fdiag;
  T* dphi;
  __nv_bfloat16* dz;
  int ldz;
  T* partial;                 // [ceil(B / 8)][2]
  unsigned* ticket;           // zero between launches
  T* loss2;
  unsigned* status;
  int* t_bump;
  unsigned long long* step_bump;
  const unsigned long long* last_step;
  AlphaTune tune;             // tune.state != null: alpha = exp(state[0]), updated at the end
};
size_t actor_loss_ws_bytes(int B, size_t elem);
template <typename T>
struct HeadFwdArgs {
  int B, A;
  const T* out;                     // [B][2A] policy output (mu, log-std)
  const float* eps;                 // [B][A] or null (Philox noise at *step_dev)
  const unsigned long long* step_dev;
  unsigned long long seed, agent;
  T* a_new;
  T* logpi;
  T* eps_used;
  __nv_bfloat16* x0;                // optional split BF16 copy of a' (see actor_head_forward)
  int x0_ld, x0_col;
  int noise_extra;                  // Philox stream word 1 + noise_extra (0: the actor; 1: the collection stub)
};
template <typename T>
struct HeadBwdArgs {
  int B, A;
  double alpha;
  const T* out;
  const T* eps_used;
  const T* da;
  T* dout;
  __nv_bfloat16* dz;                // optional BF16 output gradient (see actor_head_backward)
  int ldz;
  const double* alpha_used;         // non-null: the alpha the actor loss used (overrides alpha)
};
// Diagonal energy, dphi (T, or BF16 into dz [B][ldz] when dz != null) and the
// actor loss in one launch.  ws: actor_loss_ws_bytes(B, sizeof(T)); ticket: a
// zero-initialised device word.  t_bump: ++*t_bump; step_bump: *step_bump =
// *last_step + 1 (both optional).  as.tune.state: alpha is read from it and, when
// t_bump is set, updated (see AlphaTune).
template <typename T>
void actor_energy_and_loss(const ActorSpec& as, const T* phi, const T* psi, const T* logpi, int B, int R,
                           T* dphi, T* fdiag, T* loss2, void* ws, unsigned* ticket, unsigned* status,
                           int* t_bump, unsigned long long* step_bump, const unsigned long long* last_step,
                           cudaStream_t st, __nv_bfloat16* dz = nullptr, int ldz = 0);
// dz != null: the output gradient is written as BF16 dz [B][ldz] instead of dout.
template <typename T>
void actor_head_backward(const ActorSpec& as, const T* pi_out, const T* eps_used, const T* da, int B,
                         T* dout, cudaStream_t st, __nv_bfloat16* dz = nullptr, int ldz = 0);

class BlobCache;
// Several agents in one launch each (float tasks of the BF16 path; tables cached in `cache`).
const char* actor_loss_multi(BlobCache& cache, const std::vector<ActorLossArgs<float>>& tasks, cudaStream_t st);
const char* actor_head_backward_multi(BlobCache& cache, const std::vector<HeadBwdArgs<float>>& tasks,
                                      cudaStream_t st);

// ---------------------------------------------------------------- Adam
template <typename T>
void adam_update(T* p, const T* g, T* m, T* v, int64_t n, const int* t_dev, int t_host, float lr,
                 float b1, float b2, float eps, cudaStream_t st);

// Small device utilities.
void launch_bump_u64(unsigned long long* ctr, cudaStream_t st);
// Random-goal actor mix (App. D): g_act[b] = g[(b + 1) mod B] when (word 2 of the
// Philox block (*step_dev, b, 0, 0) keyed (seed, agent)) >> 32 < floor(alpha_rg 2^32),
// else g[b].  step_dev: the step the relabel of g used.
void launch_actor_goals(int B, int G, const float* g, float* g_act, uint64_t seed, uint64_t agent,
                        const unsigned long long* step_dev, float alpha_rg, cudaStream_t st);

// Sets the message crl_last_error(NULL) returns on the calling thread.
void set_thread_error(const std::string& msg);

}  // namespace crl
