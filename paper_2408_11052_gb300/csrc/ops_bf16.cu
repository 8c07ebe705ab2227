// Op-level BF16 entry points behind torch.autograd.Function: one encoder MLP on
// the tcgen05 grouped GEMMs, and the fused energy + InfoNCE + logsumexp penalty
// stage (BF16 operands on the tensor cores, FP32 logsumexps, penalty and loss
// reduction; the B x B logits never reach memory).  The arithmetic is the
// update step's (the same kernels and the same BF16 split input, weight pair and
// operand rounding); only the buffers differ: everything the backward needs
// lives in the caller's workspace, so every forward / backward pair is
// independent of every other.
//
// arXiv 2408.11052: §3.1 (encoders phi, psi; critic objective), App. A.2
// (energies, InfoNCE directions), Algorithm 1 (beta * logsumexp penalty).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctx.h"
#include "energy_tc.cuh"
#include "internal.h"
#include "mlp_bf16.cuh"

namespace crl {
namespace {

constexpr size_t kStatusBytes = 256;  // the device status word of op-level calls, first in the workspace

// Pieces of a caller workspace, 256-byte aligned, in a fixed order.
struct Carver {
  char* base;
  size_t off;
};
void* carve_piece(void* owner, size_t bytes) {
  Carver* c = static_cast<Carver*>(owner);
  const size_t o = (c->off + 255) / 256 * 256;
  c->off = o + bytes;
  return c->base + o;
}

// Grouped-GEMM problem tables of the op-level calls.  Their problems point at
// caller buffers, so the fixed tile rule is used (no timing per new address)
// and the tables are dropped once they pile up.
std::mutex g_ops_mutex;
GemmGroups& ops_groups() {
  static GemmGroups* g = [] {
    GemmGroups* p = new GemmGroups();
    p->allow_tune = false;
    return p;
  }();
  if (g->entries() > 512) g->reset();
  return *g;
}

// The network's BF16 buffers laid out in `saved` (after the status word) for M rows.
const char* carve_net(BfNet& n, const MlpShape& s, int M, void* saved) {
  Carver c{static_cast<char*>(saved) + kStatusBytes, 0};
  if (const char* e = bf_net_carve(n, s, M, carve_piece, &c, true)) return e;
  return bf_net_maps(n, M);
}

}  // namespace

size_t mlp_bf16_saved_bytes(const MlpShape& s, int M) {
  const size_t net = bf_net_bytes(s, M);
  return net == 0 ? 0 : kStatusBytes + net;
}

void mlp_bf16_forward(const MlpShape& s, const float* params, const float* x0, const float* x1, int M, float* y,
                      void* saved, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_ops_mutex);
  BfNet n;
  if (const char* e = carve_net(n, s, M, saved)) throw Failure(CRL_E_INVALID_ARG, e);
  // a fresh workspace: zero it (padding columns of the weight shadows are read
  // as K by the tensor cores; the LayerNorm ticket starts at zero), then the
  // ones rows, the weight shadows and the split input
  CRL_CHECK_CUDA(cudaMemsetAsync(saved, 0, mlp_bf16_saved_bytes(s, M), st));
  bf_net_fill_ones(n, st);
  bf_net_shadow(n, params, st);
  bf_net_pack_input(n, x0, x1, M, st);
  n.y = y;
  BfPass p{&n, params, nullptr, nullptr, M};
  if (const char* e = bf_forward(ops_groups(), &p, 1, static_cast<unsigned*>(saved), st))
    throw Failure(CRL_E_CUDA, e);
}

void mlp_bf16_backward(const MlpShape& s, const float* params, int M, const void* saved, const float* dy,
                       float* dparams, float* dx0, float* dx1, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_ops_mutex);
  BfNet n;
  void* sv = const_cast<void*>(saved);   // the backward writes its dz buffers there
  if (const char* e = carve_net(n, s, M, sv)) throw Failure(CRL_E_INVALID_ARG, e);
  bf_net_load_dy(n, dy, M, st);
  BfPass p{&n, params, dparams, dx1, M};
  p.dx0 = dx0;
  if (const char* e = bf_backward(ops_groups(), &p, 1, static_cast<unsigned*>(sv), st))
    throw Failure(CRL_E_CUDA, e);
}

namespace {

// The fused energy stage's operands in a caller workspace: the energy
// workspace (tickets first), then X, Y [B][R] BF16 and auxX, auxY [B].
struct EnergyWs {
  EnergyTc e;
  void* ews;
  unsigned* status;
};
const char* carve_energy(EnergyWs& w, const LossSpec& ls, int B, int R, void* ws) {
  char* base = static_cast<char*>(ws);
  w.status = reinterpret_cast<unsigned*>(base);
  Carver c{base + kStatusBytes, 0};
  w.ews = carve_piece(&c, energy_tc_ws_bytes(ls, B, R));
  w.e.R = R;
  w.e.Bmax = B;
  w.e.ldt = 0;
  w.e.X = static_cast<__nv_bfloat16*>(carve_piece(&c, (size_t)B * R * 2));
  w.e.Y = static_cast<__nv_bfloat16*>(carve_piece(&c, (size_t)B * R * 2));
  w.e.XT = w.e.YT = nullptr;
  w.e.auxX = static_cast<float*>(carve_piece(&c, (size_t)B * 4));
  w.e.auxY = static_cast<float*>(carve_piece(&c, (size_t)B * 4));
  w.e.tm_B = -1;
  return energy_tc_maps(w.e, B);
}

// The -L1 tiles move rows in 16-byte pieces.
void check_l1_alignment(const LossSpec& ls, const void* a, const void* b, const void* c, const void* d) {
  if (ls.energy != CRL_ENERGY_L1) return;
  const uintptr_t bits = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                         reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d);
  if (bits % 16 != 0) throw Failure(CRL_E_INVALID_ARG, "the fused -L1 energy needs 16-byte aligned rows");
}

}  // namespace

size_t infonce_bf16_ws_bytes(const LossSpec& ls, int B, int R) {
  Carver c{nullptr, 0};
  carve_piece(&c, energy_tc_ws_bytes(ls, B, R));
  carve_piece(&c, (size_t)B * R * 2);
  carve_piece(&c, (size_t)B * R * 2);
  carve_piece(&c, (size_t)B * 4);
  carve_piece(&c, (size_t)B * 4);
  return kStatusBytes + (c.off + 255) / 256 * 256;
}

void infonce_bf16_forward(const LossSpec& ls, const float* phi, const float* psi, int B, int R, float* loss4,
                          float* row_lse, float* col_lse, void* ws, cudaStream_t st) {
  const char* why = nullptr;
  if (!energy_tc_supported(ls, B, R, &why)) throw Failure(CRL_E_UNSUPPORTED, why);
  check_l1_alignment(ls, phi, psi, nullptr, nullptr);
  EnergyWs w;
  if (const char* e = carve_energy(w, ls, B, R, ws)) throw Failure(CRL_E_INVALID_ARG, e);
  // status word and tickets start at zero
  CRL_CHECK_CUDA(cudaMemsetAsync(ws, 0, kStatusBytes, st));
  CRL_CHECK_CUDA(cudaMemsetAsync(w.ews, 0, energy_tc_ticket_bytes(B), st));
  energy_tc_prepare(w.e, ls, phi, psi, B, st);
  energy_tc_forward(w.e, ls, B, phi, psi, loss4, row_lse, col_lse, w.ews, w.status, nullptr, st);
}

void infonce_bf16_backward(const LossSpec& ls, const float* phi, const float* psi, int B, int R, const float* row_lse,
                           const float* col_lse, double dtotal, float* dphi, float* dpsi, void* ws, cudaStream_t st) {
  const char* why = nullptr;
  if (!energy_tc_supported(ls, B, R, &why)) throw Failure(CRL_E_UNSUPPORTED, why);
  check_l1_alignment(ls, phi, psi, dphi, dpsi);
  EnergyWs w;
  if (const char* e = carve_energy(w, ls, B, R, ws)) throw Failure(CRL_E_INVALID_ARG, e);
  energy_tc_backward_f32(w.e, ls, B, phi, psi, row_lse, col_lse, dtotal, dphi, dpsi, w.ews, w.status, st);
}

}  // namespace crl
