// Argument blocks and per-pair arithmetic shared by the fused energy kernels:
// energy_tc.cu (the tcgen05 energies) and energy_l1.cu (the SIMT -L1 energy).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace crl {

using bf16 = __nv_bfloat16;

// Named (not anonymous): energy_tc.cu and energy_l1.cu pass these blocks to
// each other's host launchers.
namespace fe {

constexpr int kTile = 128;

struct Weights {
  float wf, wb, pr, pc;
};

// Weights of the InfoNCE directions (FlatNCE takes InfoNCE's gradient; the
// other objectives none) and of the penalty axes.
inline Weights loss_weights(const LossSpec& ls) {
  Weights w{0, 0, 0, 0};
  if (ls.loss == CRL_LOSS_FWD || ls.loss == CRL_LOSS_FLATNCE_FWD) w.wf = 1;
  else if (ls.loss == CRL_LOSS_BWD || ls.loss == CRL_LOSS_FLATNCE_BWD) w.wb = 1;
  else if (ls.loss == CRL_LOSS_SYM) w.wf = w.wb = (ls.sym_reduction == CRL_SYM_SUM) ? 1.f : 0.5f;
  if (ls.penalty_axis == CRL_PENALTY_ROW) w.pr = 1;
  else if (ls.penalty_axis == CRL_PENALTY_COL) w.pc = 1;
  else w.pr = w.pc = 0.5f;
  return w;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Two-lane FP32 arithmetic (one instruction for both lanes; each lane rounds
// exactly as the scalar operation does).
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 mul_x2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 add_x2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

struct FwdArgs {
  int B, R, energy, obj;  // obj: the loss code
  int n, C, nC;           // tiles per side; column tiles per chunk (at most 64) and chunks per row tile
  float inv_tau;
  const float* auxX;
  const float* auxY;
  const bf16* X;   // [B][R] operand rows (the DPO / IPO anchor F_ii)
  const bf16* Y;
  float* objpart;  // [nC][B][2] per-row objective partials over each column chunk
  float* dpre;     // [B] the anchor F_ii of DPO / IPO (written by the J = 0 tiles)
  float* kd;       // [B] k_i of DPO / IPO (written by the row merges)
  float* rowpart;  // [nC][B][2] per-row (max, sum) over each column chunk
  float* colpart;  // [nI][B][2]
  float* diag;     // [B]
  const float* phi;  // [B][R] FP32 representations (the -L1 energy reads these, not X / Y)
  const float* psi;
  unsigned* status;
  // finalize (run by the last CTA to finish)
  Weights w;
  float beta;
  float* r_out;
  float* c_out;
  float* loss4;
  int* t_bump;
  unsigned* tickets;  // [2 n + 1]: per row tile (chunks), per column tile (row tiles), final (zero between launches)
  float* tile_part;   // [2][n][3]: per row / column tile (sum of (lse - diag), sum of lse^2, objective value)
};

__device__ __forceinline__ float sigmoidf_fast(float x) { return __frcp_rn(1.f + __expf(-x)); }
__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.f) + log1pf(__expf(-fabsf(x))); }

struct BwdArgs {
  int B, R, energy, transposed;  // transposed: own = psi (the column pass)
  int obj;                       // the loss code
  float inv_tau, beta, scale;    // scale = dtotal / B
  float dtotal;
  const float* dpre;             // [B] anchor F_ii of DPO / IPO (from the forward)
  const float* kd;               // [B] k_i of DPO / IPO (from the forward)
  Weights w;
  const float* aux_own;
  const float* aux_other;
  const float* lse_own;    // r (row pass) or c (column pass)
  const float* lse_other;  // c (row pass) or r (column pass)
  const float* own_f32;    // [B][R] FP32 representation (cos: unnormalised)
  bf16* d_out;             // [B][R]
  unsigned* status;
  float* d_out_f32;        // non-null: the gradient as FP32 [B][R] here instead of d_out
  const float* other_f32;  // [B][R] FP32 representation of the other side (the -L1 energy)
};

struct HCoef {
  float a_own;    // own auxiliary (|x|^2 for the L2 energies)
  float l_own2;   // own logsumexp x log2(e)
  float k_own;    // scale (w_own + 2 beta p_own l_own)
  float k_own_tau;  // k_own / tau
  float k_diag;   // scale (w_f + w_b): the positive pair's -1 terms
  float inv_tau;
  float k1;       // log2(e) / tau
  // objectives outside InfoNCE (OBJ > 0)
  float d_own, kd_own;  // row pass: this row's anchor F_uu and k_u
  const float* dpre;    // column pass: the rows' anchors and k (read per pair)
  const float* kd;
  float c_bb, c_b, c_fb;  // dtotal / B^2, dtotal / B, dtotal / (B (B - 1))
  float dtotal;
  int transposed;
};

// Objective kinds of the coefficient tile: 0 the InfoNCE family (FlatNCE
// included), then forward-backward, DPO, IPO, SPPO, NCE-binary.
enum : int { kObjInfo = 0, kObjFB, kObjDPO, kObjIPO, kObjSPPO, kObjNCE };
inline int obj_kind(int loss) {
  switch (loss) {
    case CRL_LOSS_FB: return kObjFB;
    case CRL_LOSS_DPO: return kObjDPO;
    case CRL_LOSS_IPO: return kObjIPO;
    case CRL_LOSS_SPPO: return kObjSPPO;
    case CRL_LOSS_NCE_BINARY: return kObjNCE;
    default: return kObjInfo;
  }
}

// dtotal x (the objective's dL/dF_ij) for F = f2 / log2(e); the row of the pair
// is u in the row pass and v in the column pass (d_row, k_row: its anchor F_ii
// and k_i, the latter already divided by B^2).
template <int OBJ>
__device__ __forceinline__ float objective_coef(float f2, bool diag, float d_row, float k_row, const HCoef& hc) {
  if (OBJ == kObjFB) return diag ? -ex2(f2) * hc.c_b : ex2(2.f * f2) * hc.c_fb;
  const float F = f2 * (1.f / kLog2e);
  float o;
  if (OBJ == kObjDPO) {
    o = __frcp_rn(1.f + ex2((d_row - F) * kLog2e)) * hc.c_bb;  // sigma(F - d)
  } else if (OBJ == kObjIPO) {
    o = -2.f * (d_row - F - 1.f) * hc.c_bb;
  } else if (OBJ == kObjSPPO) {
    o = 2.f * (F + 1.f) * hc.c_bb + (diag ? 2.f * (F - 1.f) * hc.c_b : 0.f);
  } else {  // NCE-binary: sigma(F) - [i = j]
    o = (__frcp_rn(1.f + ex2(-f2)) - (diag ? 1.f : 0.f)) * hc.c_bb;
  }
  if ((OBJ == kObjDPO || OBJ == kObjIPO) && diag) o -= k_row * hc.dtotal;
  return o;
}

// ---- the -L1 energy (energy_l1.cu): SIMT tiles over the FP32 representations
// Forward tiles of one (row tile, column tile) each: the same partials as the
// tcgen05 forward with one column tile per chunk (a.C = 1, a.nC = a.n), merged
// by the same finalize.
void l1_forward(const FwdArgs& a, cudaStream_t st);
// Backward row and column passes.  part: l1_part_floats(B, R) floats of
// scratch for the per-segment partial gradients (added in segment order).
void l1_backward(const BwdArgs& row, const BwdArgs& col, float* part, cudaStream_t st);
size_t l1_part_floats(int B, int R);

}  // namespace fe
}  // namespace crl
