// Fused tcgen05 energy + InfoNCE + logsumexp penalty (see energy_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "internal.h"
#include "tables.h"

namespace crl {

// BF16 operands and per-row auxiliaries of the fused energy stage for batches up to Bmax.
struct EnergyTc {
  int R = 0, Bmax = 0, ldt = 0;
  __nv_bfloat16 *X = nullptr, *Y = nullptr;   // [Bmax][R]
  __nv_bfloat16 *XT = nullptr, *YT = nullptr; // optional transposed copies [R][ldt] (null: not written)
  float *auxX = nullptr, *auxY = nullptr;     // [Bmax]
  CUtensorMap tmX, tmY;
  int tm_B = -1;
};

bool energy_tc_supported(const LossSpec& ls, int B, int R, const char** why);
// Bytes of the workspace of energy_tc_forward / energy_tc_backward.
size_t energy_tc_ws_bytes(const LossSpec& ls, int B, int R);
const char* energy_tc_maps(EnergyTc& e, int B);
// phi, psi [B][R] FP32 -> BF16 operands and auxiliaries (nothing for -L1,
// whose tiles read phi and psi).
void energy_tc_prepare(EnergyTc& e, const LossSpec& ls, const float* phi, const float* psi, int B, cudaStream_t st);
// loss4 = {total, fwd, bwd, penalty}; r, c = row / column logsumexp.  ws:
// energy_tc_ws_bytes(ls, B, R).  phi, psi: the FP32 representations (read by
// the -L1 energy; the others read the BF16 operands).
void energy_tc_forward(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi, float* loss4,
                       float* r, float* c, void* ws, unsigned* status, int* t_bump, cudaStream_t st);
// dphi / dpsi as BF16 [B][R] (the encoders' dy layout), scaled by dtotal.
// ws: the forward's workspace (its anchors and diagonal coefficients for DPO / IPO).
void energy_tc_backward(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi, const float* r,
                        const float* c, double dtotal, __nv_bfloat16* dphi, __nv_bfloat16* dpsi, void* ws,
                        unsigned* status, cudaStream_t st);

// The same backward with dphi / dpsi as FP32 [B][R] (the op-level entry points).
void energy_tc_backward_f32(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi,
                            const float* r, const float* c, double dtotal, float* dphi, float* dpsi, void* ws,
                            unsigned* status, cudaStream_t st);
// Bytes at the start of the forward's workspace holding its tickets, which must
// be zero when a forward starts (the CTAs that use them reset them).
size_t energy_tc_ticket_bytes(int B);

// One agent of a multi-agent launch of the fused energy stage (its maps built
// by energy_tc_maps for batch B).
struct EnergyAgent {
  EnergyTc* e;
  LossSpec ls;
  int B;
  const float* phi;   // [B][R] FP32 encoder outputs
  const float* psi;
  float* loss4;
  float* r;
  float* c;
  void* ws;           // energy_tc_ws_bytes(ls, B, R), zeroed at creation
  int* t_bump;
  __nv_bfloat16* dphi;
  __nv_bfloat16* dpsi;
  unsigned* status;
};
// stage 0: prepare, 1: forward (+ loss), 2: backward -- one launch over all agents.
const char* energy_tc_multi(BlobCache& cache, const std::vector<EnergyAgent>& agents, int stage, cudaStream_t st);

}  // namespace crl
