// Logit statistics of the critic's energy matrix, a library diagnostic that is
// off by default (crl_set_logit_stats): the mean positive-pair logit
// (1 / B) sum_i F_ii and the mean negative logit (1 / (B^2 - B)) sum_{i != j} F_ij
// of every critic step, from the representations its energy was formed from
// (the encoders' FP32 outputs; FP64 on the check path).  F as in the critic
// objective (§3.1, App. A.2, temperature tau): L2 -|x - y| / tau, L2^2
// -|x - y|^2 / tau, dot <x, y> / tau, cos <x, y> / (|x| |y| tau), -L1
// -|x - y|_1 / tau.
//
// One block per 32 x 32 tile of pairs (256 threads, four pairs each), both
// operand tiles staged through shared memory 64 columns at a time; each block
// leaves its two FP64 sums in a partial slot and one block adds the slots in
// order, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"

namespace crl {
namespace {

constexpr int kT = 32;   // pairs per tile side
constexpr int kC = 64;   // representation columns per stage

template <typename T>
__global__ void __launch_bounds__(256) logit_stats_tiles(const T* __restrict__ phi, const T* __restrict__ psi, int B,
                                                         int R, int energy, double inv_tau, double* __restrict__ part) {
  pdl_enter();
  __shared__ T xs[kT][kC + 1];
  __shared__ T ys[kT][kC + 1];
  const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
  const int tx = threadIdx.x % kT, ty = threadIdx.x / kT;   // pair (i0 + ty + 8 q, j0 + tx), q = 0..3
  T acc[4] = {0, 0, 0, 0}, nx[4] = {0, 0, 0, 0}, ny[4] = {0, 0, 0, 0};
  for (int c0 = 0; c0 < R; c0 += kC) {
    for (int e = threadIdx.x; e < kT * kC; e += blockDim.x) {
      const int r = e / kC, c = e % kC;
      xs[r][c] = (i0 + r < B && c0 + c < R) ? phi[(size_t)(i0 + r) * R + c0 + c] : T(0);
      ys[r][c] = (j0 + r < B && c0 + c < R) ? psi[(size_t)(j0 + r) * R + c0 + c] : T(0);
    }
    __syncthreads();
    const int cn = min(kC, R - c0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      for (int c = 0; c < cn; ++c) {
        const T x = xs[r][c], y = ys[tx][c];
        if (energy == CRL_ENERGY_L2 || energy == CRL_ENERGY_L2SQ) acc[q] += (x - y) * (x - y);
        else if (energy == CRL_ENERGY_L1) acc[q] += fabs(x - y);
        else acc[q] += x * y;
        if (energy == CRL_ENERGY_COS) {
          nx[q] += x * x;
          ny[q] += y * y;
        }
      }
    }
    __syncthreads();
  }
  double sd = 0.0, so = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i >= B || j >= B) continue;
    double f;
    switch (energy) {
      case CRL_ENERGY_L2: f = -sqrt((double)acc[q]); break;
      case CRL_ENERGY_L2SQ: f = -(double)acc[q]; break;
      case CRL_ENERGY_L1: f = -(double)acc[q]; break;
      case CRL_ENERGY_COS: f = (double)acc[q] / sqrt((double)nx[q] * (double)ny[q]); break;
      default: f = (double)acc[q]; break;
    }
    f *= inv_tau;
    if (i == j) sd += f;
    else so += f;
  }
  // fixed-order block reduction: warp trees, then the eight warps in order
  sd = warp_sum(sd);
  so = warp_sum(so);
  __shared__ double ws[2][8];
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  if (lane == 0) {
    ws[0][warp] = sd;
    ws[1][warp] = so;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += ws[0][w];
      b += ws[1][w];
    }
    double* p = part + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    p[0] = a;
    p[1] = b;
  }
}

__global__ void __launch_bounds__(256) logit_stats_finish(const double* __restrict__ part, int nparts, int B,
                                                          float* __restrict__ out) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  double d = 0.0, o = 0.0;
  for (int k = 0; k < nparts; ++k) {
    d += part[2 * k];
    o += part[2 * k + 1];
  }
  out[0] = (float)(d / B);
  out[1] = B > 1 ? (float)(o / ((double)B * (B - 1))) : __int_as_float(0x7fc00000);   // NaN: no negatives
}

}  // namespace

void logit_stats_alloc(crl_ctx* c) {
  if (c->stats) return;
  const int nt = ceil_div(c->cfg.B, kT);
  c->stats = static_cast<float*>(c->dalloc(2 * sizeof(float)));
  c->stats_part = static_cast<double*>(c->dalloc((size_t)nt * nt * 2 * sizeof(double)));
  const float nan2[2] = {NAN, NAN};
  CRL_CHECK_CUDA(cudaMemcpy(c->stats, nan2, sizeof(nan2), cudaMemcpyHostToDevice));
}

void logit_stats_launch(crl_ctx* c, const void* phi, const void* psi, int B, bool fp64, cudaStream_t st) {
  if (!c->stats_on) return;
  const int nt = ceil_div(B, kT);
  const crl_config& cf = c->cfg;
  const double inv_tau = 1.0 / (double)cf.temperature;
  TraceLaunch tr(CRL_TRACE_AUX, st, 2.0 * B * B * cf.repr);
  if (fp64)
    launch_k(logit_stats_tiles<double>, dim3(nt, nt), dim3(256), 0, st, static_cast<const double*>(phi),
             static_cast<const double*>(psi), B, cf.repr, cf.energy, inv_tau, c->stats_part);
  else
    launch_k(logit_stats_tiles<float>, dim3(nt, nt), dim3(256), 0, st, static_cast<const float*>(phi),
             static_cast<const float*>(psi), B, cf.repr, cf.energy, inv_tau, c->stats_part);
  launch_k(logit_stats_finish, dim3(1), dim3(32), 0, st, static_cast<const double*>(c->stats_part), nt * nt, B,
           c->stats);
}

}  // namespace crl

extern "C" {

int crl_set_logit_stats(crl_ctx* ctx, int32_t on) {
  using namespace crl;
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx, CRL_E_INVALID_ARG, "null context");
    if (on) logit_stats_alloc(ctx);
    if ((on != 0) != ctx->stats_on) {
      // the captured update step changes (a sweep holding this agent rebuilds its own)
      ctx->drop_graph();
      ++ctx->bind_generation;
    }
    ctx->stats_on = on != 0;
  });
}

int crl_get_logit_stats(crl_ctx* ctx, float* out) {
  using namespace crl;
  return guarded(ctx, [&] {
    CRL_REQUIRE(ctx && out, CRL_E_INVALID_ARG, "null argument");
    if (!ctx->stats) {
      out[0] = out[1] = NAN;
      return;
    }
    CRL_CHECK_CUDA(cudaDeviceSynchronize());
    CRL_CHECK_CUDA(cudaMemcpy(out, ctx->stats, 2 * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

}  // extern "C"
