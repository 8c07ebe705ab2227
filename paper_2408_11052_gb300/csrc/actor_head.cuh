// The actor head's forward (Eq. 3, §3.2, §5.1; readings as in actor.cu): a
// device body shared by the head's own kernels and by the Adam launch that
// runs it alongside the critic's update (the head reads only the policy's
// output, never the critic's weights).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "philox.cuh"

namespace crl {

constexpr double kLogStdMin = -5.0;
constexpr double kLogStdMax = 2.0;
constexpr double kLog2 = 0.69314718055994530942;
constexpr double kHalfLog2Pi = 0.91893853320467274178;

// One warp per row b, lanes over the action dims.
// x0 != null: a' also goes into columns [x0_col, x0_col + A) of the split BF16
// network input x0 (hi, lo interleaved: element c at 2c, 2c + 1).
template <typename T>
__device__ __forceinline__ void head_forward_body(const HeadFwdArgs<T>& p, int lb) {
  const int B = p.B, A = p.A;
  const T* __restrict__ out = p.out;
  const float* __restrict__ eps = p.eps;
  T* __restrict__ a_new = p.a_new;
  T* __restrict__ eps_used = p.eps_used;
  __nv_bfloat16* __restrict__ x0 = p.x0;
  const int x0_ld = p.x0_ld, x0_col = p.x0_col;
  const unsigned long long seed = p.seed, agent = p.agent;
  const int lane = threadIdx.x % kWarp;
  const int b = lb * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (b >= B) return;
  const unsigned long long step = eps ? 0ull : *p.step_dev;
  T lp = 0;
  for (int d = lane; d < A; d += kWarp) {
    const T mu = out[(size_t)b * 2 * A + d];
    const T lraw = out[(size_t)b * 2 * A + A + d];
    const T l = fmin(fmax(lraw, T(kLogStdMin)), T(kLogStdMax));
    const T e = eps ? T(eps[(size_t)b * A + d]) : philox_normal<T>(step, b, 1ull + p.noise_extra, d, seed, agent);
    const T u = mu + dev_exp(l) * e;
    const T act = dev_tanh(u);
    a_new[(size_t)b * A + d] = act;
    if (x0) {
      const float v = (float)act;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      __nv_bfloat16* dst = x0 + (size_t)b * x0_ld + 2 * (x0_col + d);
      dst[0] = hi;
      dst[1] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    eps_used[(size_t)b * A + d] = e;
    lp += -T(0.5) * e * e - T(kHalfLog2Pi) - l - T(2) * (T(kLog2) - u - softplus(T(-2) * u));
  }
  lp = warp_sum(lp);
  if (lane == 0) p.logpi[b] = lp;
}

}  // namespace crl
