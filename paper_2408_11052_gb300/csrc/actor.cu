// Actor head of the CRL update step: tanh-squashed Gaussian policy, the
// DDPG-style objective with an entropy term, and its backward.
//
// arXiv 2408.11052: Eq. 3 (§3.2) -- the policy maximises f(s, a', g) with
// a' ~ pi(. | s, g), goals from the same trajectory (App. C, random-goal
// weight 0); §5.1 -- "a tuneable entropy coefficient".
// Readings: (mu, l) = pi(concat(s, g)), l clipped to [-5, 2], sigma = e^l,
// u = mu + sigma eps, a' = tanh(u),
//   log pi = sum_d [-eps^2/2 - log(2 pi)/2 - l - 2 (log 2 - u - softplus(-2u))],
//   L = mean_i [alpha log pi_i - f(phi(s_i, a'_i), psi(g_i)) / tau].
// Gradients: d log pi / du = 2 tanh(u); d log pi / dl = -1 (plus the u path,
// du/dl = sigma eps); the clip passes gradient only strictly inside (-5, 2).
#include "common.cuh"
#include "internal.h"
#include "philox.cuh"
#include "trace.h"

namespace crl {

constexpr double kLogStdMin = -5.0;
constexpr double kLogStdMax = 2.0;
constexpr double kLog2 = 0.69314718055994530942;
constexpr double kHalfLog2Pi = 0.91893853320467274178;
constexpr double kTwoPi = 6.28318530717958647693;

namespace {

// N(0, 1) noise for element d of row b: Box-Muller on Philox4x64-10 block
// (step, b, 1, d / 4); words (0, 1) feed elements 4q, 4q+1 and words (2, 3)
// feed 4q+2, 4q+3 (cos / sin branch).
// The FP64 path draws the noise in double; the FP32 path in float (same
// Philox words, so the two agree to float rounding).
template <typename T>
__device__ T philox_normal(unsigned long long step, int b, int d, unsigned long long seed, unsigned long long agent) {
  const Philox4 r = philox4x64_10(step, (unsigned long long)b, 1ull, (unsigned long long)(d / 4), seed, agent);
  const int pair = (d % 4) / 2;
  const double u1 = u64_to_unit_open(r.w[2 * pair]);
  const double u2 = u64_to_unit_open(r.w[2 * pair + 1]);
  if constexpr (sizeof(T) == 8) {
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(kTwoPi * u2, &s, &c);
    return (d % 2 == 0) ? rad * c : rad * s;
  } else {
    const float rad = sqrtf(-2.0f * logf((float)u1));
    float s, c;
    sincosf((float)(kTwoPi * u2), &s, &c);
    return (d % 2 == 0) ? rad * c : rad * s;
  }
}

// One warp per row b, lanes over the action dims.
template <typename T>
__global__ void __launch_bounds__(256) head_forward_kernel(int B, int A, const T* __restrict__ out,
                                                          const float* __restrict__ eps,
                                                          const unsigned long long* __restrict__ step_dev,
                                                          unsigned long long seed, unsigned long long agent,
                                                          T* __restrict__ a_new, T* __restrict__ logpi,
                                                          T* __restrict__ eps_used) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int b = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (b >= B) return;
  const unsigned long long step = eps ? 0ull : *step_dev;
  T lp = 0;
  for (int d = lane; d < A; d += kWarp) {
    const T mu = out[(size_t)b * 2 * A + d];
    const T lraw = out[(size_t)b * 2 * A + A + d];
    const T l = fmin(fmax(lraw, T(kLogStdMin)), T(kLogStdMax));
    const T e = eps ? T(eps[(size_t)b * A + d]) : philox_normal<T>(step, b, d, seed, agent);
    const T u = mu + dev_exp(l) * e;
    a_new[(size_t)b * A + d] = dev_tanh(u);
    eps_used[(size_t)b * A + d] = e;
    lp += -T(0.5) * e * e - T(kHalfLog2Pi) - l - T(2) * (T(kLog2) - u - softplus(T(-2) * u));
  }
  lp = warp_sum(lp);
  if (lane == 0) logpi[b] = lp;
}

// f_i = f(phi_i, psi_i) / tau and dphi_i = -(1/B) df_i/dphi_i.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) diag_energy_kernel(int B, int R, int energy, double tau,
                                                         const T* __restrict__ phi, const T* __restrict__ psi,
                                                         T* __restrict__ fdiag, T* __restrict__ dphi) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int i = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (i >= B) return;
  const T* x = phi + (size_t)i * R;
  const T* y = psi + (size_t)i * R;
  T sxy = 0, sxx = 0, syy = 0, sdd = 0, sad = 0;
  for (int c = lane; c < R; c += kWarp) {
    const T a = x[c], b = y[c], d = a - b;
    sxy += a * b;
    sxx += a * a;
    syy += b * b;
    sdd += d * d;
    sad += fabs(d);
  }
  sxy = warp_sum(sxy);
  sxx = warp_sum(sxx);
  syy = warp_sum(syy);
  sdd = warp_sum(sdd);
  sad = warp_sum(sad);
  const T it = T(1.0 / tau), ib = T(-1.0 / B);
  T f;
  switch (energy) {
    case CRL_ENERGY_DOT: f = sxy; break;
    case CRL_ENERGY_COS: f = sxy / (dev_sqrt(sxx) * dev_sqrt(syy)); break;
    case CRL_ENERGY_L2: f = -dev_sqrt(sdd); break;
    case CRL_ENERGY_L2SQ: f = -sdd; break;
    default: f = -sad; break;
  }
  if (lane == 0) fdiag[i] = f * it;
  const T nx = dev_sqrt(sxx), ny = dev_sqrt(syy), dist = dev_sqrt(sdd);
  for (int c = lane; c < R; c += kWarp) {
    const T a = x[c], b = y[c], d = a - b;
    T g;
    switch (energy) {
      case CRL_ENERGY_DOT: g = b; break;
      case CRL_ENERGY_COS: {
        const T xh = a / nx, yh = b / ny;
        g = (yh - xh * (sxy / (nx * ny))) / nx;
        break;
      }
      case CRL_ENERGY_L2: g = (dist >= T(1e-12)) ? -d / dist : T(0); break;
      case CRL_ENERGY_L2SQ: g = T(-2) * d; break;
      default: g = (d > T(0)) ? T(-1) : ((d < T(0)) ? T(1) : T(0)); break;
    }
    dphi[(size_t)i * R + c] = ib * it * g;
  }
}

// loss2 = {mean(alpha log pi - f), mean log pi}.  One block.
template <typename T>
__global__ void __launch_bounds__(1024) actor_loss_kernel(int B, double alpha, const T* __restrict__ logpi,
                                                         const T* __restrict__ fdiag, T* __restrict__ loss2,
                                                         unsigned* status, int* t_bump) {
  pdl_enter();
  __shared__ T sm[32];
  T a = 0, l = 0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    a += T(alpha) * logpi[i] - fdiag[i];
    l += logpi[i];
  }
  a = block_sum(a, sm);
  l = block_sum(l, sm);
  if (threadIdx.x == 0) {
    loss2[0] = a / T(B);
    loss2[1] = l / T(B);
    if (status && !finite_val(a)) atomicOr(status, CRL_STATUS_NONFINITE);
    if (t_bump) *t_bump += 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) head_backward_kernel(int B, int A, double alpha, const T* __restrict__ out,
                                                           const T* __restrict__ eps_used,
                                                           const T* __restrict__ da, T* __restrict__ dout) {
  pdl_enter();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const T ab = T(alpha / B);
  for (int d = 0; d < A; ++d) {
    const T mu = out[(size_t)b * 2 * A + d];
    const T lraw = out[(size_t)b * 2 * A + A + d];
    const T l = fmin(fmax(lraw, T(kLogStdMin)), T(kLogStdMax));
    const T sigma = dev_exp(l);
    const T e = eps_used[(size_t)b * A + d];
    const T a = dev_tanh(mu + sigma * e);
    const T du = da[(size_t)b * A + d] * (T(1) - a * a) + ab * T(2) * a;
    const T dl = du * sigma * e - ab;
    const bool inside = lraw > T(kLogStdMin) && lraw < T(kLogStdMax);
    dout[(size_t)b * 2 * A + d] = du;
    dout[(size_t)b * 2 * A + A + d] = inside ? dl : T(0);
  }
}

}  // namespace

template <typename T>
void actor_head_forward(const ActorSpec& as, const T* pi_out, const float* eps, const unsigned long long* step_dev,
                        uint64_t seed, uint64_t agent, int B, T* a_new, T* logpi, T* eps_used, cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)B * as.A * sizeof(T) * 5);
  launch_k(head_forward_kernel<T>, dim3(ceil_div(B, 8)), dim3(256), 0, st, B, as.A, pi_out, eps, step_dev, seed, agent, a_new,
                                                           logpi, eps_used);
}

template <typename T>
void actor_energy_and_loss(const ActorSpec& as, const T* phi, const T* psi, const T* logpi, int B, int R, T* dphi,
                           T* fdiag, T* loss2, unsigned* status, int* t_bump, cudaStream_t st) {
  {
    TraceLaunch tr(CRL_TRACE_ENERGY, st, 2.0 * B * R);
    launch_k(diag_energy_kernel<T>, dim3(ceil_div(B, 8)), dim3(256), 0, st, B, R, as.energy, as.tau, phi, psi, fdiag, dphi);
  }
  TraceLaunch tr(CRL_TRACE_AUX, st, 2.0 * B * sizeof(T));
  launch_k(actor_loss_kernel<T>, dim3(1), dim3(1024), 0, st, B, as.alpha, logpi, fdiag, loss2, status, t_bump);
}

template <typename T>
void actor_head_backward(const ActorSpec& as, const T* pi_out, const T* eps_used, const T* da, int B, T* dout,
                         cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)B * as.A * sizeof(T) * 6);
  launch_k(head_backward_kernel<T>, dim3(ceil_div(B, 256)), dim3(256), 0, st, B, as.A, as.alpha, pi_out, eps_used, da, dout);
}

#define CRL_INST_ACTOR(T)                                                                                        \
  template void actor_head_forward<T>(const ActorSpec&, const T*, const float*, const unsigned long long*,       \
                                      uint64_t, uint64_t, int, T*, T*, T*, cudaStream_t);                        \
  template void actor_energy_and_loss<T>(const ActorSpec&, const T*, const T*, const T*, int, int, T*, T*, T*,   \
                                         unsigned*, int*, cudaStream_t);                                         \
  template void actor_head_backward<T>(const ActorSpec&, const T*, const T*, const T*, int, T*, cudaStream_t);
CRL_INST_ACTOR(float)
CRL_INST_ACTOR(double)

}  // namespace crl
