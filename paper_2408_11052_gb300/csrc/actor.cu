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
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tables.h"
#include "actor_head.cuh"
#include "philox.cuh"
#include "trace.h"

namespace crl {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) head_forward_kernel(const __grid_constant__ HeadFwdArgs<T> p) {
  pdl_enter();
  head_forward_body(p, blockIdx.x);
}

// f_i = f(phi_i, psi_i) / tau and dphi_i = -(1/B) df_i/dphi_i, 8 rows per
// block of 4 warps (warp w: rows w and w + 4 of the block, side by side), and
// the loss loss2 = {mean(alpha log pi - f), mean log pi}: each block writes its
// partial sums (its rows in order), and the last block to finish (ticket) adds
// the partials in block order, so the result does not depend on which block
// finishes last.  dz != null: dphi is written as BF16 [B][ldz] (the phi
// network's output gradient) instead of T.
// Lane j owns the columns j, j + 32, ... of its row and sums them in that
// order; rows up to kDiagRegCols columns stay in registers between the sums
// and the gradient (one read of each row, the loads of both of the warp's rows
// in flight together), wider rows are read twice, one row after the other.
// (Two rows per warp keep a block of 8 rows to 4 warps: every block of a
// batch-8192 launch is resident at once.)
constexpr int kDiagRegCols = 256;
constexpr int kDiagThreads = 128;   // 4 warps, 2 rows each

template <typename T>
__device__ __forceinline__ T diag_grad(int energy, T a, T b, T sxy, T nx, T ny, T dist) {
  const T d = a - b;
  switch (energy) {
    case CRL_ENERGY_DOT: return b;
    case CRL_ENERGY_COS: {
      const T xh = a / nx, yh = b / ny;
      return (yh - xh * (sxy / (nx * ny))) / nx;
    }
    case CRL_ENERGY_L2: return (dist >= T(1e-12)) ? -d / dist : T(0);
    case CRL_ENERGY_L2SQ: return T(-2) * d;
    default: return (d > T(0)) ? T(-1) : ((d < T(0)) ? T(1) : T(0));
  }
}

// f_i, dphi_i and alpha log pi_i - f_i of row i from its five column sums.
template <typename T>
__device__ __forceinline__ T diag_finish(const ActorLossArgs<T>& p, int i, int lane, T sxy, T sxx, T syy, T sdd, T sad,
                                         T& f, T& nx, T& ny, T& dist) {
  sxy = warp_sum(sxy);
  sxx = warp_sum(sxx);
  syy = warp_sum(syy);
  sdd = warp_sum(sdd);
  sad = warp_sum(sad);
  const T it = T(1.0 / p.tau);
  switch (p.energy) {
    case CRL_ENERGY_DOT: f = sxy; break;
    case CRL_ENERGY_COS: f = sxy / (dev_sqrt(sxx) * dev_sqrt(syy)); break;
    case CRL_ENERGY_L2: f = -dev_sqrt(sdd); break;
    case CRL_ENERGY_L2SQ: f = -sdd; break;
    default: f = -sad; break;
  }
  f *= it;
  if (lane == 0) p.fdiag[i] = f;
  nx = dev_sqrt(sxx);
  ny = dev_sqrt(syy);
  dist = dev_sqrt(sdd);
  return sxy;
}

template <typename T>
__device__ __forceinline__ void diag_store(const ActorLossArgs<T>& p, int i, int c, T dv) {
  if (p.dz) p.dz[(size_t)i * p.ldz + c] = __float2bfloat16_rn((float)dv);
  else p.dphi[(size_t)i * p.R + c] = dv;
}

template <typename T>
__device__ __forceinline__ void diag_energy_loss_body(const ActorLossArgs<T>& p, int lb, int nb) {
  constexpr int kReg = kDiagRegCols / kWarp;
  __shared__ T s_a[8], s_l[8];
  __shared__ int s_last;
  const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
  const int B = p.B, R = p.R;
  const int rows[2] = {lb * 8 + w, lb * 8 + w + 4};
  T term[2] = {T(0), T(0)}, lpi[2] = {T(0), T(0)};
  // every block reads log alpha before its ticket; the last block updates it after all tickets
  const double alpha = p.tune.state ? exp(p.tune.state[0]) : p.alpha;
  const T scale = T(-1.0 / B) * T(1.0 / p.tau);
  if (R <= kDiagRegCols) {
    T xr[2][kReg], yr[2][kReg];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = rows[q];
      const T* x = p.phi + (size_t)(i < B ? i : 0) * R;
      const T* y = p.psi + (size_t)(i < B ? i : 0) * R;
#pragma unroll
      for (int u = 0; u < kReg; ++u) {
        const int c = lane + kWarp * u;
        xr[q][u] = (i < B && c < R) ? x[c] : T(0);
        yr[q][u] = (i < B && c < R) ? y[c] : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = rows[q];
      if (i >= B) continue;   // warp-uniform
      T sxy = 0, sxx = 0, syy = 0, sdd = 0, sad = 0;
#pragma unroll
      for (int u = 0; u < kReg; ++u) {
        if (lane + kWarp * u >= R) break;
        const T a = xr[q][u], b = yr[q][u], d = a - b;
        sxy += a * b;
        sxx += a * a;
        syy += b * b;
        sdd += d * d;
        sad += fabs(d);
      }
      T f, nx, ny, dist;
      sxy = diag_finish(p, i, lane, sxy, sxx, syy, sdd, sad, f, nx, ny, dist);
      lpi[q] = p.logpi[i];
      term[q] = T(alpha) * lpi[q] - f;
#pragma unroll
      for (int u = 0; u < kReg; ++u) {
        const int c = lane + kWarp * u;
        if (c >= R) break;
        diag_store(p, i, c, scale * diag_grad<T>(p.energy, xr[q][u], yr[q][u], sxy, nx, ny, dist));
      }
    }
  } else {
    for (int q = 0; q < 2; ++q) {
      const int i = rows[q];
      if (i >= B) continue;   // warp-uniform
      const T* x = p.phi + (size_t)i * R;
      const T* y = p.psi + (size_t)i * R;
      T sxy = 0, sxx = 0, syy = 0, sdd = 0, sad = 0;
      for (int c = lane; c < R; c += kWarp) {
        const T a = x[c], b = y[c], d = a - b;
        sxy += a * b;
        sxx += a * a;
        syy += b * b;
        sdd += d * d;
        sad += fabs(d);
      }
      T f, nx, ny, dist;
      sxy = diag_finish(p, i, lane, sxy, sxx, syy, sdd, sad, f, nx, ny, dist);
      lpi[q] = p.logpi[i];
      term[q] = T(alpha) * lpi[q] - f;
      for (int c = lane; c < R; c += kWarp)
        diag_store(p, i, c, scale * diag_grad<T>(p.energy, x[c], y[c], sxy, nx, ny, dist));
    }
  }
  if (lane == 0) {
    s_a[w] = term[0];
    s_l[w] = lpi[0];
    s_a[w + 4] = term[1];
    s_l[w + 4] = lpi[1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T a = 0, l = 0;
    for (int k = 0; k < 8; ++k) {
      a += s_a[k];
      l += s_l[k];
    }
    p.partial[2 * lb] = a;
    p.partial[2 * lb + 1] = l;
    __threadfence();
    s_last = (atomicAdd(p.ticket, 1u) == (unsigned)nb - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ T sm[32];
  // thread t adds the partials t, t + blockDim.x, ... in that order; the loads of
  // a group of four are issued before their additions
  T a = 0, l = 0;
  const int nt = blockDim.x;
  int k = threadIdx.x;
  for (; k + 3 * nt < nb; k += 4 * nt) {
    T pa[4], pl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pa[u] = __ldcg(p.partial + 2 * (k + u * nt));
      pl[u] = __ldcg(p.partial + 2 * (k + u * nt) + 1);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a += pa[u];
      l += pl[u];
    }
  }
  for (; k < nb; k += nt) {
    a += __ldcg(p.partial + 2 * k);
    l += __ldcg(p.partial + 2 * k + 1);
  }
  a = block_sum(a, sm);
  l = block_sum(l, sm);
  if (threadIdx.x == 0) {
    p.loss2[0] = a / T(B);
    p.loss2[1] = l / T(B);
    if (p.status && !finite_val(a)) atomicOr(p.status, CRL_STATUS_NONFINITE);
    if (p.t_bump) *p.t_bump += 1;
    if (p.tune.state) {
      double* s = p.tune.state;
      s[3] = exp(s[0]);
      if (p.t_bump) {
        // Adam on log alpha: gradient of -log alpha * (mean log pi + target entropy)
        const int t = *p.t_bump;
        const double g = -((double)l / B + p.tune.target_entropy);
        const double b1 = p.tune.b1, b2 = p.tune.b2;
        const double m = b1 * s[1] + (1.0 - b1) * g;
        const double v = b2 * s[2] + (1.0 - b2) * g * g;
        const double mh = m / (1.0 - pow(b1, (double)t)), vh = v / (1.0 - pow(b2, (double)t));
        s[0] -= p.tune.lr * mh / (sqrt(vh) + p.tune.eps);
        s[1] = m;
        s[2] = v;
      }
    }
    // next relabel step: the one this step's relabel used, plus one
    if (p.step_bump) *p.step_bump = *p.last_step + 1ull;
    *p.ticket = 0u;
  }
}

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) diag_energy_loss_kernel(const __grid_constant__ ActorLossArgs<T> p) {
  pdl_enter();
  diag_energy_loss_body(p, blockIdx.x, gridDim.x);
}

// One thread per element (b, d) of the B x A action gradient, consecutive
// threads along d then b (coalesced row segments).  dz != null: the gradient
// is written as BF16 dz [B][ldz] (the policy network's output gradient)
// instead of dout.
constexpr int kHeadBwdThreads = 256;
template <typename T>
__device__ __forceinline__ void head_backward_body(const HeadBwdArgs<T>& p, int lb) {
  const int B = p.B, A = p.A;
  const int idx = lb * kHeadBwdThreads + (int)threadIdx.x;
  if (idx >= B * A) return;
  const int b = idx / A, d = idx - b * A;
  const T ab = T((p.alpha_used ? *p.alpha_used : p.alpha) / B);
  const T mu = p.out[(size_t)b * 2 * A + d];
  const T lraw = p.out[(size_t)b * 2 * A + A + d];
  const T l = fmin(fmax(lraw, T(kLogStdMin)), T(kLogStdMax));
  const T sigma = dev_exp(l);
  const T e = p.eps_used[(size_t)b * A + d];
  const T a = dev_tanh(mu + sigma * e);
  const T du = p.da[(size_t)b * A + d] * (T(1) - a * a) + ab * T(2) * a;
  const T dl = du * sigma * e - ab;
  const bool inside = lraw > T(kLogStdMin) && lraw < T(kLogStdMax);
  const T dlv = inside ? dl : T(0);
  if (p.dz) {
    p.dz[(size_t)b * p.ldz + d] = __float2bfloat16_rn((float)du);
    p.dz[(size_t)b * p.ldz + A + d] = __float2bfloat16_rn((float)dlv);
  } else {
    p.dout[(size_t)b * 2 * A + d] = du;
    p.dout[(size_t)b * 2 * A + A + d] = dlv;
  }
}

template <typename T>
__global__ void __launch_bounds__(kHeadBwdThreads) head_backward_kernel(const __grid_constant__ HeadBwdArgs<T> p) {
  pdl_enter();
  head_backward_body(p, blockIdx.x);
}

// ---- several agents in one launch (BF16 path: float) ----------------------------
__global__ void __launch_bounds__(kDiagThreads)
    diag_energy_loss_multi_kernel(const ActorLossArgs<float>* __restrict__ tasks, const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(begin, n, blockIdx.x, lb, nb);
  diag_energy_loss_body(tasks[s], lb, nb);
}
__global__ void __launch_bounds__(kHeadBwdThreads)
    head_backward_multi_kernel(const HeadBwdArgs<float>* __restrict__ tasks, const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(begin, n, blockIdx.x, lb, nb);
  head_backward_body(tasks[s], lb);
}

// Device tables of `tasks` and their block offsets (items_per_block items per
// block; a task has its batch B items, or B x A with PerAction).
template <bool PerAction = false, class Task>
const char* multi_tables(BlobCache& cache, const std::vector<Task>& tasks, int items_per_block, cudaStream_t st,
                         const Task** dt, const int** db, int* blocks) {
  std::vector<int> begin(tasks.size() + 1, 0);
  for (size_t i = 0; i < tasks.size(); ++i) {
    int items = tasks[i].B;
    if constexpr (PerAction) items *= tasks[i].A;
    begin[i + 1] = begin[i] + ceil_div(items, items_per_block);
  }
  *blocks = begin.back();
  const char* err = nullptr;
  if (!(*dt = cache.get(tasks, st, &err))) return err;
  if (!(*db = cache.get(begin, st, &err))) return err;
  return nullptr;
}

}  // namespace

template <typename T>
void actor_head_forward(const ActorSpec& as, const T* pi_out, const float* eps, const unsigned long long* step_dev,
                        uint64_t seed, uint64_t agent, int B, T* a_new, T* logpi, T* eps_used, cudaStream_t st,
                        __nv_bfloat16* x0, int x0_ld, int x0_col, int noise_extra) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)B * as.A * sizeof(T) * 5);
  const HeadFwdArgs<T> p{B,        as.A, pi_out, eps,   step_dev, seed,  agent,      a_new,
                         logpi,    eps_used, x0, x0_ld, x0_col,   noise_extra};
  launch_k(head_forward_kernel<T>, dim3(ceil_div(B, 8)), dim3(256), 0, st, p);
}

const char* actor_loss_multi(BlobCache& cache, const std::vector<ActorLossArgs<float>>& tasks, cudaStream_t st) {
  if (tasks.empty()) return nullptr;
  const ActorLossArgs<float>* dt;
  const int* db;
  int blocks;
  if (const char* err = multi_tables(cache, tasks, 8, st, &dt, &db, &blocks)) return err;
  double work = 0.0;
  for (const auto& t : tasks) work += 2.0 * t.B * t.R;
  TraceLaunch tr(CRL_TRACE_ENERGY, st, work);
  launch_k(diag_energy_loss_multi_kernel, dim3(blocks), dim3(kDiagThreads), 0, st, dt, db, (int)tasks.size());
  return nullptr;
}

const char* actor_head_backward_multi(BlobCache& cache, const std::vector<HeadBwdArgs<float>>& tasks,
                                      cudaStream_t st) {
  if (tasks.empty()) return nullptr;
  const HeadBwdArgs<float>* dt;
  const int* db;
  int blocks;
  if (const char* err = multi_tables<true>(cache, tasks, kHeadBwdThreads, st, &dt, &db, &blocks)) return err;
  double bytes = 0.0;
  for (const auto& t : tasks) bytes += (double)t.B * t.A * 4.0 * 6;
  TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
  launch_k(head_backward_multi_kernel, dim3(blocks), dim3(kHeadBwdThreads), 0, st, dt, db, (int)tasks.size());
  return nullptr;
}

size_t actor_loss_ws_bytes(int B, size_t elem) { return (size_t)ceil_div(B, 8) * 2 * elem + 256; }

template <typename T>
void actor_energy_and_loss(const ActorSpec& as, const T* phi, const T* psi, const T* logpi, int B, int R, T* dphi,
                           T* fdiag, T* loss2, void* ws, unsigned* ticket, unsigned* status, int* t_bump,
                           unsigned long long* step_bump, const unsigned long long* last_step, cudaStream_t st,
                           __nv_bfloat16* dz, int ldz) {
  ActorLossArgs<T> p{B,    R,     as.energy, as.tau, as.alpha, phi,    psi,       logpi,     fdiag,
                     dphi, dz,    ldz,       static_cast<T*>(ws), ticket, loss2, status, t_bump, step_bump,
                     last_step, as.tune};
  TraceLaunch tr(CRL_TRACE_ENERGY, st, 2.0 * B * R);
  launch_k(diag_energy_loss_kernel<T>, dim3(ceil_div(B, 8)), dim3(kDiagThreads), 0, st, p);
}

template <typename T>
void actor_head_backward(const ActorSpec& as, const T* pi_out, const T* eps_used, const T* da, int B, T* dout,
                         cudaStream_t st, __nv_bfloat16* dz, int ldz) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)B * as.A * sizeof(T) * 6);
  const HeadBwdArgs<T> p{B, as.A, as.alpha, pi_out, eps_used, da, dout, dz, ldz,
                         as.tune.state ? as.tune.state + 3 : nullptr};
  launch_k(head_backward_kernel<T>, dim3(ceil_div(B * as.A, kHeadBwdThreads)), dim3(kHeadBwdThreads), 0, st, p);
}

#define CRL_INST_ACTOR(T)                                                                                        \
  template void actor_head_forward<T>(const ActorSpec&, const T*, const float*, const unsigned long long*,       \
                                      uint64_t, uint64_t, int, T*, T*, T*, cudaStream_t, __nv_bfloat16*, int,    \
                                      int, int);                                                                 \
  template void actor_energy_and_loss<T>(const ActorSpec&, const T*, const T*, const T*, int, int, T*, T*, T*,   \
                                         void*, unsigned*, unsigned*, int*, unsigned long long*,                 \
                                         const unsigned long long*, cudaStream_t, __nv_bfloat16*, int);          \
  template void actor_head_backward<T>(const ActorSpec&, const T*, const T*, const T*, int, T*, cudaStream_t,    \
                                       __nv_bfloat16*, int);
CRL_INST_ACTOR(float)
CRL_INST_ACTOR(double)

}  // namespace crl
