// Energy matrix + InfoNCE + logsumexp penalty, forward and backward: the plain
// SIMT path (FP32 / FP64), which writes the B x B matrix to HBM.
//
// arXiv 2408.11052: §3.1 (critic objective: symmetric InfoNCE over the batch,
// L2 energy), App. A.2 (energies cos, dot, -L1, -L2, -L2^2; InfoNCE forward,
// backward, symmetric), Algorithm 1 (critic loss + beta * logsumexp penalty).
// Readings: F_ij = f(phi_i, psi_j) / tau; losses averaged over the batch;
// symmetric = mean (or sum) of the two directions; penalty = beta * mean of
// the squared row (or column) logsumexp.
//
// Gradient: with P = row softmax of F, Q = column softmax, r / c the row /
// column logsumexp and (wf, wb), (pr, pc) the direction and penalty weights,
//   dL/dF_ij = (1/B) [wf (P_ij - d_ij) + wb (Q_ij - d_ij) + 2 beta (pr r_i P_ij + pc c_j Q_ij)].
// Chain rule through the energy, with H the per-pair coefficient:
//   dot:  dphi = (G/tau) psi,            dpsi = (G/tau)^T phi
//   L2:   H = G / (tau d),  dphi_i = (H psi)_i - (sum_j H_ij) phi_i,
//                           dpsi_j = (H^T phi)_j - (sum_i H_ij) psi_j   (H = 0 where d = 0)
//   L2^2: the same with H = 2 G / tau
//   cos:  the dot form on x = phi/|phi|, then dphi = (dx - x <x, dx>) / |phi|.
//   L1:   H = G / tau,  dphi_ik = -sum_j H_ij sign(phi_ik - psi_jk),
//                       dpsi_jk = -sum_i H_ij sign(psi_jk - phi_ik)   (sign(0) = 0)
//
// The other objectives of App. A.2 / §5.2 (d_i = F_ii, s = sigma, sp = softplus,
// all pair sums over j = 1..B):
//   FlatNCE fwd / bwd: value 0, dL/dF as InfoNCE fwd / bwd (wf or wb = 1).
//   FB:   value mean_i [-e^{d_i} + sum_{j != i} e^{2 F_ij} / (2 (B - 1))];
//         dL/dF_ij = e^{2 F_ij} / (B (B - 1)) (j != i), -e^{d_i} / B (j = i).
//   DPO:  value sum_ij sp(F_ij - d_i) / B^2;  e_ij = s(F_ij - d_i) / B^2.
//   IPO:  value sum_ij (d_i - F_ij - 1)^2 / B^2;  e_ij = -2 (d_i - F_ij - 1) / B^2.
//         For both, dL/dF_ij = e_ij - [i = j] k_i with k_i = sum_j e_ij.
//   SPPO: value sum_i (d_i - 1)^2 / B + sum_ij (F_ij + 1)^2 / B^2;
//         dL/dF_ij = 2 (F_ij + 1) / B^2 + [i = j] 2 (d_i - 1) / B.
//   NCE-binary: value sum_ij (sp(F_ij) - [i = j] F_ij) / B^2;  dL/dF_ij = (s(F_ij) - [i = j]) / B^2.
// One warp per row gives d_i, the row's share of the value and k_i.
#include <algorithm>

#include "common.cuh"
#include "gemm_simt.cuh"
#include "internal.h"
#include "trace.h"

namespace crl {

namespace {

template <typename T>
struct PlainWs {
  T* F;       // [B][B] energies, then the coefficient matrix H
  T* rsum;    // [B]
  T* csum;    // [B]
  T* inx;     // [B] 1/|phi_i|
  T* iny;     // [B] 1/|psi_j|
  T* dg;      // [B] F_ii (objectives outside InfoNCE)
  T* ov;      // [B] row i's share of the objective's value
  T* kd;      // [B] k_i of DPO / IPO
  T* xh;      // [B][R] phi / |phi|
  T* yh;      // [B][R] psi / |psi|
};

template <typename T>
PlainWs<T> carve_plain(int B, int R, void* ws) {
  PlainWs<T> w;
  T* p = static_cast<T*>(ws);
  w.F = p;
  p += (size_t)B * B;
  w.rsum = p;
  p += B;
  w.csum = p;
  p += B;
  w.inx = p;
  p += B;
  w.iny = p;
  p += B;
  w.dg = p;
  p += B;
  w.ov = p;
  p += B;
  w.kd = p;
  p += B;
  w.xh = p;
  p += (size_t)B * R;
  w.yh = p;
  return w;
}

template <typename T>
struct EpiEnergy {
  T* F;
  int ld;
  int energy;
  T inv_tau;
  const T* inx;
  const T* iny;
  __device__ void operator()(int m, int n, T acc) const {
    T v;
    switch (energy) {
      case CRL_ENERGY_L2: v = -dev_sqrt(acc); break;
      case CRL_ENERGY_COS: v = acc * inx[m] * iny[n]; break;
      case CRL_ENERGY_DOT: v = acc; break;
      default: v = -acc; break;  // L1, L2^2
    }
    F[(size_t)m * ld + n] = v * inv_tau;
  }
};

// Row normalisation: inv[i] = 1/|x_i|, xh = x * inv.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) normalize_rows_kernel(int B, int R, const T* __restrict__ x,
                                                            T* __restrict__ inv, T* __restrict__ xh) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= B) return;
  T s = 0;
  for (int c = lane; c < R; c += kWarp) {
    const T v = x[(size_t)row * R + c];
    s += v * v;
  }
  const T iv = T(1) / dev_sqrt(warp_sum(s));
  for (int c = lane; c < R; c += kWarp) xh[(size_t)row * R + c] = x[(size_t)row * R + c] * iv;
  if (lane == 0) inv[row] = iv;
}

// r_i = LSE_j F_ij.  One warp per row, two passes.
template <typename T>
__global__ void __launch_bounds__(256) row_lse_kernel(int B, const T* __restrict__ F, T* __restrict__ r) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= B) return;
  const T* f = F + (size_t)row * B;
  T m = -INFINITY;
  for (int c = lane; c < B; c += kWarp) m = fmax(m, f[c]);
  m = warp_max(m);
  T s = 0;
  for (int c = lane; c < B; c += kWarp) s += dev_exp(f[c] - m);
  s = warp_sum(s);
  if (lane == 0) r[row] = m + dev_log(s);
}

// c_j = LSE_i F_ij.  Block = 32 columns x 8 row groups; each thread keeps a
// running (max, sum) over its rows, then the 8 partials of a column are merged.
template <typename T>
__global__ void __launch_bounds__(256) col_lse_kernel(int B, const T* __restrict__ F, T* __restrict__ c) {
  pdl_enter();
  __shared__ T sm_m[8][33], sm_s[8][33];
  const int cx = threadIdx.x % 32, ry = threadIdx.x / 32;
  const int j = blockIdx.x * 32 + cx;
  T m = -INFINITY, s = 0;
  if (j < B) {
    for (int i = ry; i < B; i += 8) {
      const T x = F[(size_t)i * B + j];
      if (x > m) {
        s = s * dev_exp(m - x) + T(1);
        m = x;
      } else {
        s += dev_exp(x - m);
      }
    }
  }
  sm_m[ry][cx] = m;
  sm_s[ry][cx] = s;
  __syncthreads();
  if (ry == 0 && j < B) {
    T mm = sm_m[0][cx];
    for (int r = 1; r < 8; ++r) mm = fmax(mm, sm_m[r][cx]);
    T ss = 0;
    for (int r = 0; r < 8; ++r)
      if (sm_s[r][cx] > T(0)) ss += sm_s[r][cx] * dev_exp(sm_m[r][cx] - mm);
    c[j] = mm + dev_log(ss);
  }
}

// Row sums (warp per row) and column sums (thread per column) of H.
template <typename T>
__global__ void __launch_bounds__(256) row_sum_kernel(int B, const T* __restrict__ H, T* __restrict__ out) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= B) return;
  T s = 0;
  for (int c = lane; c < B; c += kWarp) s += H[(size_t)row * B + c];
  s = warp_sum(s);
  if (lane == 0) out[row] = s;
}
template <typename T>
__global__ void __launch_bounds__(256) col_sum_kernel(int B, const T* __restrict__ H, T* __restrict__ out) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B) return;
  T s = 0;
  for (int i = 0; i < B; ++i) s += H[(size_t)i * B + j];
  out[j] = s;
}

// wf, wb: weights of the InfoNCE directions in the loss and its gradient (FlatNCE
// takes InfoNCE's gradient); obj: the loss code.
struct DirWeights {
  double wf, wb, pr, pc;
  int obj;
};
inline DirWeights weights(const LossSpec& ls) {
  DirWeights w{0, 0, 0, 0, ls.loss};
  if (ls.loss == CRL_LOSS_FWD || ls.loss == CRL_LOSS_FLATNCE_FWD) w.wf = 1;
  else if (ls.loss == CRL_LOSS_BWD || ls.loss == CRL_LOSS_FLATNCE_BWD) w.wb = 1;
  else if (ls.loss == CRL_LOSS_SYM) w.wf = w.wb = (ls.sym_reduction == CRL_SYM_SUM) ? 1.0 : 0.5;
  if (ls.penalty_axis == CRL_PENALTY_ROW) w.pr = 1;
  else if (ls.penalty_axis == CRL_PENALTY_COL) w.pc = 1;
  else w.pr = w.pc = 0.5;
  return w;
}

template <typename T>
__device__ __forceinline__ T sigmoid(T x) {
  // 1 / (1 + e^{-x}) without overflow: e^{x} / (1 + e^{x}) for x < 0
  const T e = dev_exp(-fabs(x));
  return x >= T(0) ? T(1) / (T(1) + e) : e / (T(1) + e);
}

// Objectives outside InfoNCE: d_i, row i's share of the value and k_i (see the
// header comment).  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) objective_rows_kernel(int B, const T* __restrict__ F, int obj,
                                                            T* __restrict__ dg, T* __restrict__ ov,
                                                            T* __restrict__ kd) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= B) return;
  const T* f = F + (size_t)row * B;
  const T d = f[row];
  T v = 0, k = 0;
  for (int j = lane; j < B; j += kWarp) {
    const T x = f[j];
    switch (obj) {
      case CRL_LOSS_FB:
        if (j != row) v += dev_exp(T(2) * x);
        break;
      case CRL_LOSS_DPO:
        v += softplus(x - d);
        k += sigmoid(x - d);
        break;
      case CRL_LOSS_IPO: {
        const T u = d - x - T(1);
        v += u * u;
        k -= T(2) * u;
        break;
      }
      case CRL_LOSS_SPPO:
        v += (x + T(1)) * (x + T(1));
        break;
      case CRL_LOSS_NCE_BINARY:
        v += softplus(x);
        break;
      default: break;
    }
  }
  v = warp_sum(v);
  k = warp_sum(k);
  if (lane != 0) return;
  const T bb = T(B) * T(B);
  T val = 0;
  switch (obj) {
    case CRL_LOSS_FB: val = (-dev_exp(d) + v / (T(2) * T(B - 1))) / T(B); break;
    case CRL_LOSS_DPO:
    case CRL_LOSS_IPO: val = v / bb; break;
    case CRL_LOSS_SPPO: val = (T(B) * (d - T(1)) * (d - T(1)) + v) / bb; break;
    case CRL_LOSS_NCE_BINARY: val = (v - d) / bb; break;
    default: break;
  }
  dg[row] = d;
  ov[row] = val;
  kd[row] = k / bb;
}

inline bool has_rows_pass(int obj) { return obj >= CRL_LOSS_FB; }

// Loss parts from the diagonal of F and the row / column logsumexp.  One block.
// ov: per-row objective values (objectives outside InfoNCE; FlatNCE: null, value 0).
template <typename T>
__global__ void __launch_bounds__(1024) loss_kernel(int B, const T* __restrict__ F, int ldf, const T* __restrict__ r,
                                                   const T* __restrict__ c, const T* __restrict__ ov, DirWeights w,
                                                   double beta, T* __restrict__ loss4, unsigned* status,
                                                   int* t_bump) {
  pdl_enter();
  __shared__ T sm[32];
  T a_f = 0, a_b = 0, a_r2 = 0, a_c2 = 0, a_o = 0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const T d = F[(size_t)i * ldf + i];
    a_f += r[i] - d;
    a_b += c[i] - d;
    a_r2 += r[i] * r[i];
    a_c2 += c[i] * c[i];
    if (ov) a_o += ov[i];
  }
  a_f = block_sum(a_f, sm);
  a_b = block_sum(a_b, sm);
  a_r2 = block_sum(a_r2, sm);
  a_c2 = block_sum(a_c2, sm);
  a_o = block_sum(a_o, sm);
  if (threadIdx.x == 0) {
    const T inv = T(1) / T(B);
    const T lf = a_f * inv, lb = a_b * inv;
    const T pen = T(beta) * (T(w.pr) * a_r2 * inv + T(w.pc) * a_c2 * inv);
    const bool info = w.obj <= CRL_LOSS_SYM;
    const T total = (info ? T(w.wf) * lf + T(w.wb) * lb : a_o) + pen;
    loss4[0] = total;
    loss4[1] = lf;
    loss4[2] = lb;
    loss4[3] = pen;
    if (status && !finite_val(total)) atomicOr(status, CRL_STATUS_NONFINITE);
    if (t_bump) *t_bump += 1;
  }
}

// F -> H in place (see the header comment).
// dg, kd: F_ii and k_i from objective_rows_kernel (objectives outside InfoNCE).
template <typename T>
__global__ void __launch_bounds__(256) grad_coeff_kernel(int B, T* __restrict__ F, const T* __restrict__ r,
                                                        const T* __restrict__ c, const T* __restrict__ dg,
                                                        const T* __restrict__ kd, DirWeights w, double beta,
                                                        double dtotal, int energy, double tau) {
  pdl_enter();
  const size_t n = (size_t)B * B;
  const T scale = T(dtotal / B);
  const T bb = T(B) * T(B);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / B), j = (int)(e % B);
    const T f = F[e];
    const T P = dev_exp(f - r[i]);
    const T Q = dev_exp(f - c[j]);
    const T dlt = (i == j) ? T(1) : T(0);
    T g = T(w.wf) * (P - dlt) + T(w.wb) * (Q - dlt) + T(2.0 * beta) * (T(w.pr) * r[i] * P + T(w.pc) * c[j] * Q);
    g *= scale;
    if (w.obj >= CRL_LOSS_FB) {
      T o = 0;
      switch (w.obj) {
        case CRL_LOSS_FB: o = (i == j) ? -dev_exp(f) / T(B) : dev_exp(T(2) * f) / (T(B) * T(B - 1)); break;
        case CRL_LOSS_DPO: o = sigmoid(f - dg[i]) / bb - dlt * kd[i]; break;
        case CRL_LOSS_IPO: o = T(-2) * (dg[i] - f - T(1)) / bb - dlt * kd[i]; break;
        case CRL_LOSS_SPPO: o = T(2) * (f + T(1)) / bb + dlt * T(2) * (f - T(1)) / T(B); break;
        default: o = (sigmoid(f) - dlt) / bb; break;  // NCE-binary
      }
      g += T(dtotal) * o;
    }
    T h;
    switch (energy) {
      case CRL_ENERGY_L2: {
        const T d = -f * T(tau);
        h = (d >= T(1e-12)) ? g / (T(tau) * d) : T(0);
        break;
      }
      case CRL_ENERGY_L2SQ: h = T(2) * g / T(tau); break;
      default: h = g / T(tau); break;  // dot, cos
    }
    F[e] = h;
  }
}

// dphi_i = (dx_i - x_i <x_i, dx_i>) * inv_i, in place on dx.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) project_rows_kernel(int B, int R, const T* __restrict__ xh,
                                                          const T* __restrict__ inv, T* __restrict__ dx) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= B) return;
  T s = 0;
  for (int c = lane; c < R; c += kWarp) s += xh[(size_t)row * R + c] * dx[(size_t)row * R + c];
  s = warp_sum(s);
  const T iv = inv[row];
  for (int c = lane; c < R; c += kWarp) {
    const size_t o = (size_t)row * R + c;
    dx[o] = (dx[o] - xh[o] * s) * iv;
  }
}

}  // namespace

namespace {

// L1 energy gradient: out[a][k] = -sum_b Ht(a, b) sign(own[a][k] - oth[b][k]),
// Ht(a, b) = H[a][b] (transposed = 0: own = phi) or H[b][a] (transposed = 1:
// own = psi).  Block = 32 a x 32 k outputs (4 per thread), b in chunks of 32
// through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) l1_grad_kernel(int B, int R, const T* __restrict__ H, int transposed,
                                                     const T* __restrict__ own, const T* __restrict__ oth,
                                                     T* __restrict__ out) {
  pdl_enter();
  __shared__ T Hs[32][33];
  __shared__ T Os[32][33];
  const int a0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // k = k0 + tx, a = a0 + ty + 8 m
  T acc[4] = {T(0), T(0), T(0), T(0)};
  T mine[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int a = a0 + ty + 8 * m, k = k0 + tx;
    mine[m] = (a < B && k < R) ? own[(size_t)a * R + k] : T(0);
  }
  for (int b0 = 0; b0 < B; b0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int a = a0 + r, b = b0 + tx;
      T h = T(0);
      if (a < B && b < B) h = transposed ? H[(size_t)b * B + a] : H[(size_t)a * B + b];
      Hs[r][tx] = h;
      const int bb = b0 + r, k = k0 + tx;
      Os[r][tx] = (bb < B && k < R) ? oth[(size_t)bb * R + k] : T(0);
    }
    __syncthreads();
    const int nb = min(32, B - b0);
    for (int j = 0; j < nb; ++j) {
      const T o = Os[j][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const T d = mine[m] - o;
        const T sg = (d > T(0)) ? T(1) : ((d < T(0)) ? T(-1) : T(0));
        acc[m] += Hs[ty + 8 * m][j] * sg;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int a = a0 + ty + 8 * m, k = k0 + tx;
    if (a < B && k < R) out[(size_t)a * R + k] = -acc[m];
  }
}

}  // namespace

size_t infonce_ws_bytes(const LossSpec& ls, int B, int R, size_t elem, int path) {
  (void)ls;
  (void)path;
  return ((size_t)B * B + 7 * (size_t)B + 2 * (size_t)B * R) * elem;
}

template <typename T>
void infonce_forward(const LossSpec& ls, const T* phi, const T* psi, int B, int R, T* loss4, T* row_lse, T* col_lse,
                     void* ws, int path, unsigned* status, int* t_bump, cudaStream_t st) {
  (void)path;
  PlainWs<T> w = carve_plain<T>(B, R, ws);
  const int nb = ceil_div(B, 8);
  if (ls.energy == CRL_ENERGY_COS) {
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(normalize_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, phi, w.inx, w.xh); }
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(normalize_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, psi, w.iny, w.yh); }
  }
  EpiEnergy<T> ep{w.F, B, ls.energy, T(1.0 / ls.tau), w.inx, w.iny};
  LoadMK<T> la{phi, R};
  LoadNK<T> lb{psi, R};
  switch (ls.energy) {
    case CRL_ENERGY_L2:
    case CRL_ENERGY_L2SQ: gemm<T, InnerOp::kSqDiff>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
    case CRL_ENERGY_L1: gemm<T, InnerOp::kAbsDiff>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
    default: gemm<T, InnerOp::kMul>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
  }
  { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(row_lse_kernel<T>, dim3(nb), dim3(256), 0, st, B, w.F, row_lse); }
  { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(col_lse_kernel<T>, dim3(ceil_div(B, 32)), dim3(256), 0, st, B, w.F, col_lse); }
  const bool rows = has_rows_pass(ls.loss);
  if (rows) {
    TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0);
    launch_k(objective_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, (const T*)w.F, ls.loss, w.dg, w.ov, w.kd);
  }
  {
    TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0);
    launch_k(loss_kernel<T>, dim3(1), dim3(1024), 0, st, B, (const T*)w.F, B, (const T*)row_lse, (const T*)col_lse,
             rows ? (const T*)w.ov : nullptr, weights(ls), ls.beta, loss4, status, t_bump);
  }
}

template <typename T>
void infonce_backward(const LossSpec& ls, const T* phi, const T* psi, int B, int R, const T* row_lse,
                      const T* col_lse, double dtotal, T* dphi, T* dpsi, void* ws, int path, cudaStream_t st) {
  (void)path;
  PlainWs<T> w = carve_plain<T>(B, R, ws);
  const int nb = ceil_div(B, 8);
  // Recompute F (the forward's copy may have been overwritten by another call).
  if (ls.energy == CRL_ENERGY_COS) {
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(normalize_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, phi, w.inx, w.xh); }
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(normalize_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, psi, w.iny, w.yh); }
  }
  {
    EpiEnergy<T> ep{w.F, B, ls.energy, T(1.0 / ls.tau), w.inx, w.iny};
    LoadMK<T> la{phi, R};
    LoadNK<T> lb{psi, R};
    switch (ls.energy) {
      case CRL_ENERGY_L2:
      case CRL_ENERGY_L2SQ: gemm<T, InnerOp::kSqDiff>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
      case CRL_ENERGY_L1: gemm<T, InnerOp::kAbsDiff>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
      default: gemm<T, InnerOp::kMul>(B, B, R, la, lb, ep, st, CRL_TRACE_ENERGY); break;
    }
  }
  if (has_rows_pass(ls.loss)) {
    TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0);
    launch_k(objective_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, (const T*)w.F, ls.loss, w.dg, w.ov, w.kd);
  }
  const int ge = (int)std::min<int64_t>(ceil_div((int64_t)B * B, 256), 152 * 16);
  {
    TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0);
    launch_k(grad_coeff_kernel<T>, dim3(ge), dim3(256), 0, st, B, w.F, row_lse, col_lse, (const T*)w.dg,
             (const T*)w.kd, weights(ls), ls.beta, dtotal, ls.energy, ls.tau);
  }
  const T* H = w.F;
  if (ls.energy == CRL_ENERGY_L2 || ls.energy == CRL_ENERGY_L2SQ) {
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(row_sum_kernel<T>, dim3(nb), dim3(256), 0, st, B, H, w.rsum); }
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(col_sum_kernel<T>, dim3(ceil_div(B, 256)), dim3(256), 0, st, B, H, w.csum); }
    gemm<T>(B, R, B, LoadMK<T>{H, B}, LoadKN<T>{psi, R}, EpiSubRowScaled<T>{dphi, R, T(1), w.rsum, phi, R}, st,
            CRL_TRACE_ENERGY);
    gemm<T>(B, R, B, LoadTrans<T>{H, B}, LoadKN<T>{phi, R}, EpiSubRowScaled<T>{dpsi, R, T(1), w.csum, psi, R},
            st, CRL_TRACE_ENERGY);
  } else if (ls.energy == CRL_ENERGY_COS) {
    gemm<T>(B, R, B, LoadMK<T>{H, B}, LoadKN<T>{w.yh, R}, EpiScale<T>{dphi, R, T(1)}, st, CRL_TRACE_ENERGY);
    gemm<T>(B, R, B, LoadTrans<T>{H, B}, LoadKN<T>{w.xh, R}, EpiScale<T>{dpsi, R, T(1)}, st, CRL_TRACE_ENERGY);
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(project_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, w.xh, w.inx, dphi); }
    { TraceLaunch tr_(CRL_TRACE_ENERGY, st, 0.0); launch_k(project_rows_kernel<T>, dim3(nb), dim3(256), 0, st, B, R, w.yh, w.iny, dpsi); }
  } else if (ls.energy == CRL_ENERGY_L1) {
    const dim3 grid(ceil_div(R, 32), ceil_div(B, 32));
    {
      TraceLaunch tr_(CRL_TRACE_ENERGY, st, 2.0 * B * B * R);
      launch_k(l1_grad_kernel<T>, grid, dim3(256), 0, st, B, R, H, 0, phi, psi, dphi);
    }
    TraceLaunch tr_(CRL_TRACE_ENERGY, st, 2.0 * B * B * R);
    launch_k(l1_grad_kernel<T>, grid, dim3(256), 0, st, B, R, H, 1, psi, phi, dpsi);
  } else {  // dot
    gemm<T>(B, R, B, LoadMK<T>{H, B}, LoadKN<T>{psi, R}, EpiScale<T>{dphi, R, T(1)}, st, CRL_TRACE_ENERGY);
    gemm<T>(B, R, B, LoadTrans<T>{H, B}, LoadKN<T>{phi, R}, EpiScale<T>{dpsi, R, T(1)}, st, CRL_TRACE_ENERGY);
  }
}

template void infonce_forward<float>(const LossSpec&, const float*, const float*, int, int, float*, float*, float*,
                                     void*, int, unsigned*, int*, cudaStream_t);
template void infonce_forward<double>(const LossSpec&, const double*, const double*, int, int, double*, double*,
                                      double*, void*, int, unsigned*, int*, cudaStream_t);
template void infonce_backward<float>(const LossSpec&, const float*, const float*, int, int, const float*,
                                      const float*, double, float*, float*, void*, int, cudaStream_t);
template void infonce_backward<double>(const LossSpec&, const double*, const double*, int, int, const double*,
                                       const double*, double, double*, double*, void*, int, cudaStream_t);

}  // namespace crl
