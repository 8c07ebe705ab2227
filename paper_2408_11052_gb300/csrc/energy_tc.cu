// Fused energy + InfoNCE + logsumexp penalty on tcgen05 (the BF16 fused path):
// the B x B energy matrix is never written to HBM.
//
// arXiv 2408.11052: §3.1 critic objective, App. A.2 energies and InfoNCE
// directions, Algorithm 1 (critic loss + beta * logsumexp penalty).  Readings as
// in the plain path (C1-C7): F_ij = f(phi_i, psi_j) / tau, batch means, the
// penalty on the squared row (or column) logsumexp.
//
// Representations enter as BF16 X = phi (or phi / |phi| for cos) and Y = psi,
// plus a per-row FP32 auxiliary: |x|^2 of the BF16-rounded row (L2, L2^2) or
// 1 / |phi| (cos).  S = X Y^T is formed 128 x 128 at a time in TMEM; the L2
// energies use d^2 = |x|^2 + |y|^2 - 2 S (clamped at 0).
//
// forward:  one CTA per (row tile I, column tile J): S -> F tile in shared
//           memory -> per-row (max, sum) over the tile's columns and per-column
//           (max, sum) over the tile's rows, written as partials; the diagonal
//           entries F_ii.  A one-block finalize merges the partials into
//           r_i = LSE_j F_ij, c_j = LSE_i F_ij and the loss parts.
// backward: the "row pass" (one CTA per 128 rows of phi) loops over column
//           tiles: S -> coefficient tile H (dL/dF times the energy's chain-rule
//           factor) written as a BF16 K-major operand in shared memory ->
//           acc += H psi (TMEM).  dphi = acc - rowsum(H) phi (L2, L2^2), acc
//           (dot), or the tangent projection of acc (cos).  The "column pass"
//           is the same kernel with the roles of phi and psi (and of r and c)
//           exchanged.  Both write their result as BF16 dy [B][R] and dy^T
//           [R][B], the layout the encoder backward consumes.
//
// The other objectives of App. A.2 / §5.2 (FlatNCE, forward-backward, DPO, IPO,
// SPPO, NCE-binary; definitions and readings as in the plain path) ride on the
// same tiles.  FlatNCE is InfoNCE's gradient with the value 0.  For the rest the
// forward tile also sums each row's objective terms over its 128 columns
// (partials merged per row like the logsumexps), and the backward adds the
// objective's dL/dF_ij to the coefficient tile.  DPO and IPO need the anchor
// F_ii inside every tile: each forward CTA computes it for its rows from the
// BF16 operand rows (the same products the MMA sums), and the forward leaves it
// and k_i (the diagonal coefficient sum_j e_ij) for the backward.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "energy_args.cuh"
#include "energy_tc.cuh"
#include "tc_common.cuh"
#include "tc_host.h"
#include "trace.h"

namespace crl {

using namespace fe;

namespace {

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// F log2(e) of one pair from S = <x, y> and the row / column auxiliaries, with
// k1 = log2(e) / tau.  EK 0: L2, 1: L2^2, 2: dot / cos (normalised operands).
template <int EK>
__device__ __forceinline__ float energy2(float s, float ax, float ay, float k1) {
  if (EK == 0) return -sqrt_approx(fmaxf(ax + ay - 2.f * s, 0.f)) * k1;
  if (EK == 1) return -fmaxf(ax + ay - 2.f * s, 0.f) * k1;
  return s * k1;
}

// One thread's 32 columns of its row: S -> F log2(e) in place (-inf outside
// the batch: columns >= jn of an edge tile), returning their maximum.
template <int EK>
__device__ __forceinline__ float tile_row(float (&v)[32], float ax, const float* __restrict__ ay, float k1, bool full,
                                          int jn) {
  float m = -INFINITY;
  if (full) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      v[k] = energy2<EK>(v[k], ax, ay[k], k1);
      m = fmaxf(m, v[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      v[k] = (k < jn) ? energy2<EK>(v[k], ax, ay[k], k1) : -INFINITY;
      m = fmaxf(m, v[k]);
    }
  }
  return m;
}

// An interior tile row (every column inside the batch): F log2(e) in place, its
// maximum m and minimum mn, in one pass.
template <int EK>
__device__ __forceinline__ void tile_row_full(float (&v)[32], float ax, const float* __restrict__ ay, float k1,
                                              float& m, float& mn) {
  m = -INFINITY;
  mn = INFINITY;
  if constexpr (EK == 0) {
    // -L2, two columns per instruction (each lane rounds as energy2 does)
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
      const float2 t = fma_x2(make_float2(-2.f, -2.f), make_float2(v[k], v[k + 1]),
                              add_x2(make_float2(ax, ax), make_float2(ay[k], ay[k + 1])));
      const float2 f = mul_x2(make_float2(sqrt_approx(fmaxf(t.x, 0.f)), sqrt_approx(fmaxf(t.y, 0.f))),
                              make_float2(-k1, -k1));
      v[k] = f.x;
      v[k + 1] = f.y;
      m = fmaxf(m, fmaxf(f.x, f.y));
      mn = fminf(mn, fminf(f.x, f.y));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      v[k] = energy2<EK>(v[k], ax, ay[k], k1);
      m = fmaxf(m, v[k]);
      mn = fminf(mn, v[k]);
    }
  }
}

__device__ __forceinline__ float energy_of(int energy, float s, float ax, float ay, float inv_tau) {
  switch (energy) {
    case CRL_ENERGY_L2: return -sqrtf(fmaxf(ax + ay - 2.f * s, 0.f)) * inv_tau;
    case CRL_ENERGY_L2SQ: return -fmaxf(ax + ay - 2.f * s, 0.f) * inv_tau;
    default: return s * inv_tau;  // dot, cos (normalised operands)
  }
}

// ---- representation preparation ------------------------------------------------
// y [B][R] FP32 -> X [B][R] BF16 (normalised for cos), X^T [R][ldt] BF16, aux [B],
// for phi and psi in one launch.  Block = 32 rows, one warp per row; the
// transposed copy goes through a shared tile.
struct PrepSide {
  const float* y;
  bf16* X;
  bf16* XT;
  float* aux;
};
// lb: block of 32 rows.
__device__ __forceinline__ void prep_body(int B, int R, int energy, int ldt, const PrepSide& p, int lb) {
  const float* __restrict__ y = p.y;
  bf16* __restrict__ X = p.X;
  bf16* __restrict__ XT = p.XT;
  float* __restrict__ aux = p.aux;
  __shared__ float tile[32][33];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int row = lb * 32 + w;
  float scale = 1.f;
  if (row < B) {
    const float* yr = y + (size_t)row * R;
    float q = 0.f;
    for (int c = lane; c < R; c += 32) {
      const float v = yr[c];
      if (energy == CRL_ENERGY_COS) {
        q += v * v;
      } else {
        const float b = __bfloat162float(__float2bfloat16_rn(v));
        q += b * b;
      }
    }
    q = warp_sum(q);
    if (energy == CRL_ENERGY_COS) scale = rsqrtf(q);
    if (lane == 0) aux[row] = (energy == CRL_ENERGY_COS) ? scale : q;
  }
  for (int c0 = 0; c0 < R; c0 += 32) {
    const int c = c0 + lane;
    float v = 0.f;
    if (row < B && c < R) {
      v = y[(size_t)row * R + c] * scale;
      X[(size_t)row * R + c] = __float2bfloat16_rn(v);
    }
    tile[w][lane] = v;
    __syncthreads();
    const int cc = c0 + w, rr = lb * 32 + lane;
    if (XT && cc < R && rr < B) XT[(size_t)cc * ldt + rr] = __float2bfloat16_rn(tile[lane][w]);
    __syncthreads();
  }
}

// blockIdx.y = 0: phi -> X, 1: psi -> Y.
__global__ void __launch_bounds__(1024) prep_kernel(int B, int R, int energy, int ldt, PrepSide s0, PrepSide s1) {
  pdl_enter();
  prep_body(B, R, energy, ldt, blockIdx.y ? s1 : s0, blockIdx.x);
}

// ---- forward ----------------------------------------------------------------------


// Row u's share of the objective's value from its merged partials (vp: the sum
// over j of the objective's pair terms; d: F_uu; see the plain path).
__device__ __forceinline__ float objective_share(int obj, int B, float vp, float d) {
  const float bb = (float)B * (float)B;
  switch (obj) {
    case CRL_LOSS_FB: return (-__expf(d) + vp / (2.f * (float)(B - 1))) / (float)B;
    case CRL_LOSS_SPPO: return ((float)B * (d - 1.f) * (d - 1.f) + vp) / bb;
    case CRL_LOSS_NCE_BINARY: return (vp - d) / bb;
    default: return vp / bb;  // DPO, IPO
  }
}

__device__ __forceinline__ void lse_merge(float& m, float& s, float m2, float s2) {
  if (s2 <= 0.f) return;
  if (s <= 0.f) {
    m = m2;
    s = s2;
    return;
  }
  const float M = fmaxf(m, m2);
  s = s * __expf(m - M) + s2 * __expf(m2 - M);
  m = M;
}

// Merge the npart partials of the 128 rows (col = false) or columns (col = true)
// of tile T into the logsumexps and this tile's loss partials.  One block of
// 512 threads: thread (item k, quarter q) merges partials q, q + 4, ... of item
// k (independent loads in flight), then the quarters merge in order.
constexpr int kMergeThreads = 512;
__device__ void merge_tile(const FwdArgs& a, int T, int npart, bool col) {
  __shared__ float s_q[4][4][kTile];   // per quarter: m, s, objective v, objective k
  __shared__ float s_red[3][kMergeThreads / 32];
  const int B = a.B, n = a.n;
  const float* part = col ? a.colpart : a.rowpart;
  const bool objrows = !col && a.obj >= CRL_LOSS_FB;
  const int k = threadIdx.x % kTile, qd = threadIdx.x / kTile;
  const int i = T * kTile + k;
  float m = -INFINITY, s = 0.f, vp = 0.f, kp = 0.f;
  if (i < B) {
    int P = qd;
    for (; P + 12 < npart; P += 16) {
      float pm[4], ps[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* p = part + ((size_t)(P + 4 * u) * B + i) * 2;
        pm[u] = __ldcg(p);
        ps[u] = __ldcg(p + 1);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) lse_merge(m, s, pm[u], ps[u]);
    }
    for (; P < npart; P += 4) {
      const float* p = part + ((size_t)P * B + i) * 2;
      lse_merge(m, s, __ldcg(p), __ldcg(p + 1));
    }
    if (objrows)
      for (int Q = qd; Q < npart; Q += 4) {
        const float* p = a.objpart + ((size_t)Q * B + i) * 2;
        vp += __ldcg(p);
        kp += __ldcg(p + 1);
      }
  }
  s_q[qd][0][k] = m;
  s_q[qd][1][k] = s;
  s_q[qd][2][k] = vp;
  s_q[qd][3][k] = kp;
  __syncthreads();
  float sd = 0.f, s2 = 0.f, so = 0.f;
  if (qd == 0 && i < B) {
    for (int g = 1; g < 4; ++g) {
      lse_merge(m, s, s_q[g][0][k], s_q[g][1][k]);
      vp += s_q[g][2][k];
      kp += s_q[g][3][k];
    }
    const float l = m + __logf(s);
    (col ? a.c_out : a.r_out)[i] = l;
    const float d = __ldcg(a.diag + i);
    sd = l - d;
    s2 = l * l;
    if (objrows) {
      so = objective_share(a.obj, B, vp, d);
      if (a.obj == CRL_LOSS_DPO || a.obj == CRL_LOSS_IPO) a.kd[i] = kp / ((float)B * (float)B);
    }
  }
  sd = warp_sum(sd);
  s2 = warp_sum(s2);
  so = warp_sum(so);
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  if (lane == 0) {
    s_red[0][w] = sd;
    s_red[1][w] = s2;
    s_red[2][w] = so;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int u = 0; u < kMergeThreads / 32; ++u) {
      a0 += s_red[0][u];
      a1 += s_red[1][u];
      a2 += s_red[2][u];
    }
    float* tp = a.tile_part + ((size_t)(col ? n : 0) + T) * 3;
    tp[0] = a0;
    tp[1] = a1;
    tp[2] = a2;
  }
}

// The loss parts from the 2 n tile partials, added in tile order.  The block
// stages the partials in shared memory kFinTiles tiles at a time (all loads in
// flight together) and thread 0 adds them in tile order.
constexpr int kFinTiles = 256;
__device__ void finalize_loss(const FwdArgs& a, int n) {
  __shared__ float s_tp[kFinTiles][5];
  float af = 0.f, ar2 = 0.f, ab = 0.f, ac2 = 0.f, ao = 0.f;
  for (int T0 = 0; T0 < n; T0 += kFinTiles) {
    const int cnt = min(kFinTiles, n - T0);
    for (int q = threadIdx.x; q < 5 * cnt; q += blockDim.x) {
      const int T = T0 + q / 5, r = q % 5;
      const float* src = r < 3 ? a.tile_part + 3 * T + r : a.tile_part + 3 * (n + T) + (r - 3);
      s_tp[q / 5][r] = __ldcg(src);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int u = 0; u < cnt; ++u) {
        af += s_tp[u][0];
        ar2 += s_tp[u][1];
        ao += s_tp[u][2];
        ab += s_tp[u][3];
        ac2 += s_tp[u][4];
      }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const float inv = 1.f / a.B;
  const float lf = af * inv, lb = ab * inv;
  const float pen = a.beta * (a.w.pr * ar2 * inv + a.w.pc * ac2 * inv);
  // FlatNCE: value 0; the objectives outside InfoNCE: the merged row shares
  const float contrastive = a.obj <= CRL_LOSS_SYM ? a.w.wf * lf + a.w.wb * lb : (a.obj >= CRL_LOSS_FB ? ao : 0.f);
  const float total = contrastive + pen;
  a.loss4[0] = total;
  a.loss4[1] = lf;
  a.loss4[2] = lb;
  a.loss4[3] = pen;
  if (a.status && !isfinite(total)) atomicOr(a.status, CRL_STATUS_NONFINITE);
  if (a.t_bump) *a.t_bump += 1;
}

// The forward's finalize: blocks [0, n) merge the row tiles' chunk partials,
// blocks [n, 2 n) the column tiles' row-tile partials, and the block completing
// the last merge adds the tiles' loss partials in tile order.
__device__ __forceinline__ void fwd_finalize_body(const FwdArgs& a, int lb) {
  const int n = a.n;
  const bool col = lb >= n;
  merge_tile(a, col ? lb - n : lb, col ? n : a.nC, col);
  __shared__ int s_fin;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_fin = (atomicAdd(a.tickets + 2 * n, 1u) == (unsigned)(2 * n) - 1u) ? 1 : 0;
  __syncthreads();
  if (s_fin) {   // block-uniform
    __threadfence();
    finalize_loss(a, n);
    if (threadIdx.x == 0) a.tickets[2 * n] = 0u;
  }
}

__global__ void __launch_bounds__(kMergeThreads) fwd_finalize_kernel(const __grid_constant__ FwdArgs a) {
  pdl_enter();
  fwd_finalize_body(a, blockIdx.x);
}


// ---- forward: one CTA per (row tile I, chunk of C column tiles) ------------------
// 18 warps: warps 0..15 run the epilogue (warp w: TMEM lanes 32 (w % 4) .. + 31,
// i.e. rows; columns 32 (w / 4) .. + 31 of each 128-wide tile), warp 16 lane 0
// loads (the row tile X once, then the column tiles Y through a ring of 64-wide
// K chunks), warp 17 issues the MMAs (S(t) = X Y(t)^T into TMEM buffer t % 2,
// once the epilogue has read buffer t % 2 of tile t - 2) and owns the TMEM.
// The epilogue of tile t runs while the MMAs of tile t + 1 fill the other
// buffer.  Per warp and tile (a 32 x 32 block of F log2(e)): the block maximum
// M_w is the reference of both sums, so each element takes one exp2:
// e = 2^(f - M_w), the row sums add e along the thread's 32 columns and the
// column sums add e down a warp-private shared tile.  When some element of the
// block lies more than 100 (log2 units) below M_w, the block takes exact
// per-row and per-column references instead (no term can underflow there).
// Row statistics run on across the chunk's tiles in registers (online merge);
// column statistics of the four row quarters merge in shared memory per tile.
constexpr int kFwdEpiWarps = 16;
constexpr int kFwdThreads = 32 * (kFwdEpiWarps + 2);
constexpr int kFwdYStages = 4;     // 16 KiB K chunks of Y in flight
constexpr float kFwdRange = 100.f;  // log2 units below the block maximum that the shared reference covers

__device__ __forceinline__ void lse2_merge(float& m, float& s, float m2, float s2) {
  if (s2 <= 0.f) return;
  if (s <= 0.f) {
    m = m2;
    s = s2;
    return;
  }
  const float M = fmaxf(m, m2);
  s = s * ex2(m - M) + s2 * ex2(m2 - M);
  m = M;
}
__device__ __forceinline__ float warp_min_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Shared memory of the forward (offsets from the 1024-aligned base).
struct FwdSmem {
  static constexpr size_t kX = 0;                                             // nk x 16 KiB row tile
  static constexpr size_t kY = 4 * 16384;                                     // ring of Y chunks
  static constexpr size_t kBlk = kY + (size_t)kFwdYStages * 16384;           // 16 x [32][32] warp blocks (swizzled)
  static constexpr size_t kCol = kBlk + (size_t)kFwdEpiWarps * 32 * 32 * 4;  // [2][4][128] (ref, sum)
  static constexpr size_t kRow = kCol + 2 * 4 * 128 * 2 * 4;                  // [4][128] (m, s)
  static constexpr size_t kObj = kRow + 4 * 128 * 2 * 4;                      // [4][128] objective (v, k)
  static constexpr size_t kD = kObj + 4 * 128 * 2 * 4;                        // [128] anchor F_ii
  static constexpr size_t kBar = kD + 128 * 4;                                // barriers
  static constexpr size_t kBytes = kBar + 16 * 8 + 1024;
};
static_assert(FwdSmem::kBytes <= 227 * 1024, "forward shared memory");

template <bool OBJ>
__device__ __forceinline__ void fwd_body(const CUtensorMap* tmX, const CUtensorMap* tmY, const FwdArgs& a, int I,
                                         int chunk, bool global_maps) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  const int n = a.n, C = a.C;
  const int nk = a.R / 64;
  const int t0 = chunk * C, nt = min(C, n - t0);   // column tiles t0 .. t0 + nt - 1
  uint8_t* Xs = smem + FwdSmem::kX;
  uint8_t* Ys = smem + FwdSmem::kY;
  float* blk_all = reinterpret_cast<float*>(smem + FwdSmem::kBlk);
  float* colbuf = reinterpret_cast<float*>(smem + FwdSmem::kCol);
  float* rowbuf = reinterpret_cast<float*>(smem + FwdSmem::kRow);
  float* objbuf = reinterpret_cast<float*>(smem + FwdSmem::kObj);
  float* s_d = reinterpret_cast<float*>(smem + FwdSmem::kD);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + FwdSmem::kBar);
  uint64_t* xfull = bars;                          // [1]
  uint64_t* yfull = bars + 1;                      // [kFwdYStages]
  uint64_t* yempty = yfull + kFwdYStages;          // [kFwdYStages]
  uint64_t* sfull = yempty + kFwdYStages;          // [2] S(t) in TMEM buffer t % 2
  uint64_t* sfree = sfull + 2;                     // [2] the epilogue has read buffer t % 2 (16 arrivals)
  uint64_t* drain = sfree + 2;                     // every MMA of this CTA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int i0 = I * kTile;
  if (tid == 0) {
    if (global_maps) {
      tc::tmap_acquire(tmX);
      tc::tmap_acquire(tmY);
    }
    tc::prefetch_tmap(tmX);
    tc::prefetch_tmap(tmY);
    tc::mbar_init(xfull, 1);
    for (int s = 0; s < kFwdYStages; ++s) {
      tc::mbar_init(&yfull[s], 1);
      tc::mbar_init(&yempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sfull[b], 1);
      tc::mbar_init(&sfree[b], kFwdEpiWarps);
    }
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == kFwdEpiWarps + 1) {
    tc::tmem_alloc(tmem_slot, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();
  const unsigned long long lim = tc::wait_limit(a.status);

  if (warp == kFwdEpiWarps) {
    if (lane == 0) {
      // the row tile once, then every column tile's K chunks through the ring
      tc::mbar_arrive_expect_tx(xfull, (uint32_t)nk * 16384u);
      for (int kb = 0; kb < nk; ++kb)
        for (int r = 0; r < 2; ++r) tc::tma_load_2d(Xs + kb * 16384 + r * 8192, tmX, xfull, kb * 64, i0 + 64 * r);
      int issued = 0;
      bool ok = true;
      for (int t = 0; t < nt && ok; ++t) {
        const int j0 = (t0 + t) * kTile;
        for (int kb = 0; kb < nk; ++kb) {
          const int it = t * nk + kb, st = it % kFwdYStages;
          if (it >= kFwdYStages && !tc::mbar_wait(&yempty[st], ((it / kFwdYStages) - 1) & 1, lim)) {
            atomicOr(a.status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          ++issued;
          tc::mbar_arrive_expect_tx(&yfull[st], 16384u);
          for (int r = 0; r < 2; ++r)
            tc::tma_load_2d(Ys + st * 16384 + r * 8192, tmY, &yfull[st], kb * 64, j0 + 64 * r);
        }
      }
      // nothing may land in this CTA's shared memory after it leaves
      tc::mbar_wait(xfull, 0, tc::kDrainLimitNs);
      tc::drain_ring(yfull, kFwdYStages, issued);
    }
  } else if (warp == kFwdEpiWarps + 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
      bool ok = tc::mbar_wait(xfull, 0, lim);
      if (!ok) atomicOr(a.status, CRL_STATUS_TIMEOUT);
      tc::fence_after_sync();
      for (int t = 0; t < nt && ok; ++t) {
        const int b = t & 1, use = t >> 1;
        if (use > 0 && !tc::mbar_wait(&sfree[b], (use - 1) & 1, lim)) {
          atomicOr(a.status, CRL_STATUS_TIMEOUT);
          break;
        }
        tc::fence_after_sync();
        for (int kb = 0; kb < nk; ++kb) {
          const int it = t * nk + kb, st = it % kFwdYStages;
          if (!tc::mbar_wait(&yfull[st], (it / kFwdYStages) & 1, lim)) {
            atomicOr(a.status, CRL_STATUS_TIMEOUT);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint64_t dx = tc::sdesc_kmajor_sw128(Xs + kb * 16384);
          const uint64_t dy = tc::sdesc_kmajor_sw128(Ys + st * 16384);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_bf16(tmem + (uint32_t)(b * 128), dx + 2 * k, dy + 2 * k, idesc, (kb | k) ? 1u : 0u);
          tc::mma_commit(&yempty[st]);
        }
        if (ok) tc::mma_commit(&sfull[b]);
      }
      tc::mma_commit(drain);   // completes once every MMA issued above has
    }
  } else {
    // ---- epilogue warps
    const int lg = warp % 4, q = warp / 4;
    const int r = lg * 32 + lane, i = i0 + r;
    const bool row_ok = i < a.B;
    const float ax = row_ok ? a.auxX[i] : 0.f;
    const float k1 = a.inv_tau * kLog2e;
    float* blk = blk_all + warp * (32 * 32);
    const bool anchored = OBJ && (a.obj == CRL_LOSS_DPO || a.obj == CRL_LOSS_IPO);
    if (anchored) {
      // the anchor F_ii of this CTA's rows: 4 threads per row, R / 4 columns of
      // the BF16 operand rows each (8 per 16-byte load)
      const int rr = tid / 4, part4 = tid % 4, ii = i0 + rr;
      float sxy = 0.f;
      if (ii < a.B) {
        const int per = a.R / 4;
        const uint4* xr = reinterpret_cast<const uint4*>(a.X + (size_t)ii * a.R + part4 * per);
        const uint4* yr = reinterpret_cast<const uint4*>(a.Y + (size_t)ii * a.R + part4 * per);
        for (int c = 0; c < per / 8; ++c) {
          const uint4 xv = xr[c], yv = yr[c];
          const bf16* xb = reinterpret_cast<const bf16*>(&xv);
          const bf16* yb = reinterpret_cast<const bf16*>(&yv);
#pragma unroll
          for (int e = 0; e < 8; ++e) sxy = fmaf(__bfloat162float(xb[e]), __bfloat162float(yb[e]), sxy);
        }
      }
      sxy += __shfl_xor_sync(0xffffffffu, sxy, 1);
      sxy += __shfl_xor_sync(0xffffffffu, sxy, 2);
      if (part4 == 0) {
        const float d = (ii < a.B) ? energy_of(a.energy, sxy, a.auxX[ii], a.auxY[ii], a.inv_tau) : 0.f;
        s_d[rr] = d;
        if (chunk == 0 && ii < a.B) a.dpre[ii] = d;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kFwdEpiWarps));
    }
    const float dpair = anchored ? s_d[r] : 0.f;
    float row_m = -INFINITY, row_s = 0.f;   // this row's running (max, sum) over the chunk, log2 units
    float vp = 0.f, kp = 0.f;               // objective partials of this row
    bool good = true;
    for (int t = 0; t < nt; ++t) {
      const int b = t & 1;
      const int J = t0 + t, j0 = J * kTile;
      // one decision for the four warps of column group q (they share barriers below)
      const bool ok_t = tc::mbar_wait(&sfull[b], (t >> 1) & 1, lim);
      good = tc::named_barrier_and(2 + q, 128, ok_t);
      if (!good) {
        if (lane == 0) atomicOr(a.status, CRL_STATUS_TIMEOUT);
        break;
      }
      tc::fence_after_sync();
      float v[32];
      tc::tmem_ld32(tmem + (uint32_t)(b * 128) + ((uint32_t)(lg * 32) << 16) + q * 32, v);
      // the buffer may take tile t + 2's MMAs once every warp has read it
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sfree[b]);
      // F log2(e) of row r, columns j0 + 32 q + k (-inf outside the batch)
      const int jb = j0 + q * 32;
      const int jn = row_ok ? min(32, a.B - jb) : 0;
      float ay[32];
      {
        const float4* a4 = reinterpret_cast<const float4*>(a.auxY + jb);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 x = (jb + 4 * k < a.B) ? __ldg(a4 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
          ay[4 * k] = x.x;
          ay[4 * k + 1] = x.y;
          ay[4 * k + 2] = x.z;
          ay[4 * k + 3] = x.w;
        }
      }
      float m, mn;
      const bool full = i0 + kTile <= a.B && j0 + kTile <= a.B;
      if (full) {
        // interior tile: energy, maximum and minimum in one pass
        switch (a.energy) {
          case CRL_ENERGY_L2: tile_row_full<0>(v, ax, ay, k1, m, mn); break;
          case CRL_ENERGY_L2SQ: tile_row_full<1>(v, ax, ay, k1, m, mn); break;
          default: tile_row_full<2>(v, ax, ay, k1, m, mn); break;
        }
      } else {
        switch (a.energy) {
          case CRL_ENERGY_L2: m = tile_row<0>(v, ax, ay, k1, false, jn); break;
          case CRL_ENERGY_L2SQ: m = tile_row<1>(v, ax, ay, k1, false, jn); break;
          default: m = tile_row<2>(v, ax, ay, k1, false, jn); break;
        }
        mn = INFINITY;
#pragma unroll
        for (int k = 0; k < 32; ++k) mn = fminf(mn, v[k] == -INFINITY ? INFINITY : v[k]);
      }
      if (J == I && q == lg) {
        // F_ii: column r of this tile, the thread's element k = lane (selected, not indexed)
        float dv = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) dv = (k == lane) ? v[k] : dv;
        if (row_ok) a.diag[i] = dv * kLn2;
      }
      if (OBJ && a.obj >= CRL_LOSS_FB) {
        // this row's objective terms over the 32 columns, F = v[k] ln 2
        const int jd = i - jb;
        switch (a.obj) {
          case CRL_LOSS_FB:
#pragma unroll
            for (int k = 0; k < 32; ++k)
              if (k < jn && k != jd) vp += ex2(2.f * v[k]);
            break;
          case CRL_LOSS_DPO:
#pragma unroll
            for (int k = 0; k < 32; ++k)
              if (k < jn) {
                const float x = v[k] * kLn2 - dpair;
                vp += softplusf(x);
                kp += sigmoidf_fast(x);
              }
            break;
          case CRL_LOSS_IPO:
#pragma unroll
            for (int k = 0; k < 32; ++k)
              if (k < jn) {
                const float x = dpair - v[k] * kLn2 - 1.f;
                vp += x * x;
                kp -= 2.f * x;
              }
            break;
          case CRL_LOSS_SPPO:
#pragma unroll
            for (int k = 0; k < 32; ++k)
              if (k < jn) {
                const float x = v[k] * kLn2 + 1.f;
                vp += x * x;
              }
            break;
          default:  // NCE-binary
#pragma unroll
            for (int k = 0; k < 32; ++k)
              if (k < jn) vp += softplusf(v[k] * kLn2);
            break;
        }
      }
      const float Mw = warp_max_f(m);
      const float mnw = warp_min_f(mn);
      float cref, csum;   // this warp's column statistics of column 32 q + lane over its 32 rows
      if (Mw == -INFINITY) {
        cref = -INFINITY;   // the block lies outside the batch
        csum = 0.f;
      } else if (mnw >= Mw - kFwdRange) {
        // one exp2 per element against the block maximum (no term underflows);
        // row r of the block goes to blk[32 r + (k ^ sw(r))], sw(r) = 4 (r % 8):
        // 16-byte stores along the row, conflict-free reads down a column
        float s = 0.f;
        const int swz = (lane & 7) << 2;
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
          const float2 d01 = add_x2(make_float2(v[4 * k4], v[4 * k4 + 1]), make_float2(-Mw, -Mw));
          const float2 d23 = add_x2(make_float2(v[4 * k4 + 2], v[4 * k4 + 3]), make_float2(-Mw, -Mw));
          float4 e4;
          e4.x = ex2(d01.x);
          e4.y = ex2(d01.y);
          e4.z = ex2(d23.x);
          e4.w = ex2(d23.y);
          const float2 p = add_x2(make_float2(e4.x, e4.z), make_float2(e4.y, e4.w));
          s += p.x + p.y;
          *reinterpret_cast<float4*>(blk + lane * 32 + ((4 * k4) ^ swz)) = e4;
        }
        lse2_merge(row_m, row_s, Mw, s);
        __syncwarp();
        float c = 0.f;
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) c += blk[rr * 32 + (lane ^ ((rr & 7) << 2))];
        cref = Mw;
        csum = c;
        __syncwarp();
      } else {
        // wide dynamic range: exact references per row and per column
        float s = 0.f;
        if (m != -INFINITY) {
#pragma unroll
          for (int k = 0; k < 32; ++k) s += ex2(v[k] - m);
        }
        lse2_merge(row_m, row_s, m, s);
        const int swz = (lane & 7) << 2;
#pragma unroll
        for (int k = 0; k < 32; ++k) blk[lane * 32 + (k ^ swz)] = v[k];
        __syncwarp();
        float cm = -INFINITY;
#pragma unroll 8
        for (int rr = 0; rr < 32; ++rr) cm = fmaxf(cm, blk[rr * 32 + (lane ^ ((rr & 7) << 2))]);
        float c = 0.f;
        if (cm != -INFINITY) {
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) c += ex2(blk[rr * 32 + (lane ^ ((rr & 7) << 2))] - cm);
        }
        cref = cm;
        csum = c;
        __syncwarp();
      }
      // merge the column statistics of the four row quarters of column group q
      float* cb = colbuf + (size_t)b * (4 * 128 * 2);
      cb[(lg * 128 + q * 32 + lane) * 2] = cref;
      cb[(lg * 128 + q * 32 + lane) * 2 + 1] = csum;
      asm volatile("bar.sync %0, 128;" ::"r"(2 + q));
      if (lg == 0) {
        float cm = cb[(q * 32 + lane) * 2], cs = cb[(q * 32 + lane) * 2 + 1];
#pragma unroll
        for (int g = 1; g < 4; ++g)
          lse2_merge(cm, cs, cb[(g * 128 + q * 32 + lane) * 2], cb[(g * 128 + q * 32 + lane) * 2 + 1]);
        const int j = jb + lane;
        if (j < a.B) {
          float* cp = a.colpart + ((size_t)I * a.B + j) * 2;
          cp[0] = cs > 0.f ? cm * kLn2 : -INFINITY;
          cp[1] = cs;
        }
      }
    }
    // this row's statistics over the chunk: merge the four column groups
    rowbuf[(q * 128 + r) * 2] = row_m;
    rowbuf[(q * 128 + r) * 2 + 1] = row_s;
    if (OBJ) {
      objbuf[(q * 128 + r) * 2] = vp;
      objbuf[(q * 128 + r) * 2 + 1] = kp;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kFwdEpiWarps));
    if (good && q == 0 && row_ok) {
      float mm = rowbuf[r * 2], ss = rowbuf[r * 2 + 1];
      for (int g = 1; g < 4; ++g) lse2_merge(mm, ss, rowbuf[(g * 128 + r) * 2], rowbuf[(g * 128 + r) * 2 + 1]);
      float* rp = a.rowpart + ((size_t)chunk * a.B + i) * 2;
      rp[0] = ss > 0.f ? mm * kLn2 : -INFINITY;
      rp[1] = ss;
      if (OBJ && a.obj >= CRL_LOSS_FB) {
        // the four column groups in order
        float* op = a.objpart + ((size_t)chunk * a.B + i) * 2;
        op[0] = objbuf[r * 2] + objbuf[(128 + r) * 2] + objbuf[(256 + r) * 2] + objbuf[(384 + r) * 2];
        op[1] = objbuf[r * 2 + 1] + objbuf[(128 + r) * 2 + 1] + objbuf[(256 + r) * 2 + 1] +
                objbuf[(384 + r) * 2 + 1];
      }
    }
  }
  __syncwarp();   // the loader and MMA warps reconverge after their single-lane loops
  // teardown: every MMA has completed before the TMEM is freed
  if (tid == 0) tc::mbar_wait(drain, 0, tc::kDrainLimitNs);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kFwdEpiWarps + 1) tc::tmem_dealloc(tmem, 256);
}

template <bool OBJ>
__global__ void __launch_bounds__(kFwdThreads, 1) fwd_kernel(const __grid_constant__ CUtensorMap tmX,
                                                             const __grid_constant__ CUtensorMap tmY,
                                                             const __grid_constant__ FwdArgs a) {
  fwd_body<OBJ>(&tmX, &tmY, a, blockIdx.x / a.nC, blockIdx.x % a.nC, false);
}

// ---- backward ---------------------------------------------------------------------

// Offset in a 128-byte-swizzled K-major tile (8-row groups of 1024 bytes) of
// the 16-byte chunk `chunk` (8 BF16 along K) of row `row`.
__device__ __forceinline__ uint32_t sw128_offset(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Per iteration (128 columns of the other side): the other tile arrives
// (TMA), S = own other^T (MMA), then while other^T is loaded into the same
// shared region, the 16 warps turn S into the BF16 coefficient tile H (warp w:
// rows 32 (w % 4) .., columns 32 (w / 4) ..), and the MMA adds H other into
// the TMEM accumulator.
// CTAs [0, nrow) run the row pass (own = phi), CTAs [nrow, 2 nrow) the column pass (own = psi).
// Per-row constants of the coefficient tile (own side = this thread's row).

// dL/dF x (chain factor of the energy) for this thread's 32 columns 32 q ..:
// with P_own = e^(F - l_own) and P_oth = e^(F - l_oth),
//   g = P_own k_own + P_oth k_oth - [u == v] k_diag,
// which is scale (w_f (P - d) + w_b (Q - d) + 2 beta (p_r r P + p_c c Q)) with
// P = e^(F - r), Q = e^(F - c) whichever side is own.  EK 0: L2 (F = -d / tau,
// factor 1 / (tau d), zero where d < 1e-12), 1: L2^2 (F = -d^2 / tau, factor
// 2 / tau), 2: dot / cos (F = s / tau, factor 1 / tau).  The BF16-rounded
// coefficients are packed in pairs and summed into rowsum.
// LIVE: which softmax terms carry weight in this pass (0: both, 1: own only,
// 2: other only); a term whose coefficient is zero for the whole pass (one
// InfoNCE direction, a one-axis penalty) costs no exp2.
// EDGE: the tile holds the diagonal or reaches past the batch (the per-pair
// tests run); interior tiles skip them.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// NC consecutive columns cb .. cb + NC - 1 of the tile (NC = 16 or 32).  The
// other side's per-column inputs come from global memory (every lane reads the
// same 16 bytes: L1 broadcasts): aux_o = its auxiliaries, lse_o = its
// logsumexps (LIVE != 1), with k_oth = kb_oth + k2_oth * lse.
template <int EK, int OBJ, int LIVE, bool EDGE, int NC>
__device__ __forceinline__ void build_h(const float (&sv)[NC], const HCoef& hc, const float* __restrict__ aux_o,
                                        const float* __restrict__ lse_o, float kb_oth, float k2_oth, int cb, int u,
                                        int v0, int B, float& rowsum, uint32_t (&packed)[NC / 2]) {
  // the per-column inputs of four columns at a time, the next group's loads
  // issued before this group's arithmetic
  float cax[4], clse[4], ckoth[4], nax[4] = {0.f, 0.f, 0.f, 0.f}, nlse[4] = {0.f, 0.f, 0.f, 0.f};
  auto load4 = [&](int k, float (&ax)[4], float (&ls)[4]) {
    const int c4 = v0 + cb + k;
    if (EDGE) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool in = c4 + e < B;
        if (EK != 2) ax[e] = in ? __ldg(aux_o + c4 + e) : 0.f;
        if (LIVE != 1) ls[e] = in ? __ldg(lse_o + c4 + e) : 0.f;
      }
    } else {
      if (EK != 2) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(aux_o + c4));
        ax[0] = t.x, ax[1] = t.y, ax[2] = t.z, ax[3] = t.w;
      }
      if (LIVE != 1) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(lse_o + c4));
        ls[0] = t.x, ls[1] = t.y, ls[2] = t.z, ls[3] = t.w;
      }
    }
  };
  load4(0, nax, nlse);
#pragma unroll
  for (int k = 0; k < NC; k += 2) {
    if ((k & 3) == 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cax[e] = nax[e];
        clse[e] = nlse[e];
      }
      if (k + 4 < NC) load4(k + 4, nax, nlse);
      if (LIVE != 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ckoth[e] = fmaf(k2_oth, clse[e], kb_oth);
          clse[e] *= kLog2e;
        }
      }
    }
    float h2[2];
    if constexpr (EK == 0 && LIVE != 0 && !EDGE && OBJ == kObjInfo) {
      // the common case (-L2, one live softmax term, interior tile, InfoNCE),
      // both columns of the pair at once: h = 2^(-k1 d - l2) k / (tau d), with
      // k / tau per row or per column
      const int c = k & 3;
      const float2 t2 = fma_x2(make_float2(-2.f, -2.f), make_float2(sv[k], sv[k + 1]),
                               make_float2(hc.a_own + cax[c], hc.a_own + cax[c + 1]));
      const float t0 = fmaxf(t2.x, 0.f), t1 = fmaxf(t2.y, 0.f);
      const float2 rs = make_float2(t0 >= 1e-24f ? rsqrt_approx(t0) : 0.f, t1 >= 1e-24f ? rsqrt_approx(t1) : 0.f);
      const float2 d = mul_x2(make_float2(t0, t1), rs);
      float2 arg, fac;
      if (LIVE == 1) {
        arg = fma_x2(make_float2(-hc.k1, -hc.k1), d, make_float2(-hc.l_own2, -hc.l_own2));
        fac = mul_x2(make_float2(hc.k_own_tau, hc.k_own_tau), rs);
      } else {
        arg = fma_x2(make_float2(-hc.k1, -hc.k1), d, make_float2(-clse[c], -clse[c + 1]));
        fac = mul_x2(make_float2(ckoth[c] * hc.inv_tau, ckoth[c + 1] * hc.inv_tau), rs);
      }
      const float2 hv = mul_x2(make_float2(ex2(arg.x), ex2(arg.y)), fac);
      h2[0] = hv.x;
      h2[1] = hv.y;
    } else {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int cl = cb + k + e;
        const int v = v0 + cl;
        const int c = (k & 3) + e;
        const float sval = sv[k + e];
        float f2, fac;
        if (EK == 0) {
          const float t = fmaxf(fmaf(-2.f, sval, hc.a_own + cax[c]), 0.f);
          const float rs = t >= 1e-24f ? rsqrt_approx(t) : 0.f;
          f2 = -(t * rs) * hc.k1;
          fac = hc.inv_tau * rs;
        } else if (EK == 1) {
          const float t = fmaxf(fmaf(-2.f, sval, hc.a_own + cax[c]), 0.f);
          f2 = -t * hc.k1;
          fac = 2.f * hc.inv_tau;
        } else {
          f2 = sval * hc.k1;
          fac = hc.inv_tau;
        }
        float g;
        if (LIVE == 1) g = ex2(f2 - hc.l_own2) * hc.k_own;
        else if (LIVE == 2) g = ex2(f2 - clse[c]) * ckoth[c];
        else g = fmaf(ex2(f2 - hc.l_own2), hc.k_own, ex2(f2 - clse[c]) * ckoth[c]);
        if (EDGE && u == v) g -= hc.k_diag;
        if (OBJ != kObjInfo) {
          const float d_row = hc.transposed ? (v < B ? __ldg(hc.dpre + v) : 0.f) : hc.d_own;
          const float k_row = hc.transposed ? (v < B ? __ldg(hc.kd + v) : 0.f) : hc.kd_own;
          g += objective_coef<OBJ>(f2, EDGE && u == v, d_row, k_row, hc);
        }
        h2[e] = (!EDGE || (u < B && v < B)) ? g * fac : 0.f;
      }
    }
    const __nv_bfloat162 p2 = __floats2bfloat162_rn(h2[0], h2[1]);
    // the row sum takes the BF16-rounded coefficients the MMA multiplies, so
    // acc - rowsum * own stays a sum of H (other - own) terms
    rowsum += __low2float(p2) + __high2float(p2);
    packed[k / 2] = *reinterpret_cast<const uint32_t*>(&p2);
  }
}

// lb in [0, 2 nrow): the row pass for lb < nrow, else the column pass.
//
// 18 warps.  Warp 16 lane 0 loads the own tile once and the other side's tiles
// into two buffers (tile v into buffer v % 2 once the MMAs of tile v - 2 are
// done with it).  Warp 17 lane 0 issues the MMAs in whatever order their inputs
// allow (polling): S(v) = own . other(v)^T into TMEM accumulator v % 2 once
// tile v has landed and the builders have read S(v - 2), and the two halves of
// acc += H(v) other(v) (K = 64 rows of the other tile each) as the builders
// publish them.  The 16 builder warps turn S(v) into the BF16 coefficient tile
// H one 64-column half at a time (warp w: rows 32 (w % 4) .., 16 columns of each
// half): the accumulation of one half runs while the next half (or the next
// tile's first half) is built, and S(v + 1) is ready before H(v) is done.
constexpr int kBwdWarps = 16;
constexpr int kBwdThreads = 32 * (kBwdWarps + 2);

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int OBJ>
__device__ __forceinline__ void bwd_body(const CUtensorMap* tmX, const CUtensorMap* tmY, const BwdArgs& row,
                                         const BwdArgs& col, int nrow, int lb, bool global_maps) {
  const bool colpass = lb >= nrow;
  const BwdArgs& a = colpass ? col : row;   // fields read where used (no register copy)
  const CUtensorMap* tmOwn = colpass ? tmY : tmX;
  const CUtensorMap* tmOther = colpass ? tmX : tmY;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = tc::align1024(smem_raw);
  const int nk = a.R / 64;
  const uint32_t tbytes = (uint32_t)nk * 16384;          // one operand tile
  uint8_t* Xs = smem;                                     // own tile                  nk x 16 KiB
  uint8_t* Ys = Xs + tbytes;                              // other tiles, 2 buffers    2 x nk x 16 KiB
  uint8_t* Hs = Ys + 2 * tbytes;                          // H halves                  2 x 16 KiB
  float* s_red = reinterpret_cast<float*>(Hs);              // [4][128] partial sums (H is free by then)
  uint64_t* bars = reinterpret_cast<uint64_t*>(Hs + 2 * 16384);
  uint64_t* xload = bars;
  uint64_t* yfull = bars + 1;   // [2] other tile v landed in buffer v % 2
  uint64_t* sfull = bars + 3;   // [2] S(v) in accumulator v % 2
  uint64_t* sfree = bars + 5;   // [2] the 16 builder warps have read S(v)
  uint64_t* hready = bars + 7;  // [2] the 16 builder warps have written half h of H(v)
  uint64_t* hdone = bars + 9;   // [2] the accumulation of half h of H(v) is done (its region is free;
                                //     after half 1 the other tile's buffer is free as well)
  uint64_t* drain = bars + 11;  // every MMA of this CTA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 12);
  constexpr uint32_t tcols = 512;  // S, S, acc (R <= 256)

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int u0 = (lb - (colpass ? nrow : 0)) * kTile;
  const int nV = (a.B + kTile - 1) / kTile;
  if (tid == 0) {
    if (global_maps) {
      tc::tmap_acquire(tmOwn);
      tc::tmap_acquire(tmOther);
    }
    tc::prefetch_tmap(tmOwn);
    tc::prefetch_tmap(tmOther);
    tc::mbar_init(xload, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&yfull[b], 1);
      tc::mbar_init(&sfull[b], 1);
      tc::mbar_init(&sfree[b], kBwdWarps);
      tc::mbar_init(&hready[b], kBwdWarps);
      tc::mbar_init(&hdone[b], 1);
    }
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == kBwdWarps + 1) {
    tc::tmem_alloc(tmem_slot, tcols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tAcc = tmem + 256;
  pdl_wait();
  pdl_trigger();
  const unsigned long long lim = tc::wait_limit(a.status);

  if (warp == kBwdWarps) {
    if (lane == 0) {
      // loader: the own tile once, then other tile v into buffer v % 2
      tc::mbar_arrive_expect_tx(xload, tbytes);
      for (int kb = 0; kb < nk; ++kb)
        for (int rr = 0; rr < 2; ++rr)
          tc::tma_load_2d(Xs + kb * 16384 + rr * 8192, tmOwn, xload, kb * 64, u0 + 64 * rr);
      int last = -1;
      for (int v = 0; v < nV; ++v) {
        if (v >= 2 && !tc::mbar_wait(&hdone[1], (v - 2) & 1, lim)) {
          atomicOr(a.status, CRL_STATUS_TIMEOUT);
          break;
        }
        uint8_t* dst = Ys + (v & 1) * tbytes;
        tc::mbar_arrive_expect_tx(&yfull[v & 1], tbytes);
        for (int kb = 0; kb < nk; ++kb)
          for (int rr = 0; rr < 2; ++rr)
            tc::tma_load_2d(dst + kb * 16384 + rr * 8192, tmOther, &yfull[v & 1], kb * 64, v * kTile + 64 * rr);
        last = v;
      }
      // nothing may land in this CTA's shared memory after it leaves
      tc::mbar_wait(xload, 0, tc::kDrainLimitNs);
      for (int b = 0; b < 2; ++b) {
        const int v = (last & 1) == b ? last : last - 1;
        if (v >= 0) tc::mbar_wait(&yfull[b], (uint32_t)((v >> 1) & 1), tc::kDrainLimitNs);
      }
    }
  } else if (warp == kBwdWarps + 1) {
    if (lane == 0) {
      // MMA issuer: S(v) and the halves of acc(v), each as soon as its inputs are ready
      constexpr uint32_t idesc_s = tc::idesc_bf16_f32(128, 128);
      const uint32_t idesc_acc = tc::idesc_bf16_f32_bmn(128, a.R);
      bool ok = tc::mbar_wait(xload, 0, lim);
      if (!ok) atomicOr(a.status, CRL_STATUS_TIMEOUT);
      tc::fence_after_sync();
      int next_s = 0, next_h = 0;   // next S(v) to issue; next accumulation half (2 v + h)
      unsigned long long t_idle = tc::globaltimer();
      while (ok && (next_s < nV || next_h < 2 * nV)) {
        bool progress = false;
        if (next_s < nV && next_s <= next_h / 2 + 1) {
          const int v = next_s, b = v & 1;
          if (tc::mbar_test_wait(&yfull[b], (v >> 1) & 1) &&
              (v < 2 || tc::mbar_test_wait(&sfree[b], ((v >> 1) - 1) & 1))) {
            tc::fence_after_sync();
            const uint8_t* ys = Ys + b * tbytes;
            for (int kb = 0; kb < nk; ++kb) {
              const uint64_t dx = tc::sdesc_kmajor_sw128(Xs + kb * 16384);
              const uint64_t dy = tc::sdesc_kmajor_sw128(ys + kb * 16384);
#pragma unroll
              for (int k = 0; k < 4; ++k)
                tc::mma_bf16(tmem + (uint32_t)(b * 128), dx + 2 * k, dy + 2 * k, idesc_s, (kb | k) ? 1u : 0u);
            }
            tc::mma_commit(&sfull[b]);
            ++next_s;
            progress = true;
          }
        }
        if (next_h < 2 * nV && next_h / 2 < next_s) {
          const int v = next_h / 2, h = next_h % 2;
          if (tc::mbar_test_wait(&hready[h], v & 1)) {
            tc::fence_after_sync();
            // half h of H (K = other rows 64 h .. 64 h + 63) times the other tile as the MN-major
            // B operand: K steps of 16 rows are 2048 bytes, R chunks of 64 columns 16 KiB apart
            const uint8_t* ys = Ys + (v & 1) * tbytes;
            const uint64_t dh = tc::sdesc_kmajor_sw128(Hs + h * 16384);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t dt = tc::sdesc_mnmajor_sw128(ys + h * 8192 + k * 2048, 16384);
              tc::mma_bf16(tAcc, dh + 2 * k, dt, idesc_acc, (v | h | k) ? 1u : 0u);
            }
            tc::mma_commit(&hdone[h]);
            ++next_h;
            progress = true;
          }
        }
        if (progress) {
          t_idle = tc::globaltimer();
        } else if (tc::globaltimer() - t_idle > lim) {
          atomicOr(a.status, CRL_STATUS_TIMEOUT);
          ok = false;
        } else {
          __nanosleep(128);   // leave the issue slots to the builder warps
        }
      }
      tc::mma_commit(drain);   // completes once every MMA issued above has
    }
  } else {
    // ---- builder warps
    const int lg = warp % 4, q = warp / 4;
    const int r = lg * 32 + lane;  // row of this thread within the tile
    const uint32_t lane_off = (uint32_t)(lg * 32) << 16;
    const int u = u0 + r;
    const float a_own = (u < a.B) ? a.aux_own[u] : 0.f;
    const float l_own = (u < a.B) ? a.lse_own[u] : 0.f;
    // loss weights of this side (row pass: forward direction and row penalty;
    // column pass: backward direction and column penalty) and of the other
    const float w_own = a.transposed ? a.w.wb : a.w.wf, p_own = a.transposed ? a.w.pc : a.w.pr;
    const float w_oth = a.transposed ? a.w.wf : a.w.wb, p_oth = a.transposed ? a.w.pr : a.w.pc;
    HCoef hc;
    hc.a_own = a_own;
    hc.l_own2 = l_own * kLog2e;
    hc.k_own = a.scale * (w_own + 2.f * a.beta * p_own * l_own);
    hc.k_own_tau = hc.k_own * a.inv_tau;
    hc.k_diag = a.scale * (a.w.wf + a.w.wb);
    const bool own_live = w_own != 0.f || (a.beta != 0.f && p_own != 0.f);
    const bool oth_live = w_oth != 0.f || (a.beta != 0.f && p_oth != 0.f);
    const int live = (own_live && oth_live) ? 0 : (oth_live ? 2 : 1);
    hc.inv_tau = a.inv_tau;
    hc.k1 = a.inv_tau * kLog2e;
    constexpr bool kAnchored = OBJ == kObjDPO || OBJ == kObjIPO;
    hc.d_own = (kAnchored && u < a.B) ? a.dpre[u] : 0.f;
    hc.kd_own = (kAnchored && u < a.B) ? a.kd[u] : 0.f;
    hc.dpre = a.dpre;
    hc.kd = a.kd;
    hc.dtotal = a.dtotal;
    hc.c_bb = a.dtotal / ((float)a.B * (float)a.B);
    hc.c_b = a.dtotal / (float)a.B;
    hc.c_fb = a.B > 1 ? a.dtotal / ((float)a.B * (float)(a.B - 1)) : 0.f;
    hc.transposed = a.transposed;
    const int ek = a.energy == CRL_ENERGY_L2 ? 0 : (a.energy == CRL_ENERGY_L2SQ ? 1 : 2);
    const float kb_oth = a.scale * w_oth, k2_oth = 2.f * a.scale * a.beta * p_oth;
    float rowsum = 0.f;
    bool ok = true;
    // No block-wide barrier per tile: each warp waits for what it reads (S(vt),
    // a free H region) and arrives on what it produces (S read, half written).
    for (int vt = 0; vt < nV && ok; ++vt) {
      const int v0 = vt * kTile, b = vt & 1;
      ok = __all_sync(0xffffffffu, tc::mbar_wait(&sfull[b], (vt >> 1) & 1, lim) ? 1 : 0) != 0;
      if (!ok) break;
      tc::fence_after_sync();
      // (the objectives outside InfoNCE always take the tested form: fewer instantiations)
      const bool edge = OBJ != kObjInfo || u0 == v0 || u0 + kTile > a.B || v0 + kTile > a.B;
#pragma unroll 1
      for (int h = 0; h < 2 && ok; ++h) {
        const int cb = 64 * h + 16 * q;   // this warp's 16 columns of half h
        float sv[16];
        tmem_ld16(tmem + (uint32_t)(b * 128) + lane_off + cb, sv);
        if (h == 1) {
          // this warp is done with S(vt): the accumulator may take S(vt + 2)
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&sfree[b]);
        }
        uint32_t packed[8];
#define CRL_BUILD_H(EK, LV, ED)                                                                              \
  build_h<EK, OBJ, LV, (ED) || OBJ != kObjInfo, 16>(sv, hc, a.aux_other, a.lse_other, kb_oth, k2_oth, cb, u, v0, \
                                                    a.B, rowsum, packed)
        switch (2 * (3 * ek + live) + (edge ? 1 : 0)) {
          case 0: CRL_BUILD_H(0, 0, false); break;
          case 1: CRL_BUILD_H(0, 0, true); break;
          case 2: CRL_BUILD_H(0, 1, false); break;
          case 3: CRL_BUILD_H(0, 1, true); break;
          case 4: CRL_BUILD_H(0, 2, false); break;
          case 5: CRL_BUILD_H(0, 2, true); break;
          case 6: CRL_BUILD_H(1, 0, false); break;
          case 7: CRL_BUILD_H(1, 0, true); break;
          case 8: CRL_BUILD_H(1, 1, false); break;
          case 9: CRL_BUILD_H(1, 1, true); break;
          case 10: CRL_BUILD_H(1, 2, false); break;
          case 11: CRL_BUILD_H(1, 2, true); break;
          case 12: CRL_BUILD_H(2, 0, false); break;
          case 13: CRL_BUILD_H(2, 0, true); break;
          case 14: CRL_BUILD_H(2, 1, false); break;
          case 15: CRL_BUILD_H(2, 1, true); break;
          case 16: CRL_BUILD_H(2, 2, false); break;
          default: CRL_BUILD_H(2, 2, true); break;
        }
#undef CRL_BUILD_H
        // half h's region is free once the accumulation of tile vt - 1's half h is done
        if (vt >= 1) {
          ok = __all_sync(0xffffffffu, tc::mbar_wait(&hdone[h], (vt - 1) & 1, lim) ? 1 : 0) != 0;
          if (!ok) break;
        }
        // columns 16 q .. 16 q + 15 of half h: 16-byte chunks 2 q, 2 q + 1 of the
        // half's 128-byte-swizzled K-major tile
        uint8_t* hb = Hs + h * 16384;
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          const uint4 val = make_uint4(packed[4 * c2], packed[4 * c2 + 1], packed[4 * c2 + 2], packed[4 * c2 + 3]);
          *reinterpret_cast<uint4*>(hb + sw128_offset(r, 2 * q + c2)) = val;
        }
        // make the generic-proxy H writes visible to the tensor core, then publish
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&hready[h]);
      }
    }
    if (!ok && lane == 0) atomicOr(a.status, CRL_STATUS_TIMEOUT);
    // every accumulation done: the H regions become the row-sum partials
    if (ok) ok = tc::mbar_wait(&hdone[1], (nV - 1) & 1, lim);
    ok = tc::named_barrier_and(1, 32 * kBwdWarps, ok);
    s_red[q * kTile + r] = rowsum;
    tc::fence_after_sync();
    asm volatile("bar.sync 1, %0;" ::"r"(32 * kBwdWarps));
    if (ok) {
      const float rs = s_red[r] + s_red[kTile + r] + s_red[2 * kTile + r] + s_red[3 * kTile + r];
      const float* own = a.own_f32 + (size_t)(u < a.B ? u : 0) * a.R;
      float proj = 0.f;
      if (a.energy == CRL_ENERGY_COS) {
        // <x_hat, acc> over all R columns: partial per column group, then combined
        float pp = 0.f;
        for (int c = q * 32; c < a.R; c += 128) {
          float v[32];
          tc::tmem_ld32(tAcc + lane_off + c, v);
#pragma unroll
          for (int k = 0; k < 32; ++k) pp += own[c + k] * a_own * v[k];
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kBwdWarps));
        s_red[q * kTile + r] = pp;
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kBwdWarps));
        proj = s_red[r] + s_red[kTile + r] + s_red[2 * kTile + r] + s_red[3 * kTile + r];
      }
      for (int c = q * 32; c < a.R; c += 128) {
        float v[32];
        tc::tmem_ld32(tAcc + lane_off + c, v);
        if (u < a.B) {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            float d = v[k];
            if (a.energy == CRL_ENERGY_L2 || a.energy == CRL_ENERGY_L2SQ) d -= rs * own[c + k];
            else if (a.energy == CRL_ENERGY_COS) d = (d - own[c + k] * a_own * proj) * a_own;
            v[k] = d;
          }
          if (a.d_out_f32 != nullptr) {
            float4* dst = reinterpret_cast<float4*>(a.d_out_f32 + (size_t)u * a.R + c);
#pragma unroll
            for (int k = 0; k < 8; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          } else {
            alignas(16) bf16 o[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) o[k] = __float2bfloat16_rn(v[k]);
            uint4* dst = reinterpret_cast<uint4*>(a.d_out + (size_t)u * a.R + c);
#pragma unroll
            for (int k = 0; k < 4; ++k) dst[k] = reinterpret_cast<const uint4*>(o)[k];
          }
        }
      }
    } else if (tid == 0) {
      atomicOr(a.status, CRL_STATUS_TIMEOUT);
    }
  }
  __syncwarp();   // the loader and MMA warps reconverge after their single-lane loops
  // teardown: every MMA has completed before the TMEM is freed
  if (tid == 0) tc::mbar_wait(drain, 0, tc::kDrainLimitNs);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kBwdWarps + 1) tc::tmem_dealloc(tmem, tcols);
}

template <int OBJ>
__global__ void __launch_bounds__(kBwdThreads, 1) bwd_kernel(const __grid_constant__ CUtensorMap tmX,
                                                             const __grid_constant__ CUtensorMap tmY,
                                                             const __grid_constant__ BwdArgs row,
                                                             const __grid_constant__ BwdArgs col, int nrow) {
  bwd_body<OBJ>(&tmX, &tmY, row, col, nrow, blockIdx.x, false);
}

// ---- several agents in one launch ------------------------------------------------
// Per-agent arguments and tensor maps in an immutable device table; agent s
// owns the blocks [begin[s], begin[s+1]) of each launch: 2 ceil(B / 32) prep
// blocks (phi then psi), n^2 forward tiles, 2 n backward CTAs.
struct EnergyTask {   // 128-byte aligned by its tensor maps
  CUtensorMap tmX, tmY;
  FwdArgs f;
  BwdArgs row, col;
  PrepSide s0, s1;
  int B, R, energy, ldt, n;
};

__global__ void __launch_bounds__(1024) prep_multi_kernel(const EnergyTask* __restrict__ tasks,
                                                         const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const EnergyTask& t = tasks[segment_of(begin, n, blockIdx.x, lb, nb)];
  const int half = nb / 2;
  prep_body(t.B, t.R, t.energy, t.ldt, lb < half ? t.s0 : t.s1, lb < half ? lb : lb - half);
}

template <bool OBJ>
__global__ void __launch_bounds__(kFwdThreads, 1) fwd_multi_kernel(const EnergyTask* __restrict__ tasks,
                                                                   const int* __restrict__ begin, int n) {
  int lb, nb;
  const EnergyTask& t = tasks[segment_of(begin, n, blockIdx.x, lb, nb)];
  fwd_body<OBJ>(&t.tmX, &t.tmY, t.f, lb / t.f.nC, lb % t.f.nC, true);
}

__global__ void __launch_bounds__(kMergeThreads) fwd_finalize_multi_kernel(const EnergyTask* __restrict__ tasks,
                                                                          const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const EnergyTask& t = tasks[segment_of(begin, n, blockIdx.x, lb, nb)];
  fwd_finalize_body(t.f, lb);
}

template <int OBJ>
__global__ void __launch_bounds__(kBwdThreads, 1) bwd_multi_kernel(const EnergyTask* __restrict__ tasks,
                                                               const int* __restrict__ begin, int n) {
  int lb, nb;
  const EnergyTask& t = tasks[segment_of(begin, n, blockIdx.x, lb, nb)];
  bwd_body<OBJ>(&t.tmX, &t.tmY, t.row, t.col, t.n, lb, true);
}

size_t fwd_smem(int R) {
  (void)R;
  return FwdSmem::kBytes;
}

int energy_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 152;
  }
  return n;
}

// Column tiles per forward CTA for an n x n tile grid: the chunk that minimises
// (waves of n * ceil(n / C) CTAs at one CTA per SM) x (C + 3), the 3 standing
// for a CTA's fixed cost (operand fill, last epilogue, merges) in tile times.
int fwd_chunk_tiles(int n) {
  const int sms = energy_sm_count();
  int best = 1;
  long long best_cost = -1;
  for (int C = 1; C <= std::min(n, 64); ++C) {
    const long long ctas = (long long)n * ((n + C - 1) / C);
    const long long cost = ((ctas + sms - 1) / sms) * (C + 3);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = C;
    }
  }
  return best;
}
size_t bwd_smem(int R) {
  // own tile, two other tiles, H (then the row-sum partials), three per-tile arrays, barriers, alignment
  // own tile, two other tiles, the two H halves (then the row-sum partials), barriers, alignment
  return (size_t)3 * (R / 64) * 16384 + 2 * 16384 + 128 + 1024;
}

FwdArgs fwd_args(const EnergyTc& e, const LossSpec& ls, int B, void* ws, float* loss4, float* r, float* c,
                 int* t_bump, unsigned* status) {
  const int n = (B + kTile - 1) / kTile;
  char* base = static_cast<char*>(ws);
  unsigned* tickets = reinterpret_cast<unsigned*>(base);
  float* tile_part = reinterpret_cast<float*>(base + round_up((2 * n + 1) * 4, 256));
  float* rowpart = reinterpret_cast<float*>(base + round_up((2 * n + 1) * 4, 256) + round_up(6 * n * 4, 256));
  float* colpart = rowpart + (size_t)2 * n * B;
  float* diag = colpart + (size_t)2 * n * B;
  float* objpart = diag + B;
  float* dpre = objpart + (size_t)2 * n * B;
  float* kd = dpre + B;
  // member by member into zeroed storage: the arguments also key device tables
  FwdArgs f;
  memset(&f, 0, sizeof(f));
  f.B = B;
  f.R = e.R;
  f.n = n;
  f.C = fwd_chunk_tiles(n);
  f.nC = (n + f.C - 1) / f.C;
  f.energy = ls.energy;
  f.obj = ls.loss;
  f.inv_tau = (float)(1.0 / ls.tau);
  f.auxX = e.auxX;
  f.auxY = e.auxY;
  f.X = e.X;
  f.Y = e.Y;
  f.objpart = objpart;
  f.dpre = dpre;
  f.kd = kd;
  f.rowpart = rowpart;
  f.colpart = colpart;
  f.diag = diag;
  f.status = status;
  f.w = loss_weights(ls);
  f.beta = (float)ls.beta;
  f.r_out = r;
  f.c_out = c;
  f.loss4 = loss4;
  f.t_bump = t_bump;
  f.tickets = tickets;
  f.tile_part = tile_part;
  return f;
}

// Backward arguments of the row pass (own = phi), member by member into zeroed storage.
BwdArgs bwd_args(const EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* r, const float* c,
                 double dtotal, bf16* dphi, unsigned* status, const FwdArgs& f) {
  BwdArgs a;
  memset(&a, 0, sizeof(a));
  a.B = B;
  a.R = e.R;
  a.energy = ls.energy;
  a.transposed = 0;
  a.obj = ls.loss;
  a.inv_tau = (float)(1.0 / ls.tau);
  a.beta = (float)ls.beta;
  a.scale = (float)(dtotal / B);
  a.dtotal = (float)dtotal;
  a.dpre = f.dpre;
  a.kd = f.kd;
  a.w = loss_weights(ls);
  a.aux_own = e.auxX;
  a.aux_other = e.auxY;
  a.lse_own = r;
  a.lse_other = c;
  a.own_f32 = phi;
  a.d_out = dphi;
  a.status = status;
  return a;
}

const char* mk(CUtensorMap* m, const void* base, int inner, int rows, int stride) {
  const char* err = nullptr;
  if (!tc::make_tmap_bf16(m, base, (uint64_t)inner, (uint64_t)rows, (uint64_t)stride, 64, &err)) return err;
  return nullptr;
}

}  // namespace

// Workspace of the forward: tickets [2 n + 1] (zeroed when the workspace is
// created, reset by the CTAs that use them), tile loss partials [2][n][3],
// rowpart [nJ][B][2], colpart [nI][B][2], diag [B], objpart [nJ][B][2],
// dpre [B], kd [B]; for the -L1 energy then the backward's per-segment partial
// gradients.
size_t energy_tc_base_bytes(int B) {
  const int n = (B + kTile - 1) / kTile;
  return (size_t)round_up((2 * n + 1) * 4, 256) + (size_t)round_up(6 * n * 4, 256) +
         ((size_t)2 * n * B * 3 + 3 * (size_t)B) * sizeof(float);
}
size_t energy_tc_ws_bytes(const LossSpec& ls, int B, int R) {
  const size_t base = energy_tc_base_bytes(B);
  if (ls.energy != CRL_ENERGY_L1) return base;
  return round_up(base, 256) + l1_part_floats(B, R) * sizeof(float);
}
namespace {
float* l1_part(void* ws, int B) {
  return reinterpret_cast<float*>(static_cast<char*>(ws) + round_up(energy_tc_base_bytes(B), 256));
}
}  // namespace

bool energy_tc_supported(const LossSpec& ls, int B, int R, const char** why) {
  if (R % 64 != 0 || R > 256) {
    *why = "the fused path needs repr to be 64, 128, 192 or 256";
    return false;
  }
  if (B % 8 != 0) {
    *why = "the fused path needs B to be a multiple of 8";
    return false;
  }
  return true;
}

const char* energy_tc_maps(EnergyTc& e, int B) {
  if (e.tm_B == B) return nullptr;
  const char* err;
  if ((err = mk(&e.tmX, e.X, e.R, B, e.R))) return err;
  if ((err = mk(&e.tmY, e.Y, e.R, B, e.R))) return err;
  e.tm_B = B;
  return nullptr;
}

void energy_tc_prepare(EnergyTc& e, const LossSpec& ls, const float* phi, const float* psi, int B, cudaStream_t st) {
  if (ls.energy == CRL_ENERGY_L1) return;   // the -L1 tiles read the FP32 rows themselves
  TraceLaunch tr(CRL_TRACE_ENERGY, st, 0.0);
  launch_k(prep_kernel, dim3(ceil_div(B, 32), 2), dim3(1024), 0, st, B, e.R, ls.energy, e.ldt,
           PrepSide{phi, e.X, e.XT, e.auxX}, PrepSide{psi, e.Y, e.YT, e.auxY});
}

void energy_tc_forward(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi, float* loss4,
                       float* r, float* c, void* ws, unsigned* status, int* t_bump, cudaStream_t st) {
  const int n = (B + kTile - 1) / kTile;
  FwdArgs a = fwd_args(e, ls, B, ws, loss4, r, c, t_bump, status);
  if (ls.energy == CRL_ENERGY_L1) {
    // SIMT tiles, one column tile per chunk
    a.C = 1;
    a.nC = n;
    a.phi = phi;
    a.psi = psi;
    l1_forward(a, st);
  } else {
    const size_t sm = fwd_smem(e.R);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(256));
      cudaFuncSetAttribute(fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(256));
      attr = true;
    }
    TraceLaunch tr(CRL_TRACE_ENERGY, st, 2.0 * B * B * e.R);
    if (ls.loss >= CRL_LOSS_FB)
      launch_k(fwd_kernel<true>, dim3(n * a.nC), dim3(kFwdThreads), sm, st, e.tmX, e.tmY, a);
    else
      launch_k(fwd_kernel<false>, dim3(n * a.nC), dim3(kFwdThreads), sm, st, e.tmX, e.tmY, a);
  }
  TraceLaunch trf(CRL_TRACE_ENERGY, st, 0.0);
  launch_k(fwd_finalize_kernel, dim3(2 * n), dim3(kMergeThreads), 0, st, a);
}

namespace {
template <int OBJ>
void launch_bwd_t(const EnergyTc& e, const BwdArgs& a, const BwdArgs& b, int n, size_t sm, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(bwd_kernel<OBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(256));
    attr = true;
  }
  launch_k(bwd_kernel<OBJ>, dim3(2 * n), dim3(kBwdThreads), sm, st, e.tmX, e.tmY, a, b, n);
}

template <int OBJ>
void launch_bwd_multi_t(const EnergyTask* dt, const int* db, int na, int blocks, size_t sm, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(bwd_multi_kernel<OBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(256));
    attr = true;
  }
  launch_k(bwd_multi_kernel<OBJ>, dim3(blocks), dim3(kBwdThreads), sm, st, dt, db, na);
}

void launch_bwd_multi(int kind, const EnergyTask* dt, const int* db, int na, int blocks, size_t sm,
                      cudaStream_t st) {
  switch (kind) {
    case kObjFB: launch_bwd_multi_t<kObjFB>(dt, db, na, blocks, sm, st); break;
    case kObjDPO: launch_bwd_multi_t<kObjDPO>(dt, db, na, blocks, sm, st); break;
    case kObjIPO: launch_bwd_multi_t<kObjIPO>(dt, db, na, blocks, sm, st); break;
    case kObjSPPO: launch_bwd_multi_t<kObjSPPO>(dt, db, na, blocks, sm, st); break;
    case kObjNCE: launch_bwd_multi_t<kObjNCE>(dt, db, na, blocks, sm, st); break;
    default: launch_bwd_multi_t<kObjInfo>(dt, db, na, blocks, sm, st); break;
  }
}
}  // namespace

namespace {
// Both passes: the tcgen05 backward, or the SIMT one for the -L1 energy.
void backward_passes(const EnergyTc& e, const LossSpec& ls, int B, BwdArgs& a, BwdArgs& b, void* ws,
                     cudaStream_t st) {
  a.other_f32 = b.own_f32;
  b.other_f32 = a.own_f32;
  if (ls.energy == CRL_ENERGY_L1) {
    l1_backward(a, b, l1_part(ws, B), st);
    return;
  }
  const int n = (B + kTile - 1) / kTile;
  const size_t sm = bwd_smem(e.R);
  TraceLaunch tr(CRL_TRACE_ENERGY, st, 8.0 * B * B * e.R);
  switch (obj_kind(ls.loss)) {
    case kObjFB: launch_bwd_t<kObjFB>(e, a, b, n, sm, st); break;
    case kObjDPO: launch_bwd_t<kObjDPO>(e, a, b, n, sm, st); break;
    case kObjIPO: launch_bwd_t<kObjIPO>(e, a, b, n, sm, st); break;
    case kObjSPPO: launch_bwd_t<kObjSPPO>(e, a, b, n, sm, st); break;
    case kObjNCE: launch_bwd_t<kObjNCE>(e, a, b, n, sm, st); break;
    default: launch_bwd_t<kObjInfo>(e, a, b, n, sm, st); break;
  }
}

// The column pass's arguments from the row pass's: the roles of phi and psi
// (and of r and c) exchanged.
BwdArgs column_args(const EnergyTc& e, const BwdArgs& a, const float* psi, const float* r, const float* c) {
  BwdArgs b = a;
  b.transposed = 1;
  b.aux_own = e.auxY;
  b.aux_other = e.auxX;
  b.lse_own = c;
  b.lse_other = r;
  b.own_f32 = psi;
  return b;
}
}  // namespace

void energy_tc_backward(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi, const float* r,
                        const float* c, double dtotal, __nv_bfloat16* dphi, __nv_bfloat16* dpsi, void* ws,
                        unsigned* status, cudaStream_t st) {
  const FwdArgs f = fwd_args(e, ls, B, ws, nullptr, nullptr, nullptr, nullptr, status);
  BwdArgs a = bwd_args(e, ls, B, phi, r, c, dtotal, dphi, status, f);
  BwdArgs b = column_args(e, a, psi, r, c);
  b.d_out = dpsi;
  backward_passes(e, ls, B, a, b, ws, st);
}

void energy_tc_backward_f32(EnergyTc& e, const LossSpec& ls, int B, const float* phi, const float* psi,
                            const float* r, const float* c, double dtotal, float* dphi, float* dpsi, void* ws,
                            unsigned* status, cudaStream_t st) {
  const FwdArgs f = fwd_args(e, ls, B, ws, nullptr, nullptr, nullptr, nullptr, status);
  BwdArgs a = bwd_args(e, ls, B, phi, r, c, dtotal, nullptr, status, f);
  a.d_out_f32 = dphi;
  BwdArgs b = column_args(e, a, psi, r, c);
  b.d_out_f32 = dpsi;
  backward_passes(e, ls, B, a, b, ws, st);
}

size_t energy_tc_ticket_bytes(int B) {
  const int n = (B + kTile - 1) / kTile;
  return (size_t)(2 * n + 1) * 4;
}

const char* energy_tc_multi(BlobCache& cache, const std::vector<EnergyAgent>& all, int stage, cudaStream_t st) {
  // the -L1 agents run their own SIMT launches; the rest share one launch per stage
  std::vector<EnergyAgent> agents;
  for (const EnergyAgent& g : all) {
    if (g.ls.energy != CRL_ENERGY_L1) {
      agents.push_back(g);
    } else if (stage == 1) {
      energy_tc_forward(*g.e, g.ls, g.B, g.phi, g.psi, g.loss4, g.r, g.c, g.ws, g.status, g.t_bump, st);
    } else if (stage == 2) {
      energy_tc_backward(*g.e, g.ls, g.B, g.phi, g.psi, g.r, g.c, 1.0, g.dphi, g.dpsi, g.ws, g.status, st);
    }
  }
  const int na = (int)agents.size();
  if (na == 0) return nullptr;
  std::vector<EnergyTask> tasks(na);
  std::vector<int> begin(na + 1, 0);
  int Rmax = 64;
  double work = 0.0;
  for (int i = 0; i < na; ++i) {
    const EnergyAgent& g = agents[i];
    EnergyTask& t = tasks[i];
    memset(&t, 0, sizeof(t));
    const EnergyTc& e = *g.e;
    t.tmX = e.tmX;
    t.tmY = e.tmY;
    t.B = g.B;
    t.R = e.R;
    t.energy = g.ls.energy;
    t.ldt = e.ldt;
    t.n = (g.B + kTile - 1) / kTile;
    t.s0 = PrepSide{g.phi, e.X, e.XT, e.auxX};
    t.s1 = PrepSide{g.psi, e.Y, e.YT, e.auxY};
    t.f = fwd_args(e, g.ls, g.B, g.ws, g.loss4, g.r, g.c, g.t_bump, g.status);
    t.row = bwd_args(e, g.ls, g.B, g.phi, g.r, g.c, 1.0, g.dphi, g.status, t.f);
    t.col = t.row;
    t.col.transposed = 1;
    t.col.aux_own = e.auxY;
    t.col.aux_other = e.auxX;
    t.col.lse_own = g.c;
    t.col.lse_other = g.r;
    t.col.own_f32 = g.psi;
    t.col.d_out = g.dpsi;
    const int nb = stage == 0 ? 2 * ceil_div(g.B, 32) : (stage == 1 ? t.n * t.f.nC : 2 * t.n);
    begin[i + 1] = begin[i] + nb;
    Rmax = std::max(Rmax, e.R);
    work += (stage == 1 ? 2.0 : 8.0) * g.B * g.B * e.R * (stage == 0 ? 0.0 : 1.0);
  }
  const char* err = nullptr;
  const EnergyTask* dt = cache.get(tasks, st, &err);
  if (!dt) return err;
  const int* db = cache.get(begin, st, &err);
  if (!db) return err;
  if (stage == 0) {
    TraceLaunch tr(CRL_TRACE_ENERGY, st, work);
    launch_k(prep_multi_kernel, dim3(begin[na]), dim3(1024), 0, st, dt, db, na);
  } else if (stage == 1) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(fwd_multi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(256));
      cudaFuncSetAttribute(fwd_multi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(256));
      attr = true;
    }
    bool obj = false;
    for (const EnergyAgent& g : agents) obj = obj || g.ls.loss >= CRL_LOSS_FB;
    {
      TraceLaunch tr(CRL_TRACE_ENERGY, st, work);
      if (obj) launch_k(fwd_multi_kernel<true>, dim3(begin[na]), dim3(kFwdThreads), fwd_smem(Rmax), st, dt, db, na);
      else launch_k(fwd_multi_kernel<false>, dim3(begin[na]), dim3(kFwdThreads), fwd_smem(Rmax), st, dt, db, na);
    }
    // the merges: 2 n blocks per agent
    std::vector<int> fb(na + 1, 0);
    for (int i = 0; i < na; ++i) fb[i + 1] = fb[i] + 2 * tasks[i].n;
    const int* dfb = cache.get(fb, st, &err);
    if (!dfb) return err;
    TraceLaunch trf(CRL_TRACE_ENERGY, st, 0.0);
    launch_k(fwd_finalize_multi_kernel, dim3(fb[na]), dim3(kMergeThreads), 0, st, dt, dfb, na);
  } else {
    TraceLaunch tr(CRL_TRACE_ENERGY, st, work);
    // one launch per objective kind present (the agents of one kind in a table of their own)
    int kinds = 0;
    for (const EnergyAgent& g : agents) kinds |= 1 << obj_kind(g.ls.loss);
    if (kinds == 1 << kObjInfo) {
      launch_bwd_multi(kObjInfo, dt, db, na, begin[na], bwd_smem(Rmax), st);
      return nullptr;
    }
    for (int kind = 0; kind <= kObjNCE; ++kind) {
      if (!(kinds & (1 << kind))) continue;
      std::vector<EnergyTask> sub;
      std::vector<int> sb(1, 0);
      for (int i = 0; i < na; ++i)
        if (obj_kind(agents[i].ls.loss) == kind) {
          sub.push_back(tasks[i]);
          sb.push_back(sb.back() + begin[i + 1] - begin[i]);
        }
      const EnergyTask* st_t = cache.get(sub, st, &err);
      if (!st_t) return err;
      const int* st_b = cache.get(sb, st, &err);
      if (!st_b) return err;
      launch_bwd_multi(kind, st_t, st_b, (int)sub.size(), sb.back(), bwd_smem(Rmax), st);
    }
  }
  return nullptr;
}

}  // namespace crl
