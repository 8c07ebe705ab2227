// Replay buffer insert and hindsight future-goal relabelling (Algorithm 1 of
// arXiv 2408.11052: "store the trajectory", then "sample with discount a batch
// of state-action pairs and goals from their future"; §3: the future offset is
// T ~ Geom(1 - gamma); §3.1/§3.2: goals come from the same trajectory).
//
// Layout: one ring of T rows per environment; a row holds the step's
// observation, action and the absolute index of the last step of its episode
// (see BufferDev in internal.h).  All environments insert in lockstep.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "philox.cuh"
#include "trace.h"

namespace crl {

// ---------------------------------------------------------------------------
// Insert n time slices in one launch, one warp per environment:
//  1. copy the environment's newest min(n, T) slices into their ring slots,
//     with the episode marked open (-1);
//  2. walk its n done flags in order and stamp every episode they close with
//     the absolute index of its last step (one episode's stamping is spread
//     over the lanes).
// The warp's own copies precede its stamps (__syncwarp orders them).  Block 0
// records the new fill.
// lb: block index within this buffer's share of the grid (4 environments per block).
__device__ __forceinline__ void insert_body(const InsertArgs& ia, int lb) {
  const BufferDev& bd = ia.bd;
  const float* __restrict__ obs = ia.obs;
  const float* __restrict__ act = ia.act;
  const uint8_t* __restrict__ done = ia.done;
  const int n = ia.n, i0 = ia.i0;
  const long long total_before = ia.total_before;
  const int lane = threadIdx.x % kWarp;
  const int e = lb * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  const long long total_after = total_before + n;
  const long long size_after = total_after < bd.T ? total_after : bd.T;
  if (lb == 0 && threadIdx.x == 0) {
    bd.state[0] = (int32_t)size_after;
    bd.state[1] = (int32_t)total_after;
  }
  if (e >= bd.E) return;
  for (int i = i0; i < n; ++i) {
    const long long abs_i = total_before + i;
    float* dst = bd.rows + ((size_t)e * bd.T + (size_t)(abs_i % bd.T)) * bd.W;
    const float* so = obs + ((size_t)i * bd.E + e) * bd.D;
    const float* sa = act + ((size_t)i * bd.E + e) * bd.A;
    for (int c = lane; c < bd.W; c += kWarp) {
      float v;
      if (c < bd.D) v = so[c];
      else if (c < bd.D + bd.A) v = sa[c - bd.D];
      else if (c == bd.D + bd.A) v = __int_as_float(-1);
      else v = 0.f;
      dst[c] = v;
    }
  }
  __syncwarp();
  const long long win_lo = total_after - size_after;
  long long start = bd.ep_start[e];
  for (int i = 0; i < n; ++i) {
    if (done[(size_t)i * bd.E + e]) {
      const long long last = total_before + i;
      const long long lo = start > win_lo ? start : win_lo;
      for (long long a = lo + lane; a <= last; a += kWarp)
        bd.rows[((size_t)e * bd.T + (size_t)(a % bd.T)) * bd.W + bd.D + bd.A] = __int_as_float((int)last);
      start = last + 1;
    }
  }
  if (lane == 0) bd.ep_start[e] = (int32_t)start;
}

__global__ void __launch_bounds__(128) insert_kernel(const __grid_constant__ InsertArgs ia) {
  pdl_enter();
  insert_body(ia, blockIdx.x);
}

// Several buffers (agents) in one launch; arguments by value (they change every step).
__global__ void __launch_bounds__(128) insert_multi_kernel(const __grid_constant__ InsertMulti m) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(m.begin, m.n, blockIdx.x, lb, nb);
  insert_body(m.a[s], lb);
}

int insert_blocks(const BufferDev& bd) { return ceil_div(bd.E, 4); }

void launch_buffer_insert_multi(const InsertMulti& m, cudaStream_t st) {
  double bytes = 0.0;
  for (int s = 0; s < m.n; ++s) {
    const InsertArgs& a = m.a[s];
    bytes += (double)(a.n - a.i0) * a.bd.E * ((a.bd.D + a.bd.A) * 4.0 + (a.bd.D + a.bd.A + 1) * 4.0) +
             (double)a.n * a.bd.E;
  }
  TraceLaunch tr(CRL_TRACE_INSERT, st, bytes);
  launch_k(insert_multi_kernel, dim3(m.begin[m.n]), dim3(128), 0, st, m);
}

void launch_buffer_insert(const BufferDev& bd, const float* obs, const float* act, const uint8_t* done,
                          int n, int64_t total_before, cudaStream_t st) {
  const int i0 = n > bd.T ? n - bd.T : 0;
  const long long rows = (long long)(n - i0) * bd.E;
  // algorithmic bytes: read obs, act and the done flags, write the rows (obs, act, episode end)
  TraceLaunch tr(CRL_TRACE_INSERT, st,
                 (double)rows * ((bd.D + bd.A) * 4.0 + (bd.D + bd.A + 1) * 4.0) + (double)n * bd.E);
  const InsertArgs ia{bd, obs, act, done, n, i0, total_before};
  launch_k(insert_kernel, dim3(insert_blocks(bd)), dim3(128), 0, st, ia);
}

// ---------------------------------------------------------------------------
// Discount table: G[0] = 2^32, G[k] = floor(G[k-1] * gq / 2^32), gq = round(gamma 2^32).
// G[k] ~ gamma^k 2^32 in exact integer arithmetic, so the inverse CDF below
// takes the same decision as any other implementation of the same rule.
void build_discount_table(float gamma, int n, unsigned long long* out) {
  const double scaled = (double)gamma * 4294967296.0;  // exact for a float gamma
  const unsigned long long gq = (unsigned long long)(scaled + 0.5);  // round half up (scaled >= 0)
  out[0] = 1ull << 32;
  for (int k = 1; k < n; ++k) {
    // (G * gq) < 2^64 because G <= 2^32 and gq < 2^32.
    out[k] = (out[k - 1] * gq) >> 32;
  }
}

// Smallest offset k in [m, L] with  v * (G0 - G[L+1-m]) < (G0 - G[k+1-m]) * 2^32,
// i.e. the inverse CDF of the geometric distribution truncated to the episode.
// The right side reaches 2^64 only when G[k+1-m] == 0, where the test is true.
__device__ __forceinline__ int geometric_offset(unsigned long long v, int L, int m,
                                                const unsigned long long* __restrict__ gq) {
  if (L == 0 && m == 1) return 0;
  const unsigned long long g0 = gq[0];
  const unsigned long long lhs = v * (g0 - __ldg(gq + L + 1 - m));
  int lo = m, hi = L;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const unsigned long long gk = __ldg(gq + mid + 1 - m);
    const bool ok = (gk == 0ull) || (lhs < ((g0 - gk) << 32));
    if (ok) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Indices of sample b from Philox4x64-10 block (step, b, 0, 0): the
// transition (e, t), t counted from the oldest stored step, uniform over the
// E x size stored steps (word 0), and the offset k from the geometric
// distribution truncated to the episode (top half of word 1).
__device__ __forceinline__ void sample_indices(const BufferDev& bd, const RelabelArgs& ra, unsigned long long step,
                                               int b, int size, long long total, int& e, int& t, int& k) {
  const Philox4 r = philox4x64_10(step, (unsigned long long)b, 0ull, 0ull, ra.seed, ra.agent);
  const unsigned long long nstored = (unsigned long long)size * (unsigned long long)bd.E;
  const unsigned long long idx = __umul64hi(r.w[0], nstored);
  e = (int)(idx / (unsigned long long)size);
  t = (int)(idx % (unsigned long long)size);
  const long long abs_t = total - size + t;
  const float* row = bd.rows + ((size_t)e * bd.T + (size_t)(abs_t % bd.T)) * bd.W;
  const int ep_end = __float_as_int(row[bd.D + bd.A]);
  int L = (ep_end < 0) ? (size - 1 - t) : (int)(ep_end - abs_t);
  if (L < 0 || L > size - 1 - t) {
    atomicOr(ra.status, CRL_STATUS_BAD_INDEX);
    L = L < 0 ? 0 : size - 1 - t;
  }
  k = geometric_offset(r.w[1] >> 32, L, ra.offset_min, bd.gq);
}

#ifndef CRL_RELABEL_UNROLL
#define CRL_RELABEL_UNROLL 2
#endif
constexpr int kRelabelUnroll = CRL_RELABEL_UNROLL;  // samples whose loads are in flight together

// One warp per ra.spw consecutive samples (1..32).  Phase 1: lane j < spw
// draws the indices of sample b0 + j (independent Philox / episode-end /
// inverse-CDF chains side by side).  Phase 2: the warp copies each sample's
// state-action row with 16-byte loads (ring rows start on 16-byte boundaries)
// and gathers its goal dims.  Small batches take spw = 1 (a warp per sample,
// the most parallel copy); large ones up to 32 (index chains 32 wide).
// lb: block index within this sample batch's share of the grid (8 warps per block).
__device__ __forceinline__ void relabel_body(const BufferDev& bd, const RelabelArgs& ra, int lb) {
  const int lane = threadIdx.x % kWarp;
  const int spw = ra.spw;
  const int b0 = (lb * (blockDim.x / kWarp) + threadIdx.x / kWarp) * spw;
  const unsigned long long step = (ra.step == CRL_STEP_AUTO) ? *ra.step_dev : ra.step;
  if (lb == 0 && threadIdx.x == 0 && ra.last_step_dev != nullptr) *ra.last_step_dev = step;
  if (b0 >= ra.B) return;
  const int size = bd.state[0];
  const long long total = bd.state[1];
  if (size <= 0) {
    if (lane == 0) atomicOr(ra.status, CRL_STATUS_BAD_INDEX);
    return;
  }
  const int b = b0 + lane;
  int e = 0, t = 0, k = 0;
  if (lane < spw && b < ra.B) {
    sample_indices(bd, ra, step, b, size, total, e, t, k);
    if (ra.idx != nullptr) {
      ra.idx[3 * (size_t)b + 0] = e;
      ra.idx[3 * (size_t)b + 1] = t;
      ra.idx[3 * (size_t)b + 2] = k;
    }
  }
  const int nb = min(spw, ra.B - b0);
  const int D = bd.D, DA = bd.D + bd.A;
  const int nv = (DA + 3) / 4;          // float4 chunks over obs + act (the tail chunk may hold ep_end / pad)
  const bool s_vec = (D % 4) == 0;      // s rows 16-byte aligned
  const bool packs = ra.pack[0].x0 || ra.pack[1].x0 || ra.pack[2].x0;
  if (!packs && nv <= 4 * kWarp) {
    // kRelabelUnroll samples at a time: every load of the group issues before any store
    constexpr int U = kRelabelUnroll;
    for (int j0 = 0; j0 < nb; j0 += U) {
      float4 v[U][4];
      float gv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = min(j0 + u, nb - 1);
        const int ej = __shfl_sync(0xffffffffu, e, j);
        const int tj = __shfl_sync(0xffffffffu, t, j);
        const int kj = __shfl_sync(0xffffffffu, k, j);
        const long long abs_t = total - size + tj;
        const float* row = bd.rows + ((size_t)ej * bd.T + (size_t)(abs_t % bd.T)) * bd.W;
        const float* grow = bd.rows + ((size_t)ej * bd.T + (size_t)((abs_t + kj) % bd.T)) * bd.W;
        const bool live = j0 + u < nb;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int q = lane + kWarp * r;
          if (live && q < nv) v[u][r] = __ldcs(reinterpret_cast<const float4*>(row) + q);
        }
        gv[u] = (live && lane < ra.G) ? grow[ra.goal_idx[lane]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j0 + u >= nb) break;
        const int bj = b0 + j0 + u;
        float* srow = ra.s + (size_t)bj * D;
        float* arow = ra.a + (size_t)bj * bd.A;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int q = lane + kWarp * r;
          if (q >= nv) break;
          const int c = 4 * q;
          if (s_vec && c + 3 < D) {
            __stcs(reinterpret_cast<float4*>(srow + c), v[u][r]);
          } else {
            const float x[4] = {v[u][r].x, v[u][r].y, v[u][r].z, v[u][r].w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int ci = c + i;
              if (ci < D) __stcs(srow + ci, x[i]);
              else if (ci < DA) __stcs(arow + ci - D, x[i]);
            }
          }
        }
        if (lane < ra.G) __stcs(ra.g + (size_t)bj * ra.G + lane, gv[u]);
      }
    }
    return;
  }
  for (int j = 0; j < nb; ++j) {
    const int ej = __shfl_sync(0xffffffffu, e, j);
    const int tj = __shfl_sync(0xffffffffu, t, j);
    const int kj = __shfl_sync(0xffffffffu, k, j);
    const int bj = b0 + j;
    const long long abs_t = total - size + tj;
    const float* row = bd.rows + ((size_t)ej * bd.T + (size_t)(abs_t % bd.T)) * bd.W;
    const float* grow = bd.rows + ((size_t)ej * bd.T + (size_t)((abs_t + kj) % bd.T)) * bd.W;
    float* srow = ra.s + (size_t)bj * D;
    float* arow = ra.a + (size_t)bj * bd.A;
    for (int q = lane; q < nv; q += kWarp) {
      const float4 v = *reinterpret_cast<const float4*>(row + 4 * q);
      const int c = 4 * q;
      if (s_vec && c + 3 < D) {
        *reinterpret_cast<float4*>(srow + c) = v;
      } else {
        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int ci = c + i;
          if (ci < D) srow[ci] = x[i];
          else if (ci < DA) arow[ci - D] = x[i];
        }
      }
    }
    if (lane < ra.G) ra.g[(size_t)bj * ra.G + lane] = grow[ra.goal_idx[lane]];
    // BF16 split packs of the network inputs (hi, lo interleaved)
    for (int kk = 0; kk < 3; ++kk) {
      const RelabelPack& pk = ra.pack[kk];
      if (pk.x0 == nullptr) continue;
      const int ncol = (kk == 0) ? DA : (kk == 1 ? ra.G : D + ra.G);
      __nv_bfloat16* x0 = static_cast<__nv_bfloat16*>(pk.x0);
      for (int c = lane; c < ncol; c += kWarp) {
        float v;
        if (kk == 0) v = row[c];
        else if (kk == 1) v = grow[ra.goal_idx[c]];
        else v = c < D ? row[c] : grow[ra.goal_idx[c - D]];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        x0[(size_t)bj * pk.ld + 2 * c] = hi;
        x0[(size_t)bj * pk.ld + 2 * c + 1] = lo;
      }
    }
  }
}

// Columns of pack k of a relabelled sample: phi (s, a), psi (g), pi (s, g).
__device__ __host__ __forceinline__ int pack_cols(int k, int D, int A, int G) {
  return k == 0 ? D + A : (k == 1 ? G : D + G);
}

// Relabel with the BF16 network-input packs (the update step): a block of 32
// warps takes 32 consecutive samples, one per warp (lane 0 draws the indices,
// the warp copies the row and writes its sample's split inputs row-major).
__device__ __forceinline__ void relabel_pack_body(const BufferDev& bd, const RelabelArgs& ra, int lb) {
  const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
  const int b0 = lb * kWarp;
  const int b = b0 + w;
  const unsigned long long step = (ra.step == CRL_STEP_AUTO) ? *ra.step_dev : ra.step;
  if (lb == 0 && threadIdx.x == 0 && ra.last_step_dev != nullptr) *ra.last_step_dev = step;
  const int size = bd.state[0];
  const long long total = bd.state[1];
  if (size <= 0) {
    if (threadIdx.x == 0) atomicOr(ra.status, CRL_STATUS_BAD_INDEX);
    return;
  }
  const int D = bd.D, DA = bd.D + bd.A;
  if (b < ra.B) {
    int e = 0, t = 0, k = 0;
    if (lane == 0) {
      sample_indices(bd, ra, step, b, size, total, e, t, k);
      if (ra.idx != nullptr) {
        ra.idx[3 * (size_t)b + 0] = e;
        ra.idx[3 * (size_t)b + 1] = t;
        ra.idx[3 * (size_t)b + 2] = k;
      }
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    t = __shfl_sync(0xffffffffu, t, 0);
    k = __shfl_sync(0xffffffffu, k, 0);
    const long long abs_t = total - size + t;
    const float* row = bd.rows + ((size_t)e * bd.T + (size_t)(abs_t % bd.T)) * bd.W;
    const float* grow = bd.rows + ((size_t)e * bd.T + (size_t)((abs_t + k) % bd.T)) * bd.W;
    for (int c = lane; c < DA; c += kWarp) {
      const float v = row[c];
      if (c < D) ra.s[(size_t)b * D + c] = v;
      else ra.a[(size_t)b * bd.A + (c - D)] = v;
    }
    if (lane < ra.G) ra.g[(size_t)b * ra.G + lane] = grow[ra.goal_idx[lane]];
    for (int kk = 0; kk < 3; ++kk) {
      const RelabelPack& pk = ra.pack[kk];
      if (pk.x0 == nullptr) continue;
      const int ncol = pack_cols(kk, D, bd.A, ra.G);
      __nv_bfloat16* x0 = static_cast<__nv_bfloat16*>(pk.x0);
      for (int c = lane; c < ncol; c += kWarp) {
        float v;
        if (kk == 0) v = row[c];
        else if (kk == 1) v = grow[ra.goal_idx[c]];
        else v = c < D ? row[c] : grow[ra.goal_idx[c - D]];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        x0[(size_t)b * pk.ld + 2 * c] = hi;
        x0[(size_t)b * pk.ld + 2 * c + 1] = lo;
      }
    }
  }
}

__global__ void __launch_bounds__(1024) relabel_pack_kernel(const __grid_constant__ BufferDev bd,
                                                           const __grid_constant__ RelabelArgs ra) {
  pdl_enter();
  relabel_pack_body(bd, ra, blockIdx.x);
}

__global__ void __launch_bounds__(1024) relabel_pack_multi_kernel(const RelabelTask* __restrict__ tasks,
                                                                 const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(begin, n, blockIdx.x, lb, nb);
  relabel_pack_body(tasks[s].bd, tasks[s].ra, lb);
}

__global__ void __launch_bounds__(256) relabel_kernel(const __grid_constant__ BufferDev bd,
                                                     const __grid_constant__ RelabelArgs ra) {
  pdl_enter();
  relabel_body(bd, ra, blockIdx.x);
}

// Several agents' batches in one launch (per-agent arguments in an immutable device table).
__global__ void __launch_bounds__(256) relabel_multi_kernel(const RelabelTask* __restrict__ tasks,
                                                           const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(begin, n, blockIdx.x, lb, nb);
  relabel_body(tasks[s].bd, tasks[s].ra, lb);
}

int relabel_spw(int B) { return (int)std::min<long long>(32, std::max<long long>(1, (long long)B / (152 * 48))); }
bool relabel_packs(const RelabelArgs& ra) { return ra.pack[0].x0 || ra.pack[1].x0 || ra.pack[2].x0; }
int relabel_blocks(const RelabelArgs& ra) {
  return relabel_packs(ra) ? ceil_div(ra.B, kWarp) : ceil_div(ra.B, 8 * ra.spw);
}

void launch_relabel_multi(const RelabelTask* tasks, const int* begin, int n, int blocks, double bytes, bool packs,
                          size_t smem, cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_RELABEL, st, bytes);
  if (packs) {
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
      cudaFuncSetAttribute(relabel_pack_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = smem;
    }
    launch_k(relabel_pack_multi_kernel, dim3(blocks), dim3(1024), smem, st, tasks, begin, n);
  } else {
    launch_k(relabel_multi_kernel, dim3(blocks), dim3(256), 0, st, tasks, begin, n);
  }
}

void launch_relabel(const BufferDev& bd, const RelabelArgs& ra, cudaStream_t st) {
  // algorithmic bytes per sample: read obs + act + episode end + goal dims, write s, a, g (+ idx)
  const double per = (bd.D + bd.A + 1 + ra.G) * 4.0 + (bd.D + bd.A + ra.G) * 4.0 + (ra.idx ? 12.0 : 0.0);
  TraceLaunch tr(CRL_TRACE_RELABEL, st, per * ra.B);
  // samples per warp: as many warps as fill the GPU (152 SMs x 48 resident warps), at most 32
  RelabelArgs r = ra;
  r.spw = relabel_spw(ra.B);
  if (relabel_packs(r)) {
    launch_k(relabel_pack_kernel, dim3(relabel_blocks(r)), dim3(1024), 0, st, bd, r);
  } else {
    launch_k(relabel_kernel, dim3(relabel_blocks(r)), dim3(256), 0, st, bd, r);
  }
}

__global__ void bump_u64_kernel(unsigned long long* c) {
  pdl_enter();
  *c += 1ull;
}

// Random-goal actor mix (App. D): sample b takes the goal of sample (b + 1) mod B
// when the top half of word 2 of its relabel Philox block falls below thr.
__global__ void __launch_bounds__(256) actor_goals_kernel(int B, int G, const float* __restrict__ g,
                                                         float* __restrict__ g_act, unsigned long long seed,
                                                         unsigned long long agent,
                                                         const unsigned long long* __restrict__ step_dev,
                                                         unsigned long long thr) {
  pdl_enter();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Philox4 r = philox4x64_10(*step_dev, (unsigned long long)b, 0ull, 0ull, seed, agent);
  const int src = ((r.w[2] >> 32) < thr) ? (b + 1 == B ? 0 : b + 1) : b;
  for (int c = 0; c < G; ++c) g_act[(size_t)b * G + c] = g[(size_t)src * G + c];
}

void launch_actor_goals(int B, int G, const float* g, float* g_act, uint64_t seed, uint64_t agent,
                        const unsigned long long* step_dev, float alpha_rg, cudaStream_t st) {
  // floor(alpha_rg 2^32), exact for a float alpha_rg in [0, 1]
  const unsigned long long thr = (unsigned long long)std::floor((double)alpha_rg * 4294967296.0);
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)B * G * 8.0);
  launch_k(actor_goals_kernel, dim3(ceil_div(B, 256)), dim3(256), 0, st, B, G, g, g_act,
           (unsigned long long)seed, (unsigned long long)agent, step_dev, thr);
}

void launch_bump_u64(unsigned long long* ctr, cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_AUX, st, 8.0);
  launch_k(bump_u64_kernel, dim3(1), dim3(1), 0, st, ctr);
}

}  // namespace crl
