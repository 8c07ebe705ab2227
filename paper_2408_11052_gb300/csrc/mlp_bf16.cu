// BF16 tensor-core MLP forward / backward (see mlp_bf16.cuh for the scheme).
//
// Networks of arXiv 2408.11052: phi(s, a) and psi(g) (§3.1), the policy
// (§3.2); hidden [256, 256] / repr 64 (App. B.3); LayerNorm before every
// activation for the large networks (§5.4).  Readings M1-M3 as in the FP32
// path: ReLU, LayerNorm (eps 1e-6, biased variance, affine) between Linear and
// ReLU, W stored [out][in].
#include <cuda_bf16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "actor_head.cuh"
#include "common.cuh"
#include "mlp_bf16.cuh"
#include "tc_gemm.cuh"
#include "tc_host.h"
#include "trace.h"

namespace crl {

using bf16 = __nv_bfloat16;

int list_split(const std::vector<tc::GemmProblem>& probs);

namespace {

constexpr float kLnEpsF = 1e-6f;

inline int pad8(int x) { return (x + 7) / 8 * 8; }

// ---- element kernels ----------------------------------------------------------------
// 32 x 32 tile transpose-and-pack: src = concat(s0 [rows][n0], s1 [rows][n1]) (FP32)
// -> dst [rows][ld] (BF16, optional) and dstT [n0 + n1][ldt] (BF16, optional).
__global__ void __launch_bounds__(256) pack_kernel(int rows, const float* __restrict__ s0, int ld0, int n0,
                                                  const float* __restrict__ s1, int ld1, int n1, bf16* __restrict__ dst,
                                                  int ld, bf16* __restrict__ dstT, int ldt) {
  pdl_enter();
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int ncol = n0 + n1;
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float v = 0.f;
    if (row < rows && col < ncol) v = col < n0 ? s0[(size_t)row * ld0 + col] : s1[(size_t)row * ld1 + (col - n0)];
    tile[r][tx] = v;
    if (dst && row < rows && col < ncol) dst[(size_t)row * ld + col] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  if (dstT) {
    for (int c = ty; c < 32; c += 8) {
      const int col = c0 + c, row = r0 + tx;
      if (col < ncol && row < rows) dstT[(size_t)col * ldt + row] = __float2bfloat16_rn(tile[tx][c]);
    }
  }
}

// Split pack of the network input: x = concat(s0, s1) [rows][ncol] (FP32) ->
// dst [rows][ld] = (hi_0, lo_0, hi_1, lo_1, ...) and dstT [2 ncol][ldt], with
// hi = bf16(x), lo = bf16(x - hi).
__global__ void __launch_bounds__(256) pack_split_kernel(int rows, const float* __restrict__ s0, int ld0, int n0,
                                                        const float* __restrict__ s1, int ld1, int n1,
                                                        bf16* __restrict__ dst, int ld, bf16* __restrict__ dstT,
                                                        int ldt) {
  pdl_enter();
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int ncol = n0 + n1;
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float v = 0.f;
    if (row < rows && col < ncol) v = col < n0 ? s0[(size_t)row * ld0 + col] : s1[(size_t)row * ld1 + (col - n0)];
    tile[r][tx] = v;
    if (row < rows && col < ncol) {
      const bf16 hi = __float2bfloat16_rn(v);
      const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      dst[(size_t)row * ld + 2 * col] = hi;
      dst[(size_t)row * ld + 2 * col + 1] = lo;
    }
  }
  __syncthreads();
  if (!dstT) return;
  for (int c = ty; c < 32; c += 8) {
    const int col = c0 + c, row = r0 + tx;
    if (col < ncol && row < rows) {
      const float v = tile[tx][c];
      const bf16 hi = __float2bfloat16_rn(v);
      dstT[(size_t)(2 * col) * ldt + row] = hi;
      dstT[(size_t)(2 * col + 1) * ldt + row] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
}

// Weight shadows: W [out][ncol] (FP32) -> W2 [out][(nhi + 1) kp] = nhi copies
// of W_hi, then W_lo, with hi = bf16(w), lo = bf16(w - hi), each column written
// `rep` times (first layer: rep = 2 matching the split input, nhi = 1; later
// layers: rep = 1, nhi = 2 for the hi / lo activations), and the single BF16
// transpose Wt [ncol][ldt] for the input-gradient product.
__global__ void __launch_bounds__(256) pack_weights_kernel(int rows, int ncol, int rep, int nhi,
                                                          const float* __restrict__ W, bf16* __restrict__ W2, int kp,
                                                          bf16* __restrict__ Wt, int ldt) {
  pdl_enter();
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int r = ty; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + tx;
    float v = 0.f;
    if (row < rows && col < ncol) {
      v = W[(size_t)row * ncol + col];
      const bf16 hi = __float2bfloat16_rn(v);
      const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      bf16* d = W2 + (size_t)row * (nhi + 1) * kp;
      for (int q = 0; q < rep; ++q) {
        for (int c = 0; c < nhi; ++c) d[c * kp + rep * col + q] = hi;
        d[nhi * kp + rep * col + q] = lo;
      }
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int c = ty; c < 32; c += 8) {
    const int col = c0 + c, row = r0 + tx;
    if (col < ncol && row < rows) Wt[(size_t)col * ldt + row] = __float2bfloat16_rn(tile[tx][c]);
  }
}

void pack(int rows, const float* s0, int ld0, int n0, const float* s1, int ld1, int n1, bf16* dst, int ld, bf16* dstT,
          int ldt, cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)rows * (n0 + n1) * (4.0 + (dst ? 2 : 0) + (dstT ? 2 : 0)));
  dim3 grid(ceil_div(n0 + n1, 32), ceil_div(rows, 32));
  launch_k(pack_kernel, grid, dim3(256), 0, st, rows, s0, ld0, n0, s1, ld1, n1, dst, ld, dstT, ldt);
}

// LayerNorm kernels: one warp per row, 8 rows per 256-thread block.  Rows of
// up to 1024 values stay in registers (float4 pieces, lane-strided), so the
// statistics and the output take one pass over global memory; wider rows loop
// over global memory.
constexpr int kLnRows = 8;
constexpr int kLnRegVec = 8;   // float4 pieces per lane held in registers (H <= 1024)
constexpr int kLnMaxSmem = 200 * 1024;
inline int ln_vec(int H) { return (H + 127) / 128 <= kLnRegVec ? (H + 127) / 128 : 0; }
// The backward's register path stages the rows' du zhat and du ([2][8][H] FP32)
// for the column sums.
inline size_t ln_bwd_smem_bytes(int H) { return ln_vec(H) > 0 ? (size_t)2 * kLnRows * H * 4 : 0; }
// LayerNorm parameter gradients: every backward block writes its rows' column
// sums of du zhat and du ([nblk][2][H] per layer); one launch after the
// input-gradient chain adds them in block order (deterministic).
inline size_t ln_partial_floats(int Mmax, int H, int layers) {
  const int nblk = (Mmax + kLnRows - 1) / kLnRows;
  return (size_t)layers * nblk * 2 * H;
}

struct LnFwdNet {
  int M;
  float* z;
  float* rstd;
  const float* g;
  const float* beta;
  bf16* h;      // [M][ldh]: hi part in columns [0, H), lo part in [hlo, hlo + H)
  int ldh, hlo;
};
struct LnFwdGroup {
  LnFwdNet n[kMaxGroupNets];
};

// ReLU(x * g + b) of four features as BF16 hi parts (returned) and BF16 lo
// parts bf16(v - hi) (in lo).
__device__ __forceinline__ uint2 ln_relu_pack(float4 x, float4 gg, float4 bb, uint2& lo) {
  const float v0 = fmaxf(x.x * gg.x + bb.x, 0.f), v1 = fmaxf(x.y * gg.y + bb.y, 0.f);
  const float v2 = fmaxf(x.z * gg.z + bb.z, 0.f), v3 = fmaxf(x.w * gg.w + bb.w, 0.f);
  const __nv_bfloat162 p0 = __floats2bfloat162_rn(v0, v1);
  const __nv_bfloat162 p1 = __floats2bfloat162_rn(v2, v3);
  const __nv_bfloat162 q0 = __floats2bfloat162_rn(v0 - __low2float(p0), v1 - __high2float(p0));
  const __nv_bfloat162 q1 = __floats2bfloat162_rn(v2 - __low2float(p1), v3 - __high2float(p1));
  lo = make_uint2(*reinterpret_cast<const uint32_t*>(&q0), *reinterpret_cast<const uint32_t*>(&q1));
  return make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
}

// LayerNorm forward over rows of z [M][H] (FP32, replaced by zhat), rstd [M],
// h = ReLU(zhat * g + beta) written as BF16 hi / lo parts [M][ldh].
// NV > 0: the row in registers (NV float4 per lane); NV = 0: three passes.
template <int NV>
__global__ void __launch_bounds__(256) ln_fwd_kernel(int H, const __grid_constant__ LnFwdGroup grp) {
  pdl_enter();
  const LnFwdNet& a = grp.n[blockIdx.y];
  const int M = a.M;
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int row0 = blockIdx.x * kLnRows;
  if (row0 >= M) return;
  const int nv = H / 4;
  const int row = row0 + w;
  if (row < M) {
    float4* zr = reinterpret_cast<float4*>(a.z + (size_t)row * H);
    const float4* g4 = reinterpret_cast<const float4*>(a.g);
    const float4* b4 = reinterpret_cast<const float4*>(a.beta);
    uint2* hr = reinterpret_cast<uint2*>(a.h + (size_t)row * a.ldh);
    uint2* hl = reinterpret_cast<uint2*>(a.h + (size_t)row * a.ldh + a.hlo);
    if constexpr (NV > 0) {
      float4 x[NV];
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int q = lane + 32 * j;
        x[j] = q < nv ? zr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        s += (x[j].x + x[j].y) + (x[j].z + x[j].w);
      }
      const float mean = warp_sum(s) / H;
      float sq = 0.f;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        if (lane + 32 * j >= nv) continue;
        const float d0 = x[j].x - mean, d1 = x[j].y - mean, d2 = x[j].z - mean, d3 = x[j].w - mean;
        sq += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
      }
      const float rs = rsqrtf(warp_sum(sq) / H + kLnEpsF);
      if (lane == 0) a.rstd[row] = rs;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int q = lane + 32 * j;
        if (q >= nv) continue;
        float4 xn;
        xn.x = (x[j].x - mean) * rs;
        xn.y = (x[j].y - mean) * rs;
        xn.z = (x[j].z - mean) * rs;
        xn.w = (x[j].w - mean) * rs;
        zr[q] = xn;
        uint2 lo;
        hr[q] = ln_relu_pack(xn, g4[q], b4[q], lo);
        hl[q] = lo;
      }
    } else {
      float s = 0.f;
      for (int q = lane; q < nv; q += 32) {
        const float4 x = zr[q];
        s += (x.x + x.y) + (x.z + x.w);
      }
      const float mean = warp_sum(s) / H;
      float sq = 0.f;
      for (int q = lane; q < nv; q += 32) {
        const float4 x = zr[q];
        const float d0 = x.x - mean, d1 = x.y - mean, d2 = x.z - mean, d3 = x.w - mean;
        sq += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
      }
      const float rs = rsqrtf(warp_sum(sq) / H + kLnEpsF);
      if (lane == 0) a.rstd[row] = rs;
      for (int q = lane; q < nv; q += 32) {
        float4 x = zr[q];
        x.x = (x.x - mean) * rs;
        x.y = (x.y - mean) * rs;
        x.z = (x.z - mean) * rs;
        x.w = (x.w - mean) * rs;
        zr[q] = x;
        uint2 lo;
        hr[q] = ln_relu_pack(x, g4[q], b4[q], lo);
        hl[q] = lo;
      }
    }
  }
}

struct LnBwdNet {
  int M;
  const float* du;
  const float* zhat;
  const float* rstd;
  const float* g;
  bf16* dz;
  float* partial;     // null: no LayerNorm parameter gradients; else [nblk][2][H] per-block column sums
};
struct LnBwdGroup {
  LnBwdNet n[kMaxGroupNets];
};

__device__ __forceinline__ uint2 ln_bwd_pack(float4 d, float4 z, float4 gg, float s1, float s2, float rs) {
  const __nv_bfloat162 p0 =
      __floats2bfloat162_rn(rs * (d.x * gg.x - s1 - z.x * s2), rs * (d.y * gg.y - s1 - z.y * s2));
  const __nv_bfloat162 p1 =
      __floats2bfloat162_rn(rs * (d.z * gg.z - s1 - z.z * s2), rs * (d.w * gg.w - s1 - z.w * s2));
  return make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
}

// LayerNorm backward: du (ReLU-masked, FP32) -> dz = rstd (g du - mean(g du) -
// zhat mean(g du zhat)), written BF16 [M][H]; with `partial` every block also
// writes its 8 rows' column sums of du zhat and du (for dg, db; added by
// ln_param_reduce_kernel).  NV as in the forward.
template <int NV>
__global__ void __launch_bounds__(256) ln_bwd_kernel(int H, const __grid_constant__ LnBwdGroup grp) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char ln_smem[];
  // register path: [2][8][H] FP32 (du zhat, du) of the block's rows
  float* colbuf = reinterpret_cast<float*>(ln_smem);
  const LnBwdNet& a = grp.n[blockIdx.y];
  const int M = a.M;
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int row0 = blockIdx.x * kLnRows;
  if (row0 >= M) return;
  const int nv = H / 4;
  const float4* g4 = reinterpret_cast<const float4*>(a.g);
  const int row = row0 + w;
  if (row < M) {
    const float4* dr = reinterpret_cast<const float4*>(a.du + (size_t)row * H);
    const float4* zr = reinterpret_cast<const float4*>(a.zhat + (size_t)row * H);
    const float rs = a.rstd[row];
    uint2* out = reinterpret_cast<uint2*>(a.dz + (size_t)row * H);
    if constexpr (NV > 0) {
      float4 d[NV], z[NV];
      float s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int q = lane + 32 * j;
        if (q < nv) {
          d[j] = dr[q];
          z[j] = zr[q];
          const float4 gg = g4[q];
          const float e0 = d[j].x * gg.x, e1 = d[j].y * gg.y, e2 = d[j].z * gg.z, e3 = d[j].w * gg.w;
          s1 += (e0 + e1) + (e2 + e3);
          s2 += (e0 * z[j].x + e1 * z[j].y) + (e2 * z[j].z + e3 * z[j].w);
        }
      }
      s1 = warp_sum(s1) / H;
      s2 = warp_sum(s2) / H;
      float4* cz = reinterpret_cast<float4*>(colbuf + (size_t)w * H);
      float4* cd = reinterpret_cast<float4*>(colbuf + (size_t)(kLnRows + w) * H);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const int q = lane + 32 * j;
        if (q >= nv) continue;
        out[q] = ln_bwd_pack(d[j], z[j], g4[q], s1, s2, rs);
        if (a.partial != nullptr) {
          cz[q] = make_float4(d[j].x * z[j].x, d[j].y * z[j].y, d[j].z * z[j].z, d[j].w * z[j].w);
          cd[q] = d[j];
        }
      }
    } else {
      float s1 = 0.f, s2 = 0.f;
      for (int q = lane; q < nv; q += 32) {
        const float4 dd = dr[q], zz = zr[q], gg = g4[q];
        const float e0 = dd.x * gg.x, e1 = dd.y * gg.y, e2 = dd.z * gg.z, e3 = dd.w * gg.w;
        s1 += (e0 + e1) + (e2 + e3);
        s2 += (e0 * zz.x + e1 * zz.y) + (e2 * zz.z + e3 * zz.w);
      }
      s1 = warp_sum(s1) / H;
      s2 = warp_sum(s2) / H;
      for (int q = lane; q < nv; q += 32) {
        out[q] = ln_bwd_pack(dr[q], zr[q], g4[q], s1, s2, rs);
      }
    }
  }
  if (a.partial == nullptr) return;
  __syncthreads();
  // column sums of this block's rows (rows in order)
  const int rmax = min(kLnRows, M - row0);
  for (int c = threadIdx.x; c < H; c += blockDim.x) {
    float sg = 0.f, sb = 0.f;
    if constexpr (NV > 0) {
#pragma unroll
      for (int r = 0; r < kLnRows; ++r) {
        if (r >= rmax) break;
        sg += colbuf[(size_t)r * H + c];
        sb += colbuf[(size_t)(kLnRows + r) * H + c];
      }
    } else {
#pragma unroll
      for (int r = 0; r < kLnRows; ++r) {
        if (r >= rmax) break;
        const size_t o = (size_t)(row0 + r) * H + c;
        const float dv = a.du[o];
        sg += dv * a.zhat[o];
        sb += dv;
      }
    }
    a.partial[((size_t)blockIdx.x * 2 + 0) * H + c] = sg;
    a.partial[((size_t)blockIdx.x * 2 + 1) * H + c] = sb;
  }
}

// dg = sum over the blocks of their du zhat column sums, db likewise, in a
// fixed order: one item per (network, LayerNorm layer) with gradients.
struct LnReduceItem {
  const float* partial;   // [nblk][2][H]
  float* dg;
  float* db;
  int nblk;
};
constexpr int kMaxLnReduce = 64;
struct LnReduceGroup {
  LnReduceItem it[kMaxLnReduce];
};
// A block takes 32 columns; its 8 warps add consecutive eighths of the block
// sums, then warp 0 adds the 8 results in order.
__global__ void __launch_bounds__(256) ln_param_reduce_kernel(int H, const __grid_constant__ LnReduceGroup grp) {
  pdl_enter();
  __shared__ float red[2][8][32];
  const LnReduceItem& t = grp.it[blockIdx.y];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int c = blockIdx.x * 32 + lane;
  const int per = (t.nblk + 7) / 8, k0 = w * per, k1 = min(t.nblk, k0 + per);
  float sg = 0.f, sb = 0.f;
  if (c < H) {
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      sg += t.partial[((size_t)k * 2 + 0) * H + c];
      sb += t.partial[((size_t)k * 2 + 1) * H + c];
    }
  }
  red[0][w][lane] = sg;
  red[1][w][lane] = sb;
  __syncthreads();
  if (w == 0 && c < H) {
    float g = 0.f, b = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      g += red[0][j][lane];
      b += red[1][j][lane];
    }
    t.dg[c] = g;
    t.db[c] = b;
  }
}

// LayerNorm launches with the register width chosen from H.
template <int NV>
void launch_ln_fwd_t(int H, dim3 grid, cudaStream_t st, const LnFwdGroup& grp) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ln_fwd_kernel<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLnMaxSmem);
    attr = true;
  }
  launch_k(ln_fwd_kernel<NV>, grid, dim3(256), 0, st, H, grp);
}
template <int NV>
void launch_ln_bwd_t(int H, dim3 grid, cudaStream_t st, const LnBwdGroup& grp) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ln_bwd_kernel<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLnMaxSmem);
    attr = true;
  }
  launch_k(ln_bwd_kernel<NV>, grid, dim3(256), ln_bwd_smem_bytes(H), st, H, grp);
}
#define CRL_LN_DISPATCH(FN)                    \
  switch (ln_vec(H)) {                         \
    case 1: FN<1>(H, grid, st, grp); break;    \
    case 2: FN<2>(H, grid, st, grp); break;    \
    case 3: FN<3>(H, grid, st, grp); break;    \
    case 4: FN<4>(H, grid, st, grp); break;    \
    case 5: FN<5>(H, grid, st, grp); break;    \
    case 6: FN<6>(H, grid, st, grp); break;    \
    case 7: FN<7>(H, grid, st, grp); break;    \
    case 8: FN<8>(H, grid, st, grp); break;    \
    default: FN<0>(H, grid, st, grp); break;   \
  }
void launch_ln_fwd(int H, dim3 grid, cudaStream_t st, const LnFwdGroup& grp) { CRL_LN_DISPATCH(launch_ln_fwd_t) }
void launch_ln_bwd(int H, dim3 grid, cudaStream_t st, const LnBwdGroup& grp) { CRL_LN_DISPATCH(launch_ln_bwd_t) }
#undef CRL_LN_DISPATCH

// One column of a row-major BF16 matrix: p[r * ld] = v for r < rows.
__global__ void fill_col_bf16_kernel(bf16* p, int rows, int ld, float v) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x)
    p[(size_t)r * ld] = __float2bfloat16_rn(v);
}

const char* mk(CUtensorMap* m, const void* base, int inner, int rows, int stride) {
  const char* err = nullptr;
  if (!tc::make_tmap_bf16(m, base, (uint64_t)inner, (uint64_t)rows, (uint64_t)stride, 64, &err)) return err;
  return nullptr;
}



uint64_t fnv1a(const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

tc::EpiDesc epi_of(int kind) {
  tc::EpiDesc e;
  memset(&e, 0, sizeof(e));
  e.kind = kind;
  return e;
}

tc::GemmProblem problem(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, int nkA,
                        const tc::EpiDesc& e) {
  tc::GemmProblem p;
  memset(&p, 0, sizeof(p));
  p.a = a;
  p.b = b;
  p.M = M;
  p.N = N;
  p.K = K;
  p.nkA = nkA;
  p.epi = e;
  return p;
}

template <int BN, int STAGES>
void launch_gemm_cfg(const tc::GemmProblem* table, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  using S = tc::GemmSmem<BN, STAGES>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::tc_gemm_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
    attr = true;
  }
  launch_k(tc::tc_gemm_kernel<BN, STAGES>, dim3(tiles), dim3(128), S::kBytes, st, table, nprob, status);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

template <int BN, int STAGES>
void launch_gemm_persistent(const tc::GemmProblem* table, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  using S = tc::GemmSmem<BN, STAGES>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::tc_gemm_persistent_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         S::kBytes);
    attr = true;
  }
  const int grid = std::min(tiles, sm_count());
  launch_k(tc::tc_gemm_persistent_kernel<BN, STAGES>, dim3(grid), dim3(192), S::kBytes, st, table, nprob, tiles,
           status);
}

// CTA-pair kernel: clusters of two CTAs, one cluster per pair of SMs at most
// (as many as can be resident at once), walking the 256-row tiles.
int pair_clusters_max(const void* kernel, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * 64);
  cfg.blockDim = dim3(224);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = sm_count() / 2;
  }
  return n;
}

template <int BN, int STAGES>
void launch_gemm_pair(const tc::GemmProblem* table, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  using S = tc::GemmPairSmem<BN, STAGES>;
  static int clusters = 0;
  if (clusters == 0) {
    cudaFuncSetAttribute(tc::tc_gemm_pair_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
    clusters = pair_clusters_max(reinterpret_cast<const void*>(tc::tc_gemm_pair_kernel<BN, STAGES>), S::kBytes);
  }
  const int grid = 2 * std::min(tiles, clusters);
  launch_k(tc::tc_gemm_pair_kernel<BN, STAGES>, dim3(grid), dim3(224), S::kBytes, st, table, nprob, tiles, status);
}

// A GEMM configuration: tile width, ring depth and kernel (0: one tile per CTA,
// 1: persistent, 2: CTA pair with 256-row tiles), coded as 8192 * kernel + 16 * BN + stages.
constexpr int gemm_cfg(int bn, int stages, int kernel = 0) { return 8192 * kernel + 16 * bn + stages; }
constexpr int cfg_bn(int cfg) { return (cfg % 8192) / 16; }
constexpr int cfg_kernel(int cfg) { return cfg / 8192; }
constexpr int cfg_bm(int cfg) { return cfg_kernel(cfg) == 2 ? 2 * tc::kBM : tc::kBM; }
// ANY tunes over all three kernels.
bool cfg_allowed(int cfg) {
  if (g_gemm_kernel == CRL_GEMM_ONE_TILE) return cfg_kernel(cfg) == 0;
  if (g_gemm_kernel == CRL_GEMM_PERSISTENT) return cfg_kernel(cfg) == 1;
  if (g_gemm_kernel == CRL_GEMM_CTA_PAIR) return cfg_kernel(cfg) == 2;
  return true;
}
constexpr int kGemmCfgs[10] = {gemm_cfg(64, 4),     gemm_cfg(64, 8),     gemm_cfg(128, 3),    gemm_cfg(128, 6),
                               gemm_cfg(256, 4),    gemm_cfg(64, 8, 1),  gemm_cfg(128, 6, 1), gemm_cfg(256, 4, 1),
                               gemm_cfg(128, 8, 2), gemm_cfg(256, 6, 2)};

void launch_cfg(int cfg, const tc::GemmProblem* t, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  switch (cfg) {
    case gemm_cfg(128, 8, 2): launch_gemm_pair<128, 8>(t, nprob, tiles, status, st); break;
    case gemm_cfg(256, 6, 2): launch_gemm_pair<256, 6>(t, nprob, tiles, status, st); break;
    case gemm_cfg(64, 8, 1): launch_gemm_persistent<64, 8>(t, nprob, tiles, status, st); break;
    case gemm_cfg(128, 6, 1): launch_gemm_persistent<128, 6>(t, nprob, tiles, status, st); break;
    case gemm_cfg(256, 4, 1): launch_gemm_persistent<256, 4>(t, nprob, tiles, status, st); break;
    case gemm_cfg(64, 8): launch_gemm_cfg<64, 8>(t, nprob, tiles, status, st); break;
    case gemm_cfg(128, 3): launch_gemm_cfg<128, 3>(t, nprob, tiles, status, st); break;
    case gemm_cfg(128, 4): launch_gemm_cfg<128, 4>(t, nprob, tiles, status, st); break;
    case gemm_cfg(128, 6): launch_gemm_cfg<128, 6>(t, nprob, tiles, status, st); break;
    case gemm_cfg(256, 4): launch_gemm_cfg<256, 4>(t, nprob, tiles, status, st); break;
    default: launch_gemm_cfg<64, 4>(t, nprob, tiles, status, st); break;
  }
}

// Configuration without measurement: 128 x 64 tiles unless 128 x 128 tiles
// already fill the 152 SMs; 4-deep rings.
int heuristic_cfg(const std::vector<tc::GemmProblem>& probs, int min_bn) {
  long long ctas128 = 0;
  for (const auto& p : probs) ctas128 += (long long)ceil_div(p.M, 128) * ceil_div(p.N, 128);
  const int bn = std::max(ctas128 >= 148 ? 128 : 64, min_bn <= 64 ? 64 : (min_bn <= 128 ? 128 : 256));
  if (g_gemm_kernel == CRL_GEMM_PERSISTENT)
    return bn == 256 ? gemm_cfg(256, 4, 1) : (bn == 128 ? gemm_cfg(128, 6, 1) : gemm_cfg(64, 8, 1));
  if (g_gemm_kernel == CRL_GEMM_CTA_PAIR) {
    // pair tiles want width: 256 columns wherever every problem has them
    int nmin = 1 << 30;
    for (const auto& p : probs) nmin = std::min(nmin, p.N);
    return (bn == 256 || nmin >= 256) ? gemm_cfg(256, 6, 2) : gemm_cfg(128, 8, 2);
  }
  return bn == 256 ? gemm_cfg(256, 4) : (bn == 128 ? gemm_cfg(128, 4) : gemm_cfg(64, 4));
}

// Autotuner: time each candidate configuration (tile width, ring depth) on
// the launch itself (every GEMM epilogue writes a pure function of inputs the
// launch does not modify, so repeating it is harmless, and neither choice
// changes any output value), keep the fastest.  The candidates are timed in
// two rounds (one warm-up and three timed launches each), and each keeps its
// faster round, so that a clock ramp or a transient at the start of the first
// round does not decide the pick.  Runs once per distinct problem list,
// outside graph capture; returns 0 when it cannot measure (the caller falls
// back to the fixed rule).
int tune_cfg(GemmGroups& gg, std::vector<tc::GemmProblem>& probs, int min_bn, bool one_tile_only, unsigned* status,
             cudaStream_t st, double flops) {
  constexpr int kRounds = 2, kReps = 3;
  GemmGroups::TuneRecord rec = {};
  for (int cfg : kGemmCfgs) {
    if (cfg_bn(cfg) < min_bn || !cfg_allowed(cfg) || (one_tile_only && cfg_kernel(cfg) != 0)) continue;
    rec.cand[rec.ncand] = cfg;
    rec.us[rec.ncand] = -1.f;
    ++rec.ncand;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 0;
  }
  for (int round = 0; round < kRounds; ++round) {
    for (int c = 0; c < rec.ncand; ++c) {
      const int cfg = rec.cand[c];
      int tiles = 0;
      const char* err = nullptr;
      const tc::GemmProblem* t = gg.table(probs, cfg_bn(cfg), &tiles, st, &err, cfg_kernel(cfg) == 0, cfg_bm(cfg));
      if (!t || tiles == 0) continue;
      launch_cfg(cfg, t, (int)probs.size(), tiles, status, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < kReps; ++r) launch_cfg(cfg, t, (int)probs.size(), tiles, status, st);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
      const float us = 1000.f * ms / kReps;
      if (rec.us[c] < 0.f || us < rec.us[c]) rec.us[c] = us;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = -1;
  for (int c = 0; c < rec.ncand; ++c)
    if (rec.us[c] >= 0.f && (best < 0 || rec.us[c] < rec.us[best])) best = c;
  if (best < 0) return 0;
  rec.cfg = rec.cand[best];
  rec.nprob = (int)probs.size();
  rec.M0 = probs[0].M;
  rec.N0 = probs[0].N;
  rec.K0 = probs[0].K;
  rec.flops = flops;
  rec.issued = 0.0;
  for (const auto& p : probs) rec.issued += 2.0 * p.M * p.N * p.K;
  gg.add_record(rec);
  return rec.cfg;
}

// One grouped launch of `probs` with the tuned (or heuristic) tile width.
// `flops` is the algorithmic work (2 M N K of the unsplit products) for tracing.
const char* launch_group(GemmGroups& gg, std::vector<tc::GemmProblem>& probs, double flops, unsigned* status,
                         cudaStream_t st) {
  if (probs.empty()) return nullptr;
  const uint64_t key = fnv1a(probs.data(), probs.size() * sizeof(tc::GemmProblem));
  // an energy-operand epilogue needs the whole row in one tile
  int min_bn = 0;
  for (const auto& p : probs)
    if (p.epi.kind == tc::kEpiFwdOutEnergy) min_bn = std::max(min_bn, p.N);
  if (min_bn > 256) return "an energy-operand output layer wider than 256 columns";
  // a list that splits over K stays on the one-tile kernel whatever the timings
  // say, so its outputs never depend on the pick (all one-tile widths give the
  // same bits; the other kernels do not split)
  const bool one_tile_only = list_split(probs) > 1;
  const bool tune = g_autotune && gg.allow_tune;
  int cfg = tune ? gg.tuned_bn(key) : 0;
  if (cfg != 0 && !cfg_allowed(cfg)) cfg = 0;   // tuned under another kernel setting
  if (cfg == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (tune && !capturing && g_tracer == nullptr) {
      cfg = tune_cfg(gg, probs, min_bn, one_tile_only, status, st, flops);
      if (cfg) gg.set_tuned_bn(key, cfg);
    }
    if (cfg == 0) cfg = heuristic_cfg(probs, min_bn);
  }
  int tiles = 0;
  const char* err = nullptr;
  const tc::GemmProblem* t = gg.table(probs, cfg_bn(cfg), &tiles, st, &err, cfg_kernel(cfg) == 0, cfg_bm(cfg));
  if (!t) return err;
  if (tiles == 0) return nullptr;
  TraceLaunch tr(CRL_TRACE_GEMM, st, flops);
  launch_cfg(cfg, t, (int)probs.size(), tiles, status, st);
  return nullptr;
}

}  // namespace

std::string gemm_tuning_json(const GemmGroups& gg) {
  auto name = [](int cfg) {
    static const char* const kinds[] = {"one_tile", "persistent", "cta_pair"};
    char b[64];
    snprintf(b, sizeof(b), "%s %dx%d s%d", kinds[cfg_kernel(cfg)], cfg_bm(cfg), cfg_bn(cfg), cfg % 16);
    return std::string(b);
  };
  std::string js = "[";
  char b[256];
  for (size_t i = 0; i < gg.records().size(); ++i) {
    const GemmGroups::TuneRecord& r = gg.records()[i];
    snprintf(b, sizeof(b),
             "%s{\"problems\": %d, \"first_mnk\": [%d, %d, %d], \"gflop\": %.4f, \"issued_gflop\": %.4f, "
             "\"picked\": \"%s\", \"us\": {",
             i ? ", " : "", r.nprob, r.M0, r.N0, r.K0, r.flops * 1e-9, r.issued * 1e-9, name(r.cfg).c_str());
    js += b;
    for (int c = 0; c < r.ncand; ++c) {
      snprintf(b, sizeof(b), "%s\"%s\": %.2f", c ? ", " : "", name(r.cand[c]).c_str(), r.us[c]);
      js += b;
    }
    js += "}}";
  }
  return js + "]";
}

// Split-K factor of a problem list: the problems that allow it (ksplit_cap > 1)
// take one split, chosen from the list's shape alone -- about two CTAs per SM
// counted in 128 x 64 tiles -- so that it does not depend on the tile
// configuration a launch runs with (the one-tile kernel splits; the others do
// not, so a list that splits runs on the one-tile kernel only).
int list_split(const std::vector<tc::GemmProblem>& probs) {
  int mn = 0, cap = 0;
  for (const auto& p : probs) {
    mn += ceil_div(p.M, tc::kBM) * ceil_div(p.N, 64);
    if (p.ksplit_cap > 1) cap = cap == 0 ? p.ksplit_cap : std::min(cap, p.ksplit_cap);
  }
  int split = cap > 1 ? std::max(1, std::min(cap, (2 * sm_count()) / std::max(mn, 1))) : 1;
  // no problem splits into parts of fewer than 8 K-slices
  bool any = false;
  for (const auto& p : probs)
    if (p.ksplit_cap > 1 && std::min(split, ceil_div(p.K, tc::kBK) / 8) > 1) any = true;
  return any ? split : 1;
}

const tc::GemmProblem* GemmGroups::table(std::vector<tc::GemmProblem>& probs, int BN, int* total_tiles,
                                         cudaStream_t st, const char** err, bool allow_split, int BM) {
  const int split = (allow_split && BN > 0) ? list_split(probs) : 1;
  int tiles = 0;
  for (auto& p : probs) {
    if (BN == 0) break;
    p.tiles_n = ceil_div(p.N, BN);
    p.tile_begin = tiles;
    const int nk = ceil_div(p.K, tc::kBK);
    p.ksplit = (p.ksplit_cap > 1) ? std::max(1, std::min(split, nk / 8)) : 1;
    tiles += ceil_div(p.M, BM) * p.tiles_n * p.ksplit;
  }
  *total_tiles = tiles;
  const size_t bytes = probs.size() * sizeof(tc::GemmProblem);
  const uint64_t h = fnv1a(probs.data(), bytes);
  auto it = map_.find(h);
  if (it != map_.end()) {
    for (const Entry& e : it->second)
      if (e.host.size() == probs.size() && memcmp(e.host.data(), probs.data(), bytes) == 0) return e.dev;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    *err = "a grouped-GEMM problem table was first needed while the stream was being captured";
    return nullptr;
  }
  const int n = (int)probs.size();
  if (used_ + n > cap_) {
    const int cap = std::max(256, n);
    void* mem = nullptr;
    if (cudaMalloc(&mem, (size_t)cap * sizeof(tc::GemmProblem)) != cudaSuccess) {
      *err = "device allocation of a grouped-GEMM problem table failed";
      return nullptr;
    }
    chunks_.push_back(mem);
    cur_ = static_cast<tc::GemmProblem*>(mem);
    used_ = 0;
    cap_ = cap;
  }
  tc::GemmProblem* dev = cur_ + used_;
  if (cudaMemcpy(dev, probs.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "copying a grouped-GEMM problem table failed";
    return nullptr;
  }
  used_ += n;
  map_[h].push_back(Entry{dev, tiles, probs});
  return dev;
}

void GemmGroups::reset() {
  for (void* p : chunks_) cudaFree(p);
  chunks_.clear();
  map_.clear();
  tuned_.clear();
  records_.clear();
  cur_ = nullptr;
  used_ = cap_ = 0;
}

const char* bf_net_carve(BfNet& n, const MlpShape& s, int Mmax, DevAlloc alloc, void* owner, bool weight_maps) {
  n.s = s;
  n.Mmax = Mmax;
  n.layers = s.layers;
  n.tm_M = -1;
  LayerOffsets lay[CRL_MAX_LAYERS + 1];
  mlp_layout(s, lay);
  const int H = s.hidden;
  auto A = [&](size_t bytes) { return alloc(owner, bytes); };
  for (int l = 0; l <= s.layers; ++l) {
    BfLayer& L = n.L[l];
    L.in = lay[l].in;
    L.out = lay[l].out;
    L.kin = (l == 0) ? 2 * L.in : L.in;
    L.kp = (L.kin + 63) / 64 * 64;
    L.nhi = (l == 0) ? 1 : 2;
    L.in_pad = (L.nhi + 1) * L.kp;
    L.out_pad = pad8(L.out);
    L.oW = lay[l].W;
    L.ob = lay[l].b;
    L.og = lay[l].g;
    L.obeta = lay[l].beta;
    L.W = static_cast<bf16*>(A((size_t)L.out * L.in_pad * 2));
    L.Wt = static_cast<bf16*>(A((size_t)L.in * L.out_pad * 2));
    if (!L.W || !L.Wt) return "device allocation failed";
    if (weight_maps) {
      const char* e;
      if ((e = mk(&L.tmW, L.W, L.in_pad, L.out, L.in_pad))) return e;  // B of the forward (see BfLayer)
      if ((e = mk(&L.tmWt, L.Wt, L.out, L.in, L.out_pad))) return e;   // B of the input gradient (K = out)
    }
  }
  // split-K buffers of the weight gradients: K = the batch, split in up to 4
  // parts of >= 2048 rows (smaller batches have enough tiles without it)
  const int cap = std::max(1, std::min(4, Mmax / 2048));
  for (int l = 0; l <= s.layers; ++l) {
    BfLayer& L = n.L[l];
    L.wsplit_cap = cap;
    L.wpart = nullptr;
    L.wtick = nullptr;
    if (cap < 2) continue;
    const int N = (l == 0) ? 2 * L.in + 1 : L.in + 1;   // the weight-gradient product's columns
    L.wpart = static_cast<float*>(A((size_t)cap * round_up(L.out, 128) * round_up(N, 256) * 4));
    L.wtick = static_cast<unsigned*>(A((size_t)round_up(ceil_div(L.out, 128) * ceil_div(N, 64), 64) * 4));
    if (!L.wpart || !L.wtick) return "device allocation failed";
  }
  const int in = s.in(), out = s.out;
  const int Hp = (H + 63) / 64 * 64;
  n.hlo = 2 * Hp;
  n.ldh = 4 * Hp;
  n.x0 = static_cast<bf16*>(A((size_t)Mmax * pad8(2 * in + 1) * 2));
  for (int l = 0; l < s.layers; ++l) {
    n.h[l] = static_cast<bf16*>(A((size_t)Mmax * n.ldh * 2));
    if (s.layernorm) {
      n.z[l] = static_cast<float*>(A((size_t)Mmax * H * 4));
      n.rstd[l] = static_cast<float*>(A((size_t)Mmax * 4));
    }
  }
  n.y = static_cast<float*>(A((size_t)Mmax * out * 4));
  for (int l = 0; l <= s.layers; ++l) {
    const size_t w = (l == s.layers) ? (size_t)pad8(out) : (size_t)H;
    n.dz[l] = static_cast<bf16*>(A((size_t)Mmax * w * 2));
  }
  if (s.layernorm) {
    n.du = static_cast<float*>(A((size_t)Mmax * H * 4));
    n.ln_partial = static_cast<float*>(A(ln_partial_floats(Mmax, H, s.layers) * 4));
  }
  if (!n.x0 || !n.y || (s.layernorm && (!n.du || !n.ln_partial)))
    return "device allocation failed";
  return nullptr;
}

namespace {
// Counting allocator for bf_net_bytes: 256-byte aligned offsets from a fake base.
void* count_alloc(void* owner, size_t bytes) {
  size_t* off = static_cast<size_t*>(owner);
  const size_t o = (*off + 255) / 256 * 256;
  *off = o + bytes;
  return reinterpret_cast<void*>(uintptr_t(4096) + o);
}
}  // namespace

size_t bf_net_bytes(const MlpShape& s, int Mmax) {
  BfNet n;
  size_t off = 0;
  if (bf_net_carve(n, s, Mmax, count_alloc, &off, false)) return 0;
  return (off + 255) / 256 * 256;
}

void bf_net_fill_ones(BfNet& n, cudaStream_t st) {
  const int in = n.s.in(), H = n.s.hidden, Mx = n.Mmax;
  fill_col_bf16_kernel<<<ceil_div(Mx, 256), 256, 0, st>>>(n.x0 + 2 * in, Mx, bf_net_x0_ld(n), 1.f);
  for (int l = 0; l < n.layers; ++l) fill_col_bf16_kernel<<<ceil_div(Mx, 256), 256, 0, st>>>(n.h[l] + H, Mx, n.ldh, 1.f);
}

const char* bf_net_init(BfNet& n, const MlpShape& s, int Mmax, DevAlloc alloc, void* owner) {
  if (const char* e = bf_net_carve(n, s, Mmax, alloc, owner, true)) return e;
  const int in = s.in(), out = s.out, H = s.hidden;
  for (int l = 0; l <= s.layers; ++l) {
    const BfLayer& L = n.L[l];
    if (cudaMemset(L.W, 0, (size_t)L.out * L.in_pad * 2) != cudaSuccess ||
        cudaMemset(L.Wt, 0, (size_t)L.in * L.out_pad * 2) != cudaSuccess)
      return "cudaMemset failed";
    if (L.wtick) {
      const int N = (l == 0) ? 2 * L.in + 1 : L.in + 1;
      if (cudaMemset(L.wtick, 0, (size_t)round_up(ceil_div(L.out, 128) * ceil_div(N, 64), 64) * 4) != cudaSuccess)
        return "cudaMemset failed";
    }
  }
  for (int l = 0; l <= s.layers; ++l) {
    const size_t w = (l == s.layers) ? (size_t)pad8(out) : (size_t)H;
    if (cudaMemset(n.dz[l], 0, (size_t)Mmax * w * 2) != cudaSuccess) return "cudaMemset failed";
  }
  for (int l = 0; l < s.layers; ++l)   // the zero columns between the hi and lo halves are read as K
    if (cudaMemset(n.h[l], 0, (size_t)Mmax * n.ldh * 2) != cudaSuccess) return "cudaMemset failed";
  if (cudaMemset(n.x0, 0, (size_t)Mmax * pad8(2 * in + 1) * 2) != cudaSuccess) return "cudaMemset failed";
  // the ones columns of the bias gradients (never overwritten)
  bf_net_fill_ones(n, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) return "initialising the ones columns failed";
  return nullptr;
}

const char* bf_net_maps(BfNet& n, int M) {
  if (n.tm_M == M) return nullptr;
  const int in = n.s.in(), H = n.s.hidden, out = n.s.out;
  const char* e;
  const int x0ld = bf_net_x0_ld(n);
  if ((e = mk(&n.tm_x0A, n.x0, 2 * in, M, x0ld))) return e;
  if ((e = mk(&n.tm_x0B, n.x0, 2 * in + 1, M, x0ld))) return e;
  for (int l = 0; l < n.layers; ++l) {
    if ((e = mk(&n.tm_hA[l], n.h[l], n.ldh, M, n.ldh))) return e;
    if ((e = mk(&n.tm_hB[l], n.h[l], H + 1, M, n.ldh))) return e;
  }
  for (int l = 0; l <= n.layers; ++l) {
    const int width = (l == n.layers) ? out : H, ld = (l == n.layers) ? pad8(out) : H;
    if ((e = mk(&n.tm_dzA[l], n.dz[l], width, M, ld))) return e;
  }
  n.tm_M = M;
  return nullptr;
}

void bf_net_shadow(BfNet& n, const float* params, cudaStream_t st) {
  for (int l = 0; l <= n.layers; ++l) {
    BfLayer& L = n.L[l];
    TraceLaunch tr(CRL_TRACE_AUX, st, (double)L.out * L.in * 10.0);
    dim3 grid(ceil_div(L.in, 32), ceil_div(L.out, 32));
    launch_k(pack_weights_kernel, grid, dim3(256), 0, st, L.out, L.in, l == 0 ? 2 : 1, L.nhi, params + L.oW, L.W, L.kp,
             L.Wt, L.out_pad);
  }
}

int bf_net_x0_ld(const BfNet& n) { return pad8(2 * n.s.in() + 1); }

void bf_net_pack_input(BfNet& n, const float* x0, const float* x1, int M, cudaStream_t st) {
  const int in = n.s.in();
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * in * 12.0);
  dim3 grid(ceil_div(in, 32), ceil_div(M, 32));
  launch_k(pack_split_kernel, grid, dim3(256), 0, st, M, x0, n.s.in0, n.s.in0, x1, n.s.in1, n.s.in1, n.x0,
           bf_net_x0_ld(n), (bf16*)nullptr, 0);
}

void bf_net_load_dy(BfNet& n, const float* dy, int M, cudaStream_t st) {
  const int out = n.s.out;
  pack(M, dy, out, out, nullptr, 0, 0, n.dz[n.layers], pad8(out), nullptr, 0, st);
}

namespace {

// Forward problem of layer l of one network (the per-layer launch's problem).
tc::GemmProblem forward_problem(const BfPass& bp, int l, bool ln) {
  BfNet& n = *bp.net;
  const int H = n.s.hidden, layers = n.layers;
  const BfLayer& L = n.L[l];
  const float* params = bp.params;
  const CUtensorMap& A = (l == 0) ? n.tm_x0A : n.tm_hA[l - 1];
  tc::EpiDesc e;
  if (l == layers && bp.energy_out) {
    const EnergyOut& eo = *bp.energy_out;
    e = epi_of(tc::kEpiFwdOutEnergy);
    e.ld0 = L.out;
    e.out0 = n.y;
    e.out1 = eo.X;
    e.aux = eo.aux;
    e.energy = eo.energy;
  } else if (l == layers) {
    e = epi_of(tc::kEpiFwdOut);
    e.ld0 = L.out;
    e.out0 = n.y;
  } else if (ln) {
    e = epi_of(tc::kEpiFwdPreLN);
    e.ld0 = H;
    e.out0 = n.z[l];
  } else {
    e = epi_of(tc::kEpiFwdHidden);
    e.ld0 = n.ldh;
    e.c0 = n.hlo;
    e.out0 = n.h[l];
  }
  e.bias = params + L.ob;
  // layer 0: A = the split input (x_hi, x_lo interleaved) against [W_hi | W_lo];
  // later layers: A = [h_hi | h_lo] against [W_hi | W_hi | W_lo], the A slices
  // wrapping around: h_hi W_hi + h_lo W_hi + h_hi W_lo
  tc::GemmProblem p = problem(A, L.tmW, bp.M, L.out, L.in_pad, (L.nhi == 1 ? 1 : 2) * L.kp / 64, e);
  if (l > 0) {   // h_lo sits two 64-column blocks after h_hi's last slice
    p.a_gap = L.kp / 64;
    p.a_skip = L.kp / 64;
  }
  return p;
}

}  // namespace

// One grouped pass over every layer: one grouped GEMM launch per layer.
const char* bf_forward(GemmGroups& gg, const BfPass* nets, int count, unsigned* status, cudaStream_t st) {
  if (count <= 0) return nullptr;
  const BfNet& n0 = *nets[0].net;
  const int H = n0.s.hidden, layers = n0.layers;
  const bool ln = n0.s.layernorm != 0;
  for (int k = 1; k < count; ++k)
    if (nets[k].net->layers != layers || nets[k].net->s.hidden != H || (nets[k].net->s.layernorm != 0) != ln)
      return "the networks of a grouped pass differ in depth, hidden width or LayerNorm";
  std::vector<tc::GemmProblem> probs;
  for (int l = 0; l <= layers; ++l) {
    probs.clear();
    double flops = 0.0;
    for (int k = 0; k < count; ++k) {
      BfNet& n = *nets[k].net;
      const int M = nets[k].M;
      if (M <= 0) continue;
      const BfLayer& L = n.L[l];
      probs.push_back(forward_problem(nets[k], l, ln));
      flops += 2.0 * M * L.out * L.in;
    }
    if (const char* err = launch_group(gg, probs, flops, status, st)) return err;
    for (int k0 = 0; l < layers && ln && k0 < count; k0 += kMaxGroupNets) {
      const int kc = std::min(kMaxGroupNets, count - k0);
      LnFwdGroup grp;
      memset(&grp, 0, sizeof(grp));
      int Mx = 0;
      double bytes = 0.0;
      for (int k = 0; k < kc; ++k) {
        BfNet& n = *nets[k0 + k].net;
        const BfLayer& L = n.L[l];
        const float* pr = nets[k0 + k].params;
        const int M = std::max(nets[k0 + k].M, 0);
        grp.n[k] = LnFwdNet{M, n.z[l], n.rstd[l], pr + L.og, pr + L.obeta, n.h[l], n.ldh, n.hlo};
        Mx = std::max(Mx, M);
        bytes += (double)M * H * 12.0;
      }
      if (Mx == 0) continue;
      TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
      launch_ln_fwd(H, dim3(ceil_div(Mx, kLnRows), kc), st, grp);
    }
  }
  return nullptr;
}

const char* bf_backward(GemmGroups& gg, const BfPass* nets, int count, unsigned* status, cudaStream_t st) {
  if (count <= 0) return nullptr;
  const BfNet& n0 = *nets[0].net;
  const int H = n0.s.hidden, layers = n0.layers;
  const bool ln = n0.s.layernorm != 0;
  for (int k = 1; k < count; ++k)
    if (nets[k].net->layers != layers || nets[k].net->s.hidden != H || (nets[k].net->s.layernorm != 0) != ln)
      return "the networks of a grouped pass differ in depth, hidden width or LayerNorm";
  std::vector<LnReduceItem> ln_items;
  std::vector<tc::GemmProblem> probs;
  // input-gradient chain: dz[l] -> dz[l - 1]
  for (int l = layers; l >= 1; --l) {
    probs.clear();
    double flops = 0.0;
    for (int k = 0; k < count; ++k) {
      BfNet& n = *nets[k].net;
      const int M = nets[k].M;
      if (M <= 0) continue;
      const BfLayer& L = n.L[l];
      tc::EpiDesc e = epi_of(ln ? tc::kEpiBwdDXLN : tc::kEpiBwdDX);
      e.mask = n.h[l - 1];
      e.ldm = n.ldh;
      e.ld0 = H;
      e.out0 = ln ? static_cast<void*>(n.du) : static_cast<void*>(n.dz[l - 1]);
      probs.push_back(problem(n.tm_dzA[l], L.tmWt, M, H, L.out, 0, e));
      flops += 2.0 * M * H * L.out;
    }
    if (const char* err = launch_group(gg, probs, flops, status, st)) return err;
    for (int k0 = 0; ln && k0 < count; k0 += kMaxGroupNets) {
      const int kc = std::min(kMaxGroupNets, count - k0);
      LnBwdGroup grp;
      memset(&grp, 0, sizeof(grp));
      int Mx = 0;
      double bytes = 0.0;
      for (int k = 0; k < kc; ++k) {
        const BfPass& bp = nets[k0 + k];
        BfNet& n = *bp.net;
        const BfLayer& P = n.L[l - 1];
        const int M = std::max(bp.M, 0);
        const int nblk = ceil_div(n.Mmax, kLnRows);
        float* part = bp.grads ? n.ln_partial + (size_t)(l - 1) * nblk * 2 * H : nullptr;
        grp.n[k] = LnBwdNet{M, n.du, n.z[l - 1], n.rstd[l - 1], bp.params + P.og, n.dz[l - 1], part};
        if (part && M > 0) ln_items.push_back(LnReduceItem{part, bp.grads + P.og, bp.grads + P.obeta,
                                                           ceil_div(M, kLnRows)});
        Mx = std::max(Mx, M);
        bytes += (double)M * H * (bp.grads ? 24.0 : 16.0);
      }
      if (Mx == 0) continue;
      TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
      launch_ln_bwd(H, dim3(ceil_div(Mx, kLnRows), kc), st, grp);
    }
  }
  // the LayerNorm gain / shift gradients of every layer and network: block sums in order
  for (size_t i0 = 0; i0 < ln_items.size(); i0 += kMaxLnReduce) {
    const int ni = (int)std::min<size_t>(kMaxLnReduce, ln_items.size() - i0);
    LnReduceGroup grp;
    memset(&grp, 0, sizeof(grp));
    double bytes = 0.0;
    for (int i = 0; i < ni; ++i) {
      grp.it[i] = ln_items[i0 + i];
      bytes += (double)ln_items[i0 + i].nblk * 2 * H * 4;
    }
    TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
    launch_k(ln_param_reduce_kernel, dim3(ceil_div(H, 32), ni), dim3(256), 0, st, H, grp);
  }
  // every weight gradient, and the first-layer input gradients, in one launch
  probs.clear();
  double flops = 0.0;
  for (int k = 0; k < count; ++k) {
    BfNet& n = *nets[k].net;
    const int M = nets[k].M;
    if (M <= 0) continue;
    if (float* grads = nets[k].grads) {
      for (int l = 0; l <= layers; ++l) {
        const BfLayer& L = n.L[l];
        tc::EpiDesc e = epi_of(l == 0 ? tc::kEpiBwdDW0 : tc::kEpiBwdDW);
        e.kin = L.in;
        e.out0 = grads + L.oW;
        e.out1 = grads + L.ob;
        // dW = dz^T [x | 1] with K = the batch: dz [M][out] and x [M][in + 1]
        // are read as they are stored (MN-major), the ones column giving db
        if (l == 0) probs.push_back(problem(n.tm_dzA[0], n.tm_x0B, L.out, 2 * L.in + 1, M, 0, e));
        else probs.push_back(problem(n.tm_dzA[l], n.tm_hB[l - 1], L.out, L.in + 1, M, 0, e));
        probs.back().a_mn = 1;
        probs.back().b_mn = 1;
        if (L.wsplit_cap > 1) {
          probs.back().ksplit_cap = L.wsplit_cap;
          probs.back().part = L.wpart;
          probs.back().tickets = L.wtick;
        }
        flops += 2.0 * L.out * (L.in + 1) * M;
      }
    }
    if (nets[k].dx1) {
      const BfLayer& L = n.L[0];
      tc::EpiDesc e = epi_of(tc::kEpiDX0);
      e.out0 = nets[k].dx1;
      e.c0 = n.s.in0;
      e.nc = n.s.in1;
      probs.push_back(problem(n.tm_dzA[0], L.tmWt, M, L.in, L.out, 0, e));
      flops += 2.0 * M * L.in * L.out;
    }
    if (nets[k].dx0) {
      const BfLayer& L = n.L[0];
      tc::EpiDesc e = epi_of(tc::kEpiDX0);
      e.out0 = nets[k].dx0;
      e.c0 = 0;
      e.nc = n.s.in0;
      probs.push_back(problem(n.tm_dzA[0], L.tmWt, M, L.in, L.out, 0, e));
      flops += 2.0 * M * L.in * L.out;
    }
  }
  return launch_group(gg, probs, flops, status, st);
}

namespace {

struct ShadowLayer {
  int64_t oW;
  int out, in, rep, kp, ldt, nhi, pad_;
  bf16* W2;
  bf16* Wt;
};
struct AdamNetDev {
  float* p;
  const float* g;
  float* m;
  float* v;
  long long n;
  const int* t;
  float lr, b1, b2, eps;
  float log_b1, log_b2;   // ln(b1), ln(b2) (computed in double on the host)
  int nl;
  ShadowLayer L[CRL_MAX_LAYERS + 1];
};

// One block of work for the Adam + shadow kernel: a 32 x 128 tile of a weight
// matrix (layer >= 0: rows [r0, r0 + 32) of the output units, columns
// [c0, c0 + 128) of the inputs), or a flat range of the parameter array
// (layer < 0: [r0, r0 + c0) -- biases, LayerNorm gains and shifts and the
// zero padding between tensors, whose update is zero).
struct AdamUnit {
  int net, layer, r0, c0;
};

// Adam on the FP32 master parameters and the refresh of the BF16 shadows:
// W2 (nhi copies of W_hi, then W_lo; see pack_weights_kernel) row-major
// (coalesced along the tile's columns) and Wt
// (the transposed single BF16, written through a shared-memory transpose).
// Bias corrections 1 - b^t = -expm1(t ln b): accurate to a few float ulps
// where 1 - b^t is small (early steps), unlike 1 - powf(b, t).
// Blocks [nunits, gridDim.x) run the actor head's forward (head_begin: each
// task's first block, 8 rows per block) instead: it reads only the policy's
// output, so it rides in the critic's Adam launch.
// TW: the tile's columns (128 for large layers, 32 when the launch would
// otherwise have too few blocks to hide memory latency).
template <int TW>
__global__ void __launch_bounds__(256, 4) adam_shadow_kernel(const AdamNetDev* __restrict__ nets,
                                                          const AdamUnit* __restrict__ units, int nunits,
                                                          const HeadFwdArgs<float>* __restrict__ heads,
                                                          const int* __restrict__ head_begin, int nheads) {
  if ((int)blockIdx.x >= nunits) {
    pdl_enter();
    int lb, nb;
    const int s = segment_of(head_begin, nheads, (int)blockIdx.x - nunits, lb, nb);
    head_forward_body(heads[s], lb);
    return;
  }
  // the tables are immutable, and p, m, v are written by Adam alone: pull this
  // block's lines into L2 while the predecessor (which writes g) drains
  const AdamUnit u = units[blockIdx.x];
  const AdamNetDev& a = nets[u.net];
  if (u.layer < 0) {
    if (threadIdx.x < 96) {
      const float* arr = threadIdx.x < 32 ? a.p : (threadIdx.x < 64 ? a.m : a.v);
      const int j = threadIdx.x % 32;
      if (32 * j < u.c0) prefetch_l2(arr + u.r0 + 32 * j);
    }
  } else {
    // 32 rows x TW columns: TW / 32 lines of 128 bytes per row and array
    constexpr int kLines = TW / 32;
    const ShadowLayer& L = a.L[u.layer];
    for (int i = threadIdx.x; i < 3 * 32 * kLines; i += blockDim.x) {
      const int arr_i = i / (32 * kLines), j = i % (32 * kLines);
      const float* arr = arr_i == 0 ? a.p : (arr_i == 1 ? a.m : a.v);
      const int o = u.r0 + j / kLines, c = u.c0 + 32 * (j % kLines);
      if (o < L.out && c < L.in) prefetch_l2(arr + L.oW + (long long)o * L.in + c);
    }
  }
  pdl_enter();
  // the descriptor's fields in registers: the stores below cannot change them
  const float* __restrict__ g = a.g;
  float* __restrict__ m = a.m;
  float* __restrict__ v = a.v;
  float* __restrict__ p = a.p;
  const float b1 = a.b1, b2 = a.b2, eps = a.eps;
  const float t = (float)*a.t;
  const float c1 = a.lr / -expm1f(t * a.log_b1);
  const float c2 = 1.f / -expm1f(t * a.log_b2);
  // one element: moments and parameter from the gradient gi
  auto upd = [=](float pi, float gi, float& mi, float& vi) {
    mi = b1 * mi + (1.f - b1) * gi;
    vi = b2 * vi + (1.f - b2) * gi * gi;
    return pi - c1 * mi / (sqrtf(vi * c2) + eps);
  };
  auto step = [=](long long i) {
    float mi = m[i], vi = v[i];
    const float pi = upd(p[i], g[i], mi, vi);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
    return pi;
  };
  if (u.layer < 0) {
    for (int k = threadIdx.x; k < u.c0; k += blockDim.x) step((long long)u.r0 + k);
    return;
  }
  // weight tile rows [r0, r0 + 32) x columns [c0, c0 + TW): thread (rq, cq)
  // takes columns 4 cq .. 4 cq + 3 of rows rq, rq + R, ... (R = 256 / (TW / 4)
  // rows per pass; 16-byte accesses where the rows are 16-byte aligned); W_hi
  // also goes to a transposed shared tile for the coalesced Wt rows
  __shared__ bf16 tile[128][34];
  const ShadowLayer L = a.L[u.layer];
  bf16* __restrict__ W2 = L.W2;
  constexpr int kTpr = TW / 4, kRows = 256 / kTpr, kPasses = 32 / kRows;   // threads per row, rows per pass
  const int cq = threadIdx.x % kTpr, rq = threadIdx.x / kTpr;
  const int cc = 4 * cq, c = u.c0 + cc;
  const bool vec = (L.in % 4) == 0 && c + 4 <= L.in;   // oW is a multiple of 64
#pragma unroll
  for (int k = 0; k < kPasses; ++k) {
    const int rr = rq + kRows * k, o = u.r0 + rr;
    float pv[4] = {0.f, 0.f, 0.f, 0.f};
    bool live[4] = {false, false, false, false};
    if (o < L.out) {
      const long long i0 = L.oW + (long long)o * L.in + c;
      if (vec) {
        const float4 g4 = *reinterpret_cast<const float4*>(g + i0);
        const float4 m4 = *reinterpret_cast<const float4*>(m + i0);
        const float4 v4 = *reinterpret_cast<const float4*>(v + i0);
        const float4 p4 = *reinterpret_cast<const float4*>(p + i0);
        float mx = m4.x, my = m4.y, mz = m4.z, mw = m4.w, vx = v4.x, vy = v4.y, vz = v4.z, vw = v4.w;
        pv[0] = upd(p4.x, g4.x, mx, vx);
        pv[1] = upd(p4.y, g4.y, my, vy);
        pv[2] = upd(p4.z, g4.z, mz, vz);
        pv[3] = upd(p4.w, g4.w, mw, vw);
        *reinterpret_cast<float4*>(m + i0) = make_float4(mx, my, mz, mw);
        *reinterpret_cast<float4*>(v + i0) = make_float4(vx, vy, vz, vw);
        *reinterpret_cast<float4*>(p + i0) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        live[0] = live[1] = live[2] = live[3] = true;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < L.in) {
            pv[j] = step(i0 + j);
            live[j] = true;
          }
      }
    }
    // W_hi / W_lo of the four columns (zero where the column lies outside the layer)
    __nv_bfloat162 h01, h23, l01, l23;
    {
      const float x0 = live[0] ? pv[0] : 0.f, x1 = live[1] ? pv[1] : 0.f;
      const float x2 = live[2] ? pv[2] : 0.f, x3 = live[3] ? pv[3] : 0.f;
      h01 = __floats2bfloat162_rn(x0, x1);
      h23 = __floats2bfloat162_rn(x2, x3);
      l01 = __floats2bfloat162_rn(x0 - __low2float(h01), x1 - __high2float(h01));
      l23 = __floats2bfloat162_rn(x2 - __low2float(h23), x3 - __high2float(h23));
    }
    tile[cc][rr] = __low2bfloat16(h01);
    tile[cc + 1][rr] = __high2bfloat16(h01);
    tile[cc + 2][rr] = __low2bfloat16(h23);
    tile[cc + 3][rr] = __high2bfloat16(h23);
    if (o < L.out) {
      bf16* d = W2 + (size_t)o * (L.nhi + 1) * L.kp;
      if (vec && L.rep == 1) {
        const uint2 hv = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
        for (int q = 0; q < L.nhi; ++q) *reinterpret_cast<uint2*>(d + q * L.kp + c) = hv;
        *reinterpret_cast<uint2*>(d + L.nhi * L.kp + c) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (!live[j]) continue;
          const __nv_bfloat162 hp = j < 2 ? h01 : h23, lp = j < 2 ? l01 : l23;
          const bf16 hj = (j & 1) ? __high2bfloat16(hp) : __low2bfloat16(hp);
          const bf16 lj = (j & 1) ? __high2bfloat16(lp) : __low2bfloat16(lp);
          for (int q = 0; q < L.rep; ++q) {
            for (int r = 0; r < L.nhi; ++r) d[r * L.kp + L.rep * (c + j) + q] = hj;
            d[L.nhi * L.kp + L.rep * (c + j) + q] = lj;
          }
        }
      }
    }
  }
  __syncthreads();
  bf16* __restrict__ Wt = L.Wt;
  for (int e = threadIdx.x; e < TW * 32; e += blockDim.x) {
    const int ct = e / 32, rt = e % 32;
    const int o = u.r0 + rt, col = u.c0 + ct;
    if (o < L.out && col < L.in) Wt[(size_t)col * L.ldt + o] = tile[ct][rt];
  }
}

}  // namespace

const char* adam_shadow_update(BlobCache& cache, const AdamShadowNet* nets, int count, cudaStream_t st,
                               const std::vector<HeadFwdArgs<float>>* heads) {
  if (count <= 0) return nullptr;
  // 32 x 128 weight tiles when there are at least two per SM, else 32 x 32
  // (small networks: more blocks in flight hide the memory latency)
  long long wide_tiles = 0;
  for (int k = 0; k < count; ++k)
    for (int l = 0; l <= nets[k].net->layers; ++l)
      wide_tiles += (long long)ceil_div(nets[k].net->L[l].out, 32) * ceil_div(nets[k].net->L[l].in, 128);
  const bool wide = wide_tiles >= 2LL * sm_count();
  const int tw = wide ? 128 : 32;
  std::vector<AdamNetDev> devs(count);
  std::vector<AdamUnit> units;
  long long ntot = 0;
  for (int k = 0; k < count; ++k) {
    AdamNetDev& a = devs[k];
    memset(&a, 0, sizeof(a));
    const AdamShadowNet& s = nets[k];
    a.p = s.p;
    a.g = s.g;
    a.m = s.m;
    a.v = s.v;
    a.n = s.n;
    a.t = s.t_dev;
    a.lr = s.lr;
    a.b1 = s.b1;
    a.b2 = s.b2;
    a.eps = s.eps;
    a.log_b1 = (float)std::log((double)s.b1);
    a.log_b2 = (float)std::log((double)s.b2);
    a.nl = s.net->layers + 1;
    ntot += s.n;
    for (int l = 0; l <= s.net->layers; ++l) {
      const BfLayer& L = s.net->L[l];
      ShadowLayer& sl = a.L[l];   // member by member: the zeroed padding keys the device table
      sl.oW = L.oW;
      sl.out = L.out;
      sl.in = L.in;
      sl.rep = l == 0 ? 2 : 1;
      sl.nhi = L.nhi;
      sl.kp = L.kp;
      sl.ldt = L.out_pad;
      sl.W2 = L.W;
      sl.Wt = L.Wt;
      for (int r0 = 0; r0 < L.out; r0 += 32)
        for (int c0 = 0; c0 < L.in; c0 += tw) units.push_back(AdamUnit{k, l, r0, c0});
      // the layer's vectors (bias, LayerNorm gain and shift) and padding up to the next tensor
      const long long v0 = L.oW + (long long)round_up((int64_t)L.out * L.in, 64);
      const long long v1 = (l < s.net->layers) ? s.net->L[l + 1].oW : s.n;
      for (long long o = v0; o < v1; o += 1024) units.push_back(AdamUnit{k, -1, (int)o, (int)std::min<long long>(1024, v1 - o)});
    }
  }
  const char* err = nullptr;
  const AdamNetDev* dt = cache.get(devs, st, &err);
  if (!dt) return err;
  const AdamUnit* du = cache.get(units, st, &err);
  if (!du) return err;
  const HeadFwdArgs<float>* dh = nullptr;
  const int* dhb = nullptr;
  int nh = 0, head_blocks = 0;
  double head_bytes = 0.0;
  if (heads && !heads->empty()) {
    std::vector<int> begin(heads->size() + 1, 0);
    for (size_t i = 0; i < heads->size(); ++i) {
      begin[i + 1] = begin[i] + ceil_div((*heads)[i].B, 8);
      head_bytes += (double)(*heads)[i].B * (*heads)[i].A * 4.0 * 5;
    }
    head_blocks = begin.back();
    nh = (int)heads->size();
    if (!(dh = cache.get(*heads, st, &err))) return err;
    if (!(dhb = cache.get(begin, st, &err))) return err;
  }
  TraceLaunch tr(CRL_TRACE_ADAM, st, 28.0 * ntot + head_bytes);
  if (wide)
    launch_k(adam_shadow_kernel<128>, dim3((unsigned)(units.size() + head_blocks)), dim3(256), 0, st, dt, du,
             (int)units.size(), dh, dhb, nh);
  else
    launch_k(adam_shadow_kernel<32>, dim3((unsigned)(units.size() + head_blocks)), dim3(256), 0, st, dt, du,
             (int)units.size(), dh, dhb, nh);
  return nullptr;
}

}  // namespace crl
