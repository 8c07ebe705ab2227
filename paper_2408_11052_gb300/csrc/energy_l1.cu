// The -L1 energy on the fused path (arXiv 2408.11052, App. A.2: f(x, y) =
// -|x - y|_1, F_ij = f(phi_i, psi_j) / tau), with every objective and the
// logsumexp penalty of Algorithm 1 / §5.2, and no B x B matrix in memory.
//
// |x - y| has no product form, so these tiles run on the FP32 SIMT lanes, not
// the tensor cores, and read the FP32 representations (no BF16 rounding: the
// energy, its logsumexps and its gradient are FP32 throughout).
//
// forward:  one CTA per (row tile I, column tile J) of 128 x 128: F in
//           registers (8 x 8 per thread, K staged through shared memory in
//           chunks of 32), then the same partials as the tcgen05 forward with
//           one column tile per chunk: per row (max, sum) over the tile's
//           columns, per column (max, sum) over its rows, the diagonal F_ii and
//           the objectives' row terms.  The tcgen05 path's finalize merges them.
// backward: dphi_uk = -(1 / tau) sum_v g_uv sign(phi_uk - psi_vk) and
//           dpsi_vk = -(1 / tau) sum_u g_uv sign(psi_vk - phi_uk), g = dL/dF
//           (sign(0) = 0).  A CTA owns 64 rows of one side and walks a segment
//           of the other side's 64-row tiles: F tile (recomputed in the
//           forward's order, so it is bit-identical) -> coefficient tile in
//           shared memory -> the sign sums, accumulated in registers.  With
//           several segments per row tile the partial sums land in scratch and
//           a second kernel adds them in segment order (deterministic).
//
// Every F_ij is summed over k = 0 .. R - 1 in order, one |x - y| at a time, so
// the forward, the backward and the DPO / IPO anchors F_ii agree bit for bit.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "energy_args.cuh"
#include "trace.h"

namespace crl {
namespace fe {
namespace {

constexpr float kLog2eF = 1.4426950408889634f;

__device__ __forceinline__ float2 sub_x2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// acc += |x_k - y_k| for the four k of one float4, in k order.
__device__ __forceinline__ float absdiff4(float acc, float4 x, float4 y) {
  const float2 d01 = sub_x2(make_float2(x.x, x.y), make_float2(y.x, y.y));
  const float2 d23 = sub_x2(make_float2(x.z, x.w), make_float2(y.z, y.w));
  acc += fabsf(d01.x);
  acc += fabsf(d01.y);
  acc += fabsf(d23.x);
  acc += fabsf(d23.y);
  return acc;
}

// g sign(d) with sign(0) = 0.
__device__ __forceinline__ float signed_coef(float g, float d) {
  const float t = __int_as_float(__float_as_int(g) ^ (__float_as_int(d) & 0x80000000));
  return d != 0.f ? t : 0.f;
}

// 16-byte copy global -> shared, zero-filled when !valid (nothing is read then).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// F_uu = -|phi_u - psi_u|_1 / tau in the tiles' summation order.
__device__ __forceinline__ float anchor(const float* __restrict__ x, const float* __restrict__ y, int R,
                                        float inv_tau) {
  float acc = 0.f;
  for (int k = 0; k < R; k += 4)
    acc = absdiff4(acc, __ldg(reinterpret_cast<const float4*>(x + k)), __ldg(reinterpret_cast<const float4*>(y + k)));
  return acc * -inv_tau;
}

__device__ __forceinline__ float half_max(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- forward ---------------------------------------------------------------------
// 256 threads; thread (tx, ty) = (tid % 16, tid / 16) holds rows i0 + ty + 16 a
// and columns j0 + tx + 16 b (a, b = 0 .. 7).  A warp reads two X rows
// (broadcast) and 16 Y rows per float4 step: with a row pitch of 36 floats the
// 16 rows fall on distinct bank quads in two wavefronts.
constexpr int kFwdT = 256;
constexpr int kKC = 32;        // K per staged chunk
constexpr int kKCP = kKC + 4;  // row pitch in shared memory (floats)
constexpr size_t kFwdStage = (size_t)kTile * kKCP;   // floats of one operand's chunk
constexpr size_t kFwdSmemBytes = 4 * kFwdStage * sizeof(float);   // X, Y x two stages

template <bool OBJ>
__global__ void __launch_bounds__(kFwdT, 2) l1_fwd_kernel(const __grid_constant__ FwdArgs a) {
  extern __shared__ float4 l1f_smem[];
  float* sm = reinterpret_cast<float*>(l1f_smem);
  __shared__ float s_c[8][kTile];   // per warp: column maxima, then column sums
  __shared__ float s_cmax[kTile];
  __shared__ float s_d[kTile];      // DPO / IPO anchors of this CTA's rows
  const int J = blockIdx.x, I = blockIdx.y;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16, lane = tid % 32, w = tid / 32;
  const int B = a.B, R = a.R, i0 = I * kTile, j0 = J * kTile;
  const float inv_tau = a.inv_tau;
  pdl_enter();

  auto load = [&](int stage, int k0) {
    float* xs = sm + (size_t)stage * 2 * kFwdStage;
    float* ys = xs + kFwdStage;
    for (int q = tid; q < kTile * (kKC / 4); q += kFwdT) {
      const int r = q / (kKC / 4), c4 = q % (kKC / 4);
      const int gi = i0 + r, gj = j0 + r;
      cp_async16(xs + r * kKCP + 4 * c4, a.phi + (size_t)(gi < B ? gi : 0) * R + k0 + 4 * c4, gi < B);
      cp_async16(ys + r * kKCP + 4 * c4, a.psi + (size_t)(gj < B ? gj : 0) * R + k0 + 4 * c4, gj < B);
    }
  };

  const bool anchored = OBJ && (a.obj == CRL_LOSS_DPO || a.obj == CRL_LOSS_IPO);
  if (anchored && tid < kTile) {
    const int i = i0 + tid;
    float d = 0.f;
    if (i < B) {
      d = anchor(a.phi + (size_t)i * R, a.psi + (size_t)i * R, R, inv_tau);
      if (J == 0) a.dpre[i] = d;
    }
    s_d[tid] = d;
  }

  float acc[8][8];
#pragma unroll
  for (int al = 0; al < 8; ++al)
#pragma unroll
    for (int be = 0; be < 8; ++be) acc[al][be] = 0.f;
  const int nch = R / kKC;
  load(0, 0);
  cp_async_commit();
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load((c + 1) & 1, (c + 1) * kKC);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float* xs = sm + (size_t)(c & 1) * 2 * kFwdStage;
    const float* ys = xs + kFwdStage;
#pragma unroll 1
    for (int kk = 0; kk < kKC; kk += 4) {
      float4 x[8];
#pragma unroll
      for (int al = 0; al < 8; ++al) x[al] = *reinterpret_cast<const float4*>(xs + (ty + 16 * al) * kKCP + kk);
#pragma unroll
      for (int be = 0; be < 8; ++be) {
        const float4 y = *reinterpret_cast<const float4*>(ys + (tx + 16 * be) * kKCP + kk);
#pragma unroll
        for (int al = 0; al < 8; ++al) acc[al][be] = absdiff4(acc[al][be], x[al], y);
      }
    }
    __syncthreads();   // the stage is refilled by the next iteration's load
  }

  // F = -acc / tau (the anchors' expression); exponents take F log2(e)
  bool colv[8];
#pragma unroll
  for (int be = 0; be < 8; ++be) colv[be] = j0 + tx + 16 * be < B;
#pragma unroll
  for (int al = 0; al < 8; ++al)
#pragma unroll
    for (int be = 0; be < 8; ++be) acc[al][be] = acc[al][be] * -inv_tau;

  // diagonal F_ii
  if (I == J && tx == ty) {
#pragma unroll
    for (int al = 0; al < 8; ++al) {
      const int i = i0 + ty + 16 * al;
      if (i < B) a.diag[i] = acc[al][al];
    }
  }

  // rows: (max, sum) over the tile's columns, across the 16 lanes of a half warp
#pragma unroll
  for (int al = 0; al < 8; ++al) {
    const int i = i0 + ty + 16 * al;
    float m = -INFINITY;
#pragma unroll
    for (int be = 0; be < 8; ++be)
      if (colv[be]) m = fmaxf(m, acc[al][be] * kLog2eF);
    m = half_max(m);
    float s = 0.f;
#pragma unroll
    for (int be = 0; be < 8; ++be)
      if (colv[be]) s += ex2(acc[al][be] * kLog2eF - m);
    s = half_sum(s);
    float vp = 0.f, kp = 0.f;
    if (OBJ && a.obj >= CRL_LOSS_FB) {
      const float dpair = anchored ? s_d[ty + 16 * al] : 0.f;
#pragma unroll
      for (int be = 0; be < 8; ++be) {
        if (!colv[be]) continue;
        const float F = acc[al][be];
        const int j = j0 + tx + 16 * be;
        switch (a.obj) {
          case CRL_LOSS_FB:
            if (j != i) vp += ex2(2.f * (F * kLog2eF));
            break;
          case CRL_LOSS_DPO: {
            const float x = F - dpair;
            vp += softplusf(x);
            kp += sigmoidf_fast(x);
            break;
          }
          case CRL_LOSS_IPO: {
            const float x = dpair - F - 1.f;
            vp += x * x;
            kp -= 2.f * x;
            break;
          }
          case CRL_LOSS_SPPO: {
            const float x = F + 1.f;
            vp += x * x;
            break;
          }
          default:  // NCE-binary
            vp += softplusf(F);
            break;
        }
      }
      vp = half_sum(vp);
      kp = half_sum(kp);
    }
    if (tx == 0 && i < B) {
      float* rp = a.rowpart + ((size_t)J * B + i) * 2;
      rp[0] = m * kLn2;
      rp[1] = s;
      if (OBJ && a.obj >= CRL_LOSS_FB) {
        float* op = a.objpart + ((size_t)J * B + i) * 2;
        op[0] = vp;
        op[1] = kp;
      }
    }
  }

  // columns: maximum over the tile's rows, then the sum against it
  bool rowv[8];
#pragma unroll
  for (int al = 0; al < 8; ++al) rowv[al] = i0 + ty + 16 * al < B;
#pragma unroll
  for (int be = 0; be < 8; ++be) {
    float m = -INFINITY;
#pragma unroll
    for (int al = 0; al < 8; ++al)
      if (rowv[al]) m = fmaxf(m, acc[al][be] * kLog2eF);
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    if (lane < 16) s_c[w][tx + 16 * be] = m;
  }
  __syncthreads();
  if (tid < kTile) {
    float m = s_c[0][tid];
    for (int q = 1; q < 8; ++q) m = fmaxf(m, s_c[q][tid]);
    s_cmax[tid] = m;
  }
  __syncthreads();
#pragma unroll
  for (int be = 0; be < 8; ++be) {
    const float m = s_cmax[tx + 16 * be];
    float s = 0.f;
#pragma unroll
    for (int al = 0; al < 8; ++al)
      if (rowv[al]) s += ex2(acc[al][be] * kLog2eF - m);
    s += __shfl_xor_sync(0xffffffffu, s, 16);
    if (lane < 16) s_c[w][tx + 16 * be] = s;
  }
  __syncthreads();
  if (tid < kTile && j0 + tid < B) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += s_c[q][tid];
    float* cp = a.colpart + ((size_t)I * B + j0 + tid) * 2;
    cp[0] = s_cmax[tid] * kLn2;
    cp[1] = s;
  }
}

// ---- backward --------------------------------------------------------------------
// 512 threads, 64 own rows, the other side in tiles of 64 rows.
//   F tile: warp w takes the 16 x 16 block (w / 4, w % 4); lane (la, lb) =
//     (lane / 8, lane % 8) its rows 16 (w / 4) + la + 4 a (a < 4) and columns
//     16 (w % 4) + lb + 8 b (b < 2): 4 + 2 float4 reads per K step, one
//     wavefront each (4 and 8 distinct rows, pitch R + 4 floats).
//   sign sums: warp w = own rows w + 16 a (a < 4), lane = float4 columns
//     lane + 32 c (c < 2): each thread keeps its 32 own values and 32 sums in
//     registers; per other row one broadcast float4 of coefficients and one
//     or two float4 of the other row.
constexpr int kBwdT = 512;
constexpr int kTA = 64;
constexpr int kMaxSeg = 8;

struct L1Sched {
  int nA, nB, S;   // own tiles per pass, other tiles, segments per own tile
  float* part;     // S > 1: [S][2][B][R] partial gradients
};

size_t bwd_smem_bytes(int R) { return ((size_t)3 * kTA * (R + 4) + (size_t)kTA * kTA) * sizeof(float); }

template <int OBJ>
__global__ void __launch_bounds__(kBwdT, 1) l1_bwd_kernel(const __grid_constant__ BwdArgs row,
                                                          const __grid_constant__ BwdArgs col,
                                                          const __grid_constant__ L1Sched sc) {
  extern __shared__ float4 l1b_smem[];
  const int seg = blockIdx.x % sc.S, pa = blockIdx.x / sc.S;
  const bool colpass = pa >= sc.nA;
  const BwdArgs& a = colpass ? col : row;
  const int A = colpass ? pa - sc.nA : pa;
  const int B = a.B, R = a.R, RP = R + 4;
  float* ownS = reinterpret_cast<float*>(l1b_smem);   // [64][RP]
  float* othS = ownS + kTA * RP;                         // [2][64][RP]
  float* Gs = othS + 2 * kTA * RP;                       // [64 other][16 own % 16][4 own / 16]
  const int tb0 = seg * sc.nB / sc.S, tb1 = (seg + 1) * sc.nB / sc.S;
  const int u0 = A * kTA;
  const int tid = threadIdx.x, lane = tid % 32, w = tid / 32;
  pdl_enter();

  auto load_rows = [&](float* dst, const float* __restrict__ src, int r0) {
    const int n4 = R / 4;
    for (int q = tid; q < kTA * n4; q += kBwdT) {
      const int r = q / n4, c4 = q % n4, g = r0 + r;
      cp_async16(dst + r * RP + 4 * c4, src + (size_t)(g < B ? g : 0) * R + 4 * c4, g < B);
    }
  };
  load_rows(ownS, a.own_f32, u0);
  if (tb0 < tb1) load_rows(othS, a.other_f32, tb0 * kTA);
  cp_async_commit();

  // F tile roles
  const int wa = w / 4, wb = w % 4, la = lane / 8, lb = lane % 8;
  // loss weights of this side and of the other (row pass: forward direction and
  // row penalty own; column pass: backward direction and column penalty own)
  const float w_own = a.transposed ? a.w.wb : a.w.wf, p_own = a.transposed ? a.w.pc : a.w.pr;
  const float w_oth = a.transposed ? a.w.wf : a.w.wb, p_oth = a.transposed ? a.w.pr : a.w.pc;
  const float k_diag = a.scale * (a.w.wf + a.w.wb);
  HCoef hc = {};
  hc.dtotal = a.dtotal;
  hc.c_bb = a.dtotal / ((float)B * (float)B);
  hc.c_b = a.dtotal / (float)B;
  hc.c_fb = B > 1 ? a.dtotal / ((float)B * (float)(B - 1)) : 0.f;
  constexpr bool kAnchored = OBJ == kObjDPO || OBJ == kObjIPO;
  float l_own2[4], k_own[4], d_own[4], kd_own[4];
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    const int u = u0 + 16 * wa + la + 4 * al;
    const float l = u < B ? a.lse_own[u] : 0.f;
    l_own2[al] = l * kLog2eF;
    k_own[al] = a.scale * (w_own + 2.f * a.beta * p_own * l);
    d_own[al] = (kAnchored && u < B) ? a.dpre[u] : 0.f;
    kd_own[al] = (kAnchored && u < B) ? a.kd[u] : 0.f;
  }
  const float kb_oth = a.scale * w_oth, k2_oth = 2.f * a.scale * a.beta * p_oth;

  // sign-sum roles: own rows w + 16 a, float4 columns lane + 32 c
  bool kv[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) kv[c] = 4 * (lane + 32 * c) < R;
  float own[4][2][4], sum[4][2][4];
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) sum[al][c][e] = 0.f;

  for (int t = tb0; t < tb1; ++t) {
    cp_async_wait<0>();
    __syncthreads();   // tile t (and on the first pass the own rows) landed; Gs and the other buffer are free
    if (t == tb0) {
#pragma unroll
      for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (kv[c]) v = *reinterpret_cast<const float4*>(ownS + (w + 16 * al) * RP + 4 * (lane + 32 * c));
          own[al][c][0] = v.x;
          own[al][c][1] = v.y;
          own[al][c][2] = v.z;
          own[al][c][3] = v.w;
        }
    }
    if (t + 1 < tb1) load_rows(othS + (size_t)((t + 1 - tb0) & 1) * kTA * RP, a.other_f32, (t + 1) * kTA);
    cp_async_commit();
    const float* os = othS + (size_t)((t - tb0) & 1) * kTA * RP;
    const int v0 = t * kTA;

    // F tile (the forward's summation order)
    float f[4][2];
#pragma unroll
    for (int al = 0; al < 4; ++al) f[al][0] = f[al][1] = 0.f;
    const float* xr = ownS + (16 * wa + la) * RP;
    const float* yr = os + (16 * wb + lb) * RP;
#pragma unroll 2
    for (int k = 0; k < R; k += 4) {
      float4 x[4], y[2];
#pragma unroll
      for (int al = 0; al < 4; ++al) x[al] = *reinterpret_cast<const float4*>(xr + 4 * al * RP + k);
#pragma unroll
      for (int be = 0; be < 2; ++be) y[be] = *reinterpret_cast<const float4*>(yr + 8 * be * RP + k);
#pragma unroll
      for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int be = 0; be < 2; ++be) f[al][be] = absdiff4(f[al][be], x[al], y[be]);
    }
    // coefficient tile: -g / tau, g = dL/dF (0 outside the batch)
#pragma unroll
    for (int be = 0; be < 2; ++be) {
      const int bl = 16 * wb + lb + 8 * be, v = v0 + bl;
      const bool vin = v < B;
      const float lo = vin ? a.lse_other[v] : 0.f;
      const float lo2 = lo * kLog2eF, ko = fmaf(k2_oth, lo, kb_oth);
      const float d_col = (kAnchored && vin) ? a.dpre[v] : 0.f;
      const float kd_col = (kAnchored && vin) ? a.kd[v] : 0.f;
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        const int ar = 16 * wa + la + 4 * al, u = u0 + ar;
        const float f2 = (f[al][be] * -a.inv_tau) * kLog2eF;
        float g = fmaf(ex2(f2 - l_own2[al]), k_own[al], ex2(f2 - lo2) * ko);
        if (u == v) g -= k_diag;
        if (OBJ != kObjInfo) {
          const float d_row = a.transposed ? d_col : d_own[al];
          const float k_row = a.transposed ? kd_col : kd_own[al];
          g += objective_coef<OBJ>(f2, u == v, d_row, k_row, hc);
        }
        Gs[(bl * 16 + (ar % 16)) * 4 + ar / 16] = (u < B && vin) ? g * -a.inv_tau : 0.f;
      }
    }
    __syncthreads();

    // sign sums over the tile's 64 other rows
#pragma unroll 2
    for (int b = 0; b < kTA; ++b) {
      const float4 g4 = *reinterpret_cast<const float4*>(Gs + (b * 16 + w) * 4);
      const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!kv[c]) continue;
        const float4 y = *reinterpret_cast<const float4*>(os + b * RP + 4 * (lane + 32 * c));
#pragma unroll
        for (int al = 0; al < 4; ++al) {
          const float2 d01 = sub_x2(make_float2(own[al][c][0], own[al][c][1]), make_float2(y.x, y.y));
          const float2 d23 = sub_x2(make_float2(own[al][c][2], own[al][c][3]), make_float2(y.z, y.w));
          const float2 s01 = add_x2(make_float2(sum[al][c][0], sum[al][c][1]),
                                    make_float2(signed_coef(gv[al], d01.x), signed_coef(gv[al], d01.y)));
          const float2 s23 = add_x2(make_float2(sum[al][c][2], sum[al][c][3]),
                                    make_float2(signed_coef(gv[al], d23.x), signed_coef(gv[al], d23.y)));
          sum[al][c][0] = s01.x;
          sum[al][c][1] = s01.y;
          sum[al][c][2] = s23.x;
          sum[al][c][3] = s23.y;
        }
      }
    }
  }

  // results: the gradient rows, or this segment's partial sums
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    const int u = u0 + w + 16 * al;
    if (u >= B) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!kv[c]) continue;
      const int k = 4 * (lane + 32 * c);
      const float4 v = make_float4(sum[al][c][0], sum[al][c][1], sum[al][c][2], sum[al][c][3]);
      if (sc.S > 1) {
        *reinterpret_cast<float4*>(sc.part + (((size_t)seg * 2 + (colpass ? 1 : 0)) * B + u) * R + k) = v;
      } else if (a.d_out_f32) {
        *reinterpret_cast<float4*>(a.d_out_f32 + (size_t)u * R + k) = v;
      } else {
        __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(a.d_out + (size_t)u * R + k);
        o[0] = __floats2bfloat162_rn(v.x, v.y);
        o[1] = __floats2bfloat162_rn(v.z, v.w);
      }
    }
  }
}

// The segments' partial gradients added in segment order: one float4 per thread.
__global__ void __launch_bounds__(256) l1_reduce_kernel(const __grid_constant__ BwdArgs row,
                                                        const __grid_constant__ BwdArgs col,
                                                        const __grid_constant__ L1Sched sc) {
  pdl_enter();
  const size_t per = (size_t)row.B * row.R / 4;   // float4 per pass
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * per) return;
  const int pass = idx >= per ? 1 : 0;
  const size_t e = idx - (size_t)pass * per;
  const float4* p = reinterpret_cast<const float4*>(sc.part);
  float4 s = __ldcg(p + ((size_t)0 * 2 + pass) * per + e);
  for (int q = 1; q < sc.S; ++q) {
    const float4 y = __ldcg(p + ((size_t)q * 2 + pass) * per + e);
    s.x += y.x;
    s.y += y.y;
    s.z += y.z;
    s.w += y.w;
  }
  const BwdArgs& a = pass ? col : row;
  if (a.d_out_f32) {
    reinterpret_cast<float4*>(a.d_out_f32)[e] = s;
  } else {
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(a.d_out) + 2 * e;
    o[0] = __floats2bfloat162_rn(s.x, s.y);
    o[1] = __floats2bfloat162_rn(s.z, s.w);
  }
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 152;
  }
  return n;
}

// Segments per own tile: the S <= min(8, nB) minimising the time in full-range
// CTA units, ceil(2 nA S / SMs) / S (one CTA per SM); ties take the smaller S.
int segments(int nA, int nB) {
  const int sms = sm_count();
  int best = 1;
  double best_cost = 0.0;
  for (int S = 1; S <= std::min(kMaxSeg, nB); ++S) {
    const double cost = (double)((2LL * nA * S + sms - 1) / sms) / S;
    if (S == 1 || cost < best_cost - 1e-9) {
      best = S;
      best_cost = cost;
    }
  }
  return best;
}

template <int OBJ>
void launch_bwd(const BwdArgs& row, const BwdArgs& col, const L1Sched& sc, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(l1_bwd_kernel<OBJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem_bytes(256));
    attr = true;
  }
  launch_k(l1_bwd_kernel<OBJ>, dim3(2 * sc.nA * sc.S), dim3(kBwdT), bwd_smem_bytes(row.R), st, row, col, sc);
}

}  // namespace

size_t l1_part_floats(int B, int R) { return (size_t)kMaxSeg * 2 * B * R; }

void l1_forward(const FwdArgs& a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(l1_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemBytes);
    cudaFuncSetAttribute(l1_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemBytes);
    attr = true;
  }
  TraceLaunch tr(CRL_TRACE_ENERGY, st, 2.0 * a.B * a.B * a.R);
  const dim3 grid(a.n, a.n);
  if (a.obj >= CRL_LOSS_FB) launch_k(l1_fwd_kernel<true>, grid, dim3(kFwdT), kFwdSmemBytes, st, a);
  else launch_k(l1_fwd_kernel<false>, grid, dim3(kFwdT), kFwdSmemBytes, st, a);
}

void l1_backward(const BwdArgs& row, const BwdArgs& col, float* part, cudaStream_t st) {
  const int B = row.B;
  L1Sched sc;
  sc.nA = (B + kTA - 1) / kTA;
  sc.nB = sc.nA;
  sc.S = part ? segments(sc.nA, sc.nB) : 1;
  sc.part = part;
  {
    TraceLaunch tr(CRL_TRACE_ENERGY, st, 4.0 * B * B * row.R);
    switch (obj_kind(row.obj)) {
      case kObjFB: launch_bwd<kObjFB>(row, col, sc, st); break;
      case kObjDPO: launch_bwd<kObjDPO>(row, col, sc, st); break;
      case kObjIPO: launch_bwd<kObjIPO>(row, col, sc, st); break;
      case kObjSPPO: launch_bwd<kObjSPPO>(row, col, sc, st); break;
      case kObjNCE: launch_bwd<kObjNCE>(row, col, sc, st); break;
      default: launch_bwd<kObjInfo>(row, col, sc, st); break;
    }
  }
  if (sc.S > 1) {
    TraceLaunch tr(CRL_TRACE_ENERGY, st, 0.0);
    const size_t n4 = (size_t)2 * B * row.R / 4;
    launch_k(l1_reduce_kernel, dim3((unsigned)((n4 + 255) / 256)), dim3(256), 0, st, row, col, sc);
  }
}

}  // namespace fe
}  // namespace crl
