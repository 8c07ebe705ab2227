// BF16 tensor-core MLP forward / backward (see mlp_bf16.cuh for the scheme).
//
// Networks of arXiv 2408.11052: phi(s, a) and psi(g) (§3.1), the policy
// (§3.2); hidden [256, 256] / repr 64 (App. B.3); LayerNorm before every
// activation for the large networks (§5.4).  Readings M1-M3 as in the FP32
// path: ReLU, LayerNorm (eps 1e-6, biased variance, affine) between Linear and
// ReLU, W stored [out][in].
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "mlp_bf16.cuh"
#include "tc_gemm.cuh"
#include "tc_host.h"
#include "trace.h"

namespace crl {

using bf16 = __nv_bfloat16;

namespace {

constexpr float kLnEpsF = 1e-6f;

inline int pad8(int x) { return (x + 7) / 8 * 8; }

// ---- epilogues -----------------------------------------------------------------
// hidden layer without LayerNorm: h = ReLU(acc + b), written row-major and transposed
struct EpiFwdHidden {
  const float* bias;
  bf16* h;
  int ldh;
  bf16* hT;
  int ldt;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    if (col0 + 32 <= N) {
      alignas(16) bf16 o[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) o[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[col0 + i], 0.f));
      uint4* dst = reinterpret_cast<uint4*>(h + (size_t)row * ldh + col0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
#pragma unroll
      for (int i = 0; i < 32; ++i) hT[(size_t)(col0 + i) * ldt + row] = o[i];
    } else {
      for (int i = 0; i < 32 && col0 + i < N; ++i) {
        const bf16 o = __float2bfloat16_rn(fmaxf(v[i] + bias[col0 + i], 0.f));
        h[(size_t)row * ldh + col0 + i] = o;
        hT[(size_t)(col0 + i) * ldt + row] = o;
      }
    }
  }
};

// hidden layer with LayerNorm: z = acc + b (FP32), normalised by the LayerNorm kernel
struct EpiFwdPreLN {
  const float* bias;
  float* z;
  int ldz;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    for (int i = 0; i < 32 && col0 + i < N; ++i) z[(size_t)row * ldz + col0 + i] = v[i] + bias[col0 + i];
  }
};

// output layer: y = acc + b (FP32)
struct EpiFwdOut {
  const float* bias;
  float* y;
  int ldy;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    for (int i = 0; i < 32 && col0 + i < N; ++i) y[(size_t)row * ldy + col0 + i] = v[i] + bias[col0 + i];
  }
};

// input gradient of a hidden layer: du = acc * [h > 0]; BF16 dz / dz^T (no LayerNorm) or FP32 du
struct EpiBwdDX {
  const bf16* hmask;
  int ldm;
  bf16* dz;
  int ldz;
  bf16* dzT;
  int ldt;
  float* du;  // non-null: LayerNorm layer, write FP32 du instead
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    for (int i = 0; i < 32 && col0 + i < N; ++i) {
      const int c = col0 + i;
      const float x = __bfloat162float(hmask[(size_t)row * ldm + c]) > 0.f ? v[i] : 0.f;
      if (du) {
        du[(size_t)row * ldz + c] = x;
      } else {
        const bf16 o = __float2bfloat16_rn(x);
        dz[(size_t)row * ldz + c] = o;
        dzT[(size_t)c * ldt + row] = o;
      }
    }
  }
};

// weight gradient: rows = output units, columns = inputs plus the ones column (bias)
struct EpiBwdDW {
  float* dW;
  float* db;
  int kin;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    for (int i = 0; i < 32 && col0 + i < N; ++i) {
      const int c = col0 + i;
      if (c < kin) dW[(size_t)row * kin + c] = v[i];
      else db[row] = v[i];
    }
  }
};

// weight gradient of the split first layer: columns 2k (hi) and 2k+1 (lo) both
// multiply input k; column 2 kin is the ones column (bias)
struct EpiBwdDW0 {
  float* dW;
  float* db;
  int kin;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
      const int c = col0 + i;
      if (c + 1 < 2 * kin + 1 && c < 2 * kin) dW[(size_t)row * kin + c / 2] = v[i] + v[i + 1];
      else if (c == 2 * kin) db[row] = v[i];
    }
  }
};

// input gradient of the first layer, columns [c0, c0 + nc) only
struct EpiDX0 {
  float* dx;
  int c0, nc;
  __device__ void operator()(int row, int col0, const float (&v)[32], int M, int N) const {
    if (row >= M) return;
    for (int i = 0; i < 32 && col0 + i < N; ++i) {
      const int c = col0 + i - c0;
      if (c >= 0 && c < nc) dx[(size_t)row * nc + c] = v[i];
    }
  }
};

// ---- launch ---------------------------------------------------------------------
template <int BN, class Epi>
void launch_gemm_bn(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, int nkA, const Epi& epi,
                    unsigned* status, cudaStream_t st) {
  using S = tc::GemmSmem<BN>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::tc_gemm_kernel<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
    attr = true;
  }
  dim3 grid(ceil_div(N, BN), ceil_div(M, tc::kBM));
  tc::tc_gemm_kernel<BN, Epi><<<grid, 128, S::kBytes, st>>>(a, b, M, N, K, nkA, epi, status);
}

// BN 64 unless 128-wide tiles already fill the 152 SMs.
// nkA > 0: the split-weight forward (K = 2 * 64 * nkA, see tc_gemm_kernel); the
// traced work is the algorithmic 2 M N K of the unsplit product.
template <class Epi>
void tc_gemm(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, const Epi& epi, unsigned* status,
             cudaStream_t st, int nkA = 0, int k_alg = -1) {
  if (M <= 0 || N <= 0) return;
  TraceLaunch tr(CRL_TRACE_GEMM, st, 2.0 * M * N * (k_alg >= 0 ? k_alg : K));
  const long long ctas128 = (long long)ceil_div(M, 128) * ceil_div(N, 128);
  if (ctas128 >= 148) launch_gemm_bn<128>(a, b, M, N, K, nkA, epi, status, st);
  else launch_gemm_bn<64>(a, b, M, N, K, nkA, epi, status, st);
}

// ---- element kernels ----------------------------------------------------------------
// 32 x 32 tile transpose-and-pack: src = concat(s0 [rows][n0], s1 [rows][n1]) (FP32)
// -> dst [rows][ld] (BF16, optional) and dstT [n0 + n1][ldt] (BF16, optional).
__global__ void __launch_bounds__(256) pack_kernel(int rows, const float* __restrict__ s0, int ld0, int n0,
                                                  const float* __restrict__ s1, int ld1, int n1, bf16* __restrict__ dst,
                                                  int ld, bf16* __restrict__ dstT, int ldt) {
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

// Weight shadows: W [out][ncol] (FP32) -> W2 [out][2 kp] = [W_hi | W_lo] with
// hi = bf16(w), lo = bf16(w - hi), each column written `rep` times (rep = 2 for
// the first layer, matching the split input), and the single BF16 transpose
// Wt [ncol][ldt] for the input-gradient product.
__global__ void __launch_bounds__(256) pack_weights_kernel(int rows, int ncol, int rep, const float* __restrict__ W,
                                                          bf16* __restrict__ W2, int kp, bf16* __restrict__ Wt,
                                                          int ldt) {
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
      bf16* d = W2 + (size_t)row * 2 * kp;
      for (int q = 0; q < rep; ++q) {
        d[rep * col + q] = hi;
        d[kp + rep * col + q] = lo;
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
  pack_kernel<<<grid, 256, 0, st>>>(rows, s0, ld0, n0, s1, ld1, n1, dst, ld, dstT, ldt);
}

// LayerNorm forward over rows of z [M][H] (FP32, replaced by zhat), rstd [M],
// h = ReLU(zhat * g + beta) written as BF16 [M][H] and, through a shared tile,
// transposed [H][ldt].  Block = 32 rows (one warp each).
__global__ void __launch_bounds__(1024) ln_fwd_kernel(int M, int H, float* __restrict__ z, float* __restrict__ rstd,
                                                     const float* __restrict__ g, const float* __restrict__ beta,
                                                     bf16* __restrict__ h, bf16* __restrict__ hT, int ldt) {
  __shared__ float tile[32][33];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int row = blockIdx.x * 32 + w;
  float mean = 0.f, rs = 0.f;
  if (row < M) {
    const float* zr = z + (size_t)row * H;
    float s = 0.f;
    for (int c = lane; c < H; c += 32) s += zr[c];
    mean = warp_sum(s) / H;
    float q = 0.f;
    for (int c = lane; c < H; c += 32) {
      const float d = zr[c] - mean;
      q += d * d;
    }
    rs = rsqrtf(warp_sum(q) / H + kLnEpsF);
    if (lane == 0) rstd[row] = rs;
  }
  for (int c0 = 0; c0 < H; c0 += 32) {
    const int c = c0 + lane;
    float hv = 0.f;
    if (row < M && c < H) {
      const size_t o = (size_t)row * H + c;
      const float zh = (z[o] - mean) * rs;
      z[o] = zh;
      hv = fmaxf(zh * g[c] + beta[c], 0.f);
      h[o] = __float2bfloat16_rn(hv);
    }
    tile[w][lane] = hv;
    __syncthreads();
    // warp w writes column c0 + w for the block's 32 rows
    const int cc = c0 + w, rr = blockIdx.x * 32 + lane;
    if (cc < H && rr < M) hT[(size_t)cc * ldt + rr] = __float2bfloat16_rn(tile[lane][w]);
    __syncthreads();
  }
}

// LayerNorm backward: du (ReLU-masked, FP32) -> dz = rstd (g du - mean(g du) - zhat mean(g du zhat)),
// written BF16 [M][H] and transposed.  Block = 32 rows.
__global__ void __launch_bounds__(1024) ln_bwd_kernel(int M, int H, const float* __restrict__ du,
                                                     const float* __restrict__ zhat, const float* __restrict__ rstd,
                                                     const float* __restrict__ g, bf16* __restrict__ dz,
                                                     bf16* __restrict__ dzT, int ldt) {
  __shared__ float tile[32][33];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int row = blockIdx.x * 32 + w;
  float s1 = 0.f, s2 = 0.f, rs = 0.f;
  if (row < M) {
    for (int c = lane; c < H; c += 32) {
      const size_t o = (size_t)row * H + c;
      const float d = du[o] * g[c];
      s1 += d;
      s2 += d * zhat[o];
    }
    s1 = warp_sum(s1) / H;
    s2 = warp_sum(s2) / H;
    rs = rstd[row];
  }
  for (int c0 = 0; c0 < H; c0 += 32) {
    const int c = c0 + lane;
    float v = 0.f;
    if (row < M && c < H) {
      const size_t o = (size_t)row * H + c;
      v = rs * (du[o] * g[c] - s1 - zhat[o] * s2);
      dz[o] = __float2bfloat16_rn(v);
    }
    tile[w][lane] = v;
    __syncthreads();
    const int cc = c0 + w, rr = blockIdx.x * 32 + lane;
    if (cc < H && rr < M) dzT[(size_t)cc * ldt + rr] = __float2bfloat16_rn(tile[lane][w]);
    __syncthreads();
  }
}

// dgain[n] = sum_m du * zhat, dbeta[n] = sum_m du.  Block = 32 columns x 8 row groups.
__global__ void __launch_bounds__(256) ln_param_grad_kernel(int M, int H, const float* __restrict__ du,
                                                           const float* __restrict__ zhat, float* __restrict__ dg,
                                                           float* __restrict__ db) {
  __shared__ float sa[8][33], sb[8][33];
  const int cx = threadIdx.x % 32, ry = threadIdx.x / 32;
  const int n = blockIdx.x * 32 + cx;
  float a = 0.f, b = 0.f;
  if (n < H) {
    for (int m = ry; m < M; m += 8) {
      const size_t o = (size_t)m * H + n;
      a += du[o] * zhat[o];
      b += du[o];
    }
  }
  sa[ry][cx] = a;
  sb[ry][cx] = b;
  __syncthreads();
  if (ry == 0 && n < H) {
    for (int r = 1; r < 8; ++r) {
      a += sa[r][cx];
      b += sb[r][cx];
    }
    dg[n] = a;
    db[n] = b;
  }
}

__global__ void fill_bf16_kernel(bf16* p, size_t n, float v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = __float2bfloat16_rn(v);
}

const char* mk(CUtensorMap* m, const void* base, int inner, int rows, int stride) {
  const char* err = nullptr;
  if (!tc::make_tmap_bf16(m, base, (uint64_t)inner, (uint64_t)rows, (uint64_t)stride, 64, &err)) return err;
  return nullptr;
}

}  // namespace

const char* bf_net_init(BfNet& n, const MlpShape& s, int Mmax, DevAlloc alloc, void* owner) {
  n.s = s;
  n.Mmax = Mmax;
  n.layers = s.layers;
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
    L.in_pad = 2 * L.kp;
    L.out_pad = pad8(L.out);
    L.oW = lay[l].W;
    L.ob = lay[l].b;
    L.og = lay[l].g;
    L.obeta = lay[l].beta;
    L.W = static_cast<bf16*>(A((size_t)L.out * L.in_pad * 2));
    L.Wt = static_cast<bf16*>(A((size_t)L.in * L.out_pad * 2));
    if (!L.W || !L.Wt) return "device allocation failed";
    if (cudaMemset(L.W, 0, (size_t)L.out * L.in_pad * 2) != cudaSuccess ||
        cudaMemset(L.Wt, 0, (size_t)L.in * L.out_pad * 2) != cudaSuccess)
      return "cudaMemset failed";
    const char* e;
    if ((e = mk(&L.tmW, L.W, 2 * L.kp, L.out, L.in_pad))) return e;  // B of the forward: [W_hi | W_lo]
    if ((e = mk(&L.tmWt, L.Wt, L.out, L.in, L.out_pad))) return e;   // B of the input gradient (K = out)
  }
  const int in = s.in(), out = s.out;
  n.x0 = static_cast<bf16*>(A((size_t)Mmax * pad8(2 * in) * 2));
  n.x0T = static_cast<bf16*>(A((size_t)(2 * in + 1) * Mmax * 2));
  for (int l = 0; l < s.layers; ++l) {
    n.h[l] = static_cast<bf16*>(A((size_t)Mmax * H * 2));
    n.hT[l] = static_cast<bf16*>(A((size_t)(H + 1) * Mmax * 2));
    if (s.layernorm) {
      n.z[l] = static_cast<float*>(A((size_t)Mmax * H * 4));
      n.rstd[l] = static_cast<float*>(A((size_t)Mmax * 4));
    }
  }
  n.y = static_cast<float*>(A((size_t)Mmax * out * 4));
  const int wmax = std::max(H, pad8(out));
  for (int b = 0; b < 2; ++b) {
    n.dz[b] = static_cast<bf16*>(A((size_t)Mmax * wmax * 2));
    n.dzT[b] = static_cast<bf16*>(A((size_t)wmax * Mmax * 2));
  }
  if (s.layernorm) n.du = static_cast<float*>(A((size_t)Mmax * H * 4));
  if (cudaMemset(n.x0, 0, (size_t)Mmax * pad8(2 * in) * 2) != cudaSuccess) return "cudaMemset failed";
  for (int b = 0; b < 2; ++b)
    if (cudaMemset(n.dz[b], 0, (size_t)Mmax * wmax * 2) != cudaSuccess) return "cudaMemset failed";
  // the ones rows of the transposed activations (never overwritten)
  fill_bf16_kernel<<<ceil_div(Mmax, 256), 256>>>(n.x0T + (size_t)(2 * in) * Mmax, Mmax, 1.f);
  for (int l = 0; l < s.layers; ++l) fill_bf16_kernel<<<ceil_div(Mmax, 256), 256>>>(n.hT[l] + (size_t)H * Mmax, Mmax, 1.f);
  if (cudaDeviceSynchronize() != cudaSuccess) return "initialising the ones rows failed";
  return nullptr;
}

const char* bf_net_maps(BfNet& n, int M) {
  if (n.tm_M == M) return nullptr;
  const int in = n.s.in(), H = n.s.hidden, out = n.s.out, Mx = n.Mmax;
  const char* e;
  if ((e = mk(&n.tm_x0A, n.x0, 2 * in, M, pad8(2 * in)))) return e;
  if ((e = mk(&n.tm_x0TB, n.x0T, M, 2 * in + 1, Mx))) return e;
  for (int l = 0; l < n.layers; ++l) {
    if ((e = mk(&n.tm_hA[l], n.h[l], H, M, H))) return e;
    if ((e = mk(&n.tm_hTB[l], n.hT[l], M, H + 1, Mx))) return e;
  }
  // dz[0] doubles as dy of the output layer (ld out_pad); both buffers serve the hidden layers (ld H)
  if ((e = mk(&n.tm_dzA[0], n.dz[0], H, M, H))) return e;
  if ((e = mk(&n.tm_dzA[1], n.dz[1], H, M, H))) return e;
  if ((e = mk(&n.tm_dzTA[0], n.dzT[0], M, H, Mx))) return e;
  if ((e = mk(&n.tm_dzTA[1], n.dzT[1], M, H, Mx))) return e;
  (void)out;
  n.tm_M = M;
  return nullptr;
}

void bf_net_shadow(BfNet& n, const float* params, cudaStream_t st) {
  for (int l = 0; l <= n.layers; ++l) {
    BfLayer& L = n.L[l];
    TraceLaunch tr(CRL_TRACE_AUX, st, (double)L.out * L.in * 10.0);
    dim3 grid(ceil_div(L.in, 32), ceil_div(L.out, 32));
    pack_weights_kernel<<<grid, 256, 0, st>>>(L.out, L.in, l == 0 ? 2 : 1, params + L.oW, L.W, L.kp, L.Wt, L.out_pad);
  }
}

int bf_net_x0_ld(const BfNet& n) { return pad8(2 * n.s.in()); }

void bf_net_pack_input(BfNet& n, const float* x0, const float* x1, int M, cudaStream_t st) {
  const int in = n.s.in();
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * in * 12.0);
  dim3 grid(ceil_div(in, 32), ceil_div(M, 32));
  pack_split_kernel<<<grid, 256, 0, st>>>(M, x0, n.s.in0, n.s.in0, x1, n.s.in1, n.s.in1, n.x0, pad8(2 * in), n.x0T,
                                          n.Mmax);
}

void bf_net_load_dy(BfNet& n, const float* dy, int M, cudaStream_t st) {
  const int out = n.s.out;
  pack(M, dy, out, out, nullptr, 0, 0, n.dz[0], pad8(out), n.dzT[0], n.Mmax, st);
}

void bf_net_forward(BfNet& n, const float* params, int M, unsigned* status, cudaStream_t st) {
  const int H = n.s.hidden;
  const CUtensorMap* A = &n.tm_x0A;
  for (int l = 0; l < n.layers; ++l) {
    const BfLayer& L = n.L[l];
    if (n.s.layernorm) {
      tc_gemm(*A, L.tmW, M, H, 2 * L.kp, EpiFwdPreLN{params + L.ob, n.z[l], H}, status, st, L.kp / 64, L.in);
      TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * H * 12.0);
      ln_fwd_kernel<<<ceil_div(M, 32), 1024, 0, st>>>(M, H, n.z[l], n.rstd[l], params + L.og, params + L.obeta,
                                                     n.h[l], n.hT[l], n.Mmax);
    } else {
      tc_gemm(*A, L.tmW, M, H, 2 * L.kp, EpiFwdHidden{params + L.ob, n.h[l], H, n.hT[l], n.Mmax}, status, st,
              L.kp / 64, L.in);
    }
    A = &n.tm_hA[l];
  }
  const BfLayer& O = n.L[n.layers];
  tc_gemm(*A, O.tmW, M, O.out, 2 * O.kp, EpiFwdOut{params + O.ob, n.y, O.out}, status, st, O.kp / 64, O.in);
}

void bf_net_backward(BfNet& n, const float* params, int M, float* grads, float* dx1, unsigned* status,
                     cudaStream_t st) {
  const int H = n.s.hidden;
  // maps of the output-layer gradient dy (dz[0] with row stride out_pad)
  const BfLayer& O = n.L[n.layers];
  CUtensorMap tm_dyA, tm_dyTA;
  mk(&tm_dyA, n.dz[0], O.out, M, O.out_pad);
  mk(&tm_dyTA, n.dzT[0], M, O.out, n.Mmax);
  const CUtensorMap* curA = &tm_dyA;
  const CUtensorMap* curT = &tm_dyTA;
  int nout = O.out;
  int b = 1;  // next dz buffer to write
  for (int l = n.layers; l >= 0; --l) {
    const BfLayer& L = n.L[l];
    if (grads) {
      if (l == 0)
        tc_gemm(*curT, n.tm_x0TB, nout, 2 * L.in + 1, M, EpiBwdDW0{grads + L.oW, grads + L.ob, L.in}, status, st);
      else
        tc_gemm(*curT, n.tm_hTB[l - 1], nout, L.in + 1, M, EpiBwdDW{grads + L.oW, grads + L.ob, L.in}, status, st);
    }
    if (l == 0) {
      if (dx1) tc_gemm(*curA, L.tmWt, M, L.in, nout, EpiDX0{dx1, n.s.in0, n.s.in1}, status, st);
      break;
    }
    const BfLayer& P = n.L[l - 1];
    if (n.s.layernorm) {
      tc_gemm(*curA, L.tmWt, M, H, nout, EpiBwdDX{n.h[l - 1], H, nullptr, H, nullptr, 0, n.du}, status, st);
      {
        TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * H * 16.0);
        ln_bwd_kernel<<<ceil_div(M, 32), 1024, 0, st>>>(M, H, n.du, n.z[l - 1], n.rstd[l - 1], params + P.og,
                                                       n.dz[b], n.dzT[b], n.Mmax);
      }
      if (grads) {
        TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * H * 8.0);
        ln_param_grad_kernel<<<ceil_div(H, 32), 256, 0, st>>>(M, H, n.du, n.z[l - 1], grads + P.og,
                                                              grads + P.obeta);
      }
    } else {
      tc_gemm(*curA, L.tmWt, M, H, nout, EpiBwdDX{n.h[l - 1], H, n.dz[b], H, n.dzT[b], n.Mmax, nullptr}, status, st);
    }
    curA = &n.tm_dzA[b];
    curT = &n.tm_dzTA[b];
    nout = H;
    b ^= 1;
  }
}

namespace {

struct ShadowLayer {
  int64_t oW;
  int out, in, rep, kp, ldt;
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
  float lr;
  int nl;
  ShadowLayer L[CRL_MAX_LAYERS + 1];
};
struct AdamPair {
  AdamNetDev a[2];
  int count;
  float b1, b2, eps;
};

__global__ void __launch_bounds__(256) adam_shadow_kernel(AdamPair ap) {
  __shared__ float s_corr[2][2];
  if (threadIdx.x < ap.count) {
    const AdamNetDev& a = ap.a[threadIdx.x];
    const double t = (double)*a.t;
    s_corr[threadIdx.x][0] = (float)((double)a.lr / (1.0 - pow((double)ap.b1, t)));
    s_corr[threadIdx.x][1] = (float)(1.0 / (1.0 - pow((double)ap.b2, t)));
  }
  __syncthreads();
  const long long n0 = ap.a[0].n, ntot = n0 + (ap.count > 1 ? ap.a[1].n : 0);
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < ntot;
       gi += (long long)gridDim.x * blockDim.x) {
    const int w = gi < n0 ? 0 : 1;
    const AdamNetDev& a = ap.a[w];
    const long long i = gi - (w ? n0 : 0);
    const float g = a.g[i];
    const float mi = ap.b1 * a.m[i] + (1.f - ap.b1) * g;
    const float vi = ap.b2 * a.v[i] + (1.f - ap.b2) * g * g;
    a.m[i] = mi;
    a.v[i] = vi;
    const float p = a.p[i] - s_corr[w][0] * mi / (sqrtf(vi * s_corr[w][1]) + ap.eps);
    a.p[i] = p;
    for (int l = 0; l < a.nl; ++l) {
      const ShadowLayer& L = a.L[l];
      const long long off = i - L.oW;
      if (off >= 0 && off < (long long)L.out * L.in) {
        const int o = (int)(off / L.in), c = (int)(off % L.in);
        const bf16 hi = __float2bfloat16_rn(p);
        const bf16 lo = __float2bfloat16_rn(p - __bfloat162float(hi));
        bf16* d = L.W2 + (size_t)o * 2 * L.kp;
        for (int q = 0; q < L.rep; ++q) {
          d[L.rep * c + q] = hi;
          d[L.kp + L.rep * c + q] = lo;
        }
        L.Wt[(size_t)c * L.ldt + o] = hi;
        break;
      }
    }
  }
}

}  // namespace

void adam_shadow_update(const AdamShadowNet* nets, int count, float b1, float b2, float eps, cudaStream_t st) {
  AdamPair ap{};
  ap.count = count;
  ap.b1 = b1;
  ap.b2 = b2;
  ap.eps = eps;
  long long ntot = 0;
  for (int k = 0; k < count; ++k) {
    AdamNetDev& a = ap.a[k];
    const AdamShadowNet& s = nets[k];
    a.p = s.p;
    a.g = s.g;
    a.m = s.m;
    a.v = s.v;
    a.n = s.n;
    a.t = s.t_dev;
    a.lr = s.lr;
    a.nl = s.net->layers + 1;
    for (int l = 0; l <= s.net->layers; ++l) {
      const BfLayer& L = s.net->L[l];
      a.L[l] = ShadowLayer{L.oW, L.out, L.in, l == 0 ? 2 : 1, L.kp, L.out_pad, L.W, L.Wt};
    }
    ntot += s.n;
  }
  TraceLaunch tr(CRL_TRACE_ADAM, st, 28.0 * ntot);
  const int blocks = (int)std::min<long long>((ntot + 255) / 256, 152 * 8);
  adam_shadow_kernel<<<blocks, 256, 0, st>>>(ap);
}

}  // namespace crl