// BF16 tensor-core MLP forward / backward (see mlp_bf16.cuh for the scheme).
//
// Networks of arXiv 2408.11052: phi(s, a) and psi(g) (§3.1), the policy
// (§3.2); hidden [256, 256] / repr 64 (App. B.3); LayerNorm before every
// activation for the large networks (§5.4).  Readings M1-M3 as in the FP32
// path: ReLU, LayerNorm (eps 1e-6, biased variance, affine) between Linear and
// ReLU, W stored [out][in].
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>
#include <vector>

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

// Weight shadows: W [out][ncol] (FP32) -> W2 [out][2 kp] = [W_hi | W_lo] with
// hi = bf16(w), lo = bf16(w - hi), each column written `rep` times (rep = 2 for
// the first layer, matching the split input), and the single BF16 transpose
// Wt [ncol][ldt] for the input-gradient product.
__global__ void __launch_bounds__(256) pack_weights_kernel(int rows, int ncol, int rep, const float* __restrict__ W,
                                                          bf16* __restrict__ W2, int kp, bf16* __restrict__ Wt,
                                                          int ldt) {
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
  launch_k(pack_kernel, grid, dim3(256), 0, st, rows, s0, ld0, n0, s1, ld1, n1, dst, ld, dstT, ldt);
}

// ---- LayerNorm (grouped over the networks of a pass: blockIdx.y = network) ----------
struct LnFwdNet {
  int M, ldt;
  float* z;
  float* rstd;
  const float* g;
  const float* beta;
  bf16* h;
  bf16* hT;
};
struct LnFwdGroup {
  LnFwdNet n[kMaxGroupNets];
};

// LayerNorm forward over rows of z [M][H] (FP32, replaced by zhat), rstd [M],
// h = ReLU(zhat * g + beta) written as BF16 [M][H] and, through a shared tile,
// transposed [H][ldt].  Block = 32 rows (one warp each).
__global__ void __launch_bounds__(1024) ln_fwd_kernel(int H, const __grid_constant__ LnFwdGroup grp) {
  pdl_enter();
  const LnFwdNet& a = grp.n[blockIdx.y];
  const int M = a.M, ldt = a.ldt;
  float* __restrict__ z = a.z;
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
    if (lane == 0) a.rstd[row] = rs;
  }
  for (int c0 = 0; c0 < H; c0 += 32) {
    const int c = c0 + lane;
    float hv = 0.f;
    if (row < M && c < H) {
      const size_t o = (size_t)row * H + c;
      const float zh = (z[o] - mean) * rs;
      z[o] = zh;
      hv = fmaxf(zh * a.g[c] + a.beta[c], 0.f);
      a.h[o] = __float2bfloat16_rn(hv);
    }
    tile[w][lane] = hv;
    __syncthreads();
    // warp w writes column c0 + w for the block's 32 rows
    const int cc = c0 + w, rr = blockIdx.x * 32 + lane;
    if (cc < H && rr < M) a.hT[(size_t)cc * ldt + rr] = __float2bfloat16_rn(tile[lane][w]);
    __syncthreads();
  }
}

struct LnBwdNet {
  int M, ldt;
  const float* du;
  const float* zhat;
  const float* rstd;
  const float* g;
  bf16* dz;
  bf16* dzT;
  float* dg;   // ln_param_grad_kernel only
  float* db;
};
struct LnBwdGroup {
  LnBwdNet n[kMaxGroupNets];
};

// LayerNorm backward: du (ReLU-masked, FP32) -> dz = rstd (g du - mean(g du) - zhat mean(g du zhat)),
// written BF16 [M][H] and transposed.  Block = 32 rows.
__global__ void __launch_bounds__(1024) ln_bwd_kernel(int H, const __grid_constant__ LnBwdGroup grp) {
  pdl_enter();
  const LnBwdNet& a = grp.n[blockIdx.y];
  const int M = a.M, ldt = a.ldt;
  const float* __restrict__ du = a.du;
  const float* __restrict__ zhat = a.zhat;
  const float* __restrict__ g = a.g;
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
    rs = a.rstd[row];
  }
  for (int c0 = 0; c0 < H; c0 += 32) {
    const int c = c0 + lane;
    float v = 0.f;
    if (row < M && c < H) {
      const size_t o = (size_t)row * H + c;
      v = rs * (du[o] * g[c] - s1 - zhat[o] * s2);
      a.dz[o] = __float2bfloat16_rn(v);
    }
    tile[w][lane] = v;
    __syncthreads();
    const int cc = c0 + w, rr = blockIdx.x * 32 + lane;
    if (cc < H && rr < M) a.dzT[(size_t)cc * ldt + rr] = __float2bfloat16_rn(tile[lane][w]);
    __syncthreads();
  }
}

// dgain[n] = sum_m du * zhat, dbeta[n] = sum_m du.  Block = 32 columns x 8 row groups.
__global__ void __launch_bounds__(256) ln_param_grad_kernel(int H, const __grid_constant__ LnBwdGroup grp) {
  pdl_enter();
  const LnBwdNet& p = grp.n[blockIdx.y];
  const int M = p.M;
  const float* __restrict__ du = p.du;
  const float* __restrict__ zhat = p.zhat;
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
    p.dg[n] = a;
    p.db[n] = b;
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

template <int BN>
void launch_gemm_bn(const tc::GemmProblem* table, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  using S = tc::GemmSmem<BN>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
    attr = true;
  }
  launch_k(tc::tc_gemm_kernel<BN>, dim3(tiles), dim3(128), S::kBytes, st, table, nprob, status);
}

void launch_bn(int BN, const tc::GemmProblem* t, int nprob, int tiles, unsigned* status, cudaStream_t st) {
  if (BN == 256) launch_gemm_bn<256>(t, nprob, tiles, status, st);
  else if (BN == 128) launch_gemm_bn<128>(t, nprob, tiles, status, st);
  else launch_gemm_bn<64>(t, nprob, tiles, status, st);
}

// Tile width without measurement: 128 x 64 tiles unless 128 x 128 tiles already fill the 152 SMs.
int heuristic_bn(const std::vector<tc::GemmProblem>& probs) {
  long long ctas128 = 0;
  for (const auto& p : probs) ctas128 += (long long)ceil_div(p.M, 128) * ceil_div(p.N, 128);
  return ctas128 >= 148 ? 128 : 64;
}

// Autotuner: time each candidate tile width on the launch itself (every GEMM
// epilogue writes a pure function of inputs the launch does not modify, so
// repeating it is harmless and the tile width does not change any output
// value), keep the fastest.  Runs once per distinct problem list, outside
// graph capture; returns 0 when it cannot measure (the caller falls back).
int tune_bn(GemmGroups& gg, std::vector<tc::GemmProblem>& probs, unsigned* status, cudaStream_t st) {
  static const int kCand[3] = {64, 128, 256};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 0;
  }
  int best = 0;
  float best_ms = 0.f;
  for (int BN : kCand) {
    int tiles = 0;
    const char* err = nullptr;
    const tc::GemmProblem* t = gg.table(probs, BN, &tiles, st, &err);
    if (!t || tiles == 0) continue;
    launch_bn(BN, t, (int)probs.size(), tiles, status, st);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) launch_bn(BN, t, (int)probs.size(), tiles, status, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    if (best == 0 || ms < best_ms) {
      best = BN;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// One grouped launch of `probs` with the tuned (or heuristic) tile width.
// `flops` is the algorithmic work (2 M N K of the unsplit products) for tracing.
const char* launch_group(GemmGroups& gg, std::vector<tc::GemmProblem>& probs, double flops, unsigned* status,
                         cudaStream_t st) {
  if (probs.empty()) return nullptr;
  const uint64_t key = fnv1a(probs.data(), probs.size() * sizeof(tc::GemmProblem));
  int BN = gg.tuned_bn(key);
  if (BN == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (g_autotune && !capturing && g_tracer == nullptr) {
      BN = tune_bn(gg, probs, status, st);
      if (BN) gg.set_tuned_bn(key, BN);
    }
    if (BN == 0) BN = heuristic_bn(probs);
  }
  int tiles = 0;
  const char* err = nullptr;
  const tc::GemmProblem* t = gg.table(probs, BN, &tiles, st, &err);
  if (!t) return err;
  if (tiles == 0) return nullptr;
  TraceLaunch tr(CRL_TRACE_GEMM, st, flops);
  launch_bn(BN, t, (int)probs.size(), tiles, status, st);
  return nullptr;
}

}  // namespace

const tc::GemmProblem* GemmGroups::table(std::vector<tc::GemmProblem>& probs, int BN, int* total_tiles,
                                         cudaStream_t st, const char** err) {
  int tiles = 0;
  for (auto& p : probs) {
    p.tiles_n = ceil_div(p.N, BN);
    p.tile_begin = tiles;
    tiles += ceil_div(p.M, tc::kBM) * p.tiles_n;
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
  cur_ = nullptr;
  used_ = cap_ = 0;
}

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
  for (int l = 0; l <= s.layers; ++l) {
    const size_t w = (l == s.layers) ? (size_t)pad8(out) : (size_t)H;
    n.dz[l] = static_cast<bf16*>(A((size_t)Mmax * w * 2));
    n.dzT[l] = static_cast<bf16*>(A(w * Mmax * 2));
    if (cudaMemset(n.dz[l], 0, (size_t)Mmax * w * 2) != cudaSuccess) return "cudaMemset failed";
  }
  if (s.layernorm) n.du = static_cast<float*>(A((size_t)Mmax * H * 4));
  if (cudaMemset(n.x0, 0, (size_t)Mmax * pad8(2 * in) * 2) != cudaSuccess) return "cudaMemset failed";
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
  for (int l = 0; l <= n.layers; ++l) {
    const int width = (l == n.layers) ? out : H, ld = (l == n.layers) ? pad8(out) : H;
    if ((e = mk(&n.tm_dzA[l], n.dz[l], width, M, ld))) return e;
    if ((e = mk(&n.tm_dzTA[l], n.dzT[l], M, width, Mx))) return e;
  }
  n.tm_M = M;
  return nullptr;
}

void bf_net_shadow(BfNet& n, const float* params, cudaStream_t st) {
  for (int l = 0; l <= n.layers; ++l) {
    BfLayer& L = n.L[l];
    TraceLaunch tr(CRL_TRACE_AUX, st, (double)L.out * L.in * 10.0);
    dim3 grid(ceil_div(L.in, 32), ceil_div(L.out, 32));
    launch_k(pack_weights_kernel, grid, dim3(256), 0, st, L.out, L.in, l == 0 ? 2 : 1, params + L.oW, L.W, L.kp,
             L.Wt, L.out_pad);
  }
}

int bf_net_x0_ld(const BfNet& n) { return pad8(2 * n.s.in()); }

void bf_net_pack_input(BfNet& n, const float* x0, const float* x1, int M, cudaStream_t st) {
  const int in = n.s.in();
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * in * 12.0);
  dim3 grid(ceil_div(in, 32), ceil_div(M, 32));
  launch_k(pack_split_kernel, grid, dim3(256), 0, st, M, x0, n.s.in0, n.s.in0, x1, n.s.in1, n.s.in1, n.x0,
           pad8(2 * in), n.x0T, n.Mmax);
}

void bf_net_load_dy(BfNet& n, const float* dy, int M, cudaStream_t st) {
  const int out = n.s.out;
  pack(M, dy, out, out, nullptr, 0, 0, n.dz[n.layers], pad8(out), n.dzT[n.layers], n.Mmax, st);
}

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
      const float* params = nets[k].params;
      const CUtensorMap& A = (l == 0) ? n.tm_x0A : n.tm_hA[l - 1];
      tc::EpiDesc e;
      if (l == layers) {
        e = epi_of(tc::kEpiFwdOut);
        e.ld0 = L.out;
        e.out0 = n.y;
      } else if (ln) {
        e = epi_of(tc::kEpiFwdPreLN);
        e.ld0 = H;
        e.out0 = n.z[l];
      } else {
        e = epi_of(tc::kEpiFwdHidden);
        e.ld0 = H;
        e.out0 = n.h[l];
        e.ld1 = n.Mmax;
        e.out1 = n.hT[l];
      }
      e.bias = params + L.ob;
      probs.push_back(problem(A, L.tmW, M, L.out, 2 * L.kp, L.kp / 64, e));
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
        grp.n[k] = LnFwdNet{M, n.Mmax, n.z[l], n.rstd[l], pr + L.og, pr + L.obeta, n.h[l], n.hT[l]};
        Mx = std::max(Mx, M);
        bytes += (double)M * H * 12.0;
      }
      if (Mx == 0) continue;
      TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
      launch_k(ln_fwd_kernel, dim3(ceil_div(Mx, 32), kc), dim3(1024), 0, st, H, grp);
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
      e.ldm = H;
      e.ld0 = H;
      if (ln) {
        e.out0 = n.du;
      } else {
        e.out0 = n.dz[l - 1];
        e.out1 = n.dzT[l - 1];
        e.ld1 = n.Mmax;
      }
      probs.push_back(problem(n.tm_dzA[l], L.tmWt, M, H, L.out, 0, e));
      flops += 2.0 * M * H * L.out;
    }
    if (const char* err = launch_group(gg, probs, flops, status, st)) return err;
    for (int k0 = 0; ln && k0 < count; k0 += kMaxGroupNets) {
      const int kc = std::min(kMaxGroupNets, count - k0);
      LnBwdGroup grp, pg;
      memset(&grp, 0, sizeof(grp));
      memset(&pg, 0, sizeof(pg));
      int np = 0, Mx = 0;
      double bytes = 0.0, pbytes = 0.0;
      for (int k = 0; k < kc; ++k) {
        const BfPass& bp = nets[k0 + k];
        BfNet& n = *bp.net;
        const BfLayer& P = n.L[l - 1];
        const int M = std::max(bp.M, 0);
        const LnBwdNet b{M, n.Mmax, n.du, n.z[l - 1], n.rstd[l - 1], bp.params + P.og, n.dz[l - 1], n.dzT[l - 1],
                         bp.grads ? bp.grads + P.og : nullptr, bp.grads ? bp.grads + P.obeta : nullptr};
        grp.n[k] = b;
        Mx = std::max(Mx, M);
        bytes += (double)M * H * 16.0;
        if (bp.grads) {
          pg.n[np++] = b;
          pbytes += (double)M * H * 8.0;
        }
      }
      if (Mx == 0) continue;
      // the parameter gradients read du before the next layer's launch overwrites it
      if (np > 0) {
        TraceLaunch tr(CRL_TRACE_AUX, st, pbytes);
        launch_k(ln_param_grad_kernel, dim3(ceil_div(H, 32), np), dim3(256), 0, st, H, pg);
      }
      TraceLaunch tr(CRL_TRACE_AUX, st, bytes);
      launch_k(ln_bwd_kernel, dim3(ceil_div(Mx, 32), kc), dim3(1024), 0, st, H, grp);
    }
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
        if (l == 0) probs.push_back(problem(n.tm_dzTA[0], n.tm_x0TB, L.out, 2 * L.in + 1, M, 0, e));
        else probs.push_back(problem(n.tm_dzTA[l], n.tm_hTB[l - 1], L.out, L.in + 1, M, 0, e));
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
  }
  return launch_group(gg, probs, flops, status, st);
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
  float lr, b1, b2, eps;
  int nl;
  ShadowLayer L[CRL_MAX_LAYERS + 1];
};

// Adam on one network's FP32 master parameters (grid-stride over its blocks
// lb of nb) and the refresh of its BF16 shadows.  Bias corrections in double
// (1 - b^t loses most of its digits in float for small t).
__device__ __forceinline__ void adam_shadow_body(const AdamNetDev& a, int lb, int nb) {
  const float b1 = a.b1, b2 = a.b2, eps = a.eps;
  __shared__ float s_corr[2];
  if (threadIdx.x == 0) {
    const double t = (double)*a.t;
    s_corr[0] = (float)((double)a.lr / (1.0 - pow((double)b1, t)));
    s_corr[1] = (float)(1.0 / (1.0 - pow((double)b2, t)));
  }
  __syncthreads();
  for (long long i = (long long)lb * blockDim.x + threadIdx.x; i < a.n; i += (long long)nb * blockDim.x) {
    const float g = a.g[i];
    const float mi = b1 * a.m[i] + (1.f - b1) * g;
    const float vi = b2 * a.v[i] + (1.f - b2) * g * g;
    a.m[i] = mi;
    a.v[i] = vi;
    const float p = a.p[i] - s_corr[0] * mi / (sqrtf(vi * s_corr[1]) + eps);
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

// Network s owns blocks [begin[s], begin[s+1]).
__global__ void __launch_bounds__(256) adam_shadow_kernel(const AdamNetDev* __restrict__ nets,
                                                          const int* __restrict__ begin, int n) {
  pdl_enter();
  int lb, nb;
  const int s = segment_of(begin, n, blockIdx.x, lb, nb);
  // the network's descriptor (read for every element's layer lookup) into shared memory
  __shared__ AdamNetDev sa;
  static_assert(sizeof(AdamNetDev) % 4 == 0, "word copy");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(nets + s);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
  for (int i = threadIdx.x; i < (int)(sizeof(AdamNetDev) / 4); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  adam_shadow_body(sa, lb, nb);
}

}  // namespace

const char* adam_shadow_update(BlobCache& cache, const AdamShadowNet* nets, int count, cudaStream_t st) {
  if (count <= 0) return nullptr;
  std::vector<AdamNetDev> devs(count);
  std::vector<int> begin(count + 1, 0);
  long long ntot = 0;
  for (int k = 0; k < count; ++k) ntot += nets[k].n;
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
    a.nl = s.net->layers + 1;
    for (int l = 0; l <= s.net->layers; ++l) {
      const BfLayer& L = s.net->L[l];
      a.L[l] = ShadowLayer{L.oW, L.out, L.in, l == 0 ? 2 : 1, L.kp, L.out_pad, L.W, L.Wt};
    }
    // about 8 blocks per SM in total, shared in proportion to the parameter counts
    const long long share = (long long)(152 * 8) * s.n / std::max<long long>(ntot, 1) + 1;
    begin[k + 1] = begin[k] + (int)std::max<long long>(1, std::min<long long>((s.n + 255) / 256, share));
  }
  const char* err = nullptr;
  const AdamNetDev* dt = cache.get(devs, st, &err);
  if (!dt) return err;
  const int* db = cache.get(begin, st, &err);
  if (!db) return err;
  TraceLaunch tr(CRL_TRACE_ADAM, st, 28.0 * ntot);
  launch_k(adam_shadow_kernel, dim3(begin[count]), dim3(256), 0, st, dt, db, count);
  return nullptr;
}

}  // namespace crl
