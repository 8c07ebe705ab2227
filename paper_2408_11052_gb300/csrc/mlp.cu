// Encoder / actor MLPs of the CRL update step, forward and hand-written backward
// (FP32 and FP64 SIMT path).
//
// A network (arXiv 2408.11052 §3.1 phi(s,a) and psi(g); §3.2 the policy; App. B.3
// hidden [256, 256], repr 64; §5.4 LayerNorm before every activation for the
// 4 x 1024 networks) is
//     h_0 = concat(x0, x1);  z_l = h_{l-1} W_l^T + b_l;  u_l = LN(z_l) or z_l;
//     h_l = ReLU(u_l);  y = h_L W_out^T + b_out.
// LayerNorm: biased variance, eps 1e-6, learned gain and bias.
//
// Saved activations per hidden layer (for the backward): h_l [M][H] and, with
// LayerNorm, zhat_l [M][H] and rstd_l [M].  The backward scratch (three
// [M][H] buffers) follows them in the same workspace.
#include "common.cuh"
#include "gemm_simt.cuh"
#include "internal.h"
#include "trace.h"

namespace crl {

constexpr double kLnEps = 1e-6;

int64_t mlp_layout(const MlpShape& s, LayerOffsets* lay) {
  int64_t off = 0;
  auto take = [&](int64_t n) {
    const int64_t o = off;
    off += round_up(n, 64);
    return o;
  };
  for (int l = 0; l <= s.layers; ++l) {
    const int in = (l == 0) ? s.in() : s.hidden;
    const int out = (l == s.layers) ? s.out : s.hidden;
    LayerOffsets& L = lay[l];
    L.in = in;
    L.out = out;
    L.W = take((int64_t)in * out);
    L.b = take(out);
    if (s.layernorm && l < s.layers) {
      L.g = take(out);
      L.beta = take(out);
    } else {
      L.g = L.beta = -1;
    }
  }
  return off;
}

size_t mlp_saved_bytes(const MlpShape& s, int M, size_t elem) {
  size_t n = (size_t)s.layers * M * s.hidden;                 // h_l
  if (s.layernorm) n += (size_t)s.layers * ((size_t)M * s.hidden + M);  // zhat_l, rstd_l
  n += 3 * (size_t)M * s.hidden;                              // backward scratch
  return n * elem;
}

namespace {

template <typename T>
struct Saved {
  T* h[CRL_MAX_LAYERS];
  T* zhat[CRL_MAX_LAYERS];
  T* rstd[CRL_MAX_LAYERS];
  T* scratch[3];
};

template <typename T>
Saved<T> carve(const MlpShape& s, int M, void* base) {
  Saved<T> sv{};
  T* p = static_cast<T*>(base);
  const size_t mh = (size_t)M * s.hidden;
  for (int l = 0; l < s.layers; ++l) {
    sv.h[l] = p;
    p += mh;
  }
  if (s.layernorm) {
    for (int l = 0; l < s.layers; ++l) {
      sv.zhat[l] = p;
      p += mh;
      sv.rstd[l] = p;
      p += M;
    }
  }
  for (int i = 0; i < 3; ++i) {
    sv.scratch[i] = p;
    p += mh;
  }
  return sv;
}

// Row-wise LayerNorm + ReLU: z (in zhat, overwritten by zhat), rstd, h = ReLU(zhat*g + beta).
// One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) layernorm_relu_kernel(int M, int N, T* __restrict__ zhat,
                                                            T* __restrict__ rstd, T* __restrict__ h,
                                                            const T* __restrict__ gain,
                                                            const T* __restrict__ bias) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= M) return;
  T* z = zhat + (size_t)row * N;
  T sum = 0;
  for (int c = lane; c < N; c += kWarp) sum += z[c];
  const T mean = warp_sum(sum) / T(N);
  T sq = 0;
  for (int c = lane; c < N; c += kWarp) {
    const T d = z[c] - mean;
    sq += d * d;
  }
  const T var = warp_sum(sq) / T(N);
  const T rs = T(1) / dev_sqrt(var + T(kLnEps));
  for (int c = lane; c < N; c += kWarp) {
    const T zh = (z[c] - mean) * rs;
    z[c] = zh;
    const T u = zh * gain[c] + bias[c];
    h[(size_t)row * N + c] = u > T(0) ? u : T(0);
  }
  if (lane == 0) rstd[row] = rs;
}

// Row-wise LayerNorm backward: du (already masked by ReLU) -> dz.
template <typename T>
__global__ void __launch_bounds__(256) layernorm_bwd_kernel(int M, int N, const T* __restrict__ du,
                                                           const T* __restrict__ zhat,
                                                           const T* __restrict__ rstd,
                                                           const T* __restrict__ gain, T* __restrict__ dz) {
  pdl_enter();
  const int lane = threadIdx.x % kWarp;
  const int row = blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  if (row >= M) return;
  const T* d = du + (size_t)row * N;
  const T* zh = zhat + (size_t)row * N;
  T s1 = 0, s2 = 0;
  for (int c = lane; c < N; c += kWarp) {
    const T dzh = d[c] * gain[c];
    s1 += dzh;
    s2 += dzh * zh[c];
  }
  s1 = warp_sum(s1) / T(N);
  s2 = warp_sum(s2) / T(N);
  const T rs = rstd[row];
  for (int c = lane; c < N; c += kWarp) {
    const T dzh = d[c] * gain[c];
    dz[(size_t)row * N + c] = rs * (dzh - s1 - zh[c] * s2);
  }
}

// Column sums over M rows: out1[n] = sum X, out2[n] = sum X*Y (Y optional),
// out3[n] = sum Z (Z optional).  Block = 32 columns x 8 row groups.
template <typename T>
__global__ void __launch_bounds__(256) colsum_kernel(int M, int N, const T* __restrict__ X,
                                                    const T* __restrict__ Y, const T* __restrict__ Z,
                                                    T* __restrict__ out1, T* __restrict__ out2,
                                                    T* __restrict__ out3) {
  pdl_enter();
  __shared__ T sm[3][8][33];
  const int cx = threadIdx.x % 32, ry = threadIdx.x / 32;
  const int n = blockIdx.x * 32 + cx;
  T a1 = 0, a2 = 0, a3 = 0;
  if (n < N) {
    for (int m = ry; m < M; m += 8) {
      const size_t o = (size_t)m * N + n;
      const T x = X[o];
      a1 += x;
      if (Y) a2 += x * Y[o];
      if (Z) a3 += Z[o];
    }
  }
  sm[0][ry][cx] = a1;
  sm[1][ry][cx] = a2;
  sm[2][ry][cx] = a3;
  __syncthreads();
  if (ry == 0 && n < N) {
    T s1 = 0, s2 = 0, s3 = 0;
    for (int r = 0; r < 8; ++r) {
      s1 += sm[0][r][cx];
      s2 += sm[1][r][cx];
      s3 += sm[2][r][cx];
    }
    if (out1) out1[n] = s1;
    if (out2) out2[n] = s2;
    if (out3) out3[n] = s3;
  }
}

template <typename T>
void colsum(int M, int N, const T* X, const T* Y, const T* Z, T* o1, T* o2, T* o3, cudaStream_t st) {
  TraceLaunch tr(CRL_TRACE_AUX, st, (double)M * N * sizeof(T) * (1 + (Y != nullptr) + (Z != nullptr)));
  launch_k(colsum_kernel<T>, dim3(ceil_div(N, 32)), dim3(256), 0, st, M, N, X, Y, Z, o1, o2, o3);
}

}  // namespace

template <typename T, typename TX1>
void mlp_forward(const MlpShape& s, const T* params, const float* x0, const TX1* x1, int M, T* y, void* saved,
                 cudaStream_t st) {
  LayerOffsets lay[CRL_MAX_LAYERS + 1];
  mlp_layout(s, lay);
  Saved<T> sv = carve<T>(s, M, saved);
  const int H = s.hidden;
  for (int l = 0; l <= s.layers; ++l) {
    const LayerOffsets& L = lay[l];
    const bool last = (l == s.layers);
    T* out = last ? y : (s.layernorm ? sv.zhat[l] : sv.h[l]);
    const int ldo = last ? s.out : H;
    EpiBias<T> ep{out, ldo, params + L.b, (!last && !s.layernorm) ? 1 : 0};
    LoadNK<T> lb{params + L.W, L.in};
    if (l == 0) {
      LoadRowsSplit<T, float, TX1> la{x0, x1, s.in0, s.in1, s.in0};
      gemm<T>(M, L.out, L.in, la, lb, ep, st);
    } else {
      LoadRowsSplit<T, T, T> la{sv.h[l - 1], nullptr, H, 0, H};
      gemm<T>(M, L.out, L.in, la, lb, ep, st);
    }
    if (!last && s.layernorm) {
      TraceLaunch tr(CRL_TRACE_AUX, st, 4.0 * M * H * sizeof(T));
      launch_k(layernorm_relu_kernel<T>, dim3(ceil_div(M, 8)), dim3(256), 0, st, M, H, sv.zhat[l], sv.rstd[l], sv.h[l],
                                                               params + L.g, params + L.beta);
    }
  }
}

template <typename T, typename TX1>
void mlp_backward(const MlpShape& s, const T* params, const float* x0, const TX1* x1, int M, const void* saved,
                  const T* dy, T* dparams, T* dx0, T* dx1, cudaStream_t st) {
  LayerOffsets lay[CRL_MAX_LAYERS + 1];
  mlp_layout(s, lay);
  Saved<T> sv = carve<T>(s, M, const_cast<void*>(saved));
  const int H = s.hidden;
  // dcur holds dZ of the layer being processed ([M][out_l]).
  const T* dcur = dy;
  int bufi = 0;
  for (int l = s.layers; l >= 0; --l) {
    const LayerOffsets& L = lay[l];
    const int nout = L.out;
    if (dparams) {
      // db_l = colsum(dZ_l);  dW_l[n][k] = sum_m dZ_l[m][n] * in_l[m][k]
      colsum<T>(M, nout, dcur, nullptr, nullptr, dparams + L.b, nullptr, nullptr, st);
      LoadTrans<T> la{dcur, nout};
      EpiScale<T> ep{dparams + L.W, L.in, T(1)};
      if (l == 0) {
        LoadColsSplit<T, float, TX1> lb{x0, x1, s.in0, s.in1, s.in0};
        gemm<T>(nout, L.in, M, la, lb, ep, st);
      } else {
        LoadColsSplit<T, T, T> lb{sv.h[l - 1], nullptr, H, 0, H};
        gemm<T>(nout, L.in, M, la, lb, ep, st);
      }
    }
    LoadMK<T> la{dcur, nout};
    LoadKN<T> lb{params + L.W, L.in};
    if (l == 0) {
      if (dx0 || dx1) {
        EpiMaskSplit<T> ep{dx0, dx1, s.in0, s.in1, s.in0, nullptr, 0};
        gemm<T>(M, L.in, nout, la, lb, ep, st);
      }
      break;
    }
    // dU_{l-1} = (dZ_l W_l) * [h_{l-1} > 0]
    T* du = sv.scratch[bufi];
    bufi = (bufi + 1) % 2;
    EpiMaskSplit<T> ep{du, nullptr, H, 0, H, sv.h[l - 1], H};
    gemm<T>(M, H, nout, la, lb, ep, st);
    if (s.layernorm) {
      const LayerOffsets& P = lay[l - 1];
      T* dz = sv.scratch[2];
      {
        TraceLaunch tr(CRL_TRACE_AUX, st, 3.0 * M * H * sizeof(T));
        launch_k(layernorm_bwd_kernel<T>, dim3(ceil_div(M, 8)), dim3(256), 0, st, M, H, du, sv.zhat[l - 1], sv.rstd[l - 1],
                                                                params + P.g, dz);
      }
      if (dparams)
        colsum<T>(M, H, du, sv.zhat[l - 1], nullptr, dparams + P.beta, dparams + P.g, nullptr, st);
      // move dz into the ping-pong buffer so scratch[2] is free for the next LayerNorm
      dcur = dz;
      // the next GEMM reads dz (scratch[2]) and writes scratch[bufi]: no overlap.
    } else {
      dcur = du;
    }
  }
}

template void mlp_forward<float, float>(const MlpShape&, const float*, const float*, const float*, int, float*,
                                        void*, cudaStream_t);
template void mlp_forward<double, float>(const MlpShape&, const double*, const float*, const float*, int,
                                         double*, void*, cudaStream_t);
template void mlp_forward<double, double>(const MlpShape&, const double*, const float*, const double*, int,
                                          double*, void*, cudaStream_t);
template void mlp_backward<float, float>(const MlpShape&, const float*, const float*, const float*, int,
                                         const void*, const float*, float*, float*, float*, cudaStream_t);
template void mlp_backward<double, float>(const MlpShape&, const double*, const float*, const float*, int,
                                          const void*, const double*, double*, double*, double*, cudaStream_t);
template void mlp_backward<double, double>(const MlpShape&, const double*, const float*, const double*, int,
                                           const void*, const double*, double*, double*, double*, cudaStream_t);

}  // namespace crl
